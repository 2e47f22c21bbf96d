// Host side of the Algorithm 1 search (Sec. 3.2): tensor maps for the TMA tile loads, the
// split of a batch into launches of <= 32 images, and the choice of kernel variant (tile height,
// occupancy target, candidate loop schedule) through the autotuner. The kernels themselves are
// in search_kernel.cuh, instantiated in k_search_u8.cu and k_search_f16.cu.
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tune.h"
#include "variants.h"

namespace glu {

int search_launch_u8(int v, const SearchArgs* items, int n, cudaStream_t st);
int search_launch_f16(int v, const SearchArgs* items, int n, cudaStream_t st);
int read_and_clear_status_search_u8(cudaStream_t st);
int read_and_clear_status_search_f16(cudaStream_t st);

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

bool encode_map_2d(CUtensorMap* map, CUtensorMapDataType dt, size_t esize, const void* base,
                   uint64_t inner, uint64_t rows, uint64_t row_bytes, uint32_t box_inner,
                   uint32_t box_rows) {
    auto enc = get_encode();
    if (!enc || ((uintptr_t)base & 15u) != 0 || row_bytes % 16 != 0 ||
        (box_inner * esize) % 16 != 0 || box_inner > 256 || box_rows > 256 || inner == 0 ||
        rows == 0)
        return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    cuuint32_t box[2] = {box_inner, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

bool make_hr_map(const SearchArgs& a, CUtensorMap* map, int tile_h) {
    auto enc = get_encode();
    if (!enc) return false;
    const size_t esz = a.hr_dtype == GLU_U8 ? 1 : 2;
    if (((uintptr_t)a.hr & 15u) != 0 || ((size_t)a.hr_pitch * esz) % 16 != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)a.W * 3, (cuuint64_t)a.H};
    cuuint64_t strides[1] = {(cuuint64_t)a.hr_pitch * esz};
    cuuint32_t box[2] = {(cuuint32_t)kTileW * 3, (cuuint32_t)tile_h};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, a.hr_dtype == GLU_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                     2, const_cast<void*>(a.hr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int read_and_clear_status_search(cudaStream_t st) {
    const int a = read_and_clear_status_search_u8(st);
    const int b = read_and_clear_status_search_f16(st);
    return a != GLU_OK ? a : b;
}

int launch_search_batch(const SearchArgs* items, int n, cudaStream_t st) {
    static std::mutex mu;  // the kernels' staging blocks are shared
    std::lock_guard<std::mutex> lock(mu);
    for (int k0 = 0; k0 < n; k0 += kMaxSearchBatch) {
        const int m = n - k0 < kMaxSearchBatch ? n - k0 : kMaxSearchBatch;
        const SearchArgs* it = items + k0;
        int maxS = 1, mins = 1 << 30;
        long long npx = 0;
        for (int k = 0; k < m; ++k) {
            const SearchArgs& a = it[k];
            if (a.hr_dtype != it[0].hr_dtype || a.wfmt != it[0].wfmt || a.gnu != it[0].gnu ||
                a.eps255 != it[0].eps255)
                return GLU_ERR_UNSUPPORTED;  // one dtype / weight format / mode per launch
            if (a.S < 1 || a.S > 9 || (a.S & 1) == 0) return GLU_ERR_UNSUPPORTED;
            if (a.S > maxS) maxS = a.S;
            if (a.s < mins) mins = a.s;
            npx += (long long)a.H * a.W;
        }
        auto run = [&](int v) -> int {
            if (it[0].hr_dtype == GLU_U8) return search_launch_u8(v, it, m, st);
            if (it[0].hr_dtype == GLU_F16) return search_launch_f16(v, it, m, st);
            return GLU_ERR_UNSUPPORTED;
        };
        const int key[5] = {it[0].hr_dtype, it[0].gnu, maxS, mins, tune_size_class(npx)};
        int v = 0;
        int rc = tune_choose(kTuneSearch, key, kNumSearchVariants, run, st, &v);
        if (rc) return rc;
        rc = run(v);
        if (rc) return rc;
    }
    return GLU_OK;
}

int launch_search(const SearchArgs& a, cudaStream_t st) {
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    return launch_search_batch(&a, 1, st);
}

}  // namespace glu
