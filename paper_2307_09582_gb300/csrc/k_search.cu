// Algorithm 1 (Sec. 3.2) over a whole image: one CTA per 64 x 16 HR tile.
//
// The HR tile is staged into shared memory by a 2D TMA load (cp.async.bulk.tensor) completing
// on an mbarrier; while it is in flight the CTA's threads copy the LR halo (the LR rows and
// columns the tile's windows reach) into shared memory as float4 colours in 1/255 units. Each
// thread then owns whole pixels: both candidate loops of Algorithm 1 run in registers against
// the shared-memory window, so no cross-lane reduction is needed and the tie-break is the
// deterministic lowest window index.
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"
#include "search.cuh"

namespace glu {

GLU_DEFINE_STATUS(search)

// Occupancy target (CTAs per SM) and the rolled search variant: build-time tuning knobs.
#ifndef GLU_SEARCH_MINBLOCKS
#define GLU_SEARCH_MINBLOCKS 3
#endif
#ifndef GLU_SEARCH_COMPACT
#define GLU_SEARCH_COMPACT 0
#endif

constexpr int kTileW = 64;   // HR pixels per tile row (64 * 3 channels: a 16-byte multiple)
constexpr int kTileH = 16;   // HR rows per tile
constexpr int kThreads = 256;
static_assert(kThreads % kTileW == 0, "a thread keeps one tile column");

template <typename HT>
struct HrTile {
    alignas(128) HT px[kTileH][kTileW * 3];
};

template <int S, typename HT>
__global__ void __launch_bounds__(kThreads, GLU_SEARCH_MINBLOCKS)
    k_search(const __grid_constant__ CUtensorMap hr_map, const SearchArgs P, const int use_tma) {
    __shared__ HrTile<HT> tile;
    __shared__ alignas(8) uint64_t bar;
    extern __shared__ float4 region[];

    constexpr int r = (S - 1) / 2;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kTileW, y0 = blockIdx.y * kTileH;
    const int s = P.s;
    const int xe = min(x0 + kTileW, P.W), ye = min(y0 + kTileH, P.H);
    const int v0 = y0 / s - r, u0 = x0 / s - r;
    const int RH = (ye - 1) / s + r - v0 + 1, RW = (xe - 1) / s + r - u0 + 1;

    if (use_tma) {
        if (tid == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            mbar_arrive_expect_tx(&bar, (uint32_t)sizeof(tile.px));
            tma_load_2d(&tile.px[0][0], &hr_map, &bar, x0 * 3, y0);
        }
    } else {
        const HT* src = (const HT*)P.hr;
        for (int i = tid; i < kTileH * kTileW * 3; i += kThreads) {
            const int ty = i / (kTileW * 3), tx = i % (kTileW * 3);
            const int y = y0 + ty, xc = x0 * 3 + tx;
            tile.px[ty][tx] = (y < P.H && xc < P.W * 3) ? src[(int64_t)y * P.hr_pitch + xc] : HT(0);
        }
    }
    // LR halo in 1/255 units; rows/columns outside the LR image are never selected (masks)
    for (int i = tid; i < RH * RW; i += kThreads) {
        const int v = v0 + i / RW, u = u0 + i % RW;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v >= 0 && v < P.h && u >= 0 && u < P.w) {
            const int64_t o = (int64_t)v * P.lr_pitch + (int64_t)u * 3;
            if (P.lr_dtype == GLU_U8) {
                const uint8_t* L = (const uint8_t*)P.lr;
                c = make_float4((float)L[o], (float)L[o + 1], (float)L[o + 2], 0.f);
            } else if (P.lr_dtype == GLU_F16) {
                const __half* L = (const __half*)P.lr;
                c = make_float4(__half2float(L[o]) * 255.f, __half2float(L[o + 1]) * 255.f,
                                __half2float(L[o + 2]) * 255.f, 0.f);
            } else {
                const float* L = (const float*)P.lr;
                c = make_float4(L[o] * 255.f, L[o + 1] * 255.f, L[o + 2] * 255.f, 0.f);
            }
        }
        region[i] = c;
    }
    __syncthreads();
    if (use_tma && !mbar_wait_bounded(&bar, 0)) {
        set_status(GLU_ERR_TIMEOUT);
        // the copy may still land: give it another bounded wait before the CTA exits
        (void)mbar_wait_bounded(&bar, 0);
        return;
    }

    // interior tiles (every window inside the LR image) skip the validity masks
    const bool interior = v0 >= 0 && u0 >= 0 && (ye - 1) / s + r < P.h && (xe - 1) / s + r < P.w;
    // a thread keeps one column of the tile (kThreads is a multiple of kTileW) and walks rows
    const int tx = tid % kTileW, x = x0 + tx, px = x / s;
    const int col = px - r - u0;
    for (int ty = tid / kTileW; ty < kTileH; ty += kThreads / kTileW) {
        const int y = y0 + ty;
        if (y >= P.H || x >= P.W) continue;
        const float ir = Px<HT>::to255(tile.px[ty][tx * 3 + 0]);
        const float ig = Px<HT>::to255(tile.px[ty][tx * 3 + 1]);
        const float ib = Px<HT>::to255(tile.px[ty][tx * 3 + 2]);
        const int py = y / s;
        const float4* win = &region[(py - r - v0) * RW + col];
        SearchOut o;
        if (interior) {
            o = search_pixel<S, GLU_SEARCH_COMPACT != 0, true>(win, RW, 0u, 0u, ir, ig, ib, P.eps255,
                                                               P.gnu != 0);
        } else {
            uint32_t rm, cm;
            window_masks(py, px, P.h, P.w, S, rm, cm);
            o = search_pixel<S, GLU_SEARCH_COMPACT != 0>(win, RW, rm, cm, ir, ig, ib, P.eps255,
                                                         P.gnu != 0);
        }
        const int64_t p = (int64_t)y * P.W + x;
        P.code[p] = (uint16_t)(o.ka * S * S + o.kb);
        store_weight(P.weight, P.wfmt, p, o.omega);
        if (P.err) P.err[p] = o.err;
    }
}

// ----------------------------------------------------------------------------- host side

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

// 2D byte/half view of an interleaved HR image for TMA: inner dim W*3 elements, outer dim H.
static bool make_hr_map(const SearchArgs& a, CUtensorMap* map) {
    auto enc = get_encode();
    if (!enc) return false;
    const size_t esz = a.hr_dtype == GLU_U8 ? 1 : 2;
    if (((uintptr_t)a.hr & 15u) != 0 || ((size_t)a.hr_pitch * esz) % 16 != 0) return false;
    cuuint64_t dims[2] = {(cuuint64_t)a.W * 3, (cuuint64_t)a.H};
    cuuint64_t strides[1] = {(cuuint64_t)a.hr_pitch * esz};
    cuuint32_t box[2] = {(cuuint32_t)kTileW * 3, (cuuint32_t)kTileH};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, a.hr_dtype == GLU_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                     2, const_cast<void*>(a.hr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int S, typename HT>
static int launch_t(const SearchArgs& a, cudaStream_t st) {
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    const int use_tma = make_hr_map(a, &map) ? 1 : 0;
    constexpr int r = (S - 1) / 2;
    // largest LR halo any tile needs
    const int rh = (kTileH - 1) / a.s + 2 + 2 * r, rw = (kTileW - 1) / a.s + 2 + 2 * r;
    const size_t smem = sizeof(float4) * (size_t)rh * rw;
    auto kern = k_search<S, HT>;
    if (smem > 48 * 1024)
        GLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((a.W + kTileW - 1) / kTileW, (a.H + kTileH - 1) / kTileH);
    kern<<<grid, kThreads, smem, st>>>(map, a, use_tma);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

template <typename HT>
static int launch_dtype(const SearchArgs& a, cudaStream_t st) {
    switch (a.S) {
        case 1: return launch_t<1, HT>(a, st);
        case 3: return launch_t<3, HT>(a, st);
        case 5: return launch_t<5, HT>(a, st);
        case 7: return launch_t<7, HT>(a, st);
        case 9: return launch_t<9, HT>(a, st);
        default: return GLU_ERR_UNSUPPORTED;
    }
}

int launch_search(const SearchArgs& a, cudaStream_t st) {
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    if (a.hr_dtype == GLU_U8) return launch_dtype<uint8_t>(a, st);
    if (a.hr_dtype == GLU_F16) return launch_dtype<__half>(a, st);
    return GLU_ERR_UNSUPPORTED;
}

}  // namespace glu
