// Shared device/host helpers of the CUDA library: dtype access, status words, mbarrier/TMA PTX.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "glu.h"

namespace glu {

constexpr float kInf = __builtin_huge_valf();

// ------------------------------------------------------------------ device status words
// Each translation unit owns one status word (first error wins). Kernels never trap: a failed
// check or an exhausted wait records its code here and the kernel returns.
#define GLU_DEFINE_STATUS(tu)                                                            \
    static __device__ int g_status_word;                                                 \
    __device__ __forceinline__ void set_status(int code) { atomicCAS(&g_status_word, 0, code); } \
    int read_and_clear_status_##tu(cudaStream_t st) {                                    \
        int v = 0, z = 0;                                                                \
        if (cudaMemcpyFromSymbolAsync(&v, g_status_word, sizeof(int), 0,                 \
                                      cudaMemcpyDeviceToHost, st) != cudaSuccess)        \
            return GLU_ERR_CUDA;                                                         \
        if (cudaMemcpyToSymbolAsync(g_status_word, &z, sizeof(int), 0,                   \
                                    cudaMemcpyHostToDevice, st) != cudaSuccess)          \
            return GLU_ERR_CUDA;                                                         \
        if (cudaStreamSynchronize(st) != cudaSuccess) return GLU_ERR_CUDA;               \
        return v;                                                                        \
    }

// Upper bound on polls of any device-side wait before it records GLU_ERR_TIMEOUT.
constexpr uint32_t kSpinLimit = 1u << 26;

// ------------------------------------------------------------------------ dtype access
template <typename T> struct Px;
template <> struct Px<uint8_t> {
    // U8 colour values are already in 1/255 units
    static __device__ __forceinline__ float to255(uint8_t v) { return (float)v; }
    static constexpr float kToUnit = 1.0f / 255.0f;
};
template <> struct Px<__half> {
    static __device__ __forceinline__ float to255(__half v) { return __half2float(v) * 255.0f; }
};
template <> struct Px<float> {
    static __device__ __forceinline__ float to255(float v) { return v * 255.0f; }
};

__device__ __forceinline__ float ld_unit(const void* p, int dtype, int64_t i) {
    switch (dtype) {
        case GLU_U8: return (float)((const uint8_t*)p)[i] * (1.0f / 255.0f);
        case GLU_F16: return __half2float(((const __half*)p)[i]);
        default: return ((const float*)p)[i];
    }
}

// --------------------------------------------------------------------- weight formats
__device__ __forceinline__ void store_weight(void* base, int fmt, int64_t i, float w) {
    if (fmt == GLU_W_F32) {
        ((float*)base)[i] = w;
    } else if (fmt == GLU_W_F16) {
        ((__half*)base)[i] = __float2half_rn(w);
    } else {
        float q = rintf(__saturatef(w) * 65535.0f);
        ((uint16_t*)base)[i] = (uint16_t)q;
    }
}

// Re-store a weight previously read with load_weight*: float16 and unorm16 values round-trip
// exactly through float (every float16 and every k/65535 converts back to the same code).
__device__ __forceinline__ void store_weight_raw(void* base, int fmt, int64_t i, float w) {
    if (fmt == GLU_W_F32) {
        ((float*)base)[i] = w;
    } else if (fmt == GLU_W_F16) {
        ((__half*)base)[i] = __float2half_rn(w);
    } else {
        ((uint16_t*)base)[i] = (uint16_t)rintf(w * 65535.0f);
    }
}

__device__ __forceinline__ float load_weight(const void* base, int fmt, int64_t i) {
    if (fmt == GLU_W_F32) return ((const float*)base)[i];
    if (fmt == GLU_W_F16) return __half2float(((const __half*)base)[i]);
    return (float)((const uint16_t*)base)[i] * (1.0f / 65535.0f);
}

// ----------------------------------------------------------------- mbarrier and TMA PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase. Returns false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
    for (uint32_t it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// 2D tiled TMA load of box (c0 = inner element coordinate, c1 = row) into shared memory.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t c0, int32_t c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// 2D tiled TMA store of a box from shared memory (bulk-group completion); the caller fences the
// generic-proxy writes of the box first (fence_proxy_async_smem) and waits before reusing it.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int32_t c0,
                                             int32_t c1) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_store_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until all but the most recent committed bulk-store group have read their sources.
__device__ __forceinline__ void tma_store_wait_read_1() {
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// Commit this thread's bulk stores and wait until they have read their shared-memory sources.
__device__ __forceinline__ void tma_store_commit_wait_read() {
    asm volatile("cp.async.bulk.commit_group;\n\tcp.async.bulk.wait_group.read 0;" ::: "memory");
}

// 4-byte asynchronous global -> shared copy (LDGSTS), completed by cp_async_wait_all().
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialisation may
// start before the preceding kernel of its stream has finished; griddep_wait() blocks until that
// kernel has completed and its writes are visible (a no-op in a kernel launched without the
// attribute). griddep_launch_dependents() lets the dependent kernel start early.
__device__ __forceinline__ void griddep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace glu

// ------------------------------------------------------------------------ host helpers
#define GLU_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return GLU_ERR_CUDA;          \
    } while (0)

#define GLU_LAUNCH_CHECK()                                   \
    do {                                                     \
        if (cudaPeekAtLastError() != cudaSuccess) {          \
            (void)cudaGetLastError();                        \
            return GLU_ERR_CUDA;                             \
        }                                                    \
    } while (0)
