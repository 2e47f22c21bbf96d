// Eq. 1 (apply) and its adjoint.
//
// apply: one thread per group of 4 consecutive HR pixels of a row: the pair codes and weights
// stream from HBM, the two LR gathers hit L2 (the LR target is small), the result streams out.
//
// backward: grad_lr_q = sum_{p: a_p = q} w_p G_p + sum_{p: b_p = q} (1 - w_p) G_p. The pixels that
// can map to q are bounded by the window: p's block must lie within r of q. One warp owns one
// LR pixel and walks those source blocks in a fixed order (blocks in raster order, lanes strided
// over each block's pixels), then reduces lanes with a fixed butterfly: no atomics, the result
// is bit-reproducible. This is the segmented reduction over the inverse pixel-to-LR map with the
// map left implicit (the window bounds it, so it is never materialised).
#include "internal.h"
#include "common.cuh"

namespace glu {

GLU_DEFINE_STATUS(apply)

__device__ __forceinline__ float ld_f(const void* p, int dtype, int64_t i) {
    return dtype == GLU_F16 ? __half2float(((const __half*)p)[i]) : ((const float*)p)[i];
}

__device__ __forceinline__ void st_f(void* p, int dtype, int64_t i, float v) {
    if (dtype == GLU_F16)
        ((__half*)p)[i] = __float2half_rn(v);
    else
        ((float*)p)[i] = v;
}

// Decode window index k of HR pixel (y, x) into an LR offset (row * pitch + col * C). A code
// that points outside the LR image (not produced by the search) is recorded as
// GLU_ERR_DEVICE_CHECK and redirected to LR pixel (0, 0) so no access leaves the buffer.
__device__ __forceinline__ int64_t lr_off(int y, int x, int k, int s, int S, int h, int w,
                                          int64_t pitch, int C) {
    const int r = (S - 1) >> 1;
    const int v = y / s + k / S - r, u = x / s + k % S - r;
    if (v < 0 || v >= h || u < 0 || u >= w || k >= S * S) {
        set_status(GLU_ERR_DEVICE_CHECK);
        return 0;
    }
    return (int64_t)v * pitch + (int64_t)u * C;
}

template <int C>
__global__ void k_apply(const ApplyArgs P) {
    const int64_t groups_per_row = (P.W + 3) / 4;
    const int64_t total = groups_per_row * P.H;
    const int K = P.S * P.S;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(g / groups_per_row);
        const int xs = (int)(g % groups_per_row) * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = xs + j;
            if (x >= P.W) break;
            const int64_t p = (int64_t)y * P.W + x;
            const int code = P.code[p];
            const float w = load_weight(P.weight, P.wfmt, p);
            const int64_t oa = lr_off(y, x, code / K, P.s, P.S, P.h, P.w, P.T_pitch, C);
            const int64_t ob = lr_off(y, x, code % K, P.s, P.S, P.h, P.w, P.T_pitch, C);
            const int64_t oo = (int64_t)y * P.out_pitch + (int64_t)x * C;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float ta = ld_f(P.T, P.T_dtype, oa + c), tb = ld_f(P.T, P.T_dtype, ob + c);
                st_f(P.out, P.out_dtype, oo + c, __fmaf_rn(w, ta - tb, tb));
            }
        }
    }
}

template <int C>
__global__ void k_apply_backward_lr(const BackwardArgs P) {
    const int lane = threadIdx.x & 31;
    const int warps_per_block = blockDim.x >> 5;
    const int64_t nq = (int64_t)P.h * P.w;
    const int r = (P.S - 1) >> 1, K = P.S * P.S;
    for (int64_t q = blockIdx.x * (int64_t)warps_per_block + (threadIdx.x >> 5); q < nq;
         q += (int64_t)gridDim.x * warps_per_block) {
        const int v = (int)(q / P.w), u = (int)(q % P.w);
        float acc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = 0.f;
        for (int bv = max(0, v - r); bv <= min(P.h - 1, v + r); ++bv) {
            for (int bu = max(0, u - r); bu <= min(P.w - 1, u + r); ++bu) {
                // window index of q as seen from pixels of block (bv, bu)
                const int kq = (v - bv + r) * P.S + (u - bu + r);
                const int ys = bv * P.s, xs = bu * P.s;
                const int ey = min(P.s, P.H - ys), ex = min(P.s, P.W - xs);
                for (int j = lane; j < ey * ex; j += 32) {
                    const int y = ys + j / ex, x = xs + j % ex;
                    const int64_t p = (int64_t)y * P.W + x;
                    const int code = P.code[p];
                    const int ka = code / K, kb = code % K;
                    if (ka != kq && kb != kq) continue;
                    const float w = load_weight(P.weight, P.wfmt, p);
                    const float f = (ka == kq ? w : 0.f) + (kb == kq ? 1.f - w : 0.f);
                    const int64_t og = (int64_t)y * P.G_pitch + (int64_t)x * C;
#pragma unroll
                    for (int c = 0; c < C; ++c) acc[c] = __fmaf_rn(f, P.G[og + c], acc[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
        }
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < C; ++c) P.gT[(int64_t)v * P.gT_pitch + (int64_t)u * C + c] = acc[c];
        }
    }
}

template <int C>
__global__ void k_apply_backward_w(const BackwardArgs P) {
    const int64_t n = (int64_t)P.H * P.W;
    const int K = P.S * P.S;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(p / P.W), x = (int)(p % P.W);
        const int code = P.code[p];
        const int64_t oa = lr_off(y, x, code / K, P.s, P.S, P.h, P.w, P.T_pitch, C);
        const int64_t ob = lr_off(y, x, code % K, P.s, P.S, P.h, P.w, P.T_pitch, C);
        const int64_t og = (int64_t)y * P.G_pitch + (int64_t)x * C;
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) acc = __fmaf_rn(P.G[og + c], P.T[oa + c] - P.T[ob + c], acc);
        P.gw[p] = acc;
    }
}

static int grid_for(int64_t work, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sms * 16;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

int launch_apply(const ApplyArgs& a, cudaStream_t st) {
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    const int threads = 256;
    const int64_t work = (int64_t)((a.W + 3) / 4) * a.H;
    const int grid = grid_for(work, threads);
    switch (a.C) {
        case 1: k_apply<1><<<grid, threads, 0, st>>>(a); break;
        case 2: k_apply<2><<<grid, threads, 0, st>>>(a); break;
        case 3: k_apply<3><<<grid, threads, 0, st>>>(a); break;
        case 4: k_apply<4><<<grid, threads, 0, st>>>(a); break;
        default: return GLU_ERR_UNSUPPORTED;
    }
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

template <int C>
static int launch_bw_t(const BackwardArgs& a, cudaStream_t st) {
    const int threads = 256;
    const int grid_q = grid_for((int64_t)a.h * a.w * 32, threads);
    k_apply_backward_lr<C><<<grid_q, threads, 0, st>>>(a);
    GLU_LAUNCH_CHECK();
    if (a.gw) {
        k_apply_backward_w<C><<<grid_for((int64_t)a.H * a.W, threads), threads, 0, st>>>(a);
        GLU_LAUNCH_CHECK();
    }
    return GLU_OK;
}

int launch_apply_backward(const BackwardArgs& a, cudaStream_t st) {
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    switch (a.C) {
        case 1: return launch_bw_t<1>(a, st);
        case 2: return launch_bw_t<2>(a, st);
        case 3: return launch_bw_t<3>(a, st);
        case 4: return launch_bw_t<4>(a, st);
        default: return GLU_ERR_UNSUPPORTED;
    }
}

}  // namespace glu
