// Eq. 1 (apply) and its adjoint.
//
// apply, 3-channel float32 targets with aligned rows: the tiled forms below (LR region and a
// pair-code table in shared memory; plain, per-tile TMA and persistent TMA-pipeline variants,
// chosen by the autotuner). Other targets: one thread per group of 4 consecutive HR pixels of a
// row, codes and weights streaming from HBM, the two LR gathers hitting L2.
//
// backward (without a workspace; the workspace form is further down):
// grad_lr_q = sum_{p: a_p = q} w_p G_p + sum_{p: b_p = q} (1 - w_p) G_p. The pixels that
// can map to q are bounded by the window: p's block must lie within r of q. One warp owns one
// LR pixel and walks those source blocks in a fixed order (blocks in raster order, lanes strided
// over each block's pixels), then reduces lanes with a fixed butterfly: no atomics, the result
// is bit-reproducible. This is the segmented reduction over the inverse pixel-to-LR map with the
// map left implicit (the window bounds it, so it is never materialised).
#include <algorithm>

#include "internal.h"
#include "tune.h"
#include "variants.h"
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

// Theta decoded into absolute LR pixel indices (row-major, v * w + u) of a and b and float32
// weights, one thread per HR pixel. A code outside the window of its pixel writes -1 for both
// indices and records GLU_ERR_DEVICE_CHECK.
__global__ void k_theta_decode(const uint16_t* __restrict__ code, const void* weight, int wfmt,
                               int H, int W, int s, int S, int h, int w, int32_t* a, int32_t* b,
                               float* wt) {
    const int64_t np = (int64_t)H * W;
    const int K = S * S, r = (S - 1) >> 1;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(p / W), x = (int)(p % W);
        const int c = code[p];
        const int ka = c / K, kb = c % K;
        const int va = y / s + ka / S - r, ua = x / s + ka % S - r;
        const int vb = y / s + kb / S - r, ub = x / s + kb % S - r;
        const bool ok = ka < K && va >= 0 && va < h && ua >= 0 && ua < w && vb >= 0 && vb < h &&
                        ub >= 0 && ub < w;
        if (!ok) set_status(GLU_ERR_DEVICE_CHECK);
        if (a) a[p] = ok ? va * w + ua : -1;
        if (b) b[p] = ok ? vb * w + ub : -1;
        if (wt) wt[p] = load_weight(weight, wfmt, p);
    }
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

// Exact integer quotient n / d for 0 <= n < 2^22 and d >= 1 (pair codes, window indices, rows):
// (n + 0.5) / d stays at least 0.5 / d away from an integer, and the float error of
// (n + 0.5) * fl(1 / d) is below (n + 0.5) / d * 2^-23 < 0.5 / d.
__device__ __forceinline__ int qdiv(int n, float inv_d) {
    return __float2int_rd(((float)n + 0.5f) * inv_d);
}

template <int WF> struct W4;
// load: 4 weights from global memory (streaming); shared: the same from shared memory.
template <> struct W4<GLU_W_F32> {
    static __device__ __forceinline__ void decode(float4 v, float w[4]) {
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
    static __device__ __forceinline__ void load(const void* b, int64_t p, float w[4]) {
        decode(__ldcs((const float4*)b + (p >> 2)), w);
    }
    static __device__ __forceinline__ void shared(const void* b, int p, float w[4]) {
        decode(*((const float4*)b + (p >> 2)), w);
    }
};
template <> struct W4<GLU_W_F16> {
    static __device__ __forceinline__ void decode(uint2 v, float w[4]) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 c = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        w[0] = a.x; w[1] = a.y; w[2] = c.x; w[3] = c.y;
    }
    static __device__ __forceinline__ void load(const void* b, int64_t p, float w[4]) {
        decode(__ldcs((const uint2*)b + (p >> 2)), w);
    }
    static __device__ __forceinline__ void shared(const void* b, int p, float w[4]) {
        decode(*((const uint2*)b + (p >> 2)), w);
    }
};
template <> struct W4<GLU_W_UNORM16> {
    static __device__ __forceinline__ void decode(uint2 v, float w[4]) {
        w[0] = (float)(v.x & 0xFFFFu) * (1.0f / 65535.0f);
        w[1] = (float)(v.x >> 16) * (1.0f / 65535.0f);
        w[2] = (float)(v.y & 0xFFFFu) * (1.0f / 65535.0f);
        w[3] = (float)(v.y >> 16) * (1.0f / 65535.0f);
    }
    static __device__ __forceinline__ void load(const void* b, int64_t p, float w[4]) {
        decode(__ldcs((const uint2*)b + (p >> 2)), w);
    }
    static __device__ __forceinline__ void shared(const void* b, int p, float w[4]) {
        decode(*((const uint2*)b + (p >> 2)), w);
    }
};

// The 12 results of 4 pixels: three 16-byte stores (float32) or three 8-byte stores (float16).
__device__ __forceinline__ void store12(float* out, const float r[12]) {
    float4* o = (float4*)out;
    __stcs(o + 0, make_float4(r[0], r[1], r[2], r[3]));
    __stcs(o + 1, make_float4(r[4], r[5], r[6], r[7]));
    __stcs(o + 2, make_float4(r[8], r[9], r[10], r[11]));
}
// The same into shared memory (the output tile of the TMA kernel).
__device__ __forceinline__ void store12_smem(float* out, const float r[12]) {
    float4* o = (float4*)out;
    o[0] = make_float4(r[0], r[1], r[2], r[3]);
    o[1] = make_float4(r[4], r[5], r[6], r[7]);
    o[2] = make_float4(r[8], r[9], r[10], r[11]);
}
__device__ __forceinline__ void store12_smem(__half* out, const float r[12]) {
    uint2* o = (uint2*)out;
    uint32_t u[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const __half2 h = __floats2half2_rn(r[2 * k], r[2 * k + 1]);
        u[k] = *reinterpret_cast<const uint32_t*>(&h);
    }
    o[0] = make_uint2(u[0], u[1]);
    o[1] = make_uint2(u[2], u[3]);
    o[2] = make_uint2(u[4], u[5]);
}
__device__ __forceinline__ void store12(__half* out, const float r[12]) {
    uint2* o = (uint2*)out;
    uint32_t u[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const __half2 h = __floats2half2_rn(r[2 * k], r[2 * k + 1]);
        u[k] = *reinterpret_cast<const uint32_t*>(&h);
    }
    __stcs(o + 0, make_uint2(u[0], u[1]));
    __stcs(o + 1, make_uint2(u[2], u[3]));
    __stcs(o + 2, make_uint2(u[4], u[5]));
}

// Largest LR region (rows x columns) a tile of TH x kApplyTW HR pixels reaches, in float4 cells.
__host__ __device__ __forceinline__ int apply_region_cells(int th, int s, int S) {
    const int r = (S - 1) / 2;
    return ((th - 1) / s + 2 + 2 * r) * ((kApplyTW - 1) / s + 2 + 2 * r);
}

// Geometry of one tile's windows in its LR region (shared by the tiled kernels below).
struct TileGeom {
    int s, S, r, K, K2, RW, v0;
    bool interior;            // every window of the tile inside the LR image
    int wcol[4], pxj[4];      // per pixel of the thread's group: window corner column, LR column
    float invs, invK, invS;
};

// Eq. 1 for the thread's 4 consecutive pixels of HR row y: pair codes packed in cc, weights w.
// Codes that would leave the LR image (not produced by the search) are recorded as
// GLU_ERR_DEVICE_CHECK and redirected to the region's first cell.
__device__ __forceinline__ void apply_row4(const ApplyArgs& P, const float4* reg4,
                                           const uint32_t* tab, const TileGeom& g, int y,
                                           uint2 cc, const float w[4], float res[12]) {
    const int py = qdiv(y, g.invs);
    const int rowbase = (py - g.r - g.v0) * g.RW;   // region row of the window's top row
    const int code[4] = {(int)(cc.x & 0xFFFFu), (int)(cc.x >> 16), (int)(cc.y & 0xFFFFu),
                         (int)(cc.y >> 16)};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int base = rowbase + g.wcol[j];
        const int c = code[j];
        int ia, ib;
        if (c < g.K2) {
            const uint32_t t = tab[c];
            ia = base + (int)(t & 0xFFFFu);
            ib = base + (int)(t >> 16);
        } else {
            set_status(GLU_ERR_DEVICE_CHECK);
            ia = ib = 0;
        }
        if (!g.interior) {
            const int ka = qdiv(c, g.invK), kb = c - ka * g.K;
            const int ra = qdiv(ka, g.invS), rb = qdiv(kb, g.invS);
            const int va = py + ra - g.r, ua = g.pxj[j] + (ka - ra * g.S) - g.r;
            const int vb = py + rb - g.r, ub = g.pxj[j] + (kb - rb * g.S) - g.r;
            if ((unsigned)va >= (unsigned)P.h || (unsigned)ua >= (unsigned)P.w) {
                set_status(GLU_ERR_DEVICE_CHECK);
                ia = 0;
            }
            if ((unsigned)vb >= (unsigned)P.h || (unsigned)ub >= (unsigned)P.w) {
                set_status(GLU_ERR_DEVICE_CHECK);
                ib = 0;
            }
        }
        const float4 ta = reg4[ia], tb = reg4[ib];
        res[j * 3 + 0] = __fmaf_rn(w[j], ta.x - tb.x, tb.x);
        res[j * 3 + 1] = __fmaf_rn(w[j], ta.y - tb.y, tb.y);
        res[j * 3 + 2] = __fmaf_rn(w[j], ta.z - tb.z, tb.z);
    }
}

// The LR region of a tile (clamped to the image: entries outside it are never selected by a
// valid code) and the pair-code table: code -> (cell of T_a, cell of T_b) relative to the
// window corner, by float-reciprocal quotients (exact for these small operands).
__device__ __forceinline__ void stage_region_table(const ApplyArgs& P, float4* reg4, uint32_t* tab,
                                                   int RH, int RW, int v0, int u0,
                                                   const TileGeom& g, bool table = true) {
    const float* T = (const float*)P.T;
    const float invRW = 1.0f / (float)RW;
    for (int i = threadIdx.x; i < RH * RW; i += blockDim.x) {
        const int rr = qdiv(i, invRW), c1 = i - rr * RW;
        const int v = min(max(v0 + rr, 0), P.h - 1);
        const int u = min(max(u0 + c1, 0), P.w - 1);
        const float* t = T + (int64_t)v * P.T_pitch + (int64_t)u * 3;
        reg4[i] = make_float4(__ldg(t), __ldg(t + 1), __ldg(t + 2), 0.f);
    }
    if (!table) return;
    for (int c = threadIdx.x; c < g.K2; c += blockDim.x) {
        const int ka = qdiv(c, g.invK), kb = c - ka * g.K;
        const int ra = qdiv(ka, g.invS), rb = qdiv(kb, g.invS);
        const uint32_t oa = (uint32_t)(ra * RW + (ka - ra * g.S));
        const uint32_t ob = (uint32_t)(rb * RW + (kb - rb * g.S));
        tab[c] = oa | (ob << 16);
    }
}

__device__ __forceinline__ TileGeom tile_geom(const ApplyArgs& P, int x0, int y0, int xe, int ye,
                                              int xs, int RW, int v0, int u0) {
    TileGeom g;
    g.s = P.s;
    g.S = P.S;
    g.r = (P.S - 1) >> 1;
    g.K = P.S * P.S;
    g.K2 = g.K * g.K;
    g.RW = RW;
    g.v0 = v0;
    g.invs = 1.0f / (float)g.s;
    g.invK = 1.0f / (float)g.K;
    g.invS = 1.0f / (float)g.S;
    g.interior = v0 >= 0 && u0 >= 0 && qdiv(ye - 1, g.invs) + g.r < P.h &&
                 qdiv(xe - 1, g.invs) + g.r < P.w;
    // window corner columns of the 4 pixels in the region: xs / s once, then at most three
    // block boundaries within the next 3 pixels
    const int c0 = qdiv(xs, g.invs), rem = xs - c0 * g.s;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        g.pxj[j] = c0 + (rem + j >= g.s) + (rem + j >= 2 * g.s) + (rem + j >= 3 * g.s);
        g.wcol[j] = g.pxj[j] - g.r - u0;
    }
    return g;
}

// Eq. 1 fast path, tiled: a CTA owns TH x kApplyTW HR pixels (a warp per row, 4 pixels per
// lane). The LR region its windows reach is copied to shared memory with coalesced row loads,
// so the 8 gathers per 4 pixels are shared-memory reads, and a per-CTA table turns a pair code
// into the two region offsets relative to the window's corner (one lookup instead of the code's
// division into window rows and columns). Codes and weights stream in as one 8-/16-byte load
// per 4 pixels, results leave as three 16- (float32) or 8-byte (float16) streaming stores.
// Conditions: 3 channels, float32 target, W % 4 == 0, aligned rows.
template <int WF, typename OT, int TH>
__global__ void __launch_bounds__(32 * (TH < 8 ? TH : 8)) k_apply3_tile(const ApplyArgs P) {
    constexpr int NW = TH < 8 ? TH : 8;   // warps: one row each, RPW rows per warp
    constexpr int RPW = TH / NW;
    extern __shared__ float4 reg4[];   // RH x RW region (RGB_), then K*K offset pairs
    const int x0 = blockIdx.x * kApplyTW, y0 = blockIdx.y * TH;
    const int s = P.s, S = P.S, r = (S - 1) >> 1;
    const int xe = min(x0 + kApplyTW, P.W), ye = min(y0 + TH, P.H);
    const float inv_s = 1.0f / (float)s;   // exact quotients (qdiv)
    const int v0 = qdiv(y0, inv_s) - r, u0 = qdiv(x0, inv_s) - r;
    const int RH = qdiv(ye - 1, inv_s) + r - v0 + 1, RW = qdiv(xe - 1, inv_s) + r - u0 + 1;
    uint32_t* tab = (uint32_t*)(reg4 + apply_region_cells(TH, s, S));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int xs = x0 + lane * 4;
    const bool col_ok = xs < P.W;
    // this thread's codes and weights first: they do not wait for the LR region
    uint2 cc[RPW];
    float w[RPW][4];
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int y = y0 + wid + k * NW;
        cc[k] = make_uint2(0u, 0u);
        if (col_ok && y < P.H) {
            const int64_t p0 = (int64_t)y * P.W + xs;
            cc[k] = __ldcs((const uint2*)P.code + (p0 >> 2));
            W4<WF>::load(P.weight, p0, w[k]);
        }
    }
    const TileGeom g = tile_geom(P, x0, y0, xe, ye, xs, RW, v0, u0);
    stage_region_table(P, reg4, tab, RH, RW, v0, u0, g);
    __syncthreads();
    if (!col_ok) return;
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int y = y0 + wid + k * NW;
        if (y >= P.H) break;
        float res[12];
        apply_row4(P, reg4, tab, g, y, cc[k], w[k], res);
        store12((OT*)P.out + (int64_t)y * P.out_pitch + (int64_t)xs * 3, res);
    }
}

// The same tile with the tensor memory accelerator: the tile's codes and weights arrive by two
// 2D TMA loads (mbarrier completion, bounded wait) while the CTA stages the LR region; results
// go to a shared-memory output tile, written back by TMA stores (two boxes of 64 pixels x 3
// channels per row band: a box row holds at most 256 elements). Every global access of the
// streaming data is then a full-line bulk copy. Same arithmetic as k_apply3_tile.
template <int WF, typename OT, int TH>
__global__ void __launch_bounds__(256) k_apply3_tma(const ApplyArgs P,
                                                    const __grid_constant__ CUtensorMap mcode,
                                                    const __grid_constant__ CUtensorMap mw,
                                                    const __grid_constant__ CUtensorMap mout) {
    constexpr int NW = 8, RPW = TH / NW;
    constexpr int WB = WF == GLU_W_F32 ? 4 : 2;          // weight bytes
    constexpr int HALF = kApplyTW / 2 * 3;               // output elements per box row
    static_assert(TH % NW == 0, "whole rows per warp");
    extern __shared__ __align__(128) unsigned char sm_raw[];
    // TMA boxes start on 128-byte boundaries of the shared window (the launch adds 128 bytes)
    unsigned char* sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);
    uint16_t* scode = (uint16_t*)sm;                                 // [TH][128]
    unsigned char* sw = sm + TH * kApplyTW * 2;                      // [TH][128] weights
    OT* sout = (OT*)(sw + TH * kApplyTW * WB);                       // [2][TH][HALF]
    uint64_t* bar = (uint64_t*)((unsigned char*)sout + 2 * TH * HALF * sizeof(OT));
    float4* reg4 = (float4*)(bar + 2);
    const int x0 = blockIdx.x * kApplyTW, y0 = blockIdx.y * TH;
    const int s = P.s, S = P.S, r = (S - 1) >> 1;
    const int xe = min(x0 + kApplyTW, P.W), ye = min(y0 + TH, P.H);
    const float inv_s = 1.0f / (float)s;   // exact quotients (qdiv)
    const int v0 = qdiv(y0, inv_s) - r, u0 = qdiv(x0, inv_s) - r;
    const int RH = qdiv(ye - 1, inv_s) + r - v0 + 1, RW = qdiv(xe - 1, inv_s) + r - u0 + 1;
    uint32_t* tab = (uint32_t*)(reg4 + apply_region_cells(TH, s, S));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int xs = x0 + lane * 4;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)(TH * kApplyTW * (2 + WB)));
        tma_load_2d(scode, &mcode, bar, x0, y0);
        tma_load_2d(sw, &mw, bar, x0, y0);
    }
    const TileGeom g = tile_geom(P, x0, y0, xe, ye, xs, RW, v0, u0);
    stage_region_table(P, reg4, tab, RH, RW, v0, u0, g);
    __syncthreads();
    const bool ok = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(ok ? 0 : 1)) {
        if (threadIdx.x == 0) set_status(GLU_ERR_TIMEOUT);
        (void)mbar_wait_bounded(bar, 0);   // the copies may still land: wait before leaving
        return;
    }
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int row = wid + k * NW, y = y0 + row;
        float res[12];
        if (y < P.H && xs < P.W) {
            const uint2 cc = *(const uint2*)&scode[row * kApplyTW + lane * 4];
            float w[4];
            W4<WF>::shared(sw + (size_t)row * kApplyTW * WB, lane * 4, w);
            apply_row4(P, reg4, tab, g, y, cc, w, res);
        } else {
#pragma unroll
            for (int j = 0; j < 12; ++j) res[j] = 0.f;   // outside the image: not stored
        }
        store12_smem(sout + ((lane >> 4) * TH + row) * HALF + (lane & 15) * 12, res);
    }
    // the output tile is complete in shared memory: make it visible to the async proxy
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        tma_store_2d(&mout, sout, x0 * 3, y0);
        if ((x0 + kApplyTW / 2) < P.W) tma_store_2d(&mout, sout + TH * HALF, x0 * 3 + HALF, y0);
        tma_store_commit_wait_read();   // shared memory stays valid until the stores read it
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

int launch_theta_decode(const uint16_t* code, const void* weight, int wfmt, int H, int W, int s,
                        int S, int32_t* a, int32_t* b, float* wt, cudaStream_t st) {
    const int64_t np = (int64_t)H * W;
    if (np == 0) return GLU_OK;
    const int threads = 256;
    k_theta_decode<<<grid_for(np, threads), threads, 0, st>>>(
        code, weight, wfmt, H, W, s, S, (H + s - 1) / s, (W + s - 1) / s, a, b, wt);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

// The LR region of a tile copied into float4 cells (RGB_) by 4-byte asynchronous copies, one
// commit group per call (clamped to the image: cells outside it are never selected by a valid
// code); completed by cp_async_wait_all() and a barrier.
__device__ __forceinline__ void prefetch_region(const ApplyArgs& P, float4* reg4, int RH, int RW,
                                                int v0, int u0) {
    const float* T = (const float*)P.T;
    const float invRW = 1.0f / (float)RW;
    for (int i = threadIdx.x; i < RH * RW; i += blockDim.x) {
        const int rr = qdiv(i, invRW), c1 = i - rr * RW;
        const int v = min(max(v0 + rr, 0), P.h - 1);
        const int u = min(max(u0 + c1, 0), P.w - 1);
        const float* t = T + (int64_t)v * P.T_pitch + (int64_t)u * 3;
        float* d = reinterpret_cast<float*>(reg4 + i);
        cp_async4(d, t);
        cp_async4(d + 1, t + 1);
        cp_async4(d + 2, t + 2);
    }
    cp_async_commit();
}

// The pair-code table of a region of width RW (see stage_region_table).
__device__ __forceinline__ void build_pair_table(uint32_t* tab, int RW, int S) {
    const int K = S * S, K2 = K * K;
    const float invK = 1.0f / (float)K, invS = 1.0f / (float)S;
    for (int c = threadIdx.x; c < K2; c += blockDim.x) {
        const int ka = qdiv(c, invK), kb = c - ka * K;
        const int ra = qdiv(ka, invS), rb = qdiv(kb, invS);
        const uint32_t oa = (uint32_t)(ra * RW + (ka - ra * S));
        const uint32_t ob = (uint32_t)(rb * RW + (kb - rb * S));
        tab[c] = oa | (ob << 16);
    }
}

// Persistent form of k_apply3_tma: a CTA walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x,
// ... with the codes and weights of the next two tiles in flight (two TMA stages, one mbarrier
// each), the output of the previous tile still being written by its TMA store (two output
// buffers) while it computes the current one, and (nreg = 2) the next tile's LR region arriving
// by asynchronous copies into a second region buffer (each with its own pair-code table) while
// the current one is computed; with nreg = 1 (a region too large for two buffers) the region is
// refilled between tiles. The LR target is first read after griddep_wait(), so the kernel may be
// launched as the programmatic dependent of the kernel that writes the target: the codes and
// weights of its first tiles are then already loading. Same arithmetic as k_apply3_tile.
template <int WF, typename OT, int TH>
__global__ void __launch_bounds__(256) k_apply3_pipe(const ApplyArgs P,
                                                     const __grid_constant__ CUtensorMap mcode,
                                                     const __grid_constant__ CUtensorMap mw,
                                                     const __grid_constant__ CUtensorMap mout,
                                                     int tiles_x, int ntiles, int nreg) {
    constexpr int NW = 8, RPW = TH / NW;
    constexpr int WB = WF == GLU_W_F32 ? 4 : 2;
    constexpr int HALF = kApplyTW / 2 * 3;
    constexpr int IN_BYTES = TH * kApplyTW * (2 + WB);              // codes, then weights
    constexpr int OUT_BYTES = 2 * TH * HALF * (int)sizeof(OT);      // two boxes of HALF columns
    static_assert(TH % NW == 0 && IN_BYTES % 128 == 0 && OUT_BYTES % 128 == 0, "tile layout");
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);
    unsigned char* sin = sm;                                         // [2][IN_BYTES]
    OT* sout = (OT*)(sm + 2 * IN_BYTES);                             // [2][OUT_BYTES]
    uint64_t* bar = (uint64_t*)(sm + 2 * IN_BYTES + 2 * OUT_BYTES);  // [2]
    const int s = P.s, S = P.S, r = (S - 1) >> 1;
    const int cells = apply_region_cells(TH, s, S), K2 = S * S * S * S;
    float4* regb = (float4*)(bar + 2);                               // [nreg][cells]
    uint32_t* tabb = (uint32_t*)(regb + nreg * cells);               // [nreg][K2]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float inv_s = 1.0f / (float)s;   // exact quotients (qdiv)
    auto issue = [&](int stage, int t) {   // thread 0 only
        const int x0 = (t % tiles_x) * kApplyTW, y0 = (t / tiles_x) * TH;
        mbar_arrive_expect_tx(&bar[stage], (uint32_t)IN_BYTES);
        tma_load_2d(sin + stage * IN_BYTES, &mcode, &bar[stage], x0, y0);
        tma_load_2d(sin + stage * IN_BYTES + TH * kApplyTW * 2, &mw, &bar[stage], x0, y0);
    };
    int tab_rw0 = -1, tab_rw1 = -1;   // region width each buffer's table holds offsets for
    // start the region copy of tile t into buffer b (and its table if the width changed)
    auto fill = [&](int b, int t) {
        const int x0 = (t % tiles_x) * kApplyTW, y0 = (t / tiles_x) * TH;
        const int xe = min(x0 + kApplyTW, P.W), ye = min(y0 + TH, P.H);
        const int v0 = qdiv(y0, inv_s) - r, u0 = qdiv(x0, inv_s) - r;
        const int RH = qdiv(ye - 1, inv_s) + r - v0 + 1, RW = qdiv(xe - 1, inv_s) + r - u0 + 1;
        prefetch_region(P, regb + b * cells, RH, RW, v0, u0);
        int& trw = b ? tab_rw1 : tab_rw0;
        if (RW != trw) {
            build_pair_table(tabb + b * K2, RW, S);
            trw = RW;
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        if (blockIdx.x < ntiles) issue(0, blockIdx.x);
        if (blockIdx.x + gridDim.x < ntiles) issue(1, blockIdx.x + gridDim.x);
    }
    griddep_wait();   // the LR target is complete from here on
    if (blockIdx.x < ntiles) fill(0, blockIdx.x);
    int i = 0;
    bool failed = false;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const int stage = i & 1;
        const uint32_t phase = (uint32_t)(i >> 1) & 1u;
        const int rb = nreg == 2 ? stage : 0;
        const int x0 = (t % tiles_x) * kApplyTW, y0 = (t / tiles_x) * TH;
        const int xe = min(x0 + kApplyTW, P.W), ye = min(y0 + TH, P.H);
        const int v0 = qdiv(y0, inv_s) - r, u0 = qdiv(x0, inv_s) - r;
        const int RW = qdiv(xe - 1, inv_s) + r - u0 + 1;
        const int xs = x0 + lane * 4;
        const TileGeom g = tile_geom(P, x0, y0, xe, ye, xs, RW, v0, u0);
        cp_async_wait_all();   // this thread's copies of this tile's region have landed
        // this stage's output buffer was last written out two tiles ago: its store must have
        // read it (one younger store group may still be reading the other buffer)
        if (threadIdx.x == 0 && i >= 2) tma_store_wait_read_1();
        __syncthreads();   // the region and its table are complete; tile i-1 is finished
        const int tn = t + gridDim.x;
        if (nreg == 2 && tn < ntiles) fill(rb ^ 1, tn);   // the next region, while computing
        const bool ok = mbar_wait_bounded(&bar[stage], phase);
        if (__syncthreads_or(ok ? 0 : 1)) {
            failed = true;
            break;
        }
        const unsigned char* cin = sin + stage * IN_BYTES;
        OT* cout = sout + stage * (OUT_BYTES / (int)sizeof(OT));
        const float4* reg4 = regb + rb * cells;
        const uint32_t* tab = tabb + rb * K2;
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int row = wid + k * NW, y = y0 + row;
            float res[12];
            if (y < P.H && xs < P.W) {
                const uint2 cc = *(const uint2*)(cin + (row * kApplyTW + lane * 4) * 2);
                float w[4];
                W4<WF>::shared(cin + TH * kApplyTW * 2 + (size_t)row * kApplyTW * WB, lane * 4,
                               w);
                apply_row4(P, reg4, tab, g, y, cc, w, res);
            } else {
#pragma unroll
                for (int j = 0; j < 12; ++j) res[j] = 0.f;   // outside the image: not stored
            }
            store12_smem(cout + ((lane >> 4) * TH + row) * HALF + (lane & 15) * 12, res);
        }
        fence_proxy_async_smem();
        __syncthreads();   // the output tile is complete and this stage's inputs are consumed
        if (threadIdx.x == 0) {
            tma_store_2d(&mout, cout, x0 * 3, y0);
            if (x0 + kApplyTW / 2 < P.W) tma_store_2d(&mout, cout + TH * HALF, x0 * 3 + HALF, y0);
            tma_store_commit();
            if (t + 2 * (int)gridDim.x < ntiles) issue(stage, t + 2 * gridDim.x);
        }
        if (nreg == 1 && tn < ntiles) fill(0, tn);   // the single buffer is free again
    }
    cp_async_wait_all();   // no copy of this thread is left in flight
    if (threadIdx.x == 0) {
        if (failed) {
            set_status(GLU_ERR_TIMEOUT);
            // loads still in flight land before the CTA leaves (bounded waits)
            (void)mbar_wait_bounded(&bar[i & 1], (uint32_t)(i >> 1) & 1u);
            if (blockIdx.x + (i + 1) * (int)gridDim.x < ntiles)
                (void)mbar_wait_bounded(&bar[(i + 1) & 1], (uint32_t)((i + 1) >> 1) & 1u);
        }
        tma_store_commit_wait_read();   // every store has read its shared-memory source
    }
}

// k_apply3_tile / k_apply3_tma with TH rows for a weight format and output type.
template <template <int, typename, int> class KT, int TH, typename F>
static int apply_kernel_for(int wfmt, bool out_f16, F&& launch) {
    if (out_f16) {
        if (wfmt == GLU_W_F32) return launch(KT<GLU_W_F32, __half, TH>::fn());
        if (wfmt == GLU_W_F16) return launch(KT<GLU_W_F16, __half, TH>::fn());
        return launch(KT<GLU_W_UNORM16, __half, TH>::fn());
    }
    if (wfmt == GLU_W_F32) return launch(KT<GLU_W_F32, float, TH>::fn());
    if (wfmt == GLU_W_F16) return launch(KT<GLU_W_F16, float, TH>::fn());
    return launch(KT<GLU_W_UNORM16, float, TH>::fn());
}
template <int WF, typename OT, int TH> struct TileK {
    static auto fn() { return k_apply3_tile<WF, OT, TH>; }
};
template <int WF, typename OT, int TH> struct TmaK {
    static auto fn() { return k_apply3_tma<WF, OT, TH>; }
};
template <int WF, typename OT, int TH> struct PipeK {
    static auto fn() { return k_apply3_pipe<WF, OT, TH>; }
};
template <template <int, typename, int> class KT, typename F>
static int apply_rows_dispatch(int rows, int wfmt, bool out_f16, F&& launch) {
    switch (rows) {
        case 8: return apply_kernel_for<KT, 8>(wfmt, out_f16, launch);
        case 16: return apply_kernel_for<KT, 16>(wfmt, out_f16, launch);
        case 32: return apply_kernel_for<KT, 32>(wfmt, out_f16, launch);
        case 64: return apply_kernel_for<KT, 64>(wfmt, out_f16, launch);
        default: return GLU_ERR_INVALID_ARG;
    }
}

int launch_apply(const ApplyArgs& a, cudaStream_t st) {
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    const int threads = 256;
    const size_t wsz = a.wfmt == GLU_W_F32 ? 16 : 8;
    const bool in_ok = a.C == 3 && a.T_dtype == GLU_F32 && a.W % 4 == 0 && a.out_pitch % 4 == 0 &&
                       ((uintptr_t)a.code & 7u) == 0 && ((uintptr_t)a.weight & (wsz - 1)) == 0;
    const bool vec = in_ok && a.out_dtype == GLU_F32 && ((uintptr_t)a.out & 15u) == 0;
    const bool vec16 = in_ok && a.out_dtype == GLU_F16 && ((uintptr_t)a.out & 7u) == 0;
    if (vec || vec16) {
        // TMA needs 16-byte rows of codes, weights and output and 16-byte aligned bases
        const size_t wb = a.wfmt == GLU_W_F32 ? 4 : 2, ob = vec16 ? 2 : 4;
        CUtensorMap mcode, mw, mout;
        int tma_rows = -1;   // rows the three maps were encoded for
        auto maps_for = [&](int th) -> bool {
            if (tma_rows == th) return true;
            const bool ok =
                encode_map_2d(&mcode, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, a.code, a.W, a.H,
                              (uint64_t)a.W * 2, kApplyTW, th) &&
                encode_map_2d(&mw, wb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                              wb, a.weight, a.W, a.H, (uint64_t)a.W * wb, kApplyTW, th) &&
                encode_map_2d(&mout, vec16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                           : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              ob, a.out, (uint64_t)a.W * 3, a.H, (uint64_t)a.out_pitch * ob,
                              kApplyTW / 2 * 3, th);
            tma_rows = ok ? th : -1;
            return ok;
        };
        auto run = [&](int v) -> int {
            const int th = kApplyVariants[v].rows;
            const size_t region = sizeof(float4) * (size_t)apply_region_cells(th, a.s, a.S) +
                                  sizeof(uint32_t) * (size_t)(a.S * a.S) * (a.S * a.S);
            const dim3 grid((a.W + kApplyTW - 1) / kApplyTW, (a.H + th - 1) / th);
            if (kApplyVariants[v].tma == 2 && maps_for(th)) {
                const int tiles_x = (a.W + kApplyTW - 1) / kApplyTW;
                const int ntiles = tiles_x * ((a.H + th - 1) / th);
                const size_t fixed = 128 + 2 * (size_t)th * kApplyTW * (2 + wb) +
                                     4 * (size_t)th * (kApplyTW / 2 * 3) * ob + 16;
                auto launch = [&](auto kern) -> int {
                    int dev = 0, sms = 148, per_sm = 1, optin = 48 * 1024;
                    GLU_CUDA_TRY(cudaGetDevice(&dev));
                    GLU_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
                    GLU_CUDA_TRY(cudaDeviceGetAttribute(
                        &optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
                    // two region buffers when they fit (the next region loads during a tile)
                    const int nreg = fixed + 2 * region <= (size_t)optin ? 2 : 1;
                    const size_t smem = fixed + nreg * region;
                    if (smem > 48 * 1024 &&
                        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem) != cudaSuccess)
                        return GLU_ERR_CUDA;
                    GLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256,
                                                                               smem));
                    const int grid = std::max(1, std::min(ntiles, sms * std::max(per_sm, 1)));
                    cudaLaunchConfig_t cfg = {};
                    cfg.gridDim = dim3(grid);
                    cfg.blockDim = dim3(256);
                    cfg.dynamicSmemBytes = smem;
                    cfg.stream = st;
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                    attr[0].val.programmaticStreamSerializationAllowed = 1;
                    cfg.attrs = attr;
                    cfg.numAttrs = a.pdl ? 1 : 0;
                    GLU_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, a, mcode, mw, mout, tiles_x,
                                                    ntiles, nreg));
                    return GLU_OK;
                };
                return apply_rows_dispatch<PipeK>(th, a.wfmt, vec16, launch);
            }
            if (kApplyVariants[v].tma == 1 && maps_for(th)) {
                const size_t smem = 128 + (size_t)th * kApplyTW * (2 + wb) +
                                    2 * (size_t)th * (kApplyTW / 2 * 3) * ob + 16 + region;
                auto launch = [&](auto kern) -> int {
                    if (smem > 48 * 1024 &&
                        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem) != cudaSuccess)
                        return GLU_ERR_CUDA;
                    kern<<<grid, 256, smem, st>>>(a, mcode, mw, mout);
                    GLU_LAUNCH_CHECK();
                    return GLU_OK;
                };
                return apply_rows_dispatch<TmaK>(th, a.wfmt, vec16, launch);
            }
            const int nthr = 32 * (th < 8 ? th : 8);
            auto launch = [&](auto kern) -> int {
                if (region > 48 * 1024 &&
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)region) != cudaSuccess)
                    return GLU_ERR_CUDA;
                kern<<<grid, nthr, region, st>>>(a);
                GLU_LAUNCH_CHECK();
                return GLU_OK;
            };
            return apply_rows_dispatch<TileK>(th, a.wfmt, vec16, launch);
        };
        const int key[5] = {a.out_dtype, a.wfmt, a.S, a.s, tune_size_class((long long)a.H * a.W)};
        int v = 0;
        const int rc = tune_choose(kTuneApply, key, kNumApplyVariants, run, st, &v);
        if (rc) return rc;
        return run(v);
    }
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

// The LR-gradient sums of k_apply_backward_lr with the HR pixels a tile of TxT LR pixels depends
// on (its blocks within r, i.e. the pixels whose windows can reach it) staged in shared memory
// once: decoded pair, weight and upstream gradient. Every input is read from HBM about
// (1 + 2r/T)^2 times instead of (2r+1)^2 times, and the scan touches shared memory only. Same
// loops, same order, same results.
template <int C>
__global__ void __launch_bounds__(256) k_apply_backward_lr_tile(const BackwardArgs P, int T) {
    // RH x RW HR pixels of the region: pair (k_a | k_b << 8), weight, upstream gradient
    extern __shared__ float rsm[];
    const int r = (P.S - 1) >> 1, K = P.S * P.S;
    const float invK = 1.0f / (float)K;
    const int v0 = blockIdx.y * T, u0 = blockIdx.x * T;
    const int bv0 = max(v0 - r, 0), bv1 = min(v0 + T + r, P.h);
    const int bu0 = max(u0 - r, 0), bu1 = min(u0 + T + r, P.w);
    const int y0 = bv0 * P.s, y1 = min(bv1 * P.s, P.H);
    const int x0 = bu0 * P.s, x1 = min(bu1 * P.s, P.W);
    const int RW = x1 - x0, RH = y1 - y0, NR = RH * RW;
    float* rg = rsm;                                   // NR x C
    float* rw = rsm + (size_t)NR * C;                  // NR
    uint16_t* rpair = (uint16_t*)(rw + NR);            // NR
    // staged four pixels per thread at a time, loads first (each code decoded once per CTA; a
    // code outside the window range matches no LR pixel)
    constexpr int kU = 4;
    for (int i0 = threadIdx.x; i0 < NR; i0 += blockDim.x * kU) {
        int code[kU];
        float w[kU], g[kU][C];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int i = i0 + k * blockDim.x;
            code[k] = 0;
            if (i < NR) {
                const int yy = i / RW, xx = i - yy * RW;
                const int64_t p = (int64_t)(y0 + yy) * P.W + x0 + xx;
                code[k] = P.code[p];
                w[k] = load_weight(P.weight, P.wfmt, p);
                const int64_t og = (int64_t)(y0 + yy) * P.G_pitch + (int64_t)(x0 + xx) * C;
#pragma unroll
                for (int c = 0; c < C; ++c) g[k][c] = __ldcs(&P.G[og + c]);
            }
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int i = i0 + k * blockDim.x;
            if (i < NR) {
                const int ka = qdiv(code[k], invK), kb = code[k] - ka * K;
                rpair[i] = code[k] < K * K ? (uint16_t)(ka | (kb << 8)) : (uint16_t)0xFFFFu;
                rw[i] = w[k];
#pragma unroll
                for (int c = 0; c < C; ++c) rg[(size_t)i * C + c] = g[k][c];
            }
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    // a full s x s block: lane j's pixels sit at fixed offsets from the block's corner (rows
    // advance by 32 / s per step when s divides 32); blocks cut by the image edge take the
    // general loop
    const int s = P.s;
    const bool pow2 = s <= 32 && (32 % s) == 0;
    const int lane_dy = pow2 ? lane / s : 0, lane_dx = pow2 ? lane % s : 0;
    const int step = pow2 ? (32 / s) * RW : 0;
    const int nstep = pow2 ? (s * s + 31) / 32 : 0;
    const int lane_off = lane_dy * RW + lane_dx;
    for (int t = threadIdx.x >> 5; t < T * T; t += warps) {
        const int v = v0 + t / T, u = u0 + t % T;
        if (v >= P.h || u >= P.w) continue;   // warp-uniform
        float acc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = 0.f;
        for (int bv = max(0, v - r); bv <= min(P.h - 1, v + r); ++bv) {
            const int ys = bv * s;
            for (int bu = max(0, u - r); bu <= min(P.w - 1, u + r); ++bu) {
                // window index of q as seen from pixels of block (bv, bu)
                const int kq = (v - bv + r) * P.S + (u - bu + r);
                const int xs = bu * s;
                const bool full = pow2 && ys + s <= P.H && xs + s <= P.W;
                if (full) {
                    int i = (ys - y0) * RW + (xs - x0) + lane_off;
                    for (int k = 0; k < nstep; ++k, i += step) {
                        if (k * 32 + lane >= s * s) break;
                        const int pr = rpair[i];
                        const int ka = pr & 0xFF, kb = pr >> 8;
                        if (ka != kq && kb != kq) continue;
                        const float w = rw[i];
                        const float f = (ka == kq ? w : 0.f) + (kb == kq ? 1.f - w : 0.f);
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            acc[c] = __fmaf_rn(f, rg[(size_t)i * C + c], acc[c]);
                    }
                } else {
                    const int ey = min(s, P.H - ys), ex = min(s, P.W - xs);
                    const float inv_ex = 1.0f / (float)ex;
                    for (int j = lane; j < ey * ex; j += 32) {
                        const int jy = qdiv(j, inv_ex), jx = j - jy * ex;
                        const int i = (ys + jy - y0) * RW + (xs + jx - x0);
                        const int pr = rpair[i];
                        const int ka = pr & 0xFF, kb = pr >> 8;
                        if (ka != kq && kb != kq) continue;
                        const float w = rw[i];
                        const float f = (ka == kq ? w : 0.f) + (kb == kq ? 1.f - w : 0.f);
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            acc[c] = __fmaf_rn(f, rg[(size_t)i * C + c], acc[c]);
                    }
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

// grad_w of the adjoint for 3 channels, tiled like k_apply3_tile: the LR target region and the
// code -> cell table in shared memory, the upstream gradient streamed in as three 16-byte loads
// per 4 pixels, the 4 results stored as one 16-byte store. Same arithmetic and order as
// k_apply_backward_w. Conditions: float32 target and gradient, W % 4 == 0, aligned rows.
template <int TH>
__global__ void __launch_bounds__(32 * (TH < 8 ? TH : 8)) k_apply3_gw_tile(const BackwardArgs P) {
    constexpr int NW = TH < 8 ? TH : 8;
    constexpr int RPW = TH / NW;
    extern __shared__ float4 reg4[];   // RH x RW region (RGB_), then K*K offset pairs
    const int x0 = blockIdx.x * kApplyTW, y0 = blockIdx.y * TH;
    const int s = P.s, S = P.S, r = (S - 1) >> 1, K = S * S, K2 = K * K;
    const int xe = min(x0 + kApplyTW, P.W), ye = min(y0 + TH, P.H);
    const int v0 = y0 / s - r, u0 = x0 / s - r;
    const int RH = (ye - 1) / s + r - v0 + 1, RW = (xe - 1) / s + r - u0 + 1;
    uint32_t* tab = (uint32_t*)(reg4 + apply_region_cells(TH, s, S));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int xs = x0 + lane * 4;
    const bool col_ok = xs < P.W;
    uint2 cc[RPW];
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int y = y0 + wid + k * NW;
        cc[k] = make_uint2(0u, 0u);
        if (col_ok && y < P.H) cc[k] = __ldcs((const uint2*)P.code + (((int64_t)y * P.W + xs) >> 2));
    }
    for (int i = threadIdx.x; i < RH * RW; i += blockDim.x) {
        const int rr = i / RW, c1 = i - rr * RW;
        const int v = min(max(v0 + rr, 0), P.h - 1);
        const int u = min(max(u0 + c1, 0), P.w - 1);
        const float* t = P.T + (int64_t)v * P.T_pitch + (int64_t)u * 3;
        reg4[i] = make_float4(__ldg(t), __ldg(t + 1), __ldg(t + 2), 0.f);
    }
    for (int c = threadIdx.x; c < K2; c += blockDim.x) {
        const int ka = c / K, kb = c - ka * K;
        tab[c] = (uint32_t)((ka / S) * RW + ka % S) | ((uint32_t)((kb / S) * RW + kb % S) << 16);
    }
    __syncthreads();
    if (!col_ok) return;
    const bool interior = v0 >= 0 && u0 >= 0 && (ye - 1) / s + r < P.h && (xe - 1) / s + r < P.w;
    const int c0 = xs / s, rem = xs - c0 * s;
    int wcol[4], pxj[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        pxj[j] = c0 + (rem + j >= s) + (rem + j >= 2 * s) + (rem + j >= 3 * s);
        wcol[j] = pxj[j] - r - u0;
    }
    const float invK = 1.0f / (float)K, invS = 1.0f / (float)S;
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int y = y0 + wid + k * NW;
        if (y >= P.H) break;
        const float4* g4 = (const float4*)(P.G + (int64_t)y * P.G_pitch + (int64_t)xs * 3);
        const float4 ga = __ldcs(g4), gb = __ldcs(g4 + 1), gc = __ldcs(g4 + 2);
        const float g[12] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w, gc.x, gc.y, gc.z, gc.w};
        const int py = y / s;
        const int rowbase = (py - r - v0) * RW;
        const int code[4] = {(int)(cc[k].x & 0xFFFFu), (int)(cc[k].x >> 16),
                             (int)(cc[k].y & 0xFFFFu), (int)(cc[k].y >> 16)};
        float res[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int base = rowbase + wcol[j];
            const int c = code[j];
            int ia, ib;
            if (c < K2) {
                const uint32_t t = tab[c];
                ia = base + (int)(t & 0xFFFFu);
                ib = base + (int)(t >> 16);
            } else {
                set_status(GLU_ERR_DEVICE_CHECK);
                ia = ib = 0;
            }
            if (!interior) {
                const int ka = qdiv(c, invK), kb = c - ka * K;
                const int ra = qdiv(ka, invS), rb = qdiv(kb, invS);
                const int va = py + ra - r, ua = pxj[j] + (ka - ra * S) - r;
                const int vb = py + rb - r, ub = pxj[j] + (kb - rb * S) - r;
                if ((unsigned)va >= (unsigned)P.h || (unsigned)ua >= (unsigned)P.w) {
                    set_status(GLU_ERR_DEVICE_CHECK);
                    ia = 0;
                }
                if ((unsigned)vb >= (unsigned)P.h || (unsigned)ub >= (unsigned)P.w) {
                    set_status(GLU_ERR_DEVICE_CHECK);
                    ib = 0;
                }
            }
            const float4 ta = reg4[ia], tb = reg4[ib];
            float acc = 0.f;
            acc = __fmaf_rn(g[j * 3 + 0], ta.x - tb.x, acc);
            acc = __fmaf_rn(g[j * 3 + 1], ta.y - tb.y, acc);
            acc = __fmaf_rn(g[j * 3 + 2], ta.z - tb.z, acc);
            res[j] = acc;
        }
        __stcs((float4*)(P.gw + (int64_t)y * P.W + xs), make_float4(res[0], res[1], res[2], res[3]));
    }
}

// ------------------------------------------------------------------ adjoint with a workspace
//
// A pixel p of LR block B contributes to exactly two LR pixels: q_a = the pixel at window index
// k_a of B's window (w_p G_p) and q_b (of k_b, (1 - w_p) G_p). Grouping B's pixels by window
// index therefore gives, per bucket k, B's whole contribution to one LR pixel q = B + (k / S - r,
// k % S - r), of which B is neighbour K - 1 - k (the window is symmetric). Two passes, each input
// read once:
//   k_bw_block_sums: a warp per block stages its pixels in shared memory (and, with grad_w,
//     writes grad_w_p = G_p . (T_a - T_b) on the way); lane k sums bucket k (lanes k, k + 32,
//     k + 64 for windows above 32 pixels) over the block's pixels in raster order and stores the
//     sums in q's slot slots[q][K - 1 - k][a or b][c] of the workspace;
//   k_bw_gather: a thread per LR pixel adds its slots, neighbours in order, a before b.
// Every sum has a fixed order (bit-reproducible); no atomics. (Measured alternative: one fixed
// butterfly per distinct window index of each 64-pixel chunk was slower on textured guides,
// where a block holds many distinct indices.)
constexpr int kBsChunk = 64;    // pixels a warp stages at a time (two per lane)

// Stable counting sort of one 64-pixel chunk by key (key 255: not listed): pixel jj = lane +
// 32 h has key key[h]; writes the chunk indices in key order, raster order inside a key, to
// list[] and the key starts to start[0..K] (start[K] = listed pixels). cnt: per-warp scratch of
// K + 1 ints. Warp-uniform.
__device__ __forceinline__ void chunk_sort(const int (&key)[2], int K, int* cnt, int* start,
                                           uint8_t* list) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int k = lane; k <= K; k += 32) cnt[k] = 0;
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const unsigned m = __match_any_sync(0xffffffffu, key[h]);
        if (key[h] < K && (m & lt) == 0) cnt[key[h]] += __popc(m);
        __syncwarp();
    }
    int carry = 0;
    for (int k0 = 0; k0 <= K; k0 += 32) {
        const int k = k0 + lane;
        const int v = k < K ? cnt[k] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (k <= K) start[k] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    for (int k = lane; k < K; k += 32) cnt[k] = start[k];   // running positions
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const unsigned m = __match_any_sync(0xffffffffu, key[h]);
        if (key[h] < K) list[cnt[key[h]] + __popc(m & lt)] = (uint8_t)(lane + 32 * h);
        __syncwarp();
        if (key[h] < K && (m & lt) == 0) cnt[key[h]] += __popc(m);
        __syncwarp();
    }
}

template <int C, int NQ>
__global__ void __launch_bounds__(256) k_bw_block_sums(const BackwardArgs P, float* slots) {
    constexpr int CG = C == 3 ? 4 : C;           // gradient row padded to 16 bytes for C = 3
    constexpr int KM = 32 * NQ;                   // buckets covered by the warp's lanes
    __shared__ float s_w[8][kBsChunk];
    __shared__ __align__(16) float s_g[8][kBsChunk * CG];
    __shared__ float s_t[8][KM * C];              // the block's window of T (grad_w)
    __shared__ int s_cnt[8][KM + 1];
    __shared__ int s_sa[8][KM + 1], s_sb[8][KM + 1];
    __shared__ uint8_t s_la[8][kBsChunk], s_lb[8][kBsChunk];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = (P.S - 1) >> 1, S = P.S, K = S * S, s = P.s;
    const float invK = 1.0f / (float)K, invS = 1.0f / (float)S;
    const int64_t nblocks = (int64_t)P.h * P.w;
    for (int64_t blk = (int64_t)blockIdx.x * 8 + warp; blk < nblocks;
         blk += (int64_t)gridDim.x * 8) {
        const int bv = (int)(blk / P.w), bu = (int)(blk - (int64_t)bv * P.w);
        if (P.gw) {
            // window cells inside the image (codes never select the others)
            for (int k = lane; k < K; k += 32) {
                const int kr = qdiv(k, invS);
                const int v = min(max(bv + kr - r, 0), P.h - 1);
                const int u = min(max(bu + (k - kr * S) - r, 0), P.w - 1);
#pragma unroll
                for (int c = 0; c < C; ++c)
                    s_t[warp][k * C + c] = __ldg(&P.T[(int64_t)v * P.T_pitch + (int64_t)u * C + c]);
            }
            __syncwarp();
        }
        float acc_a[NQ][C], acc_b[NQ][C];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int c = 0; c < C; ++c) acc_a[q][c] = acc_b[q][c] = 0.f;
        const int ys = bv * s, xs = bu * s;
        const int ey = min(s, P.H - ys), ex = min(s, P.W - xs), n = ey * ex;
        const float inv_ex = 1.0f / (float)ex;
        for (int j0 = 0; j0 < n; j0 += kBsChunk) {
            int ka[2], kb[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jj = lane + 32 * h, j = j0 + jj;
                ka[h] = kb[h] = 255;
                if (j >= n) continue;
                const int jy = qdiv(j, inv_ex);
                const int y = ys + jy, x = xs + (j - jy * ex);
                const int64_t p = (int64_t)y * P.W + x;
                const int code = P.code[p];
                const float w = load_weight(P.weight, P.wfmt, p);
                const int64_t og = (int64_t)y * P.G_pitch + (int64_t)x * C;
                float g[C];
#pragma unroll
                for (int c = 0; c < C; ++c) g[c] = __ldcs(&P.G[og + c]);
                const bool valid = code < K * K;
                const int qa = qdiv(code, invK), qb = code - qa * K;
                if (valid) {
                    ka[h] = qa;
                    kb[h] = qb;
                }
                s_w[warp][jj] = w;
                if (C == 3) {
                    *(float4*)&s_g[warp][jj * CG] = make_float4(g[0], g[1], g[C - 1], 0.f);
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c) s_g[warp][jj * CG + c] = g[c];
                }
                if (P.gw) {
                    float gw = 0.f;
                    if (valid) {
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            gw = __fmaf_rn(g[c], s_t[warp][qa * C + c] - s_t[warp][qb * C + c], gw);
                    } else {
                        set_status(GLU_ERR_DEVICE_CHECK);
                    }
                    P.gw[p] = gw;
                }
            }
            chunk_sort(ka, K, s_cnt[warp], s_sa[warp], s_la[warp]);
            chunk_sort(kb, K, s_cnt[warp], s_sb[warp], s_lb[warp]);
            // lane k walks bucket k of each list: the chunk's pixels with that window index,
            // in raster order
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int kk = lane + 32 * q;
                if (kk >= K) continue;
                for (int e = s_sa[warp][kk]; e < s_sa[warp][kk + 1]; ++e) {
                    const int jj = s_la[warp][e];
                    const float w = s_w[warp][jj];
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        acc_a[q][c] = __fmaf_rn(w, s_g[warp][jj * CG + c], acc_a[q][c]);
                }
                for (int e = s_sb[warp][kk]; e < s_sb[warp][kk + 1]; ++e) {
                    const int jj = s_lb[warp][e];
                    const float w = 1.f - s_w[warp][jj];
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        acc_b[q][c] = __fmaf_rn(w, s_g[warp][jj * CG + c], acc_b[q][c]);
                }
            }
            __syncwarp();
        }
        // bucket k feeds q = B + (k / S - r, k % S - r) as its neighbour K - 1 - k
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int kk = lane + 32 * q;
            if (kk >= K) continue;
            const int kr = qdiv(kk, invS);
            const int qv = bv + kr - r, qu = bu + (kk - kr * S) - r;
            if (qv < 0 || qv >= P.h || qu < 0 || qu >= P.w) continue;
            float* o = slots + (((int64_t)qv * P.w + qu) * K + (K - 1 - kk)) * 2 * C;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                o[c] = acc_a[q][c];
                o[C + c] = acc_b[q][c];
            }
        }
    }
}

// The slots of 32 consecutive LR pixels are one contiguous run of 32 K 2C floats: the CTA copies
// it into shared memory with 16-byte coalesced loads, then thread i adds pixel i's slots in order.
constexpr int kGatherQ = 32;
template <int C>
__global__ void __launch_bounds__(128) k_bw_gather(const BackwardArgs P, const float* slots) {
    extern __shared__ float4 gsm4[];
    float* gsm = (float*)gsm4;
    const int r = (P.S - 1) >> 1, S = P.S, K = S * S;
    const float invS = 1.0f / (float)S;
    const int per_q = K * 2 * C;                        // floats of one LR pixel's slots
    const int64_t nq = (int64_t)P.h * P.w;
    for (int64_t q0 = (int64_t)blockIdx.x * kGatherQ; q0 < nq;
         q0 += (int64_t)gridDim.x * kGatherQ) {
        const int nqc = (int)min((int64_t)kGatherQ, nq - q0);
        const int nf = nqc * per_q;                     // a multiple of 2; of 4 when nqc = 32
        const float* src = slots + q0 * per_q;          // 16-byte aligned when q0 % 32 == 0
        __syncthreads();                                // the previous chunk's readers are done
        if (nqc == kGatherQ) {
            const float4* s4 = (const float4*)src;
            for (int i = threadIdx.x; i < nf / 4; i += blockDim.x) gsm4[i] = __ldcs(&s4[i]);
        } else {
            for (int i = threadIdx.x; i < nf; i += blockDim.x) gsm[i] = __ldcs(&src[i]);
        }
        __syncthreads();
        if (threadIdx.x < nqc) {
            const int64_t q = q0 + threadIdx.x;
            const int v = (int)(q / P.w), u = (int)(q - (int64_t)v * P.w);
            const float* sl = gsm + threadIdx.x * per_q;
            float acc[C];
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = 0.f;
            for (int n = 0; n < K; ++n) {
                // neighbour n is block q + (n / S - r, n % S - r); outside the image: no slot
                const int nr = qdiv(n, invS);
                const int bv = v + nr - r, bu = u + (n - nr * S) - r;
                if (bv < 0 || bv >= P.h || bu < 0 || bu >= P.w) continue;
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] += sl[n * 2 * C + c];
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] += sl[n * 2 * C + C + c];
            }
#pragma unroll
            for (int c = 0; c < C; ++c) P.gT[(int64_t)v * P.gT_pitch + (int64_t)u * C + c] = acc[c];
        }
    }
}

size_t apply_backward_workspace_bytes(int h, int w, int S, int C) {
    return (size_t)h * w * (size_t)S * S * 2 * (size_t)C * sizeof(float);
}

template <int C>
static int launch_bw_ws_t(const BackwardArgs& a, float* slots, cudaStream_t st) {
    const int K = a.S * a.S;
    const int64_t nblocks = (int64_t)a.h * a.w;
    const int grid1 = grid_for(nblocks * 32, 256);
    if (K <= 32) k_bw_block_sums<C, 1><<<grid1, 256, 0, st>>>(a, slots);
    else if (K <= 64) k_bw_block_sums<C, 2><<<grid1, 256, 0, st>>>(a, slots);
    else k_bw_block_sums<C, 3><<<grid1, 256, 0, st>>>(a, slots);
    GLU_LAUNCH_CHECK();
    const size_t gsm = sizeof(float) * (size_t)kGatherQ * K * 2 * C;   // <= 83 KB (9x9, c = 4)
    if (gsm > 48 * 1024 &&
        cudaFuncSetAttribute(k_bw_gather<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gsm) != cudaSuccess)
        return GLU_ERR_CUDA;
    k_bw_gather<C><<<grid_for((nblocks + kGatherQ - 1) / kGatherQ * 128, 128), 128, gsm, st>>>(
        a, slots);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

int launch_apply_backward_ws(const BackwardArgs& a, void* ws, cudaStream_t st) {
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    float* slots = (float*)ws;
    switch (a.C) {
        case 1: return launch_bw_ws_t<1>(a, slots, st);
        case 2: return launch_bw_ws_t<2>(a, slots, st);
        case 3: return launch_bw_ws_t<3>(a, slots, st);
        case 4: return launch_bw_ws_t<4>(a, slots, st);
        default: return GLU_ERR_UNSUPPORTED;
    }
}

// grad_w_p = G_p . (T_a - T_b) for every HR pixel (the tiled kernel where the layout allows).
template <int C>
static int launch_gw(const BackwardArgs& a, cudaStream_t st) {
    const int threads = 256;
    {
        const bool tiled = C == 3 && a.W % 4 == 0 && a.G_pitch == (int64_t)a.W * 3 &&
                           ((uintptr_t)a.G & 15u) == 0 && ((uintptr_t)a.gw & 15u) == 0 &&
                           ((uintptr_t)a.code & 7u) == 0;
        if (tiled) {
            constexpr int TH = 16;
            const size_t sm = sizeof(float4) * (size_t)apply_region_cells(TH, a.s, a.S) +
                              sizeof(uint32_t) * (size_t)(a.S * a.S) * (a.S * a.S);
            if (sm > 48 * 1024 &&
                cudaFuncSetAttribute(k_apply3_gw_tile<TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm) != cudaSuccess)
                return GLU_ERR_CUDA;
            const dim3 grid((a.W + kApplyTW - 1) / kApplyTW, (a.H + TH - 1) / TH);
            k_apply3_gw_tile<TH><<<grid, 32 * 8, sm, st>>>(a);
        } else {
            k_apply_backward_w<C><<<grid_for((int64_t)a.H * a.W, threads), threads, 0, st>>>(a);
        }
        GLU_LAUNCH_CHECK();
    }
    return GLU_OK;
}

template <int C>
static int launch_bw_t(const BackwardArgs& a, cudaStream_t st) {
    const int threads = 256;
    // the largest LR tile whose HR region's codes fit the shared-memory budget
    const int r = (a.S - 1) / 2;
    int T = 0;
    size_t smem = 0;
    for (int t : {8, 4, 2, 1}) {
        const size_t side = (size_t)(t + 2 * r) * a.s;
        const size_t bytes = side * side * (sizeof(float) * (C + 1) + sizeof(uint16_t));
        if (bytes <= 110 * 1024 && a.s <= 64) {
            T = t;
            smem = bytes;
            break;
        }
    }
    if (T > 0) {
        auto kern = k_apply_backward_lr_tile<C>;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
            return GLU_ERR_CUDA;
        const dim3 grid((a.w + T - 1) / T, (a.h + T - 1) / T);
        kern<<<grid, threads, smem, st>>>(a, T);
    } else {
        const int grid_q = grid_for((int64_t)a.h * a.w * 32, threads);
        k_apply_backward_lr<C><<<grid_q, threads, 0, st>>>(a);
    }
    GLU_LAUNCH_CHECK();
    if (a.gw) return launch_gw<C>(a, st);
    return GLU_OK;
}

// ------------------------------------------------------- adjoint with a precomputed plan
//
// For a Theta used by many adjoint calls (an LR operator fitted through the upsampler), the
// inverse pixel-to-LR map is built once: for every LR pixel q, the list of its contributions
// (HR pixel p, side a or b) in a fixed order: neighbour blocks B = q + (n / S - r, n % S - r) for
// n = 0 .. K - 1, inside B first the pixels with a_p = q then those with b_p = q, each in raster
// order. Layout (int32): off[nq + 1], the entries p << 1 | side (2 per HR pixel at most), and
// the per-(q, n, side) counts / starts used while building. A call then reads each LR pixel's
// list once: a warp per LR pixel, lanes strided over the entries, a fixed butterfly.
size_t apply_backward_plan_bytes(int64_t np, int64_t nq, int S) {
    return sizeof(int) * (size_t)((nq + 1) + 2 * np + nq * (int64_t)S * S * 2);
}

struct PlanArgs {
    const uint16_t* code;
    int H, W, h, w, s, S;
    int* off;    // nq + 1
    int* ent;    // 2 np
    int* cnt;    // nq K 2: counts, then starts
};

// Counts (pass 0) or entries (pass 1) of one block per warp; chunk ranks by warp match, so the
// entries of one (q, n, side) are in raster order.
template <int PASS, int NQ>
__global__ void __launch_bounds__(256) k_plan_block(const PlanArgs A) {
    __shared__ int s_run[8][2][32 * NQ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int r = (A.S - 1) >> 1, S = A.S, K = S * S, s = A.s;
    const float invK = 1.0f / (float)K, invS = 1.0f / (float)S;
    const int64_t nblocks = (int64_t)A.h * A.w;
    for (int64_t blk = (int64_t)blockIdx.x * 8 + warp; blk < nblocks;
         blk += (int64_t)gridDim.x * 8) {
        const int bv = (int)(blk / A.w), bu = (int)(blk - (int64_t)bv * A.w);
        for (int k = lane; k < 32 * NQ; k += 32) s_run[warp][0][k] = s_run[warp][1][k] = 0;
        __syncwarp();
        const int ys = bv * s, xs = bu * s;
        const int ey = min(s, A.H - ys), ex = min(s, A.W - xs), n = ey * ex;
        const float inv_ex = 1.0f / (float)ex;
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            int key[2] = {255, 255};
            int64_t p = 0;
            if (j < n) {
                const int jy = qdiv(j, inv_ex);
                p = (int64_t)(ys + jy) * A.W + xs + (j - jy * ex);
                const int code = A.code[p];
                if (code < K * K) {
                    key[0] = qdiv(code, invK);
                    key[1] = code - key[0] * K;
                } else {
                    set_status(GLU_ERR_DEVICE_CHECK);
                }
            }
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int k = key[side];
                const unsigned m = __match_any_sync(0xffffffffu, k);
                if (PASS == 1 && k < K) {
                    const int kr = qdiv(k, invS);
                    const int qv = bv + kr - r, qu = bu + (k - kr * S) - r;
                    if (qv < 0 || qv >= A.h || qu < 0 || qu >= A.w) {
                        set_status(GLU_ERR_DEVICE_CHECK);   // not a code the search produces
                    } else {
                        const int64_t q = (int64_t)qv * A.w + qu;
                        const int pos = A.cnt[(q * K + (K - 1 - k)) * 2 + side] +
                                        s_run[warp][side][k] + __popc(m & lt);
                        A.ent[pos] = (int)((p << 1) | side);
                    }
                }
                __syncwarp();
                if (k < K && (m & lt) == 0) s_run[warp][side][k] += __popc(m);
                __syncwarp();
            }
        }
        if (PASS == 0) {
            for (int k = lane; k < K; k += 32) {
                const int kr = qdiv(k, invS);
                const int qv = bv + kr - r, qu = bu + (k - kr * S) - r;
                if (qv < 0 || qv >= A.h || qu < 0 || qu >= A.w) continue;
                const int64_t q = (int64_t)qv * A.w + qu;
                A.cnt[(q * K + (K - 1 - k)) * 2 + 0] = s_run[warp][0][k];
                A.cnt[(q * K + (K - 1 - k)) * 2 + 1] = s_run[warp][1][k];
            }
        }
        __syncwarp();
    }
}

// Per LR pixel: its total (neighbours inside the image) -> off[q] (before the scan).
__global__ void k_plan_totals(const PlanArgs A) {
    const int r = (A.S - 1) >> 1, S = A.S, K = S * S;
    const float invS = 1.0f / (float)S;
    const int64_t nq = (int64_t)A.h * A.w;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(q / A.w), u = (int)(q - (int64_t)v * A.w);
        int t = 0;
        for (int nn = 0; nn < K; ++nn) {
            const int nr = qdiv(nn, invS);
            const int bv = v + nr - r, bu = u + (nn - nr * S) - r;
            if (bv < 0 || bv >= A.h || bu < 0 || bu >= A.w) continue;
            t += A.cnt[(q * K + nn) * 2] + A.cnt[(q * K + nn) * 2 + 1];
        }
        A.off[q] = t;
    }
}

// Exclusive scan of off[0 .. nq) in place (off[nq] = total): one CTA, 1024 threads, in order.
__global__ void __launch_bounds__(1024) k_plan_scan(int* off, int64_t nq) {
    __shared__ int wsum[32];
    __shared__ int carry_s;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nq; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        const int v = i < nq ? off[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int t = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        const int excl = carry_s + (wid > 0 ? wsum[wid - 1] : 0) + x - v;
        if (i < nq) off[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry_s += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[nq] = carry_s;
}

// counts -> starts: off[q] + the counts of the earlier (n, side) of q (n ascending, a then b).
__global__ void k_plan_starts(const PlanArgs A) {
    const int r = (A.S - 1) >> 1, S = A.S, K = S * S;
    const float invS = 1.0f / (float)S;
    const int64_t nq = (int64_t)A.h * A.w;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(q / A.w), u = (int)(q - (int64_t)v * A.w);
        int pos = A.off[q];
        for (int nn = 0; nn < K; ++nn) {
            const int nr = qdiv(nn, invS);
            const int bv = v + nr - r, bu = u + (nn - nr * S) - r;
            if (bv < 0 || bv >= A.h || bu < 0 || bu >= A.w) continue;
            const int ca = A.cnt[(q * K + nn) * 2], cb = A.cnt[(q * K + nn) * 2 + 1];
            A.cnt[(q * K + nn) * 2] = pos;
            A.cnt[(q * K + nn) * 2 + 1] = pos + ca;
            pos += ca + cb;
        }
    }
}

int apply_backward_plan(const uint16_t* code, int H, int W, int s, int S, void* plan,
                        cudaStream_t st) {
    PlanArgs A;
    A.code = code;
    A.H = H;
    A.W = W;
    A.s = s;
    A.S = S;
    A.h = (H + s - 1) / s;
    A.w = (W + s - 1) / s;
    const int64_t np = (int64_t)H * W, nq = (int64_t)A.h * A.w;
    A.off = (int*)plan;
    A.ent = A.off + (nq + 1);
    A.cnt = A.ent + 2 * np;
    const int K = S * S;
    const int g = grid_for(nq * 32, 256);
    auto both = [&](auto k0, auto k1) {
        k0<<<g, 256, 0, st>>>(A);
        k_plan_totals<<<grid_for(nq, 256), 256, 0, st>>>(A);
        k_plan_scan<<<1, 1024, 0, st>>>(A.off, nq);
        k_plan_starts<<<grid_for(nq, 256), 256, 0, st>>>(A);
        k1<<<g, 256, 0, st>>>(A);
    };
    if (K <= 32) both(k_plan_block<0, 1>, k_plan_block<1, 1>);
    else if (K <= 64) both(k_plan_block<0, 2>, k_plan_block<1, 2>);
    else both(k_plan_block<0, 3>, k_plan_block<1, 3>);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

// A warp per LR pixel over its plan entries (lane-strided), then a fixed butterfly.
template <int C>
__global__ void __launch_bounds__(256) k_bw_planned(const BackwardArgs P, const int* off,
                                                   const int* ent, int dense) {
    const int lane = threadIdx.x & 31;
    const int64_t nq = (int64_t)P.h * P.w;
    for (int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); q < nq;
         q += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int e0 = off[q], e1 = off[q + 1];
        float acc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = 0.f;
        // four entries per lane at a time: their loads are issued together (the sums still
        // run over the lane's entries in ascending order)
        for (int e = e0 + lane; e < e1; e += 128) {
            int x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = e + 32 * u < e1 ? __ldcs(&ent[e + 32 * u]) : -1;
            float f[4], g[4][C];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                f[u] = 0.f;
#pragma unroll
                for (int c = 0; c < C; ++c) g[u][c] = 0.f;
                if (x[u] < 0) continue;
                const int64_t p = (int64_t)(x[u] >> 1);
                const float w = load_weight(P.weight, P.wfmt, p);
                f[u] = (x[u] & 1) ? 1.f - w : w;
                const int64_t og = dense ? p * C : (p / P.W) * P.G_pitch + (p % P.W) * C;
#pragma unroll
                for (int c = 0; c < C; ++c) g[u][c] = __ldg(&P.G[og + c]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (x[u] < 0) break;
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] = __fmaf_rn(f[u], g[u][c], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        }
        if (lane == 0) {
            const int v = (int)(q / P.w), u = (int)(q - (int64_t)v * P.w);
#pragma unroll
            for (int c = 0; c < C; ++c) P.gT[(int64_t)v * P.gT_pitch + (int64_t)u * C + c] = acc[c];
        }
    }
}

template <int C>
static int launch_bw_planned_t(const BackwardArgs& a, const void* plan, cudaStream_t st) {
    const int64_t nq = (int64_t)a.h * a.w;
    const int* off = (const int*)plan;
    const int* ent = off + (nq + 1);
    k_bw_planned<C><<<grid_for(nq * 32, 256), 256, 0, st>>>(a, off, ent,
                                                            a.G_pitch == (int64_t)a.W * C);
    GLU_LAUNCH_CHECK();
    if (a.gw) return launch_gw<C>(a, st);
    return GLU_OK;
}

int launch_apply_backward_planned(const BackwardArgs& a, const void* plan, cudaStream_t st) {
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    switch (a.C) {
        case 1: return launch_bw_planned_t<1>(a, plan, st);
        case 2: return launch_bw_planned_t<2>(a, plan, st);
        case 3: return launch_bw_planned_t<3>(a, plan, st);
        case 4: return launch_bw_planned_t<4>(a, plan, st);
        default: return GLU_ERR_UNSUPPORTED;
    }
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
