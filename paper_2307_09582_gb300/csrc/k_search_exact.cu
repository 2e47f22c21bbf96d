// GLU* (Sec. 3.1, Eq. 4): for every HR pixel, every unordered pair of window pixels
// k_a < k_b with the least-squares weight w = ((I - L_b) . (L_a - L_b)) / (|L_a - L_b|^2 + eps)
// (not clamped) and its Eq. 3 error; the pair with the smallest error wins (ties: the first pair
// in (k_a, k_b) order). A window with a single pixel inside the LR image gives a = b, w = 1.
//
// The pair count is quadratic in the window (S = 5: 300 pairs), so this is plain ALU work. HR
// pixels of one LR block share their window, so a thread owns PX x PY pixels of one block (PX, PY
// divide the scale) and computes each pair's difference d = L_a - L_b, |d|^2 + eps and its
// reciprocal once for all of them; per pixel and pair it forms v = L_b - I, w = -(v . d) / den,
// the residual w d + v and its squared norm (the comparison key, exact squared error in 1/255
// units). The valid window is a rectangle (the window clipped to the LR image), so the pair loops
// run over its bounds with no per-candidate masks. The LR halo of the CTA's 32 PX x 8 PY tile
// sits in shared memory in 1/255 units.
#include "common.cuh"
#include "internal.h"
#include "search.cuh"

namespace glu {

GLU_DEFINE_STATUS(search_exact)

constexpr int kExTX = 32, kExTY = 8;

// |d|^2 + eps for the pair (c_a, c_b) and its reciprocal; d = c_a - c_b.
struct ExPair {
    float dr, dg, db, d2, rden;
};
__device__ __forceinline__ ExPair ex_pair(const float4 ca, const float4 cb, float eps2) {
    ExPair p;
    p.dr = __fsub_rn(ca.x, cb.x);
    p.dg = __fsub_rn(ca.y, cb.y);
    p.db = __fsub_rn(ca.z, cb.z);
    p.d2 = dist2(p.dr, p.dg, p.db);
    p.rden = __fdividef(1.0f, __fadd_rn(p.d2, eps2));   // eps2 > 0: the host guarantees it
    return p;
}
// Weight and squared error of the pair for guide colour (ir, ig, ib).
__device__ __forceinline__ float ex_eval(const ExPair& p, const float4 cb, float ir, float ig,
                                         float ib, float& w) {
    const float vr = __fsub_rn(cb.x, ir), vg = __fsub_rn(cb.y, ig), vb = __fsub_rn(cb.z, ib);
    const float vd = __fmaf_rn(vb, p.db, __fmaf_rn(vg, p.dg, __fmul_rn(vr, p.dr)));
    w = __fmul_rn(-vd, p.rden);
    const float er = __fmaf_rn(w, p.dr, vr), eg = __fmaf_rn(w, p.dg, vg),
                eb = __fmaf_rn(w, p.db, vb);
    return dist2(er, eg, eb);
}

template <int S, typename HT, int PX, int PY>
__global__ void __launch_bounds__(kExTX * kExTY) k_search_exact(const SearchArgs a, float eps2,
                                                                int eps_zero) {
    constexpr int r = (S - 1) / 2, K = S * S, P = PX * PY;
    constexpr int TW = kExTX * PX, TH = kExTY * PY;
    extern __shared__ float4 region[];
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int s = a.s;
    const int xe = min(x0 + TW, a.W), ye = min(y0 + TH, a.H);
    const int v0 = y0 / s - r, u0 = x0 / s - r;
    const int RH = (ye - 1) / s + r - v0 + 1, RW = (xe - 1) / s + r - u0 + 1;
    for (int k = threadIdx.x; k < RH * RW; k += blockDim.x) {
        const int v = v0 + k / RW, u = u0 + k % RW;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v >= 0 && v < a.h && u >= 0 && u < a.w) {
            const int64_t o = (int64_t)v * a.lr_pitch + (int64_t)u * 3;
            if (a.lr_dtype == GLU_U8) {
                const uint8_t* L = (const uint8_t*)a.lr;
                c = make_float4((float)L[o], (float)L[o + 1], (float)L[o + 2], 0.f);
            } else if (a.lr_dtype == GLU_F16) {
                const __half* L = (const __half*)a.lr;
                c = make_float4(__half2float(L[o]) * 255.f, __half2float(L[o + 1]) * 255.f,
                                __half2float(L[o + 2]) * 255.f, 0.f);
            } else {
                const float* L = (const float*)a.lr;
                c = make_float4(L[o] * 255.f, L[o + 1] * 255.f, L[o + 2] * 255.f, 0.f);
            }
        }
        region[k] = c;
    }
    __syncthreads();
    // the thread's pixels: columns xb .. xb + PX - 1, rows yb .. yb + PY - 1, all in one LR block
    const int xb = x0 + (threadIdx.x % kExTX) * PX, yb = y0 + (threadIdx.x / kExTX) * PY;
    if (xb >= a.W || yb >= a.H) return;
    float ir[P], ig[P], ib[P], bkey[P];
    int bidx[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int x = min(xb + q % PX, a.W - 1), y = min(yb + q / PX, a.H - 1);
        const HT* hp = (const HT*)a.hr + (int64_t)y * a.hr_pitch + (int64_t)x * 3;
        ir[q] = Px<HT>::to255(hp[0]);
        ig[q] = Px<HT>::to255(hp[1]);
        ib[q] = Px<HT>::to255(hp[2]);
        bkey[q] = kInf;
        bidx[q] = -1;
    }
    const int py = yb / s, px = xb / s;
    const int ylo = max(0, r - py), yhi = min(S - 1, a.h - 1 - py + r);
    const int xlo = max(0, r - px), xhi = min(S - 1, a.w - 1 - px + r);
    const float4* win = &region[(py - r - v0) * RW + (px - r - u0)];
    auto pair = [&](const float4 ci, const float4 cj, int code) {
        const ExPair pr = ex_pair(ci, cj, eps2);
#pragma unroll
        for (int q = 0; q < P; ++q) {
            float w;
            const float key = ex_eval(pr, cj, ir[q], ig[q], ib[q], w);
            if (key < bkey[q]) {
                bkey[q] = key;
                bidx[q] = code;
            }
        }
    };
    for (int iy = ylo; iy <= yhi; ++iy)
        for (int ix = xlo; ix <= xhi; ++ix) {
            const float4 ci = lds_f4(&win[iy * RW + ix]);
            const int ci_code = (iy * S + ix) * K;
            for (int jx = ix + 1; jx <= xhi; ++jx)
                pair(ci, lds_f4(&win[iy * RW + jx]), ci_code + iy * S + jx);
            for (int jy = iy + 1; jy <= yhi; ++jy)
                for (int jx = xlo; jx <= xhi; ++jx)
                    pair(ci, lds_f4(&win[jy * RW + jx]), ci_code + jy * S + jx);
        }
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int x = xb + q % PX, y = yb + q / PX;
        if (x >= a.W || y >= a.H) continue;
        int ka, kb;
        float omega, e2;
        if (bidx[q] < 0) {   // a single valid window pixel
            ka = kb = ylo * S + xlo;
            const float4 c = lds_f4(&win[ylo * RW + xlo]);
            omega = 1.f;
            e2 = dist2(c.x - ir[q], c.y - ig[q], c.z - ib[q]);
        } else {
            ka = bidx[q] / K;
            kb = bidx[q] % K;
            const float4 ca = lds_f4(&win[(ka / S) * RW + ka % S]);
            const float4 cb = lds_f4(&win[(kb / S) * RW + kb % S]);
            const ExPair pr = ex_pair(ca, cb, eps2);
            e2 = ex_eval(pr, cb, ir[q], ig[q], ib[q], omega);
            if (pr.d2 == 0.f) omega = eps_zero ? 1.f : 0.f;   // L_a = L_b: Eq. 4 is 0 / eps
        }
        const int64_t p = (int64_t)y * a.W + x;
        a.code[p] = (uint16_t)(ka * K + kb);
        ((float*)a.weight)[p] = omega;
        if (a.err) a.err[p] = sqrt_approx(e2) * (1.0f / 255.0f);
    }
}

template <typename HT, int PX, int PY>
static int launch_exact_t(const SearchArgs& a, float eps2, int eps_zero, cudaStream_t st) {
    constexpr int TW = kExTX * PX, TH = kExTY * PY;
    const int r = (a.S - 1) / 2;
    const size_t smem = sizeof(float4) * (size_t)((TH - 1) / a.s + 2 + 2 * r) *
                        (size_t)((TW - 1) / a.s + 2 + 2 * r);
    const dim3 grid((a.W + TW - 1) / TW, (a.H + TH - 1) / TH);
    auto run = [&](auto kern) -> int {
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
            return GLU_ERR_CUDA;
        kern<<<grid, kExTX * kExTY, smem, st>>>(a, eps2, eps_zero);
        GLU_LAUNCH_CHECK();
        return GLU_OK;
    };
    switch (a.S) {
        case 1: return run(k_search_exact<1, HT, PX, PY>);
        case 3: return run(k_search_exact<3, HT, PX, PY>);
        case 5: return run(k_search_exact<5, HT, PX, PY>);
        case 7: return run(k_search_exact<7, HT, PX, PY>);
        default: return run(k_search_exact<9, HT, PX, PY>);
    }
}

template <typename HT>
static int launch_exact_h(const SearchArgs& a, float eps2, int eps_zero, cudaStream_t st) {
    // pixels per thread must share an LR block: PX and PY divide the scale
    if (a.s % 4 == 0) return launch_exact_t<HT, 4, 2>(a, eps2, eps_zero, st);
    if (a.s % 2 == 0) return launch_exact_t<HT, 2, 2>(a, eps2, eps_zero, st);
    return launch_exact_t<HT, 1, 1>(a, eps2, eps_zero, st);
}

int launch_search_exact(const SearchArgs& a, cudaStream_t st) {
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    if (a.wfmt != GLU_W_F32) return GLU_ERR_UNSUPPORTED;   // Eq. 4 weights are not clamped
    // Eq. 4's eps adds to a squared colour distance: eps in [0, 1]^2 units is eps * 255^2 in
    // 1/255 units, i.e. eps255 * 255. The host clamps eps255 to >= 1e-12 (so the denominator is
    // never zero); at that floor eps was zero.
    const float eps2 = a.eps255 * 255.0f;
    const int eps_zero = a.eps255 <= 1e-12f;
    if (a.hr_dtype == GLU_U8) return launch_exact_h<uint8_t>(a, eps2, eps_zero, st);
    if (a.hr_dtype == GLU_F16) return launch_exact_h<__half>(a, eps2, eps_zero, st);
    return GLU_ERR_UNSUPPORTED;
}

}  // namespace glu
