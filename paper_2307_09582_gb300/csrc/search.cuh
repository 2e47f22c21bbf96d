// Per-pixel candidate search of Algorithm 1 (Sec. 3.2), shared by the full-image search kernel
// and the joint-optimisation trials so both compute bit-identical Theta and error values.
//
// Colours are floats in 1/255 units. For uint8 inputs every distance ||I_p - L_c||^2 is an
// integer below 2^24 and is computed exactly, so the nearest-colour choice of a is exact.
#pragma once

#include "common.cuh"

namespace glu {

struct SearchOut {
    int ka, kb;     // window indices
    float omega;    // Eq. 5 weight
    float err;      // Eq. 3 error ||I_p - I_hat_p|| in [0, 1] units
};

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Window colour k from shared memory. An explicit shared load per use keeps the compiler from
// holding the whole window in registers across both candidate loops (it is a broadcast read).
__device__ __forceinline__ float4 lds_f4(const float4* p) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
    return v;
}

// Squared colour distance with a fixed operation order (so a = b evaluates identically in both
// steps and uint8 inputs stay exact).
__device__ __forceinline__ float dist2(float er, float eg, float eb) {
    return __fmaf_rn(eb, eb, __fmaf_rn(eg, eg, __fmul_rn(er, er)));
}

// win: window candidate (dy, dx) at win[dy * rs + dx] (float4: r, g, b, unused), in shared
// memory. rowmask / colmask: bit i set when window row / column i lies inside the LR image
// (ignored when kInterior: the caller guarantees the whole window is inside).
// eps255 must be > 0 (the library clamps eps = 0 to a negligible positive value), so the
// Eq. 5 denominator never vanishes.
// Ties: a -> lowest k; b -> lowest k_b (strict comparisons in ascending k).
// kCompact: keep the window rows rolled (fewer registers, more resident warps). Every variant
// computes bit-identical results: the same operations on the same values.
template <int S, bool kCompact = false, bool kInterior = false>
__device__ __forceinline__ SearchOut search_pixel(const float4* __restrict__ win, int rs,
                                                  uint32_t rowmask, uint32_t colmask, float ir,
                                                  float ig, float ib, float eps255, bool gnu) {
    constexpr int K = S * S;
    constexpr int kRowUnroll = (kCompact || S > 5) ? 1 : S;
    constexpr bool kKeep = !kCompact && S <= 3;   // keep step 1's distances for step 2
    float d2s[kKeep ? K : 1];
    // Step 1: a = the window pixel with the most similar colour (squared distance, exact).
    float bd = kInf;
    int a = 0;
#pragma unroll(kRowUnroll)
    for (int dy = 0; dy < S; ++dy) {
#pragma unroll
        for (int dx = 0; dx < S; ++dx) {
            const bool ok = kInterior || ((rowmask >> dy) & (colmask >> dx) & 1u) != 0u;
            const float4 c = lds_f4(&win[dy * rs + dx]);
            const float d2 = dist2(c.x - ir, c.y - ig, c.z - ib);
            if constexpr (kKeep) d2s[dy * S + dx] = d2;
            if (ok && d2 < bd) {
                bd = d2;
                a = dy * S + dx;
            }
        }
    }
    const float4 ca = lds_f4(&win[(a / S) * rs + (a % S)]);
    const float ur = ca.x - ir, ug = ca.y - ig, ub = ca.z - ib;
    const float da = sqrt_approx(bd);
    SearchOut o;
    o.ka = a;
    if (gnu) {  // weight fixed to 1: T_hat = T_a
        o.kb = a;
        o.omega = 1.0f;
        o.err = da * (1.0f / 255.0f);
        return o;
    }
    // Step 2: fix a; for every b (b = a included) the Eq. 5 weight w = d_b / (d_a + d_b + eps)
    // and the Eq. 3 residual r = w u + (1 - w) v with u = L_a - I, v = L_b - I. The comparison
    // uses D * r = d_b u + (d_a + eps) v and D = d_a + d_b + eps: err^2 = |D r|^2 / D^2,
    // compared by cross-multiplication so no candidate needs a division.
    const float dae = da + eps255;
    float bnum = kInf, bden = 1.0f;
    int b = a;
#pragma unroll(kRowUnroll)
    for (int dy = 0; dy < S; ++dy) {
#pragma unroll
        for (int dx = 0; dx < S; ++dx) {
            const bool ok = kInterior || ((rowmask >> dy) & (colmask >> dx) & 1u) != 0u;
            const float4 c = lds_f4(&win[dy * rs + dx]);
            const float vr = c.x - ir, vg = c.y - ig, vb = c.z - ib;
            float d2b;
            if constexpr (kKeep) d2b = d2s[dy * S + dx];
            else d2b = dist2(vr, vg, vb);
            const float db = sqrt_approx(d2b);
            const float xr = __fmaf_rn(db, ur, __fmul_rn(dae, vr));
            const float xg = __fmaf_rn(db, ug, __fmul_rn(dae, vg));
            const float xb = __fmaf_rn(db, ub, __fmul_rn(dae, vb));
            const float num = dist2(xr, xg, xb);
            const float D = __fadd_rn(db, dae);
            const float den = __fmul_rn(D, D);
            if (ok && __fmul_rn(num, bden) < __fmul_rn(bnum, den)) {
                bnum = num;
                bden = den;
                b = dy * S + dx;
            }
        }
    }
    o.kb = b;
    // the winner's d_b again (same operations on the same values as in the loop)
    const float4 cb = lds_f4(&win[(b / S) * rs + (b % S)]);
    const float bdb = sqrt_approx(dist2(cb.x - ir, cb.y - ig, cb.z - ib));
    const float wden = bdb + dae;
    o.omega = __fdividef(bdb, wden);
    o.err = sqrt_approx(__fdividef(bnum, bden)) * (1.0f / 255.0f);
    return o;
}

// Row/column validity masks of the window centred on LR block (py, px) of an h x w LR image.
__device__ __forceinline__ void window_masks(int py, int px, int h, int w, int S,
                                             uint32_t& rowmask, uint32_t& colmask) {
    const int r = (S - 1) >> 1;
    rowmask = 0u;
    colmask = 0u;
    for (int i = 0; i < S; ++i) {
        const int v = py - r + i, u = px - r + i;
        rowmask |= (uint32_t)(v >= 0 && v < h) << i;
        colmask |= (uint32_t)(u >= 0 && u < w) << i;
    }
}

}  // namespace glu
