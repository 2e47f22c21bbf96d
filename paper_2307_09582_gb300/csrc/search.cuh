// Per-pixel candidate search of Algorithm 1 (Sec. 3.2), shared by the full-image search kernel
// and the joint-optimisation trials so both compute bit-identical Theta and error values. The
// pieces (step 2 for a given a, the candidate key, the chosen pair's weight and error) are also
// used by the trials' exact re-search after a few window colours change.
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

// Step-2 key of candidate b for a fixed a: the squared Eq. 3 error in 1/255 units. With the Eq. 5
// weight w = d_b / (d_a + d_b + eps) and u = L_a - I, v = L_b - I, the residual is
// r = w u + (1 - w) v = (d_b u + (d_a + eps) v) / D with D = d_a + d_b + eps. v is formed
// exactly for uint8 colours, so an exactly representable pixel (I = L_a = L_b) gets error 0.
// One float per candidate, compared exactly, so the candidate order is a total order (ties:
// lowest k) and a re-search after some candidates change can be done exactly from the previous
// winner.
struct StepB {
    float ur, ug, ub;   // u = L_a - I
    float dae;          // d_a + eps
};

__device__ __forceinline__ StepB step_b_setup(float4 ca, float d2a, float ir, float ig, float ib,
                                              float eps255) {
    StepB t;
    t.ur = ca.x - ir;
    t.ug = ca.y - ig;
    t.ub = ca.z - ib;
    t.dae = sqrt_approx(d2a) + eps255;
    return t;
}

// d2b = ||L_b - I||^2 (as dist2 computes it), (vr, vg, vb) = L_b - I.
__device__ __forceinline__ float b_key(const StepB& t, float d2b, float vr, float vg, float vb) {
    const float db = sqrt_approx(d2b);
    const float xr = __fmaf_rn(db, t.ur, __fmul_rn(t.dae, vr));
    const float xg = __fmaf_rn(db, t.ug, __fmul_rn(t.dae, vg));
    const float xb = __fmaf_rn(db, t.ub, __fmul_rn(t.dae, vb));
    const float num = dist2(xr, xg, xb);
    const float D = __fadd_rn(db, t.dae);
    return __fdividef(num, __fmul_rn(D, D));
}

// Weight and error of the chosen pair (the same operations wherever a pair is chosen).
__device__ __forceinline__ void finish_pair(const float4* win, int rs, int S, int b, float ir,
                                            float ig, float ib, float dae, float bkey,
                                            SearchOut& o) {
    const float4 cb = lds_f4(&win[(b / S) * rs + (b % S)]);
    const float bdb = sqrt_approx(dist2(cb.x - ir, cb.y - ig, cb.z - ib));
    o.kb = b;
    o.omega = __fdividef(bdb, bdb + dae);
    o.err = sqrt_approx(bkey) * (1.0f / 255.0f);
}

// Step 2 of Algorithm 1 for a fixed a (window index) at squared distance d2a: b over the whole
// window (b = a included) minimising the key, ties to the lowest k.
template <int S, bool kCompact, bool kInterior>
__device__ __forceinline__ SearchOut step_b(const float4* __restrict__ win, int rs,
                                            uint32_t rowmask, uint32_t colmask, int a, float d2a,
                                            float ir, float ig, float ib, float eps255) {
    constexpr int kRowUnroll = (kCompact || S > 5) ? 1 : S;
    const StepB t = step_b_setup(lds_f4(&win[(a / S) * rs + (a % S)]), d2a, ir, ig, ib, eps255);
    float bkey = kInf;
    int b = a;
#pragma unroll(kRowUnroll)
    for (int dy = 0; dy < S; ++dy) {
#pragma unroll
        for (int dx = 0; dx < S; ++dx) {
            const bool ok = kInterior || ((rowmask >> dy) & (colmask >> dx) & 1u) != 0u;
            const float4 c = lds_f4(&win[dy * rs + dx]);
            const float vr = c.x - ir, vg = c.y - ig, vb = c.z - ib;
            const float key = b_key(t, dist2(vr, vg, vb), vr, vg, vb);
            if (ok && key < bkey) {
                bkey = key;
                b = dy * S + dx;
            }
        }
    }
    SearchOut o;
    o.ka = a;
    finish_pair(win, rs, S, b, ir, ig, ib, t.dae, bkey, o);
    return o;
}

// Dot product with a fixed operation order.
__device__ __forceinline__ float dot3(float ar, float ag, float ab, float br, float bg, float bb) {
    return __fmaf_rn(ab, bb, __fmaf_rn(ag, bg, __fmul_rn(ar, br)));
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
    constexpr int kRowUnroll = (kCompact || S > 5) ? 1 : S;
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
            if (ok && d2 < bd) {
                bd = d2;
                a = dy * S + dx;
            }
        }
    }
    if (gnu) {  // weight fixed to 1: T_hat = T_a
        SearchOut o;
        o.ka = a;
        o.kb = a;
        o.omega = 1.0f;
        o.err = sqrt_approx(bd) * (1.0f / 255.0f);
        return o;
    }
    // Step 2: fix a; b over the window with the Eq. 5 weight and the Eq. 3 error
    return step_b<S, kCompact, kInterior>(win, rs, rowmask, colmask, a, bd, ir, ig, ib, eps255);
}

// ------------------------------------------------------------------ two pixels, packed FP32
//
// Two HR pixels of one LR block share the window, so every candidate is evaluated for both at
// once with the packed two-lane FP32 instructions (add / sub / mul / fma .rn.f32x2): each lane
// is an ordinary IEEE single-precision operation with round-to-nearest, so lane 0 computes
// exactly what the scalar search_pixel computes for pixel 0 and lane 1 for pixel 1, in the same
// order; the square roots and the divisions stay per lane (the same calls as above), and the
// comparisons and tie-breaks are per pixel. The window is read from a second shared-memory copy
// that holds each colour channel twice, (r, r, g, g) and (b, b), so a candidate arrives as three
// packed operands.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// dist2 of both lanes (the same operation order as dist2)
__device__ __forceinline__ f32x2 dist2x2(f32x2 er, f32x2 eg, f32x2 eb) {
    return fma2(eb, eb, fma2(eg, eg, mul2(er, er)));
}

// The duplicated window copy: candidate k's (r, r, g, g) at rg[k] and (b, b) at bb[k].
__device__ __forceinline__ void lds_dup(const float4* rg, const float2* bb, f32x2& r2, f32x2& g2,
                                        f32x2& b2) {
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];"
                 : "=l"(r2), "=l"(g2)
                 : "r"((uint32_t)__cvta_generic_to_shared(rg)));
    asm volatile("ld.shared.b64 %0, [%1];"
                 : "=l"(b2)
                 : "r"((uint32_t)__cvta_generic_to_shared(bb)));
}

// Algorithm 1 for two pixels (colours (ir0, ig0, ib0) and (ir1, ig1, ib1)) with the same window.
// win: the float4 copy (used for the chosen pairs); cand(idx, r2, g2, b2) delivers window cell
// idx (= dy * rs + dx) as three packed (c, c) operands. Results equal search_pixel's for each
// pixel, bit for bit.
template <int S, bool kCompact, bool kInterior, typename Cand>
__device__ __forceinline__ void search_pair_impl(const float4* __restrict__ win, Cand cand,
                                                 int rs, uint32_t rowmask, uint32_t colmask,
                                                 float ir0, float ig0, float ib0, float ir1,
                                                 float ig1, float ib1, float eps255, bool gnu,
                                                 SearchOut& o0, SearchOut& o1) {
    constexpr int kRowUnroll = (kCompact || S > 5) ? 1 : S;
    const f32x2 ir = pack2(ir0, ir1), ig = pack2(ig0, ig1), ib = pack2(ib0, ib1);
    // step 1: the nearest colour of each pixel (exact for uint8 colours), ties to the lowest k
    float bd0 = kInf, bd1 = kInf;
    int a0 = 0, a1 = 0;
#pragma unroll(kRowUnroll)
    for (int dy = 0; dy < S; ++dy) {
#pragma unroll
        for (int dx = 0; dx < S; ++dx) {
            const bool ok = kInterior || ((rowmask >> dy) & (colmask >> dx) & 1u) != 0u;
            f32x2 cr, cg, cb;
            cand(dy * rs + dx, cr, cg, cb);
            float d0, d1;
            unpack2(dist2x2(sub2(cr, ir), sub2(cg, ig), sub2(cb, ib)), d0, d1);
            const int k = dy * S + dx;
            if (ok && d0 < bd0) {
                bd0 = d0;
                a0 = k;
            }
            if (ok && d1 < bd1) {
                bd1 = d1;
                a1 = k;
            }
        }
    }
    if (gnu) {
        o0.ka = o0.kb = a0;
        o1.ka = o1.kb = a1;
        o0.omega = o1.omega = 1.0f;
        o0.err = sqrt_approx(bd0) * (1.0f / 255.0f);
        o1.err = sqrt_approx(bd1) * (1.0f / 255.0f);
        return;
    }
    // step 2: for each pixel's a, b over the window minimising the key, ties to the lowest k
    const float4 ca0 = lds_f4(&win[(a0 / S) * rs + (a0 % S)]);
    const float4 ca1 = lds_f4(&win[(a1 / S) * rs + (a1 % S)]);
    const f32x2 ur = sub2(pack2(ca0.x, ca1.x), ir);
    const f32x2 ug = sub2(pack2(ca0.y, ca1.y), ig);
    const f32x2 ub = sub2(pack2(ca0.z, ca1.z), ib);
    const float dae0 = sqrt_approx(bd0) + eps255, dae1 = sqrt_approx(bd1) + eps255;
    const f32x2 dae = pack2(dae0, dae1);
    float bkey0 = kInf, bkey1 = kInf;
    int b0 = a0, b1 = a1;
#pragma unroll(kRowUnroll)
    for (int dy = 0; dy < S; ++dy) {
#pragma unroll
        for (int dx = 0; dx < S; ++dx) {
            const bool ok = kInterior || ((rowmask >> dy) & (colmask >> dx) & 1u) != 0u;
            f32x2 cr, cg, cb;
            cand(dy * rs + dx, cr, cg, cb);
            const f32x2 vr = sub2(cr, ir), vg = sub2(cg, ig), vb = sub2(cb, ib);
            float q0, q1;
            unpack2(dist2x2(vr, vg, vb), q0, q1);
            const f32x2 db = pack2(sqrt_approx(q0), sqrt_approx(q1));
            const f32x2 xr = fma2(db, ur, mul2(dae, vr));
            const f32x2 xg = fma2(db, ug, mul2(dae, vg));
            const f32x2 xb = fma2(db, ub, mul2(dae, vb));
            const f32x2 D = add2(db, dae);
            float n0, n1, e0, e1;
            unpack2(dist2x2(xr, xg, xb), n0, n1);
            unpack2(mul2(D, D), e0, e1);
            const float key0 = __fdividef(n0, e0), key1 = __fdividef(n1, e1);
            const int k = dy * S + dx;
            if (ok && key0 < bkey0) {
                bkey0 = key0;
                b0 = k;
            }
            if (ok && key1 < bkey1) {
                bkey1 = key1;
                b1 = k;
            }
        }
    }
    o0.ka = a0;
    o1.ka = a1;
    finish_pair(win, rs, S, b0, ir0, ig0, ib0, dae0, bkey0, o0);
    finish_pair(win, rs, S, b1, ir1, ig1, ib1, dae1, bkey1, o1);
}

// With the duplicated window copy: rg / bb indexed like win.
template <int S, bool kCompact = false, bool kInterior = false>
__device__ __forceinline__ void search_pair(const float4* __restrict__ win,
                                            const float4* __restrict__ rg,
                                            const float2* __restrict__ bb, int rs,
                                            uint32_t rowmask, uint32_t colmask, float ir0,
                                            float ig0, float ib0, float ir1, float ig1,
                                            float ib1, float eps255, bool gnu, SearchOut& o0,
                                            SearchOut& o1) {
    auto cand = [&](int idx, f32x2& r2, f32x2& g2, f32x2& b2) {
        lds_dup(&rg[idx], &bb[idx], r2, g2, b2);
    };
    search_pair_impl<S, kCompact, kInterior>(win, cand, rs, rowmask, colmask, ir0, ig0, ib0, ir1,
                                             ig1, ib1, eps255, gnu, o0, o1);
}

// With the float4 window only: each candidate's channels are broadcast into packed pairs.
template <int S>
__device__ __forceinline__ void search_pair_f4(const float4* __restrict__ win, int rs,
                                               uint32_t rowmask, uint32_t colmask, float ir0,
                                               float ig0, float ib0, float ir1, float ig1,
                                               float ib1, float eps255, SearchOut& o0,
                                               SearchOut& o1) {
    auto cand = [&](int idx, f32x2& r2, f32x2& g2, f32x2& b2) {
        const float4 c = lds_f4(&win[idx]);
        r2 = pack2(c.x, c.x);
        g2 = pack2(c.y, c.y);
        b2 = pack2(c.z, c.z);
    };
    search_pair_impl<S, true, false>(win, cand, rs, rowmask, colmask, ir0, ig0, ib0, ir1, ig1,
                                     ib1, eps255, false, o0, o1);
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
