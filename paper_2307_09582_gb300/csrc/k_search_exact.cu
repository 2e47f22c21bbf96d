// GLU* (Sec. 3.1, Eq. 4): for every HR pixel, every unordered pair of window pixels
// k_a < k_b with the least-squares weight w = ((I - L_b) . (L_a - L_b)) / (|L_a - L_b|^2 + eps)
// (not clamped) and its Eq. 3 error; the pair with the smallest error wins (ties: the first pair
// in (k_a, k_b) order). A window with a single pixel inside the LR image gives a = b, w = 1.
//
// The pair count is quadratic in the window (S = 5: 300 pairs), so this is plain ALU work: one
// thread per pixel, the LR halo of a 64 x 4 tile in shared memory in 1/255 units, and per pixel
// the candidates' offsets v_k = L_k - I; the pair key is the squared error, compared exactly.
#include "common.cuh"
#include "internal.h"
#include "search.cuh"

namespace glu {

GLU_DEFINE_STATUS(search_exact)

constexpr int kExW = 64, kExH = 4;

template <int S, typename HT>
__global__ void __launch_bounds__(kExW * kExH) k_search_exact(const SearchArgs a, float eps2) {
    constexpr int r = (S - 1) / 2, K = S * S;
    extern __shared__ float4 region[];
    const int x0 = blockIdx.x * kExW, y0 = blockIdx.y * kExH;
    const int s = a.s;
    const int xe = min(x0 + kExW, a.W), ye = min(y0 + kExH, a.H);
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
    const int x = x0 + threadIdx.x % kExW, y = y0 + threadIdx.x / kExW;
    if (x >= a.W || y >= a.H) return;
    const HT* hp = (const HT*)a.hr + (int64_t)y * a.hr_pitch + (int64_t)x * 3;
    const float ir = Px<HT>::to255(hp[0]), ig = Px<HT>::to255(hp[1]), ib = Px<HT>::to255(hp[2]);
    const int py = y / s, px = x / s;
    uint32_t rm, cm;
    window_masks(py, px, a.h, a.w, S, rm, cm);
    const float4* win = &region[(py - r - v0) * RW + (px - r - u0)];
    float bkey = kInf, bw = 1.f;
    int ba = -1, bb = -1, nvalid = 0, only = 0;
    for (int i = 0; i < K; ++i) {
        if (!((rm >> (i / S)) & (cm >> (i % S)) & 1u)) continue;
        ++nvalid;
        only = i;
        const float4 ci = lds_f4(&win[(i / S) * RW + (i % S)]);
        for (int j = i + 1; j < K; ++j) {
            if (!((rm >> (j / S)) & (cm >> (j % S)) & 1u)) continue;
            const float4 cj = lds_f4(&win[(j / S) * RW + (j % S)]);
            // d = L_a - L_b, v = L_b - I: w = -(v . d) / (|d|^2 + eps), e = w d + v
            const float dr = ci.x - cj.x, dg = ci.y - cj.y, db = ci.z - cj.z;
            const float vr = cj.x - ir, vg = cj.y - ig, vb = cj.z - ib;
            const float num = -dot3(vr, vg, vb, dr, dg, db);
            const float den = __fadd_rn(dist2(dr, dg, db), eps2);
            const float w = den > 0.f ? __fdividef(num, den) : 1.f;   // eps = 0, L_a = L_b
            const float er = __fmaf_rn(w, dr, vr), eg = __fmaf_rn(w, dg, vg),
                        eb = __fmaf_rn(w, db, vb);
            const float key = dist2(er, eg, eb);
            if (key < bkey) {
                bkey = key;
                bw = w;
                ba = i;
                bb = j;
            }
        }
    }
    SearchOut o;
    if (nvalid == 1 || ba < 0) {
        const float4 c = lds_f4(&win[(only / S) * RW + (only % S)]);
        o.ka = o.kb = only;
        o.omega = 1.f;
        o.err = sqrt_approx(dist2(c.x - ir, c.y - ig, c.z - ib)) * (1.0f / 255.0f);
    } else {
        o.ka = ba;
        o.kb = bb;
        o.omega = bw;
        o.err = sqrt_approx(bkey) * (1.0f / 255.0f);
    }
    const int64_t p = (int64_t)y * a.W + x;
    a.code[p] = (uint16_t)(o.ka * K + o.kb);
    ((float*)a.weight)[p] = o.omega;
    if (a.err) a.err[p] = o.err;
}

template <typename HT>
static int launch_exact_t(const SearchArgs& a, float eps2, cudaStream_t st) {
    const int r = (a.S - 1) / 2;
    const size_t smem = sizeof(float4) * (size_t)((kExH - 1) / a.s + 2 + 2 * r) *
                        (size_t)((kExW - 1) / a.s + 2 + 2 * r);
    const dim3 grid((a.W + kExW - 1) / kExW, (a.H + kExH - 1) / kExH);
    auto run = [&](auto kern) -> int {
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
            return GLU_ERR_CUDA;
        kern<<<grid, kExW * kExH, smem, st>>>(a, eps2);
        GLU_LAUNCH_CHECK();
        return GLU_OK;
    };
    switch (a.S) {
        case 1: return run(k_search_exact<1, HT>);
        case 3: return run(k_search_exact<3, HT>);
        case 5: return run(k_search_exact<5, HT>);
        case 7: return run(k_search_exact<7, HT>);
        default: return run(k_search_exact<9, HT>);
    }
}

int launch_search_exact(const SearchArgs& a, cudaStream_t st) {
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    if (a.wfmt != GLU_W_F32) return GLU_ERR_UNSUPPORTED;   // Eq. 4 weights are not clamped
    // Eq. 4's eps adds to a squared colour distance: eps in [0, 1]^2 units is eps * 255^2 in
    // 1/255 units, i.e. eps255 * 255
    const float eps2 = a.eps255 * 255.0f;
    if (a.hr_dtype == GLU_U8) return launch_exact_t<uint8_t>(a, eps2, st);
    if (a.hr_dtype == GLU_F16) return launch_exact_t<__half>(a, eps2, st);
    return GLU_ERR_UNSUPPORTED;
}

}  // namespace glu
