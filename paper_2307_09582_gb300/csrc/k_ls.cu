// Least-squares LR colour update alternated with Algorithm 1 (an alternative to Algorithm 2's
// replace-and-roll-back joint optimisation; not the paper's method).
//
// Update, for a fixed Theta: every LR pixel q independently takes the value that minimises the
// Eq. 1 reconstruction error sum_p || T_hat_p - I_p ||^2 (T = L) with the other LR pixels held at
// their current values (a Jacobi sweep of the normal equations). Pixel p reconstructs
// c_pa L_a + c_pb L_b with c_pa = w_p, c_pb = 1 - w_p, or L_a alone (c = 1) when a_p = b_p, so
//     num_q = sum_p c_pq (I_p - c_pj L_j),   den_q = sum_p c_pq^2,   L'_q = clamp(num_q / den_q)
// over the pixels that use q (j: p's other LR pixel, if any); an LR pixel no pixel uses keeps its
// value. As in the adjoint of Eq. 1 (k_apply.cu), a pixel of LR block B reaches exactly the LR
// pixels at its two window indices, so:
//   k_ls_block_sums: a warp per block stages its pixels' contributions (num for both targets,
//     den), lane k sums bucket k over the block's pixels in raster order with Kahan
//     compensation, and stores the sums in the slot of the LR pixel the bucket feeds;
//   k_ls_gather: a thread per LR pixel adds its slots (neighbours in order, a before b) with
//     Kahan compensation and writes the new colour.
// Per-LR-pixel accumulation in FP32 with compensation, fixed order: bit-reproducible.
//
// The alternation (glu_ls_joint_optimize): L = grid downsampling, Theta / E = Algorithm 1; then N
// times: L' = update(L, Theta), Theta' / E' = Algorithm 1 on L', R' = sum_p E'_p (exact 64-bit
// fixed point, 2^-32 units); the new state is kept only while R' < R (a device-side flag; once an
// update is not kept, the later iterations change nothing).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace glu {

GLU_DEFINE_STATUS(ls)

// Exact n / d for 0 <= n < 2^22 (window and pixel indices): (n + 0.5) / d stays at least
// 0.5 / d from an integer, above the float error of (n + 0.5) * fl(1 / d).
__device__ __forceinline__ int qdiv_f(int n, float inv_d) {
    return __float2int_rd(((float)n + 0.5f) * inv_d);
}

constexpr int kLsChunk = 128;   // pixels a warp stages at a time
constexpr int kLsSlot = 8;      // floats per slot: a (num r, g, b, den), b (num r, g, b, den)

__device__ __forceinline__ void kahan(float& sum, float& comp, float v) {
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

struct LsArgs {
    const void* hr;
    int64_t hr_pitch;
    int hr_dtype;
    const uint16_t* code;
    const float* weight;
    const float* L;       // current LR colours, [0, 1], h x w x 3 (pitch in floats)
    int64_t L_pitch;
    float* Lout;          // new LR colours
    int64_t Lout_pitch;
    int H, W, h, w, s, S;
    float* slots;         // h * w * S^2 * kLsSlot floats
    const int* active;    // nullable: the update runs only while *active != 0
};

template <typename HT>
__device__ __forceinline__ float hr_unit(const void* hr, int64_t i);
template <> __device__ __forceinline__ float hr_unit<uint8_t>(const void* hr, int64_t i) {
    return (float)((const uint8_t*)hr)[i] * (1.0f / 255.0f);
}
template <> __device__ __forceinline__ float hr_unit<__half>(const void* hr, int64_t i) {
    return __half2float(((const __half*)hr)[i]);
}

template <typename HT, int NQ>
__global__ void __launch_bounds__(256) k_ls_block_sums(const LsArgs A) {
    if (A.active && *(volatile const int*)A.active == 0) return;
    __shared__ int s_pair[8][kLsChunk];
    __shared__ float4 s_ca[8][kLsChunk];   // contribution to q_a: (num r, g, b, den)
    __shared__ float4 s_cb[8][kLsChunk];   // to q_b
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = (A.S - 1) >> 1, S = A.S, K = S * S, s = A.s;
    const float invK = 1.0f / (float)K, invS = 1.0f / (float)S;
    const int64_t nblocks = (int64_t)A.h * A.w;
    for (int64_t blk = (int64_t)blockIdx.x * 8 + warp; blk < nblocks;
         blk += (int64_t)gridDim.x * 8) {
        const int bv = (int)(blk / A.w), bu = (int)(blk - (int64_t)bv * A.w);
        float sa[NQ][4], ca[NQ][4], sb[NQ][4], cb[NQ][4];   // Kahan sums and compensations
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int c = 0; c < 4; ++c) sa[q][c] = ca[q][c] = sb[q][c] = cb[q][c] = 0.f;
        const int ys = bv * s, xs = bu * s;
        const int ey = min(s, A.H - ys), ex = min(s, A.W - xs), n = ey * ex;
        const float inv_ex = 1.0f / (float)ex;
        for (int j0 = 0; j0 < n; j0 += kLsChunk) {
            const int m = min(kLsChunk, n - j0);
            for (int jj = lane; jj < m; jj += 32) {
                const int j = j0 + jj, jy = qdiv_f(j, inv_ex);
                const int y = ys + jy, x = xs + (j - jy * ex);
                const int64_t p = (int64_t)y * A.W + x;
                const int code = A.code[p];
                const float w = A.weight[p];
                const int64_t ih = (int64_t)y * A.hr_pitch + (int64_t)x * 3;
                const float ir = hr_unit<HT>(A.hr, ih), ig = hr_unit<HT>(A.hr, ih + 1),
                            ib = hr_unit<HT>(A.hr, ih + 2);
                int ka = qdiv_f(code, invK), kb = code - ka * K;
                float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
                if (code >= K * K) {
                    set_status(GLU_ERR_DEVICE_CHECK);
                    ka = kb = 255;   // matches no bucket
                } else if (ka == kb) {
                    va = make_float4(ir, ig, ib, 1.f);   // T_hat_p = L_a: coefficient 1
                    kb = 255;
                } else {
                    const int kar = qdiv_f(ka, invS), kbr = qdiv_f(kb, invS);
                    const int64_t la = (int64_t)(bv + kar - r) * A.L_pitch +
                                       (int64_t)(bu + (ka - kar * S) - r) * 3;
                    const int64_t lb = (int64_t)(bv + kbr - r) * A.L_pitch +
                                       (int64_t)(bu + (kb - kbr * S) - r) * 3;
                    const float wa = w, wb = 1.f - w;
                    va = make_float4(wa * (ir - wb * A.L[lb]), wa * (ig - wb * A.L[lb + 1]),
                                     wa * (ib - wb * A.L[lb + 2]), wa * wa);
                    vb = make_float4(wb * (ir - wa * A.L[la]), wb * (ig - wa * A.L[la + 1]),
                                     wb * (ib - wa * A.L[la + 2]), wb * wb);
                }
                s_pair[warp][jj] = ka | (kb << 8);
                s_ca[warp][jj] = va;
                s_cb[warp][jj] = vb;
            }
            __syncwarp();
            for (int jj = 0; jj < m; ++jj) {
                const int pr = s_pair[warp][jj];
                const int ka = pr & 0xFF, kb = pr >> 8;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int kk = lane + 32 * q;
                    if (ka == kk) {
                        const float4 v = s_ca[warp][jj];
                        kahan(sa[q][0], ca[q][0], v.x);
                        kahan(sa[q][1], ca[q][1], v.y);
                        kahan(sa[q][2], ca[q][2], v.z);
                        kahan(sa[q][3], ca[q][3], v.w);
                    }
                    if (kb == kk) {
                        const float4 v = s_cb[warp][jj];
                        kahan(sb[q][0], cb[q][0], v.x);
                        kahan(sb[q][1], cb[q][1], v.y);
                        kahan(sb[q][2], cb[q][2], v.z);
                        kahan(sb[q][3], cb[q][3], v.w);
                    }
                }
            }
            __syncwarp();
        }
        // bucket k feeds q = B + (k / S - r, k % S - r) as its neighbour K - 1 - k
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int kk = lane + 32 * q;
            if (kk >= K) continue;
            const int kr = qdiv_f(kk, invS);
            const int qv = bv + kr - r, qu = bu + (kk - kr * S) - r;
            if (qv < 0 || qv >= A.h || qu < 0 || qu >= A.w) continue;
            float4* o = (float4*)(A.slots + (((int64_t)qv * A.w + qu) * K + (K - 1 - kk)) * kLsSlot);
            o[0] = make_float4(sa[q][0], sa[q][1], sa[q][2], sa[q][3]);
            o[1] = make_float4(sb[q][0], sb[q][1], sb[q][2], sb[q][3]);
        }
    }
}

__global__ void __launch_bounds__(256) k_ls_gather(const LsArgs A) {
    if (A.active && *(volatile const int*)A.active == 0) return;
    const int r = (A.S - 1) >> 1, S = A.S, K = S * S;
    const float invS = 1.0f / (float)S;
    const int64_t nq = (int64_t)A.h * A.w;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(q / A.w), u = (int)(q - (int64_t)v * A.w);
        float sum[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
        const float4* sl = (const float4*)(A.slots + q * K * kLsSlot);
        for (int n = 0; n < K; ++n) {
            const int nr = qdiv_f(n, invS);
            const int bv = v + nr - r, bu = u + (n - nr * S) - r;
            if (bv < 0 || bv >= A.h || bu < 0 || bu >= A.w) continue;
            const float4 a = __ldg(&sl[2 * n]), b = __ldg(&sl[2 * n + 1]);
            kahan(sum[0], comp[0], a.x);
            kahan(sum[1], comp[1], a.y);
            kahan(sum[2], comp[2], a.z);
            kahan(sum[3], comp[3], a.w);
            kahan(sum[0], comp[0], b.x);
            kahan(sum[1], comp[1], b.y);
            kahan(sum[2], comp[2], b.z);
            kahan(sum[3], comp[3], b.w);
        }
        const int64_t li = (int64_t)v * A.L_pitch + (int64_t)u * 3;
        const int64_t lo = (int64_t)v * A.Lout_pitch + (int64_t)u * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float x = sum[3] > 0.f ? __fdiv_rn(sum[c], sum[3]) : A.L[li + c];
            A.Lout[lo + c] = fminf(fmaxf(x, 0.f), 1.f);
        }
    }
}

static int grid_cap(int64_t work, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = (work + threads - 1) / threads, cap = (int64_t)sms * 16;
    return (int)std::max<int64_t>(1, std::min(blocks, cap));
}

size_t ls_update_workspace_bytes(int h, int w, int S) {
    return (size_t)h * w * (size_t)S * S * kLsSlot * sizeof(float);
}

static int launch_ls_update(const LsArgs& a, cudaStream_t st) {
    const int K = a.S * a.S;
    const int64_t nb = (int64_t)a.h * a.w;
    const int g1 = grid_cap(nb * 32, 256);
    auto run = [&](auto kern) { kern<<<g1, 256, 0, st>>>(a); };
    if (a.hr_dtype == GLU_U8) {
        if (K <= 32) run(k_ls_block_sums<uint8_t, 1>);
        else if (K <= 64) run(k_ls_block_sums<uint8_t, 2>);
        else run(k_ls_block_sums<uint8_t, 3>);
    } else {
        if (K <= 32) run(k_ls_block_sums<__half, 1>);
        else if (K <= 64) run(k_ls_block_sums<__half, 2>);
        else run(k_ls_block_sums<__half, 3>);
    }
    GLU_LAUNCH_CHECK();
    k_ls_gather<<<grid_cap(nb, 256), 256, 0, st>>>(a);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

int ls_update(const LsUpdate& u, cudaStream_t st) {
    LsArgs a;
    a.hr = u.hr;
    a.hr_pitch = u.hr_pitch;
    a.hr_dtype = u.hr_dtype;
    a.code = u.code;
    a.weight = u.weight;
    a.L = u.L;
    a.L_pitch = u.L_pitch;
    a.Lout = u.Lout;
    a.Lout_pitch = u.Lout_pitch;
    a.H = u.H;
    a.W = u.W;
    a.h = u.h;
    a.w = u.w;
    a.s = u.s;
    a.S = u.S;
    a.slots = u.slots;
    a.active = u.active;
    if (a.H <= 0 || a.W <= 0) return GLU_OK;
    return launch_ls_update(a, st);
}

// ------------------------------------------------------------------- the alternation

struct LsCtl {
    unsigned long long R[GLU_MAX_ITERS + 1];   // residuals in 2^-32 units (R[0] = initial)
    int active;                                // 0 once an update was not kept
    int kept;                                  // updates kept
};

__global__ void k_ls_init(LsCtl* c) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int i = 0; i <= GLU_MAX_ITERS; ++i) c->R[i] = 0ull;
        c->active = 1;
        c->kept = 0;
    }
}

// R[slot] += sum_p round(2^32 E_p): exact, order-independent (one 64-bit atomic per CTA).
__global__ void __launch_bounds__(256) k_ls_resid(const float* E, int64_t n, LsCtl* c, int slot) {
    if (slot > 0 && *(volatile const int*)&c->active == 0) return;
    __shared__ unsigned long long sm[8];
    unsigned long long acc = 0ull;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        acc += __float2ull_rn(E[p] * 4294967296.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0ull;
        for (int w = 0; w < 8; ++w) t += sm[w];
        atomicAdd(&c->R[slot], t);
    }
}

// The iteration's candidate state is kept while its residual is below the current one.
__global__ void k_ls_decide(LsCtl* c, int it) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && c->active) {
        if (c->R[it] < c->R[c->kept]) {
            c->kept = it;
        } else {
            c->active = 0;
        }
    }
}

// Copy the candidate (LR colours, Theta, E) over the state when iteration `it` was kept.
__global__ void __launch_bounds__(256) k_ls_commit(const LsCtl* c, int it, const float* Lc,
                                                   int64_t Lc_pitch, float* L, int64_t L_pitch,
                                                   int h, int w, const uint16_t* codec,
                                                   const float* wc, const float* Ec,
                                                   uint16_t* code, float* weight, float* E,
                                                   int64_t n) {
    if (*(volatile const int*)&c->kept != it) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += stride) {
        code[p] = codec[p];
        weight[p] = wc[p];
        if (E) E[p] = Ec[p];
    }
    const int64_t nl = (int64_t)h * w * 3;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl; i += stride) {
        const int64_t q = i / 3, c3 = i - q * 3, v = q / w, u = q - v * w;
        L[v * L_pitch + u * 3 + c3] = Lc[v * Lc_pitch + u * 3 + c3];
    }
}

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t ls_joint_workspace_bytes(int H, int W, int s, int S) {
    const size_t np = (size_t)H * W, h = (size_t)(H + s - 1) / s, w = (size_t)(W + s - 1) / s;
    return align256(sizeof(LsCtl)) + align256(ls_update_workspace_bytes((int)h, (int)w, S)) +
           align256(h * w * 3 * sizeof(float)) +          // candidate LR colours
           align256(np * sizeof(uint16_t)) +              // candidate codes
           2 * align256(np * sizeof(float)) +             // candidate weights and E
           align256(np * sizeof(float));                  // E when the caller passes none
}

int ls_joint(const LsJoint& j, cudaStream_t st, unsigned long long* R_host, int* kept_host) {
    const int H = j.H, W = j.W, s = j.s, S = j.S;
    const int h = (H + s - 1) / s, w = (W + s - 1) / s;
    const int64_t np = (int64_t)H * W;
    char* b = (char*)j.ws;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void* p = b + off;
        off += align256(bytes);
        return p;
    };
    LsCtl* ctl = (LsCtl*)take(sizeof(LsCtl));
    float* slots = (float*)take(ls_update_workspace_bytes(h, w, S));
    float* Lc = (float*)take((size_t)h * w * 3 * sizeof(float));
    uint16_t* codec = (uint16_t*)take((size_t)np * sizeof(uint16_t));
    float* wc = (float*)take((size_t)np * sizeof(float));
    float* Ec = (float*)take((size_t)np * sizeof(float));
    float* Eown = (float*)take((size_t)np * sizeof(float));
    float* E = j.err ? j.err : Eown;
    k_ls_init<<<1, 32, 0, st>>>(ctl);
    GLU_LAUNCH_CHECK();
    // grid downsampling into the caller's float LR image, then Algorithm 1
    glu_image hri = j.hr_image, lri = j.lr_image;
    int rc = launch_downsample(hri, s, GLU_DOWN_GRID, lri, st);
    if (rc) return rc;
    SearchArgs a;
    a.hr = j.hr_image.data;
    a.hr_pitch = j.hr_image.pitch;
    a.hr_dtype = j.hr_image.dtype;
    a.lr = j.L;
    a.lr_pitch = j.L_pitch;
    a.lr_dtype = GLU_F32;
    a.H = H;
    a.W = W;
    a.h = h;
    a.w = w;
    a.s = s;
    a.S = S;
    a.eps255 = j.eps255;
    a.gnu = 0;
    a.code = j.code;
    a.weight = j.weight;
    a.wfmt = GLU_W_F32;
    a.err = E;
    rc = launch_search(a, st);
    if (rc) return rc;
    const int gr = grid_cap(np, 256);
    k_ls_resid<<<gr, 256, 0, st>>>(E, np, ctl, 0);
    GLU_LAUNCH_CHECK();
    for (int it = 1; it <= j.N; ++it) {
        LsUpdate u;
        u.hr = j.hr_image.data;
        u.hr_pitch = j.hr_image.pitch;
        u.hr_dtype = j.hr_image.dtype;
        u.code = j.code;
        u.weight = j.weight;
        u.L = j.L;
        u.L_pitch = j.L_pitch;
        u.Lout = Lc;
        u.Lout_pitch = (int64_t)w * 3;
        u.H = H;
        u.W = W;
        u.h = h;
        u.w = w;
        u.s = s;
        u.S = S;
        u.slots = slots;
        u.active = &ctl->active;
        rc = ls_update(u, st);
        if (rc) return rc;
        // Algorithm 1 on the candidate LR image (runs even once the loop has stopped; its
        // result is then not kept)
        SearchArgs c = a;
        c.lr = Lc;
        c.lr_pitch = (int64_t)w * 3;
        c.code = codec;
        c.weight = wc;
        c.err = Ec;
        rc = launch_search(c, st);
        if (rc) return rc;
        k_ls_resid<<<gr, 256, 0, st>>>(Ec, np, ctl, it);
        k_ls_decide<<<1, 32, 0, st>>>(ctl, it);
        k_ls_commit<<<gr, 256, 0, st>>>(ctl, it, Lc, (int64_t)w * 3, j.L, j.L_pitch, h, w,
                                        codec, wc, Ec, j.code, j.weight, j.err ? E : nullptr,
                                        np);
        GLU_LAUNCH_CHECK();
    }
    if (R_host || kept_host) {
        LsCtl hc;
        if (cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return GLU_ERR_CUDA;
        if (R_host)
            for (int i = 0; i <= j.N; ++i) R_host[i] = hc.R[i];
        if (kept_host) *kept_host = hc.kept;
    }
    return GLU_OK;
}

}  // namespace glu
