// Algorithm 2 (Sec. 3.3): joint optimisation of the downsampled image and Theta.
//
// Per iteration n (all launched up front; every kernel returns at once when a device-side flag
// says the loop has converged, so the host never waits in the middle):
//   threshold   E_p > tau marks the large-error set; union-find labels (parent pointers only
//               ever decrease, so every component's root is its smallest raster index)
//   merge/flat  8- (or 4-) connected unions, then every pixel points at its root
//   roots       ordered stream compaction of the roots: component j = the j-th smallest root
//   buckets     pixels and distinct LR blocks per component (counts, exclusive scan, fill)
//   trials      persistent kernel: CTAs claim components in ascending order; component j waits
//               only for earlier components whose LR blocks lie within D of its own (D = 2r for
//               STRICT, r for PAPER) — exactly the components whose trials can read or write
//               state j reads or writes — so the concurrent result equals the sequential one.
//               Waits are bounded (GLU_ERR_TIMEOUT) and can never deadlock: a component only
//               waits for lower indices, which were claimed earlier by running CTAs.
//   residual    R_n = sum_p E_p in FP64 with a fixed reduction order; stop when no trial was
//               kept or R_n >= R_{n-1}.
// Trial sums e0 / e1 are FP32 Kahan sums per LR block (fixed lane order), rounded to 2^-32 and
// added as 64-bit integers: exact and independent of the order blocks finish in.
#include "internal.h"
#include "search.cuh"

namespace glu {

GLU_DEFINE_STATUS(joint)

constexpr int kOwnSlots = 8;        // components recorded per LR pixel before overflow
constexpr int kScanTile = 4096;     // elements per scan tile
constexpr int kScanThreads = 256;   // 16 elements per thread
constexpr int kTrialThreads = 256;
constexpr int kResidChunk = 8192;

struct JointCtl {
    int active;
    int timeout;
    int iterations;
    int M_cur;
    int n_large[GLU_MAX_ITERS];
    int M[GLU_MAX_ITERS];
    int accepted[GLU_MAX_ITERS];
    int rolled[GLU_MAX_ITERS];
    int claim[GLU_MAX_ITERS];
    double residual[GLU_MAX_ITERS + 1];
    unsigned long long searched[GLU_MAX_ITERS];
};

struct JointWs {
    JointCtl* ctl;
    float* err;             // H*W
    int* lab;               // H*W: -1, union-find parent, then component id
    uint8_t* qflag;         // H*W: pixel represents its (component, LR block) pair
    int* roots;             // Mcap
    int* comp_pix;          // H*W
    int* qlist;             // H*W
    int* ulist;             // H*W
    int2* cnt;              // Mcap: (pixels, LR blocks)
    int2* fill;             // Mcap
    int2* start;            // Mcap + 1
    int* done;              // Mcap
    int* tile_a;            // tiles over H*W
    int2* tile_b;           // tiles over Mcap
    int* own;               // h*w*kOwnSlots
    uint8_t* ovf;           // h*w
    unsigned long long* stamp;  // h*w
    unsigned long long* best;   // h*w
    uint32_t* backup;       // h*w
    double* partial;        // residual partials
    int8_t* dlog;           // N * Mcap: kept (1) / rolled back (0) per component and iteration
    int64_t mcap;
};

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static inline int64_t mcap_of(int H, int W) {
    // 8-connected components of single pixels are at most ceil(H/2)*ceil(W/2); 4-connected at
    // most ceil(H*W/2) (checkerboard). Use the larger bound.
    return ((int64_t)H * W + 1) / 2 + 1;
}

// Carve the workspace; returns the bytes needed (ptr may be null to only measure).
static size_t carve(void* base, int H, int W, int h, int w, int N, JointWs* o) {
    const int64_t n = (int64_t)H * W, nl = (int64_t)h * w, mcap = mcap_of(H, W);
    const int64_t tiles_a = (n + kScanTile - 1) / kScanTile + 1;
    const int64_t tiles_b = (mcap + kScanTile - 1) / kScanTile + 1;
    const int64_t nres = (n + kResidChunk - 1) / kResidChunk + 1;
    size_t off = 0;
    char* b = (char*)base;
    auto take = [&](size_t bytes) -> void* {
        void* p = b ? (void*)(b + off) : nullptr;
        off = align256(off + bytes);
        return p;
    };
    JointWs t;
    t.ctl = (JointCtl*)take(sizeof(JointCtl));
    t.err = (float*)take(sizeof(float) * n);
    t.lab = (int*)take(sizeof(int) * n);
    t.qflag = (uint8_t*)take(n);
    t.roots = (int*)take(sizeof(int) * mcap);
    t.comp_pix = (int*)take(sizeof(int) * n);
    t.qlist = (int*)take(sizeof(int) * n);
    t.ulist = (int*)take(sizeof(int) * n);
    t.cnt = (int2*)take(sizeof(int2) * mcap);
    t.fill = (int2*)take(sizeof(int2) * mcap);
    t.start = (int2*)take(sizeof(int2) * (mcap + 1));
    t.done = (int*)take(sizeof(int) * mcap);
    t.tile_a = (int*)take(sizeof(int) * tiles_a);
    t.tile_b = (int2*)take(sizeof(int2) * tiles_b);
    t.own = (int*)take(sizeof(int) * nl * kOwnSlots);
    t.ovf = (uint8_t*)take(nl);
    t.stamp = (unsigned long long*)take(sizeof(unsigned long long) * nl);
    t.best = (unsigned long long*)take(sizeof(unsigned long long) * nl);
    t.backup = (uint32_t*)take(sizeof(uint32_t) * nl);
    t.partial = (double*)take(sizeof(double) * nres);
    t.dlog = (int8_t*)take((size_t)(N > 0 ? N : 1) * (size_t)mcap);
    t.mcap = mcap;
    if (o) *o = t;
    return off;
}

size_t joint_workspace_bytes(int H, int W, int s, int S, int N) {
    (void)S;
    const int h = (H + s - 1) / s, w = (W + s - 1) / s;
    return carve(nullptr, H, W, h, w, N, nullptr);
}

// --------------------------------------------------------------------------- small helpers

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool is_active(const JointCtl* c) {
    return *(volatile const int*)&c->active != 0;
}

// Block-wide exclusive scan of one int per thread (blockDim.x == 256). Returns the total.
__device__ __forceinline__ int block_excl_scan(int v, int* out_excl, int* smem_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < 8 ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < 8) smem_warp[lane] = t;
    }
    __syncthreads();
    const int warp_base = wid > 0 ? smem_warp[wid - 1] : 0;
    const int total = smem_warp[7];
    *out_excl = warp_base + x - v;
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------- control and init kernels

__global__ void k_ctl_init(JointCtl* c, unsigned long long* stamp, int64_t nl) {
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i0 == 0) {
        c->active = 1;
        c->timeout = 0;
        c->iterations = 0;
        c->M_cur = 0;
        for (int k = 0; k < GLU_MAX_ITERS; ++k) {
            c->n_large[k] = 0;
            c->M[k] = 0;
            c->accepted[k] = 0;
            c->rolled[k] = 0;
            c->claim[k] = 0;
            c->searched[k] = 0ull;
        }
    }
    for (int64_t i = i0; i < nl; i += (int64_t)gridDim.x * blockDim.x) stamp[i] = 0ull;
}

// Residual R = sum_p E_p in FP64: fixed chunk per CTA, fixed thread assignment, fixed tree.
__global__ void k_resid_partial(const float* err, int64_t n, double* partial, const JointCtl* c) {
    if (!is_active(c)) return;
    __shared__ double sm[256];
    const int64_t base = (int64_t)blockIdx.x * kResidChunk;
    double acc = 0.0;
    for (int i = threadIdx.x; i < kResidChunk; i += 256) {
        const int64_t p = base + i;
        if (p < n) acc += (double)err[p];
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}

// it < 0: initial residual R_0. Otherwise finish iteration it: record R, decide convergence.
__global__ void k_resid_final(const double* partial, int nb, JointCtl* c, int it) {
    if (!is_active(c)) return;
    __shared__ double sm[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) acc += partial[i];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double R = sm[0];
        if (it < 0) {
            c->residual[0] = R;
        } else {
            c->residual[it + 1] = R;
            c->iterations = it + 1;
            if (c->accepted[it] == 0 || !(R < c->residual[it])) c->active = 0;
        }
    }
}

// ----------------------------------------------------------------------- threshold and CCL

// Large-error set and union-find init; clears the per-LR-pixel owner slots.
__global__ void k_threshold(const float* err, int64_t n, float tau, int* lab, int* own,
                            uint8_t* ovf, int64_t nl, JointCtl* c, int it) {
    if (!is_active(c)) return;
    __shared__ int wsum[8];
    int local = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += stride) {
        const bool fg = err[p] > tau;
        lab[p] = fg ? (int)p : -1;
        local += fg;
    }
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nl; q += stride) {
#pragma unroll
        for (int k = 0; k < kOwnSlots; ++k) own[q * kOwnSlots + k] = -1;
        ovf[q] = 0;
    }
    // block sum then one atomic per block (integer: order-independent)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += wsum[i];
        if (t) atomicAdd(&c->n_large[it], t);
    }
}

// Root of x with path halving; parents only ever decrease (parent < child).
__device__ __forceinline__ int uf_find(int* par, int x) {
    for (;;) {
        const int p = __ldcg(&par[x]);
        if (p == x) return x;
        const int gp = __ldcg(&par[p]);
        if (gp != p) atomicMin(&par[x], gp);
        x = p;
    }
}

__device__ __forceinline__ void uf_union(int* par, int a, int b) {
    for (;;) {
        a = uf_find(par, a);
        b = uf_find(par, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        // link the larger root a under b; if a stopped being a root meanwhile, retry from there
        const int old = atomicMin(&par[a], b);
        if (old == a) return;
        a = old;
    }
}

__global__ void k_ccl_merge(int* lab, int H, int W, int conn, const JointCtl* c) {
    if (!is_active(c)) return;
    const int64_t n = (int64_t)H * W;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (__ldcg(&lab[p]) < 0) continue;
        const int y = (int)(p / W), x = (int)(p % W);
        // backward neighbours only: W, N (and NW, NE for 8-connectivity)
        if (x > 0 && __ldcg(&lab[p - 1]) >= 0) uf_union(lab, (int)p, (int)p - 1);
        if (y > 0) {
            const int64_t up = p - W;
            if (__ldcg(&lab[up]) >= 0) uf_union(lab, (int)p, (int)up);
            if (conn == 8) {
                if (x > 0 && __ldcg(&lab[up - 1]) >= 0) uf_union(lab, (int)p, (int)up - 1);
                if (x + 1 < W && __ldcg(&lab[up + 1]) >= 0) uf_union(lab, (int)p, (int)up + 1);
            }
        }
    }
}

__global__ void k_ccl_flatten(int* lab, int64_t n, const JointCtl* c) {
    if (!is_active(c)) return;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (__ldcg(&lab[p]) >= 0) lab[p] = uf_find(lab, (int)p);
    }
}

// -------------------------------------------------------------- roots: ordered compaction

// per-tile root counts (a root is a labelled pixel that is its own parent)
__global__ void k_root_count(const int* lab, int64_t n, int* tile_cnt, const JointCtl* c) {
    if (!is_active(c)) return;
    __shared__ int wsum[8];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int local = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        const int64_t p = base + i;
        if (p < n && lab[p] == (int)p) ++local;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < 8; ++i) t += wsum[i];
        tile_cnt[blockIdx.x] = t;
    }
}

// single-CTA exclusive scan of tile counts in place; the total becomes M
__global__ void k_root_scan(int* tile_cnt, int ntiles, JointCtl* c, int it) {
    if (!is_active(c)) return;
    __shared__ int wsm[8];
    int carry = 0;
    for (int base = 0; base < ntiles; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const int v = i < ntiles ? tile_cnt[i] : 0;
        int ex;
        const int tot = block_excl_scan(v, &ex, wsm);
        if (i < ntiles) tile_cnt[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        c->M[it] = carry;
        c->M_cur = carry;
        if (carry == 0) c->active = 0;  // the large-error set is empty: Algorithm 2 stops
    }
}

// scatter roots in raster order; component j's per-iteration state is cleared here
__global__ void k_root_scatter(const int* lab, int64_t n, const int* tile_off, int* roots,
                               int2* cnt, int2* fill, int* done, const JointCtl* c) {
    if (!is_active(c)) return;
    __shared__ int wsm[8];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int off = tile_off[blockIdx.x];
    // 16 consecutive elements per thread keep raster order inside the tile
    const int per = kScanTile / kScanThreads;
    const int64_t my = base + (int64_t)threadIdx.x * per;
    int flags = 0, cntl = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int64_t p = my + k;
        const bool r = p < n && lab[p] == (int)p;
        flags |= (int)r << k;
        cntl += r;
    }
    int ex;
    (void)block_excl_scan(cntl, &ex, wsm);
    int j = off + ex;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        if ((flags >> k) & 1) {
            roots[j] = (int)(my + k);
            cnt[j] = make_int2(0, 0);
            fill[j] = make_int2(0, 0);
            done[j] = 0;
            ++j;
        }
    }
}

// ------------------------------------------------------------------- per-component buckets

__device__ __forceinline__ int lower_bound_i(const int* a, int n, int key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// pixel -> component id (lab rewritten in place); counts of pixels and of distinct LR blocks;
// owner slots of each LR block list the components touching it.
__global__ void k_comp_count(int* lab, int H, int W, int s, int w, const int* roots, int2* cnt,
                             int* own, uint8_t* ovf, uint8_t* qflag, const JointCtl* c) {
    if (!is_active(c)) return;
    const int M = c->M_cur;
    const int64_t n = (int64_t)H * W;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int root = lab[p];
        if (root < 0) continue;
        const int j = lower_bound_i(roots, M, root);
        lab[p] = j;
        atomicAdd(&cnt[j].x, 1);
        const int y = (int)(p / W), x = (int)(p % W);
        const int64_t q = (int64_t)(y / s) * w + (x / s);
        int ins = -1;  // 1: inserted here, 0: already present, -1: slots full
        for (int k = 0; k < kOwnSlots; ++k) {
            const int old = atomicCAS(&own[q * kOwnSlots + k], -1, j);
            if (old == -1) { ins = 1; break; }
            if (old == j) { ins = 0; break; }
        }
        if (ins == -1) ovf[q] = 1;
        const bool rep = ins != 0;   // overflowing pixels all list their block (dedup later)
        qflag[p] = rep;
        if (rep) atomicAdd(&cnt[j].y, 1);
    }
}

// multi-CTA exclusive scan of int2 counts over M (read from the control block)
__global__ void k_comp_tile_reduce(const int2* cnt, int2* tile_sum, const JointCtl* c) {
    if (!is_active(c)) return;
    const int M = c->M_cur;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= M) return;
    __shared__ int wx[8], wy[8];
    int sx = 0, sy = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        const int64_t j = base + i;
        if (j < M) { sx += cnt[j].x; sy += cnt[j].y; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if ((threadIdx.x & 31) == 0) { wx[threadIdx.x >> 5] = sx; wy[threadIdx.x >> 5] = sy; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int tx = 0, ty = 0;
        for (int i = 0; i < 8; ++i) { tx += wx[i]; ty += wy[i]; }
        tile_sum[blockIdx.x] = make_int2(tx, ty);
    }
}

__global__ void k_comp_tile_scan(int2* tile_sum, const JointCtl* c) {
    if (!is_active(c)) return;
    const int M = c->M_cur;
    const int ntiles = (M + kScanTile - 1) / kScanTile;
    __shared__ int wsm[8];
    int cx = 0, cy = 0;
    for (int base = 0; base < ntiles; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const int2 v = i < ntiles ? tile_sum[i] : make_int2(0, 0);
        int ex, ey;
        const int tx = block_excl_scan(v.x, &ex, wsm);
        const int ty = block_excl_scan(v.y, &ey, wsm);
        if (i < ntiles) tile_sum[i] = make_int2(cx + ex, cy + ey);
        cx += tx;
        cy += ty;
    }
}

__global__ void k_comp_scan(const int2* cnt, const int2* tile_off, int2* start, const JointCtl* c) {
    if (!is_active(c)) return;
    const int M = c->M_cur;
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= M) return;
    __shared__ int wsm[8];
    const int per = kScanTile / kScanThreads;
    const int64_t my = base + (int64_t)threadIdx.x * per;
    int sx = 0, sy = 0;
    int2 v[per];
#pragma unroll
    for (int k = 0; k < per; ++k) {
        v[k] = (my + k < M) ? cnt[my + k] : make_int2(0, 0);
        sx += v[k].x;
        sy += v[k].y;
    }
    int ex, ey;
    (void)block_excl_scan(sx, &ex, wsm);
    (void)block_excl_scan(sy, &ey, wsm);
    int ox = tile_off[blockIdx.x].x + ex, oy = tile_off[blockIdx.x].y + ey;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        if (my + k < M) start[my + k] = make_int2(ox, oy);
        ox += v[k].x;
        oy += v[k].y;
        if (my + k == M - 1) start[M] = make_int2(ox, oy);
    }
}

__global__ void k_comp_fill(const int* lab, int H, int W, int s, int w, const uint8_t* qflag,
                            const int2* start, int2* fill, int* comp_pix, int* qlist,
                            const JointCtl* c) {
    if (!is_active(c)) return;
    const int64_t n = (int64_t)H * W;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int j = lab[p];
        if (j < 0) continue;
        const int pos = atomicAdd(&fill[j].x, 1);
        comp_pix[start[j].x + pos] = (int)p;
        if (qflag[p]) {
            const int y = (int)(p / W), x = (int)(p % W);
            const int qp = atomicAdd(&fill[j].y, 1);
            qlist[start[j].y + qp] = (y / s) * w + (x / s);
        }
    }
}

// ---------------------------------------------------------------------------- the trials

struct TrialArgs {
    const uint8_t* hr;
    int64_t hr_pitch;
    uint8_t* lr;
    int64_t lr_pitch;
    int H, W, h, w, s;
    float eps255;
    int strict, it;
    uint16_t* code;
    void* weight;
    int wfmt;
    float* err;
    JointWs ws;
};

__device__ __forceinline__ long long to_fixed(float x) {
    // x * 2^32 is exact in float; conversion rounds the part below 2^-32 to nearest
    return __float2ll_rn(x * 4294967296.0f);
}

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__device__ __forceinline__ uint32_t load_rgb(const uint8_t* L, int64_t pitch, int v, int u) {
    const uint8_t* p = L + (int64_t)v * pitch + (int64_t)u * 3;
    return (uint32_t)__ldcg(p) | ((uint32_t)__ldcg(p + 1) << 8) | ((uint32_t)__ldcg(p + 2) << 16);
}

__device__ __forceinline__ void store_rgb(uint8_t* L, int64_t pitch, int v, int u, uint32_t c) {
    uint8_t* p = L + (int64_t)v * pitch + (int64_t)u * 3;
    p[0] = (uint8_t)(c & 255u);
    p[1] = (uint8_t)((c >> 8) & 255u);
    p[2] = (uint8_t)((c >> 16) & 255u);
}

// Wait until done[i] is set; bounded (about a second), and abandoned at once when any other
// wait of the launch has already timed out. Returns false on timeout.
constexpr uint32_t kDoneSpinLimit = 1u << 22;
__device__ __forceinline__ bool wait_done(const int* done, int i, const JointCtl* c) {
    for (uint32_t k = 0; k < kDoneSpinLimit; ++k) {
        if (ld_acquire(&done[i]) != 0) return true;
        if (*(volatile const int*)&c->timeout) return false;
        __nanosleep(128);
    }
    return false;
}

// One warp re-searches the HR pixels of LR block (bv, bu). Sums (Kahan, fixed lane order) the
// stored errors (e0) and the re-searched ones (e1) of the pixels selected by `member`
// (comp >= 0: only pixels of that component), optionally committing Theta and E.
template <int S>
__device__ __forceinline__ void warp_block(const TrialArgs& A, float4* win, int bv, int bu,
                                           int comp, bool commit, float& e0, float& e1) {
    constexpr int r = (S - 1) / 2, K = S * S;
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < K; k += 32) {
        const int v = bv + k / S - r, u = bu + k % S - r;
        float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v >= 0 && v < A.h && u >= 0 && u < A.w) {
            const uint32_t c = load_rgb(A.lr, A.lr_pitch, v, u);
            c4 = make_float4((float)(c & 255u), (float)((c >> 8) & 255u), (float)(c >> 16), 0.f);
        }
        win[k] = c4;
    }
    __syncwarp();
    uint32_t rm, cm;
    window_masks(bv, bu, A.h, A.w, S, rm, cm);
    const int ys = bv * A.s, xs = bu * A.s;
    const int ey = min(A.s, A.H - ys), ex = min(A.s, A.W - xs);
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    int nsearched = 0;
    for (int j = lane; j < ey * ex; j += 32) {
        const int y = ys + j / ex, x = xs + j % ex;
        const int64_t p = (int64_t)y * A.W + x;
        if (comp >= 0 && __ldcg(&A.ws.lab[p]) != comp) continue;
        const uint8_t* ip = A.hr + (int64_t)y * A.hr_pitch + (int64_t)x * 3;
        const SearchOut o = search_pixel<S>(win, S, rm, cm, (float)ip[0], (float)ip[1],
                                            (float)ip[2], A.eps255, false);
        ++nsearched;
        if (commit) {
            A.code[p] = (uint16_t)(o.ka * K + o.kb);
            store_weight(A.weight, A.wfmt, p, o.omega);
            A.err[p] = o.err;
        } else {
            kahan_add(s0, c0, __ldcg(&A.err[p]));
            kahan_add(s1, c1, o.err);
        }
    }
    float t0 = s0 - c0, t1 = s1 - c1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(0xffffffffu, t0, o);
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nsearched += __shfl_xor_sync(0xffffffffu, nsearched, o);
    if (lane == 0 && nsearched) atomicAdd(&A.ws.ctl->searched[A.it], (unsigned long long)nsearched);
    e0 = t0;
    e1 = t1;
    __syncwarp();
}

template <int S>
__global__ void __launch_bounds__(kTrialThreads, 2) k_trials(const TrialArgs A) {
    constexpr int r = (S - 1) / 2;
    JointCtl* ctl = A.ws.ctl;
    if (!is_active(ctl)) return;
    __shared__ float4 wins[kTrialThreads / 32][S * S];
    __shared__ int s_j, s_nu, s_accept;
    __shared__ volatile int s_fail;
    __shared__ long long s_e0, s_e1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nwarps = kTrialThreads / 32;
    const int M = ctl->M_cur;
    const int D = A.strict ? 2 * r : r;
    const JointWs& W_ = A.ws;
    const unsigned long long tagbase = ((unsigned long long)(A.it * 4) << 40);

    for (;;) {
        if (tid == 0) {
            s_j = atomicAdd(&ctl->claim[A.it], 1);
            s_nu = 0;
            s_e0 = 0;
            s_e1 = 0;
            s_fail = 0;
        }
        __syncthreads();
        const int j = s_j;
        if (j >= M) break;
        const int2 st = W_.start[j], en = W_.start[j + 1];

        // 1. wait for every earlier component whose LR blocks lie within D of ours
        for (int t = st.y + tid; t < en.y; t += kTrialThreads) {
            const int q = W_.qlist[t];
            const int qv = q / A.w, qu = q % A.w;
            for (int bv = max(0, qv - D); bv <= min(A.h - 1, qv + D); ++bv)
                for (int bu = max(0, qu - D); bu <= min(A.w - 1, qu + D); ++bu) {
                    const int64_t b = (int64_t)bv * A.w + bu;
                    if (__ldcg(&W_.ovf[b])) {
                        for (int i = 0; i < j && !s_fail; ++i)
                            if (!wait_done(W_.done, i, ctl)) s_fail = 1;
                    } else {
                        for (int k = 0; k < kOwnSlots && !s_fail; ++k) {
                            const int i = __ldcg(&W_.own[b * kOwnSlots + k]);
                            if (i < 0) break;
                            if (i < j && !wait_done(W_.done, i, ctl)) s_fail = 1;
                        }
                    }
                }
        }
        __syncthreads();
        __threadfence();
        if (s_fail) {
            if (tid == 0) {
                set_status(GLU_ERR_TIMEOUT);
                atomicExch(&ctl->timeout, 1);
                st_release(&W_.done[j], 1);  // never leave a later component waiting on us
            }
            __syncthreads();
            continue;
        }

        // 2. the distinct LR blocks Q of the component (stamps drop duplicates)
        const unsigned long long tagQ = tagbase | (unsigned long long)(j + 1);
        for (int t = st.y + tid; t < en.y; t += kTrialThreads) {
            const int q = W_.qlist[t];
            if (atomicExch(&W_.stamp[q], tagQ) != tagQ) {
                const int u = atomicAdd(&s_nu, 1);
                W_.ulist[st.y + u] = q;
                W_.best[q] = 0ull;
            }
        }
        __syncthreads();
        const int nu = s_nu;
        // 3. per q, the largest current error among the component's pixels in its block
        //    (ties: lowest raster index)
        for (int t = st.x + tid; t < en.x; t += kTrialThreads) {
            const int p = W_.comp_pix[t];
            const int y = p / A.W, x = p % A.W;
            const int q = (y / A.s) * A.w + (x / A.s);
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(__ldcg(&A.err[p])) << 32) |
                (unsigned long long)(0xFFFFFFFFu - (uint32_t)p);
            atomicMax(&W_.best[q], key);
        }
        __syncthreads();
        // 4. back up and replace the LR colours
        for (int t = tid; t < nu; t += kTrialThreads) {
            const int q = W_.ulist[st.y + t];
            const int qv = q / A.w, qu = q % A.w;
            const uint32_t p = 0xFFFFFFFFu - (uint32_t)(__ldcg(&W_.best[q]) & 0xFFFFFFFFull);
            const int y = (int)(p / (uint32_t)A.W), x = (int)(p % (uint32_t)A.W);
            W_.backup[q] = load_rgb(A.lr, A.lr_pitch, qv, qu);
            const uint8_t* ip = A.hr + (int64_t)y * A.hr_pitch + (int64_t)x * 3;
            store_rgb(A.lr, A.lr_pitch, qv, qu,
                      (uint32_t)ip[0] | ((uint32_t)ip[1] << 8) | ((uint32_t)ip[2] << 16));
        }
        __syncthreads();

        // 5. e0 / e1 over the affected pixels (STRICT: every block within r of Q; PAPER: the
        //    component's own pixels), then 6. commit or roll back
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1 && !s_accept) break;
            const bool commit = pass == 1;
            const unsigned long long tagB = (tagbase + ((unsigned long long)(pass + 1) << 40)) |
                                            (unsigned long long)(j + 1);
            for (int t = warp; t < nu; t += nwarps) {
                const int q = W_.ulist[st.y + t];
                const int qv = q / A.w, qu = q % A.w;
                if (!A.strict) {
                    float e0, e1;
                    warp_block<S>(A, wins[warp], qv, qu, j, commit, e0, e1);
                    if (!commit && lane == 0) {
                        atomicAdd((unsigned long long*)&s_e0, (unsigned long long)to_fixed(e0));
                        atomicAdd((unsigned long long*)&s_e1, (unsigned long long)to_fixed(e1));
                    }
                    continue;
                }
                for (int bv = max(0, qv - r); bv <= min(A.h - 1, qv + r); ++bv)
                    for (int bu = max(0, qu - r); bu <= min(A.w - 1, qu + r); ++bu) {
                        const int64_t b = (int64_t)bv * A.w + bu;
                        int claimed = 0;
                        if (lane == 0) claimed = atomicExch(&W_.stamp[b], tagB) != tagB;
                        claimed = __shfl_sync(0xffffffffu, claimed, 0);
                        if (!claimed) continue;
                        float e0, e1;
                        warp_block<S>(A, wins[warp], bv, bu, -1, commit, e0, e1);
                        if (!commit && lane == 0) {
                            atomicAdd((unsigned long long*)&s_e0, (unsigned long long)to_fixed(e0));
                            atomicAdd((unsigned long long*)&s_e1, (unsigned long long)to_fixed(e1));
                        }
                    }
            }
            __syncthreads();
            if (pass == 0 && tid == 0) s_accept = !(s_e1 > s_e0);
            __syncthreads();
        }
        if (!s_accept) {
            for (int t = tid; t < nu; t += kTrialThreads) {
                const int q = W_.ulist[st.y + t];
                store_rgb(A.lr, A.lr_pitch, q / A.w, q % A.w, W_.backup[q]);
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            W_.dlog[(int64_t)A.it * W_.mcap + j] = (int8_t)(s_accept ? 1 : 0);
            if (s_accept) atomicAdd(&ctl->accepted[A.it], 1);
            else atomicAdd(&ctl->rolled[A.it], 1);
            st_release(&W_.done[j], 1);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------ host side

static int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

static int grid_cap(int64_t work, int threads, int per_sm = 16) {
    const int64_t blocks = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    return (int)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

template <int S>
static int launch_trials(const TrialArgs& A, cudaStream_t st) {
    static int blocks_per_sm = -1;
    if (blocks_per_sm < 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trials<S>, kTrialThreads, 0) !=
            cudaSuccess)
            return GLU_ERR_CUDA;
        blocks_per_sm = nb > 0 ? nb : 1;
    }
    k_trials<S><<<sm_count() * blocks_per_sm, kTrialThreads, 0, st>>>(A);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

// ---------------------------------------------------------------- phase-timing instrumentation
namespace prof {
constexpr int kSlots = 64, kMaxEv = 4 + 3 * GLU_MAX_ITERS;
static bool enabled = false;
static cudaEvent_t ev[kSlots][kMaxEv];
static int nev[kSlots];
static int used = 0;           // slots filled since the last read
static bool created = false;

static void mark(int slot, int i, cudaStream_t st) {
    if (slot >= 0) cudaEventRecord(ev[slot][i], st);
}
}  // namespace prof

int launch_joint(const JointArgs& a, void* wsp, size_t ws_bytes, glu_joint_stats* stats,
                 cudaStream_t st) {
    int slot = -1;
    if (prof::enabled && prof::used < prof::kSlots) slot = prof::used++;
    int evi = 0;
    JointWs ws;
    const size_t need = carve(wsp, a.H, a.W, a.h, a.w, a.N, &ws);
    if (ws_bytes < need) return GLU_ERR_WORKSPACE;
    float* err = a.err ? a.err : ws.err;
    const int64_t n = (int64_t)a.H * a.W, nl = (int64_t)a.h * a.w;
    const int T = 256;

    prof::mark(slot, evi++, st);
    k_ctl_init<<<grid_cap(nl, T), T, 0, st>>>(ws.ctl, ws.stamp, nl);
    GLU_LAUNCH_CHECK();
    // initialise the LR image by regular grid downsampling, Theta and E by Algorithm 1
    glu_image hr{const_cast<uint8_t*>(a.hr), a.H, a.W, 3, GLU_U8, a.hr_pitch};
    glu_image lr{a.lr, a.h, a.w, 3, GLU_U8, a.lr_pitch};
    int rc = launch_downsample(hr, a.s, GLU_DOWN_GRID, lr, st);
    if (rc) return rc;
    SearchArgs sa;
    sa.hr = a.hr; sa.hr_pitch = a.hr_pitch; sa.hr_dtype = GLU_U8;
    sa.lr = a.lr; sa.lr_pitch = a.lr_pitch; sa.lr_dtype = GLU_U8;
    sa.H = a.H; sa.W = a.W; sa.h = a.h; sa.w = a.w; sa.s = a.s; sa.S = a.S;
    sa.eps255 = a.eps255; sa.gnu = 0;
    sa.code = a.code; sa.weight = a.weight; sa.wfmt = a.wfmt; sa.err = err;
    prof::mark(slot, evi++, st);
    rc = launch_search(sa, st);
    if (rc) return rc;
    prof::mark(slot, evi++, st);
    const int nres = (int)((n + kResidChunk - 1) / kResidChunk);
    k_resid_partial<<<nres, 256, 0, st>>>(err, n, ws.partial, ws.ctl);
    k_resid_final<<<1, 256, 0, st>>>(ws.partial, nres, ws.ctl, -1);
    GLU_LAUNCH_CHECK();
    prof::mark(slot, evi++, st);

    const int tiles_a = (int)((n + kScanTile - 1) / kScanTile);
    const int64_t mcap = mcap_of(a.H, a.W);
    const int tiles_b = (int)((mcap + kScanTile - 1) / kScanTile);
    TrialArgs ta;
    ta.hr = a.hr; ta.hr_pitch = a.hr_pitch; ta.lr = a.lr; ta.lr_pitch = a.lr_pitch;
    ta.H = a.H; ta.W = a.W; ta.h = a.h; ta.w = a.w; ta.s = a.s;
    ta.eps255 = a.eps255; ta.strict = a.strict;
    ta.code = a.code; ta.weight = a.weight; ta.wfmt = a.wfmt; ta.err = err; ta.ws = ws;

    for (int it = 0; it < a.N; ++it) {
        k_threshold<<<grid_cap(n, T), T, 0, st>>>(err, n, a.tau, ws.lab, ws.own, ws.ovf, nl, ws.ctl, it);
        k_ccl_merge<<<grid_cap(n, T), T, 0, st>>>(ws.lab, a.H, a.W, a.conn, ws.ctl);
        k_ccl_flatten<<<grid_cap(n, T), T, 0, st>>>(ws.lab, n, ws.ctl);
        k_root_count<<<tiles_a, kScanThreads, 0, st>>>(ws.lab, n, ws.tile_a, ws.ctl);
        k_root_scan<<<1, kScanThreads, 0, st>>>(ws.tile_a, tiles_a, ws.ctl, it);
        k_root_scatter<<<tiles_a, kScanThreads, 0, st>>>(ws.lab, n, ws.tile_a, ws.roots, ws.cnt,
                                                         ws.fill, ws.done, ws.ctl);
        k_comp_count<<<grid_cap(n, T), T, 0, st>>>(ws.lab, a.H, a.W, a.s, a.w, ws.roots, ws.cnt,
                                                   ws.own, ws.ovf, ws.qflag, ws.ctl);
        k_comp_tile_reduce<<<tiles_b, kScanThreads, 0, st>>>(ws.cnt, ws.tile_b, ws.ctl);
        k_comp_tile_scan<<<1, kScanThreads, 0, st>>>(ws.tile_b, ws.ctl);
        k_comp_scan<<<tiles_b, kScanThreads, 0, st>>>(ws.cnt, ws.tile_b, ws.start, ws.ctl);
        k_comp_fill<<<grid_cap(n, T), T, 0, st>>>(ws.lab, a.H, a.W, a.s, a.w, ws.qflag, ws.start,
                                                  ws.fill, ws.comp_pix, ws.qlist, ws.ctl);
        GLU_LAUNCH_CHECK();
        prof::mark(slot, evi++, st);
        ta.it = it;
        switch (a.S) {
            case 1: rc = launch_trials<1>(ta, st); break;
            case 3: rc = launch_trials<3>(ta, st); break;
            case 5: rc = launch_trials<5>(ta, st); break;
            case 7: rc = launch_trials<7>(ta, st); break;
            case 9: rc = launch_trials<9>(ta, st); break;
            default: return GLU_ERR_UNSUPPORTED;
        }
        if (rc) return rc;
        prof::mark(slot, evi++, st);
        k_resid_partial<<<nres, 256, 0, st>>>(err, n, ws.partial, ws.ctl);
        k_resid_final<<<1, 256, 0, st>>>(ws.partial, nres, ws.ctl, it);
        GLU_LAUNCH_CHECK();
        prof::mark(slot, evi++, st);
    }
    if (slot >= 0) prof::nev[slot] = evi;
    if (stats) {
        JointCtl h;
        GLU_CUDA_TRY(cudaMemcpyAsync(&h, ws.ctl, sizeof(h), cudaMemcpyDeviceToHost, st));
        GLU_CUDA_TRY(cudaStreamSynchronize(st));
        memset(stats, 0, sizeof(*stats));
        stats->iterations = h.iterations;
        for (int k = 0; k < GLU_MAX_ITERS; ++k) {
            stats->n_large[k] = h.n_large[k];
            stats->components[k] = h.M[k];
            stats->accepted[k] = h.accepted[k];
            stats->rolled_back[k] = h.rolled[k];
        }
        for (int k = 0; k <= h.iterations && k <= GLU_MAX_ITERS; ++k) stats->residual[k] = h.residual[k];
        for (int k = 0; k < GLU_MAX_ITERS; ++k) stats->searched[k] = (int64_t)h.searched[k];
        if (h.timeout) return GLU_ERR_TIMEOUT;
    }
    return GLU_OK;
}

int joint_decisions(const void* wsp, size_t ws_bytes, int H, int W, int s, int N, int8_t* out,
                    int64_t cap, cudaStream_t st, int64_t* written) {
    const int h = (H + s - 1) / s, w = (W + s - 1) / s;
    JointWs ws;
    const size_t need = carve(const_cast<void*>(wsp), H, W, h, w, N, &ws);
    if (ws_bytes < need) return GLU_ERR_WORKSPACE;
    JointCtl c;
    GLU_CUDA_TRY(cudaMemcpyAsync(&c, ws.ctl, sizeof(c), cudaMemcpyDeviceToHost, st));
    GLU_CUDA_TRY(cudaStreamSynchronize(st));
    int64_t off = 0;
    for (int it = 0; it < c.iterations && it < N; ++it) {
        const int64_t m = c.M[it];
        if (off + m > cap) return GLU_ERR_INVALID_ARG;
        if (m > 0)
            GLU_CUDA_TRY(cudaMemcpyAsync(out + off, ws.dlog + (int64_t)it * ws.mcap, (size_t)m,
                                         cudaMemcpyDeviceToHost, st));
        off += m;
    }
    GLU_CUDA_TRY(cudaStreamSynchronize(st));
    *written = off;
    return GLU_OK;
}

}  // namespace glu

extern "C" int glu_joint_profile(int32_t enable) {
    using namespace glu;
    if (enable && !prof::created) {
        for (int i = 0; i < prof::kSlots; ++i)
            for (int j = 0; j < prof::kMaxEv; ++j)
                if (cudaEventCreate(&prof::ev[i][j]) != cudaSuccess) return GLU_ERR_CUDA;
        prof::created = true;
    }
    prof::enabled = enable != 0;
    return GLU_OK;
}

extern "C" int glu_joint_profile_read(float* ms, int32_t* calls) {
    using namespace glu;
    if (!ms || !calls) return GLU_ERR_INVALID_ARG;
    for (int k = 0; k < 5; ++k) ms[k] = 0.f;
    *calls = 0;
    for (int sl = 0; sl < prof::used; ++sl) {
        const int n = prof::nev[sl];
        if (n < 4) continue;
        if (cudaEventSynchronize(prof::ev[sl][n - 1]) != cudaSuccess) return GLU_ERR_CUDA;
        float t = 0.f;
        cudaEventElapsedTime(&t, prof::ev[sl][0], prof::ev[sl][1]);
        ms[0] += t;  // control init + grid downsample
        cudaEventElapsedTime(&t, prof::ev[sl][1], prof::ev[sl][2]);
        ms[1] += t;  // Algorithm 1 search kernel
        cudaEventElapsedTime(&t, prof::ev[sl][2], prof::ev[sl][3]);
        ms[4] += t;  // R_0
        // per iteration: [previous end .. components built] [.. trials] [.. residual]
        for (int i = 3; i + 3 <= n - 1; i += 3) {
            cudaEventElapsedTime(&t, prof::ev[sl][i], prof::ev[sl][i + 1]);
            ms[2] += t;
            cudaEventElapsedTime(&t, prof::ev[sl][i + 1], prof::ev[sl][i + 2]);
            ms[3] += t;
            cudaEventElapsedTime(&t, prof::ev[sl][i + 2], prof::ev[sl][i + 3]);
            ms[4] += t;
        }
        ++*calls;
    }
    prof::used = 0;
    return GLU_OK;
}
