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
    int finished[GLU_MAX_ITERS];   // components done (kept or rolled back) per iteration
    int open_tasks;                // published tasks that still have unclaimed items
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
    uint16_t* sh_code;      // H*W shadow Theta / E written by a trial, copied if it is kept
    float* sh_w;            // H*W
    float* sh_err;          // H*W
    // one task slot per persistent CTA: the block items of its component's trial or commit,
    // open to every warp of the grid
    unsigned long long* slot_word;  // (epoch << 32) | next item; odd epoch = open
    int* slot_j;
    int* slot_n;            // items
    int* slot_nu;           // distinct LR blocks of the component
    int* slot_kind;         // 0 trial, 1 commit
    unsigned long long* slot_e0;
    unsigned long long* slot_e1;
    int* slot_fin;          // items finished
};

constexpr int kMaxSlots = 4096;

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
    t.sh_code = (uint16_t*)take(sizeof(uint16_t) * n);
    t.sh_w = (float*)take(sizeof(float) * n);
    t.sh_err = (float*)take(sizeof(float) * n);
    t.slot_word = (unsigned long long*)take(sizeof(unsigned long long) * kMaxSlots);
    t.slot_j = (int*)take(sizeof(int) * kMaxSlots);
    t.slot_n = (int*)take(sizeof(int) * kMaxSlots);
    t.slot_nu = (int*)take(sizeof(int) * kMaxSlots);
    t.slot_kind = (int*)take(sizeof(int) * kMaxSlots);
    t.slot_e0 = (unsigned long long*)take(sizeof(unsigned long long) * kMaxSlots);
    t.slot_e1 = (unsigned long long*)take(sizeof(unsigned long long) * kMaxSlots);
    t.slot_fin = (int*)take(sizeof(int) * kMaxSlots);
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

__global__ void k_ctl_init(JointCtl* c, unsigned long long* stamp, int64_t nl,
                           unsigned long long* slot_word) {
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t i = i0; i < kMaxSlots; i += (int64_t)gridDim.x * blockDim.x) slot_word[i] = 0ull;
    if (i0 == 0) {
        c->active = 1;
        c->timeout = 0;
        c->iterations = 0;
        c->M_cur = 0;
        c->open_tasks = 0;
        for (int k = 0; k < GLU_MAX_ITERS; ++k) {
            c->n_large[k] = 0;
            c->M[k] = 0;
            c->accepted[k] = 0;
            c->rolled[k] = 0;
            c->claim[k] = 0;
            c->searched[k] = 0ull;
            c->finished[k] = 0;
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

#ifdef GLU_TRIAL_TRACE
// Debug builds only: per-component timestamps (claim, dependencies met, trial summed, done).
constexpr int kTraceMax = 1 << 15;
static __device__ unsigned long long g_trace[GLU_MAX_ITERS][kTraceMax][4];
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
#define GLU_TRACE(it, j, k) \
    do { if (tid == 0 && (j) < kTraceMax) g_trace[it][j][k] = gtimer(); } while (0)
#else
#define GLU_TRACE(it, j, k) do { } while (0)
#endif

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

// Weight load through L2 (the planes are written by other CTAs during the trials).
__device__ __forceinline__ float load_weight_cg(const void* base, int fmt, int64_t i) {
    if (fmt == GLU_W_F32) return __ldcg((const float*)base + i);
    if (fmt == GLU_W_F16) return __half2float(__ldcg((const __half*)base + i));
    return (float)__ldcg((const unsigned short*)base + i) * (1.0f / 65535.0f);
}

// One warp re-runs Algorithm 1 on the HR pixels of LR block (bv, bu) against the current LR
// image (comp >= 0: only the pixels of that component), writing the results in place and the
// previous values to the backup planes. The previous errors (e0) and the new ones (e1) are
// summed with Kahan compensation in a fixed lane order and reduced with a fixed butterfly.
template <int S>
__device__ __noinline__ void warp_block_trial(const TrialArgs& A, float4* win, int bv, int bu,
                                                 int comp, float& e0, float& e1) {
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
        const SearchOut o = search_pixel<S, true>(win, S, rm, cm, (float)ip[0], (float)ip[1],
                                                  (float)ip[2], A.eps255, false);
        ++nsearched;
        // the new Theta / E go in place; the old ones to the backup planes (restored if the
        // trial is rolled back)
        const float eold = __ldcg(&A.err[p]);
        A.ws.sh_code[p] = __ldcg(&A.code[p]);
        A.ws.sh_w[p] = load_weight_cg(A.weight, A.wfmt, p);
        A.ws.sh_err[p] = eold;
        A.code[p] = (uint16_t)(o.ka * K + o.kb);
        store_weight(A.weight, A.wfmt, p, o.omega);
        A.err[p] = o.err;
        kahan_add(s0, c0, eold);
        kahan_add(s1, c1, o.err);
    }
    float t0 = s0 - c0, t1 = s1 - c1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(0xffffffffu, t0, o);
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        nsearched += __shfl_xor_sync(0xffffffffu, nsearched, o);
    }
    if (lane == 0 && nsearched) atomicAdd(&A.ws.ctl->searched[A.it], (unsigned long long)nsearched);
    e0 = t0;
    e1 = t1;
    __syncwarp();
}

// Roll back a trial for LR block (bv, bu): restore Theta and E from the backup planes.
__device__ __forceinline__ void warp_block_commit(const TrialArgs& A, int bv, int bu, int comp) {
    const int lane = threadIdx.x & 31;
    const int ys = bv * A.s, xs = bu * A.s;
    const int ey = min(A.s, A.H - ys), ex = min(A.s, A.W - xs);
    for (int j = lane; j < ey * ex; j += 32) {
        const int y = ys + j / ex, x = xs + j % ex;
        const int64_t p = (int64_t)y * A.W + x;
        if (comp >= 0 && __ldcg(&A.ws.lab[p]) != comp) continue;
        A.code[p] = __ldcg(&A.ws.sh_code[p]);
        store_weight_raw(A.weight, A.wfmt, p, __ldcg(&A.ws.sh_w[p]));
        A.err[p] = __ldcg(&A.ws.sh_err[p]);
    }
}

// Block item t of component j (trial or commit enumeration): the LR block it designates, or
// false when it falls outside the LR image. STRICT: (distinct block u, neighbour nb) pairs;
// PAPER: the distinct blocks themselves.
template <int S>
__device__ __forceinline__ bool item_block(const TrialArgs& A, int stY, int t, int& bv, int& bu) {
    constexpr int r = (S - 1) / 2, NB = (2 * r + 1) * (2 * r + 1);
    const int q = A.ws.ulist[stY + (A.strict ? t / NB : t)];
    bv = q / A.w;
    bu = q % A.w;
    if (A.strict) {
        const int nb = t % NB;
        bv += nb / (2 * r + 1) - r;
        bu += nb % (2 * r + 1) - r;
        if (bv < 0 || bv >= A.h || bu < 0 || bu >= A.w) return false;
    }
    return true;
}

__device__ __forceinline__ unsigned long long trial_tag(int it, int j, int phase) {
    return ((unsigned long long)(it * 4 + phase) << 40) | (unsigned long long)(j + 1);
}

// One warp processes item t of component j: claims its block (STRICT blocks reached from several
// q are processed once), then runs the trial (kind 0, sums returned) or the commit (kind 1).
template <int S>
__device__ __forceinline__ bool process_item(const TrialArgs& A, float4* win, int j, int stY,
                                             int kind, int t, float& e0, float& e1) {
    const int lane = threadIdx.x & 31;
    e0 = 0.f;
    e1 = 0.f;
    int bv, bu;
    if (!item_block<S>(A, stY, t, bv, bu)) return false;
    if (A.strict) {
        const unsigned long long tag = trial_tag(A.it, j, kind + 1);
        int claimed = 0;
        if (lane == 0) claimed = atomicExch(&A.ws.stamp[(int64_t)bv * A.w + bu], tag) != tag;
        if (!__shfl_sync(0xffffffffu, claimed, 0)) return false;
    }
    if (kind == 0)
        warp_block_trial<S>(A, win, bv, bu, A.strict ? -1 : j, e0, e1);
    else
        warp_block_commit(A, bv, bu, A.strict ? -1 : j);
    return true;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *(volatile const unsigned long long*)p;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Backstop for every wait of the trial kernel: a launch that has run this long has gone wrong
// (the whole 4K workload takes milliseconds); give up, record GLU_ERR_TIMEOUT and return.
constexpr unsigned long long kTrialDeadlineNs = 5000000000ull;

// Warp-uniform: true when the launch must stop waiting (deadline passed or another wait
// already timed out). Lane 0 decides, every lane gets the same answer.
__device__ __forceinline__ bool warp_should_abort(const JointCtl* c, unsigned long long t0) {
    int a = 0;
    if ((threadIdx.x & 31) == 0)
        a = (*(volatile const int*)&c->timeout != 0) || (now_ns() - t0 > kTrialDeadlineNs);
    return __shfl_sync(0xffffffffu, a, 0) != 0;
}

__device__ __forceinline__ unsigned long long atom_add_acquire_u64(unsigned long long* p,
                                                                   unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.acquire.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v)
                 : "memory");
    return old;
}

__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// True when slot k holds an open task with unclaimed items (a relaxed snapshot).
__device__ __forceinline__ bool slot_has_items(const JointWs& W_, int k) {
    const unsigned long long w = ld_volatile_u64(&W_.slot_word[k]);
    return ((w >> 32) & 1ull) && (int)(w & 0xFFFFFFFFull) < *(volatile const int*)&W_.slot_n[k];
}

// One warp: take one unclaimed item of an open task — its own CTA's slot first, then the slot it
// helped last (`hint`), otherwise the open task of the smallest component — and process it.
// Returns false if no item was available.
//
// Claiming is one fetch-and-add on the slot's (epoch << 32 | next) word. An increment that lands
// on a closed slot is harmless (opening overwrites the word); one that lands on an open epoch
// owns item `next` of that epoch, whose context cannot change before that item is finished.
template <int S>
__device__ bool help_one(const TrialArgs& A, float4* win, int own, int G, int& hint) {
    const JointWs& W_ = A.ws;
    const int lane = threadIdx.x & 31;
    int s_sel = -1;
    if (lane == 0) {
        if (slot_has_items(W_, own)) s_sel = own;
        else if (hint >= 0 && slot_has_items(W_, hint)) s_sel = hint;
        else if (*(volatile const int*)&W_.ctl->open_tasks <= 0) s_sel = -2;  // nothing open
    }
    s_sel = __shfl_sync(0xffffffffu, s_sel, 0);
    if (s_sel == -2) {
        hint = -1;
        return false;
    }
    if (s_sel < 0) {
        int bj = 0x7fffffff, bs = -1;
        for (int k = lane; k < G; k += 32) {
            if (!slot_has_items(W_, k)) continue;
            const int jj = *(volatile const int*)&W_.slot_j[k];
            if (jj < bj) { bj = jj; bs = k; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            const int os = __shfl_xor_sync(0xffffffffu, bs, o);
            if (oj < bj || (oj == bj && os < bs)) { bj = oj; bs = os; }
        }
        s_sel = bs;
    }
    if (s_sel < 0) {
        hint = -1;
        return false;
    }
    int item = -1, j = 0, kind = 0, stY = 0;
    if (lane == 0) {
        const unsigned long long old = atom_add_acquire_u64(&W_.slot_word[s_sel], 1ull);
        if ((old >> 32) & 1ull) {
            const int nx = (int)(old & 0xFFFFFFFFull);
            const int n = *(volatile const int*)&W_.slot_n[s_sel];
            if (nx < n) {
                item = nx;
                j = *(volatile const int*)&W_.slot_j[s_sel];
                kind = *(volatile const int*)&W_.slot_kind[s_sel];
                stY = W_.start[j].y;
                // the claimer of the last item takes the task off the open count
                if (nx + 1 == n) atomicSub(&W_.ctl->open_tasks, 1);
            }
        }
    }
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item < 0) {
        hint = -1;
        return false;
    }
    hint = s_sel;
    j = __shfl_sync(0xffffffffu, j, 0);
    kind = __shfl_sync(0xffffffffu, kind, 0);
    stY = __shfl_sync(0xffffffffu, stY, 0);
    float e0, e1;
    const bool did = process_item<S>(A, win, j, stY, kind, item, e0, e1);
    __syncwarp();
    if (lane == 0) {
        if (did && kind == 0) {
            atomicAdd(&W_.slot_e0[s_sel], (unsigned long long)to_fixed(e0));
            atomicAdd(&W_.slot_e1[s_sel], (unsigned long long)to_fixed(e1));
        }
        // release: this warp's writes (shadow planes, Theta, E, sums) are visible to whoever
        // observes the count
        red_release_add(&W_.slot_fin[s_sel], 1);
    }
    __syncwarp();
    return true;
}

// Run the items of one task of component j. Small tasks stay inside the CTA; larger ones are
// published in the CTA's slot so idle warps anywhere in the grid can take items. Returns the
// (fixed-point) sums of a trial in e0/e1. False on an exhausted wait.
template <int S>
__device__ bool run_task(const TrialArgs& A, float4* win, int j, int stY, int nu, int kind,
                         int nitems, int G, unsigned long long* s_e0, unsigned long long* s_e1,
                         int* s_flag, unsigned long long t0) {
    const JointWs& W_ = A.ws;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int nwarps = kTrialThreads / 32;
    const int own = blockIdx.x;
    if (nitems <= nwarps) {
        for (int t = warp; t < nitems; t += nwarps) {
            float e0, e1;
            const bool did = process_item<S>(A, win, j, stY, kind, t, e0, e1);
            if (did && kind == 0 && lane == 0) {
                atomicAdd(s_e0, (unsigned long long)to_fixed(e0));
                atomicAdd(s_e1, (unsigned long long)to_fixed(e1));
            }
        }
        __syncthreads();
        return true;
    }
    if (tid == 0) {
        const unsigned long long e = W_.slot_word[own] >> 32;  // even: closed
        W_.slot_j[own] = j;
        W_.slot_n[own] = nitems;
        W_.slot_nu[own] = nu;
        W_.slot_kind[own] = kind;
        W_.slot_e0[own] = 0ull;
        W_.slot_e1[own] = 0ull;
        W_.slot_fin[own] = 0;
        atomicAdd(&W_.ctl->open_tasks, 1);
        __threadfence();
        atomicExch(&W_.slot_word[own], (e + 1ull) << 32);  // open, next item 0
        *s_flag = 0;
    }
    __syncthreads();
    // every decision below is warp-uniform (lane 0 reads, all lanes follow), so the warp-wide
    // shuffles inside help_one always run with the full warp
    int hint = -1;
    for (;;) {
        int fin = 0;
        if (lane == 0) fin = ld_acquire(&W_.slot_fin[own]) >= nitems;
        if (__shfl_sync(0xffffffffu, fin, 0)) break;
        if (!help_one<S>(A, win, own, G, hint)) __nanosleep(100);
        if (warp_should_abort(A.ws.ctl, t0)) {
            if (lane == 0) *s_flag = 1;
            break;
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (kind == 0) {
            *s_e0 = ld_volatile_u64(&W_.slot_e0[own]);
            *s_e1 = ld_volatile_u64(&W_.slot_e1[own]);
        }
        const unsigned long long w = W_.slot_word[own] >> 32;
        atomicExch(&W_.slot_word[own], (w + 1ull) << 32);  // closed
    }
    __syncthreads();
    return *s_flag == 0;
}

template <int S>
__global__ void __launch_bounds__(kTrialThreads, 3) k_trials(const TrialArgs A) {
    constexpr int r = (S - 1) / 2;
    constexpr int NB = (2 * r + 1) * (2 * r + 1);  // blocks within r of one LR pixel
    constexpr int kPend = 512;
    JointCtl* ctl = A.ws.ctl;
    if (!is_active(ctl)) return;
    __shared__ float4 wins[kTrialThreads / 32][S * S];
    __shared__ int s_j, s_nu, s_accept, s_flag, s_npend, s_povf;
    __shared__ int s_pend[kPend];
    __shared__ unsigned long long s_e0, s_e1;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int G = gridDim.x;
    const int M = ctl->M_cur;
    const int D = A.strict ? 2 * r : r;
    const int ND = (2 * D + 1) * (2 * D + 1);
    const JointWs& W_ = A.ws;
    float4* win = wins[warp];
    const unsigned long long t0 = now_ns();

    for (;;) {
        if (tid == 0) {
            s_j = atomicAdd(&ctl->claim[A.it], 1);
            s_nu = 0;
            s_e0 = 0;
            s_e1 = 0;
            s_flag = 0;
            s_npend = 0;
            s_povf = 0;
        }
        __syncthreads();
        const int j = s_j;
        if (j >= M) break;
        GLU_TRACE(A.it, j, 0);
        const int2 st = W_.start[j], en = W_.start[j + 1];

        // 1. the earlier components whose LR blocks lie within D of ours and are not done yet
        const int npairs = (en.y - st.y) * ND;
        for (int t = tid; t < npairs; t += kTrialThreads) {
            const int q = W_.qlist[st.y + t / ND];
            const int nb = t % ND;
            const int bv = q / A.w + nb / (2 * D + 1) - D, bu = q % A.w + nb % (2 * D + 1) - D;
            if (bv < 0 || bv >= A.h || bu < 0 || bu >= A.w) continue;
            const int64_t b = (int64_t)bv * A.w + bu;
            if (__ldcg(&W_.ovf[b])) {
                s_povf = 1;  // more components than owner slots: wait for every earlier one
                continue;
            }
            for (int k = 0; k < kOwnSlots; ++k) {
                const int i = __ldcg(&W_.own[b * kOwnSlots + k]);
                if (i < 0) break;
                if (i < j && ld_acquire(&W_.done[i]) == 0) {
                    const int slot = atomicAdd(&s_npend, 1);
                    if (slot < kPend) s_pend[slot] = i; else s_povf = 1;
                }
            }
        }
        __syncthreads();
        if (s_povf) {
            // rare fallback: wait in order for every earlier component
            for (int i = tid; i < j; i += kTrialThreads)
                if (!wait_done(W_.done, i, ctl)) s_flag = 1;
        } else {
            // wait, helping other components' tasks meanwhile; the loop decisions are
            // CTA-uniform (__syncthreads_or)
            const int np = min(s_npend, kPend);
            int hint = -1;
            for (;;) {
                int mine = 0;
                for (int t = tid; t < np; t += kTrialThreads) {
                    const int i = s_pend[t];
                    if (i >= 0) {
                        if (ld_acquire(&W_.done[i]) != 0) s_pend[t] = -1; else mine = 1;
                    }
                }
                if (__syncthreads_or(mine) == 0) break;
                if (!help_one<S>(A, win, blockIdx.x, G, hint)) __nanosleep(200);
                const int abort = warp_should_abort(ctl, t0) ? 1 : 0;
                if (__syncthreads_or(abort)) {
                    if (tid == 0) s_flag = 1;
                    break;
                }
            }
        }
        __syncthreads();
        __threadfence();
        if (s_flag) {
            if (tid == 0) {
                set_status(GLU_ERR_TIMEOUT);
                atomicExch(&ctl->timeout, 1);
                st_release(&W_.done[j], 1);  // never leave a later component waiting on us
                atomicAdd(&ctl->finished[A.it], 1);
            }
            __syncthreads();
            continue;
        }
        GLU_TRACE(A.it, j, 1);

        // 2. the distinct LR blocks Q of the component (stamps drop duplicates)
        const unsigned long long tagQ = trial_tag(A.it, j, 0);
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
        __threadfence();
        __syncthreads();

        // 5. trial: Algorithm 1 again on the affected pixels (STRICT: every block within r of
        //    Q; PAPER: the component's own pixels) into the shadow planes, summing e0 and e1
        const int nitems = A.strict ? nu * NB : nu;
        bool ok = run_task<S>(A, win, j, st.y, nu, 0, nitems, G, &s_e0, &s_e1, &s_flag, t0);
        if (tid == 0) s_accept = !(s_e1 > s_e0);
        __syncthreads();
        GLU_TRACE(A.it, j, 2);
        // 6. keep (nothing to do: the results are in place) or roll back: restore Theta and E
        //    from the backup planes and the LR colours from their backups
        if (!s_accept && ok) {
            ok = run_task<S>(A, win, j, st.y, nu, 1, nitems, G, &s_e0, &s_e1, &s_flag, t0);
            for (int t = tid; t < nu; t += kTrialThreads) {
                const int q = W_.ulist[st.y + t];
                store_rgb(A.lr, A.lr_pitch, q / A.w, q % A.w, W_.backup[q]);
            }
        }
        __syncthreads();
        if (tid == 0) {
            if (!ok) {
                set_status(GLU_ERR_TIMEOUT);
                atomicExch(&ctl->timeout, 1);
            }
            __threadfence();
            W_.dlog[(int64_t)A.it * W_.mcap + j] = (int8_t)(s_accept ? 1 : 0);
            if (s_accept) atomicAdd(&ctl->accepted[A.it], 1);
            else atomicAdd(&ctl->rolled[A.it], 1);
            st_release(&W_.done[j], 1);
            atomicAdd(&ctl->finished[A.it], 1);
        }
        GLU_TRACE(A.it, j, 3);
        __syncthreads();
    }
    // no component left to claim: help the running ones until every component is done
    // (per warp; lane 0 decides)
    const int lane = tid & 31;
    int hint = -1;
    for (;;) {
        int fin = 0;
        if (lane == 0) fin = *(volatile const int*)&ctl->finished[A.it] >= M;
        if (__shfl_sync(0xffffffffu, fin, 0)) break;
        if (!help_one<S>(A, win, blockIdx.x, G, hint)) __nanosleep(200);
        if (warp_should_abort(ctl, t0)) break;
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
    int grid = sm_count() * blocks_per_sm;
    if (grid > kMaxSlots) grid = kMaxSlots;
    k_trials<S><<<grid, kTrialThreads, 0, st>>>(A);
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
    k_ctl_init<<<grid_cap(nl > kMaxSlots ? nl : kMaxSlots, T), T, 0, st>>>(ws.ctl, ws.stamp, nl,
                                                                          ws.slot_word);
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

#ifdef GLU_TRIAL_TRACE
extern "C" int glu_dbg_trace(unsigned long long* host, int64_t n) {
    const size_t bytes = sizeof(unsigned long long) * (size_t)n;
    if (bytes > sizeof(glu::g_trace)) return GLU_ERR_INVALID_ARG;
    return cudaMemcpyFromSymbol(host, glu::g_trace, bytes) == cudaSuccess ? GLU_OK : GLU_ERR_CUDA;
}
#endif

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
