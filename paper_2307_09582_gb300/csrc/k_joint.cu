// Algorithm 2 (Sec. 3.3): joint optimisation of the downsampled image and Theta, for a batch of
// images (a single image is a batch of one).
//
// The images of a batch share one global HR pixel index space and one global LR index space
// (image after image, raster order inside each). Per iteration n (all launched up front; every
// kernel returns at once when device-side flags say every image has converged, so the host
// never waits in the middle, and a repeated call is replayed as a CUDA graph):
//   threshold   E_p > tau marks the large-error set of every still-active image; union-find
//               labels (parent pointers only ever decrease, so every component's root is its
//               smallest global index, i.e. its smallest raster index inside its image); the
//               set's pixels are compacted in raster order and later passes visit only them
//   merge/flat  8- (or 4-) connected unions inside each image, then every pixel points at its root
//   roots       ordered stream compaction of the roots: component j = the j-th smallest root
//   buckets     pixels and distinct LR blocks per component (counts, exclusive scan, fill)
//   graph       trial j must follow trial i < j exactly when an LR block of i lies within D of
//               one of j (D = 2r STRICT, r PAPER): those are the trials that read or write state
//               j reads or writes. Per component: the number of such predecessors and, per
//               component, the list of its successors
//   trials      persistent kernel over a ready queue: a component whose predecessors have all
//               finished is tried by one CTA (small components: entirely in shared memory; large
//               ones: block items shared with idle warps of the grid); its commit releases its
//               successors, continuing with the first it made ready. Trials that run at the same
//               time touch disjoint state, so the result equals the sequential order. Waits are
//               bounded (GLU_ERR_TIMEOUT) and cannot deadlock (edges only go from lower to
//               higher indices)
//   residual    R_n = sum_p E_p per image, exact in units of 2^-32 (64-bit integer sum of every
//               E_p rounded to a multiple of 2^-32); an image stops when its set is empty, when
//               no trial was kept, or when R_n >= R_{n-1}.
// Trial sums e0 / e1 use the same arithmetic: every pixel's error rounded to a multiple of 2^-32,
// added as 64-bit integers, so they are exact and independent of the order blocks finish in, and
// R_n = R_{n-1} + sum over the kept trials of (e1 - e0) holds exactly: only R_0 needs a pass over
// the image; the kept trials add their differences to the running residual.
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <atomic>
#include <memory>
#include <mutex>

#include "internal.h"
#include "search.cuh"
#include "tune.h"

namespace glu {

GLU_DEFINE_STATUS(joint)

constexpr int kOwnSlots = 8;        // components recorded per LR pixel before overflow
constexpr int kScanTile = 4096;     // elements per scan tile
constexpr int kScanThreads = 256;   // 16 elements per thread
constexpr int kTrialThreads = 1024;
constexpr int kResidChunk = 8192;
constexpr int kMaxSlots = 4096;
// The general path's affected blocks, listed per task slot for the first kListSlots slots (up to
// kSlotA blocks each); other tasks enumerate (block, neighbour) items and skip the ones they do
// not own.
constexpr int kListSlots = 256;
constexpr int kSlotA = 2048;
constexpr int kSmax = 9;            // largest window

// One image of a batch.
struct JImg {
    const uint8_t* hr;
    int64_t hr_pitch;
    uint8_t* lr;
    int64_t lr_pitch;
    uint16_t* code;
    void* weight;
    float* err;
    int H, W, h, w, s, S;
    int64_t p0, q0;   // first global HR / LR index
    int c0;           // first residual chunk
};

struct JBatch {
    JImg im[kMaxJointBatch];
    int n, wfmt, strict, conn;
    float eps255, tau;
    int64_t np, nq;
    int nchunks;
};

__device__ __forceinline__ int img_of_p(const JBatch& B, int64_t p) {
    int i = 0;
    while (i + 1 < B.n && B.im[i + 1].p0 <= p) ++i;
    return i;
}

struct JointCtl {
    int active_any;
    int timeout;
    int M_cur;
    int nfg;          // large-error pixels of the current iteration (all active images)
    int open_tasks;
    int small_cur;    // 1: the one-CTA list kernel built this iteration's components and graph
    int nedge;        // dependency edges listed by k_deps in the current iteration
    int multi_lists;  // bit n: iteration n's lists were built by the multi-kernel path
    int claim[GLU_MAX_ITERS];
    int finished[GLU_MAX_ITERS];
    int head[GLU_MAX_ITERS];      // ready queue: positions taken
    int tail[GLU_MAX_ITERS];      // ready queue: positions filled
    int dag_bad[GLU_MAX_ITERS];   // dependency graph did not fit: claim in index order instead
    int active[kMaxJointBatch];
    int iterations[kMaxJointBatch];
    int n_large[kMaxJointBatch][GLU_MAX_ITERS];
    int M[kMaxJointBatch][GLU_MAX_ITERS];
    int accepted[kMaxJointBatch][GLU_MAX_ITERS];
    int rolled[kMaxJointBatch][GLU_MAX_ITERS];
    unsigned long long searched[kMaxJointBatch][GLU_MAX_ITERS];
    double residual[kMaxJointBatch][GLU_MAX_ITERS + 1];
    unsigned long long racc[kMaxJointBatch];   // residual accumulators (2^-32 units)
};

struct JointWs {
    JointCtl* ctl;
    float* err;             // np: error planes of images whose caller passed no error map
    int* lab;               // np: -1, union-find parent, then component id
    uint8_t* qflag;         // np: pixel represents its (component, LR block) pair
    int* roots;             // mcap
    int* comp_pix;          // np
    int* qlist;             // np
    int* ulist;             // np
    int2* cnt;              // mcap: (pixels, LR blocks)
    int2* fill;             // mcap
    int2* start;            // mcap + 1
    int* done;              // mcap
    int* tile_a;            // tiles over np
    uint32_t* tcnt;             // tiles over np (padded to 4): large-error pixels per threshold tile
    uint32_t* tbits;            // tiles over np x kScanTile / 32: the threshold tiles' ballots
    int2* tile_b;           // tiles over mcap
    int* own;               // nq * kOwnSlots
    uint8_t* ovf;           // nq
    unsigned long long* stamp;  // nq
    int* bown;              // nq: the item that re-searches an affected block (general path)
    unsigned long long* best;   // nq
    uint32_t* backup;       // nq
    int8_t* dlog;           // N * mcap: kept (1) / rolled back (0) per component and iteration
    int64_t mcap;
    uint16_t* sh_code;      // np: Theta / E before a trial, restored if it is rolled back
    float* sh_w;            // np
    float* sh_err;          // np
    // one task slot per persistent CTA: the block items of its component's trial or rollback,
    // open to every warp of the grid
    unsigned long long* slot_word;  // (epoch << 32) | next item; odd epoch = open
    // (component j, items, image * 4 + kind, j's LR list offset); kind bit 0: rollback (else
    // trial), bit 1: items from the slot's A list
    int4* slot_info;
    unsigned long long* slot_e0;
    unsigned long long* slot_e1;
    int* slot_fin;          // items finished
    int* alist;             // kListSlots * kSlotA: per slot, the LR blocks its task re-searches
    // dependency graph of the iteration's trials: succ lists (CSR) and pending-predecessor counts
    int2* dag_cnt;          // mcap: (successors, unused)
    int2* dag_start;        // mcap + 1
    int* dag_fill;          // mcap
    int* pend;              // mcap: predecessors not yet finished
    int* queue;             // mcap: ready components in the order they became ready (-1: not yet)
    int* succ;              // ecap
    int64_t ecap;
};

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// 8-connected components of single pixels are at most ceil(H/2)*ceil(W/2) per image, 4-connected
// at most ceil(H*W/2) (checkerboard); summed over a batch, (np + n) / 2 bounds both.
static inline int64_t mcap_of(int64_t np, int n) { return (np + n) / 2 + 1; }

// Carve the workspace; returns the bytes needed (base may be null to only measure).
static size_t carve(void* base, int64_t np, int64_t nq, int nimg, int N, int64_t nchunks,
                    JointWs* o) {
    const int64_t mcap = mcap_of(np, nimg);
    const int64_t tiles_a = (np + kScanTile - 1) / kScanTile + 1;
    const int64_t tiles_b = (mcap + kScanTile - 1) / kScanTile + 1;
    size_t off = 0;
    char* b = (char*)base;
    auto take = [&](size_t bytes) -> void* {
        void* p = b ? (void*)(b + off) : nullptr;
        off = align256(off + bytes);
        return p;
    };
    JointWs t;
    t.ctl = (JointCtl*)take(sizeof(JointCtl));
    t.err = (float*)take(sizeof(float) * np);
    t.lab = (int*)take(sizeof(int) * np);
    t.qflag = (uint8_t*)take(np);
    t.roots = (int*)take(sizeof(int) * mcap);
    t.comp_pix = (int*)take(sizeof(int) * np);
    t.qlist = (int*)take(sizeof(int) * np);
    t.ulist = (int*)take(sizeof(int) * np);
    t.cnt = (int2*)take(sizeof(int2) * mcap);
    t.fill = (int2*)take(sizeof(int2) * mcap);
    t.start = (int2*)take(sizeof(int2) * (mcap + 1));
    t.done = (int*)take(sizeof(int) * mcap);
    t.tile_a = (int*)take(sizeof(int) * tiles_a);
    t.tcnt = (uint32_t*)take(sizeof(uint32_t) * (size_t)((tiles_a + 3) & ~(int64_t)3));
    t.tbits = (uint32_t*)take(sizeof(uint32_t) * (size_t)tiles_a * (kScanTile / 32));
    t.tile_b = (int2*)take(sizeof(int2) * tiles_b);
    t.own = (int*)take(sizeof(int) * nq * kOwnSlots);
    t.ovf = (uint8_t*)take(nq);
    t.stamp = (unsigned long long*)take(sizeof(unsigned long long) * nq);
    t.bown = (int*)take(sizeof(int) * nq);
    t.best = (unsigned long long*)take(sizeof(unsigned long long) * nq);
    t.backup = (uint32_t*)take(sizeof(uint32_t) * nq);
    t.dlog = (int8_t*)take((size_t)(N > 0 ? N : 1) * (size_t)mcap);
    t.mcap = mcap;
    t.sh_code = (uint16_t*)take(sizeof(uint16_t) * np);
    t.sh_w = (float*)take(sizeof(float) * np);
    t.sh_err = (float*)take(sizeof(float) * np);
    t.slot_word = (unsigned long long*)take(sizeof(unsigned long long) * kMaxSlots);
    t.slot_info = (int4*)take(sizeof(int4) * kMaxSlots);
    t.slot_e0 = (unsigned long long*)take(sizeof(unsigned long long) * kMaxSlots);
    t.slot_e1 = (unsigned long long*)take(sizeof(unsigned long long) * kMaxSlots);
    t.slot_fin = (int*)take(sizeof(int) * kMaxSlots);
    t.alist = (int*)take(sizeof(int) * kListSlots * kSlotA);
    t.ecap = std::min<int64_t>(2 * mcap + (1 << 20), (int64_t)1 << 30);
    t.dag_cnt = (int2*)take(sizeof(int2) * mcap);
    t.dag_start = (int2*)take(sizeof(int2) * (mcap + 1));
    t.dag_fill = (int*)take(sizeof(int) * mcap);
    t.pend = (int*)take(sizeof(int) * mcap);
    t.queue = (int*)take(sizeof(int) * mcap);
    t.succ = (int*)take(sizeof(int) * t.ecap);
    if (o) *o = t;
    return off;
}

// Sizes of a batch: global pixel / LR counts and residual chunks.
static void batch_sizes(const JointItem* items, int n, int64_t* np, int64_t* nq, int64_t* nch) {
    *np = 0;
    *nq = 0;
    *nch = 0;
    for (int k = 0; k < n; ++k) {
        const int64_t a = (int64_t)items[k].H * items[k].W;
        const int h = (items[k].H + items[k].s - 1) / items[k].s;
        const int w = (items[k].W + items[k].s - 1) / items[k].s;
        *np += a;
        *nq += (int64_t)h * w;
        *nch += (a + kResidChunk - 1) / kResidChunk;
    }
}

size_t joint_batch_workspace_bytes(const JointItem* items, int n, int N) {
    int64_t np, nq, nch;
    batch_sizes(items, n, &np, &nq, &nch);
    return carve(nullptr, np, nq, n, N, nch, nullptr);
}

size_t joint_workspace_bytes(int H, int W, int s, int S, int N) {
    JointItem it{};
    it.H = H;
    it.W = W;
    it.s = s;
    it.S = S;
    return joint_batch_workspace_bytes(&it, 1, N);
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

// Fetch-and-add with release and acquire semantics at GPU scope: the writes ordered before it
// (including other threads' writes ordered by a barrier) are visible to whoever observes the
// result, and the writes released by earlier updates of *p are visible after it.
__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
                 : "memory");
    return old;
}

__device__ __forceinline__ bool any_active(const JointCtl* c) {
    return *(volatile const int*)&c->active_any != 0;
}

// The list passes of the multi-kernel path run only when the one-CTA kernel (k_small_comp) did
// not already build this iteration's components and dependency graph.
__device__ __forceinline__ bool skip_lists(const JointCtl* c) {
    return !any_active(c) || *(volatile const int*)&c->small_cur != 0;
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

// Block-wide exclusive scan of one int per thread for any blockDim.x <= 1024 (a multiple of 32).
// Returns the total; smem_warp holds 32 ints.
__device__ __forceinline__ int block_excl_scan_any(int v, int* out_excl, int* smem_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        smem_warp[lane] = t;
    }
    __syncthreads();
    *out_excl = (wid > 0 ? smem_warp[wid - 1] : 0) + x - v;
    const int total = smem_warp[nw - 1];
    __syncthreads();
    return total;
}

// Warp-wide sum of a 64-bit integer (fixed butterfly; integer addition is exact).
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sums (blockDim.x a multiple of 32, at most 8 warps): every thread gets the total, added
// in a fixed order, so the result does not depend on timing.
__device__ __forceinline__ long long block_sum_ll(long long v, long long* smem_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_ll(v);
    if (lane == 0) smem_warp[wid] = v;
    __syncthreads();
    long long t = 0;
    for (int k = 0; k < nw; ++k) t += smem_warp[k];
    __syncthreads();
    return t;
}
__device__ __forceinline__ int block_sum_int(int v, int* smem_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) smem_warp[wid] = v;
    __syncthreads();
    int t = 0;
    for (int k = 0; k < nw; ++k) t += smem_warp[k];
    __syncthreads();
    return t;
}

// Verification log (test hook, null: off): log[0].x counts records, records from log[1], at most
// cap of them. Kinds: (iteration, component, LR pixel, HR pixel) for a trial's replacement
// choice; (256 + iteration, HR pixel, membership, 0) for a pixel whose FP32 error is within
// kThrLogBand of tau at the threshold pass (indices inside the pixel's image).
constexpr float kThrLogBand = 1e-5f;
__device__ __forceinline__ void log_record(int4* log, long long cap, int4 rec) {
    if (!log) return;
    const int pos = atomicAdd(&log[0].x, 1);
    if (pos < cap) log[1 + pos] = rec;
}

// ---------------------------------------------------------------- control and init kernels

// Every counter of the control block starts at zero, except the active flags of the nimg
// images and active_any; stamps and task slots are cleared.
__global__ void k_ctl_init(JointCtl* c, unsigned long long* stamp, int64_t nq,
                           unsigned long long* slot_word, int nimg, uint32_t* tcnt,
                           int64_t ntcnt) {
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = i0; i < kMaxSlots; i += stride) slot_word[i] = 0ull;
    for (int64_t i = i0; i < ntcnt; i += stride) tcnt[i] = 0u;
    for (int64_t i = i0; i < nq; i += stride) stamp[i] = 0ull;
    int* ci = (int*)c;
    constexpr int nwords = (int)(sizeof(JointCtl) / sizeof(int));
    constexpr int w_any = (int)(offsetof(JointCtl, active_any) / sizeof(int));
    constexpr int w_act = (int)(offsetof(JointCtl, active) / sizeof(int));
    for (int64_t i = i0; i < nwords; i += stride)
        ci[i] = (i == w_any || (i >= w_act && i < w_act + nimg)) ? 1 : 0;
}

// Batched regular grid downsampling (uint8): LR pixel (v, u) copies HR pixel
// (v*s + e_y/2, u*s + e_x/2), e = extent of the block.
__global__ void k_grid_batch(const __grid_constant__ JBatch B) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < B.nq;
         g += (int64_t)gridDim.x * blockDim.x) {
        int i = 0;
        while (i + 1 < B.n && B.im[i + 1].q0 <= g) ++i;
        const JImg& I = B.im[i];
        const int64_t lq = g - I.q0;
        const int v = (int)(lq / I.w), u = (int)(lq % I.w);
        const int ey = min(I.s, I.H - v * I.s), ex = min(I.s, I.W - u * I.s);
        const uint8_t* src =
            I.hr + (int64_t)(v * I.s + ey / 2) * I.hr_pitch + (int64_t)(u * I.s + ex / 2) * 3;
        uint8_t* dst = I.lr + (int64_t)v * I.lr_pitch + (int64_t)u * 3;
        dst[0] = src[0];
        dst[1] = src[1];
        dst[2] = src[2];
    }
}

// Residual R = sum_p E_p per image. Each E_p is rounded to a multiple of 2^-32 and the
// multiples are added as 64-bit integers: the sum is exact and independent of the order the
// CTAs add their chunks in (E_p <= sqrt(3), so 2^31 pixels cannot overflow), and its error
// against the real-valued sum (at most 2^-33 per pixel, unbiased) is far below that of a plain
// FP64 accumulation. The result is converted to FP64 once. A CTA per chunk of one image.
__global__ void k_resid_partial(const __grid_constant__ JBatch B, JointCtl* c) {
    if (!any_active(c)) return;
    __shared__ unsigned long long sm[8];
    const int chunk = blockIdx.x;
    int i = 0;
    while (i + 1 < B.n && B.im[i + 1].c0 <= chunk) ++i;
    if (!c->active[i]) return;   // uniform across the CTA
    const JImg& I = B.im[i];
    const int64_t n = (int64_t)I.H * I.W;
    const int64_t base = (int64_t)(chunk - I.c0) * kResidChunk;
    unsigned long long acc = 0ull;
    for (int k = threadIdx.x; k < kResidChunk; k += 256) {
        const int64_t p = base + k;
        if (p < n) acc += __float2ull_rn(__ldcg(&I.err[p]) * 4294967296.0f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0ull;
        for (int w = 0; w < 8; ++w) t += sm[w];
        atomicAdd(&c->racc[i], t);
    }
}

// it < 0: initial residuals R_0 (the accumulators hold k_resid_partial's sums). Otherwise finish
// iteration it for every active image: the accumulator holds R_{it} + the kept trials' (e1 - e0),
// i.e. R_{it+1} exactly; record it and decide whether the image stops. An image whose
// large-error set was empty stops without counting the iteration (Algorithm 2 breaks before any
// trial).
__global__ void k_resid_final(const __grid_constant__ JBatch B, JointCtl* c, int it) {
    if (!any_active(c) || threadIdx.x != 0) return;
    if (it >= 0 && !c->small_cur) c->multi_lists |= 1 << it;
    for (int i = 0; i < B.n; ++i) {
        if (!c->active[i]) continue;
        const double R = (double)c->racc[i] * (1.0 / 4294967296.0);
        if (it < 0) {
            c->residual[i][0] = R;
        } else if (c->M[i][it] == 0) {
            c->active[i] = 0;
        } else {
            c->residual[i][it + 1] = R;
            c->iterations[i] = it + 1;
            if (c->accepted[i][it] == 0 || !(R < c->residual[i][it])) c->active[i] = 0;
        }
    }
    if (it >= 0) {
        int any = 0;
        for (int i = 0; i < B.n; ++i) any |= c->active[i];
        c->active_any = any;
    }
}

// ----------------------------------------------------------------------- threshold and CCL

// Large-error set of the active images, its bitmap and its ordered list, in two passes
// over tiles of kScanTile pixels (16 per thread, in rounds of 256 consecutive pixels) with no
// waits between CTAs:
//   k_threshold_count  marks E_p > tau and stores the tile's ballots (one 32-bit word per warp
//                      and round: together a raster bitmap of the large-error set, bit p of word
//                      p / 32) and its count; iteration 0 (full_clear) also sets the label of
//                      every pixel outside the set to -1 and clears the owner slots (later
//                      iterations find them cleared by k_lists_clear, which resets only the
//                      previous lists' pixels and blocks); the large-error pixels' labels are
//                      written by the component kernels
//   k_threshold_write  adds up the counts of the tiles before its own (a fixed-order block sum
//                      over at most a few thousand L2-resident integers) and writes the tile's
//                      large-error pixels to the list in raster order from the stored ballots
// The counts end in the last tile, which records the list's length.
__global__ void __launch_bounds__(kScanThreads)
    k_threshold_count(const __grid_constant__ JBatch B, JointWs W, int it, int full_clear,
                      int4* vlog, long long vcap) {
    JointCtl* c = W.ctl;
    if (!any_active(c)) return;
    constexpr int kRounds = kScanTile / kScanThreads;   // 256 consecutive pixels per round
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int wsm[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    if (tile == 0 && tid == 0) {   // a new iteration's lists
        c->small_cur = 0;
        c->nedge = 0;
    }
    const int64_t base = (int64_t)tile * kScanTile;
    // a tile inside one image (the usual case): all sixteen error loads issue together, with no
    // per-pixel image lookup in front of them
    const int i0 = img_of_p(B, base);
    const bool one = i0 + 1 >= B.n || B.im[i0 + 1].p0 >= base + kScanTile;
    const bool act0 = c->active[i0] != 0;
    float e1[kRounds];
    if (one) {
        const float* err = B.im[i0].err - B.im[i0].p0;
#pragma unroll
        for (int k = 0; k < kRounds; ++k) {
            const int64_t p = base + k * kScanThreads + tid;
            e1[k] = act0 && p < B.np ? err[p] : 0.f;
        }
    }
    int run_img = -1, run = 0, cnt = 0;
    unsigned fgm = 0u;   // bit k: this thread's pixel of round k is a large-error pixel
    uint32_t* tb = W.tbits + (int64_t)tile * (kRounds * kWarps);
    if (one && !vlog) {
        // the usual case: one image, no verification log
        const int pl = (int)base + tid;   // pixel ids fit in 31 bits
        const int np = (int)B.np;
#pragma unroll
        for (int k = 0; k < kRounds; ++k) {
            const bool in = pl + k * kScanThreads < np;
            const bool fg = act0 && in && e1[k] > B.tau;
            if (full_clear && in && !fg) W.lab[pl + k * kScanThreads] = -1;
            const unsigned bal = __ballot_sync(0xffffffffu, fg);
            if (lane == 0) tb[k * kWarps + warp] = bal;
            fgm |= fg ? 1u << k : 0u;
        }
        run = cnt = __popc(fgm);
    } else {
#pragma unroll
        for (int k = 0; k < kRounds; ++k) {
            const int64_t p = base + k * kScanThreads + tid;
            bool fg = false;
            if (p < B.np) {
                const int i = one ? i0 : img_of_p(B, p);
                if (one ? act0 : c->active[i] != 0) {
                    const float e = one ? e1[k] : B.im[i].err[p - B.im[i].p0];
                    fg = e > B.tau;
                    if (vlog && fabsf(e - B.tau) < kThrLogBand)
                        log_record(vlog, vcap,
                                   make_int4(256 + it, (int)(p - B.im[i].p0), fg ? 1 : 0, 0));
                }
                if (full_clear && !fg) W.lab[p] = -1;
                if (fg) {
                    if (i != run_img) {
                        if (run && !one) atomicAdd(&c->n_large[run_img][it], run);
                        run_img = i;
                        run = 0;
                    }
                    ++run;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, fg);
            if (lane == 0) tb[k * kWarps + warp] = bal;
            cnt += fg ? 1 : 0;
        }
    }
    // |E| per image (one atomic per CTA for a tile inside one image) and the tile's count
    if (one) {
        const int tot = block_sum_int(run, wsm);
        if (tid == 0) {
            if (tot) atomicAdd(&c->n_large[i0][it], tot);
            W.tcnt[tile] = (uint32_t)tot;
        }
    } else {
        if (run) atomicAdd(&c->n_large[run_img][it], run);
        const int tot = block_sum_int(cnt, wsm);
        if (tid == 0) W.tcnt[tile] = (uint32_t)tot;
    }
    if (full_clear) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + tid; q < B.nq; q += stride) {
#pragma unroll
            for (int k = 0; k < kOwnSlots; ++k) W.own[q * kOwnSlots + k] = -1;
            W.ovf[q] = 0;
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) k_threshold_write(JointWs W) {
    JointCtl* c = W.ctl;
    if (!any_active(c)) return;
    constexpr int kRounds = kScanTile / kScanThreads;
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int s_cnt[kRounds * kWarps];   // per (round, warp): offset within the tile
    __shared__ int wsm[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    // a tile without large-error pixels writes nothing (the last one still records the length)
    if (tile != (int)gridDim.x - 1 && __ldcg(&W.tcnt[tile]) == 0u) return;
    // the list offset of this tile: counts of the tiles before it (four per 16-byte load, the
    // loads of a thread issued together), summed in a fixed order
    constexpr int kCntPer = 4;   // 16-byte loads per thread and round
    int part = 0;
    const uint4* c4 = reinterpret_cast<const uint4*>(W.tcnt);
    for (int g0 = tid * kCntPer; g0 * 4 < tile; g0 += kScanThreads * kCntPer) {
        uint4 v[kCntPer];
#pragma unroll
        for (int k = 0; k < kCntPer; ++k)
            v[k] = (g0 + k) * 4 < tile ? __ldcg(&c4[g0 + k]) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int k = 0; k < kCntPer; ++k) {
            const int t = (g0 + k) * 4;
            part += (t < tile ? (int)v[k].x : 0) + (t + 1 < tile ? (int)v[k].y : 0) +
                    (t + 2 < tile ? (int)v[k].z : 0) + (t + 3 < tile ? (int)v[k].w : 0);
        }
    }
    const long long excl = block_sum_int(part, wsm);
    const uint32_t* bits = W.tbits + (int64_t)tile * (kRounds * kWarps);
    const int v = tid < kRounds * kWarps ? __popc(__ldcg(&bits[tid])) : 0;
    int ex;
    const int agg = block_excl_scan(v, &ex, wsm);
    if (tid < kRounds * kWarps) s_cnt[tid] = ex;
    __syncthreads();
    if (tid == 0 && tile == (int)gridDim.x - 1) {   // the last tile knows the list's length
        c->nfg = (int)(excl + agg);
        if (excl + agg == 0) c->active_any = 0;   // every large-error set is empty
    }
    const int64_t base = (int64_t)tile * kScanTile;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kRounds; ++k) {
        const unsigned bal = __ldcg(&bits[k * kWarps + warp]);
        if ((bal >> lane) & 1u)
            W.ulist[excl + s_cnt[k * kWarps + warp] + __popc(bal & lt)] =
                (int)(base + k * kScanThreads + tid);
    }
}

// After an iteration's trials: the labels of its large-error pixels back to -1 and the owner
// slots of the LR blocks its components touched cleared (everything else is still clear), so
// the next threshold pass writes only its own pixels.
__global__ void k_lists_clear(JointWs W) {
    JointCtl* c = W.ctl;
    if (!any_active(c)) return;
    const int M = c->M_cur;
    if (c->nfg <= 0 || M <= 0) return;
    const int2 tot = W.start[M];
    const int stride = gridDim.x * blockDim.x;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot.x; e += stride)
        W.lab[__ldcg(&W.comp_pix[e])] = -1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot.y; e += stride) {
        const int64_t q = __ldcg(&W.qlist[e]);
#pragma unroll
        for (int k = 0; k < kOwnSlots; ++k) W.own[q * kOwnSlots + k] = -1;
        W.ovf[q] = 0;
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

// The same union-find on a CTA's shared-memory array.
__device__ __forceinline__ int suf_find(int* par, int x) {
    volatile int* vp = par;
    for (;;) {
        const int p = vp[x];
        if (p == x) return x;
        const int gp = vp[p];
        if (gp != p) atomicMin(&par[x], gp);
        x = p;
    }
}

__device__ __forceinline__ void suf_union(int* par, int a, int b) {
    for (;;) {
        a = suf_find(par, a);
        b = suf_find(par, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&par[a], b);
        if (old == a) return;
        a = old;
    }
}

// Components of the large-error set in two stages. Stage one (k_ccl_local): one warp per
// kCclTile x kCclTile tile of an image finds the components of the tile's own large-error
// pixels in shared memory, from the threshold pass's ballots (bit p of the raster bitmap is
// E_p > tau), and labels every large-error pixel with the smallest pixel of its tile component.
// Stage two (k_ccl_merge): the global union-find joins those labels across tile borders only.
// Rows and columns are read in raster order, so the smallest pixel of a tile component is its
// smallest global index and, after the merge, every component's root is its smallest pixel.
constexpr int kCclTile = 32;

// Neighbour rule of the border merge, for a large-error pixel with backward neighbours W, N
// (and NW, NE with 8-connectivity), each flag meaning "inside the image and large-error".
// With 8-connectivity a large-error N makes the other three redundant (W is joined to N as its
// NE neighbour, NW and NE as N's W and E neighbours, each when that pixel is handled), and a
// large-error W makes NW redundant (W's N): at most two unions per pixel. Bit 0: W, 1: N,
// 2: NW, 3: NE.
__device__ __forceinline__ unsigned ccl_edges(int conn, bool fw, bool fn, bool fnw, bool fne) {
    if (conn != 8) return (fw ? 1u : 0u) | (fn ? 2u : 0u);
    if (fn) return 2u;
    return (fw ? 1u : (fnw ? 4u : 0u)) | (fne ? 8u : 0u);
}

// One warp per tile, lane r holding row r's bits: the tile's runs (maximal horizontal
// segments, at most 16 per row) are the union-find's elements, numbered r * 16 + their order in
// the row, which is raster order of their first pixels; a run is joined to every run of the row
// above that touches it (8-connectivity: within one column to either side). With union by the
// smaller number, every tile component's root is its first run, whose first pixel is the
// component's smallest. Eight tiles side by side per CTA, no block-wide barrier: all tiles of a
// 4K image are resident at once.
constexpr int kCclRuns = kCclTile / 2;

__device__ __forceinline__ int ccl_run(unsigned starts, int r, int cl) {
    // the run holding column cl of a row whose run starts are `starts` (cl = 31: all bits)
    return r * kCclRuns + __popc(starts & ((2u << cl) - 1u)) - 1;
}

__global__ void __launch_bounds__(256) k_ccl_local(const __grid_constant__ JBatch B, JointWs W) {
    const JointCtl* c = W.ctl;
    const int i = blockIdx.z;
    const int iw = B.im[i].W, ih = B.im[i].H;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * 8 + warp) * kCclTile, y0 = blockIdx.y * kCclTile;
    if (x0 >= iw || y0 >= ih) return;
    const int64_t rowp = B.im[i].p0 + (int64_t)y0 * iw + x0;
    // the control words and the row's bitmap words in one round trip (the bitmap is read even
    // when the pass is skipped: it is always allocated)
    const int act_any = __ldcg(&c->active_any), small = __ldcg(&c->small_cur);
    const int act = __ldcg(&c->active[i]);
    unsigned m = 0u;
    if (y0 + lane < ih) {
        const int64_t p = rowp + (int64_t)lane * iw;
        const int64_t wd = p >> 5;
        const int sh = (int)(p & 31);
        const unsigned lo = __ldcg(&W.tbits[wd]);
        // the bits past the end of the batch are zero: the next word is needed only below it
        const unsigned hi = sh && (wd + 1) * 32 < B.np ? __ldcg(&W.tbits[wd + 1]) : 0u;
        m = __funnelshift_r(lo, hi, sh);
        const int wv = iw - x0;
        if (wv < kCclTile) m &= (1u << wv) - 1u;
    }
    if (!act_any || small || !act) return;
    if (!__any_sync(0xffffffffu, m != 0u)) return;
    __shared__ int par_s[8][kCclTile * kCclRuns];
    __shared__ uint8_t rstart_s[8][kCclTile * kCclRuns];   // first column of each run
    int* par = par_s[warp];
    uint8_t* rstart = rstart_s[warp];
    const unsigned st = m & ~(m << 1);   // first pixels of this row's runs
    {
        int j = 0;
        for (unsigned b = st; b; b &= b - 1, ++j) {
            par[lane * kCclRuns + j] = lane * kCclRuns + j;
            rstart[lane * kCclRuns + j] = (uint8_t)(__ffs(b) - 1);
        }
    }
    const unsigned up = __shfl_up_sync(0xffffffffu, m, 1);
    __syncwarp();
    if (lane > 0 && m && up) {
        const unsigned ust = up & ~(up << 1);
        int j = 0;
        for (unsigned b = st; b; b &= b - 1, ++j) {
            const int a = __ffs(b) - 1;
            const unsigned rest = m >> a;
            const int len = __ffs(~rest) ? __ffs(~rest) - 1 : 32 - a;   // run [a, a + len)
            const int lo = B.conn == 8 && a > 0 ? a - 1 : a;
            const int hi = B.conn == 8 ? min(a + len, kCclTile - 1) : a + len - 1;
            const unsigned span = (hi - lo == 31 ? 0xffffffffu : ((2u << (hi - lo)) - 1u)) << lo;
            const unsigned ov = up & span;
            // one union per run of the row above that touches this one
            for (unsigned t = ov & ~(ov << 1); t; t &= t - 1)
                suf_union(par, lane * kCclRuns + j, ccl_run(ust, lane - 1, __ffs(t) - 1));
        }
    }
    __syncwarp();
    // labels: each lane its own row's runs, every pixel of a run the root run's first pixel (the
    // finds of the lanes run together; a parent only decreases, so the forest stays valid)
    int j = 0;
    int* dst = W.lab + rowp + (int64_t)lane * iw;
    for (unsigned b = st; b; b &= b - 1, ++j) {
        const int a = __ffs(b) - 1;
        const unsigned rest = m >> a;
        const int len = __ffs(~rest) ? __ffs(~rest) - 1 : 32 - a;
        const int root = suf_find(par, lane * kCclRuns + j);
        const int g = (int)(rowp + (int64_t)(root / kCclRuns) * iw + rstart[root]);
        for (int k = 0; k < len; ++k) dst[a + k] = g;
    }
}

// Stage two: the edges of the neighbour rule that cross a tile border, through the global
// union-find (every large-error pixel's label is its tile component's root). Only pixels in a
// tile's first row or first or last column have such edges.
__global__ void k_ccl_merge(const __grid_constant__ JBatch B, int* lab, const int* fgl,
                            const JointCtl* c) {
    if (skip_lists(c)) return;
    const int nfg = c->nfg;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nfg; e += gridDim.x * blockDim.x) {
        const int64_t p = fgl[e];
        const JImg& I = B.im[img_of_p(B, p)];
        const int64_t lp = p - I.p0;
        const int y = (int)(lp / I.W), x = (int)(lp % I.W);
        const int r = y % kCclTile, cl = x % kCclTile;
        if (r != 0 && cl != 0 && cl != kCclTile - 1) continue;
        const int64_t up = p - I.W;
        const bool fw = x > 0 && __ldcg(&lab[p - 1]) >= 0;
        const bool fn = y > 0 && __ldcg(&lab[up]) >= 0;
        const bool fnw = B.conn == 8 && y > 0 && x > 0 && __ldcg(&lab[up - 1]) >= 0;
        const bool fne = B.conn == 8 && y > 0 && x + 1 < I.W && __ldcg(&lab[up + 1]) >= 0;
        const unsigned ed = ccl_edges(B.conn, fw, fn, fnw, fne);
        if ((ed & 1u) && cl == 0) uf_union(lab, (int)p, (int)p - 1);
        if ((ed & 2u) && r == 0) uf_union(lab, (int)p, (int)up);
        if ((ed & 4u) && (r == 0 || cl == 0)) uf_union(lab, (int)p, (int)up - 1);
        if ((ed & 8u) && (r == 0 || cl == kCclTile - 1)) uf_union(lab, (int)p, (int)up + 1);
    }
}

__global__ void k_ccl_flatten(int* lab, const int* fgl, const JointCtl* c) {
    if (skip_lists(c)) return;
    const int nfg = c->nfg;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nfg; e += gridDim.x * blockDim.x) {
        const int p = fgl[e];
        lab[p] = uf_find(lab, p);
    }
}

// -------------------------------------------------------------- roots: ordered compaction

// per-tile root counts over the large-error list (a root is a pixel that is its own parent)
__global__ void k_root_count(const int* lab, const int* fgl, int* tile_cnt, const JointCtl* c) {
    if (skip_lists(c)) return;
    __shared__ int wsum[8];
    const int nfg = c->nfg;
    // grid-stride over the list's tiles (a small grid: the list is short after iteration 1)
    for (int tile = blockIdx.x; tile * kScanTile < nfg; tile += gridDim.x) {
        const int base = tile * kScanTile;
        int local = 0;
        for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
            const int e = base + i;
            if (e < nfg) {
                const int p = fgl[e];
                if (lab[p] == p) ++local;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = local;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int i = 0; i < 8; ++i) t += wsum[i];
            tile_cnt[tile] = t;
        }
        __syncthreads();
    }
}

// single-CTA exclusive scan of tile counts in place; the total becomes nfg (OUT = 0) or M
// (OUT = 1); an empty large-error set stops every image
template <int OUT>
__global__ void k_tile_scan(int* tile_cnt, int ntiles, JointCtl* c) {
    if (skip_lists(c)) return;
    __shared__ int wsm[8];
    // the root counts cover only the list's tiles
    if (OUT == 1) ntiles = (c->nfg + kScanTile - 1) / kScanTile;
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
        if (OUT == 0) c->nfg = carry;
        else c->M_cur = carry;
        if (carry == 0) c->active_any = 0;  // every large-error set is empty: all images stop
    }
}

// scatter roots in global order; component j's per-iteration state is cleared here
__global__ void k_root_scatter(const __grid_constant__ JBatch B, const int* lab, const int* fgl,
                               const int* tile_off, int* roots, int2* cnt, int2* fill, int* done,
                               int2* dag_cnt, int* dag_fill, int* queue, JointCtl* c, int it) {
    if (skip_lists(c)) return;
    __shared__ int wsm[8];
    const int nfg = c->nfg;
    for (int tile = blockIdx.x; tile * kScanTile < nfg; tile += gridDim.x) {   // uniform
    const int base = tile * kScanTile;
    const int off = tile_off[tile];
    // 16 consecutive elements per thread keep the order inside the tile
    constexpr int per = kScanTile / kScanThreads;
    const int my = base + threadIdx.x * per;
    int flags = 0, cntl = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int e = my + k;
        bool r = false;
        if (e < nfg) {
            const int p = fgl[e];
            r = lab[p] == p;
        }
        flags |= (int)r << k;
        cntl += r;
    }
    int ex;
    (void)block_excl_scan(cntl, &ex, wsm);
    int j = off + ex;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        if ((flags >> k) & 1) {
            const int p = fgl[my + k];
            roots[j] = p;
            cnt[j] = make_int2(0, 0);
            fill[j] = make_int2(0, 0);
            done[j] = 0;
            dag_cnt[j] = make_int2(0, 0);
            dag_fill[j] = 0;
            queue[j] = -1;
            atomicAdd(&c->M[img_of_p(B, p)][it], 1);
            ++j;
        }
    }
    }
}

// ------------------------------------------------------------------- per-component buckets

// First index whose value exceeds key (a ascending), n if none.
__device__ __forceinline__ int upper_bound_i(const int* a, int n, int key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

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
__global__ void k_comp_count(const __grid_constant__ JBatch B, int* lab, const int* fgl,
                             const int* roots, int2* cnt, int* own, uint8_t* ovf, uint8_t* qflag,
                             const JointCtl* c) {
    if (skip_lists(c)) return;
    const int M = c->M_cur, nfg = c->nfg;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nfg; e += gridDim.x * blockDim.x) {
        const int64_t p = fgl[e];
        const int root = lab[p];
        const int j = lower_bound_i(roots, M, root);
        lab[p] = j;
        atomicAdd(&cnt[j].x, 1);
        const JImg& I = B.im[img_of_p(B, p)];
        const int64_t lp = p - I.p0;
        const int y = (int)(lp / I.W), x = (int)(lp % I.W);
        const int64_t q = I.q0 + (int64_t)(y / I.s) * I.w + (x / I.s);
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
    if (skip_lists(c)) return;
    const int M = c->M_cur;
    __shared__ int wx[8], wy[8];
    for (int tile = blockIdx.x; (int64_t)tile * kScanTile < M; tile += gridDim.x) {   // uniform
        const int64_t base = (int64_t)tile * kScanTile;
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
            tile_sum[tile] = make_int2(tx, ty);
        }
        __syncthreads();
    }
}

__global__ void k_comp_tile_scan(int2* tile_sum, const JointCtl* c) {
    if (skip_lists(c)) return;
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
    if (skip_lists(c)) return;
    const int M = c->M_cur;
    __shared__ int wsm[8];
    for (int tile = blockIdx.x; (int64_t)tile * kScanTile < M; tile += gridDim.x) {   // uniform
    const int64_t base = (int64_t)tile * kScanTile;
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
    int ox = tile_off[tile].x + ex, oy = tile_off[tile].y + ey;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        if (my + k < M) start[my + k] = make_int2(ox, oy);
        ox += v[k].x;
        oy += v[k].y;
        if (my + k == M - 1) start[M] = make_int2(ox, oy);
    }
    }
}

__global__ void k_comp_fill(const __grid_constant__ JBatch B, const int* lab, const int* fgl,
                            const uint8_t* qflag, const int2* start, int2* fill, int* comp_pix,
                            int* qlist, const JointCtl* c) {
    if (skip_lists(c)) return;
    const int nfg = c->nfg;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nfg; e += gridDim.x * blockDim.x) {
        const int64_t p = fgl[e];
        const int j = lab[p];
        const int pos = atomicAdd(&fill[j].x, 1);
        comp_pix[start[j].x + pos] = (int)p;
        if (qflag[p]) {
            const JImg& I = B.im[img_of_p(B, p)];
            const int64_t lp = p - I.p0;
            const int y = (int)(lp / I.W), x = (int)(lp % I.W);
            const int qp = atomicAdd(&fill[j].y, 1);
            qlist[start[j].y + qp] = (int)(I.q0 + (int64_t)(y / I.s) * I.w + (x / I.s));
        }
    }
}

#ifdef GLU_TRIAL_TRACE
// Debug builds only: per-component timestamps (claim, dependencies met, trial summed, done).
constexpr int kTraceMax = 1 << 15;
static __device__ unsigned long long g_trace[GLU_MAX_ITERS][kTraceMax][16];
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
#define GLU_TRACE(it, j, k) \
    do { if (tid == 0 && (j) < kTraceMax) g_trace[it][j][k] = gtimer(); } while (0)
#define GLU_TRACE_ANY(it, j, k) \
    do { if ((j) < kTraceMax) g_trace[it][j][k] = gtimer(); } while (0)
#else
#define GLU_TRACE(it, j, k) do { } while (0)
#define GLU_TRACE_ANY(it, j, k) do { } while (0)
#endif
#ifdef GLU_TRIAL_TRACE
// Debug builds only: per-warp stamps inside the one-CTA trials of iteration 0 (component,
// warp, [pass start, pass end, full-search start, full-search end, blocks, pixels queued]).
constexpr int kWTraceMax = 4096;
static __device__ unsigned long long g_wtrace[kWTraceMax][32][6];
#define GLU_WSTAMP(it, j, k) \
    do { if ((it) == 0 && (j) < kWTraceMax && (threadIdx.x & 31) == 0) \
        g_wtrace[j][threadIdx.x >> 5][k] = gtimer(); } while (0)
#define GLU_WVAL(it, j, k, v) \
    do { if ((it) == 0 && (j) < kWTraceMax && (threadIdx.x & 31) == 0) \
        g_wtrace[j][threadIdx.x >> 5][k] = (unsigned long long)(v); } while (0)
#else
#define GLU_WSTAMP(it, j, k) do { } while (0)
#define GLU_WVAL(it, j, k, v) do { } while (0)
#endif
#ifdef GLU_TRIAL_TRACE
// Debug builds only: per component of iteration 0, k_deps' [start, end, items, bitmap, CTA].
static __device__ unsigned long long g_deps_t[kTraceMax][5];
#endif
#ifdef GLU_TRIAL_TRACE
// Debug builds only: phase stamps of the one-CTA list kernel per iteration.
static __device__ unsigned long long g_small_t[GLU_MAX_ITERS][16];
#define GLU_SMALL_STAMP(it, k) \
    do { if (threadIdx.x == 0) g_small_t[it][k] = gtimer(); } while (0)
#else
#define GLU_SMALL_STAMP(it, k) do { } while (0)
#endif

// ------------------------------------------------------------ dependency graph of the trials
//
// Trial j reads and writes state within D LR pixels of its blocks Q_j (D = 2r STRICT: it re-runs
// Algorithm 1 on blocks within r of Q_j, whose windows reach r further; D = r PAPER). Component
// i < j must therefore finish before j starts exactly when some block of Q_i lies within D of a
// block of Q_j. k_deps finds those i for every j from the owner slots of the LR blocks around
// Q_j (or, for a block whose slots overflowed, from the labels of its pixels), removes
// duplicates, and builds: pend[j] = number of predecessors, succ lists (CSR) of every i. The
// trials then run any component whose predecessors have all finished, in any order: components
// that run concurrently never touch the same state, so the result equals the sequential one.

constexpr int kCandMax = 4096;   // predecessor candidates per component before the fallback

__device__ __forceinline__ void bitonic_sort_smem(int* a, int n2) {
    for (int k = 2; k <= n2; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int t = threadIdx.x; t < n2; t += blockDim.x) {
                const int u = t ^ jj;
                if (u > t) {
                    const int x = a[t], y = a[u];
                    const bool up = (t & k) == 0;
                    if ((x > y) == up) {
                        a[t] = y;
                        a[u] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// k_deps: per component j, pend[j] = the number of its distinct predecessors, every predecessor's
// successor count, and every (predecessor, j) edge appended to a scratch list; k_edge_scatter then
// writes the successor lists (CSR, after a scan of the counts) from that list and puts the
// components without predecessors in the ready queue. Distinct predecessors come from a
// shared-memory bitmap over component indices (one atomicOr per candidate) when M <= kDepsBits,
// else from a sorted candidate list.
constexpr int kDepsBits = 1 << 16;
// Neighbourhood bitmap of one component (dilated bounding box of its blocks), used above this
// many (block, neighbour) pairs.
constexpr int kNbBits = 1 << 15;
constexpr int kNbMinPairs = 256;
constexpr int kDepsWords = 256;   // bitmap words compacted per round (positions < 2^15: short)
static_assert(kNbBits <= 32768, "bitmap positions are stored as short");

// Multiplicative hash of a key into mask + 1 (a power of two) slots.
__device__ __forceinline__ int hash_slot(int key, int mask) {
    return (int)(((unsigned)key * 2654435761u) >> 13) & mask;
}

// The scratch list of dependency edges (i, j): the backup weight plane, free outside the trials.
__device__ __forceinline__ int2* edge_list(const JointWs& W) { return reinterpret_cast<int2*>(W.sh_w); }
__device__ __forceinline__ int edge_cap(const JBatch& B) {
    return (int)(B.np / 2 < ((int64_t)1 << 30) ? B.np / 2 : ((int64_t)1 << 30));
}

__device__ __forceinline__ void add_edge(const JBatch& B, const JointWs& W, JointCtl* c, int i,
                                         int j) {
    atomicAdd(&W.dag_cnt[i].x, 1);
    const int k = atomicAdd(&c->nedge, 1);
    if (k < edge_cap(B)) edge_list(W)[k] = make_int2(i, j);
}

__global__ void __launch_bounds__(256, 4)
    k_deps(const __grid_constant__ JBatch B, JointWs W, int it) {
    JointCtl* c = W.ctl;
    if (skip_lists(c)) return;
    __shared__ int cand[kCandMax];
    __shared__ unsigned bits[kDepsBits / 32];
    __shared__ unsigned nbits[kNbBits / 32];
    __shared__ short plist[kDepsWords * 32];   // marked bitmap positions of one round
    __shared__ int s_scan[32];
    __shared__ int s_n, s_vmin, s_vmax, s_umin, s_umax;
    // components in batches of kDepsWarps (those this CTA's grid-stride loop would visit one
    // after another): a warp takes each component of at most kWarpPairs (block, neighbour) pairs
    // on its own, its distinct predecessors in a per-warp hash set; the CTA then takes the
    // batch's larger components (and any whose set overflowed) one at a time as below
    constexpr int kDepsWarps = 8;
    constexpr int kWarpPairs = 256;
    constexpr int kWarpHash = 256;
    __shared__ int whash[kDepsWarps][kWarpHash];
    __shared__ int s_big[kDepsWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int M = c->M_cur;
    const bool use_bits = M <= kDepsBits;
    if (use_bits)
        for (int t = threadIdx.x; t < (M + 31) / 32; t += blockDim.x) bits[t] = 0u;
    // one component by one warp; false: too many pairs or predecessors (left to the CTA)
    auto warp_comp = [&](int j) -> bool {
        const int2 st = W.start[j], en = W.start[j + 1];
        const JImg& I = B.im[img_of_p(B, W.roots[j])];
        const int r = (I.S - 1) / 2;
        const int D = B.strict ? 2 * r : r;
        const int ND = (2 * D + 1) * (2 * D + 1);
        const int npairs = (en.y - st.y) * ND;
        if (npairs > kWarpPairs) return false;
        int* hs = whash[warp];
        for (int t = lane; t < kWarpHash; t += 32) hs[t] = -1;
        __syncwarp();
        bool full = false;
        auto insert = [&](int i) {
            int h = hash_slot(i, kWarpHash - 1);
            for (int k = 0; k < kWarpHash; ++k) {
                const int old = atomicCAS(&hs[h], -1, i);
                if (old == -1 || old == i) return;
                h = (h + 1) & (kWarpHash - 1);
            }
            full = true;
        };
        for (int t = lane; t < npairs; t += 32) {
            const int64_t lq = (int64_t)W.qlist[st.y + t / ND] - I.q0;
            const int nb = t % ND;
            const int bv = (int)(lq / I.w) + nb / (2 * D + 1) - D;
            const int bu = (int)(lq % I.w) + nb % (2 * D + 1) - D;
            if (bv < 0 || bv >= I.h || bu < 0 || bu >= I.w) continue;
            const int64_t bb = I.q0 + (int64_t)bv * I.w + bu;
            if (W.ovf[bb]) {
                // more components than owner slots: the block's pixel labels
                const int ys = bv * I.s, xs = bu * I.s;
                const int ey = min(I.s, I.H - ys), ex = min(I.s, I.W - xs);
                int last = -1;
                for (int e = 0; e < ey * ex; ++e) {
                    const int i = W.lab[I.p0 + (int64_t)(ys + e / ex) * I.W + xs + e % ex];
                    if (i >= 0 && i < j && i != last) {
                        insert(i);
                        last = i;
                    }
                }
            } else {
                const int4* op = reinterpret_cast<const int4*>(W.own + bb * kOwnSlots);
                const int4 o0 = op[0], o1 = op[1];
                const int sl[kOwnSlots] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
#pragma unroll
                for (int e = 0; e < kOwnSlots; ++e) {
                    if (sl[e] < 0) break;   // slots fill in order
                    if (sl[e] < j) insert(sl[e]);
                }
            }
        }
        if (__any_sync(0xffffffffu, full)) return false;
        __syncwarp();
        // the occupied slots (kWarpHash / 32 per lane) are the distinct predecessors: their edges
        // with one slot reservation for the warp
        constexpr int kPerLane = kWarpHash / 32;
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kPerLane; ++k) cnt += hs[lane * kPerLane + k] >= 0 ? 1 : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int n = __shfl_sync(0xffffffffu, incl, 31);
        int e0 = 0;
        if (lane == 0 && n) e0 = atomicAdd(&c->nedge, n);
        e0 = __shfl_sync(0xffffffffu, e0, 0);
        const int ecap = edge_cap(B);
        int pos = e0 + incl - cnt;
#pragma unroll
        for (int k = 0; k < kPerLane; ++k) {
            const int i = hs[lane * kPerLane + k];
            if (i < 0) continue;
            atomicAdd(&W.dag_cnt[i].x, 1);
            if (pos < ecap) edge_list(W)[pos] = make_int2(i, j);
            ++pos;
        }
        if (lane == 0) W.pend[j] = n;
        return true;
    };
    for (int jb = blockIdx.x; jb < M; jb += gridDim.x * kDepsWarps) {
        {
            const int jw = jb + warp * gridDim.x;
            const bool done = jw < M && warp_comp(jw);
            if (lane == 0) s_big[warp] = jw < M && !done ? jw : -1;
        }
        __syncthreads();
        for (int kb = 0; kb < kDepsWarps; ++kb) {
            const int j = s_big[kb];
            if (j < 0) continue;
            if (threadIdx.x == 0) {
                s_n = 0;
                s_vmin = s_umin = 0x7fffffff;
                s_vmax = s_umax = -1;
            }
            __syncthreads();
            const int2 st = W.start[j], en = W.start[j + 1];
            const JImg& I = B.im[img_of_p(B, W.roots[j])];
            const int r = (I.S - 1) / 2;
            const int D = B.strict ? 2 * r : r;
            const int ND = (2 * D + 1) * (2 * D + 1);
            const int npairs = (en.y - st.y) * ND;
#ifdef GLU_TRIAL_TRACE
            if (it == 0 && threadIdx.x == 0 && j < kTraceMax) g_deps_t[j][0] = gtimer();
#endif
            // a large component's (block, neighbour) pairs name each block of its neighbourhood
            // many times: mark them in a bitmap over the bounding box of its blocks dilated by D,
            // then look up every marked block once
            int nitems = npairs, BV0 = 0, BU0 = 0, BW = 1;
            bool nbmap = false;
            if (npairs > kNbMinPairs) {
                // the component's blocks, staged in cand (free until the lookups) when they fit
                const int nbq = en.y - st.y;
                const bool staged = nbq <= kCandMax;
                for (int t = (int)threadIdx.x; t < nbq; t += blockDim.x) {
                    const int lq = (int)((int64_t)W.qlist[st.y + t] - I.q0);
                    if (staged) cand[t] = lq;
                    const int v = lq / I.w, u = lq % I.w;
                    atomicMin(&s_vmin, v);
                    atomicMax(&s_vmax, v);
                    atomicMin(&s_umin, u);
                    atomicMax(&s_umax, u);
                }
                __syncthreads();
                BV0 = s_vmin - D;
                BU0 = s_umin - D;
                BW = s_umax - s_umin + 1 + 2 * D;
                const int BH = s_vmax - s_vmin + 1 + 2 * D;
                nbmap = (int64_t)BH * BW <= kNbBits;
                if (nbmap) {
                    nitems = BH * BW;
                    for (int t = threadIdx.x; t < (nitems + 31) / 32; t += blockDim.x)
                        nbits[t] = 0u;
                    __syncthreads();
                    if (staged) {
                        // per (block, row of its neighbourhood): one run of 2D + 1 positions, at
                        // most two bitmap words (D <= 8)
                        const int NR = 2 * D + 1;
                        for (int t = threadIdx.x; t < nbq * NR; t += blockDim.x) {
                            const int lq = cand[t / NR];
                            const int bv = lq / I.w + t % NR - D, qu = lq % I.w;
                            if (bv < 0 || bv >= I.h) continue;
                            const int row = (bv - BV0) * BW - BU0;
                            const int b0 = row + max(qu - D, 0), b1 = row + min(qu + D, I.w - 1);
                            const int w0 = b0 >> 5, w1 = b1 >> 5;
                            if (w0 == w1) {
                                atomicOr(&nbits[w0], (0xFFFFFFFFu >> (31 - (b1 & 31))) &
                                                         (0xFFFFFFFFu << (b0 & 31)));
                            } else {
                                atomicOr(&nbits[w0], 0xFFFFFFFFu << (b0 & 31));
                                for (int w = w0 + 1; w < w1; ++w) atomicOr(&nbits[w], 0xFFFFFFFFu);
                                atomicOr(&nbits[w1], 0xFFFFFFFFu >> (31 - (b1 & 31)));
                            }
                        }
                    } else {
                        for (int t = threadIdx.x; t < npairs; t += blockDim.x) {
                            const int64_t lq = (int64_t)W.qlist[st.y + t / ND] - I.q0;
                            const int nb = t % ND;
                            const int bv = (int)(lq / I.w) + nb / (2 * D + 1) - D;
                            const int bu = (int)(lq % I.w) + nb % (2 * D + 1) - D;
                            if (bv < 0 || bv >= I.h || bu < 0 || bu >= I.w) continue;
                            const int idx = (bv - BV0) * BW + (bu - BU0);
                            atomicOr(&nbits[idx >> 5], 1u << (idx & 31));
                        }
                    }
                    __syncthreads();
                }
            }
            // one candidate predecessor i < j: with the bitmap, the first sighting records it (its
            // edge is appended with the component's others, one slot reservation for all of them;
            // past kCandMax records, at once)
            auto offer = [&](int i) {
                if (use_bits) {
                    const unsigned bit = 1u << (i & 31);
                    if (atomicOr(&bits[i >> 5], bit) & bit) return;
                    const int slot = atomicAdd(&s_n, 1);
                    if (slot < kCandMax) cand[slot] = i;
                    else add_edge(B, W, c, i, j);
                } else {
                    const int slot = atomicAdd(&s_n, 1);
                    if (slot < kCandMax) cand[slot] = i;
                }
            };
            // kDepsBatch items (pairs, or marked bitmap positions) per thread and round, their
            // loads issued together (a block's overflow flag and its owner slots as two 16-byte
            // loads): the largest components span hundreds of LR blocks, and their CTA sets the
            // kernel's duration
            constexpr int kDepsBatch = 4;
            static_assert(kOwnSlots == 8, "owner slots are read as two int4");
            auto run_items = [&](const short* plist, int n_items) {
                for (int t0 = threadIdx.x * kDepsBatch; t0 < n_items;
                     t0 += blockDim.x * kDepsBatch) {
                    int64_t bb[kDepsBatch];
                    int bvv[kDepsBatch], buu[kDepsBatch];
#pragma unroll
                    for (int k = 0; k < kDepsBatch; ++k) {
                        bb[k] = -1;
                        const int t = t0 + k;
                        if (t >= n_items) continue;
                        if (plist) {
                            const int pos = plist[t];
                            bvv[k] = BV0 + pos / BW;
                            buu[k] = BU0 + pos % BW;
                        } else {
                            const int64_t lq = (int64_t)W.qlist[st.y + t / ND] - I.q0;
                            const int nb = t % ND;
                            bvv[k] = (int)(lq / I.w) + nb / (2 * D + 1) - D;
                            buu[k] = (int)(lq % I.w) + nb % (2 * D + 1) - D;
                            if (bvv[k] < 0 || bvv[k] >= I.h || buu[k] < 0 || buu[k] >= I.w)
                                continue;
                        }
                        bb[k] = I.q0 + (int64_t)bvv[k] * I.w + buu[k];
                    }
                    uint8_t ov[kDepsBatch];
                    int4 o0[kDepsBatch], o1[kDepsBatch];
#pragma unroll
                    for (int k = 0; k < kDepsBatch; ++k) {
                        ov[k] = 0;
                        o0[k] = o1[k] = make_int4(-1, -1, -1, -1);
                        if (bb[k] < 0) continue;
                        ov[k] = W.ovf[bb[k]];
                        const int4* op = reinterpret_cast<const int4*>(W.own + bb[k] * kOwnSlots);
                        o0[k] = op[0];
                        o1[k] = op[1];
                    }
#pragma unroll
                    for (int k = 0; k < kDepsBatch; ++k) {
                        if (bb[k] < 0) continue;
                        if (ov[k]) {
                            // more components than owner slots: read the block's pixel labels
                            const int ys = bvv[k] * I.s, xs = buu[k] * I.s;
                            const int ey = min(I.s, I.H - ys), ex = min(I.s, I.W - xs);
                            int last = -1;
                            for (int e = 0; e < ey * ex; ++e) {
                                const int i =
                                    W.lab[I.p0 + (int64_t)(ys + e / ex) * I.W + xs + e % ex];
                                if (i >= 0 && i < j && i != last) {
                                    offer(i);
                                    last = i;
                                }
                            }
                        } else {
                            // slots fill in order: the first -1 ends the list
                            const int sl[kOwnSlots] = {o0[k].x, o0[k].y, o0[k].z, o0[k].w,
                                                       o1[k].x, o1[k].y, o1[k].z, o1[k].w};
#pragma unroll
                            for (int e = 0; e < kOwnSlots; ++e) {
                                if (sl[e] < 0) break;
                                if (sl[e] < j) offer(sl[e]);
                            }
                        }
                    }
                }
            };
            if (nbmap) {
                // the marked positions only (the bounding box of a long component is mostly empty):
                // each round compacts kDepsWords bitmap words into a list, then looks it up
                const int nwords = (nitems + 31) / 32;
                for (int w0 = 0; w0 < nwords; w0 += kDepsWords) {
                    const int w = w0 + (int)threadIdx.x;
                    const unsigned word = (threadIdx.x < kDepsWords && w < nwords) ? nbits[w] : 0u;
                    int ex;
                    const int tot = block_excl_scan_any(__popc(word), &ex, s_scan);
                    for (unsigned m = word; m; m &= m - 1) plist[ex++] = (short)(w * 32 + __ffs(m) - 1);
                    __syncthreads();
                    run_items(plist, tot);
                    __syncthreads();
                }
            } else {
                run_items(nullptr, nitems);
            }
            __syncthreads();
            const int n = s_n;
            int npred;
            if (use_bits) {
                npred = n;
                const int nrec = min(n, kCandMax);
                if (threadIdx.x == 0) s_vmin = nrec ? atomicAdd(&c->nedge, nrec) : 0;
                __syncthreads();
                const int e0 = s_vmin, ecap = edge_cap(B);
                for (int t = threadIdx.x; t < nrec; t += blockDim.x) {
                    const int i = cand[t];
                    atomicAdd(&W.dag_cnt[i].x, 1);
                    if (e0 + t < ecap) edge_list(W)[e0 + t] = make_int2(i, j);
                }
                // clear the bits this component set (every set bit is one of its predecessors)
                if (n <= kCandMax) {
                    for (int t = threadIdx.x; t < n; t += blockDim.x) bits[cand[t] >> 5] = 0u;
                } else {
                    for (int t = threadIdx.x; t < (M + 31) / 32; t += blockDim.x) bits[t] = 0u;
                }
            } else {
                if (n > kCandMax) {
                    if (threadIdx.x == 0) atomicExch(&c->dag_bad[it], 1);
                    __syncthreads();
                    continue;
                }
                int n2 = 1;
                while (n2 < n) n2 <<= 1;
                for (int t = n + threadIdx.x; t < n2; t += blockDim.x) cand[t] = 0x7fffffff;
                __syncthreads();
                if (n > 1) bitonic_sort_smem(cand, n2);
                if (threadIdx.x == 0) s_n = 0;
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += blockDim.x) {
                    const int i = cand[t];
                    if (t > 0 && cand[t - 1] == i) continue;   // distinct predecessors only
                    atomicAdd(&s_n, 1);
                    add_edge(B, W, c, i, j);
                }
                __syncthreads();
                npred = s_n;
            }
            if (threadIdx.x == 0) W.pend[j] = npred;
#ifdef GLU_TRIAL_TRACE
            if (it == 0 && threadIdx.x == 0 && j < kTraceMax) {
                g_deps_t[j][1] = gtimer();
                g_deps_t[j][2] = (unsigned long long)nitems;
                g_deps_t[j][3] = (unsigned long long)(nbmap ? 1 : 0) | ((unsigned long long)npairs << 8);
                g_deps_t[j][4] = (unsigned long long)blockIdx.x;
            }
#endif
            __syncthreads();
        }
        __syncthreads();   // s_big and the warps' sets are rewritten by the next batch
    }
}

// Successor lists from the edge list (dag_start: the scanned successor counts) and the ready
// queue's first entries. The graph is dropped (the trials then claim in index order) when the
// edges did not fit the scratch list or the successor array.
__global__ void k_edge_scatter(const __grid_constant__ JBatch B, JointWs W, int it) {
    JointCtl* c = W.ctl;
    if (skip_lists(c)) return;
    const int M = c->M_cur, ne = c->nedge;
    if (*(volatile int*)&c->dag_bad[it] || ne > edge_cap(B) || (int64_t)W.dag_start[M].x > W.ecap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&c->dag_bad[it], 1);
        return;
    }
    const int2* E = edge_list(W);
    const int stride = gridDim.x * blockDim.x;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += stride) {
        const int2 e = __ldcg(&E[k]);
        W.succ[W.dag_start[e.x].x + atomicAdd(&W.dag_fill[e.x], 1)] = e.y;
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += stride) {
        if (W.pend[j] != 0) continue;
        const int pos = atomicAdd(&c->tail[it], 1);
        W.queue[pos] = j;
        GLU_TRACE_ANY(it, j, 0);
    }
}

// ------------------------------------------- small large-error lists: the whole phase in one CTA
//
// After the first iteration the large-error list is short (a few thousand pixels or fewer), and
// the multi-kernel path above spends its time in launch gaps and near-empty grids. k_small_comp
// does the same work in one 1024-thread CTA with the list in shared memory:
//   components  min-label hooking over the list's adjacencies (neighbours found by binary search
//               in the sorted list) alternated with pointer jumping until nothing changes: every
//               pass is a barrier-separated sweep of logarithmic depth, and the final root of a
//               component is its smallest index, i.e. its smallest raster index
//   buckets     components numbered in order of their roots; pixel and distinct-LR-block buckets
//               (owner slots claimed as in k_comp_count, so every later reader sees the same state)
//   graph       one flat pass over every (component block, neighbouring cell) pair: the blocks of
//               all components are hashed into cells of D + 1 LR pixels, so every block within D
//               of a block lies in the 3 x 3 cells around it; each distinct (predecessor,
//               component) edge enters a shared hash set once, which gives the predecessor counts
//               and, after a scan, the successor lists
// The kernels of the multi-kernel path then return at once (small_cur). If the hooking does not
// settle within kSmallRounds passes (it always has on the workloads), the kernel returns before
// writing anything and the multi-kernel path runs instead.
constexpr int kSmallFg = 4096;      // large-error pixels handled by the one-CTA path
constexpr int kSmallHash = 8192;    // cell hash slots (power of two, more than kSmallFg)
constexpr int kSmallEdges = 2 * kSmallFg;   // edge hash-set slots (power of two)
constexpr int kSmallThreads = 1024;
constexpr int kSmallPer = kSmallFg / kSmallThreads;   // list pixels per thread
constexpr int kSmallRounds = 64;

struct SmallSmem {
    union {
        struct {
            int p[kSmallFg];        // the list: global pixel ids, ascending
            int a[kSmallFg];        // component forest, then component ids
        } l;
        int eset[kSmallEdges];      // graph: edge keys i * kSmallFg + j (-1: empty)
    } u;
    int b[2 * kSmallFg];            // root ranks; then per component (pixels, blocks) counters
    int q[kSmallFg];                // per list pixel: its (component, block) representative
    int2 tab[kSmallHash];           // (cell key, first entry); key -1: empty
    int ecid[kSmallFg];             // entry: component
    int eq[kSmallFg];               // entry: LR block
    int enext[kSmallFg];            // next entry of the same cell
    int scan[32];
    int nent, nedge, bad;
};

__device__ __forceinline__ int img_of_q(const JBatch& B, int64_t q) {
    int i = 0;
    while (i + 1 < B.n && B.im[i + 1].q0 <= q) ++i;
    return i;
}

// Chunked exclusive scan of n values in place (each thread a contiguous chunk); returns the total.
__device__ __forceinline__ int small_scan(int* v, int n, int* scan_smem) {
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int e0 = (int)threadIdx.x * per, e1 = min(e0 + per, n);
    int s = 0;
    for (int e = e0; e < e1; ++e) s += v[e];
    int ex;
    const int tot = block_excl_scan_any(s, &ex, scan_smem);
    for (int e = e0; e < e1; ++e) {
        const int t = v[e];
        v[e] = ex;
        ex += t;
    }
    __syncthreads();
    return tot;
}

// cond / has_cond: inside a recorded graph, the condition of the conditional node that holds the
// multi-kernel path; set to 0 (skip it) when this kernel built the lists (its default, 1, runs it).
__global__ void __launch_bounds__(kSmallThreads, 1)
    k_small_comp(const __grid_constant__ JBatch B, JointWs W, int it,
                 cudaGraphConditionalHandle cond, int has_cond) {
    JointCtl* c = W.ctl;
    if (!any_active(c)) {   // converged: the multi-kernel path would return at once
        if (has_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int nfg = c->nfg;
    if (nfg <= 0 || nfg > kSmallFg) return;   // the multi-kernel path does it (small_cur is 0)
    extern __shared__ __align__(16) unsigned char small_dyn[];
    SmallSmem& S = *reinterpret_cast<SmallSmem*>(small_dyn);
    int* P = S.u.l.p;
    volatile int* A = S.u.l.a;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int e = tid; e < nfg; e += nthr) {
        P[e] = __ldcg(&W.ulist[e]);
        A[e] = e;
    }
    for (int t = tid; t < kSmallHash; t += nthr) S.tab[t] = make_int2(-1, -1);
    if (tid == 0) {
        S.nent = 0;
        S.nedge = 0;
        S.bad = 0;
    }
    __syncthreads();
    GLU_SMALL_STAMP(it, 0);
    // the backward neighbours (W, N, and NW, NE with 8-connectivity) of this thread's pixels e =
    // tid + k * nthr, as local indices (-1: not in the list)
    int nbr[kSmallPer][4];
#pragma unroll
    for (int k = 0; k < kSmallPer; ++k) {
        const int e = tid + k * nthr;
#pragma unroll
        for (int d = 0; d < 4; ++d) nbr[k][d] = -1;
        if (e >= nfg) continue;
        const int p = P[e];
        const JImg& I = B.im[img_of_p(B, p)];
        const int64_t lp = p - I.p0;
        const int y = (int)(lp / I.W), x = (int)(lp % I.W);
        int cand[4] = {x > 0 ? p - 1 : -1, y > 0 ? p - I.W : -1,
                       (y > 0 && x > 0 && B.conn == 8) ? p - I.W - 1 : -1,
                       (y > 0 && x + 1 < I.W && B.conn == 8) ? p - I.W + 1 : -1};
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            if (cand[d] < 0) continue;
            const int f = lower_bound_i(P, e, cand[d]);
            if (f < e && P[f] == cand[d]) nbr[k][d] = f;
        }
    }
    // hook every edge's two roots (the larger under the smaller), then jump pointers until every
    // tree is a star; repeat until no edge joins two trees
    bool settled = false;
#ifdef GLU_TRIAL_TRACE
    int n_jumps = 0;
#endif
    for (int round = 0; round < kSmallRounds; ++round) {
#ifdef GLU_TRIAL_TRACE
        if (threadIdx.x == 0) g_small_t[it][10] = (unsigned long long)(round + 1);
#endif
        int changed = 0;
#pragma unroll
        for (int k = 0; k < kSmallPer; ++k) {
            const int e = tid + k * nthr;
            if (e >= nfg) continue;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const int f = nbr[k][d];
                if (f < 0) continue;
                const int ra = A[e], rb = A[f];
                if (ra == rb) continue;
                atomicMin((int*)&A[max(ra, rb)], min(ra, rb));
                changed = 1;
            }
        }
        if (!__syncthreads_or(changed)) {
            settled = true;
            break;
        }
        // every tree a star again, in one round: each thread walks from its pixels to the root,
        // halving the path on the way. A parent is always a smaller index than its child and
        // the root the smallest of its tree, so the writes (atomicMin) only ever move a pixel
        // closer to its root, whichever threads walk through it, and leave each of this
        // thread's pixels under the root itself
#pragma unroll
        for (int k = 0; k < kSmallPer; ++k) {
            const int e = tid + k * nthr;
            if (e >= nfg) continue;
            int x = e;
            for (;;) {
                const int px = A[x], g = A[px];
                if (g == px) {
                    if (x != e) atomicMin((int*)&A[e], px);
                    break;
                }
                atomicMin((int*)&A[x], g);
                x = g;
            }
        }
#ifdef GLU_TRIAL_TRACE
        if (threadIdx.x == 0) g_small_t[it][11] = (unsigned long long)(++n_jumps);
#endif
        __syncthreads();
    }
    if (!settled) return;   // nothing global written yet: the multi-kernel path runs
    GLU_SMALL_STAMP(it, 1);
    GLU_SMALL_STAMP(it, 2);
    // components in order of their roots; per-component state cleared as in k_root_scatter
    int M;
    {
        const int per = (nfg + nthr - 1) / nthr;
        const int e0 = tid * per, e1 = min(e0 + per, nfg);
        int nr = 0;
        for (int e = e0; e < e1; ++e) nr += A[e] == e;
        int ex;
        M = block_excl_scan_any(nr, &ex, S.scan);
        for (int e = e0; e < e1; ++e) {
            if (A[e] != e) continue;
            const int j = ex++;
            S.b[e] = j;
            const int p = P[e];
            W.roots[j] = p;
            W.done[j] = 0;
            W.queue[j] = -1;
            atomicAdd(&c->M[img_of_p(B, p)][it], 1);
        }
    }
    __syncthreads();
    for (int e = tid; e < nfg; e += nthr) A[e] = S.b[A[e]];   // component id (root's rank)
    __syncthreads();
    for (int j = tid; j < 2 * M; j += nthr) S.b[j] = 0;
    if (tid == 0) c->M_cur = M;
    __syncthreads();
    GLU_SMALL_STAMP(it, 3);
    // buckets: label, owner slots (as k_comp_count), pixel and distinct-block counts
    int* cntp = S.b;        // pixels per component
    int* cntq = S.b + M;    // distinct LR blocks per component (owner-slot representatives)
    for (int e = tid; e < nfg; e += nthr) {
        const int p = P[e], j = A[e];
        W.lab[p] = j;
        const JImg& I = B.im[img_of_p(B, p)];
        const int64_t lp = p - I.p0;
        const int y = (int)(lp / I.W), x = (int)(lp % I.W);
        const int64_t q = I.q0 + (int64_t)(y / I.s) * I.w + (x / I.s);
        int ins = -1;
        for (int k = 0; k < kOwnSlots; ++k) {
            const int old = atomicCAS(&W.own[q * kOwnSlots + k], -1, j);
            if (old == -1) { ins = 1; break; }
            if (old == j) { ins = 0; break; }
        }
        if (ins == -1) W.ovf[q] = 1;
        const bool rep = ins != 0;
        atomicAdd(&cntp[j], 1);
        S.q[e] = rep ? (int)q : -1;   // temporarily per pixel
        if (rep) atomicAdd(&cntq[j], 1);
    }
    __syncthreads();
    GLU_SMALL_STAMP(it, 4);
    const int totp = small_scan(cntp, M, S.scan);
    const int totq = small_scan(cntq, M, S.scan);
    for (int j = tid; j < M; j += nthr) W.start[j] = make_int2(cntp[j], cntq[j]);
    if (tid == 0) W.start[M] = make_int2(totp, totq);
    __syncthreads();
    // fill comp_pix and qlist (the counters become the end of each component's range), and hash
    // every (component, block) pair into its cell
    for (int e = tid; e < nfg; e += nthr) {
        const int p = P[e], j = A[e];
        const int pos = atomicAdd(&cntp[j], 1);
        W.comp_pix[pos] = p;
        const int q = S.q[e];
        if (q < 0) continue;
        const int qp = atomicAdd(&cntq[j], 1);
        W.qlist[qp] = q;
        const JImg& I = B.im[img_of_q(B, q)];
        const int D = B.strict ? I.S - 1 : (I.S - 1) / 2;
        const int C = D + 1, cw = (I.w + C - 1) / C;
        const int lq = q - (int)I.q0;
        const int key = (int)(I.q0 + (int64_t)((lq / I.w) / C) * cw + (lq % I.w) / C);
        int h = hash_slot(key, kSmallHash - 1);
        for (int k = 0; k < kSmallHash; ++k) {
            const int old = atomicCAS(&S.tab[h].x, -1, key);
            if (old == -1 || old == key) break;
            h = (h + 1) & (kSmallHash - 1);
        }
        const int ent = atomicAdd(&S.nent, 1);
        S.ecid[ent] = j;
        S.eq[ent] = q;
        S.enext[ent] = atomicExch(&S.tab[h].y, ent);
    }
    __syncthreads();
    GLU_SMALL_STAMP(it, 5);
    // from here the list and the forest are no longer needed: their space holds the edge set
    for (int t = tid; t < kSmallEdges; t += nthr) S.u.eset[t] = -1;
    __syncthreads();
    GLU_SMALL_STAMP(it, 6);
    // graph: tpe threads per entry (one (component, block) pair of the cell hash, which holds its
    // component and block: no lookup in global memory), each working out the entry's block, cell
    // and image constants once and scanning 9 / tpe of the nine cells around it (its own and the
    // eight neighbours). tpe (1, 3 or 9) minimises rounds x (set-up + cells per thread), the
    // set-up costing about three cell scans: 9 for short lists, fewer for long ones.
    int* npred = cntp;   // per component: distinct predecessors
    for (int j = tid; j < M; j += nthr) npred[j] = 0;
    __syncthreads();
    const int nent = S.nent;
    int tpe = 9;
    {
        int best = 0x7fffffff;
        for (int t = 9; t >= 1; t /= 3) {
            const int cost = (nent * t + nthr - 1) / nthr * (3 + 9 / t);
            if (cost < best) { best = cost; tpe = t; }
        }
    }
    for (int et = tid; et < nent * tpe; et += nthr) {
        const int e = et / tpe, sub = et - e * tpe;
        const int j = S.ecid[e], q = S.eq[e];
        const JImg& I = B.im[img_of_q(B, q)];
        const int D = B.strict ? I.S - 1 : (I.S - 1) / 2;
        const int C = D + 1, cw = (I.w + C - 1) / C, ch = (I.h + C - 1) / C;
        const int lq = q - (int)I.q0;
        const int v = lq / I.w, u = lq % I.w;
        const int cv0 = v / C, cu0 = u / C;
        for (int nc = sub; nc < 9; nc += tpe) {
            const int cv = cv0 + nc / 3 - 1, cu = cu0 + nc % 3 - 1;
            if (cv < 0 || cv >= ch || cu < 0 || cu >= cw) continue;
            const int key = (int)(I.q0 + (int64_t)cv * cw + cu);
            int h = hash_slot(key, kSmallHash - 1);
            int ent = -1;
            for (int k = 0; k < kSmallHash; ++k) {
                const int kk = S.tab[h].x;
                if (kk == key) { ent = S.tab[h].y; break; }
                if (kk == -1) break;
                h = (h + 1) & (kSmallHash - 1);
            }
            for (int g = 0; ent >= 0 && g < kSmallFg; ++g, ent = S.enext[ent]) {
                const int i = S.ecid[ent];
                if (i >= j) continue;
                const int lq2 = S.eq[ent] - (int)I.q0;
                const int dv = lq2 / I.w - v, du = lq2 % I.w - u;
                if (dv < -D || dv > D || du < -D || du > D) continue;
                const int ekey = i * kSmallFg + j;
                int eh = hash_slot(ekey, kSmallEdges - 1);
                bool inserted = false;
                int k = 0;
                for (; k < kSmallEdges; ++k) {
                    const int old = atomicCAS(&S.u.eset[eh], -1, ekey);
                    if (old == -1) { inserted = true; break; }
                    if (old == ekey) break;
                    eh = (eh + 1) & (kSmallEdges - 1);
                }
                if (k == kSmallEdges) S.bad = 1;   // the set is full
                if (inserted) {
                    atomicAdd(&npred[j], 1);
                    atomicAdd(&S.nedge, 1);
                }
            }
        }
    }
    __syncthreads();
    GLU_SMALL_STAMP(it, 7);
    GLU_SMALL_STAMP(it, 8);
    const int nedge = S.nedge;
    if (S.bad || nedge > W.ecap) {
        if (tid == 0) atomicExch(&c->dag_bad[it], 1);   // the trials claim in index order
    } else {
        for (int j = tid; j < M; j += nthr) W.pend[j] = npred[j];
        int* scnt = cntq;   // successors per predecessor (the ranges are no longer needed)
        __syncthreads();
        for (int j = tid; j < M; j += nthr) scnt[j] = 0;
        __syncthreads();
        for (int t = tid; t < kSmallEdges; t += nthr) {
            const int ek = S.u.eset[t];
            if (ek >= 0) atomicAdd(&scnt[ek / kSmallFg], 1);
        }
        __syncthreads();
        const int tot = small_scan(scnt, M, S.scan);
        for (int j = tid; j < M; j += nthr) W.dag_start[j] = make_int2(scnt[j], 0);
        if (tid == 0) W.dag_start[M] = make_int2(tot, 0);
        __syncthreads();
        for (int t = tid; t < kSmallEdges; t += nthr) {
            const int ek = S.u.eset[t];
            if (ek >= 0) W.succ[atomicAdd(&scnt[ek / kSmallFg], 1)] = ek % kSmallFg;
        }
        // components without predecessors enter the ready queue
        for (int j = tid; j < M; j += nthr) {
            if (npred[j] != 0) continue;
            const int pos = atomicAdd(&c->tail[it], 1);
            W.queue[pos] = j;
            GLU_TRACE_ANY(it, j, 0);
        }
    }
    __syncthreads();
    GLU_SMALL_STAMP(it, 9);
    if (tid == 0) {
        c->small_cur = 1;
        if (has_cond) cudaGraphSetConditional(cond, 0u);
    }
}

// ---------------------------------------------------------------------------- the trials


struct TrialCtx {
    JointWs ws;
    int it;
    unsigned long long wait_limit_ns;   // 0: trial_deadline(M)
    // verification log (null: off; see log_record)
    int4* alog;
    long long alog_cap;
};

static unsigned long long g_wait_limit_ns = 0;   // test hook (glu_test_set_wait_limit)
void set_trial_wait_limit(unsigned long long ns) { g_wait_limit_ns = ns; }
static int4* g_argmax_log = nullptr;              // test hook (glu_test_joint_argmax_log)
static long long g_argmax_cap = 0;
void set_argmax_log(void* buf, long long cap) {
    g_argmax_log = (int4*)buf;
    g_argmax_cap = buf ? cap : 0;
}

// Appends one replacement choice to the verification log (one thread).
__device__ __forceinline__ void log_argmax(const TrialCtx& X, int j, int q, int lp) {
    log_record(X.alog, X.alog_cap, make_int4(X.it, j, q, lp));
}

__device__ __forceinline__ long long to_fixed(float x) {
    // x * 2^32 is exact in float; conversion rounds the part below 2^-32 to nearest
    return __float2ll_rn(x * 4294967296.0f);
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

// Shared-memory limits of the one-CTA trial path (below) and its layout.
constexpr int kFastQRaw = 512;    // LR block entries of the component (before removing repeats)
constexpr int kFastQ = 64;        // distinct LR blocks of the component
constexpr int kFastA = 256;       // blocks re-searched
constexpr int kFastPx = 4096;     // pixels re-searched
constexpr int kFastRegion = 2304; // LR pixels of the staged neighbourhood

struct FastSmem {
    float4 region[kFastRegion];
    unsigned long long best[kFastQ];
    int rawq[kFastQRaw];
    int qs[kFastQ];
    uint32_t newc[kFastQ];
    int blocks[kFastA];
    int pxoff[kFastA + 1];
    int scan[32];
    short qmap[kFastRegion];  // Q block: its index + 1
    short amap[kFastRegion];  // block to re-search: its index + 1
    uint16_t rcode[kFastPx];
    float rw[kFastPx];
    float rerr[kFastPx];
    uint32_t hrpx[kFastPx];   // guide colour of every re-searched pixel
    float eold[kFastPx];      // its error before the trial
    uint16_t code0[kFastPx];  // its pair before the trial
    int full[kFastPx];        // the component's pixels, then the pixels needing a full search
    int nfull;
};

constexpr uint16_t kNotSearched = 0xFFFFu;
constexpr int kMaxChg = 8;       // replaced LR pixels per window for the exact re-search

// One warp re-runs Algorithm 1 on the HR pixels of LR block (bv, bu) of image I against the
// current LR image (comp >= 0: only the pixels of that component), writing the results in place
// and the previous values to the backup planes. The previous errors (e0) and the new ones (e1)
// are summed exactly in 2^-32 units.
// The general path splits every LR block into chunks of HR pixels in raster order, one item each,
// so that a block is re-searched by several warps: 32 pixels (one per lane) for blocks of up to
// 1024 pixels, 1024 pixels above that (scales above 32). The sums are exact integers, so the
// grouping does not change them.
__device__ __forceinline__ int chunk_px(const JImg& I) { return I.s * I.s <= 1024 ? 32 : 1024; }
__device__ __forceinline__ int block_chunks(const JImg& I) {
    return (I.s * I.s + chunk_px(I) - 1) / chunk_px(I);
}

template <int S>
__device__ __noinline__ void warp_block_trial(const JBatch& B, const TrialCtx& X, const JImg& I,
                                              float4* win, int bv, int bu, int chunk, int comp,
                                              int img, long long& e0, long long& e1) {
    constexpr int r = (S - 1) / 2, K = S * S;
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < K; k += 32) {
        const int v = bv + k / S - r, u = bu + k % S - r;
        float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v >= 0 && v < I.h && u >= 0 && u < I.w) {
            const uint32_t c = load_rgb(I.lr, I.lr_pitch, v, u);
            c4 = make_float4((float)(c & 255u), (float)((c >> 8) & 255u), (float)(c >> 16), 0.f);
        }
        win[k] = c4;
    }
    __syncwarp();
    uint32_t rm, cm;
    window_masks(bv, bu, I.h, I.w, S, rm, cm);
    const int ys = bv * I.s, xs = bu * I.s;
    const int ey = min(I.s, I.H - ys), ex = min(I.s, I.W - xs);
    long long s0 = 0, s1 = 0;
    int nsearched = 0;
    const int cpx = chunk_px(I);
    const int jend = min(ey * ex, (chunk + 1) * cpx);
    for (int j = chunk * cpx + lane; j < jend; j += 32) {
        const int y = ys + j / ex, x = xs + j % ex;
        const int64_t lp = (int64_t)y * I.W + x, p = I.p0 + lp;
        if (comp >= 0 && __ldcg(&X.ws.lab[p]) != comp) continue;
        const uint8_t* ip = I.hr + (int64_t)y * I.hr_pitch + (int64_t)x * 3;
        const SearchOut o = search_pixel<S, true>(win, S, rm, cm, (float)ip[0], (float)ip[1],
                                                  (float)ip[2], B.eps255, false);
        ++nsearched;
        // the new Theta / E go in place; the old ones to the backup planes (restored if the
        // trial is rolled back)
        const float eold = __ldcg(&I.err[lp]);
        X.ws.sh_code[p] = __ldcg(&I.code[lp]);
        X.ws.sh_w[p] = load_weight_cg(I.weight, B.wfmt, lp);
        X.ws.sh_err[p] = eold;
        I.code[lp] = (uint16_t)(o.ka * K + o.kb);
        store_weight(I.weight, B.wfmt, lp, o.omega);
        I.err[lp] = o.err;
        s0 += to_fixed(eold);
        s1 += to_fixed(o.err);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nsearched += __shfl_xor_sync(0xffffffffu, nsearched, o);
    if (lane == 0 && nsearched)
        atomicAdd(&X.ws.ctl->searched[img][X.it], (unsigned long long)nsearched);
    e0 = warp_sum_ll(s0);
    e1 = warp_sum_ll(s1);
    __syncwarp();
}

// Roll back a trial for a chunk of LR block (bv, bu): restore Theta and E from the backup planes.
__device__ __forceinline__ void warp_block_rollback(const JBatch& B, const TrialCtx& X,
                                                    const JImg& I, int bv, int bu, int chunk,
                                                    int comp) {
    const int lane = threadIdx.x & 31;
    const int ys = bv * I.s, xs = bu * I.s;
    const int ey = min(I.s, I.H - ys), ex = min(I.s, I.W - xs);
    const int cpx = chunk_px(I);
    const int jend = min(ey * ex, (chunk + 1) * cpx);
    for (int j = chunk * cpx + lane; j < jend; j += 32) {
        const int y = ys + j / ex, x = xs + j % ex;
        const int64_t lp = (int64_t)y * I.W + x, p = I.p0 + lp;
        if (comp >= 0 && __ldcg(&X.ws.lab[p]) != comp) continue;
        I.code[lp] = __ldcg(&X.ws.sh_code[p]);
        store_weight_raw(I.weight, B.wfmt, lp, __ldcg(&X.ws.sh_w[p]));
        I.err[lp] = __ldcg(&X.ws.sh_err[p]);
    }
}

// Block item t of component j (global LR list offset stY) of image I: the LR block it
// designates, or false when it falls outside the LR image. STRICT: (distinct block u,
// neighbour nb) pairs; PAPER: the distinct blocks themselves.
__device__ __forceinline__ bool item_block(const JBatch& B, const TrialCtx& X, const JImg& I,
                                           int stY, int t, int& bv, int& bu) {
    const int r = (I.S - 1) / 2, NB = (2 * r + 1) * (2 * r + 1);
    const int64_t lq = (int64_t)X.ws.ulist[stY + (B.strict ? t / NB : t)] - I.q0;
    bv = (int)(lq / I.w);
    bu = (int)(lq % I.w);
    if (B.strict) {
        const int nb = t % NB;
        bv += nb / (2 * r + 1) - r;
        bu += nb % (2 * r + 1) - r;
        if (bv < 0 || bv >= I.h || bu < 0 || bu >= I.w) return false;
    }
    return true;
}

__device__ __forceinline__ unsigned long long trial_tag(int it, int j, int phase) {
    return ((unsigned long long)(it * 4 + phase) << 40) | (unsigned long long)(j + 1);
}

// One warp processes item t of component j of image img: chunk t % nch of the block of block
// item t / nch (STRICT: only if that block item owns the block, so a block reached from several
// q is processed once), running the trial (kind bit 0 clear, sums returned) or the rollback.
// With kind bit 1 the block items are the blocks listed in task slot `slot`'s A list.
__device__ __noinline__ bool process_item(const JBatch& B, const TrialCtx& X, float4* win,
                                             int j, int img, int stY, int kind, int t, int slot,
                                             long long& e0, long long& e1) {
    const JImg& I = B.im[img];
    e0 = 0;
    e1 = 0;
    const int nch = block_chunks(I), t0 = t / nch, chunk = t % nch;
    int bv, bu;
    if (kind & 2) {   // a listed block: owned by this task, inside the image
        const int lq = __ldcg(&X.ws.alist[(int64_t)slot * kSlotA + t0]);
        bv = lq / I.w;
        bu = lq % I.w;
    } else {
        if (!item_block(B, X, I, stY, t0, bv, bu)) return false;
        if (B.strict && __ldcg(&X.ws.bown[I.q0 + (int64_t)bv * I.w + bu]) != t0) return false;
    }
    const int comp = B.strict ? -1 : j;
    if ((kind & 1) == 0) {
        switch (I.S) {
            case 1: warp_block_trial<1>(B, X, I, win, bv, bu, chunk, comp, img, e0, e1); break;
            case 3: warp_block_trial<3>(B, X, I, win, bv, bu, chunk, comp, img, e0, e1); break;
            case 5: warp_block_trial<5>(B, X, I, win, bv, bu, chunk, comp, img, e0, e1); break;
            case 7: warp_block_trial<7>(B, X, I, win, bv, bu, chunk, comp, img, e0, e1); break;
            default: warp_block_trial<9>(B, X, I, win, bv, bu, chunk, comp, img, e0, e1); break;
        }
    } else {
        warp_block_rollback(B, X, I, bv, bu, chunk, comp);
    }
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
// (the whole 4K workload takes milliseconds); give up, record GLU_ERR_TIMEOUT and return. The
// allowance grows with the iteration's component count (a trial at scale 128 re-searches
// 150 K pixels, and tens of thousands of them can depend on one another), up to a cap.
constexpr unsigned long long kTrialDeadlineNs = 5000000000ull;
constexpr unsigned long long kDeadlinePerComponentNs = 500000ull;
constexpr unsigned long long kTrialDeadlineCapNs = 30000000000ull;
__device__ __forceinline__ unsigned long long trial_deadline(int M) {
    const unsigned long long d = kTrialDeadlineNs + (unsigned long long)M * kDeadlinePerComponentNs;
    return d < kTrialDeadlineCapNs ? d : kTrialDeadlineCapNs;
}

// Warp-uniform: true when the launch must stop waiting (its deadline, an absolute global-timer
// value, has passed, or another wait already timed out). Lane 0 decides, every lane gets the
// same answer.
__device__ __forceinline__ bool warp_should_abort(const JointCtl* c, unsigned long long deadline) {
    int a = 0;
    if ((threadIdx.x & 31) == 0)
        a = (*(volatile const int*)&c->timeout != 0) || now_ns() > deadline;
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
    return ((w >> 32) & 1ull) &&
           (int)(w & 0xFFFFFFFFull) < *(volatile const int*)&W_.slot_info[k].y;
}

__device__ __forceinline__ int4 ld_volatile_i4(const int4* p) {
    int4 v;
    asm volatile("ld.volatile.global.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Lane 0: claim the next item of slot k (item -1 if the slot is closed or has none left).
__device__ __forceinline__ int claim_item(const JointWs& W_, int k, int4& info) {
    const unsigned long long old = atom_add_acquire_u64(&W_.slot_word[k], 1ull);
    if (!((old >> 32) & 1ull)) return -1;
    const int nx = (int)(old & 0xFFFFFFFFull);
    info = ld_volatile_i4(&W_.slot_info[k]);
    if (nx >= info.y) return -1;
    // the claimer of the last item takes the task off the open count
    if (nx + 1 == info.y) atomicSub(&W_.ctl->open_tasks, 1);
    return nx;
}

// One warp: take one unclaimed item of an open task — its own CTA's slot first, then the slot it
// helped last (`hint`), otherwise the open task of the smallest component — and process it.
// Returns false if no item was available. own_left: the caller's own slot is open and may still
// have items; it is claimed from directly (no snapshot first), and own_left cleared once it has
// none. own_only: take no item of another slot.
//
// Claiming is one fetch-and-add on the slot's (epoch << 32 | next) word. An increment that lands
// on a closed slot is harmless (opening overwrites the word); one that lands on an open epoch
// owns item `next` of that epoch, whose context cannot change before that item is finished.
__device__ __noinline__ bool help_one(const JBatch& B, const TrialCtx& X, float4* win, int own, int G,
                         int& hint, bool& own_left, bool own_only = false) {
    const JointWs& W_ = X.ws;
    const int lane = threadIdx.x & 31;
    int s_sel = -1, item = -1;
    int4 info = make_int4(0, 0, 0, 0);
    if (own_left) {
        if (lane == 0) {
            item = claim_item(W_, own, info);
            if (item >= 0) s_sel = own;
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item < 0) own_left = false;
    }
    if (item < 0 && own_only) return false;
    if (item < 0) {
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
                const int jj = *(volatile const int*)&W_.slot_info[k].x;
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
        if (lane == 0) item = claim_item(W_, s_sel, info);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item < 0) {
            hint = -1;
            return false;
        }
    }
    s_sel = __shfl_sync(0xffffffffu, s_sel, 0);
    hint = s_sel;
    const int j = __shfl_sync(0xffffffffu, info.x, 0);
    const int ik = __shfl_sync(0xffffffffu, info.z, 0);
    const int stY = __shfl_sync(0xffffffffu, info.w, 0);
    const int img = ik >> 2, kind = ik & 3;
#ifdef GLU_TRIAL_TRACE
    const unsigned long long tr0 = gtimer();
    if (lane == 0 && s_sel != (int)blockIdx.x && j < kTraceMax && (kind & 1) == 0)
        atomicAdd(&g_trace[X.it][j][8], 1ull);
#endif
    long long e0, e1;
    const bool did = process_item(B, X, win, j, img, stY, kind, item, s_sel, e0, e1);
#ifdef GLU_TRIAL_TRACE
    if (lane == 0 && j < kTraceMax && (kind & 1) == 0) {
        const unsigned long long tr1 = gtimer();
        atomicMax(&g_trace[X.it][j][11], tr1);
        atomicAdd(&g_trace[X.it][j][13], tr1 - tr0);
        if (item + 1 == info.y) g_trace[X.it][j][10] = tr0;   // the last item claimed
    }
#endif
    __syncwarp();
    if (lane == 0) {
        if (did && (kind & 1) == 0) {
            atomicAdd(&W_.slot_e0[s_sel], (unsigned long long)e0);
            atomicAdd(&W_.slot_e1[s_sel], (unsigned long long)e1);
        }
        // release: this warp's writes (backup planes, Theta, E, sums) are visible to whoever
        // observes the count
        red_release_add(&W_.slot_fin[s_sel], 1);
    }
    __syncwarp();
    return true;
}

// Run the items of one task of component j. Small tasks stay inside the CTA; larger ones are
// published in the CTA's slot so idle warps anywhere in the grid can take items. Returns the
// (fixed-point) sums of a trial in e0/e1. False on an exhausted wait.
__device__ bool run_task(const JBatch& B, const TrialCtx& X, float4* win, int j, int img, int stY,
                         int kind, int nitems, int G, unsigned long long* s_e0,
                         unsigned long long* s_e1, int* s_flag, unsigned long long deadline) {
    const JointWs& W_ = X.ws;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int nwarps = kTrialThreads / 32;
    const int own = blockIdx.x;
    if (nitems <= nwarps) {
        for (int t = warp; t < nitems; t += nwarps) {
            long long e0, e1;
            const bool did = process_item(B, X, win, j, img, stY, kind, t, own, e0, e1);
            if (did && (kind & 1) == 0 && lane == 0) {
                atomicAdd(s_e0, (unsigned long long)e0);
                atomicAdd(s_e1, (unsigned long long)e1);
            }
        }
        __syncthreads();
        return true;
    }
    if (tid == 0) {
        const unsigned long long e = W_.slot_word[own] >> 32;  // even: closed
        W_.slot_info[own] = make_int4(j, nitems, img * 4 + kind, stY);
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
    // the owner's warps take only this task's items, then wait for its last ones: a warp busy
    // with another task's item would hold the CTA back after this task is done
    int hint = -1;
    bool own_left = true;
    for (;;) {
        int fin = 0;
        if (lane == 0) fin = ld_acquire(&W_.slot_fin[own]) >= nitems;
        if (__shfl_sync(0xffffffffu, fin, 0)) break;
        if (!help_one(B, X, win, own, G, hint, own_left, true)) __nanosleep(64);
        if (warp_should_abort(X.ws.ctl, deadline)) {
            if (lane == 0) *s_flag = 1;
            break;
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if ((kind & 1) == 0) {
            *s_e0 = ld_volatile_u64(&W_.slot_e0[own]);
            *s_e1 = ld_volatile_u64(&W_.slot_e1[own]);
        }
        const unsigned long long w = W_.slot_word[own] >> 32;
        atomicExch(&W_.slot_word[own], (w + 1ull) << 32);  // closed
    }
    __syncthreads();
    return *s_flag == 0;
}

// ------------------------------------------------------ trials of small components in one CTA
//
// A component whose blocks, re-searched pixels and LR neighbourhood fit in shared memory is tried
// by its CTA alone: the LR neighbourhood (with the replacements applied) is staged in shared
// memory, every affected block is re-searched by one warp against it, and the new Theta / E stay
// in shared memory until the decision. A kept trial writes them (and the new LR colours) out; a
// rolled-back trial writes nothing, so the global state never holds a rejected trial. The
// arithmetic is that of the general path below, and so are the sums: every pixel's error rounded
// to 2^-32 units and added as 64-bit integers, exact in any order.

// The re-search of a trial in two passes, so that the few pixels that need a full search do not
// hold up whole warps:
//   pass 1 (a warp per block): with `incr` (STRICT: Theta is Algorithm 1 on the LR image before
//     the trial) re-search each pixel exactly from its previous pair when the replaced LR pixels
//     in its window (at most kMaxChg) are neither its a nor its b and do not become its a;
//     otherwise queue it for a full search (entry: pixel index, block, and the new a when only
//     step 2 must be redone);
//   pass 2 (every thread of the CTA): the queued searches.
// e1 is summed as the pixels finish in either pass; e0 was summed while the pixels were staged.

__device__ __forceinline__ int full_entry(int pix, int bi, int a_known) {
    return pix | (bi << 12) | ((a_known + 1) << 20);
}

template <int S>
__device__ __noinline__ void fast_block_pass(const JBatch& B, const JointWs& W_, const JImg& I,
                                             FastSmem& F, int RW, int RV0, int RU0, int bi,
                                             int comp, bool incr, long long& e1) {
    constexpr int r = (S - 1) / 2, K = S * S;
    const int lane = threadIdx.x & 31;
    const int c = F.blocks[bi], off = F.pxoff[bi];
    const int bv = RV0 + c / RW, bu = RU0 + c % RW;
    uint32_t rm, cm;
    window_masks(bv, bu, I.h, I.w, S, rm, cm);
    const float4* win = &F.region[(bv - r - RV0) * RW + (bu - r - RU0)];
    // the replaced LR pixels in this block's window as a bit set over window indices (the same
    // in every lane of the warp, so the loops over it below run in step)
    constexpr int NW = (K + 31) / 32;
    uint32_t chg[NW];
    int nchg = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        chg[w] = 0u;
        if (incr) {
            const int k = w * 32 + lane;
            bool is = false;
            if (k < K)
                is = F.qmap[(bv - r + k / S - RV0) * RW + (bu - r + k % S - RU0)] != 0;
            chg[w] = __ballot_sync(0xffffffffu, is);
            nchg += __popc(chg[w]);
        }
    }
    auto changed = [&](int k) -> bool {
        uint32_t m = chg[0];
#pragma unroll
        for (int w = 1; w < NW; ++w)
            if ((k >> 5) == w) m = chg[w];
        return (m >> (k & 31)) & 1u;
    };
    const bool use_incr = incr && nchg <= kMaxChg;
    const int ys = bv * I.s, xs = bu * I.s;
    const int ey = min(I.s, I.H - ys), ex = min(I.s, I.W - xs);
    for (int jp0 = 0; jp0 < ey * ex; jp0 += 32) {
        const int jp = jp0 + lane;
        // queue decisions of the whole warp go out as one shared atomic per warp
        int want = -2;   // -2: none; -1: full search; >= 0: step 2 for this a
        int a = 0, b = 0;
        float bd = 0.f, ir = 0.f, ig = 0.f, ib = 0.f;
        float4 ca0 = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool live = jp < ey * ex && F.rcode[off + jp] != kNotSearched;
        if (live) {
            const uint32_t rgb = F.hrpx[off + jp];
            ir = (float)(rgb & 255u);
            ig = (float)((rgb >> 8) & 255u);
            ib = (float)(rgb >> 16);
            if (!use_incr) {
                want = -1;
            } else {
                const int code0 = (int)F.code0[off + jp];
                const int a0 = code0 / K, b0 = code0 % K;
                const bool redo_a = changed(a0), redo_b = changed(b0);
                if (redo_a) {
                    want = -1;
                } else {
                    // step 1 from the previous a: only a replaced pixel can be nearer
                    // (ties: lowest k)
                    ca0 = lds_f4(&win[(a0 / S) * RW + (a0 % S)]);
                    bd = dist2(ca0.x - ir, ca0.y - ig, ca0.z - ib);
                    a = a0;
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        for (uint32_t m = chg[w]; m; m &= m - 1u) {   // ascending window index
                            const int k = w * 32 + __ffs(m) - 1;
                            const float4 cc = lds_f4(&win[(k / S) * RW + (k % S)]);
                            const float d2 = dist2(cc.x - ir, cc.y - ig, cc.z - ib);
                            if (d2 < bd || (d2 == bd && k < a)) {
                                bd = d2;
                                a = k;
                            }
                        }
                    }
                    if (a != a0 || redo_b) want = a;
                    b = b0;
                }
            }
        }
        const unsigned q = __ballot_sync(0xffffffffu, want != -2);
        if (q) {
            int base = 0;
            if (lane == __ffs(q) - 1) base = atomicAdd(&F.nfull, __popc(q));
            base = __shfl_sync(0xffffffffu, base, __ffs(q) - 1);
            if (want != -2) F.full[base + __popc(q & ((1u << lane) - 1u))] = full_entry(off + jp, bi, want);
        }
        if (!live || want != -2) continue;
        // step 2 from the previous b: only a replaced pixel can beat it (ties: lowest k)
        const StepB sb = step_b_setup(ca0, bd, ir, ig, ib, B.eps255);
        const float4 cb0 = lds_f4(&win[(b / S) * RW + (b % S)]);
        float vr = cb0.x - ir, vg = cb0.y - ig, vb = cb0.z - ib;
        float bkey = b_key(sb, dist2(vr, vg, vb), vr, vg, vb);
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            for (uint32_t m = chg[w]; m; m &= m - 1u) {   // ascending window index
                const int k = w * 32 + __ffs(m) - 1;
                const float4 cc = lds_f4(&win[(k / S) * RW + (k % S)]);
                vr = cc.x - ir;
                vg = cc.y - ig;
                vb = cc.z - ib;
                const float key = b_key(sb, dist2(vr, vg, vb), vr, vg, vb);
                if (key < bkey || (key == bkey && k < b)) {
                    bkey = key;
                    b = k;
                }
            }
        }
        SearchOut o;
        o.ka = a;
        finish_pair(win, RW, S, b, ir, ig, ib, sb.dae, bkey, o);
        F.rcode[off + jp] = (uint16_t)(o.ka * K + o.kb);
        F.rw[off + jp] = o.omega;
        F.rerr[off + jp] = o.err;
        e1 += to_fixed(o.err);
    }
}

// Queued full searches (entries from fast_block_pass). While one round of the CTA covers them: a
// team of TEAM consecutive lanes per entry (4, 2 or 1: the widest that fits), each lane scanning
// every TEAM-th window candidate; the team reduces (value, k) lexicographically, which is exactly
// the first minimum the sequential scan finds (values compare exactly). More entries than
// threads: one thread per two entries, which
// run as one packed two-pixel search (search_pair_f4) when they lie in one block (they share the
// window), else one after the other (search_pixel). An entry whose a is known (step 1 decided it
// exactly: integer distances) skips step 1 in the team form and is searched in full in the
// packed form, which finds the same a: the results are those of the scalar search either way.
template <int TEAM>
__device__ __forceinline__ void team_min(float& v, int& k, unsigned mask) {
#pragma unroll
    for (int o = 1; o < TEAM; o <<= 1) {
        const float ov = __shfl_xor_sync(mask, v, o);
        const int ok = __shfl_xor_sync(mask, k, o);
        if (ov < v || (ov == v && ok < k)) {
            v = ov;
            k = ok;
        }
    }
}

__device__ __forceinline__ void full_put(FastSmem& F, int K, int pix, const SearchOut& o,
                                         long long& acc) {
    F.rcode[pix] = (uint16_t)(o.ka * K + o.kb);
    F.rw[pix] = o.omega;
    F.rerr[pix] = o.err;
    acc += to_fixed(o.err);
}

__device__ __forceinline__ void full_colour(const FastSmem& F, int pix, float& ir, float& ig,
                                            float& ib) {
    const uint32_t rgb = F.hrpx[pix];
    ir = (float)(rgb & 255u);
    ig = (float)((rgb >> 8) & 255u);
    ib = (float)(rgb >> 16);
}

template <int S>
__device__ __forceinline__ const float4* full_window(const JImg& I, const FastSmem& F, int RW,
                                                     int RV0, int RU0, int bi, uint32_t& rm,
                                                     uint32_t& cm) {
    constexpr int r = (S - 1) / 2;
    const int c = F.blocks[bi];
    const int bv = RV0 + c / RW, bu = RU0 + c % RW;
    window_masks(bv, bu, I.h, I.w, S, rm, cm);
    return &F.region[(bv - r - RV0) * RW + (bu - r - RU0)];
}

// One entry by a team of TEAM lanes (scalar arithmetic).
template <int S, int TEAM>
__device__ __noinline__ void fast_full_search(const JBatch& B, const JImg& I, FastSmem& F, int RW,
                                              int RV0, int RU0, int e, int tl, unsigned mask,
                                              long long& acc) {
    constexpr int K = S * S;
    const int pix = e & 0xFFF, bi = (e >> 12) & 0xFF;
    uint32_t rm, cm;
    const float4* win = full_window<S>(I, F, RW, RV0, RU0, bi, rm, cm);
    float ir, ig, ib;
    full_colour(F, pix, ir, ig, ib);
    float bd = kInf;
    int a = ((e >> 20) & 0xFF) - 1;   // >= 0: step 1 already decided a (exactly: integer distances)
    if (a >= 0) {
        const float4 ca = lds_f4(&win[(a / S) * RW + (a % S)]);
        bd = dist2(ca.x - ir, ca.y - ig, ca.z - ib);
    } else {
        a = K;
        for (int k = tl; k < K; k += TEAM) {
            const int dy = k / S, dx = k % S;
            if (!((rm >> dy) & (cm >> dx) & 1u)) continue;
            const float4 cc = lds_f4(&win[dy * RW + dx]);
            const float d2 = dist2(cc.x - ir, cc.y - ig, cc.z - ib);
            if (d2 < bd) {
                bd = d2;
                a = k;
            }
        }
        team_min<TEAM>(bd, a, mask);
    }
    const StepB sb = step_b_setup(lds_f4(&win[(a / S) * RW + (a % S)]), bd, ir, ig, ib, B.eps255);
    float bkey = kInf;
    int b = K;
    for (int k = tl; k < K; k += TEAM) {
        const int dy = k / S, dx = k % S;
        if (!((rm >> dy) & (cm >> dx) & 1u)) continue;
        const float4 cc = lds_f4(&win[dy * RW + dx]);
        const float vr = cc.x - ir, vg = cc.y - ig, vb = cc.z - ib;
        const float key = b_key(sb, dist2(vr, vg, vb), vr, vg, vb);
        if (key < bkey) {
            bkey = key;
            b = k;
        }
    }
    team_min<TEAM>(bkey, b, mask);
    if (tl == 0) {
        SearchOut o;
        o.ka = a;
        finish_pair(win, RW, S, b, ir, ig, ib, sb.dae, bkey, o);
        full_put(F, K, pix, o, acc);
    }
}

// Two entries by one thread (packed when they share the block).
template <int S>
__device__ __noinline__ void fast_full_pair(const JBatch& B, const JImg& I, FastSmem& F, int RW,
                                            int RV0, int RU0, int e0, int e1, long long& acc) {
    constexpr int K = S * S;
    const int pix0 = e0 & 0xFFF, bi0 = (e0 >> 12) & 0xFF;
    const int pix1 = e1 & 0xFFF, bi1 = e1 >= 0 ? (e1 >> 12) & 0xFF : -1;
    uint32_t rm, cm;
    const float4* win = full_window<S>(I, F, RW, RV0, RU0, bi0, rm, cm);
    float ir0, ig0, ib0;
    full_colour(F, pix0, ir0, ig0, ib0);
    if (bi1 == bi0) {
        float ir1, ig1, ib1;
        full_colour(F, pix1, ir1, ig1, ib1);
        SearchOut o0, o1;
        search_pair_f4<S>(win, RW, rm, cm, ir0, ig0, ib0, ir1, ig1, ib1, B.eps255, o0, o1);
        full_put(F, K, pix0, o0, acc);
        full_put(F, K, pix1, o1, acc);
        return;
    }
    full_put(F, K, pix0, search_pixel<S, true>(win, RW, rm, cm, ir0, ig0, ib0, B.eps255, false),
             acc);
    if (e1 < 0) return;
    win = full_window<S>(I, F, RW, RV0, RU0, bi1, rm, cm);
    float ir1, ig1, ib1;
    full_colour(F, pix1, ir1, ig1, ib1);
    full_put(F, K, pix1, search_pixel<S, true>(win, RW, rm, cm, ir1, ig1, ib1, B.eps255, false),
             acc);
}

constexpr int kSuccCache = 32;   // successors of a one-CTA trial's component staged for its commit

struct FastShared {
    int nq, vmin, vmax, umin, umax, na, npx, ok;
    unsigned long long e0, e1;
    int searched;
    int s0, s1;            // the component's successor range (s1 < 0: not staged)
    int sc[kSuccCache];    // its first successors
};

// Tries component j in this CTA if it fits (returns false, having changed nothing, if it does
// not). On return *accept holds the decision and the global state holds its outcome.
//
// stage: the iteration's dependency graph exists; the last warp then stages j's successor list
// in sh while the others write the kept trial out, so the commit does not wait for it.
__device__ bool fast_trial(const JBatch& B, const TrialCtx& X, const JImg& I, int img, int j,
                          int2 st, int2 en, FastSmem& F, FastShared& sh, int* accept,
                          bool stage) {
    const JointWs& W_ = X.ws;
    const int tid = threadIdx.x, warp = tid >> 5, nthr = blockDim.x, nwarps = nthr >> 5;
    const int r = (I.S - 1) / 2;
    const int Rm = B.strict ? 2 * r : r, Am = B.strict ? r : 0;
    const int nraw = en.y - st.y;
    if (tid == 0) sh.s1 = -1;   // read by the commit after later barriers
    if (nraw > kFastQRaw) return false;   // uniform: from global values every thread read
    if (tid == 0) {
        sh.nq = 0;
        sh.vmin = 0x7fffffff;
        sh.umin = 0x7fffffff;
        sh.vmax = -1;
        sh.umax = -1;
        sh.e0 = 0ull;
        sh.e1 = 0ull;
        sh.searched = 0;
        sh.ok = 1;
    }
    __syncthreads();
    // the component's LR blocks (repeats are possible where owner slots overflowed) and their
    // bounding box
    for (int t = tid; t < nraw; t += nthr) {
        const int q = (int)((int64_t)W_.qlist[st.y + t] - I.q0);
        F.rawq[t] = q;
        const int v = q / I.w, u = q % I.w;
        atomicMin(&sh.vmin, v);
        atomicMax(&sh.vmax, v);
        atomicMin(&sh.umin, u);
        atomicMax(&sh.umax, u);
    }
    __syncthreads();
    const int RV0 = sh.vmin - Rm, RU0 = sh.umin - Rm;
    const int RH = sh.vmax - sh.vmin + 1 + 2 * Rm, RW = sh.umax - sh.umin + 1 + 2 * Rm;
    if (RH * RW > kFastRegion) return false;
    // region maps: Q blocks (index + 1) and the blocks to re-search
    for (int t = tid; t < RH * RW; t += nthr) {
        F.qmap[t] = 0;
        F.amap[t] = 0;
    }
    __syncthreads();
    // distinct blocks Q: the first entry to claim a block's cell in the map numbers it (the
    // numbering order does not matter: only the block <-> index pairing is used)
    for (int t = tid; t < nraw; t += nthr) {
        const int q = F.rawq[t];
        const int cell = (q / I.w - RV0) * RW + (q % I.w - RU0);
        unsigned short* qm = reinterpret_cast<unsigned short*>(&F.qmap[cell]);
        if (atomicCAS(qm, (unsigned short)0, (unsigned short)0xFFFFu) != 0) continue;
        const int idx = atomicAdd(&sh.nq, 1);
        if (idx < kFastQ) {
            F.qs[idx] = q;
            F.qmap[cell] = (short)(idx + 1);
        }
    }
    __syncthreads();
    const int nq = sh.nq;
    if (nq > kFastQ) return false;
    const int NA = (2 * Am + 1) * (2 * Am + 1);
    for (int t = tid; t < nq * NA; t += nthr) {
        const int q = F.qs[t / NA], nb = t % NA;
        const int v = q / I.w + nb / (2 * Am + 1) - Am, u = q % I.w + nb % (2 * Am + 1) - Am;
        if (v >= 0 && v < I.h && u >= 0 && u < I.w) F.amap[(v - RV0) * RW + (u - RU0)] = 1;
    }
    __syncthreads();
    // the blocks to re-search in raster order, with their pixel offsets
    const int ncell = RH * RW;
    const int per = (ncell + nthr - 1) / nthr;
    const int c_beg = tid * per, c_end = min(c_beg + per, ncell);
    int myb = 0, mypx = 0;
    for (int c = c_beg; c < c_end; ++c) {
        if (!F.amap[c]) continue;
        const int bv = RV0 + c / RW, bu = RU0 + c % RW;
        ++myb;
        mypx += min(I.s, I.H - bv * I.s) * min(I.s, I.W - bu * I.s);
    }
    int bex, pex;
    const int na = block_excl_scan_any(myb, &bex, F.scan);
    const int npx = block_excl_scan_any(mypx, &pex, F.scan);
    if (na > kFastA || npx > kFastPx) return false;
    GLU_TRACE(X.it, j, 4);
    for (int c = c_beg, k = bex, o = pex; c < c_end; ++c) {
        if (!F.amap[c]) continue;
        const int bv = RV0 + c / RW, bu = RU0 + c % RW;
        F.blocks[k] = c;
        F.pxoff[k] = o;
        F.amap[c] = (short)(k + 1);
        ++k;
        o += min(I.s, I.H - bv * I.s) * min(I.s, I.W - bu * I.s);
    }
    const int ncomp = en.x - st.x;
    __syncthreads();
    // one round of loads: the LR neighbourhood in 1/255 units (zero outside the image: masked by
    // the search), every re-searched pixel's guide colour, error and pair (PAPER: its label),
    // and the component's pixel list
    for (int t = tid; t < ncell; t += nthr) {
        const int v = RV0 + t / RW, u = RU0 + t % RW;
        float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v >= 0 && v < I.h && u >= 0 && u < I.w) {
            const uint32_t c = load_rgb(I.lr, I.lr_pitch, v, u);
            c4 = make_float4((float)(c & 255u), (float)((c >> 8) & 255u), (float)(c >> 16), 0.f);
        }
        F.region[t] = c4;
    }
    // e0 (the searched pixels' previous errors, exact in 2^-32 units) and the number searched
    // are summed here; e1 as the searches finish
    long long acc0 = 0;
    int nsr = 0;
    for (int w0 = warp; w0 < na; w0 += nwarps) {
        const int c = F.blocks[w0], off = F.pxoff[w0];
        const int bv = RV0 + c / RW, bu = RU0 + c % RW;
        const int ys = bv * I.s, xs = bu * I.s;
        const int ey = min(I.s, I.H - ys), ex = min(I.s, I.W - xs);
        for (int jp = (tid & 31); jp < ey * ex; jp += 32) {
            const int y = ys + jp / ex, x = xs + jp % ex;
            const int64_t lp = (int64_t)y * I.W + x;
            const uint8_t* ip = I.hr + (int64_t)y * I.hr_pitch + (int64_t)x * 3;
            F.hrpx[off + jp] = (uint32_t)__ldg(ip) | ((uint32_t)__ldg(ip + 1) << 8) |
                               ((uint32_t)__ldg(ip + 2) << 16);
            const float eo = __ldcg(&I.err[lp]);
            F.eold[off + jp] = eo;
            F.code0[off + jp] = __ldcg(&I.code[lp]);
            const bool sr = B.strict || __ldcg(&W_.lab[I.p0 + lp]) == j;
            F.rcode[off + jp] = sr ? (uint16_t)0 : kNotSearched;
            if (sr) {
                acc0 += to_fixed(eo);
                ++nsr;
            }
        }
    }
    {
        const long long w0s = warp_sum_ll(acc0);
        int wn = nsr;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wn += __shfl_xor_sync(0xffffffffu, wn, o);
        if ((tid & 31) == 0 && wn) {
            atomicAdd(&sh.e0, (unsigned long long)w0s);
            atomicAdd(&sh.searched, wn);
        }
    }
    for (int t = tid; t < ncomp; t += nthr) F.full[t] = W_.comp_pix[st.x + t];
    for (int t = tid; t < nq; t += nthr) F.best[t] = 0ull;
    __syncthreads();
    // per q, the component's largest current error in the block (ties: lowest raster index)
    for (int t = tid; t < ncomp; t += nthr) {
        const int64_t lp = (int64_t)F.full[t] - I.p0;
        const int y = (int)(lp / I.W), x = (int)(lp % I.W);
        const int cell = (y / I.s - RV0) * RW + (x / I.s - RU0);
        const int ai = F.amap[cell] - 1;
        const int ex = min(I.s, I.W - (x / I.s) * I.s);
        const int pix = F.pxoff[ai] + (y % I.s) * ex + (x % I.s);
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(F.eold[pix]) << 32) |
            (unsigned long long)(0xFFFFFFFFu - (uint32_t)lp);
        atomicMax(&F.best[F.qmap[cell] - 1], key);
    }
    __syncthreads();
    // the replacement colours (guide colours of the argmax pixels), applied to the staged
    // neighbourhood only
    for (int t = tid; t < nq; t += nthr) {
        const uint32_t lp = 0xFFFFFFFFu - (uint32_t)(F.best[t] & 0xFFFFFFFFull);
        const int y = (int)(lp / (uint32_t)I.W), x = (int)(lp % (uint32_t)I.W);
        const int cell = (y / I.s - RV0) * RW + (x / I.s - RU0);
        const int ex = min(I.s, I.W - (x / I.s) * I.s);
        const uint32_t c = F.hrpx[F.pxoff[F.amap[cell] - 1] + (y % I.s) * ex + (x % I.s)];
        F.newc[t] = c;
        log_argmax(X, j, F.qs[t], (int)lp);
        F.region[cell] = make_float4((float)(c & 255u), (float)((c >> 8) & 255u),
                                     (float)(c >> 16), 0.f);
    }
    __syncthreads();
    GLU_TRACE(X.it, j, 5);
    // the trial: Algorithm 1 on the affected blocks
    const int comp = B.strict ? -1 : j;
    const bool incr = B.strict != 0;   // PAPER leaves Theta stale outside components: no re-search
    if (tid == 0) F.nfull = 0;
    __syncthreads();
    long long acc1 = 0;
    GLU_WSTAMP(X.it, j, 0);
    for (int bi = warp; bi < na; bi += nwarps) {
        switch (I.S) {
            case 1: fast_block_pass<1>(B, W_, I, F, RW, RV0, RU0, bi, comp, incr, acc1); break;
            case 3: fast_block_pass<3>(B, W_, I, F, RW, RV0, RU0, bi, comp, incr, acc1); break;
            case 5: fast_block_pass<5>(B, W_, I, F, RW, RV0, RU0, bi, comp, incr, acc1); break;
            case 7: fast_block_pass<7>(B, W_, I, F, RW, RV0, RU0, bi, comp, incr, acc1); break;
            default: fast_block_pass<9>(B, W_, I, F, RW, RV0, RU0, bi, comp, incr, acc1); break;
        }
    }
    GLU_WSTAMP(X.it, j, 1);
    __syncthreads();
    const int nfull = F.nfull;
    GLU_TRACE(X.it, j, 7);
#ifdef GLU_TRIAL_TRACE
    if (tid == 0 && j < kTraceMax) g_trace[X.it][j][9] = (unsigned long long)nfull;
#endif
    GLU_WSTAMP(X.it, j, 2);
    // one round of the CTA: teams of 4, 2 or 1 lanes per queued pixel (a CTA-uniform choice, see
    // fast_full_search); longer queues: one thread per two pixels (packed when they share a block)
    const int team = nfull <= nthr / 4 ? 4 : nfull <= nthr / 2 ? 2 : nfull <= nthr ? 1 : 0;
    auto teams = [&](auto tw) {
        constexpr int TW = decltype(tw)::value;
        const int tl = tid % TW;
        const unsigned mask = ((TW == 32 ? 0xFFFFFFFFu : (1u << TW) - 1u)) << ((tid & 31) - tl);
        for (int t = tid / TW; t < nfull; t += nthr / TW) {
            const int e = F.full[t];
            switch (I.S) {
                case 1: fast_full_search<1, TW>(B, I, F, RW, RV0, RU0, e, tl, mask, acc1); break;
                case 3: fast_full_search<3, TW>(B, I, F, RW, RV0, RU0, e, tl, mask, acc1); break;
                case 5: fast_full_search<5, TW>(B, I, F, RW, RV0, RU0, e, tl, mask, acc1); break;
                case 7: fast_full_search<7, TW>(B, I, F, RW, RV0, RU0, e, tl, mask, acc1); break;
                default: fast_full_search<9, TW>(B, I, F, RW, RV0, RU0, e, tl, mask, acc1); break;
            }
        }
    };
    if (team == 4) {
        teams(std::integral_constant<int, 4>());
    } else if (team == 2) {
        teams(std::integral_constant<int, 2>());
    } else if (team == 1) {
        teams(std::integral_constant<int, 1>());
    } else {
        for (int t = tid; 2 * t < nfull; t += nthr) {
            const int e0 = F.full[2 * t], e1 = 2 * t + 1 < nfull ? F.full[2 * t + 1] : -1;
            switch (I.S) {
                case 1: fast_full_pair<1>(B, I, F, RW, RV0, RU0, e0, e1, acc1); break;
                case 3: fast_full_pair<3>(B, I, F, RW, RV0, RU0, e0, e1, acc1); break;
                case 5: fast_full_pair<5>(B, I, F, RW, RV0, RU0, e0, e1, acc1); break;
                case 7: fast_full_pair<7>(B, I, F, RW, RV0, RU0, e0, e1, acc1); break;
                default: fast_full_pair<9>(B, I, F, RW, RV0, RU0, e0, e1, acc1); break;
            }
        }
    }
    GLU_WSTAMP(X.it, j, 3);
    GLU_WVAL(X.it, j, 4, na);
    GLU_WVAL(X.it, j, 5, nfull);
    {
        const long long w1 = warp_sum_ll(acc1);
        if ((tid & 31) == 0 && w1) atomicAdd(&sh.e1, (unsigned long long)w1);
    }
    __syncthreads();
    GLU_TRACE(X.it, j, 8);
    GLU_TRACE(X.it, j, 6);
    const bool keep = !((long long)sh.e1 > (long long)sh.e0);
    if (stage && warp == nwarps - 1) {
        const int lane = tid & 31;
        const int s0 = W_.dag_start[j].x, s1 = W_.dag_start[j + 1].x;
        for (int t = lane; t < min(s1 - s0, kSuccCache); t += 32) sh.sc[t] = W_.succ[s0 + t];
        if (lane == 0) {
            sh.s0 = s0;
            sh.s1 = s1;
        }
    }
    if (keep) {
        // write the kept trial: Theta / E of every re-searched pixel, then the LR colours
        for (int bi = warp; bi < na; bi += nwarps) {
            const int c = F.blocks[bi];
            const int bv = RV0 + c / RW, bu = RU0 + c % RW;
            const int ys = bv * I.s, xs = bu * I.s;
            const int ey = min(I.s, I.H - ys), ex = min(I.s, I.W - xs);
            const int off = F.pxoff[bi];
            for (int jp = (threadIdx.x & 31); jp < ey * ex; jp += 32) {
                const uint16_t code = F.rcode[off + jp];
                if (code == kNotSearched) continue;
                const int64_t lp = (int64_t)(ys + jp / ex) * I.W + xs + jp % ex;
                I.code[lp] = code;
                store_weight(I.weight, B.wfmt, lp, F.rw[off + jp]);
                I.err[lp] = F.rerr[off + jp];
            }
        }
        for (int t = tid; t < nq; t += nthr) {
            const int q = F.qs[t];
            store_rgb(I.lr, I.lr_pitch, q / I.w, q % I.w, F.newc[t]);
        }
    }
    if (tid == 0 && sh.searched)
        atomicAdd(&X.ws.ctl->searched[img][X.it], (unsigned long long)sh.searched);
    *accept = keep ? 1 : 0;
    return true;
}

// General path (components too large for fast_trial): in place with backup planes, block items
// shared with every idle warp of the grid, explicit rollback. Returns false on an exhausted wait.
__device__ bool big_trial(const JBatch& B, const TrialCtx& X, const JImg& I, int img, int j,
                          int2 st, int2 en, float4* win, int G, int* s_nu, int* s_na,
                          unsigned long long* s_e0, unsigned long long* s_e1, int* s_flag,
                          int* accept, unsigned long long deadline) {
    const JointWs& W_ = X.ws;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int r = (I.S - 1) / 2;
    if (tid == 0) {
        *s_nu = 0;
        *s_na = 0;
        *s_e0 = 0ull;
        *s_e1 = 0ull;
        *s_flag = 0;
    }
    __syncthreads();
    // the distinct LR blocks Q of the component (stamps drop duplicates)
    const unsigned long long tagQ = trial_tag(X.it, j, 0);
    for (int t = st.y + tid; t < en.y; t += nthr) {
        const int q = W_.qlist[t];
        if (atomicExch(&W_.stamp[q], tagQ) != tagQ) {
            const int u = atomicAdd(s_nu, 1);
            W_.ulist[st.y + u] = q;
            W_.best[q] = 0ull;
        }
    }
    __syncthreads();
    const int nu = *s_nu;
    // per q, the largest current error among the component's pixels in its block
    // (ties: lowest raster index)
    for (int t = st.x + tid; t < en.x; t += nthr) {
        const int p = W_.comp_pix[t];
        const int64_t lp = p - I.p0;
        const int y = (int)(lp / I.W), x = (int)(lp % I.W);
        const int64_t q = I.q0 + (int64_t)(y / I.s) * I.w + (x / I.s);
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(__ldcg(&I.err[lp])) << 32) |
            (unsigned long long)(0xFFFFFFFFu - (uint32_t)lp);
        atomicMax(&W_.best[q], key);
    }
    __syncthreads();
    // back up and replace the LR colours
    for (int t = tid; t < nu; t += nthr) {
        const int64_t lq = (int64_t)W_.ulist[st.y + t] - I.q0;
        const int qv = (int)(lq / I.w), qu = (int)(lq % I.w);
        const uint32_t lp = 0xFFFFFFFFu - (uint32_t)(__ldcg(&W_.best[I.q0 + lq]) & 0xFFFFFFFFull);
        const int y = (int)(lp / (uint32_t)I.W), x = (int)(lp % (uint32_t)I.W);
        W_.backup[I.q0 + lq] = load_rgb(I.lr, I.lr_pitch, qv, qu);
        log_argmax(X, j, (int)lq, (int)lp);
        const uint8_t* ip = I.hr + (int64_t)y * I.hr_pitch + (int64_t)x * 3;
        store_rgb(I.lr, I.lr_pitch, qv, qu,
                  (uint32_t)ip[0] | ((uint32_t)ip[1] << 8) | ((uint32_t)ip[2] << 16));
    }
    // STRICT: every affected block (within r of Q) gets one owner among the block items that
    // reach it; the owners also go to this slot's A list, so that the tasks claim only items
    // with work (without the list, most (block, neighbour) items find another owner)
    const int NB = (2 * r + 1) * (2 * r + 1);
    const bool listed = B.strict && blockIdx.x < kListSlots;
    if (B.strict) {
        const unsigned long long tagA = trial_tag(X.it, j, 1);
        int* al = W_.alist + (int64_t)blockIdx.x * kSlotA;
        for (int t = tid; t < nu * NB; t += nthr) {
            int bv, bu;
            if (!item_block(B, X, I, st.y, t, bv, bu)) continue;
            const int64_t b = I.q0 + (int64_t)bv * I.w + bu;
            if (atomicExch(&W_.stamp[b], tagA) != tagA) {
                W_.bown[b] = t;
                if (listed) {
                    const int k = atomicAdd(s_na, 1);
                    if (k < kSlotA) al[k] = bv * I.w + bu;
                }
            }
        }
    }
    // visible to this CTA after the barrier, and to helpers through the fence thread 0 issues
    // before it publishes the task (cumulative over what the barrier ordered before it)
    __syncthreads();
    // trial: Algorithm 1 again on the affected pixels (STRICT: every block within r of Q; PAPER:
    // the component's own pixels), in place, summing e0 and e1; every block in several items
    const bool use_list = listed && *s_na <= kSlotA;
    const int nitems = (use_list ? *s_na : B.strict ? nu * NB : nu) * block_chunks(I);
    const int lk = use_list ? 2 : 0;
    GLU_TRACE(X.it, j, 4);
#ifdef GLU_TRIAL_TRACE
    if (tid == 0 && j < kTraceMax) g_trace[X.it][j][9] = (unsigned long long)nitems;
#endif
    bool ok = run_task(B, X, win, j, img, st.y, lk, nitems, G, s_e0, s_e1, s_flag, deadline);
    GLU_TRACE(X.it, j, 5);
    const bool keep = !((long long)*s_e1 > (long long)*s_e0);
    __syncthreads();
    // keep (the results are in place) or roll back: Theta and E from the backup planes, the LR
    // colours from their backups
    if (!keep && ok) {
        ok = run_task(B, X, win, j, img, st.y, 1 | lk, nitems, G, s_e0, s_e1, s_flag, deadline);
        GLU_TRACE(X.it, j, 7);
        for (int t = tid; t < nu; t += nthr) {
            const int64_t lq = (int64_t)W_.ulist[st.y + t] - I.q0;
            store_rgb(I.lr, I.lr_pitch, (int)(lq / I.w), (int)(lq % I.w), W_.backup[I.q0 + lq]);
        }
    }
    *accept = keep ? 1 : 0;
    return ok;
}

// The persistent trial kernel. With the dependency graph (the normal case) a CTA takes the next
// position of the ready queue, waits until a component is published there and tries it; when it
// finishes, every successor whose last predecessor it was enters the queue. Without it (graph
// too large for the workspace) components are claimed in index order and each waits for its
// earlier neighbours. Waiting warps help with the block items of large components' trials.
__global__ void __launch_bounds__(kTrialThreads, 1)
    k_trials(const __grid_constant__ JBatch B, const TrialCtx X) {
    constexpr int kPend = 512;
    JointCtl* ctl = X.ws.ctl;
    if (!any_active(ctl)) return;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    FastSmem& F = *reinterpret_cast<FastSmem*>(dyn_smem);
    __shared__ float4 wins[kTrialThreads / 32][kSmax * kSmax];
    __shared__ int s_j, s_idx, s_nu, s_na, s_accept, s_flag, s_npend, s_povf, s_next;
    __shared__ int s_pend[kPend];
    __shared__ unsigned long long s_e0, s_e1;
    __shared__ FastShared sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    bool no_own = false;   // help_one: this CTA has no task of its own open here
    const int G = gridDim.x;
    const int M = ctl->M_cur;
    const JointWs& W_ = X.ws;
    float4* win = wins[warp];
    const unsigned long long deadline =
        now_ns() + (X.wait_limit_ns ? X.wait_limit_ns : trial_deadline(M));
    const bool dag = *(volatile int*)&ctl->dag_bad[X.it] == 0;
    bool stop = false;
    int next = -1;   // a successor this CTA made ready itself: tried next, without the queue

    while (!stop) {
        int j;
        if (dag && next >= 0) {
            j = next;
        } else if (dag) {
            if (tid == 0) {
                s_idx = atomicAdd(&ctl->head[X.it], 1);
                s_flag = 0;
            }
            __syncthreads();
            const int idx = s_idx;
            if (idx >= M) break;
            // wait for the component published at this position, helping meanwhile: thread 0
            // polls closely while no large trial has items open, then the CTA helps a round
            int hint = -1;
            for (;;) {
                if (tid == 0) {
                    int v = -1;
                    for (int k = 0; k < 64; ++k) {
                        v = ld_acquire(&W_.queue[idx]);
                        if (v >= 0 || *(volatile const int*)&ctl->open_tasks > 0) break;
                        // components taken by continuation never pass through the queue: a
                        // position can stay empty, and every component may already be done
                        if (*(volatile const int*)&ctl->finished[X.it] >= M) {
                            v = -2;
                            break;
                        }
                        __nanosleep(32);
                    }
                    s_j = v;
                }
                __syncthreads();
                if (s_j >= 0 || s_j == -2) break;
                if (!help_one(B, X, win, blockIdx.x, G, hint, no_own)) __nanosleep(200);
                if (__syncthreads_or(warp_should_abort(ctl, deadline) ? 1 : 0)) {
                    if (tid == 0) s_flag = 1;
                    __syncthreads();
                    break;
                }
            }
            if (s_flag) {
                if (tid == 0) {
                    set_status(GLU_ERR_TIMEOUT);
                    atomicExch(&ctl->timeout, 1);
                }
                break;
            }
            if (s_j == -2) break;
            j = s_j;
        } else {
            if (tid == 0) {
                s_j = atomicAdd(&ctl->claim[X.it], 1);
                s_flag = 0;
                s_npend = 0;
                s_povf = 0;
            }
            __syncthreads();
            j = s_j;
            if (j >= M) break;
            GLU_TRACE(X.it, j, 0);
            const int2 st = W_.start[j], en = W_.start[j + 1];
            const JImg& I = B.im[img_of_p(B, W_.roots[j])];
            const int r = (I.S - 1) / 2;
            const int D = B.strict ? 2 * r : r;
            const int ND = (2 * D + 1) * (2 * D + 1);
            // the earlier components whose LR blocks lie within D of ours and are not done yet
            const int npairs = (en.y - st.y) * ND;
            for (int t = tid; t < npairs; t += kTrialThreads) {
                const int64_t lq = (int64_t)W_.qlist[st.y + t / ND] - I.q0;
                const int nb = t % ND;
                const int bv = (int)(lq / I.w) + nb / (2 * D + 1) - D;
                const int bu = (int)(lq % I.w) + nb % (2 * D + 1) - D;
                if (bv < 0 || bv >= I.h || bu < 0 || bu >= I.w) continue;
                const int64_t b = I.q0 + (int64_t)bv * I.w + bu;
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
                    if (!help_one(B, X, win, blockIdx.x, G, hint, no_own)) __nanosleep(200);
                    if (__syncthreads_or(warp_should_abort(ctl, deadline) ? 1 : 0)) {
                        if (tid == 0) s_flag = 1;
                        break;
                    }
                }
            }
            __syncthreads();
            if (s_flag) {
                if (tid == 0) {
                    set_status(GLU_ERR_TIMEOUT);
                    atomicExch(&ctl->timeout, 1);
                    st_release(&W_.done[j], 1);  // never leave a later component waiting on us
                    atomicAdd(&ctl->finished[X.it], 1);
                }
                __syncthreads();
                continue;
            }
        }
        GLU_TRACE(X.it, j, 1);
        const int2 st = W_.start[j], en = W_.start[j + 1];
        const int img = img_of_p(B, W_.roots[j]);
        const JImg& I = B.im[img];
        int accept = 0;
        bool ok = true;
        const bool fast = fast_trial(B, X, I, img, j, st, en, F, sh, &accept, dag);
        if (!fast)
            ok = big_trial(B, X, I, img, j, st, en, win, G, &s_nu, &s_na, &s_e0, &s_e1, &s_flag,
                           &accept, deadline);
        if (tid == 0) s_accept = accept;
        GLU_TRACE(X.it, j, 2);
#ifdef GLU_TRIAL_TRACE
        if (tid == 0 && j < kTraceMax) {
            g_trace[X.it][j][14] = fast ? 1ull : 2ull;
            g_trace[X.it][j][15] = (unsigned long long)blockIdx.x;
        }
#endif
        // the outcome is visible before any successor can start: every write precedes the
        // barrier, and each thread that publishes (a successor, the done flag) does so with
        // release semantics after it
        __syncthreads();
        if (tid == 0) {
            if (!ok) {
                set_status(GLU_ERR_TIMEOUT);
                atomicExch(&ctl->timeout, 1);
            }
            W_.dlog[(int64_t)X.it * W_.mcap + j] = (int8_t)(s_accept ? 1 : 0);
            if (s_accept) {
                atomicAdd(&ctl->accepted[img][X.it], 1);
                // the running residual: exact, since e0 / e1 and R sum the same rounded errors
                const unsigned long long d = fast ? sh.e1 - sh.e0 : s_e1 - s_e0;
                if (d) atomicAdd(&ctl->racc[img], d);
            } else {
                atomicAdd(&ctl->rolled[img][X.it], 1);
            }
        }
        if (dag) {
            if (tid == 0) s_next = -1;
            __syncthreads();
            const bool staged = sh.s1 >= 0;   // by the one-CTA trial (written before a barrier)
            const int s0 = staged ? sh.s0 : W_.dag_start[j].x;
            const int s1 = staged ? sh.s1 : W_.dag_start[j + 1].x;
            for (int k = s0 + tid; k < s1; k += kTrialThreads) {
                const int sj = (staged && k - s0 < kSuccCache) ? sh.sc[k - s0] : W_.succ[k];
                // release: this CTA's writes before the count drops; acquire: the other
                // predecessors' writes
                if (atom_add_acq_rel(&W_.pend[sj], -1) == 1) {
                    GLU_TRACE_ANY(X.it, sj, 0);   // the time it became ready
#ifdef GLU_TRIAL_TRACE
                    if (sj < kTraceMax) g_trace[X.it][sj][12] = (unsigned long long)(j + 1);
#endif
                    // the first successor this CTA made ready is tried here next; the others
                    // go to the queue
                    if (atomicCAS(&s_next, -1, sj) != -1) {
                        const int pos = atomicAdd(&ctl->tail[X.it], 1);
                        st_release(&W_.queue[pos], sj);
                    }
                }
            }
        }
        if (tid == 0) {
            // done[] is read only by the in-order fallback (no dependency graph)
            if (!dag) st_release(&W_.done[j], 1);
            atomicAdd(&ctl->finished[X.it], 1);
        }
        GLU_TRACE(X.it, j, 3);
        if (!ok) stop = true;
        __syncthreads();
        next = dag ? s_next : -1;
    }
    // no component left to take: help the running ones until every component is done
    // (per warp; lane 0 decides)
    const int lane = tid & 31;
    int hint = -1;
    for (;;) {
        int fin = 0;
        if (lane == 0) fin = *(volatile const int*)&ctl->finished[X.it] >= M;
        if (__shfl_sync(0xffffffffu, fin, 0)) break;
        if (!help_one(B, X, win, blockIdx.x, G, hint, no_own)) __nanosleep(200);
        if (warp_should_abort(ctl, deadline)) break;
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

// Opt-in shared memory of the one-CTA list kernel (once per process).
static int small_comp_setup() {
    static std::once_flag once;
    static int rc = GLU_OK;
    std::call_once(once, [] {
        if (cudaFuncSetAttribute(k_small_comp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(SmallSmem)) != cudaSuccess)
            rc = GLU_ERR_CUDA;
        // k_deps: four CTAs per SM (its whole grid resident) need the largest shared-memory split
        if (cudaFuncSetAttribute(k_deps, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            rc = GLU_ERR_CUDA;
    });
    return rc;
}

static int launch_trials(const JBatch& B, const TrialCtx& X, cudaStream_t st) {
    static std::atomic<int> blocks_per_sm{-1};   // the same on every device of one kind
    const size_t smem = sizeof(FastSmem);
    int bps = blocks_per_sm.load();
    if (bps < 0) {
        if (cudaFuncSetAttribute(k_trials, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return GLU_ERR_CUDA;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trials, kTrialThreads, smem) !=
            cudaSuccess)
            return GLU_ERR_CUDA;
        bps = nb > 0 ? nb : 1;
        blocks_per_sm.store(bps);
    }
    int grid = sm_count() * bps;
    if (grid > kMaxSlots) grid = kMaxSlots;
    k_trials<<<grid, kTrialThreads, smem, st>>>(B, X);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

// ---------------------------------------------------------------- phase-timing instrumentation
namespace prof {
// Slots 0 .. kSlots-1: calls issued directly; slot kSlots: the events inside the recorded graph
// (external event nodes, recorded again at every replay; each replay's times are collected
// before the next replay is launched).
constexpr int kSlots = 64, kGraphSlot = kSlots, kMaxEv = 4 + 3 * GLU_MAX_ITERS;
static bool enabled = false;
static cudaEvent_t ev[kSlots + 1][kMaxEv];
static int nev[kSlots + 1];
static int used = 0;           // direct slots filled since the last read
static bool created = false;
static bool graph_pending = false;
static float gacc[5];
static int gcalls = 0;

static void mark(int slot, int i, cudaStream_t st) {
    if (slot < 0) return;
    if (slot == kGraphSlot) cudaEventRecordWithFlags(ev[slot][i], st, cudaEventRecordExternal);
    else cudaEventRecord(ev[slot][i], st);
}

// Phase times of one slot's events: [control init + grid downsample, search, components,
// trials, residuals].
static int phase_times(int sl, float ms[5]) {
    for (int k = 0; k < 5; ++k) ms[k] = 0.f;
    const int n = nev[sl];
    if (n < 4) return GLU_ERR_INVALID_ARG;
    if (cudaEventSynchronize(ev[sl][n - 1]) != cudaSuccess) return GLU_ERR_CUDA;
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[sl][0], ev[sl][1]);
    ms[0] += t;
    cudaEventElapsedTime(&t, ev[sl][1], ev[sl][2]);
    ms[1] += t;
    cudaEventElapsedTime(&t, ev[sl][2], ev[sl][3]);
    ms[4] += t;
    // per iteration: [previous end .. components built] [.. trials] [.. residual]
    for (int i = 3; i + 3 <= n - 1; i += 3) {
        cudaEventElapsedTime(&t, ev[sl][i], ev[sl][i + 1]);
        ms[2] += t;
        cudaEventElapsedTime(&t, ev[sl][i + 1], ev[sl][i + 2]);
        ms[3] += t;
        cudaEventElapsedTime(&t, ev[sl][i + 2], ev[sl][i + 3]);
        ms[4] += t;
    }
    return GLU_OK;
}

// Adds the last graph replay's phase times to the running sums (waits for that replay).
static int collect_graph() {
    if (!graph_pending) return GLU_OK;
    graph_pending = false;
    float t[5];
    const int rc = phase_times(kGraphSlot, t);
    if (rc) return rc;
    for (int k = 0; k < 5; ++k) gacc[k] += t[k];
    ++gcalls;
    return GLU_OK;
}
}  // namespace prof

#ifdef GLU_TRIAL_TRACE
// Trace build: an event after every launch of a directly issued call (glu_dbg_marks reads them).
namespace dbgm {
constexpr int kMax = 1024;
static cudaEvent_t ev[kMax];
static int tag[kMax];
static int n = 0;
static bool on = false;
static void mark(cudaStream_t st, int t) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!on || n >= kMax || cudaStreamIsCapturing(st, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
        return;
    if (!ev[n]) cudaEventCreate(&ev[n]);
    tag[n] = t;
    cudaEventRecord(ev[n++], st);
}
}  // namespace dbgm
#define GLU_DBG_MARK(st, t) dbgm::mark(st, t)
#else
#define GLU_DBG_MARK(st, t)
#endif

// Every launch of one Algorithm 2 call on `st` (phase events into profiling slot `slot`, if
// >= 0). The sequence depends only on the arguments: iterations after an image's convergence
// still launch and return at once, so the sequence can be replayed as a CUDA graph.
// body: a second stream when `st` is recording a graph (the multi-kernel list path of every
// iteration then goes into a conditional node that the one-CTA kernel switches off), else null.
static int issue_joint(const JointItem* items, int n, const JointCommon& cm, const JointWs& ws,
                       int64_t np, int64_t nq, int slot, cudaStream_t st,
                       cudaStream_t body = nullptr) {
    int evi = 0;

    JBatch B;   // host staging of the parameter block (copied into each launch)
    memset(&B, 0, sizeof(B));
    int64_t p0 = 0, q0 = 0;
    int c0 = 0;
    for (int k = 0; k < n; ++k) {
        const JointItem& a = items[k];
        JImg& I = B.im[k];
        I.hr = a.hr;
        I.hr_pitch = a.hr_pitch;
        I.lr = a.lr;
        I.lr_pitch = a.lr_pitch;
        I.code = a.code;
        I.weight = a.weight;
        I.err = a.err ? a.err : ws.err + p0;
        I.H = a.H; I.W = a.W; I.s = a.s; I.S = a.S;
        I.h = (a.H + a.s - 1) / a.s;
        I.w = (a.W + a.s - 1) / a.s;
        I.p0 = p0;
        I.q0 = q0;
        I.c0 = c0;
        p0 += (int64_t)a.H * a.W;
        q0 += (int64_t)I.h * I.w;
        c0 += (int)(((int64_t)a.H * a.W + kResidChunk - 1) / kResidChunk);
    }
    B.n = n;
    B.wfmt = cm.wfmt;
    B.strict = cm.strict;
    B.conn = cm.conn;
    B.eps255 = cm.eps255;
    B.tau = cm.tau;
    B.np = np;
    B.nq = nq;
    B.nchunks = c0;
    const int T = 256;

    {
        const int rc0 = small_comp_setup();
        if (rc0) return rc0;
    }
    prof::mark(slot, evi++, st);
    k_ctl_init<<<grid_cap(nq > kMaxSlots ? nq : kMaxSlots, T), T, 0, st>>>(
        ws.ctl, ws.stamp, nq, ws.slot_word, n, ws.tcnt,
        (((np + kScanTile - 1) / kScanTile + 1) + 3) & ~(int64_t)3);
    GLU_DBG_MARK(st, 1);
    // initialise every LR image by regular grid downsampling, Theta and E by Algorithm 1
    k_grid_batch<<<grid_cap(nq, T), T, 0, st>>>(B);
    GLU_DBG_MARK(st, 2);
    GLU_LAUNCH_CHECK();
    SearchArgs sa[kMaxJointBatch];
    for (int k = 0; k < n; ++k) {
        const JImg& I = B.im[k];
        SearchArgs& a = sa[k];
        a.hr = I.hr; a.hr_pitch = I.hr_pitch; a.hr_dtype = GLU_U8;
        a.lr = I.lr; a.lr_pitch = I.lr_pitch; a.lr_dtype = GLU_U8;
        a.H = I.H; a.W = I.W; a.h = I.h; a.w = I.w; a.s = I.s; a.S = I.S;
        a.eps255 = cm.eps255; a.gnu = 0;
        a.code = I.code; a.weight = I.weight; a.wfmt = cm.wfmt; a.err = I.err;
    }
    prof::mark(slot, evi++, st);
    int rc = launch_search_batch(sa, n, st);
    GLU_DBG_MARK(st, 3);
    if (rc) return rc;
    prof::mark(slot, evi++, st);
    k_resid_partial<<<B.nchunks, 256, 0, st>>>(B, ws.ctl);
    GLU_DBG_MARK(st, 4);
    k_resid_final<<<1, 32, 0, st>>>(B, ws.ctl, -1);
    GLU_DBG_MARK(st, 5);
    GLU_LAUNCH_CHECK();
    prof::mark(slot, evi++, st);

    const int tiles_a = (int)((np + kScanTile - 1) / kScanTile);
    int wmax = 1, hmax = 1;
    for (int k = 0; k < n; ++k) {
        wmax = std::max(wmax, B.im[k].W);
        hmax = std::max(hmax, B.im[k].H);
    }
    const dim3 ccl_grid((wmax + 8 * kCclTile - 1) / (8 * kCclTile), (hmax + kCclTile - 1) / kCclTile,
                        n);
    const int tiles_b = (int)((ws.mcap + kScanTile - 1) / kScanTile);
    // the list passes over tiles of the large-error list or of the components: grid-stride
    // over a small grid (the lists are short after the first iteration)
    const int list_grid_a = std::min(tiles_a, 2 * sm_count());
    const int list_grid_b = std::min(tiles_b, 2 * sm_count());
    TrialCtx X;
    X.ws = ws;
    X.wait_limit_ns = cm.wait_limit_ns;
    X.alog = cm.argmax_log;
    X.alog_cap = cm.argmax_cap;

    for (int it = 0; it < cm.N; ++it) {
        // large-error set, its ordered list, and its components (the list is the Q-list
        // scratch of the trials, free until then)
        int* fgl = ws.ulist;
        const int lgrid = 2 * sm_count();   // list passes: a thread per large-error pixel or so
        k_threshold_count<<<tiles_a, kScanThreads, 0, st>>>(B, ws, it, it == 0 ? 1 : 0,
                                                             cm.argmax_log, cm.argmax_cap);
        GLU_DBG_MARK(st, 6);
        k_threshold_write<<<tiles_a, kScanThreads, 0, st>>>(ws);
        GLU_DBG_MARK(st, 7);
        // a short list: the whole phase in one CTA, and the multi-kernel path below is skipped:
        // inside a recorded graph by a conditional node, otherwise its kernels return at once
        cudaGraphConditionalHandle cond = 0;
        cudaStream_t ls = st;   // the stream of the multi-kernel path
        if (body) {
            cudaStreamCaptureStatus cs;
            cudaGraph_t g = nullptr;
            GLU_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g));
            if (cs != cudaStreamCaptureStatusActive || !g) return GLU_ERR_CUDA;
            GLU_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault));
        }
        k_small_comp<<<1, kSmallThreads, sizeof(SmallSmem), st>>>(B, ws, it, cond, body ? 1 : 0);
        GLU_DBG_MARK(st, 8);
        if (body) {
            cudaStreamCaptureStatus cs;
            cudaGraph_t g = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            const cudaGraphEdgeData* edata = nullptr;
            size_t nd = 0;
            GLU_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edata, &nd));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = cond;
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 1;
            cudaGraphNode_t node = nullptr;
            GLU_CUDA_TRY(cudaGraphAddNode(&node, g, deps, edata, nd, &cp));
            GLU_CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                                             cudaStreamSetCaptureDependencies));
            GLU_CUDA_TRY(cudaStreamBeginCaptureToGraph(body, cp.conditional.phGraph_out[0], nullptr,
                                                       nullptr, 0, cudaStreamCaptureModeRelaxed));
            ls = body;
        }
        k_ccl_local<<<ccl_grid, 256, 0, ls>>>(B, ws);
        GLU_DBG_MARK(ls, 27);
        k_ccl_merge<<<lgrid, T, 0, ls>>>(B, ws.lab, fgl, ws.ctl);
        GLU_DBG_MARK(ls, 9);
        k_ccl_flatten<<<lgrid, T, 0, ls>>>(ws.lab, fgl, ws.ctl);
        GLU_DBG_MARK(ls, 10);
        k_root_count<<<list_grid_a, kScanThreads, 0, ls>>>(ws.lab, fgl, ws.tile_a, ws.ctl);
        GLU_DBG_MARK(ls, 11);
        k_tile_scan<1><<<1, kScanThreads, 0, ls>>>(ws.tile_a, tiles_a, ws.ctl);
        GLU_DBG_MARK(ls, 12);
        k_root_scatter<<<list_grid_a, kScanThreads, 0, ls>>>(B, ws.lab, fgl, ws.tile_a, ws.roots,
                                                         ws.cnt, ws.fill, ws.done, ws.dag_cnt,
                                                         ws.dag_fill, ws.queue, ws.ctl, it);
        GLU_DBG_MARK(ls, 13);
        k_comp_count<<<lgrid, T, 0, ls>>>(B, ws.lab, fgl, ws.roots, ws.cnt, ws.own,
                                                         ws.ovf, ws.qflag, ws.ctl);
        GLU_DBG_MARK(ls, 14);
        k_comp_tile_reduce<<<list_grid_b, kScanThreads, 0, ls>>>(ws.cnt, ws.tile_b, ws.ctl);
        GLU_DBG_MARK(ls, 15);
        k_comp_tile_scan<<<1, kScanThreads, 0, ls>>>(ws.tile_b, ws.ctl);
        GLU_DBG_MARK(ls, 16);
        k_comp_scan<<<list_grid_b, kScanThreads, 0, ls>>>(ws.cnt, ws.tile_b, ws.start, ws.ctl);
        GLU_DBG_MARK(ls, 17);
        k_comp_fill<<<lgrid, T, 0, ls>>>(B, ws.lab, fgl, ws.qflag, ws.start,
                                                        ws.fill, ws.comp_pix, ws.qlist, ws.ctl);
        GLU_DBG_MARK(ls, 18);
        // the trials' dependency graph
        k_deps<<<grid_cap(ws.mcap, 1, 4), 256, 0, ls>>>(B, ws, it);
        GLU_DBG_MARK(ls, 19);
        k_comp_tile_reduce<<<list_grid_b, kScanThreads, 0, ls>>>(ws.dag_cnt, ws.tile_b, ws.ctl);
        GLU_DBG_MARK(ls, 20);
        k_comp_tile_scan<<<1, kScanThreads, 0, ls>>>(ws.tile_b, ws.ctl);
        GLU_DBG_MARK(ls, 21);
        k_comp_scan<<<list_grid_b, kScanThreads, 0, ls>>>(ws.dag_cnt, ws.tile_b, ws.dag_start, ws.ctl);
        GLU_DBG_MARK(ls, 22);
        k_edge_scatter<<<list_grid_b, 256, 0, ls>>>(B, ws, it);
        GLU_DBG_MARK(ls, 23);
        GLU_LAUNCH_CHECK();
        if (body) {
            cudaGraph_t done = nullptr;
            GLU_CUDA_TRY(cudaStreamEndCapture(body, &done));
        }
        prof::mark(slot, evi++, st);
        X.it = it;
        rc = launch_trials(B, X, st);
        GLU_DBG_MARK(st, 24);
        if (rc) return rc;
        k_lists_clear<<<list_grid_a, kScanThreads, 0, st>>>(ws);
        GLU_DBG_MARK(st, 25);
        prof::mark(slot, evi++, st);
        // R_{it+1} = R_it + the kept trials' differences (added by the trials themselves)
        k_resid_final<<<1, 32, 0, st>>>(B, ws.ctl, it);
        GLU_DBG_MARK(st, 26);
        GLU_LAUNCH_CHECK();
        prof::mark(slot, evi++, st);
    }
    if (slot >= 0) prof::nev[slot] = evi;
    return GLU_OK;
}

// One recorded call: the arguments it was recorded for and its executable graph.
struct JointGraph {
    bool valid, profiled;
    int device, n, seen;
    JointItem items[kMaxJointBatch];
    JointCommon cm;
    void* ws;
    size_t ws_bytes;
    cudaGraphExec_t exec;
};

static bool same_call(const JointGraph& g, int device, const JointItem* items, int n,
                      const JointCommon& cm, void* ws, size_t ws_bytes) {
    return g.device == device && g.n == n && g.ws == ws && g.ws_bytes == ws_bytes &&
           memcmp(&g.cm, &cm, sizeof(cm)) == 0 &&
           memcmp(g.items, items, sizeof(JointItem) * (size_t)n) == 0;
}

static std::atomic<long long> g_graphs_recorded{0};
long long joint_graphs_recorded() { return g_graphs_recorded.load(); }

// Copies the control block's statistics to the host records (synchronises st).
static int read_stats(const JointWs& ws, int n, glu_joint_stats* stats, cudaStream_t st) {
    std::unique_ptr<JointCtl> h(new JointCtl);
    GLU_CUDA_TRY(cudaMemcpyAsync(h.get(), ws.ctl, sizeof(JointCtl), cudaMemcpyDeviceToHost, st));
    GLU_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i) {
        glu_joint_stats& o = stats[i];
        memset(&o, 0, sizeof(o));
        o.iterations = h->iterations[i];
        for (int k = 0; k < GLU_MAX_ITERS; ++k) {
            o.n_large[k] = h->n_large[i][k];
            o.components[k] = h->M[i][k];
            o.accepted[k] = h->accepted[i][k];
            o.rolled_back[k] = h->rolled[i][k];
            o.searched[k] = (int64_t)h->searched[i][k];
        }
        o.multi_kernel_lists = (uint32_t)h->multi_lists;
        for (int k = 0; k <= h->iterations[i] && k <= GLU_MAX_ITERS; ++k)
            o.residual[k] = h->residual[i][k];
    }
    return h->timeout ? GLU_ERR_TIMEOUT : GLU_OK;
}

int launch_joint_batch(const JointItem* items, int n, const JointCommon& cm, void* wsp,
                       size_t ws_bytes, glu_joint_stats* stats, cudaStream_t st) {
    if (n <= 0) return GLU_OK;
    if (n > kMaxJointBatch) return GLU_ERR_UNSUPPORTED;
    // the graph cache, the capture stream and the profiling slots are shared by every call
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    int64_t np, nq, nch;
    batch_sizes(items, n, &np, &nq, &nch);
    if (np >= (int64_t)0x7fffffff) return GLU_ERR_UNSUPPORTED;  // 32-bit pixel ids
    JointWs ws;
    const size_t need = carve(wsp, np, nq, n, cm.N, nch, &ws);
    if (ws_bytes < need) return GLU_ERR_WORKSPACE;
    // Launch gaps dominate the small kernels of late iterations: a call repeated with the same
    // arguments is recorded as a CUDA graph on its second occurrence (the first runs directly,
    // so the autotuner can time its kernels) and replayed from then on. Profiling runs directly.
    JointItem key[kMaxJointBatch];
    memset(key, 0, sizeof(key));
    memcpy(key, items, sizeof(JointItem) * (size_t)n);
    JointCommon ckey;
    memset(&ckey, 0, sizeof(ckey));
    ckey = cm;
    ckey.wait_limit_ns = g_wait_limit_ns;   // part of the graph key: a changed limit re-records
    ckey.argmax_log = g_argmax_log;
    ckey.argmax_cap = g_argmax_cap;
    if (cm.direct) {
        // every launch straight onto the caller's stream; the graph cache is left alone
        TuneTimingOff no_timing;
        const int slot = prof::enabled && prof::used < prof::kSlots ? prof::used++ : -1;
        const int rc = issue_joint(key, n, ckey, ws, np, nq, slot, st);
        if (rc) return rc;
        return stats ? read_stats(ws, n, stats, st) : GLU_OK;
    }
    int device = 0;
    GLU_CUDA_TRY(cudaGetDevice(&device));
    static JointGraph g = {};
    int rc = GLU_OK;
    const bool same = g.valid && g.profiled == prof::enabled &&
                      same_call(g, device, key, n, ckey, wsp, ws_bytes);
    if (prof::enabled && (same || g.valid)) {
        rc = prof::collect_graph();   // the previous replay's phase times
        if (rc) return rc;
    }
    if (same && g.exec) {
        GLU_CUDA_TRY(cudaGraphLaunch(g.exec, st));
        if (prof::enabled) prof::graph_pending = true;
    } else if (same && g.seen >= 1) {
        static cudaStream_t cap = nullptr, cap_body = nullptr;
        static int cap_device = -1;
        if (!cap || cap_device != device) {
            if (cap) cudaStreamDestroy(cap);
            if (cap_body) cudaStreamDestroy(cap_body);
            cap = cap_body = nullptr;
            GLU_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            GLU_CUDA_TRY(cudaStreamCreateWithFlags(&cap_body, cudaStreamNonBlocking));
            cap_device = device;
        }
        cudaGraph_t graph = nullptr;
        GLU_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
        rc = issue_joint(key, n, ckey, ws, np, nq, prof::enabled ? prof::kGraphSlot : -1, cap,
                         cap_body);
        {   // a failure in the middle of a conditional body leaves that capture open: close it
            cudaStreamCaptureStatus bs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(cap_body, &bs) == cudaSuccess &&
                bs != cudaStreamCaptureStatusNone) {
                cudaGraph_t bg = nullptr;
                (void)cudaStreamEndCapture(cap_body, &bg);
                if (rc == GLU_OK) rc = GLU_ERR_CUDA;
            }
        }
        const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
        cudaGraphExec_t exec = nullptr;
        if (rc == GLU_OK && ec == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
            g.exec = exec;
            ++g_graphs_recorded;
            GLU_CUDA_TRY(cudaGraphLaunch(g.exec, st));
            if (prof::enabled) prof::graph_pending = true;
        } else {
            // recording failed (a CUDA call refused inside the capture): issue directly
            (void)cudaGetLastError();
            if (rc == GLU_OK || rc == GLU_ERR_CUDA) {
                const int slot = prof::enabled && prof::used < prof::kSlots ? prof::used++ : -1;
                rc = issue_joint(key, n, ckey, ws, np, nq, slot, st);
            }
        }
        if (graph) cudaGraphDestroy(graph);
    } else {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = JointGraph{};
        g.valid = true;
        g.profiled = prof::enabled;
        g.device = device;
        g.n = n;
        memcpy(g.items, key, sizeof(key));
        g.cm = ckey;
        g.ws = wsp;
        g.ws_bytes = ws_bytes;
        g.seen = 1;
        const int slot = prof::enabled && prof::used < prof::kSlots ? prof::used++ : -1;
        rc = issue_joint(key, n, ckey, ws, np, nq, slot, st);
    }
    if (rc) return rc;
    return stats ? read_stats(ws, n, stats, st) : GLU_OK;
}

int launch_joint(const JointArgs& a, void* ws, size_t ws_bytes, glu_joint_stats* stats,
                 cudaStream_t st, int direct) {
    JointItem it;
    it.hr = a.hr;
    it.hr_pitch = a.hr_pitch;
    it.lr = a.lr;
    it.lr_pitch = a.lr_pitch;
    it.H = a.H;
    it.W = a.W;
    it.s = a.s;
    it.S = a.S;
    it.code = a.code;
    it.weight = a.weight;
    it.err = a.err;
    JointCommon cm;
    cm.eps255 = a.eps255;
    cm.tau = a.tau;
    cm.N = a.N;
    cm.strict = a.strict;
    cm.conn = a.conn;
    cm.wfmt = a.wfmt;
    cm.wait_limit_ns = 0;
    cm.direct = direct;
    return launch_joint_batch(&it, 1, cm, ws, ws_bytes, stats, st);
}

int joint_decisions(const void* wsp, size_t ws_bytes, int H, int W, int s, int N, int8_t* out,
                    int64_t cap, cudaStream_t st, int64_t* written) {
    JointItem it{};
    it.H = H;
    it.W = W;
    it.s = s;
    int64_t np, nq, nch;
    batch_sizes(&it, 1, &np, &nq, &nch);
    JointWs ws;
    const size_t need = carve(const_cast<void*>(wsp), np, nq, 1, N, nch, &ws);
    if (ws_bytes < need) return GLU_ERR_WORKSPACE;
    std::unique_ptr<JointCtl> c(new JointCtl);
    GLU_CUDA_TRY(cudaMemcpyAsync(c.get(), ws.ctl, sizeof(JointCtl), cudaMemcpyDeviceToHost, st));
    GLU_CUDA_TRY(cudaStreamSynchronize(st));
    int64_t off = 0;
    for (int k = 0; k < c->iterations[0] && k < N; ++k) {
        const int64_t m = c->M[0][k];
        if (off + m > cap) return GLU_ERR_INVALID_ARG;
        if (m > 0)
            GLU_CUDA_TRY(cudaMemcpyAsync(out + off, ws.dlog + (int64_t)k * ws.mcap, (size_t)m,
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

extern "C" int glu_dbg_wtrace(unsigned long long* host) {
    return cudaMemcpyFromSymbol(host, glu::g_wtrace, sizeof(glu::g_wtrace)) == cudaSuccess
               ? GLU_OK : GLU_ERR_CUDA;
}

extern "C" int glu_dbg_deps_times(unsigned long long* host) {
    return cudaMemcpyFromSymbol(host, glu::g_deps_t, sizeof(glu::g_deps_t)) == cudaSuccess
               ? GLU_OK : GLU_ERR_CUDA;
}

extern "C" int glu_dbg_small_times(unsigned long long* host) {
    return cudaMemcpyFromSymbol(host, glu::g_small_t, sizeof(glu::g_small_t)) == cudaSuccess
               ? GLU_OK : GLU_ERR_CUDA;
}

extern "C" int glu_dbg_marks(int enable, float* ms, int* tags, int cap) {
    using namespace glu;
    int k = 0;
    if (dbgm::n > 0 && ms && tags) {
        if (cudaEventSynchronize(dbgm::ev[dbgm::n - 1]) != cudaSuccess) return -1;
        for (int i = 1; i < dbgm::n && k < cap; ++i, ++k) {
            cudaEventElapsedTime(&ms[k], dbgm::ev[i - 1], dbgm::ev[i]);
            tags[k] = dbgm::tag[i];
        }
    }
    dbgm::n = 0;
    dbgm::on = enable != 0;
    return k;
}

extern "C" int glu_dbg_trace_clear(void) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, glu::g_trace) != cudaSuccess) return GLU_ERR_CUDA;
    return cudaMemset(p, 0, sizeof(glu::g_trace)) == cudaSuccess ? GLU_OK : GLU_ERR_CUDA;
}
#endif

extern "C" int glu_joint_profile(int32_t enable) {
    using namespace glu;
    if (enable && !prof::created) {
        for (int i = 0; i <= prof::kSlots; ++i)
            for (int j = 0; j < prof::kMaxEv; ++j)
                if (cudaEventCreate(&prof::ev[i][j]) != cudaSuccess) return GLU_ERR_CUDA;
        prof::created = true;
    }
    if (!enable && prof::enabled) {
        const int rc = prof::collect_graph();
        if (rc) return rc;
    }
    prof::enabled = enable != 0;
    return GLU_OK;
}

extern "C" int glu_joint_profile_read(float* ms, int32_t* calls) {
    using namespace glu;
    if (!ms || !calls) return GLU_ERR_INVALID_ARG;
    int rc = prof::collect_graph();
    if (rc) return rc;
    for (int k = 0; k < 5; ++k) ms[k] = prof::gacc[k];
    *calls = prof::gcalls;
    for (int sl = 0; sl < prof::used; ++sl) {
        float t[5];
        rc = prof::phase_times(sl, t);
        if (rc == GLU_ERR_INVALID_ARG) continue;
        if (rc) return rc;
        for (int k = 0; k < 5; ++k) ms[k] += t[k];
        ++*calls;
    }
    prof::used = 0;
    prof::gcalls = 0;
    for (int k = 0; k < 5; ++k) prof::gacc[k] = 0.f;
    return GLU_OK;
}
