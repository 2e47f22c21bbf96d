// Algorithm 1 (Sec. 3.2) over a batch of images in one persistent launch: the kernel template
// and its host-side launcher. Instantiated per guide dtype in k_search_u8.cu / k_search_f16.cu
// for every variant of the tuning table below; the including file defines set_status().
//
// Work items are 64 x TH HR tiles of every image of the batch (one global tile index space);
// each CTA walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... so images of uneven sizes,
// scales and window sizes share one launch. A single image is a batch of one.
//
// Per tile, the HR tile is staged into shared memory by a 2D TMA load (cp.async.bulk.tensor)
// completing on an mbarrier (one tensor map per image, kept in the kernel's parameter block);
// while it is in flight the CTA's threads copy the LR halo (the LR rows and columns the tile's
// windows reach) into shared memory as float4 colours in 1/255 units, plus a copy with every
// channel duplicated for the packed two-pixel search. Each thread then owns whole pixels, two
// vertically adjacent ones of one LR block at a time: both candidate loops of Algorithm 1 run in
// registers against the shared-memory window with packed two-lane FP32 arithmetic (one lane per
// pixel; search_pair), so no cross-lane reduction is needed and the tie-break is the
// deterministic lowest window index. Every variant computes the same arithmetic in the same
// order: results are bit-identical across variants and to the one-pixel search_pixel.
#pragma once

#include <cudaTypedefs.h>
#include <string.h>

#include "internal.h"
#include "search.cuh"
#include "variants.h"

namespace glu {

constexpr int kThreads = 256;
constexpr int kMaxBatch = kMaxSearchBatch;
static_assert(kThreads % kTileW == 0, "a thread keeps one tile column");

struct SImg {
    const void* hr;
    int64_t hr_pitch;
    const void* lr;
    int64_t lr_pitch;
    uint16_t* code;
    void* weight;
    float* err;
    int lr_dtype;
    int H, W, h, w, s, S;
    int tiles_x;   // tiles per tile row
    int tile0;     // first global tile index of this image
    int use_tma;
};

struct SBatch {
    CUtensorMap maps[kMaxBatch];
    SImg im[kMaxBatch];
    int n, total_tiles;
    int wfmt, gnu;
    float eps255;
    int region_cap;   // LR halo cells of the largest tile: the shared copies' stride
};

// Shared-memory bytes of the LR halo copies for region_cap cells: float4 colours, then the
// duplicated (r, r, g, g) float4 and (b, b) float2 copies.
__host__ __device__ constexpr size_t region_bytes(int cells) {
    return (size_t)cells * (sizeof(float4) * 2 + sizeof(float2));
}

template <typename HT, int TH>
struct HrTile {
    alignas(128) HT px[TH][kTileW * 3];
};

// One tile of image I: (x0, y0) its top-left HR pixel. `phase` is the mbarrier parity to wait on.
template <int S, typename HT, int TH, bool CP>
__device__ __forceinline__ bool search_tile(const SBatch& B, int i, int x0, int y0,
                                            HrTile<HT, TH>& tile, uint64_t* bar, uint32_t phase,
                                            float4* region) {
    float4* const rg = region + B.region_cap;
    float2* const bbuf = reinterpret_cast<float2*>(rg + B.region_cap);
    const SImg& I = B.im[i];
    constexpr int r = (S - 1) / 2;
    const int tid = threadIdx.x;
    const int s = I.s;
    const int xe = min(x0 + kTileW, I.W), ye = min(y0 + TH, I.H);
    const int v0 = y0 / s - r, u0 = x0 / s - r;
    const int RH = (ye - 1) / s + r - v0 + 1, RW = (xe - 1) / s + r - u0 + 1;

    if (I.use_tma) {
        if (tid == 0) {
            fence_proxy_async_smem();  // earlier generic reads of the tile buffer come first
            mbar_arrive_expect_tx(bar, (uint32_t)sizeof(tile.px));
            tma_load_2d(&tile.px[0][0], &B.maps[i], bar, x0 * 3, y0);
        }
    } else {
        const HT* src = (const HT*)I.hr;
        for (int k = tid; k < TH * kTileW * 3; k += kThreads) {
            const int ty = k / (kTileW * 3), tx = k % (kTileW * 3);
            const int y = y0 + ty, xc = x0 * 3 + tx;
            tile.px[ty][tx] = (y < I.H && xc < I.W * 3) ? src[(int64_t)y * I.hr_pitch + xc] : HT(0);
        }
    }
    // LR halo in 1/255 units; rows/columns outside the LR image are never selected (masks)
    for (int k = tid; k < RH * RW; k += kThreads) {
        const int v = v0 + k / RW, u = u0 + k % RW;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v >= 0 && v < I.h && u >= 0 && u < I.w) {
            const int64_t o = (int64_t)v * I.lr_pitch + (int64_t)u * 3;
            if (I.lr_dtype == GLU_U8) {
                const uint8_t* L = (const uint8_t*)I.lr;
                c = make_float4((float)L[o], (float)L[o + 1], (float)L[o + 2], 0.f);
            } else if (I.lr_dtype == GLU_F16) {
                const __half* L = (const __half*)I.lr;
                c = make_float4(__half2float(L[o]) * 255.f, __half2float(L[o + 1]) * 255.f,
                                __half2float(L[o + 2]) * 255.f, 0.f);
            } else {
                const float* L = (const float*)I.lr;
                c = make_float4(L[o] * 255.f, L[o + 1] * 255.f, L[o + 2] * 255.f, 0.f);
            }
        }
        region[k] = c;
        rg[k] = make_float4(c.x, c.x, c.y, c.y);
        bbuf[k] = make_float2(c.z, c.z);
    }
    __syncthreads();
    if (I.use_tma && !mbar_wait_bounded(bar, phase)) {
        set_status(GLU_ERR_TIMEOUT);
        // the copy may still land: give it another bounded wait before the CTA moves on
        (void)mbar_wait_bounded(bar, phase);
        return false;
    }

    // interior tiles (every window inside the LR image) skip the validity masks
    const bool interior = v0 >= 0 && u0 >= 0 && (ye - 1) / s + r < I.h && (xe - 1) / s + r < I.w;
    // a thread keeps one column of the tile (kThreads is a multiple of kTileW) and walks pairs
    // of rows (ty, ty + 1); the warps of one row pair decide alike whether both rows lie in one
    // LR block (then they share the window and are searched together) or not
    static_assert(TH % (2 * (kThreads / kTileW)) == 0, "row pairs tile the tile");
    const int tx = tid % kTileW, x = x0 + tx, px = x / s;
    const int col = px - r - u0;
    auto store = [&](int y, const SearchOut& o) {
        const int64_t p = (int64_t)y * I.W + x;
        I.code[p] = (uint16_t)(o.ka * S * S + o.kb);
        store_weight(I.weight, B.wfmt, p, o.omega);
        if (I.err) I.err[p] = o.err;
    };
    auto one = [&](int ty) {
        const int y = y0 + ty, py = y / s;
        const float ir = Px<HT>::to255(tile.px[ty][tx * 3 + 0]);
        const float ig = Px<HT>::to255(tile.px[ty][tx * 3 + 1]);
        const float ib = Px<HT>::to255(tile.px[ty][tx * 3 + 2]);
        const float4* win = &region[(py - r - v0) * RW + col];
        SearchOut o;
        if (interior) {
            o = search_pixel<S, CP, true>(win, RW, 0u, 0u, ir, ig, ib, B.eps255, B.gnu != 0);
        } else {
            uint32_t rm, cm;
            window_masks(py, px, I.h, I.w, S, rm, cm);
            o = search_pixel<S, CP>(win, RW, rm, cm, ir, ig, ib, B.eps255, B.gnu != 0);
        }
        store(y, o);
    };
    for (int ty = 2 * (tid / kTileW); ty < TH; ty += 2 * (kThreads / kTileW)) {
        const int y = y0 + ty;
        if (y >= I.H || x >= I.W) continue;
        const bool two = y + 1 < I.H && y / s == (y + 1) / s;
        if (!two) {
            one(ty);
            if (y + 1 < I.H) one(ty + 1);
            continue;
        }
        const int py = y / s;
        const int wo = (py - r - v0) * RW + col;
        SearchOut o0, o1;
        const float ir0 = Px<HT>::to255(tile.px[ty][tx * 3 + 0]);
        const float ig0 = Px<HT>::to255(tile.px[ty][tx * 3 + 1]);
        const float ib0 = Px<HT>::to255(tile.px[ty][tx * 3 + 2]);
        const float ir1 = Px<HT>::to255(tile.px[ty + 1][tx * 3 + 0]);
        const float ig1 = Px<HT>::to255(tile.px[ty + 1][tx * 3 + 1]);
        const float ib1 = Px<HT>::to255(tile.px[ty + 1][tx * 3 + 2]);
        if (interior) {
            search_pair<S, CP, true>(&region[wo], &rg[wo], &bbuf[wo], RW, 0u, 0u, ir0, ig0, ib0,
                                     ir1, ig1, ib1, B.eps255, B.gnu != 0, o0, o1);
        } else {
            uint32_t rm, cm;
            window_masks(py, px, I.h, I.w, S, rm, cm);
            search_pair<S, CP>(&region[wo], &rg[wo], &bbuf[wo], RW, rm, cm, ir0, ig0, ib0, ir1,
                               ig1, ib1, B.eps255, B.gnu != 0, o0, o1);
        }
        store(y, o0);
        store(y + 1, o1);
    }
    __syncthreads();  // the tile buffers are reused by the next tile
    return true;
}

template <typename HT, int TH, int MINB, bool CP>
__global__ void __launch_bounds__(kThreads, MINB) k_search(const __grid_constant__ SBatch B) {
    __shared__ HrTile<HT, TH> tile;
    __shared__ alignas(8) uint64_t bar;
    extern __shared__ float4 region[];
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t uses = 0;  // completed phases of the mbarrier (TMA tiles issued by this CTA)
    for (int t = blockIdx.x; t < B.total_tiles; t += gridDim.x) {
        int i = 0;
        while (i + 1 < B.n && B.im[i + 1].tile0 <= t) ++i;
        const SImg& I = B.im[i];
        const int lt = t - I.tile0;
        const int x0 = (lt % I.tiles_x) * kTileW, y0 = (lt / I.tiles_x) * TH;
        const uint32_t phase = uses & 1u;
        bool ok = true;
        switch (I.S) {
            case 1: ok = search_tile<1, HT, TH, CP>(B, i, x0, y0, tile, &bar, phase, region); break;
            case 3: ok = search_tile<3, HT, TH, CP>(B, i, x0, y0, tile, &bar, phase, region); break;
            case 5: ok = search_tile<5, HT, TH, CP>(B, i, x0, y0, tile, &bar, phase, region); break;
            case 7: ok = search_tile<7, HT, TH, CP>(B, i, x0, y0, tile, &bar, phase, region); break;
            default: ok = search_tile<9, HT, TH, CP>(B, i, x0, y0, tile, &bar, phase, region); break;
        }
        if (!ok) return;
        if (I.use_tma) ++uses;
    }
}

// 2D byte/half view of an interleaved HR image for TMA: inner dim W*3 elements, outer dim H,
// box (kTileW*3, tile_h). Defined in k_search.cu.
bool make_hr_map(const SearchArgs& a, CUtensorMap* map, int tile_h);

template <typename HT, int TH, int MINB, bool CP>
int launch_search_chunk(const SearchArgs* items, int n, cudaStream_t st) {
    SBatch B;  // host staging of the parameter block (copied into the launch)
    memset(&B, 0, sizeof(B));
    int cap = 0;
    int tiles = 0;
    for (int k = 0; k < n; ++k) {
        const SearchArgs& a = items[k];
        SImg& I = B.im[k];
        I.hr = a.hr;
        I.hr_pitch = a.hr_pitch;
        I.lr = a.lr;
        I.lr_pitch = a.lr_pitch;
        I.lr_dtype = a.lr_dtype;
        I.code = a.code;
        I.weight = a.weight;
        I.err = a.err;
        I.H = a.H; I.W = a.W; I.h = a.h; I.w = a.w; I.s = a.s; I.S = a.S;
        I.tiles_x = (a.W + kTileW - 1) / kTileW;
        I.tile0 = tiles;
        I.use_tma = make_hr_map(a, &B.maps[k], TH) ? 1 : 0;
        tiles += I.tiles_x * ((a.H + TH - 1) / TH);
        const int r = (a.S - 1) / 2;
        const int rh = (TH - 1) / a.s + 2 + 2 * r, rw = (kTileW - 1) / a.s + 2 + 2 * r;
        if (rh * rw > cap) cap = rh * rw;
    }
    const size_t smem = region_bytes(cap);
    B.region_cap = cap;
    B.n = n;
    B.total_tiles = tiles;
    B.wfmt = items[0].wfmt;
    B.gnu = items[0].gnu;
    B.eps255 = items[0].eps255;
    if (tiles == 0) return GLU_OK;
    auto kern = k_search<HT, TH, MINB, CP>;
    if (smem > 48 * 1024)
        GLU_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 148, per_sm = 1;
    GLU_CUDA_TRY(cudaGetDevice(&dev));
    GLU_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GLU_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const int grid = tiles < sms * per_sm ? tiles : sms * per_sm;
    kern<<<grid, kThreads, smem, st>>>(B);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

// Variant v of the table for one chunk of <= kMaxBatch images of guide dtype HT.
template <typename HT>
int search_dispatch(int v, const SearchArgs* items, int n, cudaStream_t st) {
#define GLU_SEARCH_CASE(k)                                                                  \
    case k:                                                                                 \
        return launch_search_chunk<HT, kSearchVariants[k].tile_h, kSearchVariants[k].min_blocks, \
                                   kSearchVariants[k].compact != 0>(items, n, st)
    static_assert(kNumSearchVariants == 5, "one case per variant");
    switch (v) {
        GLU_SEARCH_CASE(0);
        GLU_SEARCH_CASE(1);
        GLU_SEARCH_CASE(2);
        GLU_SEARCH_CASE(3);
        GLU_SEARCH_CASE(4);
        default: return GLU_ERR_INVALID_ARG;
    }
#undef GLU_SEARCH_CASE
}

}  // namespace glu
