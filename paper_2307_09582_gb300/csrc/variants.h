// Implementation variants the autotuner chooses from (every variant of a kernel computes the
// same arithmetic in the same order, so results are bit-identical across variants).
#pragma once

namespace glu {

constexpr int kTileW = 64;   // HR pixels per search tile row (64 * 3 channels: a 16-byte multiple)

// Algorithm 1 search: tile height, CTAs per SM the registers are sized for, and the candidate
// loop schedule (window rows unrolled, or rolled loops).
struct SearchVariant {
    int tile_h, min_blocks, compact;
};
constexpr SearchVariant kSearchVariants[] = {
    {32, 2, 0}, {16, 2, 0}, {8, 2, 0}, {16, 3, 1}, {16, 4, 1},
};
constexpr int kNumSearchVariants = (int)(sizeof(kSearchVariants) / sizeof(kSearchVariants[0]));

// Eq. 1 apply, 3-channel float targets: rows of the 128-pixel-wide tiles, and how the tile's
// codes, weights and output move: plain loads and stores (0), TMA per tile (1), or TMA in a
// persistent two-stage pipeline (2). Where the arrays do not allow TMA, a variant runs the
// plain tiled kernel with the same rows.
constexpr int kApplyTW = 128;
struct ApplyVariant {
    int rows, tma;
};
constexpr ApplyVariant kApplyVariants[] = {{16, 0}, {8, 0}, {32, 0}, {64, 0}, {16, 1},
                                           {8, 1},  {32, 1}, {16, 2}, {8, 2},  {32, 2}};
constexpr int kNumApplyVariants = (int)(sizeof(kApplyVariants) / sizeof(kApplyVariants[0]));

}  // namespace glu
