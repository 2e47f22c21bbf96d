/*
 * Seeded synthetic piecewise-smooth RGB images: Voronoi cells, each filled with its own linear
 * colour gradient, plus isolated square dots and one-pixel lines of random colour, plus
 * per-channel Gaussian noise, rounded and clamped to uint8.
 *
 * This file is the input generator shared by the CPU oracle tests and the GPU path. It contains
 * none of the upsampling method's arithmetic. Every random number comes from a counter-based
 * hash (SplitMix64's finaliser applied to a packed counter), so a pixel's value does not depend
 * on the order pixels are generated in and the OpenMP-parallel render is bit-reproducible.
 *
 * Video mode: frame f translates every cell seed by f * cell_dx_per_frame pixels along x, and
 * dot i is re-drawn every dot_period frames with a per-dot phase, so 1/dot_period of the dots
 * vanish and reappear elsewhere on each frame. Lines are static. Noise is fresh per frame.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t width, height;
    int32_t n_cells, n_dots, n_lines;
    double noise_sigma;        /* per-channel N(0, sigma) in uint8 units */
    double grad_max;           /* cell gradient entries ~ U[-grad_max, grad_max] per pixel */
    uint64_t seed;
    int32_t frame;             /* video frame index; 0 for still images */
    double cell_dx_per_frame;  /* seed translation per frame (pixels, +x) */
    int32_t dot_period;        /* 0: static dots; P: each dot is re-drawn every P frames */
} synth_scene;

/* Stream tags keep the draws of different scene elements independent. */
enum { TAG_CELL = 1, TAG_DOT = 2, TAG_LINE = 3, TAG_NOISE = 4, TAG_PHASE = 5 };

static inline uint64_t fmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Hash of (seed, tag, a, b, c): chained finaliser rounds. */
static inline uint64_t hash5(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint64_t c) {
    uint64_t h = fmix64(seed ^ (tag << 56));
    h = fmix64(h ^ a);
    h = fmix64(h ^ (b * 0xD6E8FEB86659FD93ull));
    h = fmix64(h ^ (c * 0xA0761D6478BD642Full));
    return h;
}

static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

typedef struct {
    double sx, sy;          /* seed position */
    double c0[3];           /* colour at the seed */
    double gx[3], gy[3];    /* colour gradient per pixel */
} cell_t;

static void make_cell(const synth_scene* sc, int32_t i, cell_t* c) {
    const uint64_t s = sc->seed;
    c->sx = u01(hash5(s, TAG_CELL, (uint64_t)i, 0, 0)) * sc->width +
            sc->cell_dx_per_frame * (double)sc->frame;
    c->sy = u01(hash5(s, TAG_CELL, (uint64_t)i, 1, 0)) * sc->height;
    for (int ch = 0; ch < 3; ++ch) {
        c->c0[ch] = 255.0 * u01(hash5(s, TAG_CELL, (uint64_t)i, 2, (uint64_t)ch));
        c->gx[ch] = sc->grad_max * (2.0 * u01(hash5(s, TAG_CELL, (uint64_t)i, 3, (uint64_t)ch)) - 1.0);
        c->gy[ch] = sc->grad_max * (2.0 * u01(hash5(s, TAG_CELL, (uint64_t)i, 4, (uint64_t)ch)) - 1.0);
    }
}

static inline double clamp255(double v) { return v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v); }

/* Nearest seed by exhaustive scan of a bucket grid, ring by ring; ties go to the lower index. */
typedef struct {
    int32_t bw, bh;        /* bucket grid size */
    double bsize;          /* bucket edge in pixels */
    double ox;             /* x origin of the grid (seeds may sit left of 0 after translation) */
    int32_t* start;        /* bw*bh+1 offsets */
    int32_t* items;        /* cell indices sorted by bucket */
} bucket_grid;

static int build_buckets(const cell_t* cells, int32_t n, const synth_scene* sc, bucket_grid* g) {
    double minx = 0.0, maxx = (double)sc->width;
    for (int32_t i = 0; i < n; ++i) {
        if (cells[i].sx < minx) minx = cells[i].sx;
        if (cells[i].sx > maxx) maxx = cells[i].sx;
    }
    double area = (maxx - minx + 1.0) * (double)sc->height;
    g->bsize = sqrt(area / (double)(n > 0 ? n : 1));
    if (g->bsize < 4.0) g->bsize = 4.0;
    g->ox = minx;
    g->bw = (int32_t)ceil((maxx - minx + 1.0) / g->bsize);
    g->bh = (int32_t)ceil(((double)sc->height + 1.0) / g->bsize);
    if (g->bw < 1) g->bw = 1;
    if (g->bh < 1) g->bh = 1;
    int32_t nb = g->bw * g->bh;
    g->start = (int32_t*)calloc((size_t)nb + 1, sizeof(int32_t));
    g->items = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* fill = (int32_t*)calloc((size_t)nb, sizeof(int32_t));
    if (!g->start || !g->items || !fill) { free(fill); return -1; }
    int32_t* bidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!bidx) { free(fill); return -1; }
    for (int32_t i = 0; i < n; ++i) {
        int32_t bx = (int32_t)floor((cells[i].sx - g->ox) / g->bsize);
        int32_t by = (int32_t)floor(cells[i].sy / g->bsize);
        if (bx < 0) bx = 0;
        if (bx >= g->bw) bx = g->bw - 1;
        if (by < 0) by = 0;
        if (by >= g->bh) by = g->bh - 1;
        bidx[i] = by * g->bw + bx;
        g->start[bidx[i] + 1]++;
    }
    for (int32_t b = 0; b < nb; ++b) g->start[b + 1] += g->start[b];
    for (int32_t i = 0; i < n; ++i) g->items[g->start[bidx[i]] + fill[bidx[i]]++] = i;
    free(fill);
    free(bidx);
    return 0;
}

static int32_t nearest_cell(const cell_t* cells, const bucket_grid* g, double px, double py) {
    int32_t bx = (int32_t)floor((px - g->ox) / g->bsize);
    int32_t by = (int32_t)floor(py / g->bsize);
    if (bx < 0) bx = 0;
    if (bx >= g->bw) bx = g->bw - 1;
    if (by < 0) by = 0;
    if (by >= g->bh) by = g->bh - 1;
    double best = INFINITY;
    int32_t besti = -1;
    int32_t maxr = g->bw > g->bh ? g->bw : g->bh;
    for (int32_t R = 0; R <= maxr; ++R) {
        for (int32_t yy = by - R; yy <= by + R; ++yy) {
            if (yy < 0 || yy >= g->bh) continue;
            for (int32_t xx = bx - R; xx <= bx + R; ++xx) {
                if (xx < 0 || xx >= g->bw) continue;
                if (yy != by - R && yy != by + R && xx != bx - R && xx != bx + R) continue;
                int32_t b = yy * g->bw + xx;
                for (int32_t t = g->start[b]; t < g->start[b + 1]; ++t) {
                    int32_t i = g->items[t];
                    double dx = px - cells[i].sx, dy = py - cells[i].sy;
                    double d = dx * dx + dy * dy;
                    if (d < best || (d == best && i < besti)) { best = d; besti = i; }
                }
            }
        }
        /* every seed in ring R+1 or beyond is at least R*bsize away */
        double lim = (double)R * g->bsize;
        if (besti >= 0 && best < lim * lim) break;
    }
    return besti;
}

static void put_px(uint8_t* out, const synth_scene* sc, int32_t x, int32_t y, const double c[3]) {
    if (x < 0 || y < 0 || x >= sc->width || y >= sc->height) return;
    uint8_t* p = out + ((size_t)y * (size_t)sc->width + (size_t)x) * 3;
    for (int ch = 0; ch < 3; ++ch) p[ch] = (uint8_t)lround(clamp255(c[ch]));
}

/* Box-Muller standard normal from two uniforms of the per-(frame, pixel, channel) counter. */
static inline double noise_at(const synth_scene* sc, int32_t x, int32_t y, int32_t ch) {
    uint64_t pix = (uint64_t)y * (uint64_t)sc->width + (uint64_t)x;
    uint64_t h1 = hash5(sc->seed, TAG_NOISE, (uint64_t)sc->frame, pix, (uint64_t)(2 * ch));
    uint64_t h2 = hash5(sc->seed, TAG_NOISE, (uint64_t)sc->frame, pix, (uint64_t)(2 * ch + 1));
    double u1 = u01(h1), u2 = u01(h2);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/*
 * Render one frame into out (height x width x 3 bytes, row-major, channel-interleaved).
 * threads <= 0 uses the OpenMP default. Returns 0, or -1 on bad arguments / allocation failure.
 */
int synth_render_u8(const synth_scene* sc, uint8_t* out, int32_t threads) {
    if (!sc || !out || sc->width <= 0 || sc->height <= 0 || sc->n_cells <= 0) return -1;
    const int32_t W = sc->width, H = sc->height;
    cell_t* cells = (cell_t*)malloc(sizeof(cell_t) * (size_t)sc->n_cells);
    if (!cells) return -1;
    for (int32_t i = 0; i < sc->n_cells; ++i) make_cell(sc, i, &cells[i]);
    bucket_grid g;
    memset(&g, 0, sizeof(g));
    if (build_buckets(cells, sc->n_cells, sc, &g) != 0) {
        free(cells); free(g.start); free(g.items);
        return -1;
    }
#ifdef _OPENMP
    int nthr = threads > 0 ? threads : 0;
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthr > 0 ? nthr : omp_get_max_threads())
#endif
    for (int32_t y = 0; y < H; ++y) {
        for (int32_t x = 0; x < W; ++x) {
            /* pixel centre convention: the seed comparison uses integer pixel coordinates */
            int32_t i = nearest_cell(cells, &g, (double)x, (double)y);
            const cell_t* c = &cells[i];
            double col[3];
            for (int ch = 0; ch < 3; ++ch)
                col[ch] = c->c0[ch] + c->gx[ch] * ((double)x - c->sx) + c->gy[ch] * ((double)y - c->sy);
            put_px(out, sc, x, y, col);
        }
    }
    free(cells); free(g.start); free(g.items);

    /* dots: squares of side 1..3 */
    for (int32_t i = 0; i < sc->n_dots; ++i) {
        uint64_t gen = 0;
        if (sc->dot_period > 0) {
            uint64_t phase = hash5(sc->seed, TAG_PHASE, (uint64_t)i, 0, 0) % (uint64_t)sc->dot_period;
            gen = ((uint64_t)sc->frame + phase) / (uint64_t)sc->dot_period;
        }
        int32_t side = 1 + (int32_t)(hash5(sc->seed, TAG_DOT, (uint64_t)i, gen, 0) % 3u);
        int32_t x0 = (int32_t)(u01(hash5(sc->seed, TAG_DOT, (uint64_t)i, gen, 1)) * W);
        int32_t y0 = (int32_t)(u01(hash5(sc->seed, TAG_DOT, (uint64_t)i, gen, 2)) * H);
        double col[3];
        for (int ch = 0; ch < 3; ++ch)
            col[ch] = floor(256.0 * u01(hash5(sc->seed, TAG_DOT, (uint64_t)i, gen, 3 + (uint64_t)ch)));
        for (int32_t dy = 0; dy < side; ++dy)
            for (int32_t dx = 0; dx < side; ++dx) put_px(out, sc, x0 + dx, y0 + dy, col);
    }

    /* lines: one-pixel Bresenham segments between random endpoints */
    for (int32_t i = 0; i < sc->n_lines; ++i) {
        int32_t x0 = (int32_t)(u01(hash5(sc->seed, TAG_LINE, (uint64_t)i, 0, 0)) * W);
        int32_t y0 = (int32_t)(u01(hash5(sc->seed, TAG_LINE, (uint64_t)i, 1, 0)) * H);
        int32_t x1 = (int32_t)(u01(hash5(sc->seed, TAG_LINE, (uint64_t)i, 2, 0)) * W);
        int32_t y1 = (int32_t)(u01(hash5(sc->seed, TAG_LINE, (uint64_t)i, 3, 0)) * H);
        double col[3];
        for (int ch = 0; ch < 3; ++ch)
            col[ch] = floor(256.0 * u01(hash5(sc->seed, TAG_LINE, (uint64_t)i, 4, (uint64_t)ch)));
        int32_t dx = abs(x1 - x0), sx = x0 < x1 ? 1 : -1;
        int32_t dy = -abs(y1 - y0), sy = y0 < y1 ? 1 : -1;
        int32_t err = dx + dy;
        for (;;) {
            put_px(out, sc, x0, y0, col);
            if (x0 == x1 && y0 == y1) break;
            int32_t e2 = 2 * err;
            if (e2 >= dy) { err += dy; x0 += sx; }
            if (e2 <= dx) { err += dx; y0 += sy; }
        }
    }

    /* noise */
    if (sc->noise_sigma > 0.0) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthr > 0 ? nthr : omp_get_max_threads())
#endif
        for (int32_t y = 0; y < H; ++y) {
            for (int32_t x = 0; x < W; ++x) {
                uint8_t* p = out + ((size_t)y * (size_t)W + (size_t)x) * 3;
                for (int ch = 0; ch < 3; ++ch) {
                    double v = (double)p[ch] + sc->noise_sigma * noise_at(sc, x, y, ch);
                    p[ch] = (uint8_t)lround(clamp255(v));
                }
            }
        }
    }
    return 0;
}
