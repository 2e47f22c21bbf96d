/*
 * FP64 CPU oracle for Guided Linear Upsampling (GLU; Song et al., ACM TOG 2023).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library. It shares no code, header, table or helper with the CUDA library; both
 * sides only receive the same seeded inputs.
 *
 * Everything is plain double-precision loops in the order the paper states the steps. OpenMP is
 * used only across independent HR pixels (Algorithm 1 is per pixel) so the oracle can be timed
 * on many host cores; the component loop of Algorithm 2 is sequential, as the paper writes it.
 *
 * Conventions (readings of points the paper leaves open):
 *  - Images are row-major H x W x C doubles in the caller's colour units: `unit` is the value of
 *    colour 1.0 (255 for raw uint8 values, 1 for colours already in [0, 1]). The paper's
 *    tau = 30/255 and eps = 1e-3 (Sec. 3.1, Sec. 5.3) are given in [0, 1] units and scaled here
 *    (eps of Eq. 5 and tau by unit, eps of Eq. 4 by unit^2, being a squared-colour term);
 *    errors are returned in [0, 1] units. Working on raw uint8 values keeps every squared
 *    distance an exact integer, so exact ties stay exact and go to the lowest window index.
 *  - ||.|| is the Euclidean norm over the colour channels.
 *  - Scale s: LR size h = ceil(H / s), w = ceil(W / s). The downscaled coordinate of HR pixel
 *    (y, x) is p_down = (floor(y / s), floor(x / s)), i.e. the LR block that contains it (Eq. 1).
 *  - Window Omega(p_down): LR pixels (v, u) with |v - p_down.y| <= r and |u - p_down.x| <= r,
 *    r = (S - 1) / 2, clipped to the LR image. Window index k = (dy + r) * S + (dx + r).
 *  - Regular grid downsampling (Sec. 3.3, Algorithm 2 init) takes, for every LR pixel, the HR
 *    pixel floor(e / 2) into its block along each axis, e being the block's extent (s, or the
 *    remainder for the last, partial block). Box downsampling is the plain block mean.
 *  - Algorithm 1 (FAST): a = argmin over the window of ||I_p - L_a||, ties to the lowest k;
 *    then b ranges over the whole window including b = a (the paper counts 9 pairs for a 3x3
 *    window), with the Eq. 5 weight; the pair minimising the Eq. 3 error wins, ties to the
 *    lowest k_b. With eps = 0 and d_a = d_b = 0 the weight is taken as 1.
 *  - GLU* (EXACT, Sec. 3.1): every unordered pair k_a < k_b of valid window pixels, weight by
 *    Eq. 4 (not clamped); minimum error wins, ties to the lowest (k_a, k_b). A window with a
 *    single valid pixel yields a = b, weight 1. With eps = 0 and L_a = L_b the weight is 1.
 *  - GNU: the weight is fixed to 1, so T_p = T_a with a from Algorithm 1's first step.
 *  - Algorithm 2: components are 8-connected (4-connected optional), processed in ascending
 *    order of their smallest raster index; membership of the large-error set is fixed when an
 *    iteration starts, while e0, the replacement argmax and the re-optimisation read the
 *    current state. The argmax over [q_up] intersected with C_i breaks ties to the lowest HR
 *    raster index. A trial is rolled back only if e1 > e0 (equality is accepted).
 *    PAPER mode re-optimises and sums over C_i exactly as Algorithm 2 lists it. STRICT mode
 *    re-optimises and sums over A_i, every HR pixel whose window contains a replaced LR pixel:
 *    the paper's text says a replacement is kept only if it reduces the total error, and the
 *    total error can change only on A_i, so STRICT compares exactly the total error.
 *    The iteration loop stops when the large-error set is empty, after N iterations, when an
 *    iteration accepts no trial (the state is then unchanged, so later iterations repeat it),
 *    or when the residual R_n = sum_p E_p does not decrease.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

static inline int imin(int a, int b) { return a < b ? a : b; }

void oracle_lr_dims(int H, int W, int s, int* h, int* w) {
    *h = (H + s - 1) / s;
    *w = (W + s - 1) / s;
}

static inline double dist3(const double* a, const double* b) {
    double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

static inline int same3(const double* a, const double* b) {
    return a[0] == b[0] && a[1] == b[1] && a[2] == b[2];
}

/* ------------------------------------------------------------------ downsampling (Sec. 3.3) */

int oracle_downsample_grid(const double* I, int H, int W, int C, int s, double* L) {
    if (!I || !L || H <= 0 || W <= 0 || C <= 0 || s <= 0) return OR_EINVAL;
    int h, w;
    oracle_lr_dims(H, W, s, &h, &w);
    for (int v = 0; v < h; ++v) {
        int ey = imin(s, H - v * s);
        int y = v * s + ey / 2;
        for (int u = 0; u < w; ++u) {
            int ex = imin(s, W - u * s);
            int x = u * s + ex / 2;
            for (int c = 0; c < C; ++c) L[((size_t)v * w + u) * C + c] = I[((size_t)y * W + x) * C + c];
        }
    }
    return OR_OK;
}

int oracle_downsample_box(const double* I, int H, int W, int C, int s, double* L) {
    if (!I || !L || H <= 0 || W <= 0 || C <= 0 || s <= 0) return OR_EINVAL;
    int h, w;
    oracle_lr_dims(H, W, s, &h, &w);
    for (int v = 0; v < h; ++v)
        for (int u = 0; u < w; ++u)
            for (int c = 0; c < C; ++c) {
                double acc = 0.0;
                int n = 0;
                for (int y = v * s; y < imin(H, v * s + s); ++y)
                    for (int x = u * s; x < imin(W, u * s + s); ++x) {
                        acc += I[((size_t)y * W + x) * C + c];
                        ++n;
                    }
                L[((size_t)v * w + u) * C + c] = acc / n;
            }
    return OR_OK;
}

/* --------------------------------------------------------------------- window helpers (Eq. 1) */

typedef struct {
    int n;          /* valid candidates */
    int k[81];      /* window index of each valid candidate, ascending */
    const double* col[81];
} window_t;

static void gather_window(const double* L, int h, int w, int s, int S, int y, int x, window_t* win) {
    int r = (S - 1) / 2, py = y / s, px = x / s;
    win->n = 0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
            int v = py + dy, u = px + dx;
            if (v < 0 || v >= h || u < 0 || u >= w) continue;
            win->k[win->n] = (dy + r) * S + (dx + r);
            win->col[win->n] = &L[((size_t)v * w + u) * 3];
            win->n++;
        }
}

/* Eq. 5 weight and the Eq. 3 error of the pair (a, b) for colour Ip. */
static void fast_pair_eval(const double* Ip, const double* La, const double* Lb, double eps,
                           double* omega, double* err) {
    double da = dist3(Ip, La), db = dist3(Ip, Lb);
    double den = da + db + eps;
    double om = den > 0.0 ? db / den : 1.0;
    double rec[3];
    for (int c = 0; c < 3; ++c) rec[c] = om * La[c] + (1.0 - om) * Lb[c];
    *omega = om;
    *err = dist3(rec, Ip);
}

/* Eq. 4 weight (projection on the colour line through La, Lb) and its Eq. 3 error. */
static void exact_pair_eval(const double* Ip, const double* La, const double* Lb, double eps,
                            double* omega, double* err) {
    double num = 0.0, den = 0.0;
    for (int c = 0; c < 3; ++c) {
        num += (Ip[c] - Lb[c]) * (La[c] - Lb[c]);
        den += (La[c] - Lb[c]) * (La[c] - Lb[c]);
    }
    den += eps;
    double om = den > 0.0 ? num / den : 1.0;
    double rec[3];
    for (int c = 0; c < 3; ++c) rec[c] = om * La[c] + (1.0 - om) * Lb[c];
    *omega = om;
    *err = dist3(rec, Ip);
}

/* Algorithm 1 for one HR pixel. Gaps: distance from the winner to the best candidate whose
 * colour differs from the winner's (exact ties of equal colours resolve identically anywhere). */
static void fast_pixel(const double* I, int H, int W, const double* L, int h, int w, int s, int S,
                       double eps, int y, int x, int32_t* ka, int32_t* kb, double* omega,
                       double* err, double* gap_a, double* gap_b) {
    (void)H;
    window_t win;
    gather_window(L, h, w, s, S, y, x, &win);
    const double* Ip = &I[((size_t)y * W + x) * 3];
    /* step 1: a is the window pixel with the most similar colour */
    int ia = 0;
    double da = INFINITY;
    for (int i = 0; i < win.n; ++i) {
        double d = dist3(Ip, win.col[i]);
        if (d < da) { da = d; ia = i; }
    }
    /* step 2: fix a, choose b and the Eq. 5 weight minimising Eq. 3 */
    int ib = 0;
    double best = INFINITY, best_om = 1.0;
    for (int i = 0; i < win.n; ++i) {
        double om, e;
        fast_pair_eval(Ip, win.col[ia], win.col[i], eps, &om, &e);
        if (e < best) { best = e; best_om = om; ib = i; }
    }
    *ka = win.k[ia];
    *kb = win.k[ib];
    *omega = best_om;
    *err = best;
    if (gap_a) {
        double g = INFINITY;
        for (int i = 0; i < win.n; ++i)
            if (!same3(win.col[i], win.col[ia])) {
                double d = dist3(Ip, win.col[i]) - da;
                if (d < g) g = d;
            }
        *gap_a = g;
    }
    if (gap_b) {
        double g = INFINITY;
        for (int i = 0; i < win.n; ++i)
            if (!same3(win.col[i], win.col[ib])) {
                double om, e;
                fast_pair_eval(Ip, win.col[ia], win.col[i], eps, &om, &e);
                if (e - best < g) g = e - best;
            }
        *gap_b = g;
    }
}

static int check_common(const double* I, int H, int W, const double* L, int s, int S) {
    if (!I || !L || H <= 0 || W <= 0 || s <= 0 || S < 1 || S > 9 || (S % 2) == 0) return OR_EINVAL;
    return OR_OK;
}

int oracle_glu_fast(const double* I, int H, int W, const double* L, int s, int S, double eps,
                    double unit, int32_t* ka, int32_t* kb, double* omega, double* err,
                    double* gap_a, double* gap_b, int threads) {
    if (check_common(I, H, W, L, s, S) || !ka || !kb || !omega || !err || !(unit > 0.0))
        return OR_EINVAL;
    int h, w;
    oracle_lr_dims(H, W, s, &h, &w);
    eps *= unit;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(threads > 0 ? threads : omp_get_max_threads())
#endif
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            fast_pixel(I, H, W, L, h, w, s, S, eps, y, x, &ka[p], &kb[p], &omega[p], &err[p],
                       gap_a ? &gap_a[p] : NULL, gap_b ? &gap_b[p] : NULL);
            err[p] /= unit;
            if (gap_a) gap_a[p] /= unit;
            if (gap_b) gap_b[p] /= unit;
        }
    (void)threads;
    return OR_OK;
}

/* Evaluate a given window pair (k_a, k_b) at HR pixel (y, x) with the Eq. 5 weight. */
int oracle_fast_pair(const double* I, int H, int W, const double* L, int s, int S, double eps,
                     double unit, int y, int x, int ka, int kb, double* omega, double* err) {
    if (check_common(I, H, W, L, s, S) || y < 0 || y >= H || x < 0 || x >= W || !(unit > 0.0))
        return OR_EINVAL;
    int h, w, r = (S - 1) / 2;
    oracle_lr_dims(H, W, s, &h, &w);
    int va = y / s + ka / S - r, ua = x / s + ka % S - r;
    int vb = y / s + kb / S - r, ub = x / s + kb % S - r;
    if (va < 0 || va >= h || ua < 0 || ua >= w || vb < 0 || vb >= h || ub < 0 || ub >= w)
        return OR_EINVAL;
    fast_pair_eval(&I[((size_t)y * W + x) * 3], &L[((size_t)va * w + ua) * 3],
                   &L[((size_t)vb * w + ub) * 3], eps * unit, omega, err);
    *err /= unit;
    return OR_OK;
}

/* GLU* of Sec. 3.1: exhaustive pairs with the least-squares weight of Eq. 4. */
int oracle_glu_exact(const double* I, int H, int W, const double* L, int s, int S, double eps,
                     double unit, int32_t* ka, int32_t* kb, double* omega, double* err,
                     int threads) {
    if (check_common(I, H, W, L, s, S) || !ka || !kb || !omega || !err || !(unit > 0.0))
        return OR_EINVAL;
    int h, w;
    oracle_lr_dims(H, W, s, &h, &w);
    eps *= unit * unit;  /* Eq. 4's eps adds to a squared colour distance */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(threads > 0 ? threads : omp_get_max_threads())
#endif
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            window_t win;
            gather_window(L, h, w, s, S, y, x, &win);
            const double* Ip = &I[p * 3];
            if (win.n == 1) {
                ka[p] = kb[p] = win.k[0];
                omega[p] = 1.0;
                err[p] = dist3(Ip, win.col[0]) / unit;
                continue;
            }
            double best = INFINITY, bom = 1.0;
            int ba = 0, bb = 1;
            for (int i = 0; i < win.n; ++i)
                for (int j = i + 1; j < win.n; ++j) {
                    double om, e;
                    exact_pair_eval(Ip, win.col[i], win.col[j], eps, &om, &e);
                    if (e < best) { best = e; bom = om; ba = i; bb = j; }
                }
            ka[p] = win.k[ba];
            kb[p] = win.k[bb];
            omega[p] = bom;
            err[p] = best / unit;
        }
    (void)threads;
    return OR_OK;
}

/* GNU: weight fixed to 1 (Sec. 3.2), so the reconstruction is the nearest-colour LR pixel. */
int oracle_glu_gnu(const double* I, int H, int W, const double* L, int s, int S, double unit,
                   int32_t* ka, double* err) {
    if (check_common(I, H, W, L, s, S) || !ka || !err || !(unit > 0.0)) return OR_EINVAL;
    int h, w;
    oracle_lr_dims(H, W, s, &h, &w);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            window_t win;
            gather_window(L, h, w, s, S, y, x, &win);
            int ia = 0;
            double da = INFINITY;
            for (int i = 0; i < win.n; ++i) {
                double d = dist3(&I[p * 3], win.col[i]);
                if (d < da) { da = d; ia = i; }
            }
            ka[p] = win.k[ia];
            err[p] = da / unit;
        }
    return OR_OK;
}

/* ------------------------------------------------------------------ apply (Eq. 1) and adjoint */

static inline size_t lr_index(int y, int x, int s, int S, int k, int w) {
    int r = (S - 1) / 2;
    int v = y / s + k / S - r, u = x / s + k % S - r;
    return (size_t)v * w + u;
}

int oracle_apply(const int32_t* ka, const int32_t* kb, const double* omega, int H, int W, int s,
                 int S, const double* T, int C, double* out) {
    if (!ka || !kb || !omega || !T || !out || H <= 0 || W <= 0 || s <= 0 || C <= 0) return OR_EINVAL;
    int h, w;
    oracle_lr_dims(H, W, s, &h, &w);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            size_t a = lr_index(y, x, s, S, ka[p], w), b = lr_index(y, x, s, S, kb[p], w);
            for (int c = 0; c < C; ++c)
                out[p * C + c] = omega[p] * T[a * C + c] + (1.0 - omega[p]) * T[b * C + c];
        }
    return OR_OK;
}

/* Adjoint of Eq. 1 for a loss with gradient G w.r.t. the HR output: the LR target receives
 * omega * G_p at a_p and (1 - omega) * G_p at b_p; d/d omega_p = G_p . (T_a - T_b).
 * Sums run in raster order of p. */
int oracle_apply_adjoint(const int32_t* ka, const int32_t* kb, const double* omega, int H, int W,
                         int s, int S, const double* T, int C, const double* G, double* gT,
                         double* gomega) {
    if (!ka || !kb || !omega || !T || !G || !gT || H <= 0 || W <= 0 || s <= 0 || C <= 0) return OR_EINVAL;
    int h, w;
    oracle_lr_dims(H, W, s, &h, &w);
    memset(gT, 0, sizeof(double) * (size_t)h * w * C);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            size_t a = lr_index(y, x, s, S, ka[p], w), b = lr_index(y, x, s, S, kb[p], w);
            double go = 0.0;
            for (int c = 0; c < C; ++c) {
                gT[a * C + c] += omega[p] * G[p * C + c];
                gT[b * C + c] += (1.0 - omega[p]) * G[p * C + c];
                go += G[p * C + c] * (T[a * C + c] - T[b * C + c]);
            }
            if (gomega) gomega[p] = go;
        }
    return OR_OK;
}

/* ------------------------------------- least-squares LR colour update (non-paper, NEXT-F4) */

/* One update of the LR colours L for a fixed Theta: every LR pixel q independently takes the
 * value that minimises the reconstruction error sum_p || T_hat_p - I_p ||^2 of Eq. 1 (T = L)
 * with every other LR pixel held at its current value (a Jacobi sweep of the normal equations).
 * Pixel p reconstructs c_pa L_a + c_pb L_b with c_pa = omega_p, c_pb = 1 - omega_p, or L_a alone
 * (c = 1) when a_p = b_p; so q collects, over the pixels that use it,
 *     num_q += c_pq (I_p - c_pj L_j)   (j the other LR pixel of p, if any),   den_q += c_pq^2,
 * and L'_q = num_q / den_q clamped to the colour range [0, unit]; an LR pixel no pixel uses keeps
 * its value. Sums in raster order of p. */
int oracle_ls_update(const double* I, int H, int W, const double* L, int s, int S,
                     const int32_t* ka, const int32_t* kb, const double* omega, double unit,
                     double* Lout) {
    if (!I || !L || !ka || !kb || !omega || !Lout || H <= 0 || W <= 0 || s <= 0 || S <= 0 ||
        !(S & 1) || !(unit > 0.0))
        return OR_EINVAL;
    int h, w;
    oracle_lr_dims(H, W, s, &h, &w);
    size_t nq = (size_t)h * w;
    double* num = (double*)calloc(nq * 3, sizeof(double));
    double* den = (double*)calloc(nq, sizeof(double));
    if (!num || !den) {
        free(num);
        free(den);
        return OR_ENOMEM;
    }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            size_t a = lr_index(y, x, s, S, ka[p], w), b = lr_index(y, x, s, S, kb[p], w);
            const double* Ip = &I[p * 3];
            if (a == b) {
                for (int c = 0; c < 3; ++c) num[a * 3 + c] += Ip[c];
                den[a] += 1.0;
                continue;
            }
            double ca = omega[p], cb = 1.0 - omega[p];
            for (int c = 0; c < 3; ++c) {
                num[a * 3 + c] += ca * (Ip[c] - cb * L[b * 3 + c]);
                num[b * 3 + c] += cb * (Ip[c] - ca * L[a * 3 + c]);
            }
            den[a] += ca * ca;
            den[b] += cb * cb;
        }
    for (size_t q = 0; q < nq; ++q)
        for (int c = 0; c < 3; ++c) {
            double v = den[q] > 0.0 ? num[q * 3 + c] / den[q] : L[q * 3 + c];
            Lout[q * 3 + c] = v < 0.0 ? 0.0 : (v > unit ? unit : v);
        }
    free(num);
    free(den);
    return OR_OK;
}

/* --------------------------------------------------- connected components (Algorithm 2, step 3) */

/* Label the set pixels of mask; components numbered 0..M-1 in ascending order of their smallest
 * raster index (a raster scan meets each component first at that pixel). Returns M or < 0. */
int oracle_label_components(const uint8_t* mask, int H, int W, int conn, int32_t* labels) {
    if (!mask || !labels || H <= 0 || W <= 0 || (conn != 4 && conn != 8)) return OR_EINVAL;
    size_t n = (size_t)H * W;
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
    if (!queue) return OR_ENOMEM;
    for (size_t p = 0; p < n; ++p) labels[p] = -1;
    int M = 0;
    for (size_t p0 = 0; p0 < n; ++p0) {
        if (!mask[p0] || labels[p0] >= 0) continue;
        size_t head = 0, tail = 0;
        queue[tail++] = (int32_t)p0;
        labels[p0] = M;
        while (head < tail) {
            int32_t p = queue[head++];
            int y = p / W, x = p % W;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dy && !dx) continue;
                    if (conn == 4 && dy && dx) continue;
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    size_t q = (size_t)yy * W + xx;
                    if (mask[q] && labels[q] < 0) {
                        labels[q] = M;
                        queue[tail++] = (int32_t)q;
                    }
                }
        }
        ++M;
    }
    free(queue);
    return M;
}

/* --------------------------------------------------------------- joint optimisation (Alg. 2) */

/* Per-iteration statistics, 11 doubles each, after a leading R_0:
 *   [n_large, M, accepted, rolled_back, residual, min nonzero |e1 - e0|, min |E_p - tau|,
 *    pixels searched, decisions replayed, argmax near-ties, argmax choices replayed]
 * An argmax near-tie is a block [q_up] of a component where the largest error and the error of
 * another pixel of a different colour are within 1e-6: a lower-precision implementation may
 * then pick the other pixel, which is as correct to its precision.
 *
 * Replay (verification of a lower-precision implementation): when `force` is given, a trial
 * whose FP64 margin |e1 - e0| is at most force_tol (in [0, 1] units) takes the decision
 * force[t] (t counts trials across iterations in order) instead of its own; such a margin is
 * below the resolution of the other implementation's sums, so either decision is correct.
 * Every other trial decides by the rule e1 > e0 as usual.
 *
 * Argmax replay (same purpose): `amax` holds amax_n records of four int32 (iteration from 0,
 * component, LR pixel, HR pixel), sorted by (iteration, component, LR pixel): the other
 * implementation's choice of the pixel whose colour replaces that LR pixel. Where that pixel
 * differs from the oracle's own argmax, belongs to the component and to the block, and its FP64
 * error is within amax_tol (in [0, 1] units) of the block's largest, the oracle takes it: the
 * two errors are then closer than the other implementation's resolution, so either choice is
 * correct. Any other record is ignored (a different choice then shows up as a difference).
 * Records (256 + iteration, HR pixel, membership, 0) in the same array give the other
 * implementation's large-error membership of pixels near tau; where the oracle's own error is
 * within thr_tol of tau (FP64), it takes that membership. */
#define JSTAT 12

/* Index of record (it, j, q) in the sorted array, or -1. */
static int64_t find_amax(const int32_t* a, int64_t n, int32_t it, int32_t j, int32_t q) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        const int32_t* r = &a[mid * 4];
        const int less = r[0] < it || (r[0] == it && (r[1] < j || (r[1] == j && r[2] < q)));
        if (less) lo = mid + 1; else hi = mid;
    }
    if (lo < n && a[lo * 4] == it && a[lo * 4 + 1] == j && a[lo * 4 + 2] == q) return lo;
    return -1;
}

int oracle_joint(const double* I, int H, int W, int s, int S, double eps, double tau,
                 double unit, int N, int strict, int conn, double* L, int32_t* ka, int32_t* kb,
                 double* omega, double* err, double* stats, int8_t* accept_log, int64_t log_cap,
                 const int8_t* force, int64_t force_n, double force_tol, const int32_t* amax,
                 int64_t amax_n, double amax_tol, double thr_tol, int threads) {
    if (!I || !L || !ka || !kb || !omega || !err || H <= 0 || W <= 0 || s <= 0 || S < 1 ||
        S > 9 || (S % 2) == 0 || N < 0 || (conn != 4 && conn != 8) || !(unit > 0.0))
        return OR_EINVAL;
    /* E, e0, e1 and the residual are kept in the caller's units internally (err is converted
     * to [0, 1] units on return); tau is compared in the same units */
    tau *= unit;
    int h, w, r = (S - 1) / 2;
    oracle_lr_dims(H, W, s, &h, &w);
    size_t n = (size_t)H * W, nl = (size_t)h * w;

    /* initialise the LR image by regular grid downsampling, then Theta and E by Algorithm 1 */
    eps *= unit;
    oracle_downsample_grid(I, H, W, 3, s, L);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(threads > 0 ? threads : omp_get_max_threads())
#endif
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            fast_pixel(I, H, W, L, h, w, s, S, eps, y, x, &ka[p], &kb[p], &omega[p], &err[p],
                       NULL, NULL);
        }

    uint8_t* mask = (uint8_t*)malloc(n);
    int32_t* lab = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * n);     /* pixels grouped by component */
    int32_t* cstart = (int32_t*)malloc(sizeof(int32_t) * (n + 1));
    int32_t* lr_stamp = (int32_t*)malloc(sizeof(int32_t) * nl);
    int32_t* lr_list = (int32_t*)malloc(sizeof(int32_t) * nl);
    int32_t* aff = (int32_t*)malloc(sizeof(int32_t) * n);       /* A_i pixel list */
    double* backup = (double*)malloc(sizeof(double) * 3 * nl);
    int32_t* tka = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* tkb = (int32_t*)malloc(sizeof(int32_t) * n);
    double* tom = (double*)malloc(sizeof(double) * n);
    double* ter = (double*)malloc(sizeof(double) * n);
    double* qval = (double*)malloc(sizeof(double) * 3 * nl);
    double* qbest = (double*)malloc(sizeof(double) * nl);
    int32_t* qpix = (int32_t*)malloc(sizeof(int32_t) * nl);
    int rc = OR_OK;
    if (!mask || !lab || !order || !cstart || !lr_stamp || !lr_list || !aff || !backup || !tka ||
        !tkb || !tom || !ter || !qval || !qbest || !qpix) {
        rc = OR_ENOMEM;
        goto done;
    }
    for (size_t q = 0; q < nl; ++q) lr_stamp[q] = -1;

    double R_prev = 0.0;
    for (size_t p = 0; p < n; ++p) R_prev += err[p];
    if (stats) stats[0] = R_prev / unit;
    int64_t nlog = 0;
    int32_t stamp = 0;

    for (int it = 1; it <= N; ++it) {
        double* st = stats ? &stats[1 + (size_t)(it - 1) * JSTAT] : NULL;
        /* the set of pixels with large error */
        size_t nlarge = 0;
        double thr_margin = INFINITY;
        int thr_replayed = 0;
        for (size_t p = 0; p < n; ++p) {
            mask[p] = err[p] > tau;
            double m = fabs(err[p] - tau);
            if (m < thr_margin) thr_margin = m;
            if (amax && m <= thr_tol * unit) {
                /* the record's third field is the membership: look for either value */
                int64_t k = find_amax(amax, amax_n, 256 + it - 1, (int32_t)p, 0);
                if (k < 0) k = find_amax(amax, amax_n, 256 + it - 1, (int32_t)p, 1);
                if (k >= 0 && (uint8_t)(amax[k * 4 + 2] != 0) != mask[p]) {
                    mask[p] = amax[k * 4 + 2] != 0;
                    ++thr_replayed;
                }
            }
            nlarge += mask[p];
        }
        if (st) {
            for (int j = 0; j < JSTAT; ++j) st[j] = 0.0;
            st[0] = (double)nlarge;
            st[6] = thr_margin / unit;
            st[11] = thr_replayed;
        }
        if (nlarge == 0) break;
        int M = oracle_label_components(mask, H, W, conn, lab);
        if (M < 0) { rc = M; goto done; }
        /* group pixels by component, raster order inside each */
        for (int i = 0; i <= M; ++i) cstart[i] = 0;
        for (size_t p = 0; p < n; ++p)
            if (lab[p] >= 0) cstart[lab[p] + 1]++;
        for (int i = 0; i < M; ++i) cstart[i + 1] += cstart[i];
        {
            int32_t* fillp = tka; /* scratch reuse: per-component fill cursor */
            for (int i = 0; i < M; ++i) fillp[i] = cstart[i];
            for (size_t p = 0; p < n; ++p)
                if (lab[p] >= 0) order[fillp[lab[p]]++] = (int32_t)p;
        }
        int accepted = 0, rolled = 0, replayed = 0, argmax_ties = 0, amax_replayed = 0;
        double min_dec = INFINITY, searched = 0.0;

        for (int ci = 0; ci < M; ++ci) {
            const int32_t* Cp = &order[cstart[ci]];
            int csz = cstart[ci + 1] - cstart[ci];
            /* Q: LR pixels whose HR block meets C_i; per q the largest-error pixel of C_i there */
            ++stamp;
            int nq = 0;
            for (int t = 0; t < csz; ++t) {
                int p = Cp[t], y = p / W, x = p % W;
                int q = (y / s) * w + (x / s);
                if (lr_stamp[q] != stamp) {
                    lr_stamp[q] = stamp;
                    lr_list[nq++] = q;
                    qbest[q] = -1.0;
                }
                if (err[p] > qbest[q]) { /* strict: the lowest raster index wins ties */
                    qbest[q] = err[p];
                    qpix[q] = p;
                    for (int c = 0; c < 3; ++c) qval[(size_t)q * 3 + c] = I[(size_t)p * 3 + c];
                }
            }
            for (int t = 0; t < csz; ++t) {
                int p = Cp[t], y = p / W, x = p % W;
                int q = (y / s) * w + (x / s);
                if (p != qpix[q] && !same3(&I[(size_t)p * 3], &I[(size_t)qpix[q] * 3]) &&
                    qbest[q] - err[p] <= 1e-6 * unit)
                    ++argmax_ties;
            }
            if (amax) {
                for (int t = 0; t < nq; ++t) {
                    int q = lr_list[t];
                    int64_t k = find_amax(amax, amax_n, it - 1, ci, q);
                    if (k < 0) continue;
                    int pg = amax[k * 4 + 3];
                    if (pg == qpix[q] || pg < 0 || (size_t)pg >= n || lab[pg] != ci) continue;
                    if ((pg / W) / s * w + (pg % W) / s != q) continue;
                    if (!(err[pg] >= qbest[q] - amax_tol * unit)) continue;
                    qpix[q] = pg;
                    for (int c = 0; c < 3; ++c) qval[(size_t)q * 3 + c] = I[(size_t)pg * 3 + c];
                    ++amax_replayed;
                }
            }
            /* the pixels whose Theta and E are re-optimised and summed */
            int na = 0;
            if (strict) {
                ++stamp;
                int nb = 0;
                for (int t = 0; t < nq; ++t) {
                    int q = lr_list[t], qv = q / w, qu = q % w;
                    for (int dv = -r; dv <= r; ++dv)
                        for (int du = -r; du <= r; ++du) {
                            int v = qv + dv, u = qu + du;
                            if (v < 0 || v >= h || u < 0 || u >= w) continue;
                            int b = v * w + u;
                            if (lr_stamp[b] == stamp) continue;
                            lr_stamp[b] = stamp;
                            aff[nb++] = b; /* temporarily the LR block list */
                        }
                }
                /* expand blocks to HR pixels; the block list is tiny relative to aff's size */
                int32_t* blocks = (int32_t*)malloc(sizeof(int32_t) * (nb ? nb : 1));
                if (!blocks) { rc = OR_ENOMEM; goto done; }
                memcpy(blocks, aff, sizeof(int32_t) * nb);
                for (int t = 0; t < nb; ++t) {
                    int v = blocks[t] / w, u = blocks[t] % w;
                    for (int y = v * s; y < imin(H, v * s + s); ++y)
                        for (int x = u * s; x < imin(W, u * s + s); ++x) aff[na++] = y * W + x;
                }
                free(blocks);
            } else {
                for (int t = 0; t < csz; ++t) aff[na++] = Cp[t];
            }
            /* e0 over the current error map */
            double e0 = 0.0;
            for (int t = 0; t < na; ++t) e0 += err[aff[t]];
            /* back up and replace the LR colours of Q */
            for (int t = 0; t < nq; ++t) {
                int q = lr_list[t];
                for (int c = 0; c < 3; ++c) {
                    backup[(size_t)t * 3 + c] = L[(size_t)q * 3 + c];
                    L[(size_t)q * 3 + c] = qval[(size_t)q * 3 + c];
                }
            }
            /* re-run Algorithm 1 on the affected pixels */
            double e1 = 0.0;
            for (int t = 0; t < na; ++t) {
                int p = aff[t];
                fast_pixel(I, H, W, L, h, w, s, S, eps, p / W, p % W, &tka[t], &tkb[t], &tom[t],
                           &ter[t], NULL, NULL);
                e1 += ter[t];
            }
            searched += na;
            double dm = fabs(e1 - e0);
            if (dm > 0.0 && dm < min_dec) min_dec = dm;
            int accept = !(e1 > e0);
            if (force && nlog < force_n && dm <= force_tol * unit && (force[nlog] & ~1) == 0 &&
                force[nlog] != accept) {
                accept = force[nlog];
                ++replayed;
            }
            if (accept) {
                for (int t = 0; t < na; ++t) {
                    int p = aff[t];
                    ka[p] = tka[t]; kb[p] = tkb[t]; omega[p] = tom[t]; err[p] = ter[t];
                }
                ++accepted;
            } else {
                for (int t = 0; t < nq; ++t) {
                    int q = lr_list[t];
                    for (int c = 0; c < 3; ++c) L[(size_t)q * 3 + c] = backup[(size_t)t * 3 + c];
                }
                ++rolled;
            }
            if (accept_log && nlog < log_cap) accept_log[nlog] = (int8_t)accept;
            ++nlog;
        }
        double R = 0.0;
        for (size_t p = 0; p < n; ++p) R += err[p];
        if (st) {
            st[1] = M; st[2] = accepted; st[3] = rolled; st[4] = R / unit; st[5] = min_dec / unit;
            st[7] = searched; st[8] = replayed; st[9] = argmax_ties; st[10] = amax_replayed;
            st[11] = thr_replayed;
        }
        if (accepted == 0 || !(R < R_prev)) break;
        R_prev = R;
    }
done:
    for (size_t p = 0; p < n; ++p) err[p] /= unit;
    free(mask); free(lab); free(order); free(cstart); free(lr_stamp); free(lr_list); free(aff);
    free(backup); free(tka); free(tkb); free(tom); free(ter); free(qval); free(qbest); free(qpix);
    return rc;
}

/* ------------------------------------------- LR operators (the black-box f of the workloads) */

/* 3x3 box blur with clamped (replicated) edges. */
int oracle_op_box3(const double* X, int h, int w, int C, double* Y) {
    for (int v = 0; v < h; ++v)
        for (int u = 0; u < w; ++u)
            for (int c = 0; c < C; ++c) {
                double acc = 0.0;
                for (int dv = -1; dv <= 1; ++dv)
                    for (int du = -1; du <= 1; ++du) {
                        int vv = v + dv < 0 ? 0 : (v + dv >= h ? h - 1 : v + dv);
                        int uu = u + du < 0 ? 0 : (u + du >= w ? w - 1 : u + du);
                        acc += X[((size_t)vv * w + uu) * C + c];
                    }
                Y[((size_t)v * w + u) * C + c] = acc / 9.0;
            }
    return OR_OK;
}

/* 3x3 Gaussian [1 2 1]/4 x [1 2 1]/4 with clamped edges. */
int oracle_op_gauss3(const double* X, int h, int w, int C, double* Y) {
    static const double k[3] = {0.25, 0.5, 0.25};
    for (int v = 0; v < h; ++v)
        for (int u = 0; u < w; ++u)
            for (int c = 0; c < C; ++c) {
                double acc = 0.0;
                for (int dv = -1; dv <= 1; ++dv)
                    for (int du = -1; du <= 1; ++du) {
                        int vv = v + dv < 0 ? 0 : (v + dv >= h ? h - 1 : v + dv);
                        int uu = u + du < 0 ? 0 : (u + du >= w ? w - 1 : u + du);
                        acc += k[dv + 1] * k[du + 1] * X[((size_t)vv * w + uu) * C + c];
                    }
                Y[((size_t)v * w + u) * C + c] = acc;
            }
    return OR_OK;
}

/* Saturation about the Rec. 601 luma: Y + f (c - Y), clamped to [0, 1]. In place allowed. */
int oracle_op_saturation(const double* X, size_t npix, double f, double* Y) {
    for (size_t p = 0; p < npix; ++p) {
        double luma = 0.299 * X[p * 3] + 0.587 * X[p * 3 + 1] + 0.114 * X[p * 3 + 2];
        for (int c = 0; c < 3; ++c) {
            double v = luma + f * (X[p * 3 + c] - luma);
            Y[p * 3 + c] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
        }
    }
    return OR_OK;
}

/* Per-channel gamma x^g on [0, 1]. In place allowed. */
int oracle_op_gamma(const double* X, size_t n, double g, double* Y) {
    for (size_t i = 0; i < n; ++i) Y[i] = X[i] > 0.0 ? pow(X[i], g) : 0.0;
    return OR_OK;
}
