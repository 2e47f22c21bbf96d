/*
 * glu.h — C ABI of the GB300 (sm_103a) Guided Linear Upsampling library (libglu.so).
 *
 * Method: Song et al., "Guided Linear Upsampling", ACM TOG 2023. Every HR pixel p is represented
 * as T_p = w * T_a + (1 - w) * T_b with a, b two LR pixels of a small window around p's LR
 * position (Eq. 1); the pair and weight are chosen on the guide image alone (Eq. 3, Algorithm 1)
 * and can then be applied to any processed LR image. The LR image itself can be re-optimised
 * jointly with the parameters (Eq. 6, Algorithm 2).
 *
 * Conventions shared by every call
 *  - All image / parameter buffers are DEVICE memory owned by the caller, unless a comment says
 *    "host". The library never allocates on these calls and keeps no pointer after returning.
 *  - Host threads: every entry point may be called from several host threads at once (each on
 *    its own stream); host-side parameter blocks are per call. The joint calls share one graph
 *    cache and are serialised by a library-wide lock while they issue their launches. The
 *    profiling switch (glu_joint_profile) and the test hooks are process-wide settings.
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy
 *    default stream) unless stated otherwise. Errors in the arguments are reported
 *    synchronously by the return value; no exception crosses the ABI.
 *  - Return value: GLU_OK (0) or a negative GLU_ERR_* code; glu_status_string() names it.
 *  - Colour units: GLU_U8 images hold colour * 255 (0..255); GLU_F16 / GLU_F32 images hold
 *    colours in [0, 1]. Error maps, eps and tau are in [0, 1] colour units.
 *  - Geometry: for an H x W HR image and integer scale s, the LR image is h x w with
 *    h = ceil(H / s), w = ceil(W / s). HR pixel (y, x) lies in LR block (y / s, x / s).
 *    The window of that block is the S x S LR neighbourhood centred on it, clipped to the
 *    image; window index k = (dy + r) * S + (dx + r), r = (S - 1) / 2.
 *  - Theta (the paper's 3 x H x W parameter tensor) is stored as a uint16 pair code
 *    code = k_a * S * S + k_b per HR pixel (row-major, H x W, no padding) plus a weight plane.
 */
#ifndef GLU_H
#define GLU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------- status codes */
#define GLU_OK 0
#define GLU_ERR_INVALID_ARG (-1)   /* null pointer, bad enum, bad parameter value */
#define GLU_ERR_SHAPE (-2)         /* image sizes inconsistent with each other or the scale */
#define GLU_ERR_UNSUPPORTED (-3)   /* valid but not implemented combination (dtype, S, ...) */
#define GLU_ERR_WORKSPACE (-4)     /* workspace missing or smaller than *_workspace_size() */
#define GLU_ERR_CUDA (-5)          /* a CUDA runtime call failed (launch, copy, attribute) */
#define GLU_ERR_DEVICE_CHECK (-6)  /* a kernel's own bounds/consistency check fired */
#define GLU_ERR_TIMEOUT (-7)       /* a bounded device-side wait gave up */

/* ------------------------------------------------------------------------------- types */
typedef enum { GLU_U8 = 0, GLU_F16 = 1, GLU_F32 = 2 } glu_dtype;

/* An image: h rows of w pixels with c interleaved channels; row r starts at
 * data + r * pitch elements (pitch >= w * c). */
typedef struct {
    void* data;
    int32_t h, w, c;
    int32_t dtype;      /* glu_dtype */
    int64_t pitch;      /* elements between consecutive row starts */
} glu_image;

typedef enum { GLU_W_F32 = 0, GLU_W_F16 = 1, GLU_W_UNORM16 = 2 } glu_wfmt;

/* Theta for an H x W HR image at scale `scale` with an S x S window. */
typedef struct {
    uint16_t* code;     /* H * W pair codes, k_a * S * S + k_b */
    void* weight;       /* H * W weights w in [0, 1] (Eq. 5) stored as `wfmt` */
    int32_t H, W, scale, S;  /* 0 < H < 2^22 */
    int32_t wfmt;       /* glu_wfmt; UNORM16 stores round(w * 65535) */
} glu_theta;

/* FAST: Algorithm 1 (Eq. 5 weight). GNU: weight fixed to 1. EXACT: GLU* (Sec. 3.1) — every
 * unordered pair k_a < k_b of window pixels with the Eq. 4 least-squares weight (not clamped, so
 * weights may leave [0, 1]: float32 weight storage only); quadratic in the window size. */
typedef enum { GLU_MODE_FAST = 0, GLU_MODE_GNU = 1, GLU_MODE_EXACT = 2 } glu_mode;
typedef enum { GLU_JOINT_STRICT = 0, GLU_JOINT_PAPER = 1 } glu_joint_mode;
typedef enum { GLU_DOWN_GRID = 0, GLU_DOWN_BOX = 1 } glu_down_mode;

typedef struct {
    int32_t S;            /* odd window size 1..9 (the paper uses 3, Sec. 5.3) */
    float eps;            /* epsilon of Eq. 4 / Eq. 5 (paper: 1e-3, Sec. 3.1) */
    float tau;            /* large-error threshold of Algorithm 2 (paper: 30/255) */
    int32_t N;            /* maximum iterations of Algorithm 2 (paper: 3), <= GLU_MAX_ITERS */
    int32_t mode;         /* glu_mode: Algorithm 1, the weight-1 special case (GNU), or GLU* */
    int32_t joint;        /* glu_joint_mode: STRICT (default) or PAPER reading of Algorithm 2 */
    int32_t connectivity; /* 8 (default) or 4: adjacency of large-error components */
} glu_params;

#define GLU_MAX_ITERS 32

/* Host-side statistics of glu_joint_optimize. */
typedef struct {
    int32_t iterations;                  /* iterations whose trials ran */
    int32_t n_large[GLU_MAX_ITERS];      /* |E| = #{p : E_p > tau} at the start of iteration n */
    int32_t components[GLU_MAX_ITERS];   /* M, connected components of that set */
    int32_t accepted[GLU_MAX_ITERS];     /* trials kept (e1 <= e0) */
    int32_t rolled_back[GLU_MAX_ITERS];  /* trials undone (e1 > e0) */
    double residual[GLU_MAX_ITERS + 1];  /* R_0 .. R_n = sum_p E_p, FP64, fixed-order reduction */
    int64_t searched[GLU_MAX_ITERS];     /* HR pixels re-run through Algorithm 1 by the trials */
    uint32_t multi_kernel_lists;         /* bit n: iteration n's components and trial dependency
                                            graph were built by the multi-kernel path (a large-
                                            error list of more than 4096 pixels or one the single
                                            CTA could not finish); clear: by one CTA (or nothing
                                            to build) and, inside a recorded graph, the path's 15
                                            kernels did not launch (the whole batch; per call) */
} glu_joint_stats;

/* Fill *p with the paper's parameters: S = 3, eps = 1e-3, tau = 30/255, N = 3, FAST, STRICT,
 * 8-connectivity (Sec. 3.1 and Sec. 5.3). */
void glu_params_default(glu_params* p);

/* ------------------------------------------------------------------------- entry points */

/* Downsample an HR image by integer factor `scale` (Sec. 3.3).
 *  GLU_DOWN_GRID: regular grid sampling — LR pixel (v, u) copies HR pixel
 *      (v*s + e_y/2, u*s + e_x/2), e = extent of the block (s, or less for the last one).
 *      hr: U8/F16/F32; lr: same dtype as hr, or F32.
 *  GLU_DOWN_BOX: mean of the block (not the paper's default; a filtered LR image for GLU
 *      without joint optimisation). hr: U8/F16/F32; lr: F32 or F16.
 *  c must be equal on both sides (1..4); lr->h, lr->w must be ceil(H/s), ceil(W/s). */
int glu_downsample(const glu_image* hr, int32_t scale, int32_t mode, glu_image* lr, void* stream);

/* Algorithm 1 (Sec. 3.2) for every HR pixel: a = the window pixel nearest in colour to I_p
 * (ties: lowest k), then b over the whole window (b = a included) with the Eq. 5 weight,
 * minimising the Eq. 3 error (ties: lowest k_b). mode GNU fixes w = 1 (b = a).
 *  hr: U8 or F16, c = 3. lr: U8, F16 or F32, c = 3, h x w = ceil(H/s) x ceil(W/s) where
 *  s = theta->scale. theta: H, W, scale, S (= params->S) and wfmt set by the caller; code and
 *  weight are written. err_map (nullable): H * W floats, E_p = ||I_p - I_hat_p|| in [0, 1]
 *  units, row-major without padding. */
int glu_optimize(const glu_image* hr, const glu_image* lr, const glu_params* params,
                 glu_theta* theta, float* err_map, void* stream);

/* Algorithm 2 (Sec. 3.3): joint optimisation of the downsampled image and Theta.
 * Initialises lr_out by regular grid downsampling of hr, Theta and E by Algorithm 1, then
 * runs up to params->N iterations of: threshold E > tau, 8-connected components in order of
 * their smallest raster index, and per component the trial replacement of the LR colours of
 * the blocks it meets by its largest-error pixel there, re-optimisation and rollback if the
 * summed error grows. STRICT sums and re-optimises every pixel whose window contains a replaced
 * LR pixel (exactly the pixels whose error can change); PAPER only the component's own pixels.
 * Stops early when the set is empty, when an iteration keeps no trial, or when the FP64
 * residual R_n = sum_p E_p stops decreasing. Components that cannot influence each other are
 * tried concurrently; the result equals the sequential order.
 *  hr: U8, c = 3. lr_out: U8, c = 3, ceil(H/s) x ceil(W/s). theta as for glu_optimize.
 *  err_map (nullable) as for glu_optimize. stats (HOST, nullable): if given, the call
 *  synchronises `stream` before returning and fills it. ws / ws_bytes: device workspace of at
 *  least glu_joint_workspace_size() bytes, 256-byte aligned; its contents need no init.
 *  A call repeated with identical arguments (pointers, sizes, parameters, workspace) is recorded
 *  as a CUDA graph on its second occurrence and replayed from then on (same kernels, same
 *  results, fewer launch gaps); the library keeps the most recent one. */
int glu_joint_optimize(const glu_image* hr, int32_t scale, const glu_params* params,
                       glu_image* lr_out, glu_theta* theta, float* err_map,
                       glu_joint_stats* stats, void* ws, size_t ws_bytes, void* stream);

/* Allocation-free variant of glu_joint_optimize (the paper has no counterpart: this is a
 * deployment aid). For callers that cannot allocate device memory — a plug-in inside an
 * application that owns every device allocation, or a streaming loop that must not risk the
 * device-wide synchronisation cudaMalloc / cudaFree can cause — the workspace is a fixed
 * GLU_JOINT_STATIC_BYTES array in the library's own device memory (held by every GPU that loads
 * the library until the process exits). Arguments and results as glu_joint_optimize, minus the
 * workspace. Returns GLU_ERR_WORKSPACE, before any launch, when glu_joint_workspace_size() for
 * this image exceeds GLU_JOINT_STATIC_BYTES: at scale 8, 5x5 window, 5 iterations that is about
 * 0.88 megapixels (1248 x 702 is the largest 16:9 image that fits, 1024 x 768 fits, 1280 x 720
 * does not). The first call in each device context looks up the array's device address with
 * that device current (and loads the library's device code there); make that first call before
 * any stream capture. All calls on a device share the array (each call initialises what it
 * reads); calls that overlap on the GPU race, so issue them one after another. Allocates
 * nothing and creates no stream, event or graph: every launch goes directly onto `stream`
 * (repeated calls are not recorded as a graph, unlike glu_joint_optimize) and the autotuner does
 * not time variants during the call. */
#define GLU_JOINT_STATIC_BYTES (64u << 20)
int glu_joint_optimize_static(const glu_image* hr, int32_t scale, const glu_params* params,
                              glu_image* lr_out, glu_theta* theta, float* err_map,
                              glu_joint_stats* stats, void* stream);

/* Workspace bytes glu_joint_optimize needs for an H x W image (0 on invalid arguments). */
size_t glu_joint_workspace_size(int32_t H, int32_t W, int32_t scale, const glu_params* params);

/* Verification aid (not part of the method): after a glu_joint_optimize call that used the
 * workspace ws (same H, W, scale, params), copy its trial decisions to HOST memory `out`:
 * for each iteration that ran, one byte per component in component order (1 kept, 0 rolled
 * back), iterations concatenated. Synchronous on `stream`. Returns the number of bytes written
 * or a negative GLU_ERR_* (GLU_ERR_INVALID_ARG if cap is too small). */
int64_t glu_joint_decisions(const void* ws, size_t ws_bytes, int32_t H, int32_t W, int32_t scale,
                            const glu_params* params, int8_t* out, int64_t cap, void* stream);

/* One image of a batched call (all pointers device memory). */
typedef struct {
    glu_image hr;       /* guide; U8 (or F16 for glu_optimize_batched), c = 3 */
    glu_image lr;       /* LR image: read by glu_optimize_batched, written by the joint call */
    glu_theta theta;    /* scale, S and wfmt per item; code and weight are written */
    float* err_map;     /* nullable, as for glu_optimize */
} glu_batch_item;

/* Algorithm 1 over n images of different sizes, scales and windows in one persistent launch
 * (per 32 images): every item's result equals a glu_optimize call on it alone. Each item's
 * window is item.theta.S (params->S is not used); eps and mode come from params. Every item must
 * share the guide dtype and theta.wfmt (GLU_ERR_UNSUPPORTED otherwise). n = 0 is a no-op. */
int glu_optimize_batched(const glu_batch_item* items, int32_t n, const glu_params* params,
                         void* stream);

/* Algorithm 2 over n <= 32 images in one set of launches: every item's LR image, Theta, error
 * map and statistics equal a glu_joint_optimize call on it alone (each image keeps its own
 * large-error sets, components, residuals and stopping rule). Each item's window is
 * item.theta.S; eps, tau, N, joint mode and connectivity come from params; all items share
 * theta.wfmt. stats: HOST array of n records, or null. ws: at least
 * glu_joint_batched_workspace_size() bytes, 256-byte aligned. */
int glu_joint_optimize_batched(const glu_batch_item* items, int32_t n, const glu_params* params,
                               glu_joint_stats* stats, void* ws, size_t ws_bytes, void* stream);

/* Workspace bytes glu_joint_optimize_batched needs (0 on invalid arguments). Reads only the
 * items' sizes and scales. */
size_t glu_joint_batched_workspace_size(const glu_batch_item* items, int32_t n,
                                        const glu_params* params);

/* Workspace bytes of one call of operation `op` for an H x W guide at `scale` with params (S, N):
 * the same number as that operation's own *_workspace_size query (the adjoint forms for c = 3
 * channels). 0 for an operation that takes no workspace (downsample, optimize, apply, theta
 * decode) and for invalid arguments, which the operation itself then reports. */
typedef enum {
    GLU_OP_DOWNSAMPLE = 0, GLU_OP_OPTIMIZE = 1, GLU_OP_APPLY = 2, GLU_OP_THETA_DECODE = 3,
    GLU_OP_JOINT = 4,               /* glu_joint_optimize */
    GLU_OP_LS_JOINT = 5,            /* glu_ls_joint_optimize */
    GLU_OP_LS_UPDATE = 6,           /* glu_ls_update */
    GLU_OP_APPLY_BACKWARD = 7,      /* glu_apply_backward_ws */
    GLU_OP_APPLY_BACKWARD_PLAN = 8  /* glu_apply_backward_plan's plan buffer */
} glu_op;
size_t glu_workspace_size(int32_t op, int32_t H, int32_t W, int32_t scale,
                          const glu_params* params);

/* Benchmark instrumentation (not part of the method). glu_joint_profile(1) makes later
 * glu_joint_optimize calls record CUDA events on their stream around their phases (calls replayed
 * as a CUDA graph record them as event nodes of the graph; each replay's times are collected
 * before the next replay is launched, which waits for it). The events of up to 64 directly issued
 * calls are kept. glu_joint_profile_read() waits for them, writes the summed milliseconds of
 * [control init + grid downsample, the Algorithm 1 search kernel, large-error set and components,
 * trials, residuals (R_0 and every R_n)] to ms[0..4] and the number of calls to *calls, then
 * forgets them. glu_joint_profile(0) stops recording. Host-side state; not thread-safe. */
int glu_joint_profile(int32_t enable);
int glu_joint_profile_read(float* ms, int32_t* calls);

/* Eq. 1: out_p = w_p * T_a + (1 - w_p) * T_b for every HR pixel (Algorithm 1, last step).
 *  lr_target: F32 or F16, c = 1..4, ceil(H/s) x ceil(W/s). hr_out: F32 or F16, same c,
 *  H x W. */
int glu_apply(const glu_theta* theta, const glu_image* lr_target, glu_image* hr_out,
              void* stream);

/* Theta decoded (Eq. 1's pair of LR pixels and weight, per HR pixel): for HR pixel p = y * W + x
 * with pair code k_a * S * S + k_b, a[p] = v_a * w + u_a where (v_a, u_a) = (y / s + k_a / S - r,
 * x / s + k_a % S - r), r = (S - 1) / 2 and w = ceil(W / s), likewise b[p] from k_b, and
 * w_out[p] the weight as float32. a, b, w_out: DEVICE buffers of H * W elements (row-major),
 * caller-owned; any of them may be null (not all three). A code that points outside its pixel's
 * (image-clipped) window writes -1 to a[p] and b[p] and records GLU_ERR_DEVICE_CHECK for
 * glu_device_status(). Asynchronous on `stream`. */
int glu_theta_decode(const glu_theta* theta, int32_t* a, int32_t* b, float* w_out, void* stream);

/* Adjoint of Eq. 1 with the pair choice held fixed. For an upstream gradient G (grad_hr,
 * F32, H x W x c):
 *   grad_lr_q = sum_{p : a_p = q} w_p G_p + sum_{p : b_p = q} (1 - w_p) G_p      (F32, h x w x c)
 *   grad_w_p  = G_p . (T_a - T_b)                                (nullable, F32, H * W, dense)
 * Each LR pixel sums its contributions in a fixed order (no atomics): results are
 * bit-reproducible. lr_target: F32, as passed to glu_apply. */
int glu_apply_backward(const glu_theta* theta, const glu_image* lr_target,
                       const glu_image* grad_hr, glu_image* grad_lr, float* grad_w, void* stream);

/* The same adjoint with a caller workspace (device memory, 16-byte aligned, at least
 * glu_apply_backward_workspace_size(theta, c) bytes: 8 c S^2 bytes per LR pixel; contents
 * scratch). A pixel of LR block B reaches exactly two LR pixels, one per window index, so every
 * block sums its pixels' contributions per window index once (raster order) into the slot of the
 * LR pixel it feeds, and each LR pixel then adds its S^2 slots (neighbour order, a before b):
 * every input is read once. Fixed summation order, no atomics: bit-reproducible (the order
 * differs from glu_apply_backward's, so the two agree to rounding). GLU_ERR_WORKSPACE if ws is
 * missing, misaligned or too small. */
size_t glu_apply_backward_workspace_size(const glu_theta* theta, int32_t c);

/* The adjoint for a Theta used by many calls (an LR operator fitted through the upsampler): a
 * plan, the inverse pixel-to-LR map of Theta's codes (every LR pixel's contributing HR pixels
 * and sides, neighbour blocks in order, a then b, raster order inside), is built once
 * (glu_apply_backward_plan: device memory of glu_apply_backward_plan_size bytes, 4-byte
 * aligned; valid while the codes do not change: the weights may), and each
 * glu_apply_backward_planned call reads every LR pixel's list once (a warp per LR pixel, lanes
 * strided over its entries, a fixed butterfly: bit-reproducible). Same results contract as
 * glu_apply_backward (its summation order differs). */
size_t glu_apply_backward_plan_size(const glu_theta* theta);
int glu_apply_backward_plan(const glu_theta* theta, void* plan, size_t plan_bytes, void* stream);
int glu_apply_backward_planned(const glu_theta* theta, const void* plan,
                               const glu_image* lr_target, const glu_image* grad_hr,
                               glu_image* grad_lr, float* grad_w, void* stream);
int glu_apply_backward_ws(const glu_theta* theta, const glu_image* lr_target,
                          const glu_image* grad_hr, glu_image* grad_lr, float* grad_w, void* ws,
                          size_t ws_bytes, void* stream);

/* Least-squares LR colour update (an alternative joint scheme beside Algorithm 2; not the
 * paper's method). For a fixed Theta every LR pixel q takes, independently, the colour that
 * minimises the Eq. 1 reconstruction error sum_p || T_hat_p - I_p ||^2 (T = the LR image) with
 * the other LR pixels held at their current values: with c_pa = w_p, c_pb = 1 - w_p (or the single
 * coefficient 1 when a_p = b_p), num_q = sum_p c_pq (I_p - c_pj L_j), den_q = sum_p c_pq^2 over the
 * pixels that use q, L'_q = num_q / den_q clamped to [0, 1]; an LR pixel no pixel uses keeps its
 * colour. Per-LR-pixel sums in FP32 with Kahan compensation in a fixed order (bit-reproducible).
 *  hr: U8 or F16 guide (3 channels); theta: F32 weights; lr_in / lr_out: F32, 3 channels, LR size
 *  (distinct buffers); ws: glu_ls_update_workspace_size(theta) bytes (32 S^2 per LR pixel),
 *  16-byte aligned. */
size_t glu_ls_update_workspace_size(const glu_theta* theta);
int glu_ls_update(const glu_image* hr, const glu_theta* theta, const glu_image* lr_in,
                  glu_image* lr_out, void* ws, size_t ws_bytes, void* stream);

/* Alternation of Algorithm 1 (reassignment) and glu_ls_update (LR colour update), starting from
 * grid downsampling: after each update Algorithm 1 runs on the new LR image, and the new state
 * (LR image, Theta, E) is kept only if its residual R = sum_p E_p is below the current one; the
 * first update that is not kept ends the loop (the remaining iterations change nothing). At most
 * params->N iterations; params->mode must be GLU_MODE_FAST. lr_out: F32, 3 channels; theta: F32
 * weights; err_map nullable; stats (nullable, host) synchronises the stream once at the end.
 * ws: glu_ls_joint_workspace_size bytes, 256-byte aligned. */
typedef struct {
    double R0;                          /* residual of the grid-downsampled start */
    double residual[GLU_MAX_ITERS];     /* residual of each iteration's candidate state (0 for
                                           iterations after the loop stopped) */
    int32_t iterations;                 /* candidate states computed (N) */
    int32_t kept;                       /* the last kept iteration (0: none) */
} glu_ls_stats;
size_t glu_ls_joint_workspace_size(int32_t H, int32_t W, int32_t scale, const glu_params* params);
int glu_ls_joint_optimize(const glu_image* hr, int32_t scale, const glu_params* params,
                          glu_image* lr_out, glu_theta* theta, float* err_map,
                          glu_ls_stats* stats, void* ws, size_t ws_bytes, void* stream);

/* Verification aid (not part of the method): log the decisions of Algorithm 2 that FP32 takes
 * on real-valued comparisons, so that an FP64 reference can follow them where its own values are
 * closer than FP32 resolution. While set, glu_joint_optimize / glu_joint_optimize_batched append
 * records of four int32 to the DEVICE buffer buf (16-byte aligned): buf[0] counts the records
 * written so far (the caller zeroes it before a call), the records follow from byte 16, at most
 * cap of them (further ones are counted, not stored), in no fixed order:
 *   (iteration, component, LR pixel, HR pixel): for each LR pixel a trial replaces, the HR pixel
 *       whose colour replaces it (the component's largest-error pixel in that block);
 *   (256 + iteration, HR pixel, 1 if in the large-error set else 0, 0): every pixel whose error
 *       is within 1e-5 of tau at that iteration's threshold pass.
 * Pixel indices are inside the pixel's own image. buf = NULL turns the log off. Process-wide;
 * not thread-safe. */
int glu_test_joint_argmax_log(void* buf, int64_t cap);

/* Test hook: the number of CUDA graphs glu_joint_optimize / glu_joint_optimize_batched have
 * recorded in this process so far (a repeated call is recorded once, then replayed). */
int64_t glu_test_joint_graph_count(void);

/* Test hook (failure detection): the deadline, in nanoseconds, of the waits of Algorithm 2's
 * trial kernel (the ready queue, the general path's items, the in-order fallback); 0 restores
 * the default (5 s plus 0.5 ms per component, at most 30 s). With a limit that runs out, the
 * waits give up, the kernel records GLU_ERR_TIMEOUT in its status word and returns, the call
 * with stats returns GLU_ERR_TIMEOUT and glu_device_status() reports it; the context stays
 * usable. Process-wide; not thread-safe. */
int glu_test_set_wait_limit(uint64_t ns);

/* Autotuner (not part of the method: implementation choice only). The Algorithm 1 search
 * (GLU_TUNE_SEARCH: tile height x CTAs per SM x candidate loop schedule) and the tiled Eq. 1
 * apply (GLU_TUNE_APPLY: tile height) have several implementation variants that compute the same
 * arithmetic in the same order, so every variant gives bit-identical results. A launch picks, in
 * order: the variant forced by glu_tune_force(); the cached choice for its shape class (guide or
 * output dtype, weight format or mode, window, scale, ceil(log2(pixels))); with tuning on
 * (glu_tune_mode(1)) and the stream not capturing a graph, the fastest variant timed on the
 * call's own inputs (that first call synchronises its stream and runs every variant 4 times);
 * otherwise variant 0. Choices are process-wide; glu_tune_export() / glu_tune_import() move them
 * between processes as text lines "kernel k0 k1 k2 k3 k4 variant ms". Thread-safe. */
#define GLU_TUNE_SEARCH 0
#define GLU_TUNE_APPLY 1
int glu_tune_mode(int32_t on);
/* Number of variants of a kernel, or GLU_ERR_INVALID_ARG. */
int32_t glu_tune_variants(int32_t kernel);
/* Description of a variant into buf (NUL-terminated, truncated to cap). */
int glu_tune_variant_name(int32_t kernel, int32_t variant, char* buf, int32_t cap);
/* Force a variant for every later launch of the kernel (-1: back to cached / tuned choices). */
int glu_tune_force(int32_t kernel, int32_t variant);
/* Write the cached choices to buf if cap is large enough; returns the bytes needed (with NUL). */
int64_t glu_tune_export(char* buf, int64_t cap);
/* Merge choices from text written by glu_tune_export(); GLU_ERR_INVALID_ARG on a bad line
 * (nothing merged then). */
int glu_tune_import(const char* text);
/* Forget every cached choice. */
int glu_tune_clear(void);

/* Name of a status code (static string). */
const char* glu_status_string(int status);

/* Read and clear the device-side status words the kernels set (bounds checks, bounded waits).
 * Synchronous: waits for `stream`. Returns GLU_OK or the first recorded GLU_ERR_*. */
int glu_device_status(void* stream);

/* Library version string. */
const char* glu_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GLU_H */
