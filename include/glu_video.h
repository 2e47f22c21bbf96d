/*
 * glu_video.h — a per-frame Guided Linear Upsampling pipeline replayed as CUDA graphs
 * (exported by libglu.so).
 *
 * Per frame, the pipeline of Sec. 3 for image operators f_k applied at low resolution:
 *   1. lr = BOX downsample of the HR frame by `scale`                        (glu_downsample)
 *   2. T_k = f_k(lr) for every operator k: a 3x3 filter, then saturation and gamma
 *                                                                           (glu_fx_filter3 / _point)
 *   3. Theta = Algorithm 1 of the HR frame against lr, once                 (glu_optimize)
 *   4. out_k = Eq. 1 of Theta on T_k for every operator k                   (glu_apply)
 * Theta depends on the guide alone (the method is target-free, Sec. 3), so one optimisation
 * serves every operator of the frame, and steps 2 and 3 are independent: with `overlap` set,
 * operator k runs on a stream of its own forked beside step 3, and once Theta is ready applies it
 * to T_k there; the branches join at the end of the frame. Each step's results equal the
 * separate calls'.
 *
 * A pipeline holds up to GLU_VIDEO_MAX_SLOTS slots. glu_video_bind() records one frame's launches
 * for a given (HR frame, output) buffer pair into a CUDA graph once; glu_video_launch() replays
 * it with one call. A ring of input buffers (a decoder or an upload writing into a fixed set of
 * frames) binds one slot per buffer. glu_video_run() issues the same launches directly, without a
 * graph.
 *
 * Ownership: the caller owns every buffer, including the device workspace (at least
 * glu_video_workspace_size() bytes, 256-byte aligned) that holds lr, T and Theta; the library
 * owns the handle, two events, one stream for the forked branch and one for recording.
 * All frames of one pipeline share that workspace: launch them in order on one stream.
 * Not thread-safe per handle. Errors: GLU_ERR_* codes of glu.h; argument errors are reported
 * before any launch.
 */
#ifndef GLU_VIDEO_H
#define GLU_VIDEO_H

#include <stddef.h>
#include <stdint.h>

#include "glu.h"
#include "glu_lrops.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GLU_VIDEO_MAX_SLOTS 256
#define GLU_VIDEO_MAX_OPS 4

typedef struct {
    int32_t H, W;          /* frame size */
    int32_t hr_dtype;      /* GLU_U8 or GLU_F16 frames, c = 3, row pitch W * 3 */
    int32_t out_dtype;     /* GLU_F16 or GLU_F32 outputs, c = 3, row pitch W * 3 */
    int32_t scale;         /* s */
    glu_params params;     /* S, eps, mode (FAST or GNU) for Algorithm 1 */
    int32_t wfmt;          /* weight storage of Theta */
    int32_t n_ops;         /* 1 .. GLU_VIDEO_MAX_OPS operators sharing the frame's Theta */
    glu_lr_op ops[GLU_VIDEO_MAX_OPS];   /* operator k (glu_lrops.h): target T_k, output k */
    int32_t overlap;       /* 1: each operator runs on a forked stream beside Algorithm 1 */
} glu_video_desc;

typedef struct glu_video glu_video;  /* opaque */

/* Device workspace bytes for a pipeline with this description (0 on invalid arguments). */
size_t glu_video_workspace_size(const glu_video_desc* desc);

/* Create a pipeline on the current device. ws: device workspace (see above). */
int glu_video_create(const glu_video_desc* desc, void* ws, size_t ws_bytes, glu_video** out);

/* Record slot `slot`'s graph: one frame from `hr` (device, H x W x 3 of hr_dtype) into
 * outs[0 .. n_ops) (HOST array of device pointers, each H x W x 3 of out_dtype; outs[k] receives
 * operator k's upsampled result). Re-binding a slot replaces its graph. Synchronous on the host
 * (records and instantiates; launches nothing). */
int glu_video_bind(glu_video* v, int32_t slot, const void* hr, void* const* outs);

/* Replay slot `slot`'s graph on `stream` (cudaStream_t as void*). */
int glu_video_launch(glu_video* v, int32_t slot, void* stream);

/* The same launches for one frame without a graph (outs as for glu_video_bind). */
int glu_video_run(glu_video* v, const void* hr, void* const* outs, void* stream);

/* Device views of the pipeline's working images (valid while the workspace lives): the BOX
 * downsampled frame lr and the processed targets T_k (targets: HOST array of n_ops records; all
 * h x w x 3 float32), and Theta. Any argument may be null. */
int glu_video_views(const glu_video* v, glu_image* lr, glu_image* targets, glu_theta* theta);

/* Destroy graphs, events, streams and the handle (not the workspace). Null is a no-op. */
int glu_video_destroy(glu_video* v);

#ifdef __cplusplus
}
#endif
#endif /* GLU_VIDEO_H */
