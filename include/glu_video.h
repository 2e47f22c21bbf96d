/*
 * glu_video.h — a per-frame Guided Linear Upsampling pipeline replayed as CUDA graphs
 * (exported by libglu.so).
 *
 * Per frame, the pipeline of Sec. 3 for an image operator f applied at low resolution:
 *   1. lr = BOX downsample of the HR frame by `scale`                        (glu_downsample)
 *   2. T  = f(lr): a 3x3 filter, then saturation and gamma                  (glu_fx_filter3 / _point)
 *   3. Theta = Algorithm 1 of the HR frame against lr                       (glu_optimize)
 *   4. out = Eq. 1 of Theta on T                                            (glu_apply)
 * Step 3 does not depend on T and step 2 does not depend on Theta (the method is target-free:
 * Theta is computed from the guide alone), so with `overlap` set, step 2 runs on a second stream
 * beside step 3 and the two join before step 4. Each step's results equal the separate calls'.
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

#ifdef __cplusplus
extern "C" {
#endif

#define GLU_VIDEO_MAX_SLOTS 256

typedef struct {
    int32_t H, W;          /* frame size */
    int32_t hr_dtype;      /* GLU_U8 or GLU_F16 frames, c = 3, row pitch W * 3 */
    int32_t out_dtype;     /* GLU_F16 or GLU_F32 output, c = 3, row pitch W * 3 */
    int32_t scale;         /* s */
    glu_params params;     /* S, eps, mode (FAST or GNU) for Algorithm 1 */
    int32_t wfmt;          /* weight storage of Theta */
    int32_t filter;        /* -1: none, 0: 3x3 box, 1: 3x3 Gaussian [1 2 1]/4 */
    float saturation;      /* 1 = unchanged */
    float gamma;           /* 1 = unchanged */
    int32_t overlap;       /* 1: the LR operator runs on a forked stream beside Algorithm 1 */
} glu_video_desc;

typedef struct glu_video glu_video;  /* opaque */

/* Device workspace bytes for a pipeline with this description (0 on invalid arguments). */
size_t glu_video_workspace_size(const glu_video_desc* desc);

/* Create a pipeline on the current device. ws: device workspace (see above). */
int glu_video_create(const glu_video_desc* desc, void* ws, size_t ws_bytes, glu_video** out);

/* Record slot `slot`'s graph: one frame from `hr` (device, H x W x 3 of hr_dtype) into `out`
 * (device, H x W x 3 of out_dtype). Re-binding a slot replaces its graph. Synchronous on the
 * host (records and instantiates; launches nothing). */
int glu_video_bind(glu_video* v, int32_t slot, const void* hr, void* out);

/* Replay slot `slot`'s graph on `stream` (cudaStream_t as void*). */
int glu_video_launch(glu_video* v, int32_t slot, void* stream);

/* The same launches for one frame without a graph. */
int glu_video_run(glu_video* v, const void* hr, void* out, void* stream);

/* Device views of the pipeline's working images (valid while the workspace lives): the BOX
 * downsampled frame lr and the processed target T (both h x w x 3 float32), and Theta. Any
 * argument may be null. */
int glu_video_views(const glu_video* v, glu_image* lr, glu_image* target, glu_theta* theta);

/* Destroy graphs, events, streams and the handle (not the workspace). Null is a no-op. */
int glu_video_destroy(glu_video* v);

#ifdef __cplusplus
}
#endif
#endif /* GLU_VIDEO_H */
