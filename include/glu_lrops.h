/*
 * glu_lrops.h — LR operators of the benchmark workloads (exported by libglu.so).
 *
 * These are NOT part of Guided Linear Upsampling. The method treats the image operator f as a
 * black box applied to the downsampled image (Sec. 3, problem statement); these kernels are
 * stand-ins for f so the workloads can run the whole pipeline (downsample -> f -> upsample) on
 * the device: a 3x3 box blur, a 3x3 [1 2 1]/4 Gaussian, a saturation change and a gamma curve.
 *
 * All buffers are device memory owned by the caller; images are float32, h x w x C interleaved,
 * colours in [0, 1], rows `pitch` elements apart. Calls are asynchronous on `stream`
 * (cudaStream_t as void*). Return GLU_OK or a negative GLU_ERR_* code from glu.h (argument
 * errors are reported synchronously, before any launch).
 */
#ifndef GLU_LROPS_H
#define GLU_LROPS_H

#include <stddef.h>
#include <stdint.h>

#include "glu.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One LR operator: the 3x3 filter, then saturation, then gamma (each optional). */
typedef struct {
    int32_t filter;        /* -1: none, 0: 3x3 box, 1: 3x3 Gaussian [1 2 1]/4 */
    float saturation;      /* 1 = unchanged */
    float gamma;           /* 1 = unchanged */
} glu_lr_op;

/* 3x3 filter with clamped (replicated) edges: op 0 = box (1/9 each), op 1 = Gaussian
 * [1 2 1]/4 x [1 2 1]/4. C = 1..4 channels. X and Y must not alias. */
int glu_fx_filter3(const float* X, int32_t h, int32_t w, int32_t C, int64_t pitch, float* Y,
                   int64_t ypitch, int32_t op, void* stream);

/* The same filter on a uint8 image (colour * 255, e.g. an optimised LR image of
 * glu_joint_optimize), each value read as x / 255 (correctly rounded). */
int glu_fx_filter3_u8(const uint8_t* X, int32_t h, int32_t w, int32_t C, int64_t pitch, float* Y,
                      int64_t ypitch, int32_t op, void* stream);

/* Per-pixel RGB (C = 3): saturation about the Rec. 601 luma, Y = l + sat * (c - l) clamped
 * to [0, 1] (sat = 1 disables), then per-channel c^gamma (gamma = 1 disables). X may equal Y. */
int glu_fx_point(const float* X, int32_t h, int32_t w, int64_t pitch, float* Y, int64_t ypitch,
                 float sat, float gamma, void* stream);

/* The operator, then Eq. 1, as one issue: lr_target = f(lr) (lr: U8, read as x / 255, or F32;
 * 3 channels, ceil(H/s) x ceil(W/s); lr_target: F32, 3 channels, the same size, caller-owned;
 * it holds f(lr) afterwards), then hr_out = glu_apply(theta, lr_target). One kernel computes the
 * whole operator per LR pixel (the values glu_fx_filter3(_u8) followed by glu_fx_point give); the
 * apply is launched as its programmatic dependent, so on the persistent TMA path the codes and
 * weights of its first tiles load while the operator runs, and it reads lr_target only once the
 * operator has finished. hr_out is bit-identical to the three separate calls. lr, lr_target and
 * hr_out must not overlap. */
int glu_apply_lrop(const glu_theta* theta, const glu_image* lr, const glu_lr_op* op,
                   glu_image* lr_target, glu_image* hr_out, void* stream);

/* ------------------------------------------------ the benchmark pipeline on host buffers
 *
 * One call runs the whole optimise-then-upsample flow of the method (Sec. 3: Theta from the
 * guide, the operator on the LR image, Eq. 1 back to full resolution) with the guide and the
 * result in HOST memory: the guide hr_host (H x W x 3 uint8, rows W * 3 bytes apart) is copied
 * to the device; Algorithm 2 (params: FAST mode, window S, N iterations) optimises the LR image
 * and Theta (unorm16 weights) at scale `scale`; the LR operator (3x3 filter op, then sat and
 * gamma) turns the optimised LR image into T and Eq. 1 upsamples T (glu_apply_lrop);
 * the H x W x 3 float32 result is copied to out_host (rows W * 3 floats apart). Host buffers in
 * pinned (page-locked) memory give the copies full bandwidth; pageable memory works, slower.
 *
 * ws: device workspace of glu_pipeline_host_workspace_size() bytes, 256-byte aligned, owned by
 * the caller; it holds the device copies of the guide, the LR images, Theta, the result and
 * Algorithm 2's workspace. Repeated calls with the same buffers replay Algorithm 2 as a CUDA
 * graph. The call returns after out_host holds the result (it synchronises `stream`); argument
 * errors return before any copy. 0 if the sizes are invalid. */
size_t glu_pipeline_host_workspace_size(int32_t H, int32_t W, int32_t scale,
                                        const glu_params* params);
int glu_pipeline_host(const uint8_t* hr_host, int32_t H, int32_t W, int32_t scale,
                      const glu_params* params, int32_t op, float sat, float gamma,
                      float* out_host, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GLU_LROPS_H */
