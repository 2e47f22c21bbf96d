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

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* 3x3 filter with clamped (replicated) edges: op 0 = box (1/9 each), op 1 = Gaussian
 * [1 2 1]/4 x [1 2 1]/4. C = 1..4 channels. X and Y must not alias. */
int glu_fx_filter3(const float* X, int32_t h, int32_t w, int32_t C, int64_t pitch, float* Y,
                   int64_t ypitch, int32_t op, void* stream);

/* Per-pixel RGB (C = 3): saturation about the Rec. 601 luma, Y = l + sat * (c - l) clamped
 * to [0, 1] (sat = 1 disables), then per-channel c^gamma (gamma = 1 disables). X may equal Y. */
int glu_fx_point(const float* X, int32_t h, int32_t w, int64_t pitch, float* Y, int64_t ypitch,
                 float sat, float gamma, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GLU_LROPS_H */
