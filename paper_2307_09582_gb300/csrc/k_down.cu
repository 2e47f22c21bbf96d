// Downsampling (Sec. 3.3: regular grid; block mean as the filtered alternative) and the LR
// operators the workloads apply to the downsampled image (the black-box f the method
// upsamples; not part of the method itself).
#include "internal.h"
#include "common.cuh"

namespace glu {

GLU_DEFINE_STATUS(down)

__device__ __forceinline__ void st_any(void* p, int dtype, int64_t i, float unit) {
    if (dtype == GLU_U8)
        ((uint8_t*)p)[i] = (uint8_t)rintf(__saturatef(unit) * 255.0f);
    else if (dtype == GLU_F16)
        ((__half*)p)[i] = __float2half_rn(unit);
    else
        ((float*)p)[i] = unit;
}

// one thread per LR pixel; GRID copies the pixel floor(e/2) into the block (raw element copy
// when the dtypes match, so uint8 stays exact).
__global__ void k_down_grid(const glu_image hr, const glu_image lr, int s) {
    const int64_t n = (int64_t)lr.h * lr.w;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / lr.w), u = (int)(i % lr.w);
        const int ey = min(s, hr.h - v * s), ex = min(s, hr.w - u * s);
        const int y = v * s + ey / 2, x = u * s + ex / 2;
        const int64_t si = (int64_t)y * hr.pitch + (int64_t)x * hr.c;
        const int64_t di = (int64_t)v * lr.pitch + (int64_t)u * lr.c;
        for (int c = 0; c < hr.c; ++c) {
            if (hr.dtype == lr.dtype) {
                if (hr.dtype == GLU_U8)
                    ((uint8_t*)lr.data)[di + c] = ((const uint8_t*)hr.data)[si + c];
                else if (hr.dtype == GLU_F16)
                    ((__half*)lr.data)[di + c] = ((const __half*)hr.data)[si + c];
                else
                    ((float*)lr.data)[di + c] = ((const float*)hr.data)[si + c];
            } else {
                st_any(lr.data, lr.dtype, di + c, ld_unit(hr.data, hr.dtype, si + c));
            }
        }
    }
}

// BOX: block mean; uint8 sums are exact integers, divided once.
__global__ void k_down_box(const glu_image hr, const glu_image lr, int s) {
    const int64_t n = (int64_t)lr.h * lr.w;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / lr.w), u = (int)(i % lr.w);
        const int y1 = min(hr.h, v * s + s), x1 = min(hr.w, u * s + s);
        const float inv = 1.0f / (float)((y1 - v * s) * (x1 - u * s));
        for (int c = 0; c < hr.c; ++c) {
            float acc = 0.f;
            for (int y = v * s; y < y1; ++y)
                for (int x = u * s; x < x1; ++x) {
                    const int64_t si = (int64_t)y * hr.pitch + (int64_t)x * hr.c + c;
                    acc += hr.dtype == GLU_U8 ? (float)((const uint8_t*)hr.data)[si]
                                              : ld_unit(hr.data, hr.dtype, si);
                }
            float m = acc * inv;
            if (hr.dtype == GLU_U8) m *= (1.0f / 255.0f);
            st_any(lr.data, lr.dtype, (int64_t)v * lr.pitch + (int64_t)u * lr.c + c, m);
        }
    }
}

static int grid_for(int64_t work, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sms * 16;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

int launch_downsample(const glu_image& hr, int s, int mode, const glu_image& lr, cudaStream_t st) {
    const int threads = 256;
    const int grid = grid_for((int64_t)lr.h * lr.w, threads);
    if (mode == GLU_DOWN_GRID)
        k_down_grid<<<grid, threads, 0, st>>>(hr, lr, s);
    else
        k_down_box<<<grid, threads, 0, st>>>(hr, lr, s);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

// ------------------------------------------------------------------------------ LR operators
// op codes: 0 box3, 1 gauss3 (both with clamped edges, [0,1] units, C channels). Input float32,
// or uint8 read as x / 255 (correctly rounded, as a separate float division would give).
__device__ __forceinline__ float op_in(float x) { return x; }
__device__ __forceinline__ float op_in(uint8_t x) { return __fdiv_rn((float)x, 255.0f); }

// Channel c of the 3x3 filter at (v, u): the nine taps in raster order, one FMA each.
template <typename TX>
__device__ __forceinline__ float filter3_at(const TX* X, int h, int w, int C, int64_t pitch, int v,
                                            int u, int c, int op) {
    const float kg[3] = {0.25f, 0.5f, 0.25f};
    float acc = 0.f;
    for (int dv = -1; dv <= 1; ++dv)
        for (int du = -1; du <= 1; ++du) {
            const int vv = min(max(v + dv, 0), h - 1), uu = min(max(u + du, 0), w - 1);
            const float wgt = op == 0 ? (1.0f / 9.0f) : kg[dv + 1] * kg[du + 1];
            acc = __fmaf_rn(wgt, op_in(X[(int64_t)vv * pitch + (int64_t)uu * C + c]), acc);
        }
    return acc;
}

// Saturation about the Rec. 601 luma (clamped to [0, 1]), then per-channel gamma; either is
// skipped at 1.
__device__ __forceinline__ void point_op(float c3[3], float sat, float gamma) {
    if (sat != 1.0f) {
        const float l = __fmaf_rn(0.114f, c3[2], __fmaf_rn(0.587f, c3[1], __fmul_rn(0.299f, c3[0])));
        for (int c = 0; c < 3; ++c) c3[c] = __saturatef(__fmaf_rn(sat, __fsub_rn(c3[c], l), l));
    }
    if (gamma != 1.0f)
        for (int c = 0; c < 3; ++c) c3[c] = c3[c] > 0.f ? powf(c3[c], gamma) : 0.f;
}

template <typename TX>
__global__ void k_op_filter3(const TX* X, int h, int w, int C, int64_t pitch, float* Y,
                             int64_t ypitch, int op) {
    const int64_t n = (int64_t)h * w;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / w), u = (int)(i % w);
        for (int c = 0; c < C; ++c)
            Y[(int64_t)v * ypitch + (int64_t)u * C + c] = filter3_at(X, h, w, C, pitch, v, u, c, op);
    }
}

// pointwise: saturation then gamma (point_op). In place allowed.
__global__ void k_op_point(const float* X, int h, int w, int64_t pitch, float* Y, int64_t ypitch,
                           float sat, float gamma) {
    const int64_t n = (int64_t)h * w;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / w), u = (int)(i % w);
        const float* x = X + (int64_t)v * pitch + (int64_t)u * 3;
        float c3[3] = {x[0], x[1], x[2]};
        point_op(c3, sat, gamma);
        float* y = Y + (int64_t)v * ypitch + (int64_t)u * 3;
        for (int c = 0; c < 3; ++c) y[c] = c3[c];
    }
}

// The whole operator (filter -1: none, else k_op_filter3's op) per 3-channel LR pixel: the same
// values as k_op_filter3 followed by k_op_point (the intermediate is a float either way). A CTA
// owns a kLrTile x kLrTile tile: it stages the tile and a one-pixel ring (coordinates clamped to
// the image, so the ring repeats the edge as the filter's clamped taps do) in shared memory with
// coalesced row loads, converted to [0, 1] once there (x / 255 for uint8: the same value every
// tap would compute), then every thread filters its pixel from there, taps in the same order.
constexpr int kLrTile = 16;

template <typename TX>
__global__ void __launch_bounds__(kLrTile * kLrTile)
    k_op_lr(const TX* X, int h, int w, int64_t pitch, float* Y, int64_t ypitch, int filter,
            float sat, float gamma) {
    griddep_launch_dependents();   // a dependent apply may start loading codes and weights
    constexpr int RW = kLrTile + 2;
    __shared__ float tile[RW * RW * 3];
    const int v0 = blockIdx.y * kLrTile, u0 = blockIdx.x * kLrTile;
    for (int i = threadIdx.x; i < RW * RW * 3; i += blockDim.x) {
        const int rr = i / (RW * 3), rem = i - rr * (RW * 3), cc = rem / 3, c = rem - cc * 3;
        const int v = min(max(v0 - 1 + rr, 0), h - 1), u = min(max(u0 - 1 + cc, 0), w - 1);
        tile[i] = op_in(X[(int64_t)v * pitch + (int64_t)u * 3 + c]);
    }
    __syncthreads();
    const int tv = threadIdx.x / kLrTile, tu = threadIdx.x % kLrTile;
    const int v = v0 + tv, u = u0 + tu;
    if (v >= h || u >= w) return;
    float c3[3];
    for (int c = 0; c < 3; ++c)
        c3[c] = filter < 0 ? tile[((tv + 1) * RW + tu + 1) * 3 + c]
                           : filter3_at(tile + (tv * RW + tu) * 3 + c, 3, 3, 3, RW * 3, 1, 1, 0,
                                        filter);
    point_op(c3, sat, gamma);
    float* y = Y + (int64_t)v * ypitch + (int64_t)u * 3;
    for (int c = 0; c < 3; ++c) y[c] = c3[c];
}

int launch_lr_op(const void* X, int x_dtype, int h, int w, int64_t pitch, float* Y, int64_t ypitch,
                 int filter, float sat, float gamma, cudaStream_t st) {
    const dim3 grid((w + kLrTile - 1) / kLrTile, (h + kLrTile - 1) / kLrTile);
    if (grid.y > 65535u) return GLU_ERR_UNSUPPORTED;
    if (x_dtype == GLU_U8)
        k_op_lr<<<grid, kLrTile * kLrTile, 0, st>>>((const uint8_t*)X, h, w, pitch, Y, ypitch,
                                                    filter, sat, gamma);
    else
        k_op_lr<<<grid, kLrTile * kLrTile, 0, st>>>((const float*)X, h, w, pitch, Y, ypitch,
                                                    filter, sat, gamma);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

}  // namespace glu

extern "C" {

int glu_fx_filter3(const float* X, int32_t h, int32_t w, int32_t C, int64_t pitch, float* Y,
                   int64_t ypitch, int32_t op, void* stream) {
    if (!X || !Y || h <= 0 || w <= 0 || C < 1 || C > 4 || (op != 0 && op != 1) ||
        pitch < (int64_t)w * C || ypitch < (int64_t)w * C || X == Y)
        return GLU_ERR_INVALID_ARG;
    const int threads = 256;
    glu::k_op_filter3<<<glu::grid_for((int64_t)h * w, threads), threads, 0, (cudaStream_t)stream>>>(
        X, h, w, C, pitch, Y, ypitch, op);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

int glu_fx_filter3_u8(const uint8_t* X, int32_t h, int32_t w, int32_t C, int64_t pitch, float* Y,
                      int64_t ypitch, int32_t op, void* stream) {
    if (!X || !Y || h <= 0 || w <= 0 || C < 1 || C > 4 || (op != 0 && op != 1) ||
        pitch < (int64_t)w * C || ypitch < (int64_t)w * C)
        return GLU_ERR_INVALID_ARG;
    const int threads = 256;
    glu::k_op_filter3<<<glu::grid_for((int64_t)h * w, threads), threads, 0, (cudaStream_t)stream>>>(
        X, h, w, C, pitch, Y, ypitch, op);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

int glu_fx_point(const float* X, int32_t h, int32_t w, int64_t pitch, float* Y, int64_t ypitch,
                 float sat, float gamma, void* stream) {
    if (!X || !Y || h <= 0 || w <= 0 || pitch < (int64_t)w * 3 || ypitch < (int64_t)w * 3 ||
        !(sat >= 0.f) || !(gamma > 0.f))
        return GLU_ERR_INVALID_ARG;
    const int threads = 256;
    glu::k_op_point<<<glu::grid_for((int64_t)h * w, threads), threads, 0, (cudaStream_t)stream>>>(
        X, h, w, pitch, Y, ypitch, sat, gamma);
    GLU_LAUNCH_CHECK();
    return GLU_OK;
}

}  // extern "C"
