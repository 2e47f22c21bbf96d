// The benchmark pipeline with host buffers (glu_pipeline_host): the guide in, Algorithm 2 (the LR
// image and Theta), the LR operator, Eq. 1, the result out — one stream, one call. Every step is
// a library call on device buffers carved from the caller's workspace; the only host work is the
// argument checks and the two copies.
#include "common.cuh"
#include "glu_lrops.h"
#include "internal.h"

namespace {

struct PipeBufs {
    uint8_t* hr;        // H x W x 3, the device copy of the guide
    uint8_t* lr;        // h x w x 3, the optimised LR image
    uint16_t* code;     // H x W pair codes
    uint16_t* weight;   // H x W unorm16 weights
    float* t2;          // h x w x 3, T
    float* out;         // H x W x 3, Eq. 1
    void* jws;          // Algorithm 2's workspace
    size_t jws_bytes;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes needed (0: invalid sizes); with base != null, also the buffers.
size_t carve_pipe(int H, int W, int s, const glu_params* p, void* base, PipeBufs* o) {
    const size_t jws = glu_joint_workspace_size(H, W, s, p);
    if (!jws) return 0;
    const size_t h = (size_t)((H + s - 1) / s), w = (size_t)((W + s - 1) / s);
    const size_t np = (size_t)H * (size_t)W;
    char* b = (char*)base;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        void* q = b ? (void*)(b + off) : nullptr;
        off = align256(off + bytes);
        return q;
    };
    PipeBufs t;
    t.jws = take(jws);   // first: 256-byte aligned like the workspace itself
    t.jws_bytes = jws;
    t.hr = (uint8_t*)take(np * 3);
    t.lr = (uint8_t*)take(h * w * 3);
    t.code = (uint16_t*)take(np * sizeof(uint16_t));
    t.weight = (uint16_t*)take(np * sizeof(uint16_t));
    t.t2 = (float*)take(h * w * 3 * sizeof(float));
    t.out = (float*)take(np * 3 * sizeof(float));
    if (o) *o = t;
    return off;
}

}  // namespace

extern "C" {

size_t glu_pipeline_host_workspace_size(int32_t H, int32_t W, int32_t scale,
                                        const glu_params* params) {
    if (H <= 0 || W <= 0 || scale < 1 || !params) return 0;
    return carve_pipe(H, W, scale, params, nullptr, nullptr);
}

int glu_pipeline_host(const uint8_t* hr_host, int32_t H, int32_t W, int32_t scale,
                      const glu_params* params, int32_t op, float sat, float gamma,
                      float* out_host, void* ws, size_t ws_bytes, void* stream) {
    if (!hr_host || !out_host || !params || H <= 0 || H >= (1 << 22) || W <= 0 || scale < 1 ||
        (op != 0 && op != 1) || !(sat >= 0.f) || !(gamma > 0.f))
        return GLU_ERR_INVALID_ARG;
    if (params->mode != GLU_MODE_FAST) return GLU_ERR_UNSUPPORTED;
    const size_t need = glu_pipeline_host_workspace_size(H, W, scale, params);
    if (!need) return GLU_ERR_INVALID_ARG;
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255u) != 0) return GLU_ERR_WORKSPACE;
    PipeBufs b;
    carve_pipe(H, W, scale, params, ws, &b);
    const int h = (H + scale - 1) / scale, w = (W + scale - 1) / scale;
    cudaStream_t st = (cudaStream_t)stream;
    GLU_CUDA_TRY(cudaMemcpyAsync(b.hr, hr_host, (size_t)H * W * 3, cudaMemcpyHostToDevice, st));
    glu_image hr{b.hr, H, W, 3, GLU_U8, (int64_t)W * 3};
    glu_image lr{b.lr, h, w, 3, GLU_U8, (int64_t)w * 3};
    glu_theta th{b.code, b.weight, H, W, scale, params->S, GLU_W_UNORM16};
    int rc = glu_joint_optimize(&hr, scale, params, &lr, &th, nullptr, nullptr, b.jws,
                                b.jws_bytes, stream);
    if (rc) return rc;
    // the operator and Eq. 1 as one issue (the apply starts while the operator runs)
    const glu_lr_op f{op, sat, gamma};
    glu_image t{b.t2, h, w, 3, GLU_F32, (int64_t)w * 3};
    glu_image out{b.out, H, W, 3, GLU_F32, (int64_t)W * 3};
    rc = glu_apply_lrop(&th, &lr, &f, &t, &out, stream);
    if (rc) return rc;
    GLU_CUDA_TRY(cudaMemcpyAsync(out_host, b.out, (size_t)H * W * 3 * sizeof(float),
                                 cudaMemcpyDeviceToHost, st));
    GLU_CUDA_TRY(cudaStreamSynchronize(st));
    return GLU_OK;
}

}  // extern "C"
