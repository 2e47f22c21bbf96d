// Per-frame pipeline (downsample -> LR operators -> Algorithm 1 once -> Eq. 1 per operator)
// replayed as CUDA graphs. Theta is computed from the guide alone (Sec. 3), so one optimisation
// serves every operator of the frame; each operator's branch forks onto a stream of its own
// beside Algorithm 1 and applies Theta to its target once Theta is ready; the branches join at
// the end of the frame.
#include <new>

#include "common.cuh"
#include "glu_lrops.h"
#include "glu_video.h"
#include "internal.h"

using namespace glu;

struct glu_video {
    glu_video_desc d;
    int h, w;
    float* lr;                       // h x w x 3: BOX downsample of the frame
    float* t1[GLU_VIDEO_MAX_OPS];    // h x w x 3: filtered, per operator
    float* T[GLU_VIDEO_MAX_OPS];     // h x w x 3: processed target, per operator
    uint16_t* code;                  // H x W
    void* weight;                    // H x W
    int device;
    cudaStream_t side[GLU_VIDEO_MAX_OPS];   // forked branches, one per operator
    cudaStream_t rec;                // recording stream for graph capture
    cudaEvent_t fork, theta_ready;
    cudaEvent_t join[GLU_VIDEO_MAX_OPS];
    cudaGraphExec_t exec[GLU_VIDEO_MAX_SLOTS];
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int wbytes(int wfmt) { return wfmt == GLU_W_F32 ? 4 : 2; }

bool desc_ok(const glu_video_desc* d) {
    if (!d || d->H <= 0 || d->W <= 0 || d->scale < 1) return false;
    if (d->hr_dtype != GLU_U8 && d->hr_dtype != GLU_F16) return false;
    if (d->out_dtype != GLU_F16 && d->out_dtype != GLU_F32) return false;
    const glu_params& p = d->params;
    if (p.S < 1 || p.S > 9 || !(p.S & 1) || !(p.eps >= 0.f)) return false;
    if (p.mode != GLU_MODE_FAST && p.mode != GLU_MODE_GNU) return false;
    if (d->wfmt < GLU_W_F32 || d->wfmt > GLU_W_UNORM16) return false;
    if (d->n_ops < 1 || d->n_ops > GLU_VIDEO_MAX_OPS) return false;
    for (int k = 0; k < d->n_ops; ++k) {
        const glu_lr_op& o = d->ops[k];
        if (o.filter < -1 || o.filter > 1) return false;
        if (!(o.saturation >= 0.f) || !(o.gamma > 0.f)) return false;
    }
    return true;
}

size_t layout(const glu_video_desc* d, char* base, glu_video* v) {
    const int h = (d->H + d->scale - 1) / d->scale, w = (d->W + d->scale - 1) / d->scale;
    const size_t lrb = sizeof(float) * 3 * (size_t)h * w;
    const size_t np = (size_t)d->H * d->W;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off = a256(off + bytes);
        return p;
    };
    char* lr = take(lrb);
    char* t1[GLU_VIDEO_MAX_OPS];
    char* T[GLU_VIDEO_MAX_OPS];
    for (int k = 0; k < d->n_ops; ++k) {
        t1[k] = take(lrb);
        T[k] = take(lrb);
    }
    char* code = take(sizeof(uint16_t) * np);
    char* weight = take((size_t)wbytes(d->wfmt) * np);
    if (v) {
        v->h = h;
        v->w = w;
        v->lr = (float*)lr;
        for (int k = 0; k < d->n_ops; ++k) {
            v->t1[k] = (float*)t1[k];
            v->T[k] = (float*)T[k];
        }
        v->code = (uint16_t*)code;
        v->weight = weight;
    }
    return off;
}

// Operator k on the LR image (on stream st).
int issue_op(glu_video* v, int k, cudaStream_t st) {
    const glu_lr_op& o = v->d.ops[k];
    const int64_t pitch = (int64_t)v->w * 3;
    const float* src = v->lr;
    if (o.filter >= 0) {
        const int rc = glu_fx_filter3(v->lr, v->h, v->w, 3, pitch, v->t1[k], pitch, o.filter, st);
        if (rc) return rc;
        src = v->t1[k];
    }
    return glu_fx_point(src, v->h, v->w, pitch, v->T[k], pitch, o.saturation, o.gamma, st);
}

// Eq. 1 of the frame's Theta on target k into out (on stream st).
int issue_apply(glu_video* v, int k, void* out, cudaStream_t st) {
    const glu_video_desc& d = v->d;
    ApplyArgs p;
    p.code = v->code;
    p.weight = v->weight;
    p.wfmt = d.wfmt;
    p.H = d.H;
    p.W = d.W;
    p.s = d.scale;
    p.S = d.params.S;
    p.h = v->h;
    p.w = v->w;
    p.C = 3;
    p.T = v->T[k];
    p.T_pitch = (int64_t)v->w * 3;
    p.T_dtype = GLU_F32;
    p.out = out;
    p.out_pitch = (int64_t)d.W * 3;
    p.out_dtype = d.out_dtype;
    return launch_apply(p, st);
}

// One frame's launches on `st` (the fork / join events make the side streams part of the same
// work).
int issue(glu_video* v, const void* hr, void* const* outs, cudaStream_t st) {
    const glu_video_desc& d = v->d;
    glu_image hi{const_cast<void*>(hr), d.H, d.W, 3, d.hr_dtype, (int64_t)d.W * 3};
    glu_image li{v->lr, v->h, v->w, 3, GLU_F32, (int64_t)v->w * 3};
    int rc = launch_downsample(hi, d.scale, GLU_DOWN_BOX, li, st);
    if (rc) return rc;
    if (d.overlap) {
        GLU_CUDA_TRY(cudaEventRecord(v->fork, st));
        for (int k = 0; k < d.n_ops; ++k) {
            GLU_CUDA_TRY(cudaStreamWaitEvent(v->side[k], v->fork, 0));
            rc = issue_op(v, k, v->side[k]);
            if (rc) return rc;
        }
    } else {
        for (int k = 0; k < d.n_ops; ++k) {
            rc = issue_op(v, k, st);
            if (rc) return rc;
        }
    }
    SearchArgs a;
    a.hr = hr;
    a.hr_pitch = (int64_t)d.W * 3;
    a.hr_dtype = d.hr_dtype;
    a.lr = v->lr;
    a.lr_pitch = (int64_t)v->w * 3;
    a.lr_dtype = GLU_F32;
    a.H = d.H;
    a.W = d.W;
    a.h = v->h;
    a.w = v->w;
    a.s = d.scale;
    a.S = d.params.S;
    a.eps255 = fmaxf(d.params.eps * 255.0f, 1e-12f);
    a.gnu = d.params.mode == GLU_MODE_GNU;
    a.code = v->code;
    a.weight = v->weight;
    a.wfmt = d.wfmt;
    a.err = nullptr;
    rc = launch_search(a, st);
    if (rc) return rc;
    if (!d.overlap) {
        for (int k = 0; k < d.n_ops; ++k) {
            rc = issue_apply(v, k, outs[k], st);
            if (rc) return rc;
        }
        return GLU_OK;
    }
    GLU_CUDA_TRY(cudaEventRecord(v->theta_ready, st));
    for (int k = 0; k < d.n_ops; ++k) {
        GLU_CUDA_TRY(cudaStreamWaitEvent(v->side[k], v->theta_ready, 0));
        rc = issue_apply(v, k, outs[k], v->side[k]);
        if (rc) return rc;
        GLU_CUDA_TRY(cudaEventRecord(v->join[k], v->side[k]));
    }
    for (int k = 0; k < d.n_ops; ++k) GLU_CUDA_TRY(cudaStreamWaitEvent(st, v->join[k], 0));
    return GLU_OK;
}

void release(glu_video* v) {
    for (auto& e : v->exec)
        if (e) cudaGraphExecDestroy(e);
    if (v->fork) cudaEventDestroy(v->fork);
    if (v->theta_ready) cudaEventDestroy(v->theta_ready);
    for (int k = 0; k < GLU_VIDEO_MAX_OPS; ++k) {
        if (v->join[k]) cudaEventDestroy(v->join[k]);
        if (v->side[k]) cudaStreamDestroy(v->side[k]);
    }
    if (v->rec) cudaStreamDestroy(v->rec);
    delete v;
}

bool outs_ok(const glu_video* v, void* const* outs) {
    if (!outs) return false;
    for (int k = 0; k < v->d.n_ops; ++k)
        if (!outs[k]) return false;
    return true;
}

}  // namespace

extern "C" {

size_t glu_video_workspace_size(const glu_video_desc* desc) {
    if (!desc_ok(desc)) return 0;
    return layout(desc, nullptr, nullptr);
}

int glu_video_create(const glu_video_desc* desc, void* ws, size_t ws_bytes, glu_video** out) {
    if (!out || !desc_ok(desc)) return GLU_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ws || ((uintptr_t)ws & 255u) != 0 || ws_bytes < layout(desc, nullptr, nullptr))
        return GLU_ERR_WORKSPACE;
    glu_video* v = new (std::nothrow) glu_video();
    if (!v) return GLU_ERR_CUDA;
    v->d = *desc;
    layout(desc, (char*)ws, v);
    bool ok = cudaGetDevice(&v->device) == cudaSuccess &&
              cudaStreamCreateWithFlags(&v->rec, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&v->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&v->theta_ready, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < desc->n_ops; ++k)
        ok = cudaStreamCreateWithFlags(&v->side[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&v->join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        release(v);
        return GLU_ERR_CUDA;
    }
    *out = v;
    return GLU_OK;
}

int glu_video_bind(glu_video* v, int32_t slot, const void* hr, void* const* outs) {
    if (!v || !hr || !outs_ok(v, outs) || slot < 0 || slot >= GLU_VIDEO_MAX_SLOTS)
        return GLU_ERR_INVALID_ARG;
    cudaGraph_t g = nullptr;
    GLU_CUDA_TRY(cudaStreamBeginCapture(v->rec, cudaStreamCaptureModeRelaxed));
    const int rc = issue(v, hr, outs, v->rec);
    const cudaError_t ec = cudaStreamEndCapture(v->rec, &g);
    if (rc != GLU_OK || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return rc != GLU_OK ? rc : GLU_ERR_CUDA;
    }
    cudaGraphExec_t e = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&e, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return GLU_ERR_CUDA;
    if (v->exec[slot]) cudaGraphExecDestroy(v->exec[slot]);
    v->exec[slot] = e;
    return GLU_OK;
}

int glu_video_launch(glu_video* v, int32_t slot, void* stream) {
    if (!v || slot < 0 || slot >= GLU_VIDEO_MAX_SLOTS || !v->exec[slot]) return GLU_ERR_INVALID_ARG;
    GLU_CUDA_TRY(cudaGraphLaunch(v->exec[slot], (cudaStream_t)stream));
    return GLU_OK;
}

int glu_video_run(glu_video* v, const void* hr, void* const* outs, void* stream) {
    if (!v || !hr || !outs_ok(v, outs)) return GLU_ERR_INVALID_ARG;
    return issue(v, hr, outs, (cudaStream_t)stream);
}

int glu_video_views(const glu_video* v, glu_image* lr, glu_image* targets, glu_theta* theta) {
    if (!v) return GLU_ERR_INVALID_ARG;
    if (lr) *lr = glu_image{v->lr, v->h, v->w, 3, GLU_F32, (int64_t)v->w * 3};
    if (targets)
        for (int k = 0; k < v->d.n_ops; ++k)
            targets[k] = glu_image{v->T[k], v->h, v->w, 3, GLU_F32, (int64_t)v->w * 3};
    if (theta)
        *theta = glu_theta{v->code, v->weight, v->d.H, v->d.W, v->d.scale, v->d.params.S,
                           v->d.wfmt};
    return GLU_OK;
}

int glu_video_destroy(glu_video* v) {
    if (v) release(v);
    return GLU_OK;
}

}  // extern "C"
