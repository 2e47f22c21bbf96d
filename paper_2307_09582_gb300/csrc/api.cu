// C-ABI entry points of libglu.so: argument validation, then launches on the caller's stream.
#include <string.h>

#include "internal.h"
#include "glu_lrops.h"

using namespace glu;

namespace {

int dtype_size(int dt) {
    switch (dt) {
        case GLU_U8: return 1;
        case GLU_F16: return 2;
        case GLU_F32: return 4;
        default: return 0;
    }
}

bool image_ok(const glu_image* im) {
    return im && im->data && im->h > 0 && im->w > 0 && im->c >= 1 && im->c <= 4 &&
           dtype_size(im->dtype) > 0 && im->pitch >= (int64_t)im->w * im->c;
}

bool params_ok(const glu_params* p) {
    return p && p->S >= 1 && p->S <= 9 && (p->S & 1) && p->eps >= 0.f && p->tau >= 0.f &&
           p->N >= 0 && p->N <= GLU_MAX_ITERS &&
           (p->mode == GLU_MODE_FAST || p->mode == GLU_MODE_GNU || p->mode == GLU_MODE_EXACT) &&
           (p->joint == GLU_JOINT_STRICT || p->joint == GLU_JOINT_PAPER) &&
           (p->connectivity == 4 || p->connectivity == 8);
}

// (fewer than 2^22 rows: the kernels divide row indices by the scale in float)
bool theta_ok(const glu_theta* t) {
    return t && t->code && t->weight && t->H > 0 && t->H < (1 << 22) && t->W > 0 &&
           t->scale >= 1 && t->S >= 1 &&
           t->S <= 9 && (t->S & 1) && t->wfmt >= GLU_W_F32 && t->wfmt <= GLU_W_UNORM16;
}

int lr_dim(int n, int s) { return (n + s - 1) / s; }

}  // namespace

namespace glu {

int joint_optimize(const glu_image* hr, int32_t scale, const glu_params* params,
                   glu_image* lr_out, glu_theta* theta, float* err_map, glu_joint_stats* stats,
                   void* ws, size_t ws_bytes, void* stream, int direct) {
    if (!image_ok(hr) || !image_ok(lr_out) || !params_ok(params) || !theta_ok(theta) || scale < 1)
        return GLU_ERR_INVALID_ARG;
    if (hr->dtype != GLU_U8 || lr_out->dtype != GLU_U8 || hr->c != 3 || lr_out->c != 3)
        return GLU_ERR_UNSUPPORTED;
    if (params->mode != GLU_MODE_FAST) return GLU_ERR_UNSUPPORTED;
    if (theta->H != hr->h || theta->W != hr->w || theta->S != params->S || theta->scale != scale ||
        lr_out->h != lr_dim(hr->h, scale) || lr_out->w != lr_dim(hr->w, scale))
        return GLU_ERR_SHAPE;
    const size_t need = joint_workspace_bytes(hr->h, hr->w, scale, params->S, params->N);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255u) != 0) return GLU_ERR_WORKSPACE;
    JointArgs a;
    a.hr = (const uint8_t*)hr->data;
    a.hr_pitch = hr->pitch;
    a.lr = (uint8_t*)lr_out->data;
    a.lr_pitch = lr_out->pitch;
    a.H = hr->h;
    a.W = hr->w;
    a.h = lr_out->h;
    a.w = lr_out->w;
    a.s = scale;
    a.S = params->S;
    a.eps255 = fmaxf(params->eps * 255.0f, 1e-12f);  // > 0: see search.cuh
    a.tau = params->tau;
    a.N = params->N;
    a.strict = params->joint == GLU_JOINT_STRICT;
    a.conn = params->connectivity;
    a.code = theta->code;
    a.weight = theta->weight;
    a.wfmt = theta->wfmt;
    a.err = err_map;
    return launch_joint(a, ws, ws_bytes, stats, (cudaStream_t)stream, direct);
}

}  // namespace glu

extern "C" {

void glu_params_default(glu_params* p) {
    if (!p) return;
    p->S = 3;
    p->eps = 1e-3f;
    p->tau = 30.0f / 255.0f;
    p->N = 3;
    p->mode = GLU_MODE_FAST;
    p->joint = GLU_JOINT_STRICT;
    p->connectivity = 8;
}

const char* glu_status_string(int s) {
    switch (s) {
        case GLU_OK: return "GLU_OK";
        case GLU_ERR_INVALID_ARG: return "GLU_ERR_INVALID_ARG";
        case GLU_ERR_SHAPE: return "GLU_ERR_SHAPE";
        case GLU_ERR_UNSUPPORTED: return "GLU_ERR_UNSUPPORTED";
        case GLU_ERR_WORKSPACE: return "GLU_ERR_WORKSPACE";
        case GLU_ERR_CUDA: return "GLU_ERR_CUDA";
        case GLU_ERR_DEVICE_CHECK: return "GLU_ERR_DEVICE_CHECK";
        case GLU_ERR_TIMEOUT: return "GLU_ERR_TIMEOUT";
        default: return "GLU_ERR_UNKNOWN";
    }
}

const char* glu_version(void) { return "glu-gb300 0.1 (sm_103a)"; }

int glu_device_status(void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int codes[6] = {read_and_clear_status_search(st), read_and_clear_status_apply(st),
                    read_and_clear_status_down(st), read_and_clear_status_joint(st),
                    read_and_clear_status_search_exact(st), read_and_clear_status_ls(st)};
    for (int c : codes)
        if (c != GLU_OK) return c;
    return GLU_OK;
}

int glu_downsample(const glu_image* hr, int32_t scale, int32_t mode, glu_image* lr, void* stream) {
    if (!image_ok(hr) || !image_ok(lr) || scale < 1) return GLU_ERR_INVALID_ARG;
    if (mode != GLU_DOWN_GRID && mode != GLU_DOWN_BOX) return GLU_ERR_INVALID_ARG;
    if (hr->c != lr->c || lr->h != lr_dim(hr->h, scale) || lr->w != lr_dim(hr->w, scale))
        return GLU_ERR_SHAPE;
    if (mode == GLU_DOWN_GRID && lr->dtype != hr->dtype && lr->dtype != GLU_F32)
        return GLU_ERR_UNSUPPORTED;
    if (mode == GLU_DOWN_BOX && lr->dtype == GLU_U8) return GLU_ERR_UNSUPPORTED;
    return launch_downsample(*hr, scale, mode, *lr, (cudaStream_t)stream);
}

int glu_optimize(const glu_image* hr, const glu_image* lr, const glu_params* params,
                 glu_theta* theta, float* err_map, void* stream) {
    if (!image_ok(hr) || !image_ok(lr) || !params_ok(params) || !theta_ok(theta))
        return GLU_ERR_INVALID_ARG;
    if (hr->c != 3 || lr->c != 3) return GLU_ERR_UNSUPPORTED;
    if (hr->dtype != GLU_U8 && hr->dtype != GLU_F16) return GLU_ERR_UNSUPPORTED;
    const int s = theta->scale;
    if (theta->H != hr->h || theta->W != hr->w || theta->S != params->S ||
        lr->h != lr_dim(hr->h, s) || lr->w != lr_dim(hr->w, s))
        return GLU_ERR_SHAPE;
    // Eq. 4 weights are not clamped to [0, 1]: only the float32 format holds them
    if (params->mode == GLU_MODE_EXACT && theta->wfmt != GLU_W_F32) return GLU_ERR_UNSUPPORTED;
    SearchArgs a;
    a.hr = hr->data;
    a.hr_pitch = hr->pitch;
    a.hr_dtype = hr->dtype;
    a.lr = lr->data;
    a.lr_pitch = lr->pitch;
    a.lr_dtype = lr->dtype;
    a.H = hr->h;
    a.W = hr->w;
    a.h = lr->h;
    a.w = lr->w;
    a.s = s;
    a.S = params->S;
    a.eps255 = fmaxf(params->eps * 255.0f, 1e-12f);  // > 0: see search.cuh
    a.gnu = params->mode == GLU_MODE_GNU;
    a.code = theta->code;
    a.weight = theta->weight;
    a.wfmt = theta->wfmt;
    a.err = err_map;
    if (params->mode == GLU_MODE_EXACT) return launch_search_exact(a, (cudaStream_t)stream);
    return launch_search(a, (cudaStream_t)stream);
}

int glu_apply(const glu_theta* theta, const glu_image* lr_target, glu_image* hr_out, void* stream) {
    if (!theta_ok(theta) || !image_ok(lr_target) || !image_ok(hr_out)) return GLU_ERR_INVALID_ARG;
    if (lr_target->dtype == GLU_U8 || hr_out->dtype == GLU_U8) return GLU_ERR_UNSUPPORTED;
    const int s = theta->scale;
    if (hr_out->h != theta->H || hr_out->w != theta->W || lr_target->c != hr_out->c ||
        lr_target->h != lr_dim(theta->H, s) || lr_target->w != lr_dim(theta->W, s))
        return GLU_ERR_SHAPE;
    ApplyArgs a;
    a.code = theta->code;
    a.weight = theta->weight;
    a.wfmt = theta->wfmt;
    a.H = theta->H;
    a.W = theta->W;
    a.s = s;
    a.S = theta->S;
    a.h = lr_target->h;
    a.w = lr_target->w;
    a.C = lr_target->c;
    a.T = lr_target->data;
    a.T_pitch = lr_target->pitch;
    a.T_dtype = lr_target->dtype;
    a.out = hr_out->data;
    a.out_pitch = hr_out->pitch;
    a.out_dtype = hr_out->dtype;
    return launch_apply(a, (cudaStream_t)stream);
}

int glu_apply_lrop(const glu_theta* theta, const glu_image* lr, const glu_lr_op* op,
                   glu_image* lr_target, glu_image* hr_out, void* stream) {
    if (!theta_ok(theta) || !image_ok(lr) || !image_ok(lr_target) || !image_ok(hr_out) || !op)
        return GLU_ERR_INVALID_ARG;
    if ((lr->dtype != GLU_U8 && lr->dtype != GLU_F32) || lr_target->dtype != GLU_F32 ||
        hr_out->dtype == GLU_U8 || lr->c != 3 || lr_target->c != 3 || hr_out->c != 3)
        return GLU_ERR_UNSUPPORTED;
    if (op->filter < -1 || op->filter > 1 || !(op->saturation >= 0.f) || !(op->gamma > 0.f))
        return GLU_ERR_INVALID_ARG;
    const int s = theta->scale, h = lr_dim(theta->H, s), w = lr_dim(theta->W, s);
    if (hr_out->h != theta->H || hr_out->w != theta->W || lr->h != h || lr->w != w ||
        lr_target->h != h || lr_target->w != w)
        return GLU_ERR_SHAPE;
    if (lr->data == lr_target->data) return GLU_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_lr_op(lr->data, lr->dtype, h, w, lr->pitch, (float*)lr_target->data,
                          lr_target->pitch, op->filter, op->saturation, op->gamma, st);
    if (rc) return rc;
    ApplyArgs a;
    a.code = theta->code;
    a.weight = theta->weight;
    a.wfmt = theta->wfmt;
    a.H = theta->H;
    a.W = theta->W;
    a.s = s;
    a.S = theta->S;
    a.h = h;
    a.w = w;
    a.C = 3;
    a.T = lr_target->data;
    a.T_pitch = lr_target->pitch;
    a.T_dtype = GLU_F32;
    a.out = hr_out->data;
    a.out_pitch = hr_out->pitch;
    a.out_dtype = hr_out->dtype;
    a.pdl = 1;
    return launch_apply(a, st);
}

}  // extern "C"

namespace {
// Arguments of the adjoint (shared by both entry points).
int backward_args(const glu_theta* theta, const glu_image* lr_target, const glu_image* grad_hr,
                  glu_image* grad_lr, float* grad_w, BackwardArgs& a) {
    if (!theta_ok(theta) || !image_ok(lr_target) || !image_ok(grad_hr) || !image_ok(grad_lr))
        return GLU_ERR_INVALID_ARG;
    if (lr_target->dtype != GLU_F32 || grad_hr->dtype != GLU_F32 || grad_lr->dtype != GLU_F32)
        return GLU_ERR_UNSUPPORTED;
    const int s = theta->scale;
    if (grad_hr->h != theta->H || grad_hr->w != theta->W || grad_hr->c != lr_target->c ||
        grad_lr->c != lr_target->c || lr_target->h != lr_dim(theta->H, s) ||
        lr_target->w != lr_dim(theta->W, s) || grad_lr->h != lr_target->h ||
        grad_lr->w != lr_target->w)
        return GLU_ERR_SHAPE;
    a.code = theta->code;
    a.weight = theta->weight;
    a.wfmt = theta->wfmt;
    a.H = theta->H;
    a.W = theta->W;
    a.s = s;
    a.S = theta->S;
    a.h = lr_target->h;
    a.w = lr_target->w;
    a.C = lr_target->c;
    a.T = (const float*)lr_target->data;
    a.T_pitch = lr_target->pitch;
    a.G = (const float*)grad_hr->data;
    a.G_pitch = grad_hr->pitch;
    a.gT = (float*)grad_lr->data;
    a.gT_pitch = grad_lr->pitch;
    a.gw = grad_w;
    return GLU_OK;
}
}  // namespace

extern "C" {

int glu_apply_backward(const glu_theta* theta, const glu_image* lr_target,
                       const glu_image* grad_hr, glu_image* grad_lr, float* grad_w, void* stream) {
    BackwardArgs a;
    const int rc = backward_args(theta, lr_target, grad_hr, grad_lr, grad_w, a);
    return rc ? rc : launch_apply_backward(a, (cudaStream_t)stream);
}

size_t glu_ls_update_workspace_size(const glu_theta* theta) {
    if (!theta_ok(theta)) return 0;
    return ls_update_workspace_bytes(lr_dim(theta->H, theta->scale),
                                     lr_dim(theta->W, theta->scale), theta->S);
}

int glu_ls_update(const glu_image* hr, const glu_theta* theta, const glu_image* lr_in,
                  glu_image* lr_out, void* ws, size_t ws_bytes, void* stream) {
    if (!image_ok(hr) || !theta_ok(theta) || !image_ok(lr_in) || !image_ok(lr_out))
        return GLU_ERR_INVALID_ARG;
    if ((hr->dtype != GLU_U8 && hr->dtype != GLU_F16) || hr->c != 3 || lr_in->c != 3 ||
        lr_out->c != 3 || lr_in->dtype != GLU_F32 || lr_out->dtype != GLU_F32 ||
        theta->wfmt != GLU_W_F32 || lr_in->data == lr_out->data)
        return GLU_ERR_UNSUPPORTED;
    const int s = theta->scale, h = lr_dim(theta->H, s), w = lr_dim(theta->W, s);
    if (hr->h != theta->H || hr->w != theta->W || lr_in->h != h || lr_in->w != w ||
        lr_out->h != h || lr_out->w != w)
        return GLU_ERR_SHAPE;
    if (!ws || ((uintptr_t)ws & 15u) != 0 || ws_bytes < ls_update_workspace_bytes(h, w, theta->S))
        return GLU_ERR_WORKSPACE;
    LsUpdate u;
    u.hr = hr->data;
    u.hr_pitch = hr->pitch;
    u.hr_dtype = hr->dtype;
    u.code = theta->code;
    u.weight = (const float*)theta->weight;
    u.L = (const float*)lr_in->data;
    u.L_pitch = lr_in->pitch;
    u.Lout = (float*)lr_out->data;
    u.Lout_pitch = lr_out->pitch;
    u.H = theta->H;
    u.W = theta->W;
    u.h = h;
    u.w = w;
    u.s = s;
    u.S = theta->S;
    u.slots = (float*)ws;
    u.active = nullptr;
    return ls_update(u, (cudaStream_t)stream);
}

size_t glu_ls_joint_workspace_size(int32_t H, int32_t W, int32_t scale, const glu_params* params) {
    if (H <= 0 || W <= 0 || H >= (1 << 22) || scale < 1 || !params_ok(params)) return 0;
    return ls_joint_workspace_bytes(H, W, scale, params->S);
}

int glu_ls_joint_optimize(const glu_image* hr, int32_t scale, const glu_params* params,
                          glu_image* lr_out, glu_theta* theta, float* err_map,
                          glu_ls_stats* stats, void* ws, size_t ws_bytes, void* stream) {
    if (!image_ok(hr) || !image_ok(lr_out) || !params_ok(params) || !theta_ok(theta) || scale < 1)
        return GLU_ERR_INVALID_ARG;
    if ((hr->dtype != GLU_U8 && hr->dtype != GLU_F16) || hr->c != 3 || lr_out->c != 3 ||
        lr_out->dtype != GLU_F32 || theta->wfmt != GLU_W_F32 || params->mode != GLU_MODE_FAST)
        return GLU_ERR_UNSUPPORTED;
    if (theta->H != hr->h || theta->W != hr->w || theta->S != params->S || theta->scale != scale ||
        lr_out->h != lr_dim(hr->h, scale) || lr_out->w != lr_dim(hr->w, scale))
        return GLU_ERR_SHAPE;
    const size_t need = ls_joint_workspace_bytes(hr->h, hr->w, scale, params->S);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255u) != 0) return GLU_ERR_WORKSPACE;
    LsJoint j;
    j.hr_image = *hr;
    j.lr_image = *lr_out;
    j.L = (float*)lr_out->data;
    j.L_pitch = lr_out->pitch;
    j.code = theta->code;
    j.weight = (float*)theta->weight;
    j.err = err_map;
    j.H = hr->h;
    j.W = hr->w;
    j.s = scale;
    j.S = params->S;
    j.N = params->N;
    j.eps255 = fmaxf(params->eps * 255.0f, 1e-12f);
    j.ws = ws;
    unsigned long long R[GLU_MAX_ITERS + 1];
    int kept = 0;
    const int rc = ls_joint(j, (cudaStream_t)stream, stats ? R : nullptr, stats ? &kept : nullptr);
    if (rc) return rc;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->R0 = (double)R[0] * (1.0 / 4294967296.0);
        for (int i = 1; i <= params->N; ++i)
            stats->residual[i - 1] = (double)R[i] * (1.0 / 4294967296.0);
        stats->iterations = params->N;
        stats->kept = kept;
    }
    return GLU_OK;
}

int glu_test_set_wait_limit(uint64_t ns) {
    set_trial_wait_limit((unsigned long long)ns);
    return GLU_OK;
}

size_t glu_apply_backward_plan_size(const glu_theta* theta) {
    if (!theta_ok(theta) || (int64_t)theta->H * theta->W >= ((int64_t)1 << 30)) return 0;
    const int s = theta->scale;
    return apply_backward_plan_bytes((int64_t)theta->H * theta->W,
                                     (int64_t)lr_dim(theta->H, s) * lr_dim(theta->W, s), theta->S);
}

int glu_apply_backward_plan(const glu_theta* theta, void* plan, size_t plan_bytes, void* stream) {
    const size_t need = glu_apply_backward_plan_size(theta);
    if (need == 0) return GLU_ERR_INVALID_ARG;
    if (!plan || ((uintptr_t)plan & 3u) != 0 || plan_bytes < need) return GLU_ERR_WORKSPACE;
    return apply_backward_plan(theta->code, theta->H, theta->W, theta->scale, theta->S, plan,
                               (cudaStream_t)stream);
}

int glu_apply_backward_planned(const glu_theta* theta, const void* plan,
                               const glu_image* lr_target, const glu_image* grad_hr,
                               glu_image* grad_lr, float* grad_w, void* stream) {
    BackwardArgs a;
    const int rc = backward_args(theta, lr_target, grad_hr, grad_lr, grad_w, a);
    if (rc) return rc;
    if (!plan || ((uintptr_t)plan & 3u) != 0) return GLU_ERR_WORKSPACE;
    return launch_apply_backward_planned(a, plan, (cudaStream_t)stream);
}

size_t glu_apply_backward_workspace_size(const glu_theta* theta, int32_t c) {
    if (!theta_ok(theta) || c < 1 || c > 4) return 0;
    return apply_backward_workspace_bytes(lr_dim(theta->H, theta->scale),
                                          lr_dim(theta->W, theta->scale), theta->S, c);
}

int glu_apply_backward_ws(const glu_theta* theta, const glu_image* lr_target,
                          const glu_image* grad_hr, glu_image* grad_lr, float* grad_w, void* ws,
                          size_t ws_bytes, void* stream) {
    BackwardArgs a;
    const int rc = backward_args(theta, lr_target, grad_hr, grad_lr, grad_w, a);
    if (rc) return rc;
    if (!ws || ((uintptr_t)ws & 15u) != 0 ||
        ws_bytes < apply_backward_workspace_bytes(a.h, a.w, a.S, a.C))
        return GLU_ERR_WORKSPACE;
    return launch_apply_backward_ws(a, ws, (cudaStream_t)stream);
}

int glu_theta_decode(const glu_theta* theta, int32_t* a, int32_t* b, float* w, void* stream) {
    if (!theta_ok(theta) || (!a && !b && !w)) return GLU_ERR_INVALID_ARG;
    if ((int64_t)lr_dim(theta->H, theta->scale) * lr_dim(theta->W, theta->scale) >
        (int64_t)INT32_MAX)
        return GLU_ERR_SHAPE;
    return launch_theta_decode(theta->code, theta->weight, theta->wfmt, theta->H, theta->W,
                               theta->scale, theta->S, a, b, w, (cudaStream_t)stream);
}

size_t glu_workspace_size(int32_t op, int32_t H, int32_t W, int32_t scale,
                          const glu_params* params) {
    if (H <= 0 || W <= 0 || H >= (1 << 22) || scale < 1 || !params_ok(params)) return 0;
    const int h = lr_dim(H, scale), w = lr_dim(W, scale);
    switch (op) {
        case GLU_OP_JOINT: return joint_workspace_bytes(H, W, scale, params->S, params->N);
        case GLU_OP_LS_JOINT: return ls_joint_workspace_bytes(H, W, scale, params->S);
        case GLU_OP_LS_UPDATE: return ls_update_workspace_bytes(h, w, params->S);
        case GLU_OP_APPLY_BACKWARD: return apply_backward_workspace_bytes(h, w, params->S, 3);
        case GLU_OP_APPLY_BACKWARD_PLAN:
            if ((int64_t)H * W >= ((int64_t)1 << 30)) return 0;
            return apply_backward_plan_bytes((int64_t)H * W, (int64_t)h * w, params->S);
        default: return 0;
    }
}

size_t glu_joint_workspace_size(int32_t H, int32_t W, int32_t scale, const glu_params* params) {
    if (H <= 0 || W <= 0 || scale < 1 || !params_ok(params)) return 0;
    return joint_workspace_bytes(H, W, scale, params->S, params->N);
}

int64_t glu_joint_decisions(const void* ws, size_t ws_bytes, int32_t H, int32_t W, int32_t scale,
                            const glu_params* params, int8_t* out, int64_t cap, void* stream) {
    if (!ws || !out || cap < 0 || H <= 0 || W <= 0 || scale < 1 || !params_ok(params))
        return GLU_ERR_INVALID_ARG;
    int64_t n = 0;
    const int rc = joint_decisions(ws, ws_bytes, H, W, scale, params->N, out, cap,
                                   (cudaStream_t)stream, &n);
    return rc != GLU_OK ? rc : n;
}

int glu_joint_optimize(const glu_image* hr, int32_t scale, const glu_params* params,
                       glu_image* lr_out, glu_theta* theta, float* err_map,
                       glu_joint_stats* stats, void* ws, size_t ws_bytes, void* stream) {
    return joint_optimize(hr, scale, params, lr_out, theta, err_map, stats, ws, ws_bytes, stream,
                          0);
}

int64_t glu_test_joint_graph_count(void) { return joint_graphs_recorded(); }

int glu_test_joint_argmax_log(void* buf, int64_t cap) {
    if (buf && (cap < 0 || ((uintptr_t)buf & 15u) != 0)) return GLU_ERR_INVALID_ARG;
    set_argmax_log(buf, buf ? cap : 0);
    return GLU_OK;
}

}  // extern "C"

namespace {

// Checks shared by the batched entry points; fills the launcher's item.
int search_item(const glu_batch_item& it, const glu_params* p, SearchArgs* a) {
    const glu_image* hr = &it.hr;
    const glu_image* lr = &it.lr;
    const glu_theta* th = &it.theta;
    if (!image_ok(hr) || !image_ok(lr) || !theta_ok(th)) return GLU_ERR_INVALID_ARG;
    if (hr->c != 3 || lr->c != 3) return GLU_ERR_UNSUPPORTED;
    if (hr->dtype != GLU_U8 && hr->dtype != GLU_F16) return GLU_ERR_UNSUPPORTED;
    const int s = th->scale;
    if (th->H != hr->h || th->W != hr->w || lr->h != lr_dim(hr->h, s) ||
        lr->w != lr_dim(hr->w, s))
        return GLU_ERR_SHAPE;
    a->hr = hr->data;
    a->hr_pitch = hr->pitch;
    a->hr_dtype = hr->dtype;
    a->lr = lr->data;
    a->lr_pitch = lr->pitch;
    a->lr_dtype = lr->dtype;
    a->H = hr->h;
    a->W = hr->w;
    a->h = lr->h;
    a->w = lr->w;
    a->s = s;
    a->S = th->S;
    a->eps255 = fmaxf(p->eps * 255.0f, 1e-12f);
    a->gnu = p->mode == GLU_MODE_GNU;
    a->code = th->code;
    a->weight = th->weight;
    a->wfmt = th->wfmt;
    a->err = it.err_map;
    return GLU_OK;
}

int joint_item(const glu_batch_item& it, JointItem* o) {
    const glu_image* hr = &it.hr;
    const glu_image* lr = &it.lr;
    const glu_theta* th = &it.theta;
    if (!image_ok(hr) || !image_ok(lr) || !theta_ok(th)) return GLU_ERR_INVALID_ARG;
    if (hr->dtype != GLU_U8 || lr->dtype != GLU_U8 || hr->c != 3 || lr->c != 3)
        return GLU_ERR_UNSUPPORTED;
    const int s = th->scale;
    if (th->H != hr->h || th->W != hr->w || lr->h != lr_dim(hr->h, s) ||
        lr->w != lr_dim(hr->w, s))
        return GLU_ERR_SHAPE;
    o->hr = (const uint8_t*)hr->data;
    o->hr_pitch = hr->pitch;
    o->lr = (uint8_t*)lr->data;
    o->lr_pitch = lr->pitch;
    o->H = hr->h;
    o->W = hr->w;
    o->s = s;
    o->S = th->S;
    o->code = th->code;
    o->weight = th->weight;
    o->err = it.err_map;
    return GLU_OK;
}

// Sizes only (for the workspace query).
int joint_item_sizes(const glu_batch_item& it, JointItem* o) {
    if (it.hr.h <= 0 || it.hr.w <= 0 || it.theta.scale < 1 || it.theta.S < 1 || it.theta.S > 9 ||
        !(it.theta.S & 1))
        return GLU_ERR_INVALID_ARG;
    *o = JointItem{};
    o->H = it.hr.h;
    o->W = it.hr.w;
    o->s = it.theta.scale;
    o->S = it.theta.S;
    return GLU_OK;
}

}  // namespace

extern "C" {

int glu_optimize_batched(const glu_batch_item* items, int32_t n, const glu_params* params,
                         void* stream) {
    if (n < 0 || (n > 0 && !items) || !params_ok(params)) return GLU_ERR_INVALID_ARG;
    if (n == 0) return GLU_OK;
    constexpr int kChunk = 64;
    SearchArgs a[kChunk];
    for (int k0 = 0; k0 < n; k0 += kChunk) {
        const int m = n - k0 < kChunk ? n - k0 : kChunk;
        for (int k = 0; k < m; ++k) {
            const int rc = search_item(items[k0 + k], params, &a[k]);
            if (rc) return rc;
            if (a[k].hr_dtype != items[0].hr.dtype || a[k].wfmt != items[0].theta.wfmt)
                return GLU_ERR_UNSUPPORTED;
        }
        if (params->mode == GLU_MODE_EXACT) {
            if (a[0].wfmt != GLU_W_F32) return GLU_ERR_UNSUPPORTED;
            for (int k = 0; k < m; ++k) {
                const int rc = launch_search_exact(a[k], (cudaStream_t)stream);
                if (rc) return rc;
            }
            continue;
        }
        const int rc = launch_search_batch(a, m, (cudaStream_t)stream);
        if (rc) return rc;
    }
    return GLU_OK;
}

size_t glu_joint_batched_workspace_size(const glu_batch_item* items, int32_t n,
                                        const glu_params* params) {
    if (n <= 0 || n > kMaxJointBatch || !items || !params_ok(params)) return 0;
    JointItem it[kMaxJointBatch];
    for (int k = 0; k < n; ++k)
        if (joint_item_sizes(items[k], &it[k])) return 0;
    return joint_batch_workspace_bytes(it, n, params->N);
}

int glu_joint_optimize_batched(const glu_batch_item* items, int32_t n, const glu_params* params,
                               glu_joint_stats* stats, void* ws, size_t ws_bytes, void* stream) {
    if (n < 0 || (n > 0 && !items) || !params_ok(params)) return GLU_ERR_INVALID_ARG;
    if (n == 0) return GLU_OK;
    if (n > kMaxJointBatch) return GLU_ERR_UNSUPPORTED;
    if (params->mode != GLU_MODE_FAST) return GLU_ERR_UNSUPPORTED;
    JointItem it[kMaxJointBatch];
    for (int k = 0; k < n; ++k) {
        const int rc = joint_item(items[k], &it[k]);
        if (rc) return rc;
        if (items[k].theta.wfmt != items[0].theta.wfmt) return GLU_ERR_UNSUPPORTED;
    }
    const size_t need = joint_batch_workspace_bytes(it, n, params->N);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255u) != 0) return GLU_ERR_WORKSPACE;
    JointCommon cm;
    cm.eps255 = fmaxf(params->eps * 255.0f, 1e-12f);
    cm.tau = params->tau;
    cm.N = params->N;
    cm.strict = params->joint == GLU_JOINT_STRICT;
    cm.conn = params->connectivity;
    cm.wfmt = items[0].theta.wfmt;
    cm.wait_limit_ns = 0;
    return launch_joint_batch(it, n, cm, ws, ws_bytes, stats, (cudaStream_t)stream);
}

}  // extern "C"
