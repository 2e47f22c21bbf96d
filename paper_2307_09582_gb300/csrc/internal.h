// Host-side launcher interfaces between the C-ABI layer (api.cu) and the kernel files.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "glu.h"

namespace glu {

// Arguments of the Algorithm 1 search over a whole image (or a batch item).
struct SearchArgs {
    const void* hr;
    int64_t hr_pitch;  // elements
    int hr_dtype;
    const void* lr;
    int64_t lr_pitch;  // elements
    int lr_dtype;
    int H, W, h, w, s, S;
    float eps255;      // eps in 1/255 colour units
    int gnu;
    uint16_t* code;
    void* weight;
    int wfmt;
    float* err;        // nullable
};

// 2D tiled TMA tensor map over a row-major array: `inner` elements of `esize` bytes per row,
// `rows` rows `row_bytes` apart, box of box_inner x box_rows elements, out-of-bounds elements
// zero-filled on loads and skipped on stores. False when TMA cannot describe the array (base
// not 16-byte aligned, row_bytes or the box row not a multiple of 16 bytes, box side > 256).
bool encode_map_2d(CUtensorMap* map, CUtensorMapDataType dt, size_t esize, const void* base,
                   uint64_t inner, uint64_t rows, uint64_t row_bytes, uint32_t box_inner,
                   uint32_t box_rows);

int launch_search(const SearchArgs& a, cudaStream_t st);
// GLU* (Eq. 4, every pair of window pixels); float32 weights only.
int launch_search_exact(const SearchArgs& a, cudaStream_t st);
constexpr int kMaxSearchBatch = 32;  // images per search launch (the kernel's parameter block)
// Several images in one persistent launch; every item shares hr_dtype, wfmt, gnu and eps255.
int launch_search_batch(const SearchArgs* items, int n, cudaStream_t st);

struct ApplyArgs {
    const uint16_t* code;
    const void* weight;
    int wfmt;
    int H, W, s, S, h, w, C;
    const void* T;
    int64_t T_pitch;
    int T_dtype;
    void* out;
    int64_t out_pitch;
    int out_dtype;
    int pdl = 0;   // 1: the preceding kernel of the stream writes T and triggers its dependents
                   // (the persistent pipeline starts loading codes and weights before it ends)
};

int launch_apply(const ApplyArgs& a, cudaStream_t st);
// The LR operator f (3x3 filter, then saturation and gamma) of a uint8 or float32 3-channel LR
// image into a float32 image T, one thread per LR pixel; the kernel lets a programmatic
// dependent launch start at once (its dependent waits for it before reading T).
int launch_lr_op(const void* X, int x_dtype, int h, int w, int64_t pitch, float* Y, int64_t ypitch,
                 int filter, float sat, float gamma, cudaStream_t st);
int launch_theta_decode(const uint16_t* code, const void* weight, int wfmt, int H, int W, int s,
                        int S, int32_t* a, int32_t* b, float* wt, cudaStream_t st);

struct BackwardArgs {
    const uint16_t* code;
    const void* weight;
    int wfmt;
    int H, W, s, S, h, w, C;
    const float* T;
    int64_t T_pitch;
    const float* G;      // H x W x C upstream gradient
    int64_t G_pitch;
    float* gT;           // h x w x C
    int64_t gT_pitch;
    float* gw;           // nullable, H * W
};

int launch_apply_backward(const BackwardArgs& a, cudaStream_t st);
// The same with a caller workspace of apply_backward_workspace_bytes(h, w, S, C) bytes
// (16-byte aligned): per-block window-bucket sums, then one gather per LR pixel.
size_t apply_backward_workspace_bytes(int h, int w, int S, int C);
int launch_apply_backward_ws(const BackwardArgs& a, void* ws, cudaStream_t st);
// The inverse pixel-to-LR map of a Theta (built once, apply_backward_plan_bytes, 4-byte aligned)
// and the adjoint that reads it.
size_t apply_backward_plan_bytes(int64_t np, int64_t nq, int S);
int apply_backward_plan(const uint16_t* code, int H, int W, int s, int S, void* plan,
                        cudaStream_t st);
int launch_apply_backward_planned(const BackwardArgs& a, const void* plan, cudaStream_t st);

int launch_downsample(const glu_image& hr, int s, int mode, const glu_image& lr, cudaStream_t st);

// Least-squares LR colour update for a fixed Theta (k_ls.cu; float32 weights, float32 LR colours
// in [0, 1]) and its alternation with Algorithm 1.
struct LsUpdate {
    const void* hr;
    int64_t hr_pitch;
    int hr_dtype;
    const uint16_t* code;
    const float* weight;
    const float* L;
    int64_t L_pitch;
    float* Lout;
    int64_t Lout_pitch;
    int H, W, h, w, s, S;
    float* slots;         // ls_update_workspace_bytes(h, w, S), 16-byte aligned
    const int* active;    // nullable (device flag)
};
size_t ls_update_workspace_bytes(int h, int w, int S);
int ls_update(const LsUpdate& u, cudaStream_t st);
struct LsJoint {
    glu_image hr_image, lr_image;   // guide (U8 / F16) and the float32 LR image (L below)
    float* L;
    int64_t L_pitch;
    uint16_t* code;
    float* weight;
    float* err;                     // nullable
    int H, W, s, S, N;
    float eps255;
    void* ws;                       // ls_joint_workspace_bytes, 256-byte aligned
};
size_t ls_joint_workspace_bytes(int H, int W, int s, int S);
int ls_joint(const LsJoint& j, cudaStream_t st, unsigned long long* R_host, int* kept_host);

// Status words of each translation unit (read and cleared; synchronous on st).
int read_and_clear_status_search(cudaStream_t st);
int read_and_clear_status_apply(cudaStream_t st);
int read_and_clear_status_down(cudaStream_t st);
int read_and_clear_status_joint(cudaStream_t st);
int read_and_clear_status_ls(cudaStream_t st);
int read_and_clear_status_search_exact(cudaStream_t st);

// Joint optimisation (Algorithm 2).
struct JointArgs {
    const uint8_t* hr;
    int64_t hr_pitch;   // bytes
    uint8_t* lr;
    int64_t lr_pitch;   // bytes
    int H, W, h, w, s, S;
    float eps255, tau;
    int N, strict, conn;
    uint16_t* code;
    void* weight;
    int wfmt;
    float* err;         // nullable: a workspace plane is used otherwise
};

size_t joint_workspace_bytes(int H, int W, int s, int S, int N);
int joint_decisions(const void* ws, size_t ws_bytes, int H, int W, int s, int N, int8_t* out,
                    int64_t cap, cudaStream_t st, int64_t* written);
int launch_joint(const JointArgs& a, void* ws, size_t ws_bytes, glu_joint_stats* stats,
                 cudaStream_t st, int direct = 0);
// Argument checks and launch of glu_joint_optimize; direct as in JointCommon.
int joint_optimize(const glu_image* hr, int32_t scale, const glu_params* params,
                   glu_image* lr_out, glu_theta* theta, float* err_map, glu_joint_stats* stats,
                   void* ws, size_t ws_bytes, void* stream, int direct);
// CUDA graphs recorded by the joint calls so far (test hook).
long long joint_graphs_recorded();

// Algorithm 2 over a batch of images in one set of launches.
constexpr int kMaxJointBatch = 32;
struct JointItem {
    const uint8_t* hr;
    int64_t hr_pitch;   // bytes
    uint8_t* lr;
    int64_t lr_pitch;   // bytes
    int H, W, s, S;
    uint16_t* code;
    void* weight;
    float* err;         // nullable: a workspace plane is used otherwise
};
struct JointCommon {
    float eps255, tau;
    int N, strict, conn, wfmt;
    unsigned long long wait_limit_ns = 0;  // set by launch_joint_batch (0: the default deadline)
    int4* argmax_log = nullptr;            // set by launch_joint_batch (test hook; null: off)
    long long argmax_cap = 0;
    // 1: every launch issued directly on the caller's stream: never recorded as a CUDA graph
    // (no stream creation, capture or instantiation) and no autotuner timing
    int direct = 0;
    int pad_ = 0;   // no implicit padding: the graph cache compares these bytes
};
static_assert(sizeof(JointCommon) == 56, "JointCommon has no implicit padding");
// Test hook: the deadline of the trial kernel's waits (0 restores the default).
void set_trial_wait_limit(unsigned long long ns);
// Test hook: log every trial's replacement choice (see glu_test_joint_argmax_log); null: off.
void set_argmax_log(void* buf, long long cap);
size_t joint_batch_workspace_bytes(const JointItem* items, int n, int N);
// stats: null or an array of n records
int launch_joint_batch(const JointItem* items, int n, const JointCommon& cm, void* ws,
                       size_t ws_bytes, glu_joint_stats* stats, cudaStream_t st);

}  // namespace glu
