// glu_joint_optimize_static: Algorithm 2 without any device allocation by the caller.
//
// Some callers cannot allocate device memory: a plug-in hosted by an application that owns
// every device allocation (it hands out no scratch and forbids its own cudaMalloc), or a
// latency-critical streaming loop where cudaMalloc / cudaFree can synchronise the device and
// stall it. For them the joint optimisation's workspace is a fixed array in the library's own
// device memory, GLU_JOINT_STATIC_BYTES (64 MiB) large. That holds the workspace of images up to
// about 0.88 megapixels at scale 8 with a 5x5 window and 5 iterations: the largest 16:9 image
// that fits is 1248 x 702 (63.5 MiB); 1024 x 768 fits (57.6 MiB); 1280 x 720 needs 66.4 MiB and
// is refused. Every GPU that loads the library keeps this array until the process exits.
//
// The array is shared by all calls on a device and keeps the previous call's contents; the
// optimisation initialises everything it reads. Calls that overlap on the GPU (for example on two
// streams at once) would use the same array and race: issue them one after another.
//
// The call allocates nothing on the device and creates no stream or graph: its launches go
// directly onto the caller's stream (the graph replay that glu_joint_optimize does for repeated
// calls is not used here), and the autotuner does not time variants during it.
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_joint_scratch[GLU_JOINT_STATIC_BYTES];

constexpr int kMaxDevices = 256;
struct ScratchAddr {
    unsigned long long ctx_id;   // id of the CUDA context the address belongs to (0: none yet)
    void* addr;
};
ScratchAddr g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;
std::once_flag g_driver_once;

void load_driver_entry_points() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
        g_ctx_current = (PFN_cuCtxGetCurrent_v4000)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
        g_ctx_id = (PFN_cuCtxGetId_v12000)p;
}

// Unique id of the context current on this thread (0 if none or unknown). Ids are never reused
// within a process, so an address cached for a context that was destroyed (cudaDeviceReset)
// never matches the context created after it.
unsigned long long current_context_id() {
    std::call_once(g_driver_once, load_driver_entry_points);
    if (!g_ctx_current || !g_ctx_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the array in the current device's context. The array's name is only a
// host-side stand-in and must never be passed to a kernel; cudaGetSymbolAddress, called with the
// device current, gives the address kernels use. It is looked up on the first call in each
// context (which also loads the library's device code there) and cached for that context.
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GLU_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long id = current_context_id();
    ScratchAddr& e = g_scratch[dev];
    if (id != 0 && e.ctx_id == id && e.addr) {
        *out = e.addr;
        return GLU_OK;
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_joint_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return GLU_ERR_CUDA;
    }
    // the lookup makes the device's primary context current if no context was yet
    e.ctx_id = id != 0 ? id : current_context_id();
    e.addr = p;
    *out = p;
    return GLU_OK;
}

}  // namespace

extern "C" int glu_joint_optimize_static(const glu_image* hr, int32_t scale,
                                         const glu_params* params, glu_image* lr_out,
                                         glu_theta* theta, float* err_map, glu_joint_stats* stats,
                                         void* stream) {
    if (!hr || !params || scale < 1) return GLU_ERR_INVALID_ARG;
    const size_t need = glu_joint_workspace_size(hr->h, hr->w, scale, params);
    if (need == 0) return GLU_ERR_INVALID_ARG;
    if (need > (size_t)GLU_JOINT_STATIC_BYTES) return GLU_ERR_WORKSPACE;  // image too large
    void* ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc != GLU_OK) return rc;
    return glu::joint_optimize(hr, scale, params, lr_out, theta, err_map, stats, ws,
                               (size_t)GLU_JOINT_STATIC_BYTES, stream, /*direct=*/1);
}
