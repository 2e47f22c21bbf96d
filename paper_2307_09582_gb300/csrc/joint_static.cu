// glu_joint_optimize_static: Algorithm 2 without any device allocation by the caller.
//
// Some callers cannot allocate device memory: a plug-in hosted by an application that owns
// every device allocation (it hands out no scratch and forbids its own cudaMalloc), or a
// latency-critical streaming loop where cudaMalloc / cudaFree can synchronise the device and
// stall it. For them the joint optimisation's workspace is a fixed array in the library's own
// device memory, sized for images up to GLU_JOINT_STATIC_BYTES of workspace (about 1.3 megapixels
// at scale 8 with a 5x5 window and 5 iterations). Every GPU that loads the library keeps this
// array until the process exits.
//
// The array is shared by all calls on a device and keeps the previous call's contents; the
// optimisation initialises everything it reads. Calls that overlap on the GPU (for example on two
// streams at once) would use the same array and race: issue them one after another.
#include <mutex>

#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_joint_scratch[GLU_JOINT_STATIC_BYTES];

constexpr int kMaxDevices = 256;
void* g_scratch_addr[kMaxDevices];   // device address of g_joint_scratch, per device
std::mutex g_scratch_mu;

// Device address of the array on the current device, looked up once per device (the name is a
// host-side stand-in and must not be passed to a kernel). The lookup happens on the first call
// on each device, with that device current.
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GLU_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_joint_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return GLU_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
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
    return glu_joint_optimize(hr, scale, params, lr_out, theta, err_map, stats, ws,
                              (size_t)GLU_JOINT_STATIC_BYTES, stream);
}
