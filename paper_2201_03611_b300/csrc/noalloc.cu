// Backward pass for callers that cannot allocate device memory.
//
// shine_pipeline_bwd needs a caller-supplied device workspace for its per-warp partial sums of
// d kappa, d Wx and d Wy. Some callers have no way to provide one: a plug-in whose host hands
// it only the input and output buffers, a real-time loop that forbids any allocation after
// start-up, or code running where the framework owns all device memory. For them this file
// keeps the partial sums in one fixed array in the library's own device memory and runs the
// ordinary backward pass on it, calling no allocating routine at all.
#include <cuda_runtime.h>

#include <mutex>

#include "harris_kernels.h"
#include "shine.h"
#include "shine_host.h"
#include "entry.h"

namespace shine {
namespace {

// Partial-sum slots per parameter cotangent. The backward pass uses at most 64 warps per SM
// (one slot each), so this covers any image on a GPU with up to 256 SMs.
constexpr int64_t kNoAllocWarps = 16384;
constexpr size_t kNoAllocBytes =
    kWorkspaceHeader + (size_t)kParamSlots * kNoAllocWarps * sizeof(double);  // ~2.5 MB

// Lives on every GPU that loads the library, until the process exits. In host code this
// name is only a stand-in for the symbol, never a device address: the address is looked up
// per device below.
__device__ __align__(256) double g_bwd_partials[kNoAllocBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_partials_ptr[kMaxDevices] = {};

// Device address of g_bwd_partials on the current device, looked up once per device.
shine_status partials_on_current_device(void** ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return SHINE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_partials_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bwd_partials);
        if (e != cudaSuccess) return cuda_status(e);
        g_partials_ptr[dev] = p;
    }
    *ptr = g_partials_ptr[dev];
    return SHINE_OK;
}

}  // namespace
}  // namespace shine

extern "C" shine_status shine_pipeline_bwd_noalloc(const void* img, int64_t H, int64_t W, int64_t img_pitch,
                                                   shine_dtype dt, shine_border border, const float* kappa,
                                                   const float* wx, const float* wy, const void* grad_out,
                                                   int64_t gout_pitch, shine_dtype gout_dt, void* grad_img,
                                                   int64_t gimg_pitch, float* grad_kappa, float* grad_wx,
                                                   float* grad_wy, void* stream) {
    SHINE_ENTRY("shine_pipeline_bwd_noalloc");
    if (!img || !kappa || !wx || !wy || !grad_out) return SHINE_ERR_INVALID_ARG;  // before touching a GPU
    size_t need = 0;
    shine_status st = shine_pipeline_bwd_workspace(H, W, border, &need);
    if (st != SHINE_OK) return st;
    if (need > shine::kNoAllocBytes) return SHINE_ERR_UNSUPPORTED;  // more partial sums than the array holds
    void* partials = nullptr;
    st = shine::partials_on_current_device(&partials);
    if (st != SHINE_OK) return st;
    unsigned int* flag = shine::wait_flag();
    if (flag == nullptr) return SHINE_ERR_CUDA;
    // Every launch writes all the partial sums its finalize step reads, so nothing left in the
    // array by an earlier call is ever used and nothing needs clearing. A bounded wait that gives
    // up is reported in the library-wide flag that shine_wait_status reads (the caller has no
    // workspace to pass to shine_workspace_status).
    return shine::run_bwd(img, H, W, img_pitch, dt, border, kappa, wx, wy, grad_out, gout_pitch, gout_dt, nullptr, 0,
                          grad_img, gimg_pitch, grad_kappa, grad_wx, grad_wy, partials, shine::kNoAllocBytes, stream,
                          flag);
}
