// Forward + backward of an image held in host memory, with the host<->device copies overlapped
// with the kernels.
//
// The image is cut into row bands. Band b's rows are uploaded on one stream; the forward and
// adjoint kernels for band b run on a second stream once band b+1 (which holds band b's halo
// rows) has arrived; R and d img of band b are downloaded on a third stream once its kernels are
// done. Uploads, kernels and downloads of different bands therefore run at the same time, and
// the step costs about the larger of the two transfer directions instead of their sum. The band
// kernels are the single-image kernels restricted to a row range of the full image (clamping
// only at the true image border), so every pixel's result equals the single-call result; the
// parameter cotangents of all bands are reduced together in one fixed-order pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "harris_kernels.h"
#include "shine.h"
#include "shine_host.h"
#include "entry.h"

namespace shine {
namespace {

constexpr int kMaxBands = 64;
constexpr int kMaxDevices = 64;

// Streams and events of the pipeline, created once per device on first use and kept for the
// life of the process (they are not device memory).
struct DeviceStreams {
    cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
    cudaEvent_t start = nullptr, comp_done = nullptr, down_done = nullptr;
    cudaEvent_t in[kMaxBands] = {}, k[kMaxBands] = {};
    std::mutex mu;  // one pipeline call at a time per device
    bool ready = false;
};
DeviceStreams g_dev[kMaxDevices];
std::mutex g_init;

shine_status device_streams(DeviceStreams** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    if (dev < 0 || dev >= kMaxDevices) return SHINE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_init);
    DeviceStreams& d = g_dev[dev];
    if (!d.ready) {
        const unsigned ef = cudaEventDisableTiming;
        e = cudaStreamCreateWithFlags(&d.up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d.comp, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d.down, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.start, ef);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.comp_done, ef);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.down_done, ef);
        for (int i = 0; i < kMaxBands && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&d.in[i], ef);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.k[i], ef);
        }
        if (e != cudaSuccess) return cuda_status(e);
        d.ready = true;
    }
    *out = &d;
    return SHINE_OK;
}

// Rows [lo, hi) of band b when H rows are cut into n bands.
void band_rows(int64_t H, int n, int b, int64_t& lo, int64_t& hi) {
    balanced_slice(H, n, b, lo, hi);
}

}  // namespace
}  // namespace shine

using namespace shine;

extern "C" {

shine_status shine_pipeline_host_workspace(int64_t H, int64_t W, shine_border border, int32_t nbands,
                                           size_t* bytes) {
    if (!bytes || nbands < 1 || nbands > kMaxBands) return SHINE_ERR_INVALID_ARG;
    shine_status st = check_shape(H, W, border);
    if (st != SHINE_OK) return st;
    Geometry g = bwd_geometry(H, W, border);
    *bytes = kWorkspaceHeader + (size_t)kParamSlots * (size_t)nbands * (size_t)bwd_max_warps(g) * sizeof(double);
    return SHINE_OK;
}

shine_status shine_pipeline_host(const void* img_h, const void* gout_h, void* out_h, void* gimg_h, int64_t H,
                                 int64_t W, shine_dtype dt, shine_border border, const float* kappa, const float* wx,
                                 const float* wy, float* grad_params, void* dev_img, void* dev_gout, void* dev_out,
                                 void* dev_gimg, void* workspace, size_t ws_bytes, int32_t nbands, void* stream) {
    SHINE_ENTRY("shine_pipeline_host");
    if (!img_h || !gout_h || !kappa || !wx || !wy || !dev_img || !dev_gout || !dev_out || !dev_gimg)
        return SHINE_ERR_INVALID_ARG;
    if (!dtype_ok(dt) || nbands < 1 || nbands > kMaxBands) return SHINE_ERR_INVALID_ARG;
    shine_status st = check_shape(H, W, border);
    if (st != SHINE_OK) return st;
    if (H < 8 * (int64_t)nbands) return SHINE_ERR_INVALID_ARG;  // a band must hold its neighbours' halo
    size_t need = 0;
    shine_pipeline_host_workspace(H, W, border, nbands, &need);
    if (!workspace || ws_bytes < need) return SHINE_ERR_WORKSPACE;
    const size_t si = dtype_size(dt);
    if (!aligned_to(dev_img, 16) || !aligned_to(dev_gout, 16) || !aligned_to(dev_out, 16) ||
        !aligned_to(dev_gimg, 16) || !aligned_to(workspace, 16) || !aligned_to(kappa, 4) || !aligned_to(wx, 4) ||
        !aligned_to(wy, 4) || (grad_params && !aligned_to(grad_params, 4)))
        return SHINE_ERR_ALIGNMENT;
    DeviceStreams* ds = nullptr;
    st = device_streams(&ds);
    if (st != SHINE_OK) return st;
    std::lock_guard<std::mutex> lock(ds->mu);

    const int64_t Ho = border == SHINE_VALID ? H - 4 : H, Wo = border == SHINE_VALID ? W - 4 : W;
    const int oy = border == SHINE_VALID ? 2 : 0;
    const size_t img_row = (size_t)3 * W * si, map_row = (size_t)Wo * si;
    const Geometry gb = bwd_geometry(H, W, border);
    const int64_t tmax = bwd_max_warps(gb);
    double* partials = reinterpret_cast<double*>(static_cast<char*>(workspace) + kWorkspaceHeader);
    unsigned int* err = static_cast<unsigned int*>(workspace);
    cudaStream_t caller = static_cast<cudaStream_t>(stream);

#define SHINE_TRY(x)                                   \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

    // Order the pipeline after the caller's earlier work.
    SHINE_TRY(cudaEventRecord(ds->start, caller));
    SHINE_TRY(cudaStreamWaitEvent(ds->up, ds->start, 0));
    SHINE_TRY(cudaStreamWaitEvent(ds->comp, ds->start, 0));
    SHINE_TRY(cudaStreamWaitEvent(ds->down, ds->start, 0));
    SHINE_TRY(cudaMemsetAsync(workspace, 0, need, ds->comp));
    (void)err;

    // Uploads: band b's image rows and the cotangent rows of the same image rows.
    for (int b = 0; b < nbands; ++b) {
        int64_t lo, hi;
        band_rows(H, nbands, b, lo, hi);
        SHINE_TRY(cudaMemcpyAsync(static_cast<char*>(dev_img) + lo * img_row,
                                  static_cast<const char*>(img_h) + lo * img_row, (hi - lo) * img_row,
                                  cudaMemcpyHostToDevice, ds->up));
        const int64_t glo = std::max<int64_t>(lo - oy, 0), ghi = std::min<int64_t>(hi - oy, Ho);
        if (ghi > glo)
            SHINE_TRY(cudaMemcpyAsync(static_cast<char*>(dev_gout) + glo * map_row,
                                      static_cast<const char*>(gout_h) + glo * map_row, (ghi - glo) * map_row,
                                      cudaMemcpyHostToDevice, ds->up));
        SHINE_TRY(cudaEventRecord(ds->in[b], ds->up));
    }
    // Kernels of band b once band b+1 (its lower halo) is on the device; downloads once done.
    for (int b = 0; b < nbands; ++b) {
        int64_t lo, hi;
        band_rows(H, nbands, b, lo, hi);
        SHINE_TRY(cudaStreamWaitEvent(ds->comp, ds->in[std::min(b + 1, nbands - 1)], 0));
        FwdArgs f;
        static_cast<Geometry&>(f) = fwd_geometry(H, W, border);
        f.ylo = (int)std::max<int64_t>(f.ylo, lo);
        f.yhi = (int)std::min<int64_t>(f.yhi, hi);
        if (f.yhi > f.ylo) {
            f.img = dev_img; f.img_pitch = 3 * W; f.out = dev_out; f.out_pitch = Wo;
            f.kappa = kappa; f.wx = wx; f.wy = wy;
            f.aligned = (img_row % (si == 4 ? 16 : 8)) == 0;  // vector staging needs aligned rows
            f.out_vec = border == SHINE_CLAMP && (Wo * si) % 16 == 0 && aligned_to(dev_out, 16);
            f.tma = SHINE_FWD_TMA && (img_row % 16) == 0;
            f.err = wait_flag();
            SHINE_TRY(launch_harris_fwd(f, dt, dt, ds->comp));
        }
        BwdArgs a;
        static_cast<Geometry&>(a) = gb;
        a.ylo = (int)lo;
        a.yhi = (int)hi;
        a.img = dev_img; a.img_pitch = 3 * W;
        a.gout = dev_gout; a.gout_pitch = Wo; a.gho = (int)Ho; a.gwo = (int)Wo;
        a.gimg = dev_gimg; a.gimg_pitch = 3 * W;
        a.kappa = kappa; a.wx = wx; a.wy = wy;
        a.partials = partials;
        a.pstride = (int64_t)nbands * tmax;
        a.poffset = (int64_t)b * tmax;
        a.err = err;
        const size_t chunk = si == 4 ? 16 : 8;
        a.aligned = (img_row % chunk) == 0;
        a.g_aligned = border == SHINE_CLAMP && (map_row % (4 * si)) == 0;
        a.gimg_vec = (img_row % chunk) == 0;
        a.tma = SHINE_BWD_TMA && (img_row % 16) == 0 && (map_row % 16) == 0 && border == SHINE_CLAMP;
        a.rout = nullptr; a.rout_pitch = 0; a.rout_vec = 0;
        SHINE_TRY(launch_harris_bwd(a, dt, dt, (int)tmax, ds->comp, nullptr));
        SHINE_TRY(cudaEventRecord(ds->k[b], ds->comp));
        SHINE_TRY(cudaStreamWaitEvent(ds->down, ds->k[b], 0));
        if (out_h) {
            const int64_t olo = std::max<int64_t>(lo - oy, 0), ohi = std::min<int64_t>(hi - oy, Ho);
            if (ohi > olo)
                SHINE_TRY(cudaMemcpyAsync(static_cast<char*>(out_h) + olo * map_row,
                                          static_cast<const char*>(dev_out) + olo * map_row, (ohi - olo) * map_row,
                                          cudaMemcpyDeviceToHost, ds->down));
        }
        if (gimg_h)
            SHINE_TRY(cudaMemcpyAsync(static_cast<char*>(gimg_h) + lo * img_row,
                                      static_cast<const char*>(dev_gimg) + lo * img_row, (hi - lo) * img_row,
                                      cudaMemcpyDeviceToHost, ds->down));
    }
    if (grad_params)
        SHINE_TRY(launch_finalize_params(partials, (int64_t)nbands * tmax, grad_params, grad_params + 1,
                                         grad_params + 10, ds->comp));
    SHINE_TRY(cudaEventRecord(ds->comp_done, ds->comp));
    SHINE_TRY(cudaEventRecord(ds->down_done, ds->down));
    SHINE_TRY(cudaStreamWaitEvent(caller, ds->comp_done, 0));
    SHINE_TRY(cudaStreamWaitEvent(caller, ds->down_done, 0));
#undef SHINE_TRY
    return SHINE_OK;
}

}  // extern "C"
