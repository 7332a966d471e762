// extern "C" entry points of libshine (declared in include/shine.h): argument validation on
// the host, the work decomposition, and the kernel launches. Nothing here allocates device
// memory except shine_plan_create (in batched.cu), and nothing synchronises except the two
// status queries (shine_workspace_status, shine_wait_status).
#include <cuda_runtime.h>

#include <mutex>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "harris_kernels.h"
#include "shine.h"
#include "entry.h"
#include "shine_host.h"

namespace shine {

thread_local int g_last_cuda_error = 0;

// Set (atomically, to 1) by a kernel launched without a workspace -- the forward, corner and
// window kernels -- when one of its bounded waits gives up; read and cleared by
// shine_wait_status. One word per GPU that loads the library.
__device__ unsigned int g_wait_flag;
std::mutex g_wait_mutex;
unsigned int* g_wait_ptr[64] = {};

// Debug builds: the index-check violation word, one per GPU (see SHINE_CHECK).
__device__ unsigned int g_bounds_flag;
unsigned int* g_bounds_ptr[64] = {};

shine_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SHINE_OK;
    g_last_cuda_error = (int)e;
    return SHINE_ERR_CUDA;
}

size_t dtype_size(int dt) { return dt == SHINE_F32 ? 4 : 2; }
bool dtype_ok(int dt) { return dt == SHINE_F32 || dt == SHINE_BF16 || dt == SHINE_F16; }
bool border_ok(int b) { return b == SHINE_VALID || b == SHINE_CLAMP; }

unsigned int* wait_flag() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_wait_mutex);
    if (g_wait_ptr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_wait_flag) != cudaSuccess) return nullptr;
        g_wait_ptr[dev] = static_cast<unsigned int*>(p);
    }
    return g_wait_ptr[dev];
}

unsigned int* bounds_flag() {
    if constexpr (!SHINE_DEBUG_BOUNDS) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_wait_mutex);
    if (g_bounds_ptr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bounds_flag) != cudaSuccess) return nullptr;
        g_bounds_ptr[dev] = static_cast<unsigned int*>(p);
    }
    return g_bounds_ptr[dev];
}

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
    return n;
}

shine_status check_shape(int64_t H, int64_t W, int border) {
    if (!border_ok(border)) return SHINE_ERR_INVALID_ARG;
    const int64_t lo = border == SHINE_VALID ? 5 : 1;
    if (H < lo || W < lo || H > kMaxDim || W > kMaxDim) return SHINE_ERR_INVALID_ARG;
    return SHINE_OK;
}

void fill_geometry(Geometry& g, int64_t H, int64_t W, int border, bool full_image, int band_rows) {
    g.H = (int)H;
    g.W = (int)W;
    g.valid = border == SHINE_VALID;
    if (g.valid && !full_image) {
        g.xlo = 2; g.xhi = (int)W - 2; g.ylo = 2; g.yhi = (int)H - 2; g.ox = 2; g.oy = 2;
    } else {
        g.xlo = 0; g.xhi = (int)W; g.ylo = 0; g.yhi = (int)H;
        g.ox = g.valid ? 2 : 0; g.oy = g.valid ? 2 : 0;
    }
    g.x0 = 0;
    g.nseg = (g.xhi + kSegOut - 1) / kSegOut;
    g.band_rows = band_rows;
    g.nband = (g.yhi - g.ylo + band_rows - 1) / band_rows;
    g.nwarps = 0;
    g.dbg = bounds_flag();
}

Geometry fwd_geometry(int64_t H, int64_t W, int border) {
    Geometry g;
    fill_geometry(g, H, W, border, false, (int)H);
    g.x0 = kFwdSegmentOrigin;
    g.nseg = (g.xhi - g.x0 + kSegOut - 1) / kSegOut;
    return g;
}

Geometry bwd_geometry(int64_t H, int64_t W, int border) {
    Geometry g;
    fill_geometry(g, H, W, border, true, (int)H);
    g.x0 = kBwdSegmentOrigin;
    g.nseg = (g.xhi - g.x0 + kSegOut - 1) / kSegOut;
    return g;
}

int64_t bwd_max_warps(const Geometry& g) {
    const int64_t units = (int64_t)(g.yhi - g.ylo) * g.nseg;
    return std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * kMaxWarpsPerSm, units / kBwdMinRows));
}

bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

shine_status injected_fault(const char* name) {
    const char* spec = std::getenv("SHINE_FAULT_INJECT");
    if (spec == nullptr || *spec == '\0') return SHINE_OK;
    const size_t nlen = std::strlen(name);
    for (const char* p = spec; *p != '\0';) {
        const char* end = std::strchr(p, ',');
        if (end == nullptr) end = p + std::strlen(p);
        const char* eq = static_cast<const char*>(std::memchr(p, '=', (size_t)(end - p)));
        if (eq != nullptr) {
            const size_t klen = (size_t)(eq - p);
            if ((klen == 1 && *p == '*') || (klen == nlen && std::strncmp(p, name, nlen) == 0)) {
                const int v = std::atoi(eq + 1);
                if (v >= SHINE_ERR_INVALID_ARG && v <= SHINE_ERR_CUDA) return static_cast<shine_status>(v);
            }
        }
        p = *end != '\0' ? end + 1 : end;
    }
    return SHINE_OK;
}

}  // namespace shine

using namespace shine;

extern "C" {

const char* shine_status_string(shine_status s) {
    switch (s) {
        case SHINE_OK: return "ok";
        case SHINE_ERR_INVALID_ARG: return "invalid argument";
        case SHINE_ERR_ALIGNMENT: return "misaligned pointer";
        case SHINE_ERR_WORKSPACE: return "workspace missing or too small";
        case SHINE_ERR_UNSUPPORTED: return "unsupported combination";
        case SHINE_ERR_CUDA: return "CUDA error";
    }
    return "unknown status";
}

int shine_last_cuda_error(void) { return g_last_cuda_error; }

shine_status shine_partition(int64_t nseg, int64_t rows, int64_t t, int64_t w, int32_t band_major,
                             int32_t edge_weight4, int64_t* lo, int64_t* hi) {
    if (!lo || !hi || nseg < 1 || rows < 1 || t < 1 || w < 0 || w >= t || edge_weight4 < 1 || edge_weight4 > 64)
        return SHINE_ERR_INVALID_ARG;
    warp_work(band_major != 0, nseg, rows, t, w, *lo, *hi, edge_weight4);
    return SHINE_OK;
}

shine_status shine_wait_status(int* failed, int clear) {
    if (!failed) return SHINE_ERR_INVALID_ARG;
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_wait_flag, sizeof v);
    if (e != cudaSuccess) return cuda_status(e);
    *failed = v != 0;
    if (clear) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_wait_flag, &zero, sizeof zero);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return SHINE_OK;
}

shine_status shine_debug_bounds_status(int* instrumented, unsigned int* bits, int clear) {
    if (!instrumented || !bits) return SHINE_ERR_INVALID_ARG;
    *instrumented = SHINE_DEBUG_BOUNDS;
    *bits = 0;
    if constexpr (SHINE_DEBUG_BOUNDS) {
        unsigned int v = 0;
        cudaError_t e = cudaMemcpyFromSymbol(&v, g_bounds_flag, sizeof v);
        if (e != cudaSuccess) return cuda_status(e);
        *bits = v;
        if (clear) {
            const unsigned int zero = 0;
            e = cudaMemcpyToSymbol(g_bounds_flag, &zero, sizeof zero);
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    return SHINE_OK;
}

shine_status shine_workspace_status(const void* workspace, int* failed) {
    if (!workspace || !failed) return SHINE_ERR_INVALID_ARG;
    unsigned int v = 0;
    cudaError_t e = cudaMemcpy(&v, workspace, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    *failed = v != 0;
    return SHINE_OK;
}

shine_status shine_output_shape(int64_t H, int64_t W, shine_border border, int64_t* H_out, int64_t* W_out) {
    if (!H_out || !W_out) return SHINE_ERR_INVALID_ARG;
    shine_status st = check_shape(H, W, border);
    if (st != SHINE_OK) return st;
    *H_out = border == SHINE_VALID ? H - 4 : H;
    *W_out = border == SHINE_VALID ? W - 4 : W;
    return SHINE_OK;
}

shine_status shine_pipeline_fwd(const void* img, int64_t H, int64_t W, int64_t img_pitch, shine_dtype dt,
                                shine_border border, const float* kappa, const float* wx, const float* wy,
                                void* out, int64_t out_pitch, shine_dtype out_dt, void* stream) {
    SHINE_ENTRY("shine_pipeline_fwd");
    if (!img || !kappa || !wx || !wy || !out) return SHINE_ERR_INVALID_ARG;
    if (!dtype_ok(dt) || !dtype_ok(out_dt)) return SHINE_ERR_INVALID_ARG;
    if (!(out_dt == dt || out_dt == SHINE_F32)) return SHINE_ERR_UNSUPPORTED;
    shine_status st = check_shape(H, W, border);
    if (st != SHINE_OK) return st;
    const int64_t Ho = border == SHINE_VALID ? H - 4 : H, Wo = border == SHINE_VALID ? W - 4 : W;
    if (img_pitch < 3 * W || out_pitch < Wo) return SHINE_ERR_INVALID_ARG;
    (void)Ho;
    const size_t si = dtype_size(dt), so = dtype_size(out_dt);
    if (!aligned_to(img, si) || !aligned_to(out, so) || !aligned_to(kappa, 4) || !aligned_to(wx, 4) ||
        !aligned_to(wy, 4))
        return SHINE_ERR_ALIGNMENT;
    FwdArgs a;
    static_cast<Geometry&>(a) = fwd_geometry(H, W, border);
    a.img = img; a.img_pitch = img_pitch; a.out = out; a.out_pitch = out_pitch;
    a.kappa = kappa; a.wx = wx; a.wy = wy;
    const size_t chunk = si == 4 ? 16 : 8;
    a.aligned = aligned_to(img, chunk) && ((size_t)img_pitch * si) % chunk == 0;
    a.out_vec = border == SHINE_CLAMP && aligned_to(out, 16) && ((size_t)out_pitch * so) % 16 == 0;
    a.tma = SHINE_FWD_TMA && aligned_to(img, 16) && ((size_t)img_pitch * si) % 16 == 0;
    a.err = wait_flag();
    return cuda_status(launch_harris_fwd(a, dt, out_dt, static_cast<cudaStream_t>(stream)));
}

shine_status shine_corners(const void* img, int64_t H, int64_t W, int64_t img_pitch, shine_dtype dt,
                           shine_border border, const float* kappa, const float* wx, const float* wy, float threshold,
                           uint8_t* mask, int64_t mask_pitch, void* out, int64_t out_pitch, shine_dtype out_dt,
                           void* stream) {
    SHINE_ENTRY("shine_corners");
    if (!img || !kappa || !wx || !wy || !mask) return SHINE_ERR_INVALID_ARG;
    if (!dtype_ok(dt) || (out && !dtype_ok(out_dt))) return SHINE_ERR_INVALID_ARG;
    if (out && !(out_dt == dt || out_dt == SHINE_F32)) return SHINE_ERR_UNSUPPORTED;
    shine_status st = check_shape(H, W, border);
    if (st != SHINE_OK) return st;
    const int64_t Wo = border == SHINE_VALID ? W - 4 : W;
    if (img_pitch < 3 * W || mask_pitch < Wo || (out && out_pitch < Wo)) return SHINE_ERR_INVALID_ARG;
    const size_t si = dtype_size(dt), so = out ? dtype_size(out_dt) : si;
    if (!aligned_to(img, si) || (out && !aligned_to(out, so)) || !aligned_to(kappa, 4) || !aligned_to(wx, 4) ||
        !aligned_to(wy, 4))
        return SHINE_ERR_ALIGNMENT;
    CornerArgs c;
    FwdArgs& a = c.f;
    static_cast<Geometry&>(a) = fwd_geometry(H, W, border);
    a.img = img; a.img_pitch = img_pitch; a.out = out; a.out_pitch = out ? out_pitch : 0;
    a.kappa = kappa; a.wx = wx; a.wy = wy;
    const size_t chunk = si == 4 ? 16 : 8;
    a.aligned = aligned_to(img, chunk) && ((size_t)img_pitch * si) % chunk == 0;
    a.out_vec = out && border == SHINE_CLAMP && aligned_to(out, 16) && ((size_t)out_pitch * so) % 16 == 0;
    a.tma = SHINE_FWD_TMA && aligned_to(img, 16) && ((size_t)img_pitch * si) % 16 == 0;
    a.err = wait_flag();
    c.mask = mask;
    c.mask_pitch = mask_pitch;
    c.threshold = threshold;
    c.mask_vec = border == SHINE_CLAMP && aligned_to(mask, 8) && mask_pitch % 8 == 0;
    return cuda_status(launch_harris_corners(c, dt, out ? out_dt : dt, static_cast<cudaStream_t>(stream)));
}

shine_status shine_pipeline_bwd_workspace(int64_t H, int64_t W, shine_border border, size_t* bytes) {
    if (!bytes) return SHINE_ERR_INVALID_ARG;
    shine_status st = check_shape(H, W, border);
    if (st != SHINE_OK) return st;
    Geometry g = bwd_geometry(H, W, border);
    *bytes = kWorkspaceHeader + (size_t)kParamSlots * (size_t)bwd_max_warps(g) * sizeof(double);
    return SHINE_OK;
}

}  // extern "C"

namespace shine {

shine_status run_bwd(const void* img, int64_t H, int64_t W, int64_t img_pitch, shine_dtype dt,
                     shine_border border, const float* kappa, const float* wx, const float* wy,
                     const void* grad_out, int64_t gout_pitch, shine_dtype gout_dt, void* out,
                     int64_t out_pitch, void* grad_img, int64_t gimg_pitch, float* grad_kappa,
                     float* grad_wx, float* grad_wy, void* workspace, size_t ws_bytes, void* stream,
                     unsigned int* err_word) {
    if (!img || !kappa || !wx || !wy || !grad_out) return SHINE_ERR_INVALID_ARG;
    if (!dtype_ok(dt) || !dtype_ok(gout_dt)) return SHINE_ERR_INVALID_ARG;
    if (!(gout_dt == dt || gout_dt == SHINE_F32)) return SHINE_ERR_UNSUPPORTED;
    shine_status st = check_shape(H, W, border);
    if (st != SHINE_OK) return st;
    const int64_t Ho = border == SHINE_VALID ? H - 4 : H, Wo = border == SHINE_VALID ? W - 4 : W;
    if (img_pitch < 3 * W || gout_pitch < Wo || (grad_img && gimg_pitch < 3 * W) || (out && out_pitch < Wo))
        return SHINE_ERR_INVALID_ARG;
    const size_t si = dtype_size(dt), sg = dtype_size(gout_dt);
    if (!aligned_to(img, si) || !aligned_to(grad_out, sg) || (grad_img && !aligned_to(grad_img, si)) ||
        (out && !aligned_to(out, si)) || !aligned_to(kappa, 4) || !aligned_to(wx, 4) || !aligned_to(wy, 4) ||
        (grad_kappa && !aligned_to(grad_kappa, 4)) || (grad_wx && !aligned_to(grad_wx, 4)) ||
        (grad_wy && !aligned_to(grad_wy, 4)))
        return SHINE_ERR_ALIGNMENT;
    BwdArgs a;
    static_cast<Geometry&>(a) = bwd_geometry(H, W, border);
    const int64_t max_warps = bwd_max_warps(a);
    const size_t need = kWorkspaceHeader + (size_t)kParamSlots * (size_t)max_warps * sizeof(double);
    if (!workspace || ws_bytes < need) return SHINE_ERR_WORKSPACE;
    if (!aligned_to(workspace, 16)) return SHINE_ERR_ALIGNMENT;
    if (!out && !grad_img && !grad_kappa && !grad_wx && !grad_wy) return SHINE_OK;
    a.img = img; a.img_pitch = img_pitch;
    a.gout = grad_out; a.gout_pitch = gout_pitch; a.gho = (int)Ho; a.gwo = (int)Wo;
    a.gimg = grad_img; a.gimg_pitch = gimg_pitch;
    a.kappa = kappa; a.wx = wx; a.wy = wy;
    // bounded-wait failures go to the workspace header (cleared below), or to err_word when given
    a.err = err_word != nullptr ? err_word : static_cast<unsigned int*>(workspace);
    a.partials = reinterpret_cast<double*>(static_cast<char*>(workspace) + kWorkspaceHeader);
    a.pstride = 0;
    a.poffset = 0;
    const size_t chunk = si == 4 ? 16 : 8;
    a.aligned = aligned_to(img, chunk) && ((size_t)img_pitch * si) % chunk == 0;
    a.g_aligned = border == SHINE_CLAMP && aligned_to(grad_out, 4 * sg) && ((size_t)gout_pitch * sg) % (4 * sg) == 0;
    a.gimg_vec = grad_img && aligned_to(grad_img, chunk) && ((size_t)gimg_pitch * si) % chunk == 0;
    a.tma = SHINE_BWD_TMA && aligned_to(img, 16) && ((size_t)img_pitch * si) % 16 == 0 &&
            aligned_to(grad_out, 16) && ((size_t)gout_pitch * sg) % 16 == 0 && border == SHINE_CLAMP;
    a.rout = out; a.rout_pitch = out_pitch;
    a.rout_vec = out && border == SHINE_CLAMP && aligned_to(out, 4 * si) && ((size_t)out_pitch * si) % (4 * si) == 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (err_word == nullptr) {
        st = cuda_status(cudaMemsetAsync(a.err, 0, sizeof(unsigned int), s));
        if (st != SHINE_OK) return st;
    }
    int used = 0;
    st = cuda_status(launch_harris_bwd(a, dt, gout_dt, (int)max_warps, s, &used));
    if (st != SHINE_OK) return st;
    if (grad_kappa || grad_wx || grad_wy)
        st = cuda_status(launch_finalize_params(a.partials, used, grad_kappa, grad_wx, grad_wy, s));
    return st;
}

}  // namespace shine

extern "C" {

shine_status shine_pipeline_bwd(const void* img, int64_t H, int64_t W, int64_t img_pitch, shine_dtype dt,
                                shine_border border, const float* kappa, const float* wx, const float* wy,
                                const void* grad_out, int64_t gout_pitch, shine_dtype gout_dt, void* grad_img,
                                int64_t gimg_pitch, float* grad_kappa, float* grad_wx, float* grad_wy,
                                void* workspace, size_t ws_bytes, void* stream) {
    SHINE_ENTRY("shine_pipeline_bwd");
    return run_bwd(img, H, W, img_pitch, dt, border, kappa, wx, wy, grad_out, gout_pitch, gout_dt, nullptr, 0,
                   grad_img, gimg_pitch, grad_kappa, grad_wx, grad_wy, workspace, ws_bytes, stream, nullptr);
}

shine_status shine_pipeline_fwd_bwd(const void* img, int64_t H, int64_t W, int64_t img_pitch, shine_dtype dt,
                                    shine_border border, const float* kappa, const float* wx, const float* wy,
                                    const void* grad_out, int64_t gout_pitch, void* out, int64_t out_pitch,
                                    void* grad_img, int64_t gimg_pitch, float* grad_kappa, float* grad_wx,
                                    float* grad_wy, void* workspace, size_t ws_bytes, void* stream) {
    SHINE_ENTRY("shine_pipeline_fwd_bwd");
    return run_bwd(img, H, W, img_pitch, dt, border, kappa, wx, wy, grad_out, gout_pitch, dt, out, out_pitch,
                   grad_img, gimg_pitch, grad_kappa, grad_wx, grad_wy, workspace, ws_bytes, stream, nullptr);
}

}  // extern "C"
