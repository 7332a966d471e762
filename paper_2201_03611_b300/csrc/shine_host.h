// Host-side helpers shared by the entry points (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "harris_kernels.h"
#include "shine.h"

namespace shine {

constexpr int64_t kMaxDim = int64_t(1) << 30;

shine_status cuda_status(cudaError_t e);
size_t dtype_size(int dt);
bool dtype_ok(int dt);
bool border_ok(int b);
int sm_count();
// Device address of the library's bounded-wait failure flag on the current device (or null).
unsigned int* wait_flag();
// Debug builds: device address of the index-check violation word on the current device; null in
// release builds.
unsigned int* bounds_flag();
shine_status check_shape(int64_t H, int64_t W, int border);
bool aligned_to(const void* p, size_t a);
void fill_geometry(Geometry& g, int64_t H, int64_t W, int border, bool full_image, int band_rows);
Geometry fwd_geometry(int64_t H, int64_t W, int border);
Geometry bwd_geometry(int64_t H, int64_t W, int border);
// Upper bound of the warps a backward launch uses (its partials need kParamSlots doubles each).
int64_t bwd_max_warps(const Geometry& g);
// The backward pass behind shine_pipeline_bwd / shine_pipeline_fwd_bwd (out: the fused pass's R,
// nullable). A bounded wait that gives up sets the workspace's header word, which this call
// clears first; when err_word is given it sets that word instead (nothing is cleared), and the
// workspace header is left unused.
shine_status run_bwd(const void* img, int64_t H, int64_t W, int64_t img_pitch, shine_dtype dt,
                     shine_border border, const float* kappa, const float* wx, const float* wy,
                     const void* grad_out, int64_t gout_pitch, shine_dtype gout_dt, void* out,
                     int64_t out_pitch, void* grad_img, int64_t gimg_pitch, float* grad_kappa,
                     float* grad_wx, float* grad_wy, void* workspace, size_t ws_bytes, void* stream,
                     unsigned int* err_word);

}  // namespace shine
