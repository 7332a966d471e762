// Fused forward kernel: A1 gray -> A2 Sobel -> A3 products -> A4 box sum -> A5 response,
// with only the response written to global memory (the paper's map-fusion and fuseReduceMap
// rules, Sec. 4.2, applied to the whole pipeline; toMem(Global) of the result, Sec. 5.3).
// One warp streams one (column segment, row band); see harris_fwd_strip.cuh.
#include "harris_fwd_strip.cuh"

namespace shine {

namespace {

template <typename TI, typename TO, int NS, bool ALIGNED>
__global__ void __launch_bounds__(kFwdThreads) harris_fwd_kernel(FwdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (kFwdThreads / 32) + warp;
    const int seg = gw % a.nseg;
    const int band = gw / a.nseg;
    if (band >= a.nband) return;  // whole warp
    const int xb = a.x0 + seg * kSegOut;
    const int x = xb - 4 + 4 * lane;
    const int y0 = a.ylo + band * a.band_rows;
    const int y1 = min(y0 + a.band_rows, a.yhi);
    TI* ring = reinterpret_cast<TI*>(smem_raw) + (warp * 32 + lane) * NS * 12;
    Params P;
    load_params(P, a.wx, a.wy, a.kappa);
    const bool edge = (xb - 4 < 0) || (xb + kSegOut + 4 > a.W) || a.valid;
    if (edge) fwd_strip<TI, TO, NS, true, ALIGNED>(a, P, lane, x, y0, y1, ring);
    else fwd_strip<TI, TO, NS, false, ALIGNED>(a, P, lane, x, y0, y1, ring);
}

template <typename TI, typename TO>
cudaError_t launch_fwd_t(const FwdArgs& a, cudaStream_t s) {
    constexpr int NS = kFwdStages;
    const int64_t warps = (int64_t)a.nseg * a.nband;
    const int64_t blocks = (warps + kFwdThreads / 32 - 1) / (kFwdThreads / 32);
    const size_t smem = (size_t)kFwdThreads * NS * 12 * sizeof(TI);
    if (blocks <= 0) return cudaSuccess;
    if (a.aligned) {
        harris_fwd_kernel<TI, TO, NS, true><<<(unsigned)blocks, kFwdThreads, smem, s>>>(a);
    } else {
        harris_fwd_kernel<TI, TO, NS, false><<<(unsigned)blocks, kFwdThreads, smem, s>>>(a);
    }
    return cudaPeekAtLastError();
}

}  // namespace

cudaError_t launch_harris_fwd(const FwdArgs& a, int dt, int out_dt, cudaStream_t s) {
#define SHINE_FWD_CASE(I, O, TI, TO) \
    if (dt == I && out_dt == O) return launch_fwd_t<TI, TO>(a, s);
    SHINE_FWD_CASE(0, 0, float, float)
    SHINE_FWD_CASE(1, 1, __nv_bfloat16, __nv_bfloat16)
    SHINE_FWD_CASE(2, 2, __half, __half)
    SHINE_FWD_CASE(1, 0, __nv_bfloat16, float)
    SHINE_FWD_CASE(2, 0, __half, float)
#undef SHINE_FWD_CASE
    return cudaErrorInvalidValue;
}

}  // namespace shine
