// Fused forward kernel: A1 gray -> A2 Sobel -> A3 products -> A4 box sum -> A5 response,
// with only the response written to global memory (the paper's map-fusion and fuseReduceMap
// rules, Sec. 4.2, applied to the whole pipeline; toMem(Global) of the result, Sec. 5.3).
// One warp streams one (column segment, row band); see harris_fwd_strip.cuh.
#include <algorithm>

#include "harris_fwd_strip.cuh"

namespace shine {

namespace {

template <typename TI, typename TO, int NS, bool ALIGNED>
__global__ void __launch_bounds__(kFwdThreads, SHINE_FWD_MIN_BLOCKS) harris_fwd_kernel(FwdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (kFwdThreads / 32) + warp;
    if (gw >= a.nwarps) return;  // whole warp
    TI* ring = reinterpret_cast<TI*>(smem_raw) + warp * NS * kLanes * 12 + lane * 12;
    Params P;
    load_params(P, a.wx, a.wy, a.kappa);
    // This warp's equal share of the (segment, row) units, walked segment by segment.
    const int64_t rows = a.yhi - a.ylo;
    int64_t lo, hi;
    warp_work(SHINE_FWD_BAND_MAJOR, a.nseg, rows, a.nwarps, gw, lo, hi);
    while (lo < hi) {
        const int seg = (int)(lo / rows);
        const int r0 = (int)(lo % rows);
        const int r1 = (int)(rows < r0 + (hi - lo) ? rows : r0 + (hi - lo));
        const int xb = a.x0 + seg * kSegOut;
        const int x = xb - 4 + 4 * lane;
        const bool edge = (xb - 4 < 0) || (xb + kSegOut + 4 > a.W) || a.valid;
        if (edge) fwd_strip<TI, TO, NS, true, ALIGNED>(a, P, lane, x, a.ylo + r0, a.ylo + r1, ring);
        else fwd_strip<TI, TO, NS, false, ALIGNED>(a, P, lane, x, a.ylo + r0, a.ylo + r1, ring);
        lo += r1 - r0;
    }
}

template <typename K>
int resident_warps(K kernel, int threads, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    return per_sm * sms * (threads / 32);
}

template <typename TI, typename TO>
cudaError_t launch_fwd_t(FwdArgs a, cudaStream_t s) {
    constexpr int NS = kFwdStages;
    const size_t smem = (size_t)kFwdThreads * NS * 12 * sizeof(TI);
    auto kern = a.aligned ? harris_fwd_kernel<TI, TO, NS, true> : harris_fwd_kernel<TI, TO, NS, false>;
    const int64_t units = (int64_t)(a.yhi - a.ylo) * a.nseg;
    if (units <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t t = resident_warps(kern, kFwdThreads, smem);
    t = std::min<int64_t>(t, std::max<int64_t>(1, units / kFwdMinRows));
    a.nwarps = (int)t;
    const int64_t blocks = (t + kFwdThreads / 32 - 1) / (kFwdThreads / 32);
    kern<<<(unsigned)blocks, kFwdThreads, smem, s>>>(a);
    return cudaPeekAtLastError();
}

}  // namespace

cudaError_t launch_harris_fwd(FwdArgs a, int dt, int out_dt, cudaStream_t s) {
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
