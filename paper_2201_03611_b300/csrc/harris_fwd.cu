// Fused forward kernel: A1 gray -> A2 Sobel -> A3 products -> A4 box sum -> A5 response,
// with only the response written to global memory (the paper's map-fusion and fuseReduceMap
// rules, Sec. 4.2, applied to the whole pipeline; toMem(Global) of the result, Sec. 5.3).
// One warp streams one (column segment, row band); see harris_fwd_strip.cuh.
#include <algorithm>

#include "harris_fwd_strip.cuh"

namespace shine {

namespace {

template <typename TI, typename TO, int D, bool ALIGNED, bool TMA>
__global__ void __launch_bounds__(kFwdThreads, SHINE_FWD_MIN_BLOCKS) harris_fwd_kernel(FwdArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int NS = kFwdBulkStages;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (kFwdThreads / 32) + warp;
    if (gw >= a.nwarps) return;  // whole warp
    FwdBulk bulk;
    bulk.seq = 0;
    bulk.failed = false;
    TI* ring = nullptr;
    if constexpr (TMA) {
        ring = reinterpret_cast<TI*>(smem_raw) + warp * NS * kLanes * 12 + lane * 12;
        uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kFwdThreads * NS * 12 * sizeof(TI)) + warp * NS;
        bulk.bars = smem_u32(bars);
        if (lane == 0)
            for (int i = 0; i < NS; ++i) mbar_init(bulk.bars + 8 * i, 1);
        mbar_init_fence();
        __syncwarp();
    }
    Params P;
    load_params(P, a.wx, a.wy, a.kappa);
    // This warp's share of the (segment, row) units, walked segment by segment.
    const int64_t rows = a.yhi - a.ylo;
    int64_t lo, hi;
    warp_work(SHINE_FWD_BAND_MAJOR, a.nseg, rows, a.nwarps, gw, lo, hi, SHINE_FWD_EDGE_WEIGHT4);
    while (lo < hi && !bulk.failed) {
        const int seg = (int)(lo / rows);
        const int r0 = (int)(lo % rows);
        const int r1 = (int)(rows < r0 + (hi - lo) ? rows : r0 + (hi - lo));
        const int xb = a.x0 + seg * kSegOut;
        const int x = xb - 4 + 4 * lane;
        const bool edge = (xb - 4 < 0) || (xb + kSegOut + 4 > a.W) || a.valid;
        if (edge) fwd_strip<TI, TO, kFwdEdgeStages, true, ALIGNED>(a, P, lane, x, a.ylo + r0, a.ylo + r1);
        else if constexpr (TMA) fwd_strip_bulk<TI, TO, NS>(a, P, lane, x, a.ylo + r0, a.ylo + r1, ring, bulk);
        else fwd_strip<TI, TO, D, false, ALIGNED>(a, P, lane, x, a.ylo + r0, a.ylo + r1);
        lo += r1 - r0;
    }
    if (bulk.failed && lane == 0 && a.err != nullptr) atomicOr(a.err, 1u);
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
    constexpr int D = kFwdStages;
    constexpr int NS = kFwdBulkStages;
    const bool tma = a.tma && a.aligned && a.out_vec;  // the bulk strips store R with vector stores
    const size_t smem = tma ? (size_t)kFwdThreads * NS * 12 * sizeof(TI) + (kFwdThreads / 32) * NS * 8 : 0;
    auto kern = tma ? harris_fwd_kernel<TI, TO, D, true, true>
                    : (a.aligned ? harris_fwd_kernel<TI, TO, D, true, false> : harris_fwd_kernel<TI, TO, D, false, false>);
    const int64_t units = (int64_t)(a.yhi - a.ylo) * a.nseg;
    if (units <= 0) return cudaSuccess;
    if (tma) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
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
