// Corner detection: the forward pass (A1-A5) followed, in the same kernel, by a threshold and a
// 3x3 non-maximum suppression of R -- the downstream step of the corner-detection image
// pipeline, one more map over slide2D(3,1) windows fused after A5 (map fusion, Sec. 4.2). R
// only reaches global memory when the caller asks for it; the mask is one byte per output pixel.
//
// A warp streams its strip exactly as the forward does (eight columns per lane, the row sources
// of harris_fwd_wide.cuh), over one extra R row above and below the rows it owns (clipped to the
// output region). Each R row is widened to 10 columns (its 8 and one from each neighbouring
// lane: lanes 0 and 31 hold valid R at the columns next to the segment) and reduced to
// horizontal 3-maxima; a row is decided once the row below it has arrived.
#include <algorithm>
#include <type_traits>

#include "harris_fwd_wide.cuh"
#include "shine_host.h"

namespace shine {

namespace {

// Maximum that returns NaN when either operand is NaN (max.NaN): a NaN in a window makes its
// maximum NaN, and no value compares >= NaN, so a pixel with a NaN neighbour is no corner, as
// the definition (R >= each neighbour) has it.
__device__ __forceinline__ float max_nan(float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float max3_nan(float a, float b, float c) {
    float d;
    asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// out_vec: R rows allow 16-byte stores; mask_vec: mask rows allow 8-byte stores.
template <typename TI, typename TO, bool SMEM>
__global__ void __launch_bounds__(kFwdThreads, SHINE_WIDE_CORNERS_MIN_BLOCKS) harris_corners_kernel(CornerArgs c) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const FwdArgs& a = c.f;
    constexpr int NS = SHINE_WIDE_BULK_STAGES;
    constexpr uint32_t kSlotBytes = kWSegLoad * 3 * sizeof(TI);
    constexpr bool kBulk = sizeof(TI) == 4 ? SHINE_WIDE_BULK_F32 : SHINE_WIDE_BULK_16;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (kFwdThreads / 32) + warp;
    if (gw >= a.nwarps) return;  // whole warp
    WideBulkState bs;
    bs.seq = 0;
    bs.failed = false;
    uint32_t ring0 = 0;
    if constexpr (SMEM && kBulk) {
        ring0 = smem_u32(smem_raw) + (uint32_t)warp * NS * kSlotBytes;
        bs.bars = smem_u32(smem_raw) + (uint32_t)(kFwdThreads / 32) * NS * kSlotBytes + (uint32_t)warp * NS * 8;
        if (lane == 0)
            for (int i = 0; i < NS; ++i) mbar_init(bs.bars + 8 * i, 1);
        mbar_init_fence();
        __syncwarp();
    }
    Params P;
    load_params(P, a.wx, a.wy, a.kappa);
    const bool producer = lane >= 1 && lane <= 30;
    const float kNegInf = __int_as_float(0xff800000);
    TO* out = static_cast<TO*>(a.out);
    const int64_t rows = a.yhi - a.ylo;
    int64_t lo, hi;
    warp_work(SHINE_FWD_BAND_MAJOR, a.nseg, rows, a.nwarps, gw, lo, hi, SHINE_FWD_EDGE_WEIGHT4);
    while (lo < hi && !bs.failed) {
        const int seg = (int)(lo / rows);
        const int r0 = (int)(lo % rows);
        const int r1 = (int)(rows < r0 + (hi - lo) ? rows : r0 + (hi - lo));
        const int xb = a.x0 + seg * kWSegOut;
        const int x = xb - kWCols + kWCols * lane;
        const bool edge = (xb - kWCols < 0) || (xb + kWSegOut + kWCols > a.W) || a.valid;
        const int y0 = a.ylo + r0, y1 = a.ylo + r1;      // rows this warp decides
        const int ys = y0 - 1 > a.ylo ? y0 - 1 : a.ylo;  // R rows it computes
        const int ye = y1 + 1 < a.yhi ? y1 + 1 : a.yhi;
        // Row y-1 is a corner where R(y-1) exceeds the threshold and is >= every value of its 3x3
        // window, i.e. >= max(hm(y-2), hm(y-1)) (tested when row y-1 arrives, one bit per column
        // in cand) and >= hm(y) (tested when row y arrives); hm are horizontal 3-maxima that
        // propagate NaN. State: cand, hb = hm(y-1), cen = R(y-1).
        uint32_t cand = 0;
        float hb[8], cen[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) hb[j] = cen[j] = kNegInf;
        // a lane column inside the output region (others read as -inf: no neighbour)
        auto col_in = [&](int j) { return x + j >= a.xlo && x + j < a.xhi; };
        // decide row y (cand and cen describe it) against the horizontal maxima of the row below
        // (-inf at the region's last row)
        auto emit = [&](auto edge_tag, int y, const float* below) {
            constexpr bool E = decltype(edge_tag)::value;
            uint32_t b0 = 0, b1 = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool lo_on = ((cand >> j) & 1u) && (below == nullptr || cen[j] >= below[j]);
                const bool hi_on = ((cand >> (4 + j)) & 1u) && (below == nullptr || cen[4 + j] >= below[4 + j]);
                b0 |= (lo_on ? 1u : 0u) << (8 * j);
                b1 |= (hi_on ? 1u : 0u) << (8 * j);
            }
            if (!producer) return;
            SHINE_CHECK(a.dbg, y >= a.ylo && y < a.yhi, kDbgFwdStore);
            uint8_t* mrow = c.mask + (int64_t)(y - a.oy) * c.mask_pitch;
            if (!E && c.mask_vec) {
                *reinterpret_cast<uint2*>(mrow + (x - a.ox)) = make_uint2(b0, b1);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (!E || col_in(j)) mrow[x + j - a.ox] = (uint8_t)(((j < 4 ? b0 : b1) >> (8 * (j & 3))) & 0xffu);
            }
        };
        auto store = [&](auto edge_tag, int y, const float R[8]) {
            constexpr bool E = decltype(edge_tag)::value;
            if (out != nullptr && producer && y >= y0 && y < y1) {
                TO* orow = out + (int64_t)(y - a.oy) * a.out_pitch;
                if (!E && a.out_vec) {
                    store8(orow + x, R);
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (!E || col_in(j)) orow[x + j - a.ox] = Conv<TO>::st(R[j]);
                }
            }
            float r[8], r10[10], hm[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] = (!E || col_in(j)) ? R[j] : kNegInf;
            widen10<false>(r, r10, x, 0);
#pragma unroll
            for (int j = 0; j < 8; ++j) hm[j] = max3_nan(r10[j], r10[j + 1], r10[j + 2]);
            if (y - 1 >= y0) emit(edge_tag, y - 1, hm);
            uint32_t nc = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                nc |= ((r[j] > c.threshold && r[j] >= max_nan(hb[j], hm[j])) ? 1u : 0u) << j;
                hb[j] = hm[j];
                cen[j] = r[j];
            }
            cand = nc;
        };
        const std::integral_constant<bool, true> on_edge{};
        const std::integral_constant<bool, false> inside{};
        auto st_edge = [&](int y, const float R[8]) { store(on_edge, y, R); };
        auto st_in = [&](int y, const float R[8]) { store(inside, y, R); };
        if constexpr (SMEM) {
            if constexpr (kBulk) {
                if (!edge) wide_rows_bulk<TI, NS>(a, P, lane, x, ys, ye, ring0, bs, st_in);
                else if constexpr (SHINE_WIDE_EDGE_LANES) wide_rows_edge<TI, NS>(a, P, lane, x, ys, ye, ring0, st_edge);
                else wide_rows_pf<TI, true>(a, P, lane, x, ys, ye, st_edge);
            } else {
                if (edge) wide_rows_pf<TI, true>(a, P, lane, x, ys, ye, st_edge);
                else wide_rows_pf<TI, false>(a, P, lane, x, ys, ye, st_in);
            }
        } else {
            if (edge) wide_rows_elem<TI, true>(a, P, x, ys, ye, st_edge);
            else wide_rows_elem<TI, false>(a, P, x, ys, ye, st_in);
        }
        if (ye == y1 && !bs.failed) {  // the region's last row: nothing below it
            if (edge) emit(on_edge, y1 - 1, static_cast<const float*>(nullptr));
            else emit(inside, y1 - 1, static_cast<const float*>(nullptr));
        }
        lo += r1 - r0;
    }
    if (bs.failed && lane == 0 && a.err != nullptr) atomicOr(a.err, 1u);
}

template <typename TI, typename TO>
cudaError_t launch_corners_t(CornerArgs c, cudaStream_t s) {
    constexpr int NS = SHINE_WIDE_BULK_STAGES;
    constexpr bool kBulk = sizeof(TI) == 4 ? SHINE_WIDE_BULK_F32 : SHINE_WIDE_BULK_16;
    FwdArgs& a = c.f;
    const bool smem_stage = a.tma;
    const size_t smem = smem_stage && kBulk ? (size_t)(kFwdThreads / 32) * NS * (kWSegLoad * 3 * sizeof(TI) + 8) : 0;
    auto kern = smem_stage ? harris_corners_kernel<TI, TO, true> : harris_corners_kernel<TI, TO, false>;
    // the wide layout: segments of kWSegOut output columns, segment 0 at the storage type's origin
    a.x0 = wide_origin<TI>();
    a.nseg = (a.xhi - a.x0 + kWSegOut - 1) / kWSegOut;
    const int64_t units = (int64_t)(a.yhi - a.ylo) * a.nseg;
    if (units <= 0) return cudaSuccess;
    if (smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFwdThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t t = (int64_t)per_sm * sm_count() * (kFwdThreads / 32);
    t = std::min<int64_t>(t, std::max<int64_t>(1, units / kFwdMinRows));
    a.nwarps = (int)t;
    const int64_t blocks = (t + kFwdThreads / 32 - 1) / (kFwdThreads / 32);
    kern<<<(unsigned)blocks, kFwdThreads, smem, s>>>(c);
    return cudaPeekAtLastError();
}

}  // namespace

cudaError_t launch_harris_corners(CornerArgs c, int dt, int out_dt, cudaStream_t s) {
#define SHINE_CORNERS_CASE(I, O, TI, TO) \
    if (dt == I && out_dt == O) return launch_corners_t<TI, TO>(c, s);
    SHINE_CORNERS_CASE(0, 0, float, float)
    SHINE_CORNERS_CASE(1, 1, __nv_bfloat16, __nv_bfloat16)
    SHINE_CORNERS_CASE(2, 2, __half, __half)
    SHINE_CORNERS_CASE(1, 0, __nv_bfloat16, float)
    SHINE_CORNERS_CASE(2, 0, __half, float)
#undef SHINE_CORNERS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace shine
