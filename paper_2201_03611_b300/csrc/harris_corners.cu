// Corner detection: the forward pass (A1-A5) followed, in the same kernel, by a threshold and a
// 3x3 non-maximum suppression of R -- the downstream step of the corner-detection image
// pipeline, one more map over slide2D(3,1) windows fused after A5 (map fusion, Sec. 4.2). R
// only reaches global memory when the caller asks for it; the mask is one byte per output pixel.
//
// A warp streams its strip exactly as the forward does, over one extra R row above and below
// the rows it owns (clipped to the output region). Each R row is widened to 6 columns (its 4
// and one from each neighbouring lane: lanes 0 and 31 hold valid R at the columns next to the
// segment) and reduced to horizontal 3-maxima; running maxima of the last rows then decide row
// y-1 when row y arrives.
#include <algorithm>
#include <type_traits>

#include "harris_fwd_strip.cuh"
#include "shine_host.h"

namespace shine {

namespace {

// float32 register cap: the bulk-staged variant fits 128 registers (16 warps per SM) without
// spilling; the others keep 168 (12 warps), where they do not spill either.
template <typename TI, typename TO, int D, bool ALIGNED, bool TMA>
__global__ void __launch_bounds__(kFwdThreads, sizeof(TI) == 4 ? (TMA ? 4 : 3) : SHINE_FWD_MIN_BLOCKS)
    harris_corners_kernel(CornerArgs c) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const FwdArgs& a = c.f;
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
    const bool producer = lane >= 1 && lane <= 30;
    const float kNegInf = __int_as_float(0xff800000);
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
        const int y0 = a.ylo + r0, y1 = a.ylo + r1;                      // rows this warp decides
        const int ys = y0 - 1 > a.ylo ? y0 - 1 : a.ylo;                  // R rows it computes
        const int ye = y1 + 1 < a.yhi ? y1 + 1 : a.yhi;
        // Columns of the lane inside the output region (others read as -inf: no neighbour).
        bool cin[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) cin[j] = x + j >= a.xlo && x + j < a.xhi;
        // Push form of the 3x3 maximum (max is exact, so any grouping gives the same value):
        // each R row arrives as its horizontal 3-maxima hm; the decision of row y-1 needs
        // max(hm(y-2), hm(y-1), hm(y)) and R(y-1) itself.
        float ha[4], hb[4], cen[4];  // max(hm(y-2), hm(y-1)); hm(y-1); R(y-1)
#pragma unroll
        for (int j = 0; j < 4; ++j) ha[j] = hb[j] = cen[j] = kNegInf;

        // Decide row y: corner where the centre exceeds the threshold and equals the maximum of
        // its 3x3 window (that is, is >= each of its 8 neighbours). E: an edge segment (or the
        // VALID region), where some of the lane's columns may lie outside the output region;
        // interior segments know at compile time that all four are inside.
        auto emit = [&](auto edge_tag, int y, const float nb[4]) {
            constexpr bool E = decltype(edge_tag)::value;
            uint32_t bits = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t on = (cen[j] > c.threshold && cen[j] >= nb[j]) ? 1u : 0u;
                bits |= on << (8 * j);
            }
            if (!producer) return;
            uint8_t* mrow = c.mask + (int64_t)(y - a.oy) * c.mask_pitch;
            if (!E && c.mask_vec) {
                *reinterpret_cast<uint32_t*>(mrow + (x - a.ox)) = bits;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (!E || cin[j]) mrow[x + j - a.ox] = (uint8_t)((bits >> (8 * j)) & 0xffu);
            }
        };
        auto store = [&](auto edge_tag, int y, const float R[4]) {
            constexpr bool E = decltype(edge_tag)::value;
            if (a.out != nullptr && producer && y >= y0 && y < y1) {
                TO* orow = static_cast<TO*>(a.out) + (int64_t)(y - a.oy) * a.out_pitch;
                if (!E && a.out_vec) {
                    store4(orow + x, R);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (!E || cin[j]) orow[x + j - a.ox] = Conv<TO>::st(R[j]);
                }
            }
            float r[4], r6[6], hm[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) r[j] = (!E || cin[j]) ? R[j] : kNegInf;
            make_row6(r, r6);
#pragma unroll
            for (int j = 0; j < 4; ++j) hm[j] = fmaxf(fmaxf(r6[j], r6[j + 1]), r6[j + 2]);
            if (y - 1 >= y0) {
                float nb[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) nb[j] = fmaxf(ha[j], hm[j]);
                emit(edge_tag, y - 1, nb);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ha[j] = fmaxf(hb[j], hm[j]);
                hb[j] = hm[j];
                cen[j] = r[j];
            }
        };
        const std::integral_constant<bool, true> on_edge{};
        const std::integral_constant<bool, false> inside{};
        if (edge) {
            fwd_rows<TI, kFwdEdgeStages, true, ALIGNED>(a, P, x, ys, ye,
                                                        [&](int y, const float R[4]) { store(on_edge, y, R); });
        } else if constexpr (TMA) {
            fwd_rows_bulk<TI, NS>(a, P, lane, x, ys, ye, ring, bulk,
                                  [&](int y, const float R[4]) { store(inside, y, R); });
        } else {
            fwd_rows<TI, D, false, ALIGNED>(a, P, x, ys, ye, [&](int y, const float R[4]) { store(inside, y, R); });
        }
        if (ye == y1 && !bulk.failed) {  // the region's last row: nothing below it
            if (edge) emit(on_edge, y1 - 1, ha);
            else emit(inside, y1 - 1, ha);
        }
        lo += r1 - r0;
    }
    if (bulk.failed && lane == 0 && a.err != nullptr) atomicOr(a.err, 1u);
}

template <typename TI, typename TO>
cudaError_t launch_corners_t(CornerArgs c, cudaStream_t s) {
    constexpr int D = kFwdStages;
    constexpr int NS = kFwdBulkStages;
    FwdArgs& a = c.f;
    const bool tma = a.tma && a.aligned && (a.out == nullptr || a.out_vec) && c.mask_vec;
    const size_t smem = tma ? (size_t)kFwdThreads * NS * 12 * sizeof(TI) + (kFwdThreads / 32) * NS * 8 : 0;
    auto kern = tma ? harris_corners_kernel<TI, TO, D, true, true>
                    : (a.aligned ? harris_corners_kernel<TI, TO, D, true, false>
                                 : harris_corners_kernel<TI, TO, D, false, false>);
    const int64_t units = (int64_t)(a.yhi - a.ylo) * a.nseg;
    if (units <= 0) return cudaSuccess;
    if (tma) {
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
