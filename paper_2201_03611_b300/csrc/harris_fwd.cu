// Fused forward kernel: A1 gray -> A2 Sobel -> A3 products -> A4 box sum -> A5 response,
// with only the response written to global memory (the paper's map-fusion and fuseReduceMap
// rules, Sec. 4.2, applied to the whole pipeline; toMem(Global) of the result, Sec. 5.3).
// One warp streams one (column segment, row band), eight columns per lane; see
// harris_fwd_wide.cuh.
#include <algorithm>
#include <type_traits>

#include "harris_fwd_wide.cuh"

namespace shine {

namespace {

// Stores of R: 16-byte stores on lanes whose 8 columns are all output columns of a row that
// allows them, else element by element.
template <typename TO>
__device__ __forceinline__ void store_row(const FwdArgs& a, TO* orow, int x, bool vec, const float R[8]) {
    if (vec && x >= a.xlo && x + kWCols <= a.xhi) {
        store8(orow + (x - a.ox), R);
    } else {
#pragma unroll
        for (int j = 0; j < kWCols; ++j) {
            const int c = x + j;
            if (c >= a.xlo && c < a.xhi) orow[c - a.ox] = Conv<TO>::st(R[j]);
        }
    }
}

// Stores of R on an interior segment (no output offset, every column an output column).
template <typename TO>
__device__ __forceinline__ void store_row_interior(const FwdArgs& a, TO* p, const float R[8]) {
    if (a.out_vec) {
        store8(p, R);
    } else {
#pragma unroll
        for (int j = 0; j < kWCols; ++j) p[j] = Conv<TO>::st(R[j]);
    }
}

// Forward strips: a row source of harris_fwd_wide.cuh per staging kind, with R stored by the
// producer lanes (element by element where a lane's columns leave the output region).
template <typename TI, typename TO, bool EDGE>
__device__ __forceinline__ void wide_strip_elem(const FwdArgs& a, const Params& P, int lane, int x, int y0, int y1) {
    TO* out = static_cast<TO*>(a.out);
    const bool producer = lane >= 1 && lane <= 30;
    wide_rows_elem<TI, EDGE>(a, P, x, y0, y1, [&](int y, const float R[8]) {
        if (producer) {
            SHINE_CHECK(a.dbg, y >= a.ylo && y < a.yhi, kDbgFwdStore);
            store_row(a, out + (int64_t)(y - a.oy) * a.out_pitch, x, a.out_vec, R);
        }
    });
}

template <typename TI, typename TO, bool EDGE>
__device__ __forceinline__ void wide_strip_pf(const FwdArgs& a, const Params& P, int lane, int x, int y0, int y1) {
    TO* out = static_cast<TO*>(a.out);
    const bool producer = lane >= 1 && lane <= 30;
    wide_rows_pf<TI, EDGE>(a, P, lane, x, y0, y1, [&](int y, const float R[8]) {
        if (producer) {
            SHINE_CHECK(a.dbg, y >= a.ylo && y < a.yhi, kDbgFwdStore);
            if constexpr (!EDGE) SHINE_CHECK(a.dbg, x >= a.xlo && x + kWCols <= a.xhi && a.ox == 0 && a.oy == 0, kDbgFwdStore);
            if constexpr (EDGE) store_row(a, out + (int64_t)(y - a.oy) * a.out_pitch, x, a.out_vec, R);
            else store_row_interior(a, out + (int64_t)y * a.out_pitch + x, R);
        }
    });
}

template <typename TI, typename TO, int NS>
__device__ __forceinline__ void wide_strip_edge(const FwdArgs& a, const Params& P, int lane, int x, int y0, int y1,
                                                uint32_t ring0) {
    TO* out = static_cast<TO*>(a.out);
    const bool producer = lane >= 1 && lane <= 30;
    wide_rows_edge<TI, NS>(a, P, lane, x, y0, y1, ring0, [&](int y, const float R[8]) {
        if (producer) {
            SHINE_CHECK(a.dbg, y >= a.ylo && y < a.yhi, kDbgFwdStore);
            store_row(a, out + (int64_t)(y - a.oy) * a.out_pitch, x, a.out_vec, R);
        }
    });
}

// Interior segment staged by bulk copies (written out here rather than through wide_rows_bulk:
// the running output pointer set up after the copies are issued measured 1.5% faster).
template <typename TI, typename TO, int NS>
__device__ __forceinline__ void wide_strip_bulk(const FwdArgs& a, const Params& P, int lane, int x, int y0, int y1,
                                                uint32_t ring0, WideBulkState& bs) {
    const int H = a.H;
    const int n = (y1 == H ? y1 - y0 + 3 : y1 - y0 + 4);  // gray rows y0-2 .. min(y1+1, H)
    SHINE_CHECK(a.dbg, x - kWCols * lane >= 0 && x - kWCols * lane + kWSegLoad <= a.W, kDbgFwdStage);
    SHINE_CHECK(a.dbg, smem_in(ring0, NS * WideBulk<TI, NS>::kBytes), kDbgSmem);
    SHINE_CHECK(a.dbg, y0 >= a.ylo && y1 <= a.yhi && x >= a.xlo && x + kWCols <= a.xhi, kDbgFwdStore);
    WideBulk<TI, NS> src(bs, static_cast<const TI*>(a.img), a.img_pitch, x - kWCols * lane, ring0, lane, y0 - 2, n, H);
    TO* orow = static_cast<TO*>(a.out) + (int64_t)y0 * a.out_pitch + x;  // interior: no output offset
    const int64_t opitch = a.out_pitch;
    const bool producer = lane >= 1 && lane <= 30;
    auto take = [&](float g10[10]) {
        WideRaw<TI> r;
        src.take_raw(r);
        float c[8];
        gray8<TI>(r, c);
        widen10<false>(c, g10, x, 0);
    };
    auto store = [&](int, const float R[8]) {
        if (producer) store_row_interior(a, orow, R);
        orow += opitch;
    };
    wide_strip_core<false>(P, x, a.W, H, y0, y1, take, store, [&] { return !bs.failed; });
    src.finish();
}

// Staging by bulk copies into a shared-memory ring (interior segments) or in registers with L2
// prefetch, per storage type; chosen by measurement.
template <typename TI> constexpr bool wide_bulk() { return sizeof(TI) == 4 ? SHINE_WIDE_BULK_F32 : SHINE_WIDE_BULK_16; }

// ALIGNED: the image rows are 16-byte aligned: interior segments are staged by bulk copies
// (wide_bulk) or in registers with L2 prefetch, edge segments in registers with L2 prefetch;
// otherwise every lane loads its pixels element by element.
template <typename TI, typename TO, bool SMEM>
__global__ void __launch_bounds__(kFwdThreads, SHINE_WIDE_MIN_BLOCKS) harris_fwd_kernel(FwdArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int NS = SHINE_WIDE_BULK_STAGES;
    constexpr uint32_t kSlotBytes = kWSegLoad * 3 * sizeof(TI);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (kFwdThreads / 32) + warp;
    if (gw >= a.nwarps) return;  // whole warp
    WideBulkState bs;
    bs.seq = 0;
    bs.failed = false;
    uint32_t ring0 = 0;
    if constexpr (SMEM && wide_bulk<TI>()) {
        ring0 = smem_u32(smem_raw) + (uint32_t)warp * NS * kSlotBytes;
        bs.bars = smem_u32(smem_raw) + (uint32_t)(kFwdThreads / 32) * NS * kSlotBytes + (uint32_t)warp * NS * 8;
        if (lane == 0)
            for (int i = 0; i < NS; ++i) mbar_init(bs.bars + 8 * i, 1);
        mbar_init_fence();
        __syncwarp();
    }
    Params P;
    load_params(P, a.wx, a.wy, a.kappa);
    // This warp's share of the (segment, row) units, walked segment by segment.
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
        if constexpr (SMEM) {
            if constexpr (wide_bulk<TI>()) {
                if (!edge) wide_strip_bulk<TI, TO, NS>(a, P, lane, x, a.ylo + r0, a.ylo + r1, ring0, bs);
                else if constexpr (SHINE_WIDE_EDGE_LANES) wide_strip_edge<TI, TO, NS>(a, P, lane, x, a.ylo + r0, a.ylo + r1, ring0);
                else wide_strip_pf<TI, TO, true>(a, P, lane, x, a.ylo + r0, a.ylo + r1);
            } else {
                if (edge) wide_strip_pf<TI, TO, true>(a, P, lane, x, a.ylo + r0, a.ylo + r1);
                else wide_strip_pf<TI, TO, false>(a, P, lane, x, a.ylo + r0, a.ylo + r1);
            }
        } else {
            if (edge) wide_strip_elem<TI, TO, true>(a, P, lane, x, a.ylo + r0, a.ylo + r1);
            else wide_strip_elem<TI, TO, false>(a, P, lane, x, a.ylo + r0, a.ylo + r1);
        }
        lo += r1 - r0;
    }
    if (bs.failed && lane == 0 && a.err != nullptr) atomicOr(a.err, 1u);
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
    constexpr int NS = SHINE_WIDE_BULK_STAGES;
    // shared-memory staging needs 16-byte aligned image rows (bulk copies, 16-byte cp.async)
    const bool smem_stage = a.tma;
    const size_t smem = smem_stage && wide_bulk<TI>() ? (size_t)(kFwdThreads / 32) * NS * (kWSegLoad * 3 * sizeof(TI) + 8) : 0;
    auto kern = smem_stage ? harris_fwd_kernel<TI, TO, true> : harris_fwd_kernel<TI, TO, false>;
    // the wide layout: segments of kWSegOut output columns, segment 0 at the storage type's origin
    a.x0 = wide_origin<TI>();
    a.nseg = (a.xhi - a.x0 + kWSegOut - 1) / kWSegOut;
    const int64_t units = (int64_t)(a.yhi - a.ylo) * a.nseg;
    if (units <= 0) return cudaSuccess;
    if (smem > 0) {
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
