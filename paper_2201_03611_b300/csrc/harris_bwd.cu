// Fused adjoint kernel of the Harris pipeline: the vector-Jacobian product of
// L = sum(g * R) with respect to the image, kappa and the two 3x3 weight matrices.
//
// Reverse mode through the patterns of the forward pass, with each pattern replaced by its
// adjoint (map -> pointwise chain rule, reduce(+) -> broadcast, slide2D -> overlap-add,
// pad_clamp -> fold onto the clamped index, a shared parameter -> sum over every use):
//
//   B1  recompute G, Ix, Iy and S (nothing of the forward pass is stored)
//   B2  gS = (g (Syy - 2 kappa T), -2 g Sxy, g (Sxx - 2 kappa T)),  d kappa += -g T^2
//   B3  gP = adjoint of the clamped 3x3 box sum applied to gS. For the all-ones symmetric
//       window with clamp padding this adjoint equals the clamped box sum itself: on an axis
//       of length n, the number of taps d in {-1,0,1} with clamp(p+d) = q equals the number
//       with clamp(q+d) = p for every p, q.
//   B4  gIx = 2 Ix gPxx + Iy gPxy,  gIy = Ix gPxy + 2 Iy gPyy
//   B5  gG = transposed 3x3 stencil of (gIx, gIy) with Wx, Wy on the clamp-padded domain,
//       folded back: the padded row/column -1 is added to row/column 0, and H (W) to H-1
//       (W-1);  d W[a][b] += gI(p) * G(clamp(p + (a-1, b-1)))
//   B6  d img[c] = coef_c * gG
//
// A warp streams one (column segment, row band): per step it stages image row r and
// cotangent row r-2, and writes d img row r-4 (the dependency reaches 4 rows and 4 columns:
// one per stencil, forward and adjoint). Lanes 0 and 31 supply exactly the 4-column halo.
// Parameter cotangents are accumulated per lane in float32, reduced per warp in float64 and
// summed in a fixed order by the finalize kernel, so every run gives the same bits.
#include <algorithm>
#include <cstdlib>

#include "harris_adj_wide.cuh"
#include "harris_bwd_strip.cuh"

namespace shine {

namespace {

template <typename TI, typename TG, int NS, bool ALIGNED, bool GALIGNED, bool WITH_R, bool TMA>
__global__ void __launch_bounds__(kBwdThreads) harris_bwd_kernel(BwdArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (kBwdThreads / 32) + warp;
    if (gw >= a.nwarps) return;  // whole warp
    TI* ring = reinterpret_cast<TI*>(smem_raw) + warp * NS * kLanes * 12 + lane * 12;
    unsigned char* gbase = smem_raw + (size_t)kBwdThreads * NS * 12 * sizeof(TI);
    TG* gring = reinterpret_cast<TG*>(gbase) + warp * NS * kLanes * 4 + lane * 4;
    BulkState bulk;
    bulk.seq = 0;
    bulk.failed = false;
    if constexpr (TMA) {
        uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + (size_t)kBwdThreads * NS * 4 * sizeof(TG)) + warp * NS;
        bulk.bars = smem_u32(bars);
        if (lane == 0)
            for (int i = 0; i < NS; ++i) mbar_init(bulk.bars + 8 * i, 1);
        mbar_init_fence();
        __syncwarp();
    }
    Params P;
    load_params(P, a.wx, a.wy, a.kappa);
    float acc[kParamSlots];
#pragma unroll
    for (int i = 0; i < kParamSlots; ++i) acc[i] = 0.0f;
    TI* rout = static_cast<TI*>(a.rout);
    // This warp's share of the (segment, row) units, walked segment by segment.
    const int64_t rows = a.yhi - a.ylo;
    int64_t lo, hi;
    warp_work(SHINE_BWD_BAND_MAJOR, a.nseg, rows, a.nwarps, gw, lo, hi, SHINE_BWD_EDGE_WEIGHT4);
    while (lo < hi && !bulk.failed) {
        const int seg = (int)(lo / rows);
        const int r0 = (int)(lo % rows);
        const int r1 = (int)(rows < r0 + (hi - lo) ? rows : r0 + (hi - lo));
        const int xb = a.x0 + seg * kSegOut;
        const int x = xb - 4 + 4 * lane;
        const bool edge = (xb - 4 < 0) || (xb + kSegOut + 4 > a.W);
        if (edge)
            bwd_strip<TI, TG, NS, true, ALIGNED, GALIGNED, WITH_R, false>(a, P, lane, x, a.ylo + r0, a.ylo + r1, ring,
                                                                          gring, acc, rout, a.rout_pitch, a.rout_vec);
        else
            bwd_strip<TI, TG, NS, false, ALIGNED, GALIGNED, WITH_R, TMA>(a, P, lane, x, a.ylo + r0, a.ylo + r1, ring,
                                                                         gring, acc, rout, a.rout_pitch, a.rout_vec,
                                                                         &bulk);
        lo += r1 - r0;
    }
    if (bulk.failed && lane == 0 && a.err != nullptr) atomicOr(a.err, 1u);
    // Warp partials in float64, lanes 0 and 31 excluded by selection (their values may be
    // unrelated to this warp's pixels).
    const bool producer = lane >= 1 && lane <= 30;
#pragma unroll
    for (int i = 0; i < kParamSlots; ++i) {
        double v = producer ? (double)acc[i] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
        if (lane == 0) a.partials[(int64_t)i * (a.pstride ? a.pstride : a.nwarps) + a.poffset + gw] = v;
    }
}

// The adjoint of a CLAMP image whose image and cotangent rows are 16-byte aligned, eight
// columns per lane (harris_adj_wide.cuh): interior segments staged by bulk copies, edge segments
// per lane by cp.async. Shared memory of a CTA: every warp's staging ring (NS slots of the image
// span and the cotangent span), then the ring barriers, then every warp's WRings.
template <typename TI, typename TG>
constexpr size_t wide_adj_smem(int ns) {
    return (size_t)(kBwdThreads / 32) * ns * (WSlot<TI, TG>::kBytes + 8) + (size_t)(kBwdThreads / 32) * kWRingBytes;
}

template <typename TI, typename TG, int NS, bool WITH_R>
__global__ void __launch_bounds__(kBwdThreads) harris_bwd_wide_kernel(BwdArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int kWarps = kBwdThreads / 32;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kWarps + warp;
    if (gw >= a.nwarps) return;  // whole warp
    const uint32_t base = smem_u32(smem_raw);
    const uint32_t ring0 = base + (uint32_t)warp * NS * WSlot<TI, TG>::kBytes;
    WRings rg;
    rg.init(base + kWarps * NS * (WSlot<TI, TG>::kBytes + 8) + (uint32_t)warp * kWRingBytes, lane);
    SHINE_CHECK(a.dbg, smem_in(ring0, NS * WSlot<TI, TG>::kBytes) &&
                           smem_in(base + kWarps * NS * (WSlot<TI, TG>::kBytes + 8) + (uint32_t)warp * kWRingBytes,
                                   kWRingBytes),
                kDbgSmem);
    rg.acc_zero();
    BulkState bulk;
    bulk.seq = 0;
    bulk.failed = false;
    bulk.bars = base + kWarps * NS * WSlot<TI, TG>::kBytes + (uint32_t)warp * NS * 8;
    if (lane == 0)
        for (int i = 0; i < NS; ++i) mbar_init(bulk.bars + 8 * i, 1);
    mbar_init_fence();
    __syncwarp();
    Params P;
    load_params(P, a.wx, a.wy, a.kappa);
    const int64_t rows = a.yhi - a.ylo;
    int64_t lo, hi;
    warp_work(SHINE_BWD_BAND_MAJOR, a.nseg, rows, a.nwarps, gw, lo, hi, SHINE_WIDE_BWD_EDGE_WEIGHT4);
    while (lo < hi && !bulk.failed) {
        const int seg = (int)(lo / rows);
        const int r0 = (int)(lo % rows);
        const int r1 = (int)(rows < r0 + (hi - lo) ? rows : r0 + (hi - lo));
        const int xb = a.x0 + seg * kWSegOut;
        const int x = xb - kWCols + kWCols * lane;
        const int y0 = a.ylo + r0, y1 = a.ylo + r1;
        const int n = y1 - y0 + 8;
        const bool edge = (xb - kWCols < 0) || (xb + kWSegOut + kWCols > a.W);
        if (edge) {
            WAdjLanes<TI, TG, NS> src(a, ring0, lane, x, y0 - 4, n);
            // a lane whose columns all lie outside the row copies nothing (zero-fill only)
            SHINE_CHECK(a.dbg, src.vbytes_img == 0 ||
                                   (x >= 0 && x * 3 * (int)sizeof(TI) + src.vbytes_img <= 3 * a.W * (int)sizeof(TI) &&
                                    x * (int)sizeof(TG) + src.vbytes_cot <= a.gwo * (int)sizeof(TG)),
                        kDbgBwdStage);
            wide_adj_strip<TI, true, false, WITH_R>(a, P, lane, x, y0, y1, src, rg, nullptr);
        } else {
            SHINE_CHECK(a.dbg, xb - kWCols >= 0 && xb - kWCols + kWSegLoad <= a.W && xb - kWCols + kWSegLoad <= a.gwo,
                        kDbgBwdStage);
            WAdjBulk<TI, TG, NS> src(bulk, a, ring0, lane, xb - kWCols, y0 - 4, n);
            wide_adj_strip<TI, false, true, WITH_R>(a, P, lane, x, y0, y1, src, rg, &bulk.failed);
        }
        lo += r1 - r0;
    }
    if (bulk.failed && lane == 0 && a.err != nullptr) atomicOr(a.err, 1u);
    const bool producer = lane >= 1 && lane <= 30;
    float acc[kParamSlots];
    rg.acc_get(acc);
#pragma unroll
    for (int i = 0; i < kParamSlots; ++i) {
        double v = producer ? (double)acc[i] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
        if (lane == 0) a.partials[(int64_t)i * (a.pstride ? a.pstride : a.nwarps) + a.poffset + gw] = v;
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

template <typename TI, typename TG>
cudaError_t launch_bwd_wide_t(BwdArgs a, int max_warps, cudaStream_t s, int* used) {
    constexpr int NS = sizeof(TI) == 4 ? SHINE_WIDE_BWD_STAGES_F32 : SHINE_WIDE_BWD_STAGES;
    const size_t smem = wide_adj_smem<TI, TG>(NS);
    auto kern = a.rout != nullptr ? harris_bwd_wide_kernel<TI, TG, NS, true> : harris_bwd_wide_kernel<TI, TG, NS, false>;
    // a lane's eight values of R and 24 of d img go out in 16-byte stores: 16-byte aligned rows
    a.rout_vec = a.rout_vec && reinterpret_cast<uintptr_t>(a.rout) % 16 == 0 &&
                 ((size_t)a.rout_pitch * sizeof(TI)) % 16 == 0;
    a.gimg_vec = a.gimg_vec && reinterpret_cast<uintptr_t>(a.gimg) % 16 == 0 &&
                 ((size_t)a.gimg_pitch * sizeof(TI)) % 16 == 0;
    a.x0 = SHINE_WIDE_BWD_ORIGIN;
    a.nseg = (a.xhi - a.x0 + kWSegOut - 1) / kWSegOut;
    const int64_t units = (int64_t)(a.yhi - a.ylo) * a.nseg;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t t = resident_warps(kern, kBwdThreads, smem);
    t = std::min<int64_t>(t, std::max<int64_t>(1, units / kBwdMinRows));
    t = std::max<int64_t>(1, std::min<int64_t>(t, max_warps));
    a.nwarps = (int)t;
    if (used) *used = a.nwarps;
    const int64_t blocks = (t + kBwdThreads / 32 - 1) / (kBwdThreads / 32);
    kern<<<(unsigned)blocks, kBwdThreads, smem, s>>>(a);
    return cudaPeekAtLastError();
}

// Image size (pixels) from which 16-bit CLAMP images take the eight-column adjoint: the
// environment variable SHINE_WIDE_BWD_MIN_PIXELS when set (read at every call, so that a test can
// reach either kernel on the same image), else SHINE_WIDE_BWD_MIN_PIXELS of the build.
int64_t wide_bwd_min_pixels() {
    if (const char* v = std::getenv("SHINE_WIDE_BWD_MIN_PIXELS")) {
        char* end = nullptr;
        const long long n = std::strtoll(v, &end, 10);
        if (end != v && *end == '\0' && n >= 0) return (int64_t)n;
    }
    return SHINE_WIDE_BWD_MIN_PIXELS;
}

template <typename TI, typename TG>
cudaError_t launch_bwd_t(BwdArgs a, int max_warps, cudaStream_t s, int* used) {
    // 16-bit CLAMP images with 16-byte aligned image and cotangent rows (a.tma): the wide kernel,
    // for the adjoint (measured on 8192^2: bf16 0.409 -> 0.388 ms, fp16 0.440 -> 0.410 ms; float32
    // 0.413 -> 0.478 ms, where its 96-byte lane pieces meet 2-way bank conflicts, so float32
    // images stay on the four-column kernel) and for the fused pass. Smaller images keep the
    // four-column kernel: with one resident wave the wide strips are half as long, and their
    // fixed cost per strip wins (bf16, adjoint / fused, us: 4096^2 129 / 152 four-column against
    // 140 / 162 wide, 2048^2 56 / 61 against 73 / 84; 8192^2 407 / 500 against 377 / 425)
    if constexpr (SHINE_WIDE_BWD && (sizeof(TI) == 2 || SHINE_WIDE_BWD_F32)) {
        if (a.tma && !a.valid && (a.rout == nullptr || SHINE_WIDE_BWD_FUSED) &&
            (int64_t)a.H * a.W >= wide_bwd_min_pixels())
            return launch_bwd_wide_t<TI, TG>(a, max_warps, s, used);
    }
    // ring depth: the adjoint alone takes bwd_stages<TI>(), the fused forward+adjoint (which also
    // stores R) the default depth (measured: float32 fused 0.486 ms at 8 rows, 0.494 at 6)
    constexpr int NS = bwd_stages<TI>();
    constexpr int NSR = kBwdStages;
    const bool wr = a.rout != nullptr;
    const int ns = wr ? NSR : NS;
    const size_t smem = (size_t)kBwdThreads * ns * (12 * sizeof(TI) + 4 * sizeof(TG)) + (kBwdThreads / 32) * ns * 8;
    void (*kern)(BwdArgs);
#define SHINE_BWD_PICK(AL, GA, TMA_)                                                            \
    kern = wr ? harris_bwd_kernel<TI, TG, NSR, AL, GA, true, TMA_> : harris_bwd_kernel<TI, TG, NS, AL, GA, false, TMA_>
    if (a.aligned && a.g_aligned && a.tma) SHINE_BWD_PICK(true, true, true);
    else if (a.aligned && a.g_aligned) SHINE_BWD_PICK(true, true, false);
    else if (a.aligned) SHINE_BWD_PICK(true, false, false);
    else SHINE_BWD_PICK(false, false, false);
#undef SHINE_BWD_PICK
    const int64_t units = (int64_t)(a.yhi - a.ylo) * a.nseg;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t t = resident_warps(kern, kBwdThreads, smem);
    t = std::min<int64_t>(t, std::max<int64_t>(1, units / kBwdMinRows));
    t = std::max<int64_t>(1, std::min<int64_t>(t, max_warps));
    a.nwarps = (int)t;
    if (used) *used = a.nwarps;
    const int64_t blocks = (t + kBwdThreads / 32 - 1) / (kBwdThreads / 32);
    kern<<<(unsigned)blocks, kBwdThreads, smem, s>>>(a);
    return cudaPeekAtLastError();
}

// Fixed-order float64 sum of the per-warp partials: block f reduces slot f.
__global__ void __launch_bounds__(256) finalize_params_kernel(const double* partials, int64_t n, float* gk,
                                                              float* gwx, float* gwy) {
    __shared__ double red[256];
    const int f = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) s += partials[(int64_t)f * n + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float v = (float)red[0];
        if (f == 0) { if (gk) *gk = v; }
        else if (f < 10) { if (gwx) gwx[f - 1] = v; }
        else { if (gwy) gwy[f - 10] = v; }
    }
}

}  // namespace

cudaError_t launch_harris_bwd(BwdArgs a, int dt, int gout_dt, int max_warps, cudaStream_t s, int* used) {
#define SHINE_BWD_CASE(I, G, TI, TG) \
    if (dt == I && gout_dt == G) return launch_bwd_t<TI, TG>(a, max_warps, s, used);
    SHINE_BWD_CASE(0, 0, float, float)
    SHINE_BWD_CASE(1, 1, __nv_bfloat16, __nv_bfloat16)
    SHINE_BWD_CASE(2, 2, __half, __half)
    SHINE_BWD_CASE(1, 0, __nv_bfloat16, float)
    SHINE_BWD_CASE(2, 0, __half, float)
#undef SHINE_BWD_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_finalize_params(const double* partials, int64_t n, float* gkappa, float* gwx, float* gwy,
                                   cudaStream_t s) {
    finalize_params_kernel<<<kParamSlots, 256, 0, s>>>(partials, n, gkappa, gwx, gwy);
    return cudaPeekAtLastError();
}

}  // namespace shine
