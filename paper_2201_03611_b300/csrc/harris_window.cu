// Harris with a weighted K-tap window at A4 (K = 3, 5, 7): the pipeline A1 gray -> A2 Sobel ->
// A3 products -> A4' separable window (weights gv down the columns, gh along the rows, over the
// clamp-padded products) -> A5 response, fused into one kernel with only R written -- a
// multi-stage fusion of two generalised stencil stages (3x3 and K x K) with pointwise maps
// between them (map fusion and fuseReduceMap, Sec. 4.2). A Gaussian window is the usual choice.
//
// A warp streams a column segment as the forward does. Down the rows everything is in push
// form: gray rows complete Sobel rows (push_gray), each product row position p (p = y0-r ..
// y1-1+r, clamped to the image at the product stage by re-using the edge Sobel row) is added
// with its K window weights into the K output rows it belongs to, and the oldest completes.
// Along the row the completed vertical sums are widened by r columns from the neighbouring lanes
// (lanes 0 and 31 hold valid Sobel rows up to 3 columns beyond the segment), clamped at the image
// edge, and weighted with gh. Window weights are host values passed in the kernel parameters.
// The xx and yy planes travel as one packed float32 pair through both window passes (each half
// rounds as the scalar operation would), the xy plane alone.
#include <algorithm>

#include "harris_fwd_strip.cuh"
#include "shine_host.h"
#include "entry.h"

namespace shine {
namespace {

constexpr int kWinMaxK = 7;

struct WindowArgs {
    FwdArgs f;  // CLAMP geometry, image, R output, kappa, Wx, Wy
    float gv[kWinMaxK];
    float gh[kWinMaxK];
};

// Register staging of a warp's gray-row stream (rows g_first, g_first+1, ...; any segment and
// alignment): the next two rows are in flight in registers.
template <typename TI, bool EDGE, bool ALIGNED>
struct RegGray {
    const RegRows<TI, EDGE, ALIGNED> rows;
    const int H, x, W;
    int gnext;
    RawRow<TI> n0, n1;
    __device__ __forceinline__ RegGray(const FwdArgs& a, int x_, int g_first)
        : rows(static_cast<const TI*>(a.img), a.img_pitch, x_, a.W), H(a.H), x(x_), W(a.W), gnext(g_first) {
        rows.load(clampi(gnext, H), n0);
        rows.load(clampi(gnext + 1, H), n1);
    }
    __device__ __forceinline__ void take(float g6[6]) {
        float v[12];
        RegRows<TI, EDGE, ALIGNED>::unpack(n0, v);
        n0 = n1;
        rows.load(clampi(gnext + 2, H), n1);
        ++gnext;
        gray_row<EDGE>(v, g6, x, W);
    }
    __device__ __forceinline__ void finish() {}
};

// Output rows y0 .. y1-1 of a strip; src delivers the gray rows from max(y0 - r, 0) - 1 on.
template <typename TO, int K, bool EDGE, typename Src>
__device__ __forceinline__ void window_strip(const WindowArgs& wa, const Params& P, int lane, int x, int y0, int y1,
                                             Src& src) {
    const FwdArgs& a = wa.f;
    constexpr int R = (K - 1) / 2;
    constexpr int NA = K - 1;  // partial output rows in flight
    const int H = a.H, W = a.W;
    const int s_first = y0 - R > 0 ? y0 - R : 0;  // first Sobel row used
    auto take_gray = [&](float g6[6]) { src.take(g6); };
    float2 gv[K], gh[K];  // window weights, duplicated into both halves of a packed pair
#pragma unroll
    for (int i = 0; i < K; ++i) { gv[i] = dup2(wa.gv[i]); gh[i] = dup2(wa.gh[i]); }
    StripRun st;
#pragma unroll
    for (int j = 0; j < 4; ++j) st.P1[j] = st.P2[j] = make_float2(0.0f, 0.0f);
    float g[6];
#pragma unroll 1
    for (int i = 0; i < 3; ++i) {
        take_gray(g);
        push_gray(P, g, st);  // after the third: S = Sobel row s_first
    }
    int cur_s = s_first;

    // Partial vertical window sums: the xx and yy planes packed in one pair, xy alone.
    float2 vacc[NA][4];
    float vaxy[NA][4];
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { vacc[i][j] = make_float2(0.0f, 0.0f); vaxy[i][j] = 0.0f; }
    const bool producer = lane >= 1 && lane <= 30;
    TO* out = static_cast<TO*>(a.out);

#pragma unroll 1
    for (int p = y0 - R; p < y1 + R; ++p) {
        const int s = p < 0 ? 0 : (p > H - 1 ? H - 1 : p);
        if (s > cur_s) {  // the next Sobel row (the clamped positions re-use the edge row)
            take_gray(g);
            push_gray(P, g, st);
            ++cur_s;
        }
        // window position q = p - (y0 - R): output row p - R completes once q >= K-1
        float2 done[4];
        float dxy[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 p2 = __fmul2_rn(st.S[j], st.S[j]);  // (Sx^2, Sy^2)
            const float pxy = __fmul_rn(st.S[j].x, st.S[j].y);
            done[j] = __ffma2_rn(gv[K - 1], p2, vacc[0][j]);
            dxy[j] = fmaf(gv[K - 1].x, pxy, vaxy[0][j]);
#pragma unroll
            for (int i = 0; i + 1 < NA; ++i) {
                vacc[i][j] = __ffma2_rn(gv[K - 2 - i], p2, vacc[i + 1][j]);
                vaxy[i][j] = fmaf(gv[K - 2 - i].x, pxy, vaxy[i + 1][j]);
            }
            vacc[NA - 1][j] = __ffma2_rn(gv[0], p2, make_float2(0.0f, 0.0f));
            vaxy[NA - 1][j] = fmaf(gv[0].x, pxy, 0.0f);
        }
        if (p - (y0 - R) < K - 1) continue;
        const int y = p - R;
        float S3[3][4];
        {
            float ex[4 + 2 * R], ey[4 + 2 * R], exy[4 + 2 * R];
            float cx[4], cy[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) { cx[j] = done[j].x; cy[j] = done[j].y; }
            widen<R>(cx, ex);
            widen<R>(cy, ey);
            widen<R>(dxy, exy);
            if constexpr (EDGE) {
                clamp_widened<4 + 2 * R>(ex, x - R, W);
                clamp_widened<4 + 2 * R>(ey, x - R, W);
                clamp_widened<4 + 2 * R>(exy, x - R, W);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 t = make_float2(0.0f, 0.0f);
                float txy = 0.0f;
#pragma unroll
                for (int b = 0; b < K; ++b) {
                    t = __ffma2_rn(gh[b], make_float2(ex[j + b], ey[j + b]), t);
                    txy = fmaf(gh[b].x, exy[j + b], txy);
                }
                S3[0][j] = t.x;
                S3[1][j] = txy;
                S3[2][j] = t.y;
            }
        }
        float Rv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) Rv[j] = response(S3[0][j], S3[1][j], S3[2][j], P.kappa);
        TO* orow = out + (int64_t)y * a.out_pitch;
        if (!EDGE && a.out_vec) {
            if (producer) store4(orow + x, Rv);
        } else if (producer) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x + j >= 0 && x + j < W) orow[x + j] = Conv<TO>::st(Rv[j]);
        }
    }
}

// Register caps by measurement: K = 3 at 128 registers (16 warps per SM, 36 bytes spilled; 16%
// faster than at 12); K = 5 and 7 at 168 (12 warps instead of 8): K = 5 fits without spilling
// (1.1x faster), K = 7 spills ~200 bytes per thread and is still 4% faster.
template <typename TI, typename TO, int K, bool ALIGNED, bool TMA>
__global__ void __launch_bounds__(kFwdThreads, K <= 3 ? 4 : 3) harris_window_kernel(const __grid_constant__ WindowArgs wa) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const FwdArgs& a = wa.f;
    constexpr int NS = kFwdBulkStages;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (kFwdThreads / 32) + warp;
    if (gw >= a.nwarps) return;
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
    constexpr int R = (K - 1) / 2;
    const int64_t rows = a.yhi - a.ylo;
    int64_t lo, hi;
    warp_work(1, a.nseg, rows, a.nwarps, gw, lo, hi, SHINE_FWD_EDGE_WEIGHT4);
    while (lo < hi && !bulk.failed) {
        const int seg = (int)(lo / rows);
        const int r0 = (int)(lo % rows);
        const int r1 = (int)(rows < r0 + (hi - lo) ? rows : r0 + (hi - lo));
        const int xb = a.x0 + seg * kSegOut;
        const int x = xb - 4 + 4 * lane;
        const bool edge = (xb - 4 < 0) || (xb + kSegOut + 4 > a.W);
        const int y0 = a.ylo + r0, y1 = a.ylo + r1;
        const int s_first = y0 - R > 0 ? y0 - R : 0;
        const int s_last = y1 - 1 + R < a.H - 1 ? y1 - 1 + R : a.H - 1;
        if (edge) {
            RegGray<TI, true, ALIGNED> src(a, x, s_first - 1);
            window_strip<TO, K, true>(wa, P, lane, x, y0, y1, src);
        } else if constexpr (TMA) {
            BulkGray<TI, NS> src(a, bulk, ring, lane, x, s_first - 1, s_last - s_first + 3);
            window_strip<TO, K, false>(wa, P, lane, x, y0, y1, src);
            src.finish();
        } else {
            RegGray<TI, false, ALIGNED> src(a, x, s_first - 1);
            window_strip<TO, K, false>(wa, P, lane, x, y0, y1, src);
        }
        lo += r1 - r0;
    }
    if (bulk.failed && lane == 0 && a.err != nullptr) atomicOr(a.err, 1u);
}

template <typename TI, typename TO, int K>
cudaError_t launch_window_k(WindowArgs& wa, cudaStream_t s) {
    FwdArgs& a = wa.f;
    constexpr int NS = kFwdBulkStages;
    const bool tma = a.tma && a.aligned;
    const size_t smem = tma ? (size_t)kFwdThreads * NS * 12 * sizeof(TI) + (kFwdThreads / 32) * NS * 8 : 0;
    auto kern = tma ? harris_window_kernel<TI, TO, K, true, true>
                    : (a.aligned ? harris_window_kernel<TI, TO, K, true, false>
                                 : harris_window_kernel<TI, TO, K, false, false>);
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
    kern<<<(unsigned)blocks, kFwdThreads, smem, s>>>(wa);
    return cudaPeekAtLastError();
}

template <typename TI, typename TO>
cudaError_t launch_window_t(WindowArgs& wa, int K, cudaStream_t s) {
    switch (K) {
        case 3: return launch_window_k<TI, TO, 3>(wa, s);
        case 5: return launch_window_k<TI, TO, 5>(wa, s);
        case 7: return launch_window_k<TI, TO, 7>(wa, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace shine

using namespace shine;

extern "C" shine_status shine_harris_window(const void* img, int64_t H, int64_t W, int64_t img_pitch, shine_dtype dt,
                                            const float* kappa, const float* wx, const float* wy, int32_t K,
                                            const float* gv, const float* gh, void* out, int64_t out_pitch,
                                            shine_dtype out_dt, void* stream) {
    SHINE_ENTRY("shine_harris_window");
    if (!img || !kappa || !wx || !wy || !gv || !gh || !out) return SHINE_ERR_INVALID_ARG;
    if (K != 3 && K != 5 && K != 7) return SHINE_ERR_INVALID_ARG;
    if (!dtype_ok(dt) || !dtype_ok(out_dt)) return SHINE_ERR_INVALID_ARG;
    if (!((dt == SHINE_F32 && out_dt == SHINE_F32) || (dt == SHINE_BF16 && (out_dt == SHINE_BF16 || out_dt == SHINE_F32))))
        return SHINE_ERR_UNSUPPORTED;
    shine_status st = check_shape(H, W, SHINE_CLAMP);
    if (st != SHINE_OK) return st;
    if (img_pitch < 3 * W || out_pitch < W) return SHINE_ERR_INVALID_ARG;
    const size_t si = dtype_size(dt), so = dtype_size(out_dt);
    if (!aligned_to(img, si) || !aligned_to(out, so) || !aligned_to(kappa, 4) || !aligned_to(wx, 4) ||
        !aligned_to(wy, 4))
        return SHINE_ERR_ALIGNMENT;
    WindowArgs wa;
    FwdArgs& a = wa.f;
    static_cast<Geometry&>(a) = fwd_geometry(H, W, SHINE_CLAMP);
    a.img = img; a.img_pitch = img_pitch; a.out = out; a.out_pitch = out_pitch;
    a.kappa = kappa; a.wx = wx; a.wy = wy;
    const size_t chunk = si == 4 ? 16 : 8;
    a.aligned = aligned_to(img, chunk) && ((size_t)img_pitch * si) % chunk == 0;
    a.out_vec = aligned_to(out, 4 * so) && ((size_t)out_pitch * so) % (4 * so) == 0;
    a.tma = SHINE_FWD_TMA && aligned_to(img, 16) && ((size_t)img_pitch * si) % 16 == 0;
    a.err = wait_flag();
    for (int i = 0; i < kWinMaxK; ++i) {
        wa.gv[i] = i < K ? gv[i] : 0.0f;
        wa.gh[i] = i < K ? gh[i] : 0.0f;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaErrorInvalidValue;
    if (dt == SHINE_F32) e = launch_window_t<float, float>(wa, K, s);
    else if (out_dt == SHINE_BF16) e = launch_window_t<__nv_bfloat16, __nv_bfloat16>(wa, K, s);
    else e = launch_window_t<__nv_bfloat16, float>(wa, K, s);
    return cuda_status(e);
}
