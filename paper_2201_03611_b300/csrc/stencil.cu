// Generalised stencil: one fused slide2D(K, 1) + reduce stage with K x K weights (K odd, <= 9),
//   out = map(map(nbh => reduce(+, 0)(map(*)(zip(join nbh, join W)))))(slide2D(K, 1)(pad(x)))
// with pad = pad_clamp2D((K-1)/2) (CLAMP) or none (VALID), and the separable form (a K-tap
// stage down the columns with wv, then a K-tap stage along the rows with wh). The same strip
// machinery as the Harris kernels, generalised over K:
//   * a warp streams a column segment (120 output columns, 4 per lane; lanes 0 and 31 supply
//     the r = (K-1)/2 halo columns on each side through shuffles), one input row per step;
//   * push form (Sec. 4.2's fusion taken down the rows): each arriving row is added, with its
//     K weight rows, into the K output rows it belongs to; the oldest completes and is stored.
//     No window of input rows is kept, and the K-1 partial rows advance by renaming in place;
//   * clamp padding is index clamping of the loads, so every lane's values, halos included,
//     are those of the padded array.
// The weights are passed by value in the kernel parameters, so each multiply-add reads its
// weight from the constant bank instead of a register.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "harris_common.cuh"
#include "harris_kernels.h"
#include "shine.h"
#include "shine_host.h"
#include "entry.h"

namespace shine {
namespace {

constexpr int kStThreads = 128;
constexpr int kStMaxK = 9;

struct StencilArgs {
    const void* in;
    int64_t in_pitch;  // elements
    void* out;
    int64_t out_pitch;  // elements
    int H, W;
    int xlo, xhi, ylo, yhi;  // output region in input coordinates
    int ox, oy;              // input coordinates of output element (0, 0)
    int x0, nseg, nwarps;
    int aligned;  // input rows allow the lane's 4-element vector load
    int out_vec;  // output rows allow 4-element vector stores
    float w[kStMaxK * kStMaxK];
    float wv[kStMaxK];
    float wh[kStMaxK];
};

// The lane's 4 input values of row y (clamped), at columns x .. x+3 (clamped to [0, W)).
template <typename T, bool FAST>
__device__ __forceinline__ void load4(const StencilArgs& a, int x, int y, float c[4]) {
    const T* row = static_cast<const T*>(a.in) + (int64_t)clampi(y, a.H) * a.in_pitch;
    if constexpr (FAST) {
        if constexpr (sizeof(T) == 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(row + x));
            c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
        } else {
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(row + x));
            c[0] = Bits16<T>::to_f(v.x & 0xffffu);
            c[1] = Bits16<T>::to_f(v.x >> 16);
            c[2] = Bits16<T>::to_f(v.y & 0xffffu);
            c[3] = Bits16<T>::to_f(v.y >> 16);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = Conv<T>::ld(row[clampi(x + j, a.W)]);
    }
}

template <int K, bool SEP, typename TI, typename TO, bool EDGE, bool ALIGNED>
__device__ __forceinline__ void stencil_strip(const StencilArgs& a, int lane, int x, int y0, int y1) {
    constexpr int R = (K - 1) / 2;
    constexpr int NA = K > 1 ? K - 1 : 1;  // partial rows in flight
    constexpr bool FAST = ALIGNED && !EDGE;
    const bool producer = lane >= 1 && lane <= 30;
    bool cin[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cin[j] = x + j >= a.xlo && x + j < a.xhi;
    float acc[NA][4];  // partial output rows (push form), oldest first
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

    auto emit = [&](int o, const float v[4]) {
        if (!producer) return;
        TO* orow = static_cast<TO*>(a.out) + (int64_t)(o - a.oy) * a.out_pitch;
        if (!EDGE && a.out_vec) {
            if constexpr (sizeof(TO) == 4) {
                *reinterpret_cast<float4*>(orow + (x - a.ox)) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
                TO t[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) t[j] = Conv<TO>::st(v[j]);
                *reinterpret_cast<uint2*>(orow + (x - a.ox)) = *reinterpret_cast<const uint2*>(t);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (cin[j]) orow[x + j - a.ox] = Conv<TO>::st(v[j]);
        }
    };

    // One input row q (image row y0 - R + q) arrives with values c; completes output row
    // y0 + q - (K-1) when q >= K-1.
    auto push = [&](int q, const float c[4]) {
        const bool completes = q >= K - 1;
        float done[4];
        if constexpr (!SEP) {
            float e[4 + 2 * R];
            widen<R>(c, e);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float d = K > 1 ? acc[0][j] : 0.0f;
#pragma unroll
                for (int b = 0; b < K; ++b) d = fmaf(a.w[(K - 1) * K + b], e[j + b], d);
                done[j] = d;
#pragma unroll
                for (int i = 0; i + 1 < NA; ++i) {
                    float t = acc[i + 1][j];
#pragma unroll
                    for (int b = 0; b < K; ++b) t = fmaf(a.w[(K - 2 - i) * K + b], e[j + b], t);
                    acc[i][j] = t;
                }
                if constexpr (K > 1) {
                    float t = 0.0f;
#pragma unroll
                    for (int b = 0; b < K; ++b) t = fmaf(a.w[b], e[j + b], t);
                    acc[NA - 1][j] = t;
                }
            }
        } else {
            float vd[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                vd[j] = fmaf(a.wv[K - 1], c[j], K > 1 ? acc[0][j] : 0.0f);
#pragma unroll
                for (int i = 0; i + 1 < NA; ++i) acc[i][j] = fmaf(a.wv[K - 2 - i], c[j], acc[i + 1][j]);
                if constexpr (K > 1) acc[NA - 1][j] = fmaf(a.wv[0], c[j], 0.0f);
            }
            if (completes) {
                float e[4 + 2 * R];
                widen<R>(vd, e);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float d = 0.0f;
#pragma unroll
                    for (int b = 0; b < K; ++b) d = fmaf(a.wh[b], e[j + b], d);
                    done[j] = d;
                }
            }
        }
        if (completes) emit(y0 + q - (K - 1), done);
    };

    // register staging: the row two steps ahead is in flight
    const int nrows = y1 - y0 + K - 1;
    float c0[4], c1[4];
    load4<TI, FAST>(a, x, y0 - R, c0);
    if (nrows > 1) load4<TI, FAST>(a, x, y0 - R + 1, c1);
#pragma unroll 1
    for (int q = 0; q < nrows; q += 2) {
        float c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = c0[j];
        if (q + 2 < nrows) load4<TI, FAST>(a, x, y0 - R + q + 2, c0);
        push(q, c);
        if (q + 1 < nrows) {
#pragma unroll
            for (int j = 0; j < 4; ++j) c[j] = c1[j];
            if (q + 3 < nrows) load4<TI, FAST>(a, x, y0 - R + q + 3, c1);
            push(q + 1, c);
        }
    }
}

// Register caps by measurement: K = 5 at 102 registers (20 warps per SM instead of 16; 7%
// faster, the separable form 12%); K = 9 at 168 (12 warps instead of 8, 72 bytes spilled;
// 10% faster); K = 7 compiled with an explicit one-CTA minimum came out 3% faster than with
// none; K = 3 already fits more warps and is slower under any cap.
template <int K, bool SEP, typename TI, typename TO, bool ALIGNED>
__global__ void __launch_bounds__(kStThreads, K == 5 ? 5 : (K == 9 ? 3 : (K == 7 ? 1 : 0))) stencil_kernel(const __grid_constant__ StencilArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (kStThreads / 32) + (threadIdx.x >> 5);
    if (gw >= a.nwarps) return;
    const int64_t rows = a.yhi - a.ylo;
    int64_t lo, hi;
    warp_work(1, a.nseg, rows, a.nwarps, gw, lo, hi, SHINE_FWD_EDGE_WEIGHT4);
    while (lo < hi) {
        const int seg = (int)(lo / rows);
        const int r0 = (int)(lo % rows);
        const int r1 = (int)(rows < r0 + (hi - lo) ? rows : r0 + (hi - lo));
        const int xb = a.x0 + seg * kSegOut;
        const int x = xb - 4 + 4 * lane;
        const bool edge = (xb - 4 < 0) || (xb + kSegOut + 4 > a.W);
        if (edge) stencil_strip<K, SEP, TI, TO, true, ALIGNED>(a, lane, x, a.ylo + r0, a.ylo + r1);
        else stencil_strip<K, SEP, TI, TO, false, ALIGNED>(a, lane, x, a.ylo + r0, a.ylo + r1);
        lo += r1 - r0;
    }
}

template <int K, bool SEP, typename TI, typename TO>
cudaError_t launch_stencil_k(StencilArgs& a, cudaStream_t s) {
    auto kern = a.aligned ? stencil_kernel<K, SEP, TI, TO, true> : stencil_kernel<K, SEP, TI, TO, false>;
    const int64_t units = (int64_t)(a.yhi - a.ylo) * a.nseg;
    if (units <= 0) return cudaSuccess;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kStThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t t = (int64_t)per_sm * sm_count() * (kStThreads / 32);
    t = std::min<int64_t>(t, std::max<int64_t>(1, units / kFwdMinRows));
    a.nwarps = (int)t;
    const int64_t blocks = (t + kStThreads / 32 - 1) / (kStThreads / 32);
    kern<<<(unsigned)blocks, kStThreads, 0, s>>>(a);
    return cudaPeekAtLastError();
}

template <bool SEP, typename TI, typename TO>
cudaError_t launch_stencil_t(StencilArgs& a, int K, cudaStream_t s) {
    switch (K) {
        case 1: return launch_stencil_k<1, SEP, TI, TO>(a, s);
        case 3: return launch_stencil_k<3, SEP, TI, TO>(a, s);
        case 5: return launch_stencil_k<5, SEP, TI, TO>(a, s);
        case 7: return launch_stencil_k<7, SEP, TI, TO>(a, s);
        case 9: return launch_stencil_k<9, SEP, TI, TO>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <bool SEP>
cudaError_t launch_stencil(StencilArgs& a, int K, int dt, int out_dt, cudaStream_t s) {
    if (dt == SHINE_F32 && out_dt == SHINE_F32) return launch_stencil_t<SEP, float, float>(a, K, s);
    if (dt == SHINE_BF16 && out_dt == SHINE_BF16) return launch_stencil_t<SEP, __nv_bfloat16, __nv_bfloat16>(a, K, s);
    if (dt == SHINE_BF16 && out_dt == SHINE_F32) return launch_stencil_t<SEP, __nv_bfloat16, float>(a, K, s);
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace shine

using namespace shine;

extern "C" shine_status shine_stencil2d(const void* in, int64_t H, int64_t W, int64_t in_pitch, shine_dtype dt,
                                        shine_border border, int32_t K, const float* weights, const float* wv,
                                        const float* wh, void* out, int64_t out_pitch, shine_dtype out_dt,
                                        void* stream) {
    SHINE_ENTRY("shine_stencil2d");
    if (!in || !out) return SHINE_ERR_INVALID_ARG;
    if (K < 1 || K > kStMaxK || K % 2 == 0) return SHINE_ERR_INVALID_ARG;
    const bool sep = weights == nullptr;
    if (sep && (!wv || !wh)) return SHINE_ERR_INVALID_ARG;
    if (!dtype_ok(dt) || !dtype_ok(out_dt) || !border_ok(border)) return SHINE_ERR_INVALID_ARG;
    if (!((dt == SHINE_F32 && out_dt == SHINE_F32) || (dt == SHINE_BF16 && (out_dt == SHINE_BF16 || out_dt == SHINE_F32))))
        return SHINE_ERR_UNSUPPORTED;
    const int r = (K - 1) / 2;
    if (H < 1 || W < 1 || H > kMaxDim || W > kMaxDim) return SHINE_ERR_INVALID_ARG;
    if (border == SHINE_VALID && (H < K || W < K)) return SHINE_ERR_INVALID_ARG;
    const int64_t Ho = border == SHINE_VALID ? H - 2 * r : H, Wo = border == SHINE_VALID ? W - 2 * r : W;
    if (in_pitch < W || out_pitch < Wo) return SHINE_ERR_INVALID_ARG;
    (void)Ho;
    const size_t si = dtype_size(dt), so = dtype_size(out_dt);
    if (!aligned_to(in, si) || !aligned_to(out, so)) return SHINE_ERR_ALIGNMENT;
    StencilArgs a;
    a.in = in; a.in_pitch = in_pitch; a.out = out; a.out_pitch = out_pitch;
    a.H = (int)H; a.W = (int)W;
    if (border == SHINE_VALID) {
        a.xlo = r; a.xhi = (int)W - r; a.ylo = r; a.yhi = (int)H - r; a.ox = r; a.oy = r;
    } else {
        a.xlo = 0; a.xhi = (int)W; a.ylo = 0; a.yhi = (int)H; a.ox = 0; a.oy = 0;
    }
    a.x0 = kFwdSegmentOrigin;  // interior segments' lane columns are multiples of 4
    a.nseg = (a.xhi - a.x0 + kSegOut - 1) / kSegOut;
    a.nwarps = 0;
    a.aligned = aligned_to(in, 4 * si) && ((size_t)in_pitch * si) % (4 * si) == 0;
    a.out_vec = border == SHINE_CLAMP && aligned_to(out, 4 * so) && ((size_t)out_pitch * so) % (4 * so) == 0;
    // The weights travel by value in the kernel parameters (copied from the host here).
    for (int i = 0; i < kStMaxK * kStMaxK; ++i) a.w[i] = (!sep && i < K * K) ? weights[i] : 0.0f;
    for (int i = 0; i < kStMaxK; ++i) {
        a.wv[i] = (sep && i < K) ? wv[i] : 0.0f;
        a.wh[i] = (sep && i < K) ? wh[i] : 0.0f;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return cuda_status(sep ? launch_stencil<true>(a, K, dt, out_dt, s) : launch_stencil<false>(a, K, dt, out_dt, s));
}
