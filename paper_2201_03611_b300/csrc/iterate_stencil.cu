// iterate with a size-preserving body (Sec. 6 with n = 1): k rounds of the clamp-padded 3x3
// stencil
//   body(x) = map(map(nbh => reduce(+, 0)(map(*)(zip(join nbh, join W)))))(slide2D(3, 1)(pad_clamp2D(1)(x)))
// on an H x W float32 array, each round's output the next round's input. The two buffers of the
// double buffer live in shared memory, one pair per tile (temporal blocking):
//   * a CTA owns a 64 x 112 output tile (default knobs below) and stages a 64 + 2(k-1) row by
//     128 column region of every intermediate round (8 halo columns on each side, k-1 halo rows
//     above and below: a round reaches one row and one column further, and round 0 reads its
//     own row halo);
//   * round 0 reads the input straight from global memory (no copy into the double buffer:
//     clamped loads, through L1), rounds 1 .. k-2 ping-pong between the two buffers, and round
//     k-1 writes the output tile to global memory -- the swap / done structure of the paper's
//     double buffer with the intended condition (swap after every round but the last);
//   * per-stage clamp padding: after each intermediate round, a tile that touches the image
//     border overwrites the positions outside the image with the round's values at the clamped
//     positions, so the next round's stencil reads exactly pad_clamp2D(1) of that round;
//   * each warp owns a band of rows and each lane a 4-column strip of it (SHINE_ITS_PX); the
//     lane slides a 3-row register window down its strip, four new rows loaded together (16-byte
//     loads; the neighbouring columns come from the adjacent lanes by shuffles), the 9 taps a
//     fused multiply-add chain in row-major order from zero.
// The outermost staged columns have no neighbour in the warp, so each round's values go stale
// one column (and, for rounds 1.., one row) further in from the staged region's edge; the halos
// are sized so the stale band never reaches the output tile (k <= 8).
#include <cuda_runtime.h>

#include <algorithm>

#include "shine.h"
#include "shine_host.h"
#include "entry.h"

namespace shine {
namespace {

// Tile shape knobs (measured on 8192^2, k = 4: 4 columns per lane and 64 rows 0.23 ms; 4 and 32
// rows 0.28 ms; 8 columns and 32 rows 0.29 ms; 8 and 64 rows, one CTA per SM, 0.36 ms).
#ifndef SHINE_ITS_PX
#define SHINE_ITS_PX 4
#endif
#ifndef SHINE_ITS_TH
#define SHINE_ITS_TH 64
#endif
constexpr int kItsWarps = 8;                            // row bands per tile
constexpr int kItsThreads = 32 * kItsWarps;
constexpr int kItsPx = SHINE_ITS_PX;                    // columns per lane (a multiple of 4)
constexpr int kItsQ = kItsPx / 4;                       // 16-byte chunks per lane and row
constexpr int kItsTH = SHINE_ITS_TH;                    // output rows per tile
constexpr int kItsHalo = 8;                             // staged columns on each side (>= k)
constexpr int kItsCols = 32 * kItsPx;                   // staged columns
constexpr int kItsTW = kItsCols - 2 * kItsHalo;         // output columns per tile
static_assert(kItsPx % 4 == 0 && kItsHalo % kItsPx == 0, "whole 16-byte chunks per lane; halo of whole lanes");
constexpr int kItsMaxK = kItsHalo;
constexpr unsigned kItsFull = 0xffffffffu;

struct ItsArgs {
    const float* in;
    int64_t in_pitch;  // elements
    float* out;
    int64_t out_pitch;  // elements
    int H, W, k;
    int tiles_x;
    int vec_in;   // input rows allow 16-byte loads
    int vec_out;  // output rows allow 16-byte stores
    float w[9];
};

__device__ __forceinline__ int clampi_its(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

__device__ __forceinline__ float4 its_lds128(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr)
                 : "memory");
    return v;
}
__device__ __forceinline__ void its_sts128(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// The lane's kItsPx values widened by one column from each neighbouring lane (columns
// P lane - 1 .. P lane + P); lanes 0 and 31 repeat their own edge value (stale columns).
__device__ __forceinline__ void its_widen(const float4 q[kItsQ], float v[kItsPx + 2]) {
#pragma unroll
    for (int u = 0; u < kItsQ; ++u) {
        v[1 + 4 * u] = q[u].x; v[2 + 4 * u] = q[u].y; v[3 + 4 * u] = q[u].z; v[4 + 4 * u] = q[u].w;
    }
    v[0] = __shfl_up_sync(kItsFull, q[kItsQ - 1].w, 1);
    v[kItsPx + 1] = __shfl_down_sync(kItsFull, q[0].x, 1);
}

// One output row of the strip: rows r0 (above), r1, r2 (below) hold the widened columns.
__device__ __forceinline__ void its_row(const ItsArgs& a, const float r0[kItsPx + 2], const float r1[kItsPx + 2],
                                        const float r2[kItsPx + 2], float o[kItsPx]) {
#pragma unroll
    for (int j = 0; j < kItsPx; ++j) {
        float t = 0.0f;
#pragma unroll
        for (int b = 0; b < 3; ++b) t = fmaf(a.w[b], r0[j + b], t);
#pragma unroll
        for (int b = 0; b < 3; ++b) t = fmaf(a.w[3 + b], r1[j + b], t);
#pragma unroll
        for (int b = 0; b < 3; ++b) t = fmaf(a.w[6 + b], r2[j + b], t);
        o[j] = t;
    }
}

// Rows [r0, r1) of one round for this lane's strip: load(r, v) delivers a widened input row,
// emit(r, o) takes an output row. Four new rows are loaded together per iteration so that
// every lane keeps four loads in flight.
template <typename Load, typename Emit>
__device__ __forceinline__ void its_band(const ItsArgs& a, int r0, int r1, Load&& load, Emit&& emit) {
    float A[kItsPx + 2], B[kItsPx + 2], C[kItsPx + 2], D[kItsPx + 2], E[kItsPx + 2], F[kItsPx + 2], o[kItsPx];
    load(r0 - 1, A);
    load(r0, B);
    int r = r0;
    for (; r + 4 <= r1; r += 4) {
        load(r + 1, C);
        load(r + 2, D);
        load(r + 3, E);
        load(r + 4, F);
        its_row(a, A, B, C, o); emit(r, o);
        its_row(a, B, C, D, o); emit(r + 1, o);
        its_row(a, C, D, E, o); emit(r + 2, o);
        its_row(a, D, E, F, o); emit(r + 3, o);
#pragma unroll
        for (int j = 0; j < kItsPx + 2; ++j) { A[j] = E[j]; B[j] = F[j]; }
    }
    for (; r < r1; ++r) {
        load(r + 1, C);
        its_row(a, A, B, C, o); emit(r, o);
#pragma unroll
        for (int j = 0; j < kItsPx + 2; ++j) { A[j] = B[j]; B[j] = C[j]; }
    }
}

__global__ void __launch_bounds__(kItsThreads) iterate_stencil_kernel(const __grid_constant__ ItsArgs a) {
    extern __shared__ __align__(16) float its_smem[];
    const int lane = threadIdx.x & 31;
    const int band = threadIdx.x >> 5;
    const int k = a.k;
    const int TH2 = kItsTH + 2 * (k - 1);  // staged rows
    const int ty0 = (int)(blockIdx.x / a.tiles_x) * kItsTH;
    const int tx0 = (int)(blockIdx.x % a.tiles_x) * kItsTW;
    const int gy0 = ty0 - (k - 1);   // global row of staged row 0
    const int gx0 = tx0 - kItsHalo;  // global column of staged column 0
    const int gx = gx0 + kItsPx * lane;  // the lane's first column
    const bool border = gy0 < 0 || gx0 < 0 || gy0 + TH2 > a.H || gx0 + kItsCols > a.W;
    const uint32_t sbuf0 = (uint32_t)__cvta_generic_to_shared(its_smem);
    const uint32_t sbuf_bytes = (uint32_t)TH2 * kItsCols * 4u;
    const uint32_t lane_off = 4u * kItsPx * (uint32_t)lane;

    // Row r (staged coordinates) of round 0's input: global, clamped.
    auto load_global = [&](int r, float v[kItsPx + 2]) {
        const float* row = a.in + (int64_t)clampi_its(gy0 + r, a.H) * a.in_pitch;
        float4 q[kItsQ];
        if (a.vec_in && gx >= 0 && gx + kItsPx - 1 < a.W) {
#pragma unroll
            for (int u = 0; u < kItsQ; ++u) q[u] = __ldg(reinterpret_cast<const float4*>(row + gx) + u);
        } else {
#pragma unroll
            for (int u = 0; u < kItsQ; ++u) {
                q[u].x = __ldg(row + clampi_its(gx + 4 * u, a.W));
                q[u].y = __ldg(row + clampi_its(gx + 4 * u + 1, a.W));
                q[u].z = __ldg(row + clampi_its(gx + 4 * u + 2, a.W));
                q[u].w = __ldg(row + clampi_its(gx + 4 * u + 3, a.W));
            }
        }
        its_widen(q, v);
    };
    // The final round's rows go to the output tile (the staged columns between the halos, rows
    // inside the image).
    const bool store_lane = lane >= kItsHalo / kItsPx && lane < (kItsHalo + kItsTW) / kItsPx;
    const bool out_lane = store_lane && gx < a.W;
    const bool out_vec = a.vec_out && gx + kItsPx - 1 < a.W;
    auto emit_global = [&](int r, const float o[kItsPx]) {
        const int gy = gy0 + r;
        if (out_lane && gy < a.H) {
            float* orow = a.out + (int64_t)gy * a.out_pitch + gx;
            if (out_vec) {
#pragma unroll
                for (int u = 0; u < kItsQ; ++u)
                    reinterpret_cast<float4*>(orow)[u] = make_float4(o[4 * u], o[4 * u + 1], o[4 * u + 2], o[4 * u + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < kItsPx; ++j)
                    if (gx + j < a.W) orow[j] = o[j];
            }
        }
    };

    // Tiles whose staged region, plus the row above and below it that round 0 reads, lies
    // inside the image (with 16-byte aligned rows) take loads and stores with no clamp or bound
    // test: a per-lane test there is turned into predicated code that issues both paths.
    const bool fast = gy0 >= 1 && gy0 + TH2 + 1 <= a.H && gx0 >= 0 && gx0 + kItsCols <= a.W && a.vec_in && a.vec_out;
    auto load_global_fast = [&](int r, float v[kItsPx + 2]) {
        const float4* row = reinterpret_cast<const float4*>(a.in + (int64_t)(gy0 + r) * a.in_pitch + gx);
        float4 q[kItsQ];
#pragma unroll
        for (int u = 0; u < kItsQ; ++u) q[u] = __ldg(row + u);
        its_widen(q, v);
    };
    auto emit_global_fast = [&](int r, const float o[kItsPx]) {
        float4* orow = reinterpret_cast<float4*>(a.out + (int64_t)(gy0 + r) * a.out_pitch + gx);
        if (store_lane)
#pragma unroll
            for (int u = 0; u < kItsQ; ++u) orow[u] = make_float4(o[4 * u], o[4 * u + 1], o[4 * u + 2], o[4 * u + 3]);
    };

    for (int i = 0; i < k; ++i) {
        const bool last = i == k - 1;
        const uint32_t src = sbuf0 + ((i - 1) & 1) * sbuf_bytes + lane_off;  // rounds >= 1
        const uint32_t dst = sbuf0 + (i & 1) * sbuf_bytes + lane_off;
        const int lo = i, hi = TH2 - i;  // rows this round produces (round 0: all staged rows)
        const int per = (hi - lo + kItsWarps - 1) / kItsWarps;
        const int r0 = lo + band * per;
        const int r1 = min(r0 + per, hi);
        auto load_shared = [&](int r, float v[kItsPx + 2]) {
            float4 q[kItsQ];
#pragma unroll
            for (int u = 0; u < kItsQ; ++u) q[u] = its_lds128(src + (uint32_t)r * (kItsCols * 4) + 16u * u);
            its_widen(q, v);
        };
        auto emit_shared = [&](int r, const float o[kItsPx]) {
#pragma unroll
            for (int u = 0; u < kItsQ; ++u)
                its_sts128(dst + (uint32_t)r * (kItsCols * 4) + 16u * u, o[4 * u], o[4 * u + 1], o[4 * u + 2], o[4 * u + 3]);
        };
        if (r0 < r1) {  // whole warp (r0, r1 depend on the band only)
            if (i == 0) {
                if (fast) {
                    if (last) its_band(a, r0, r1, load_global_fast, emit_global_fast);
                    else its_band(a, r0, r1, load_global_fast, emit_shared);
                } else {
                    if (last) its_band(a, r0, r1, load_global, emit_global);
                    else its_band(a, r0, r1, load_global, emit_shared);
                }
            } else {
                if (last) {
                    if (fast) its_band(a, r0, r1, load_shared, emit_global_fast);
                    else its_band(a, r0, r1, load_shared, emit_global);
                } else {
                    its_band(a, r0, r1, load_shared, emit_shared);
                }
            }
        }
        if (last) break;
        __syncthreads();
        if (border) {
            // pad_clamp2D(1) of this round for the next: staged positions outside the image take
            // the round's value at the clamped position (inside the image, so not written here).
            float* d = its_smem + (size_t)(i & 1) * TH2 * kItsCols;
            const int n = TH2 * kItsCols;
            for (int e = threadIdx.x; e < n; e += kItsThreads) {
                const int r = e / kItsCols, c = e % kItsCols;
                const int gy = gy0 + r, gxe = gx0 + c;
                if (gy < 0 || gy >= a.H || gxe < 0 || gxe >= a.W) {
                    const int rr = clampi_its(gy, a.H) - gy0, cc = clampi_its(gxe, a.W) - gx0;
                    if (rr >= 0 && rr < TH2 && cc >= 0 && cc < kItsCols) d[e] = d[(size_t)rr * kItsCols + cc];
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace
}  // namespace shine

using namespace shine;

extern "C" shine_status shine_iterate_stencil(const float* in, int64_t H, int64_t W, int64_t in_pitch,
                                              const float* weights, int32_t k, float* out, int64_t out_pitch,
                                              void* stream) {
    SHINE_ENTRY("shine_iterate_stencil");
    if (!in || !out || !weights) return SHINE_ERR_INVALID_ARG;
    if (k < 1 || k > kItsMaxK) return SHINE_ERR_INVALID_ARG;
    if (H < 1 || W < 1 || H > kMaxDim || W > kMaxDim) return SHINE_ERR_INVALID_ARG;
    if (in_pitch < W || out_pitch < W) return SHINE_ERR_INVALID_ARG;
    if (!aligned_to(in, 4) || !aligned_to(out, 4)) return SHINE_ERR_ALIGNMENT;
    // The tiles read their input halos while other tiles write their outputs: no overlap.
    const uintptr_t ib = reinterpret_cast<uintptr_t>(in), ob = reinterpret_cast<uintptr_t>(out);
    const uintptr_t ie = ib + (uintptr_t)((H - 1) * in_pitch + W) * 4, oe = ob + (uintptr_t)((H - 1) * out_pitch + W) * 4;
    if (ib < oe && ob < ie) return SHINE_ERR_INVALID_ARG;
    ItsArgs a;
    a.in = in; a.in_pitch = in_pitch; a.out = out; a.out_pitch = out_pitch;
    a.H = (int)H; a.W = (int)W; a.k = k;
    a.tiles_x = (int)((W + kItsTW - 1) / kItsTW);
    const int64_t tiles = (int64_t)a.tiles_x * ((H + kItsTH - 1) / kItsTH);
    if (tiles > 0x7fffffff) return SHINE_ERR_INVALID_ARG;
    a.vec_in = aligned_to(in, 16) && (in_pitch % 4) == 0;
    a.vec_out = aligned_to(out, 16) && (out_pitch % 4) == 0;
    for (int i = 0; i < 9; ++i) a.w[i] = weights[i];
    const size_t smem = k > 1 ? (size_t)2 * (kItsTH + 2 * (k - 1)) * kItsCols * sizeof(float) : 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(iterate_stencil_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
    }
    iterate_stencil_kernel<<<(unsigned)tiles, kItsThreads, smem, s>>>(a);
    return cuda_status(cudaPeekAtLastError());
}
