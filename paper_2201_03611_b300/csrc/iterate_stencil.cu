// iterate with a size-preserving body (Sec. 6 with n = 1): k rounds of the clamp-padded 3x3
// stencil
//   body(x) = map(map(nbh => reduce(+, 0)(map(*)(zip(join nbh, join W)))))(slide2D(3, 1)(pad_clamp2D(1)(x)))
// on an H x W float32 array, each round's output the next round's input. The two buffers of the
// double buffer live in shared memory, one pair per tile (temporal blocking):
//   * a CTA owns a 64 x 112 output tile and stages a 64 + 2(k-1) row by 128 column region of
//     every intermediate round (8 halo columns on each side, k-1 halo rows above and below: a
//     round reaches one row and one column further, and round 0 reads its own row halo);
//   * round 0 reads the input straight from global memory (no copy into the double buffer:
//     clamped loads, through L1), rounds 1 .. k-2 ping-pong between the two buffers, and round
//     k-1 writes the output tile to global memory -- the swap / done structure of the paper's
//     double buffer with the intended condition (swap after every round but the last);
//   * per-stage clamp padding: after each intermediate round, a tile that touches the image
//     border overwrites the positions outside the image with the round's values at the clamped
//     positions, so the next round's stencil reads exactly pad_clamp2D(1) of that round;
//   * each warp owns a band of rows and each lane a 4-column strip of it; the lane slides a
//     3-row register window down its strip, four new rows loaded together (one 16-byte load per
//     row; the neighbouring columns come from the adjacent lanes by shuffles), the 9 taps a
//     fused multiply-add chain in row-major order from zero.
// The outermost staged columns have no neighbour in the warp, so each round's values go stale
// one column (and, for rounds 1.., one row) further in from the staged region's edge; the halos
// are sized so the stale band never reaches the output tile (k <= 8).
#include <cuda_runtime.h>

#include <algorithm>

#include "shine.h"
#include "shine_host.h"

namespace shine {
namespace {

constexpr int kItsWarps = 8;                            // row bands per tile
constexpr int kItsThreads = 32 * kItsWarps;
constexpr int kItsTH = 64;                              // output rows per tile
constexpr int kItsHalo = 8;                             // staged columns on each side (>= k)
constexpr int kItsCols = 128;                           // staged columns: 4 per lane
constexpr int kItsTW = kItsCols - 2 * kItsHalo;         // 112 output columns per tile
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

// The lane's 4 values widened by one column from each neighbouring lane (row6: columns
// 4 lane - 1 .. 4 lane + 4); lanes 0 and 31 repeat their own edge value (stale columns).
__device__ __forceinline__ void its_widen(float4 q, float v[6]) {
    v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
    v[0] = __shfl_up_sync(kItsFull, q.w, 1);
    v[5] = __shfl_down_sync(kItsFull, q.x, 1);
}

// One output row of the strip: rows r0 (above), r1, r2 (below) hold columns 4 lane - 1 .. +4.
__device__ __forceinline__ void its_row(const ItsArgs& a, const float r0[6], const float r1[6], const float r2[6],
                                        float o[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
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
    float A[6], B[6], C[6], D[6], E[6], F[6], o[4];
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
        for (int j = 0; j < 6; ++j) { A[j] = E[j]; B[j] = F[j]; }
    }
    for (; r < r1; ++r) {
        load(r + 1, C);
        its_row(a, A, B, C, o); emit(r, o);
#pragma unroll
        for (int j = 0; j < 6; ++j) { A[j] = B[j]; B[j] = C[j]; }
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
    const int gx = gx0 + 4 * lane;   // the lane's first column
    const bool border = gy0 < 0 || gx0 < 0 || gy0 + TH2 > a.H || gx0 + kItsCols > a.W;
    const uint32_t sbuf0 = (uint32_t)__cvta_generic_to_shared(its_smem);
    const uint32_t sbuf_bytes = (uint32_t)TH2 * kItsCols * 4u;
    const uint32_t lane_off = 16u * (uint32_t)lane;

    // Row r (staged coordinates) of round 0's input: global, clamped.
    auto load_global = [&](int r, float v[6]) {
        const float* row = a.in + (int64_t)clampi_its(gy0 + r, a.H) * a.in_pitch;
        float4 q;
        if (a.vec_in && gx >= 0 && gx + 3 < a.W) {
            q = __ldg(reinterpret_cast<const float4*>(row + gx));
        } else {
            q.x = __ldg(row + clampi_its(gx, a.W));
            q.y = __ldg(row + clampi_its(gx + 1, a.W));
            q.z = __ldg(row + clampi_its(gx + 2, a.W));
            q.w = __ldg(row + clampi_its(gx + 3, a.W));
        }
        its_widen(q, v);
    };
    // The final round's rows go to the output tile (staged columns 8 .. 119, rows inside it).
    const bool out_lane = lane >= kItsHalo / 4 && lane < (kItsHalo + kItsTW) / 4 && gx < a.W;
    const bool out_vec = a.vec_out && gx + 3 < a.W;
    auto emit_global = [&](int r, const float o[4]) {
        const int gy = gy0 + r;
        if (out_lane && gy < a.H) {
            float* orow = a.out + (int64_t)gy * a.out_pitch + gx;
            if (out_vec) {
                *reinterpret_cast<float4*>(orow) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (gx + j < a.W) orow[j] = o[j];
            }
        }
    };

    // Tiles whose staged region, plus the row above and below it that round 0 reads, lies
    // inside the image (with 16-byte aligned rows) take loads and stores with no clamp or bound
    // test: a per-lane test there is turned into predicated code that issues both paths.
    const bool fast = gy0 >= 1 && gy0 + TH2 + 1 <= a.H && gx0 >= 0 && gx0 + kItsCols <= a.W && a.vec_in && a.vec_out;
    const bool store_lane = lane >= kItsHalo / 4 && lane < (kItsHalo + kItsTW) / 4;
    auto load_global_fast = [&](int r, float v[6]) {
        its_widen(__ldg(reinterpret_cast<const float4*>(a.in + (int64_t)(gy0 + r) * a.in_pitch + gx)), v);
    };
    auto emit_global_fast = [&](int r, const float o[4]) {
        if (store_lane)
            *reinterpret_cast<float4*>(a.out + (int64_t)(gy0 + r) * a.out_pitch + gx) = make_float4(o[0], o[1], o[2], o[3]);
    };

    for (int i = 0; i < k; ++i) {
        const bool last = i == k - 1;
        const uint32_t src = sbuf0 + ((i - 1) & 1) * sbuf_bytes + lane_off;  // rounds >= 1
        const uint32_t dst = sbuf0 + (i & 1) * sbuf_bytes + lane_off;
        const int lo = i, hi = TH2 - i;  // rows this round produces (round 0: all staged rows)
        const int per = (hi - lo + kItsWarps - 1) / kItsWarps;
        const int r0 = lo + band * per;
        const int r1 = min(r0 + per, hi);
        auto load_shared = [&](int r, float v[6]) { its_widen(its_lds128(src + (uint32_t)r * (kItsCols * 4)), v); };
        auto emit_shared = [&](int r, const float o[4]) {
            its_sts128(dst + (uint32_t)r * (kItsCols * 4), o[0], o[1], o[2], o[3]);
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
