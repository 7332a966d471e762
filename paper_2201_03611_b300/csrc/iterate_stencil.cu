// iterate with a size-preserving body (Sec. 6 with n = 1): k rounds of the clamp-padded 3x3
// stencil
//   body(x) = map(map(nbh => reduce(+, 0)(map(*)(zip(join nbh, join W)))))(slide2D(3, 1)(pad_clamp2D(1)(x)))
// on an H x W float32 array, each round's output the next round's input. The two buffers of the
// double buffer live in shared memory, one pair per tile (temporal blocking):
//   * a CTA owns a 64 x 128 output tile and stages a 64 + 2(k-1) row by 144 column region of
//     every intermediate round (8 halo columns on each side, k-1 halo rows above and below: a
//     round reaches one row and one column further, and round 0 reads its own halo);
//   * round 0 reads the input straight from global memory (no copy into the double buffer:
//     clamped loads, through L1), rounds 1 .. k-2 ping-pong between the two buffers, and round
//     k-1 writes the output tile to global memory -- the swap / done structure of the paper's
//     double buffer with the intended condition (swap after every round but the last);
//   * per-stage clamp padding: after each intermediate round, a tile that touches the image
//     border overwrites the positions outside the image with the round's values at the clamped
//     positions, so the next round's stencil reads exactly pad_clamp2D(1) of that round;
//   * each thread owns a 4-column strip of a band of rows and slides a 3-row register window
//     down it (one new row per output row: a 16-byte shared load plus one value from each
//     neighbouring strip), the 9 taps a fused multiply-add chain in row-major order from zero.
// Each round's values near the tile edge go stale one row / column per round (their neighbours
// were never staged); the halos are sized so the stale band never reaches the output tile.
#include <cuda_runtime.h>

#include <algorithm>

#include "shine.h"
#include "shine_host.h"

namespace shine {
namespace {

constexpr int kItsThreads = 256;
constexpr int kItsTH = 64;                              // output rows per tile
constexpr int kItsTW = 128;                             // output columns per tile
constexpr int kItsHalo = 8;                             // staged columns on each side (>= k - 1)
constexpr int kItsMaxK = kItsHalo + 1;
constexpr int kItsCols = kItsTW + 2 * kItsHalo;         // 144 staged columns
constexpr int kItsStrips = kItsCols / 4;                // 36 four-column strips
constexpr int kItsBands = kItsThreads / kItsStrips;     // 7 row bands (252 threads busy)

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

// One output row of the strip: rows r0 (above), r1, r2 (below) hold columns 4s-1 .. 4s+4.
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

__global__ void __launch_bounds__(kItsThreads) iterate_stencil_kernel(const __grid_constant__ ItsArgs a) {
    extern __shared__ __align__(16) float its_smem[];
    const int tid = threadIdx.x;
    const int s = tid % kItsStrips;   // strip: staged columns 4s .. 4s+3
    const int band = tid / kItsStrips;
    const bool busy = band < kItsBands;
    const int k = a.k;
    const int TH2 = kItsTH + 2 * (k - 1);  // staged rows
    const int ty0 = (int)(blockIdx.x / a.tiles_x) * kItsTH;
    const int tx0 = (int)(blockIdx.x % a.tiles_x) * kItsTW;
    const int gy0 = ty0 - (k - 1);   // global row of staged row 0
    const int gx0 = tx0 - kItsHalo;  // global column of staged column 0
    const bool border = gy0 < 0 || gx0 < 0 || gy0 + TH2 > a.H || gx0 + kItsCols > a.W;
    float* buf[2] = {its_smem, its_smem + (size_t)TH2 * kItsCols};

    // Row r (staged coordinates) of round 0's input: global, clamped.
    auto load_global = [&](int r, float v[6]) {
        const int gy = clampi_its(gy0 + r, a.H);
        const float* row = a.in + (int64_t)gy * a.in_pitch;
        const int gx = gx0 + 4 * s;
        if (a.vec_in && gx >= 0 && gx + 3 < a.W) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(row + gx));
            v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) v[1 + j] = __ldg(row + clampi_its(gx + j, a.W));
        }
        v[0] = __ldg(row + clampi_its(gx - 1, a.W));
        v[5] = __ldg(row + clampi_its(gx + 4, a.W));
    };
    // Row r of a staged buffer (the strips at the region's two ends read their own edge value
    // for the missing neighbour column: stale positions, never used for the output).
    auto load_shared = [&](const float* src, int r, float v[6]) {
        const float* row = src + (size_t)r * kItsCols + 4 * s;
        const float4 q = *reinterpret_cast<const float4*>(row);
        v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
        v[0] = s > 0 ? row[-1] : q.x;
        v[5] = s < kItsStrips - 1 ? row[4] : q.w;
    };

    for (int i = 0; i < k; ++i) {
        const bool last = i == k - 1;
        const float* src = i == 0 ? nullptr : buf[(i - 1) & 1];
        float* dst = buf[i & 1];
        const int lo = i, hi = TH2 - i;  // rows this round produces (round 0: all staged rows)
        if (busy) {
            const int per = (hi - lo + kItsBands - 1) / kItsBands;
            const int r0 = lo + band * per;
            const int r1 = min(r0 + per, hi);
            auto load = [&](int r, float v[6]) {
                if (i == 0) load_global(r, v);
                else load_shared(src, r, v);
            };
            auto emit = [&](int r, const float o[4]) {
                if (!last) {
                    *reinterpret_cast<float4*>(dst + (size_t)r * kItsCols + 4 * s) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
                    const int gy = gy0 + r, gx = gx0 + 4 * s;
                    if (s >= kItsHalo / 4 && s < (kItsHalo + kItsTW) / 4 && gy < a.H && gx < a.W) {
                        float* orow = a.out + (int64_t)gy * a.out_pitch;
                        if (a.vec_out && gx + 3 < a.W) {
                            *reinterpret_cast<float4*>(orow + gx) = make_float4(o[0], o[1], o[2], o[3]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (gx + j < a.W) orow[gx + j] = o[j];
                        }
                    }
                }
            };
            if (r0 < r1) {
                // sliding 3-row window; the loop rotates the three registers by name, so no
                // row is copied
                float A[6], B[6], C[6], o[4];
                load(r0 - 1, A);
                load(r0, B);
                int r = r0;
                for (; r + 3 <= r1; r += 3) {
                    load(r + 1, C); its_row(a, A, B, C, o); emit(r, o);
                    load(r + 2, A); its_row(a, B, C, A, o); emit(r + 1, o);
                    load(r + 3, B); its_row(a, C, A, B, o); emit(r + 2, o);
                }
                if (r < r1) {
                    load(r + 1, C); its_row(a, A, B, C, o); emit(r, o);
                    if (r + 1 < r1) { load(r + 2, A); its_row(a, B, C, A, o); emit(r + 1, o); }
                }
            }
        }
        if (last) break;
        __syncthreads();
        if (border) {
            // pad_clamp2D(1) of this round for the next: staged positions outside the image take
            // the round's value at the clamped position (inside the image, so not written here).
            const int n = TH2 * kItsCols;
            for (int e = tid; e < n; e += kItsThreads) {
                const int r = e / kItsCols, c = e % kItsCols;
                const int gy = gy0 + r, gx = gx0 + c;
                if (gy < 0 || gy >= a.H || gx < 0 || gx >= a.W) {
                    const int rr = clampi_its(gy, a.H) - gy0, cc = clampi_its(gx, a.W) - gx0;
                    if (rr >= 0 && rr < TH2 && cc >= 0 && cc < kItsCols) dst[e] = dst[(size_t)rr * kItsCols + cc];
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
