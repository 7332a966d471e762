// Matrix-vector multiply, the paper's running example (Sec. 4): y = map(row => reduce(+, 0)
// (map(*)(zip(row, x))))(A).
//
// The B300 form is the split-join rewrite (Sec. 4.2) applied to each row's reduce: a warp owns
// a row, its 32 lanes split the row into 16-byte chunks taken round-robin, each lane reduces
// its chunks sequentially with fused multiply-adds (fuseReduceMap: the products never exist
// as an array), and the 32 partial sums are joined by a fixed butterfly of shuffles. Warps walk
// the rows grid-stride from one resident wave. The row is streamed once from HBM with 16-byte
// loads that bypass L1 allocation; x is read through the read-only path and stays in L1/L2.
// The kernel is HBM-bound: M * N * sizeof(T) bytes of A per launch.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "shine.h"
#include "shine_host.h"
#include "entry.h"

namespace shine {
namespace {

constexpr int kMvThreads = 256;
// 16-byte chunks a lane has in flight per row: 4 for float32, 8 for 16-bit types (their chunks
// carry twice the elements, and with 4 in flight the bf16 GEMV stayed at 67% of the copy
// bandwidth; 8 measured 16384^2 bf16 0.128 -> 0.102 ms, float32 unchanged).
template <typename T> constexpr int mv_unroll() { return sizeof(T) == 4 ? 4 : 8; }
constexpr unsigned kMvFull = 0xffffffffu;

template <typename T> struct MvElem;
template <> struct MvElem<float> {
    static constexpr int kPer = 4;  // elements per 16-byte chunk
    __device__ static float to_f(float v) { return v; }
};
template <> struct MvElem<__nv_bfloat16> {
    static constexpr int kPer = 8;
    __device__ static float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <> struct MvElem<__half> {
    static constexpr int kPer = 8;
    __device__ static float to_f(__half v) { return __half2float(v); }
};

__device__ __forceinline__ uint4 ld_stream16(const void* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

// acc += the dot product of one 16-byte chunk of A (elements j .. j+kPer-1) with x[j ..].
template <typename T>
__device__ __forceinline__ float chunk_dot(uint4 raw, const float* x, int64_t j, float acc) {
    if constexpr (sizeof(T) == 4) {
        const float4 xv = __ldg(reinterpret_cast<const float4*>(x + j));
        acc = fmaf(__uint_as_float(raw.x), xv.x, acc);
        acc = fmaf(__uint_as_float(raw.y), xv.y, acc);
        acc = fmaf(__uint_as_float(raw.z), xv.z, acc);
        acc = fmaf(__uint_as_float(raw.w), xv.w, acc);
    } else {
        const float4 x0 = __ldg(reinterpret_cast<const float4*>(x + j));
        const float4 x1 = __ldg(reinterpret_cast<const float4*>(x + j + 4));
        const T* e = reinterpret_cast<const T*>(&raw);
        const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) acc = fmaf(MvElem<T>::to_f(e[i]), xs[i], acc);
    }
    return acc;
}

// VEC: A and lda * sizeof(T) are 16-byte aligned and x is 16-byte aligned. Each lane sums its
// chunks c = lane, lane + 32, ... in order into U = mv_unroll<T>() accumulators (chunk c goes
// to accumulator (c / 32) % U), which are then added pairwise as a balanced tree
// ((a0 + a1) + (a2 + a3)) [+ ((a4 + a5) + (a6 + a7))]; the tail
// elements beyond the last whole chunk are added by the lanes that own them; then the
// butterfly. !VEC: each lane sums elements j = lane, lane + 32, ... sequentially.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kMvThreads) mv_kernel(const T* __restrict__ A, int64_t M, int64_t N, int64_t lda,
                                                        const float* __restrict__ x, float* __restrict__ y,
                                                        int64_t nwarps) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (kMvThreads / 32) + (threadIdx.x >> 5);
    constexpr int kPer = MvElem<T>::kPer;
    constexpr int kMvUnroll = mv_unroll<T>();
    for (int64_t row = gw; row < M; row += nwarps) {
        const T* r = A + row * lda;
        float s;
        if constexpr (VEC) {
            const int64_t nchunks = N / kPer;
            float acc[kMvUnroll];
#pragma unroll
            for (int u = 0; u < kMvUnroll; ++u) acc[u] = 0.0f;
            int64_t c = lane;
            // whole groups of kMvUnroll chunks per lane: all loads issued before the sums
            for (; c + 32 * (kMvUnroll - 1) < nchunks; c += 32 * kMvUnroll) {
                uint4 raw[kMvUnroll];
#pragma unroll
                for (int u = 0; u < kMvUnroll; ++u) raw[u] = ld_stream16(r + (c + 32 * u) * kPer);
#pragma unroll
                for (int u = 0; u < kMvUnroll; ++u) acc[u] = chunk_dot<T>(raw[u], x, (c + 32 * u) * kPer, acc[u]);
            }
#pragma unroll
            for (int u = 0; u < kMvUnroll; ++u) {
                if (c < nchunks) {
                    acc[u] = chunk_dot<T>(ld_stream16(r + c * kPer), x, c * kPer, acc[u]);
                    c += 32;
                }
            }
            s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
            if constexpr (kMvUnroll == 8) s = s + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
            for (int64_t j = nchunks * kPer + lane; j < N; j += 32) s = fmaf(MvElem<T>::to_f(r[j]), x[j], s);
        } else {
            s = 0.0f;
            for (int64_t j = lane; j < N; j += 32) s = fmaf(MvElem<T>::to_f(r[j]), x[j], s);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kMvFull, s, off);
        if (lane == 0) y[row] = s;
    }
}

template <typename T>
cudaError_t launch_mv(const void* A, int64_t M, int64_t N, int64_t lda, const float* x, float* y, cudaStream_t s) {
    const bool vec = aligned_to(A, 16) && aligned_to(x, 16) && ((size_t)lda * sizeof(T)) % 16 == 0;
    auto kern = vec ? mv_kernel<T, true> : mv_kernel<T, false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMvThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    // One resident wave; every warp gets the same number of rows (ceil(M / resident)), so no
    // warp is left with an extra row at the end while the others idle.
    const int64_t warps_per_block = kMvThreads / 32;
    const int64_t resident = (int64_t)per_sm * sm_count() * warps_per_block;
    const int64_t rows_per_warp = (M + resident - 1) / resident;
    const int64_t nwarps = (M + rows_per_warp - 1) / rows_per_warp;
    const int64_t blocks = (nwarps + warps_per_block - 1) / warps_per_block;
    kern<<<(unsigned)blocks, kMvThreads, 0, s>>>(static_cast<const T*>(A), M, N, lda, x, y, nwarps);
    return cudaPeekAtLastError();
}

}  // namespace
}  // namespace shine

using namespace shine;

extern "C" shine_status shine_mv(const void* A, int64_t M, int64_t N, int64_t lda, shine_dtype dt, const float* x,
                                 float* y, void* stream) {
    SHINE_ENTRY("shine_mv");
    if (M < 0 || N < 0 || M > ((int64_t)1 << 31) || N > ((int64_t)1 << 31) || lda < std::max<int64_t>(N, 1))
        return SHINE_ERR_INVALID_ARG;
    if (!dtype_ok(dt)) return SHINE_ERR_INVALID_ARG;
    if (M == 0) return SHINE_OK;
    if (!y || (N > 0 && (!A || !x))) return SHINE_ERR_INVALID_ARG;
    const size_t si = dtype_size(dt);
    if (!aligned_to(y, 4) || (N > 0 && (!aligned_to(x, 4) || !aligned_to(A, si)))) return SHINE_ERR_ALIGNMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (N == 0) {
        e = cudaMemsetAsync(y, 0, (size_t)M * sizeof(float), s);  // reduce(+, 0) of an empty row
    } else if (dt == SHINE_F32) {
        e = launch_mv<float>(A, M, N, lda, x, y, s);
    } else if (dt == SHINE_BF16) {
        e = launch_mv<__nv_bfloat16>(A, M, N, lda, x, y, s);
    } else {
        e = launch_mv<__half>(A, M, N, lda, x, y, s);
    }
    return cuda_status(e);
}
