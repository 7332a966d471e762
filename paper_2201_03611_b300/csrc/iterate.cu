// iterate with double buffering (Sec. 6): k rounds of the body split(n) >> map(reduce(op, id))
// over Array[(n^k) m], each round folding every n consecutive values from the left, starting
// at the operator's identity (+ from 0, max from -inf, min from +inf), so out[j] is the
// level-by-level tree reduction of in[j n^k .. (j+1) n^k).
//
// A CTA takes G whole output groups at a time (G n^(k-1) <= kIterBuf). Round 0 reads the input
// straight from global memory (the double buffer's first input is the overall input, no copy)
// and writes buffer 0 in shared memory; rounds 1 .. k-2 read one shared buffer and write the
// other (swap); the last round writes the output in global memory (done). The swap/done choice
// is the one the paper's double-buffer code intends: the destination of round i is the output
// when i == k-1 and buffer i mod 2 otherwise; the source is the input when i == 0 and buffer
// (i-1) mod 2 otherwise. Every round keeps the fold order of reduce, so the result equals a
// float32 evaluation of the pattern definition bit for bit. Round 0 streams the input once
// (HBM-bound: (n^k) m 4 bytes); the later rounds run in shared memory.
#include <cuda_runtime.h>

#include <algorithm>

#include "shine.h"
#include "shine_host.h"
#include "entry.h"

namespace shine {
namespace {

constexpr int kIterThreads = 256;
constexpr int kIterBuf = 6144;  // floats per shared-memory buffer (two buffers: 48 KB)
constexpr int kIterUnroll = 4;  // round-0 values a thread has in flight

// The fold operator: + (rounded to nearest), max or min (IEEE maxNum / minNum: a NaN operand is
// ignored unless both are NaN), with its identity.
template <int OP> struct FoldOp;
template <> struct FoldOp<SHINE_REDUCE_SUM> {
    __device__ static float id() { return 0.0f; }
    __device__ static float f(float a, float b) { return __fadd_rn(a, b); }
};
template <> struct FoldOp<SHINE_REDUCE_MAX> {
    __device__ static float id() { return __int_as_float(0xff800000); }
    __device__ static float f(float a, float b) { return fmaxf(a, b); }
};
template <> struct FoldOp<SHINE_REDUCE_MIN> {
    __device__ static float id() { return __int_as_float(0x7f800000); }
    __device__ static float f(float a, float b) { return fminf(a, b); }
};

// Left fold of n consecutive values from the identity (N > 0: n == N known at compile time, so
// all its loads are issued together).
template <int N, int OP>
__device__ __forceinline__ float fold_global(const float* __restrict__ p, int n) {
    using F = FoldOp<OP>;
    float s = F::id();
    if constexpr (N > 0 && N % 4 == 0) {
        float4 v[N / 4];
#pragma unroll
        for (int e = 0; e < N / 4; ++e) v[e] = __ldcs(reinterpret_cast<const float4*>(p) + e);  // streamed once
#pragma unroll
        for (int e = 0; e < N / 4; ++e) s = F::f(F::f(F::f(F::f(s, v[e].x), v[e].y), v[e].z), v[e].w);
    } else if constexpr (N > 0) {
        float v[N];
#pragma unroll
        for (int e = 0; e < N; ++e) v[e] = __ldcs(p + e);
#pragma unroll
        for (int e = 0; e < N; ++e) s = F::f(s, v[e]);
    } else {
        for (int e = 0; e < n; ++e) s = F::f(s, __ldcs(p + e));
    }
    return s;
}

template <int OP>
__device__ __forceinline__ float fold_shared(const float* p, int n) {
    using F = FoldOp<OP>;
    float s = F::id();
    for (int e = 0; e < n; ++e) s = F::f(s, p[e]);
    return s;
}

template <int N, int OP>
__global__ void __launch_bounds__(kIterThreads) iterate_kernel(const float* __restrict__ in, int64_t m, int n,
                                                                   int k, int64_t span1, int64_t G,
                                                                   float* __restrict__ out) {
    // span1 = n^(k-1): level-1 values per output group; G groups per pass (G * span1 <= kIterBuf)
    __shared__ float buf[2][kIterBuf];
    if constexpr (N > 0) n = N;
    const int64_t passes = (m + G - 1) / G;
    for (int64_t pass = blockIdx.x; pass < passes; pass += gridDim.x) {
        const int64_t g0 = pass * G;
        const int64_t groups = (m - g0) < G ? (m - g0) : G;
        int64_t count = groups * span1;  // values after round 0
        // round 0: the input (global) -> buffer 0, or the output when k == 1
        const float* src0 = in + g0 * span1 * n;
        float* dst0 = k == 1 ? out + g0 : buf[0];
        for (int64_t v0 = threadIdx.x; v0 < count; v0 += kIterThreads * kIterUnroll) {
            float r[kIterUnroll];
#pragma unroll
            for (int u = 0; u < kIterUnroll; ++u) {
                const int64_t v = v0 + (int64_t)u * kIterThreads;
                r[u] = v < count ? fold_global<N, OP>(src0 + v * n, n) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < kIterUnroll; ++u) {
                const int64_t v = v0 + (int64_t)u * kIterThreads;
                if (v < count) dst0[v] = r[u];
            }
        }
        // rounds 1 .. k-1: swap between the two buffers; the last writes the output (done)
        for (int i = 1; i < k; ++i) {
            __syncthreads();
            const float* src = buf[(i - 1) & 1];
            float* dst = i == k - 1 ? out + g0 : buf[i & 1];
            count /= n;
            for (int64_t v = threadIdx.x; v < count; v += kIterThreads) dst[v] = fold_shared<OP>(src + v * n, n);
        }
        __syncthreads();  // the buffers are reused by the next pass
    }
}

template <int N, int OP>
cudaError_t launch_iterate(const float* in, int64_t m, int n, int k, int64_t span1, int64_t G, float* out,
                           cudaStream_t s) {
    const int64_t passes = (m + G - 1) / G;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iterate_kernel<N, OP>, kIterThreads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(passes, (int64_t)per_sm * sm_count()));
    iterate_kernel<N, OP><<<(unsigned)blocks, kIterThreads, 0, s>>>(in, m, n, k, span1, G, out);
    return cudaPeekAtLastError();
}

// Round 0 reads groups of n consecutive floats: with 16-byte loads when n is a multiple of 4
// and the input is 16-byte aligned.
template <int OP>
cudaError_t launch_iterate_op(const float* in, int64_t m, int n, int k, int64_t span1, int64_t G, float* out,
                              cudaStream_t s) {
    const bool vec = aligned_to(in, 16);
    if (n == 2) return launch_iterate<2, OP>(in, m, n, k, span1, G, out, s);
    if (n == 4 && vec) return launch_iterate<4, OP>(in, m, n, k, span1, G, out, s);
    if (n == 8 && vec) return launch_iterate<8, OP>(in, m, n, k, span1, G, out, s);
    if (n == 16 && vec) return launch_iterate<16, OP>(in, m, n, k, span1, G, out, s);
    return launch_iterate<0, OP>(in, m, n, k, span1, G, out, s);
}

}  // namespace
}  // namespace shine

using namespace shine;

extern "C" shine_status shine_iterate_reduce(const float* in, int64_t m, int32_t n, int32_t k, shine_reduce_op op,
                                             float* out, void* stream) {
    SHINE_ENTRY("shine_iterate_reduce");
    if (m < 0 || n < 1 || k < 0) return SHINE_ERR_INVALID_ARG;
    if (op != SHINE_REDUCE_SUM && op != SHINE_REDUCE_MAX && op != SHINE_REDUCE_MIN) return SHINE_ERR_INVALID_ARG;
    // n^k and n^(k-1) without overflow
    int64_t span = 1, span1 = 1;
    for (int i = 0; i < k; ++i) {
        if (span > ((int64_t)1 << 40) / n) return SHINE_ERR_INVALID_ARG;
        span1 = span;
        span *= n;
    }
    if (m > 0 && span > (((int64_t)1 << 40) / m)) return SHINE_ERR_INVALID_ARG;
    if (m == 0) return SHINE_OK;
    if (!in || !out) return SHINE_ERR_INVALID_ARG;
    if (!aligned_to(in, 4) || !aligned_to(out, 4)) return SHINE_ERR_ALIGNMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k == 0)  // zero rounds: the input itself
        return cuda_status(cudaMemcpyAsync(out, in, (size_t)m * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (k > 1 && span1 > kIterBuf) return SHINE_ERR_UNSUPPORTED;  // one group's level-1 values must fit
    const int64_t G = k > 1 ? kIterBuf / span1 : kIterBuf;
    cudaError_t e;
    if (op == SHINE_REDUCE_SUM) e = launch_iterate_op<SHINE_REDUCE_SUM>(in, m, n, k, span1, G, out, s);
    else if (op == SHINE_REDUCE_MAX) e = launch_iterate_op<SHINE_REDUCE_MAX>(in, m, n, k, span1, G, out, s);
    else e = launch_iterate_op<SHINE_REDUCE_MIN>(in, m, n, k, span1, G, out, s);
    return cuda_status(e);
}

extern "C" shine_status shine_iterate_sum(const float* in, int64_t m, int32_t n, int32_t k, float* out,
                                          void* stream) {
    SHINE_ENTRY("shine_iterate_sum");
    return shine_iterate_reduce(in, m, n, k, SHINE_REDUCE_SUM, out, stream);
}
