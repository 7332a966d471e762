// Device building blocks shared by the fused Harris kernels (sm_103a).
//
// Work decomposition (the split/join tiling of the paper's Sec. 4.2, lowered by hand):
//   * the image is cut into column segments of kSegOut = 120 output columns; one warp owns a
//     segment and a band of rows, and streams down the band row by row (a sequential map over
//     rows, the mapSeq choice of Sec. 4.2), keeping the 3-row stencil windows in registers;
//   * each lane owns kCols = 4 adjacent columns; lanes 1..30 produce output, lanes 0 and 31
//     only provide the 2-column halo each stencil needs (read from neighbours by warp
//     shuffles, so no shared-memory round trip and no block-wide barrier is needed);
//   * the lane's 4 input pixels of each row are staged through a ring of NS rows in shared
//     memory with cp.async (the toMem(Local) choice), so NS-1 rows are always in flight while
//     the current one is computed; a slot holds the 32 lanes' chunks side by side (lane
//     stride 48 bytes for float32), so the 16-byte shared loads of a quarter-warp hit 8
//     distinct 16-byte bank groups;
//   * arithmetic is float32; the x and y halves of the Sobel and adjoint stencils run as
//     packed float32x2 operations (each half rounds exactly like the scalar operation);
//   * per-stage clamp padding is applied where it matters: at the image border, the value a
//     stencil reads beyond the edge is replaced by the edge value of THAT stage (gray, the
//     vertical product sums, ...), which is exactly pad_clamp before each slide2D.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "harris_kernels.h"

namespace shine {

constexpr unsigned kFull = 0xffffffffu;

// Luminance weights of A1 (nearest float32 values of 0.299, 0.587, 0.114).
constexpr float kGrayR = 0.299f, kGrayG = 0.587f, kGrayB = 0.114f;

__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

// A1 for one pixel.
__device__ __forceinline__ float gray_of(float r, float g, float b) {
    return fmaf(kGrayB, b, fmaf(kGrayG, g, kGrayR * r));
}

// ---------------------------------------------------------------------------------------------
// Storage types: float32 arithmetic, float32 / bf16 / fp16 storage (round to nearest even).
// ---------------------------------------------------------------------------------------------
template <typename T> struct Conv;
template <> struct Conv<float> {
    __device__ __forceinline__ static float ld(float v) { return v; }
    __device__ __forceinline__ static float st(float v) { return v; }
};
template <> struct Conv<__nv_bfloat16> {
    __device__ __forceinline__ static float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ __forceinline__ static __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};
template <> struct Conv<__half> {
    __device__ __forceinline__ static float ld(__half v) { return __half2float(v); }
    __device__ __forceinline__ static __half st(float v) { return __float2half_rn(v); }
};

// 16-bit types are moved as raw bits.
template <typename T> struct Bits16;
template <> struct Bits16<__nv_bfloat16> {
    __device__ __forceinline__ static float to_f(uint32_t b16) { return __uint_as_float(b16 << 16); }
};
template <> struct Bits16<__half> {
    __device__ __forceinline__ static float to_f(uint32_t b16) {
        return __half2float(__ushort_as_half((unsigned short)b16));
    }
};

// 16-bit channel values unpacked from a word holding two of them (element 0 in the low half).
__device__ __forceinline__ uint32_t lo16_to_hi(uint32_t w) {  // low half moved up, low half zero
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, 0x1044;" : "=r"(d) : "r"(w));
    return d;
}
template <typename T> struct Unpack16;
template <> struct Unpack16<__nv_bfloat16> {
    __device__ __forceinline__ static float lo(uint32_t w) { return __uint_as_float(lo16_to_hi(w)); }
    __device__ __forceinline__ static float hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
};
template <> struct Unpack16<__half> {
    __device__ __forceinline__ static float lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
    __device__ __forceinline__ static float hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
};

// Gray values of two adjacent 16-bit pixels from their three words (pixel 0: r, g in w0, b in the
// low half of w1; pixel 1: r in the high half of w1, g, b in w2), unpacked straight into the
// (pixel 0, pixel 1) pair of each channel and weighed with packed multiply-adds; each half is the
// scalar chain fma(kB, b, fma(kG, g, kR * r)) of gray_of.
template <typename T>
__device__ __forceinline__ float2 gray2_16(uint32_t w0, uint32_t w1, uint32_t w2) {
    const float2 r = make_float2(Unpack16<T>::lo(w0), Unpack16<T>::hi(w1));
    const float2 g = make_float2(Unpack16<T>::hi(w0), Unpack16<T>::lo(w2));
    const float2 b = make_float2(Unpack16<T>::lo(w1), Unpack16<T>::hi(w2));
    return __ffma2_rn(make_float2(kGrayB, kGrayB), b,
                      __ffma2_rn(make_float2(kGrayG, kGrayG), g, __fmul2_rn(make_float2(kGrayR, kGrayR), r)));
}

// ---------------------------------------------------------------------------------------------
// cp.async (LDGSTS) helpers. src_bytes < cp-size zero-fills the rest of the chunk and reads
// only src_bytes from global memory.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Bulk (TMA) copies into shared memory completing on an mbarrier. A warp owns NS barriers, one
// per ring slot; lane 0 arms a slot's barrier with the expected byte count and issues the
// copies, every lane waits on the slot's phase. Waits are bounded: after kMaxSpins polls the
// wait gives up, and the caller records the failure instead of hanging the GPU.
// ---------------------------------------------------------------------------------------------
constexpr int kMaxSpins = 1 << 22;

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// Loads from a shared-memory address (explicitly in the shared state space).
__device__ __forceinline__ float4 lds128(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ uint2 lds64(uint32_t addr) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "r"(addr) : "memory");
    return v;
}
// Debug builds: whether [addr, addr + bytes) lies inside the CTA's dynamic shared memory.
__device__ __forceinline__ bool smem_in(uint32_t addr, uint32_t bytes) {
    extern __shared__ unsigned char shine_dyn_smem[];
    uint32_t size;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(shine_dyn_smem));
    return addr >= base && addr + bytes <= base + size;
}

// Generic-proxy accesses to shared memory before async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Wait until the barrier's phase with the given parity has completed; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int max_spins = kMaxSpins) {
    for (int it = 0; it < max_spins; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Warp-wide wait for a bulk copy: lane 0 polls the barrier (bounded); once it has seen the
// phase complete, every lane waits on it once more, which succeeds at once and gives each lane
// its own acquire of the copied data. One polling lane instead of 32 keeps the barrier traffic
// of many waiting warps from slowing the copies they wait for (measured: the forward, 16 warps
// per SM, streams ~12% faster; the adjoint, 8 warps per SM with longer steps, is better off with
// the shorter all-lane wait). False on every lane when the poll gave up.
__device__ __forceinline__ bool warp_mbar_wait(uint32_t bar, uint32_t parity, int lane) {
    bool ok = true;
    if (lane == 0) ok = mbar_wait(bar, parity);
    if (!__shfl_sync(kFull, ok, 0)) return false;
    return __all_sync(kFull, mbar_wait(bar, parity));
}

// ---------------------------------------------------------------------------------------------
// PixelRows: the lane's 4 pixels (12 elements) of successive image rows.
//   ALIGNED: staged through a per-lane ring of NS rows in shared memory with cp.async; the
//            image pointer and the row pitch in bytes are multiples of the chunk size
//            (16 bytes for float32, 8 bytes for 16-bit types).
//   !ALIGNED: read element by element from global memory when needed (slow path).
// EDGE: some of the lane's pixels may lie outside [0, W): those read as zero and are never
// read from memory.
// ---------------------------------------------------------------------------------------------
template <typename T, int NS, bool EDGE, bool ALIGNED>
struct PixelRows {
    static constexpr int kChunk = sizeof(T) == 4 ? 16 : 8;
    static constexpr int kSlot = kLanes * 12;  // elements per ring slot (all 32 lanes)
    T* ring;         // this lane's 12 elements of slot 0; slot s is ring + s * kSlot
    const T* img;
    int64_t pitch;   // elements
    int x;           // first column of the lane
    int W;
    int valid_bytes; // bytes of the lane's 12 elements inside the row (EDGE only)

    __device__ __forceinline__ PixelRows(T* ring_, const T* img_, int64_t pitch_, int x_, int W_)
        : ring(ring_), img(img_), pitch(pitch_), x(x_), W(W_) {
        int npx = x < 0 ? 0 : (W - x >= kCols ? kCols : (W - x > 0 ? W - x : 0));
        valid_bytes = npx * 3 * (int)sizeof(T);
    }

    // Start staging image row yc (already clamped to [0, H)) into ring slot `slot`.
    __device__ __forceinline__ void fetch(int slot, int yc) const {
        if constexpr (ALIGNED) {
            const char* src = reinterpret_cast<const char*>(img + (int64_t)yc * pitch + (int64_t)x * 3);
            uint32_t dst = smem_u32(ring + slot * kSlot);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                int nb = kChunk;
                const char* s = src + i * kChunk;
                if constexpr (EDGE) {
                    nb = valid_bytes - i * kChunk;
                    nb = nb < 0 ? 0 : (nb > kChunk ? kChunk : nb);
                    if (nb == 0) s = reinterpret_cast<const char*>(img);
                }
                if constexpr (kChunk == 16) cp_async16(dst + i * 16, s, nb);
                else cp_async8(dst + i * 8, s, nb);
            }
        }
    }

    // The 12 channel values (float32) of the lane's pixels in image row yc (slot for ALIGNED).
    __device__ __forceinline__ void read(int slot, int yc, float v[12]) const {
        if constexpr (ALIGNED) {
            if constexpr (sizeof(T) == 4) {
                const float4* s = reinterpret_cast<const float4*>(ring + slot * kSlot);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float4 q = s[i];
                    v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
                }
            } else {
                const uint2* s = reinterpret_cast<const uint2*>(ring + slot * kSlot);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    uint2 q = s[i];
                    v[4 * i] = Bits16<T>::to_f(q.x & 0xffffu);
                    v[4 * i + 1] = Bits16<T>::to_f(q.x >> 16);
                    v[4 * i + 2] = Bits16<T>::to_f(q.y & 0xffffu);
                    v[4 * i + 3] = Bits16<T>::to_f(q.y >> 16);
                }
            }
        } else {
            const T* row = img + (int64_t)yc * pitch;
#pragma unroll
            for (int j = 0; j < kCols; ++j) {
                int c = x + j;
                bool in = !EDGE || (c >= 0 && c < W);
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
                    v[3 * j + ch] = in ? Conv<T>::ld(row[(int64_t)c * 3 + ch]) : 0.0f;
            }
        }
    }
};

// ---------------------------------------------------------------------------------------------
// RegRows: the lane's 4 pixels of an image row loaded straight into registers (128-bit loads for
// float32, 64-bit for 16-bit types) and kept there until used, so a warp keeps several rows in
// flight with no shared-memory round trip. Measured on B300, this staging streams the column
// strips at the copy bandwidth, where cp.async staging through shared memory topped out near
// 60% of it.
//   ALIGNED: the image pointer and the row pitch in bytes allow the vector loads.
//   EDGE: the lane's pixels may lie partly outside [0, W); those read as zero.
// ---------------------------------------------------------------------------------------------
template <typename T> struct RawRow;
template <> struct RawRow<float> { float4 q[3]; };
template <> struct RawRow<__nv_bfloat16> { uint2 q[3]; };
template <> struct RawRow<__half> { uint2 q[3]; };

template <typename T, bool EDGE, bool ALIGNED>
struct RegRows {
    const T* img;
    int64_t pitch;  // elements
    int x;          // first column of the lane
    int W;
    bool full;      // all 4 pixels inside [0, W)

    __device__ __forceinline__ RegRows(const T* img_, int64_t pitch_, int x_, int W_)
        : img(img_), pitch(pitch_), x(x_), W(W_), full(x_ >= 0 && x_ + kCols <= W_) {}

    // Issue the loads of image row yc (already clamped to [0, H)).
    __device__ __forceinline__ void load(int yc, RawRow<T>& r) const {
        const T* row = img + (int64_t)yc * pitch;
        if (ALIGNED && (!EDGE || full)) {
            if constexpr (sizeof(T) == 4) {
                const float4* s = reinterpret_cast<const float4*>(row + (int64_t)x * 3);
#pragma unroll
                for (int i = 0; i < 3; ++i) r.q[i] = __ldg(s + i);
            } else {
                const uint2* s = reinterpret_cast<const uint2*>(row + (int64_t)x * 3);
#pragma unroll
                for (int i = 0; i < 3; ++i) r.q[i] = __ldg(s + i);
            }
        } else {
            T e[12];
#pragma unroll
            for (int j = 0; j < kCols; ++j) {
                const int c = x + j;
                const bool in = !EDGE || (c >= 0 && c < W);
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) e[3 * j + ch] = in ? row[(int64_t)c * 3 + ch] : Conv<T>::st(0.0f);
            }
            r = *reinterpret_cast<const RawRow<T>*>(e);
        }
    }

    // The 12 channel values (float32) of a loaded row.
    __device__ __forceinline__ static void unpack(const RawRow<T>& r, float v[12]) {
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                v[4 * i] = r.q[i].x; v[4 * i + 1] = r.q[i].y; v[4 * i + 2] = r.q[i].z; v[4 * i + 3] = r.q[i].w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                v[4 * i] = Bits16<T>::to_f(r.q[i].x & 0xffffu);
                v[4 * i + 1] = Bits16<T>::to_f(r.q[i].x >> 16);
                v[4 * i + 2] = Bits16<T>::to_f(r.q[i].y & 0xffffu);
                v[4 * i + 3] = Bits16<T>::to_f(r.q[i].y >> 16);
            }
        }
    }
};

// ---------------------------------------------------------------------------------------------
// Warp-level neighbour exchange and per-stage clamp at the image border.
// A "row6" holds the 6 values of columns x-1 .. x+4 of one stage: the lane's own 4 and one
// from each neighbouring lane.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void make_row6(const float c[4], float r6[6]) {
    r6[0] = __shfl_up_sync(kFull, c[3], 1);
    r6[1] = c[0]; r6[2] = c[1]; r6[3] = c[2]; r6[4] = c[3];
    r6[5] = __shfl_down_sync(kFull, c[0], 1);
}
__device__ __forceinline__ void make_row6(const float2 c[4], float2 r6[6]) {
    r6[0].x = __shfl_up_sync(kFull, c[3].x, 1);
    r6[0].y = __shfl_up_sync(kFull, c[3].y, 1);
    r6[1] = c[0]; r6[2] = c[1]; r6[3] = c[2]; r6[4] = c[3];
    r6[5].x = __shfl_down_sync(kFull, c[0].x, 1);
    r6[5].y = __shfl_down_sync(kFull, c[0].y, 1);
}

// The lane's 4 values widened by R columns on each side from the neighbouring lanes (R <= 4).
template <int R>
__device__ __forceinline__ void widen(const float c[4], float e[4 + 2 * R]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) e[R + j] = c[j];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        e[i] = __shfl_up_sync(kFull, c[4 - R + i], 1);
        e[R + 4 + i] = __shfl_down_sync(kFull, c[i], 1);
    }
}

// pad_clamp at this stage for a widened row of N values at columns xs .. xs+N-1: values at
// columns outside [0, W) become the value at column 0 or W-1 (those columns are in the row
// whenever a position needs them, except on lanes wholly outside the image, whose values are
// never stored).
template <int N>
__device__ __forceinline__ void clamp_widened(float e[N], int xs, int W) {
    const int i0 = -xs, iw = W - 1 - xs;
    float v0 = e[0], vw = e[N - 1];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i == i0) v0 = e[i];
        if (i == iw) vw = e[i];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (xs + i < 0) e[i] = v0;
        else if (xs + i >= W) e[i] = vw;
    }
}

// pad_clamp at this stage: the value at column -1 becomes the value at column 0 and the
// value at column W becomes the value at column W-1. Only the stencil reads of in-image
// columns matter, and those read at most one column beyond the edge.
template <typename V>
__device__ __forceinline__ void clamp_row6(V r6[6], int x, int W) {
    if (x == 0) r6[0] = r6[1];
#pragma unroll
    for (int p = 1; p < 6; ++p)
        if (x - 1 + p == W) r6[p] = r6[p - 1];
}


__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// Loop-invariant parameters, read once per warp from device memory: w[k] = (Wx[k], Wy[k]).
struct Params {
    float2 w[9];
    float kappa;
};

__device__ __forceinline__ void load_params(Params& P, const float* wx, const float* wy, const float* kappa) {
#pragma unroll
    for (int i = 0; i < 9; ++i) P.w[i] = make_float2(__ldg(wx + i), __ldg(wy + i));
    P.kappa = __ldg(kappa);
}

// A2 on one lane: Sobel correlation of three 6-wide gray rows (r0 = row above) at the lane's
// 4 columns; I[j] = (Ix, Iy). Each half is the scalar fused multiply-add chain over the taps
// in row-major order, so every kernel that calls this gets the same bits.
__device__ __forceinline__ void sobel(const Params& P, const float r0[6], const float r1[6], const float r2[6],
                                      float2 I[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int b = 0; b < 3; ++b) acc = __ffma2_rn(P.w[b], dup2(r0[j + b]), acc);
#pragma unroll
        for (int b = 0; b < 3; ++b) acc = __ffma2_rn(P.w[3 + b], dup2(r1[j + b]), acc);
#pragma unroll
        for (int b = 0; b < 3; ++b) acc = __ffma2_rn(P.w[6 + b], dup2(r2[j + b]), acc);
        I[j] = acc;
    }
}

// A3 + vertical half of A4: the product sums over Sobel rows a (above), m, b (below), each
// already clamped by the caller, accumulated in the order the rows arrive when streaming
// down: V = fma(b, b, fma(m, m, a * a)) per plane. v2 = (xx, yy) sums, vxy = xy sums.
__device__ __forceinline__ void vertical_products(const float2 a[4], const float2 m[4], const float2 b[4],
                                                  float2 v2[4], float vxy[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v2[j] = __ffma2_rn(b[j], b[j], __ffma2_rn(m[j], m[j], __fmul2_rn(a[j], a[j])));
        vxy[j] = fmaf(b[j].x, b[j].y, fmaf(m[j].x, m[j].y, __fmul_rn(a[j].x, a[j].y)));
    }
}
// Running state of a warp streaming down a column strip in push form: every gray row and
// every Sobel row is added into the sums it contributes to when it arrives and is then
// dropped, so no window of rows is kept or shifted.
struct StripRun {
    float2 P1[4], P2[4];   // Sobel rows r and r+1 with two and one gray rows of taps added
    float2 S[4];           // the Sobel row completed last
    float2 A[4], B[4];     // (xx, yy): products of the last two Sobel rows summed; of the last one
    float Axy[4], Bxy[4];  // the same for the xy plane
};

// Gray row r arrives: it completes Sobel row r-1 into S and adds its taps to rows r and r+1.
// Each Sobel output is the fused multiply-add chain over its nine taps in row-major order,
// starting from zero, exactly as sobel() computes it.
__device__ __forceinline__ void push_gray(const Params& P, const float g[6], StripRun& st) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float2 s = st.P1[j], p1 = st.P2[j], p2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float2 gg = dup2(g[j + b]);
            s = __ffma2_rn(P.w[6 + b], gg, s);
            p1 = __ffma2_rn(P.w[3 + b], gg, p1);
            p2 = __ffma2_rn(P.w[b], gg, p2);
        }
        st.S[j] = s; st.P1[j] = p1; st.P2[j] = p2;
    }
}

// Sobel row S (row y+1) arrives: V = the vertical product sums of row y, as
// vertical_products(row y-1, row y, S) computes them; the running sums move down one row. At
// the bottom image row the caller leaves S at row y (the clamped row below), which gives
// vertical_products(row y-1, row y, row y).
__device__ __forceinline__ void push_products(StripRun& st, float2 v2[4], float vxy[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 s = st.S[j];
        v2[j] = __ffma2_rn(s, s, st.A[j]);
        vxy[j] = fmaf(s.x, s.y, st.Axy[j]);
        st.A[j] = __ffma2_rn(s, s, st.B[j]);
        st.Axy[j] = fmaf(s.x, s.y, st.Bxy[j]);
        st.B[j] = __fmul2_rn(s, s);
        st.Bxy[j] = __fmul_rn(s.x, s.y);
    }
}
// The product of the Sobel row S alone (B), or with the row above (A = fma(S, S, B)).
__device__ __forceinline__ void square_S(StripRun& st) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        st.B[j] = __fmul2_rn(st.S[j], st.S[j]);
        st.Bxy[j] = __fmul_rn(st.S[j].x, st.S[j].y);
    }
}
__device__ __forceinline__ void add_S(StripRun& st) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        st.A[j] = __ffma2_rn(st.S[j], st.S[j], st.B[j]);
        st.Axy[j] = fmaf(st.S[j].x, st.S[j].y, st.Bxy[j]);
    }
}

// Horizontal half of a 3x3 box sum (with the per-stage clamp on EDGE warps).
template <bool EDGE>
__device__ __forceinline__ void horizontal_box(const float v[4], float s[4], int x, int W) {
    float r6[6];
    make_row6(v, r6);
    if constexpr (EDGE) clamp_row6(r6, x, W);
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = __fadd_rn(__fadd_rn(r6[j], r6[j + 1]), r6[j + 2]);
}
template <bool EDGE>
__device__ __forceinline__ void horizontal_box(const float2 v[4], float2 s[4], int x, int W) {
    float2 r6[6];
    make_row6(v, r6);
    if constexpr (EDGE) clamp_row6(r6, x, W);
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = __fadd2_rn(__fadd2_rn(r6[j], r6[j + 1]), r6[j + 2]);
}

// A5 in float32 (det - kappa * trace^2 cancels, so it is never done in a narrower type).
__device__ __forceinline__ float response(float sxx, float sxy, float syy, float kappa) {
    const float tr = __fadd_rn(sxx, syy);
    const float det = fmaf(sxx, syy, -__fmul_rn(sxy, sxy));
    return fmaf(-__fmul_rn(kappa, tr), tr, det);
}

}  // namespace shine
