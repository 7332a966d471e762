// Wide forward strip: one warp computes R over one (column segment, row band) of one image,
// eight columns per lane.
//
// The same pipeline and the same arithmetic as harris_fwd_strip.cuh (push form: an arriving gray
// row completes one Sobel row and advances the next two; a completed Sobel row completes one row
// of vertical product sums), so R is bit-identical to every other kernel of the library. What
// changes is the shape of the work: a lane owns 8 adjacent columns, a warp 256 staged and 240
// computed ones (lanes 0 and 31 only supply the 2-column halos), so the fixed cost of a row step
// -- the staging wait, the copy issue, the neighbour shuffles, the loop -- is spread over twice
// as many pixels. For 16-bit storage, which halves the bytes of a row but not its arithmetic, that
// fixed cost had been the limit.
#pragma once

#include <type_traits>

#include "harris_common.cuh"
#include "harris_kernels.h"

namespace shine {

constexpr int kWCols = 8;                        // pixels per lane
constexpr int kWSegLoad = kLanes * kWCols;       // 256 staged columns per warp segment
constexpr int kWSegOut = (kLanes - 2) * kWCols;  // 240 computed columns per warp segment

// pad_clamp of a widened row of N = 8 + 2 values at columns x-1 .. x+8: the value at column -1
// becomes the value at column 0, the value at column W the value at column W-1 (the stencils of
// in-image columns read at most one column beyond the edge).
template <typename V>
__device__ __forceinline__ void clamp_row10(V r[10], int x, int W) {
    if (x == 0) r[0] = r[1];
#pragma unroll
    for (int p = 1; p < 10; ++p)
        if (x - 1 + p == W) r[p] = r[p - 1];
}

template <typename V>
__device__ __forceinline__ V shfl_up1(V v);
template <>
__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(kFull, v, 1); }
template <>
__device__ __forceinline__ float2 shfl_up1(float2 v) {
    return make_float2(__shfl_up_sync(kFull, v.x, 1), __shfl_up_sync(kFull, v.y, 1));
}
template <typename V>
__device__ __forceinline__ V shfl_down1(V v);
template <>
__device__ __forceinline__ float shfl_down1(float v) { return __shfl_down_sync(kFull, v, 1); }
template <>
__device__ __forceinline__ float2 shfl_down1(float2 v) {
    return make_float2(__shfl_down_sync(kFull, v.x, 1), __shfl_down_sync(kFull, v.y, 1));
}

// The lane's 8 values widened by one column from each neighbouring lane (clamped on EDGE warps).
template <bool EDGE, typename V>
__device__ __forceinline__ void widen10(const V c[8], V r[10], int x, int W) {
    r[0] = shfl_up1(c[7]);
#pragma unroll
    for (int j = 0; j < 8; ++j) r[1 + j] = c[j];
    r[9] = shfl_down1(c[0]);
    if constexpr (EDGE) clamp_row10(r, x, W);
}

// Horizontal half of a 3x3 box sum over 8 columns: (r[j] + r[j+1]) + r[j+2], as everywhere else.
template <bool EDGE>
__device__ __forceinline__ void hbox8(const float2 v[8], float2 s[8], int x, int W) {
    float2 r[10];
    widen10<EDGE>(v, r, x, W);
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] = __fadd2_rn(__fadd2_rn(r[j], r[j + 1]), r[j + 2]);
}
template <bool EDGE>
__device__ __forceinline__ void hbox8(const float v[8], float s[8], int x, int W) {
    float r[10];
    widen10<EDGE>(v, r, x, W);
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] = __fadd_rn(__fadd_rn(r[j], r[j + 1]), r[j + 2]);
}

// Running state of a warp streaming down its strip (push form; see StripRun).
struct WideRun {
    float2 P1[8], P2[8];   // Sobel rows r and r+1 with two and one gray rows of taps added
    float2 S[8];           // the Sobel row completed last
    float2 A[8], B[8];     // (xx, yy): products of the last two Sobel rows summed; of the last one
    float Axy[8], Bxy[8];  // the same for the xy plane
};

// Gray row r (10 wide) arrives: it completes Sobel row r-1 into S and adds its taps to rows r
// and r+1 (the nine-tap fused multiply-add chain in row-major order from zero, as sobel()).
__device__ __forceinline__ void wide_push_gray(const Params& P, const float g[10], WideRun& st) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
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

// Sobel row S (row y+1) arrives: v = the vertical product sums of row y (see push_products).
__device__ __forceinline__ void wide_push_products(WideRun& st, float2 v2[8], float vxy[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float2 s = st.S[j];
        v2[j] = __ffma2_rn(s, s, st.A[j]);
        vxy[j] = fmaf(s.x, s.y, st.Axy[j]);
        st.A[j] = __ffma2_rn(s, s, st.B[j]);
        st.Axy[j] = fmaf(s.x, s.y, st.Bxy[j]);
        st.B[j] = __fmul2_rn(s, s);
        st.Bxy[j] = __fmul_rn(s.x, s.y);
    }
}
__device__ __forceinline__ void wide_square_S(WideRun& st) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        st.B[j] = __fmul2_rn(st.S[j], st.S[j]);
        st.Bxy[j] = __fmul_rn(st.S[j].x, st.S[j].y);
    }
}
__device__ __forceinline__ void wide_add_S(WideRun& st) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        st.A[j] = __ffma2_rn(st.S[j], st.S[j], st.B[j]);
        st.Axy[j] = fmaf(st.S[j].x, st.S[j].y, st.Bxy[j]);
    }
}

// ---------------------------------------------------------------------------------------------
// Gray values of the lane's 8 pixels (24 channel values). 16-bit pixels are unpacked two at a
// time straight into the (pixel j, pixel j+1) pairs of each channel and weighed with packed
// multiply-adds; each half is the scalar chain fma(kB, b, fma(kG, g, kR * r)) of gray_of.
// ---------------------------------------------------------------------------------------------
// 16-bit: w[0..11] are the 12 words of 24 channel values (pixel 2i in words 3i, 3i+1 low half;
// pixel 2i+1 in words 3i+1 high half, 3i+2).
template <typename T>
__device__ __forceinline__ void gray8_16(const uint32_t w[12], float c[8]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 y = gray2_16<T>(w[3 * i], w[3 * i + 1], w[3 * i + 2]);
        c[2 * i] = y.x;
        c[2 * i + 1] = y.y;
    }
}
__device__ __forceinline__ void gray8_32(const float v[24], float c[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j] = gray_of(v[3 * j], v[3 * j + 1], v[3 * j + 2]);
}

// The lane's raw row: 24 channel values as 6 (float32) or 3 (16-bit) 16-byte chunks.
template <typename T> struct WideRaw { uint4 q[sizeof(T) == 4 ? 6 : 3]; };

template <typename T>
__device__ __forceinline__ void gray8(const WideRaw<T>& r, float c[8]) {
    if constexpr (sizeof(T) == 4) {
        float v[24];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            v[4 * i] = __uint_as_float(r.q[i].x); v[4 * i + 1] = __uint_as_float(r.q[i].y);
            v[4 * i + 2] = __uint_as_float(r.q[i].z); v[4 * i + 3] = __uint_as_float(r.q[i].w);
        }
        gray8_32(v, c);
    } else {
        uint32_t w[12];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            w[4 * i] = r.q[i].x; w[4 * i + 1] = r.q[i].y; w[4 * i + 2] = r.q[i].z; w[4 * i + 3] = r.q[i].w;
        }
        gray8_16<T>(w, c);
    }
}

// The lane's 24 channel values of image row yc loaded into registers: 16-byte loads when the
// lane's pixels all lie inside the image (FULL: known to) and VEC (16-byte aligned rows), else
// element by element with the pixels outside [0, W) read as zero.
template <typename T, bool VEC, bool FULL = false>
__device__ __forceinline__ void wide_load(const T* img, int64_t pitch, int yc, int x, int W, WideRaw<T>& r) {
    const T* row = img + (int64_t)yc * pitch;
    constexpr int NQ = sizeof(T) == 4 ? 6 : 3;
    if (VEC && (FULL || (x >= 0 && x + kWCols <= W))) {
        const uint4* s = reinterpret_cast<const uint4*>(row + (int64_t)x * 3);
#pragma unroll
        for (int i = 0; i < NQ; ++i) r.q[i] = __ldg(s + i);
    } else {
        T e[24];
#pragma unroll
        for (int j = 0; j < kWCols; ++j) {
            const int c = x + j;
            const bool in = c >= 0 && c < W;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) e[3 * j + ch] = in ? row[(int64_t)c * 3 + ch] : Conv<T>::st(0.0f);
        }
        r = *reinterpret_cast<const WideRaw<T>*>(e);
    }
}

// R of the lane's 8 columns, converted to the output type and stored with 16-byte stores.
template <typename TO>
__device__ __forceinline__ void store8(TO* p, const float R[8]) {
    if constexpr (sizeof(TO) == 4) {
        float4* d = reinterpret_cast<float4*>(p);
        d[0] = make_float4(R[0], R[1], R[2], R[3]);
        d[1] = make_float4(R[4], R[5], R[6], R[7]);
    } else {
        uint32_t u[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if constexpr (std::is_same<TO, __nv_bfloat16>::value) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(R[2 * i], R[2 * i + 1]);
                u[i] = *reinterpret_cast<const uint32_t*>(&h);
            } else {
                const __half2 h = __floats2half2_rn(R[2 * i], R[2 * i + 1]);
                u[i] = *reinterpret_cast<const uint32_t*>(&h);
            }
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(u[0], u[1], u[2], u[3]);
    }
}

// ---------------------------------------------------------------------------------------------
// The strip walk: y0 .. y1-1 are the output rows; take(g) delivers the next gray row of the
// sequence y0-2, y0-1, ... (image rows, clamped to [0, H)), widened to 10 columns;
// store(y, R) writes R[y]; go() is false once the staging has failed. At the bottom image row the
// Sobel row is not advanced (the product stage's clamp reuses row H-1), so the strip that ends
// there takes one gray row fewer.
// ---------------------------------------------------------------------------------------------
template <bool EDGE, typename Take, typename Store, typename Go>
__device__ __forceinline__ void wide_strip_core(const Params& P, int x, int W, int H, int y0, int y1, Take&& take,
                                                Store&& store, Go&& go) {
    WideRun st;
#pragma unroll
    for (int j = 0; j < 8; ++j) st.P1[j] = st.P2[j] = make_float2(0.0f, 0.0f);
    float g[10];
    // gray rows y0-2 .. y0+1: S = Sobel row y0-1 after the third, Sobel row y0 after the fourth
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        take(g);
        wide_push_gray(P, g, st);
        if (i == 2) wide_square_S(st);
    }
    if (y0 == 0) wide_square_S(st);  // the product row above the image is the clamped copy of row 0
    wide_add_S(st);
    wide_square_S(st);
#pragma unroll 1
    for (int y = y0; y < y1; ++y) {
        if (!go()) return;
        // gray row y+2 completes Sobel row y+1; at the bottom image row S stays at row H-1, the
        // clamped row below it at the product stage (and no gray row is taken)
        if (y != H - 1) {
            take(g);
            wide_push_gray(P, g, st);
        }
        float2 v2[8];
        float vxy[8], sxy[8], R[8];
        wide_push_products(st, v2, vxy);
        hbox8<EDGE>(vxy, sxy, x, W);
        float2 r[10];
        widen10<EDGE>(v2, r, x, W);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 s2 = __fadd2_rn(__fadd2_rn(r[j], r[j + 1]), r[j + 2]);
            R[j] = response(s2.x, sxy[j], s2.y, P.kappa);
        }
        store(y, R);
    }
}

// L2 prefetch of a byte range of global memory (a hint; completes on its own, nothing waits).
__device__ __forceinline__ void prefetch_l2_pred(uint32_t issue, const void* p, uint32_t bytes) {
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q cp.async.bulk.prefetch.L2.global [%1], %2;\n}\n"
                 ::"r"(issue), "l"(p), "r"(bytes) : "memory");
}

// Bulk (TMA) staging of a warp's gray-row stream on an interior segment with 16-byte aligned
// rows: lane 0 moves each row's 256-pixel span into a ring of NS shared-memory slots with one
// copy completing on the slot's mbarrier. Per row: a barrier check (all lanes test the phase
// once; only when the copy is late does lane 0 poll, bounded, before the lanes test again), the
// lane's 16-byte shared loads, one copy issue into the slot just read (predicated on lane 0, no
// branch), and the gray arithmetic. Ring position and row pointers advance incrementally.
struct WideBulkState {
    uint32_t bars;  // shared address of this warp's NS barriers
    uint32_t seq;   // rows staged by this warp so far (row n sits in slot n % NS)
    bool failed;    // a bounded wait gave up
};

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Lane 0 (issue != 0) re-arms the slot's barrier for `bytes` and starts the copy; the proxy fence
// orders the lanes' earlier shared loads of the slot before the copy's writes.
__device__ __forceinline__ void bulk_issue_pred(uint32_t issue, uint32_t bar, uint32_t dst, const void* src,
                                                uint32_t bytes) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %0, 0;\n"
        "@p fence.proxy.async.shared::cta;\n"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%1], %2;\n"
        "@p cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%3], [%4], %2, [%1];\n}\n"
        ::"r"(issue), "r"(bar), "r"(bytes), "r"(dst), "l"(src)
        : "memory");
}

template <typename TI, int NS>
struct WideBulk {
    static constexpr uint32_t kBytes = kWSegLoad * 3 * sizeof(TI);  // one slot: 256 pixels
    WideBulkState& bs;
    const int lane, n;           // rows of the stream
    uint32_t bar, dst, lane_src;  // current slot: barrier, warp slot base, this lane's chunk
    uint32_t slot, phase;
    uint32_t bar0, dst0;         // slot 0
    const char* src;             // global row of the next copy
    int64_t pitch_bytes;
    int frow, last_row;          // image row of the next copy (unclamped), H - 1
    int fq = 0, tq = 0, failed_q = 0;

    __device__ __forceinline__ WideBulk(WideBulkState& bs_, const TI* img, int64_t pitch, int xs, uint32_t ring0,
                                        int lane_, int g_first, int n_, int H)
        : bs(bs_), lane(lane_), n(n_) {
        slot = bs.seq % NS;
        phase = (bs.seq / NS) & 1u;
        bar0 = bs.bars;
        dst0 = ring0;
        bar = bar0 + 8 * slot;
        dst = dst0 + slot * kBytes;
        lane_src = dst + lane * (kWCols * 3 * sizeof(TI));
        pitch_bytes = pitch * (int64_t)sizeof(TI);
        frow = g_first;
        last_row = H - 1;
        src = reinterpret_cast<const char*>(img + (int64_t)clampi(g_first, H) * pitch + (int64_t)xs * 3);
        // prologue: the first NS rows, into consecutive slots from the current one
        uint32_t b = bar, d = dst, s = slot;
#pragma unroll 1
        for (int i = 0; i < NS && i < n; ++i) {
            bulk_issue_pred(lane == 0, b, d, src, kBytes);
            advance_src();
            ++fq;
            if (++s == NS) { s = 0; b = bar0; d = dst0; } else { b += 8; d += kBytes; }
        }
    }
    __device__ __forceinline__ void advance_src() {
        if (frow >= 0 && frow < last_row) src += pitch_bytes;  // rows below the image repeat row H-1
        ++frow;
    }
    // The next row's 24 channel values (as raw chunks); the slot is then refilled with the row NS
    // further on.
    __device__ __forceinline__ void take_raw(WideRaw<TI>& r) {
        bool ok = mbar_test(bar, phase);
        if (!__all_sync(kFull, ok)) {
            ok = warp_mbar_wait(bar, phase, lane);
            if (!ok && !bs.failed) { bs.failed = true; failed_q = tq; }
        }
        ++tq;
        constexpr int NQ = sizeof(TI) == 4 ? 6 : 3;
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const float4 t = lds128(lane_src + 16 * i);
            r.q[i] = make_uint4(__float_as_uint(t.x), __float_as_uint(t.y), __float_as_uint(t.z),
                                __float_as_uint(t.w));
        }
        __syncwarp();  // every lane has read the slot before the copy that overwrites it
        const bool more = fq < n;
        bulk_issue_pred(lane == 0 && more && !bs.failed, bar, dst, src, kBytes);
        if (more) { advance_src(); ++fq; }
        if (++slot == NS) {
            slot = 0; phase ^= 1u; bar = bar0; dst = dst0;
        } else {
            bar += 8; dst += kBytes;
        }
        lane_src = dst + lane * (kWCols * 3 * sizeof(TI));
    }
    __device__ __forceinline__ void finish() {
        if (bs.failed) {
            // Drain the copies issued but not seen complete (bounded waits), so that no bulk copy
            // still writes this warp's shared memory when the kernel returns.
            for (int q = failed_q; q < fq; ++q) {
                const uint32_t m = bs.seq + (uint32_t)q;
                mbar_wait(bar0 + 8 * (m % NS), (m / NS) & 1u);
            }
        }
        bs.seq += (uint32_t)n;
    }
};

// Per-lane staging of a warp's gray-row stream on an edge segment (16-byte aligned rows): each
// lane copies its own 24 channel values of a row into its place in the ring slot with cp.async,
// the pixels outside [0, W) zero-filled (never read from memory); NS-1 rows are in flight. Each
// lane reads back only what it copied itself, so no barrier or fence between lanes is needed.
template <typename TI, int NS>
struct WideLaneStage {
    static constexpr uint32_t kSlotBytes = kWSegLoad * 3 * sizeof(TI);
    static constexpr int kLaneBytes = kWCols * 3 * sizeof(TI);  // 96 (float32) or 48 (16-bit)
    const TI* img;
    int64_t pitch;
    int x, H, n;          // lane's first column, image rows, rows of the stream
    int g_first;          // image row (unclamped) of stream row 0
    int valid_bytes;      // bytes of the lane's 24 values inside the row
    uint32_t lane0;       // this lane's chunk of slot 0
    int fq = 0, tq = 0;   // next row to fetch, rows taken

    __device__ __forceinline__ WideLaneStage(const TI* img_, int64_t pitch_, int x_, int W, int H_, uint32_t ring0,
                                             int lane, int g_first_, int n_)
        : img(img_), pitch(pitch_), x(x_), H(H_), n(n_), g_first(g_first_) {
        const int npx = x < 0 ? 0 : (W - x >= kWCols ? kWCols : (W - x > 0 ? W - x : 0));
        valid_bytes = npx * 3 * (int)sizeof(TI);
        lane0 = ring0 + lane * kLaneBytes;
#pragma unroll 1
        for (int i = 0; i < NS - 1; ++i) fetch();
    }
    __device__ __forceinline__ void fetch() {
        if (fq < n) {
            const char* src = reinterpret_cast<const char*>(img + (int64_t)clampi(g_first + fq, H) * pitch +
                                                             (int64_t)(x < 0 ? 0 : x) * 3);
            const uint32_t dst = lane0 + (uint32_t)(fq % NS) * kSlotBytes;
#pragma unroll
            for (int i = 0; i < kLaneBytes / 16; ++i) {
                int nb = valid_bytes - 16 * i;
                nb = nb < 0 ? 0 : (nb > 16 ? 16 : nb);
                cp_async16(dst + 16 * i, nb > 0 ? src + 16 * i : src, nb);
            }
        }
        cp_async_commit();
        ++fq;
    }
    __device__ __forceinline__ void take_raw(WideRaw<TI>& r) {
        cp_async_wait<NS - 2>();  // the oldest row in flight has landed
        const uint32_t src = lane0 + (uint32_t)(tq % NS) * kSlotBytes;
        constexpr int NQ = kLaneBytes / 16;
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const float4 t = lds128(src + 16 * i);
            r.q[i] = make_uint4(__float_as_uint(t.x), __float_as_uint(t.y), __float_as_uint(t.z),
                                __float_as_uint(t.w));
        }
        ++tq;
        fetch();  // row tq + NS - 2 goes to the slot read one step earlier
    }
    __device__ __forceinline__ void finish() { cp_async_wait<0>(); }
};

// ---------------------------------------------------------------------------------------------
// Row sources of the wide strip, one per staging kind: each stages the gray rows of the strip
// (rows y0-2 .. y1+1, clamped) and runs wide_strip_core over the rows [y0, y1), handing every R
// row to store(y, R) on every lane (the forward stores it, the corner kernel suppresses
// non-maxima first).
// ---------------------------------------------------------------------------------------------

// Rows that are not 16-byte aligned: each lane loads its pixels of the next row element by
// element, one row ahead.
template <typename TI, bool EDGE, typename Store>
__device__ __forceinline__ void wide_rows_elem(const FwdArgs& a, const Params& P, int x, int y0, int y1,
                                               Store&& store) {
    const int H = a.H, W = a.W;
    const TI* img = static_cast<const TI*>(a.img);
    int row = y0 - 2;  // image row (unclamped) of the next gray row
    WideRaw<TI> buf;
    wide_load<TI, false>(img, a.img_pitch, clampi(row, H), x, W, buf);
    auto take = [&](float g10[10]) {
        float c[8];
        gray8<TI>(buf, c);
        ++row;
        wide_load<TI, false>(img, a.img_pitch, clampi(row, H), x, W, buf);
        widen10<EDGE>(c, g10, x, W);
    };
    wide_strip_core<EDGE>(P, x, W, H, y0, y1, take, store, [] { return true; });
}

// 16-byte aligned rows staged in registers: each lane loads its 8 pixels of the next row with
// 16-byte loads one row ahead (element by element where a lane straddles the image edge), and
// lane 0 prefetches the warp's span of the row kWidePfRows ahead into L2 with one bulk prefetch,
// so the register loads hit L2. Nothing waits on the prefetch.
template <typename TI, bool EDGE, typename Store>
__device__ __forceinline__ void wide_rows_pf(const FwdArgs& a, const Params& P, int lane, int x, int y0, int y1,
                                             Store&& store) {
    constexpr int K = kWidePfRows;
    const int H = a.H, W = a.W;
    const TI* img = static_cast<const TI*>(a.img);
    // the warp's 256 staged pixels clipped to the image, in whole 16-byte chunks
    const int xs = x - kWCols * lane;
    const int plo = xs < 0 ? 0 : xs, phi = xs + kWSegLoad < W ? xs + kWSegLoad : W;
    const uint32_t pbytes = (uint32_t)((phi - plo) * 3 * (int)sizeof(TI)) & ~15u;
    const char* prow = reinterpret_cast<const char*>(img + (int64_t)plo * 3);
    const int64_t pitch_b = a.img_pitch * (int64_t)sizeof(TI);
    SHINE_CHECK(a.dbg, pbytes <= (uint32_t)((phi - plo) * 3 * (int)sizeof(TI)), kDbgFwdStage);
    if constexpr (!EDGE) SHINE_CHECK(a.dbg, x >= 0 && x + kWCols <= W, kDbgFwdLoad);
    int pr = y0 - 2;  // next row to prefetch (unclamped)
    const uint32_t lead = lane == 0 && pbytes != 0;
    auto prefetch_next = [&]() {
        prefetch_l2_pred(lead && pr >= 0 && pr < H, prow + (int64_t)(pr < 0 ? 0 : pr) * pitch_b, pbytes);
        ++pr;
    };
#pragma unroll 1
    for (int i = 0; i < K; ++i) prefetch_next();
    int row = y0 - 2;  // image row (unclamped) of the next gray row
    WideRaw<TI> buf;
    wide_load<TI, true, !EDGE>(img, a.img_pitch, clampi(row, H), x, W, buf);
    auto take = [&](float g10[10]) {
        float c[8];
        gray8<TI>(buf, c);
        ++row;
        wide_load<TI, true, !EDGE>(img, a.img_pitch, clampi(row, H), x, W, buf);  // one row ahead
        prefetch_next();
        widen10<EDGE>(c, g10, x, W);
    };
    wide_strip_core<EDGE>(P, x, W, H, y0, y1, take, store, [] { return true; });
}

// An edge segment of a 16-byte aligned image, staged per lane by cp.async.
template <typename TI, int NS, typename Store>
__device__ __forceinline__ void wide_rows_edge(const FwdArgs& a, const Params& P, int lane, int x, int y0, int y1,
                                               uint32_t ring0, Store&& store) {
    const int H = a.H, W = a.W;
    const int n = (y1 == H ? y1 - y0 + 3 : y1 - y0 + 4);  // gray rows y0-2 .. min(y1+1, H)
    SHINE_CHECK(a.dbg, smem_in(ring0, NS * WideLaneStage<TI, NS>::kSlotBytes), kDbgSmem);
    WideLaneStage<TI, NS> src(static_cast<const TI*>(a.img), a.img_pitch, x, W, H, ring0, lane, y0 - 2, n);
    // a lane whose columns all lie outside the row copies nothing (zero-fill only)
    SHINE_CHECK(a.dbg, src.valid_bytes == 0 || (x >= 0 && (x + kWCols <= W ? kWCols : W - x) * 3 * (int)sizeof(TI) ==
                                                              src.valid_bytes),
                kDbgFwdStage);
    auto take = [&](float g10[10]) {
        WideRaw<TI> r;
        src.take_raw(r);
        float c[8];
        gray8<TI>(r, c);
        widen10<true>(c, g10, x, W);
    };
    wide_strip_core<true>(P, x, W, H, y0, y1, take, store, [] { return true; });
    src.finish();
}

// An interior segment of a 16-byte aligned image, staged by bulk copies.
template <typename TI, int NS, typename Store>
__device__ __forceinline__ void wide_rows_bulk(const FwdArgs& a, const Params& P, int lane, int x, int y0, int y1,
                                               uint32_t ring0, WideBulkState& bs, Store&& store) {
    const int H = a.H;
    const int n = (y1 == H ? y1 - y0 + 3 : y1 - y0 + 4);  // gray rows y0-2 .. min(y1+1, H)
    SHINE_CHECK(a.dbg, x - kWCols * lane >= 0 && x - kWCols * lane + kWSegLoad <= a.W, kDbgFwdStage);
    SHINE_CHECK(a.dbg, smem_in(ring0, NS * WideBulk<TI, NS>::kBytes), kDbgSmem);
    WideBulk<TI, NS> src(bs, static_cast<const TI*>(a.img), a.img_pitch, x - kWCols * lane, ring0, lane, y0 - 2, n, H);
    auto take = [&](float g10[10]) {
        WideRaw<TI> r;
        src.take_raw(r);
        float c[8];
        gray8<TI>(r, c);
        widen10<false>(c, g10, x, 0);
    };
    wide_strip_core<false>(P, x, a.W, H, y0, y1, take, store, [&] { return !bs.failed; });
    src.finish();
}

}  // namespace shine
