// Wide adjoint strip: one warp computes the vector-Jacobian product over one (column segment,
// row band) of a CLAMP image with 16-byte aligned rows, eight columns per lane; see
// harris_bwd.cu for the adjoint chain B1-B6.
//
// The arithmetic, and its order, is that of harris_bwd_strip.cuh (d img is bit-identical; the
// parameter cotangents are the same terms summed over a different partition). What changes is
// the shape of the work: a lane owns 8 adjacent columns and a warp 256 staged, 240 computed
// columns, so the fixed cost of a step is spread over twice as many pixels. The registers that
// doubles are found by keeping in registers only what every step reads and writes (the Sobel push
// partials, the running gS sums of the box adjoint, the running d gray rows of the transposed
// stencil, the weight-cotangent partial sums), and by moving to shared memory what a step touches
// once: the gray rows the weight cotangent pairs with gI row k (a 4-row ring), the Sobel rows of
// the product stage and of B4 (a 4-row ring) and the per-lane parameter-cotangent sums.
#pragma once

#include <type_traits>

#include "harris_bwd_strip.cuh"
#include "harris_common.cuh"
#include "harris_fwd_wide.cuh"
#include "harris_kernels.h"

namespace shine {

// Per-warp rings (besides the staging ring), slot-major; within a slot the lanes' entries of
// each 16-byte (or 8-byte) piece are contiguous, so every access of a warp is conflict-free.
//   gray slot:  [32 x values 0..3][32 x values 4..7][32 x (left, right) neighbour values]
//   Sobel slot: [32 x (I0, I1)][32 x (I2, I3)][32 x (I4, I5)][32 x (I6, I7)]
constexpr uint32_t kWGraySlot = kLanes * (16 + 16 + 8);
constexpr uint32_t kWSobelSlot = kLanes * 64;
constexpr uint32_t kWAccStride = 80;  // 19 floats per lane, 16-byte rows
constexpr uint32_t kWRingBytes = 4 * kWGraySlot + 4 * kWSobelSlot + kLanes * kWAccStride;

__device__ __forceinline__ void st_shared4(uint32_t a, float x, float y, float z, float w) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}
__device__ __forceinline__ void st_shared2(uint32_t a, float x, float y) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(x), "f"(y) : "memory");
}
__device__ __forceinline__ float2 ld_shared2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}

struct WRings {
    uint32_t gray, sobel, acc;  // this lane's entries of gray slot 0, Sobel slot 0, and its sums

    __device__ __forceinline__ void init(uint32_t base, int lane) {
        gray = base + lane * 16;
        sobel = base + 4 * kWGraySlot + lane * 16;
        acc = base + 4 * kWGraySlot + 4 * kWSobelSlot + lane * kWAccStride;
    }
    __device__ __forceinline__ void gray_get(uint32_t slot, int lane, float g[10]) const {
        const uint32_t a = gray + slot * kWGraySlot;
        const float4 lo = lds128(a), hi = lds128(a + kLanes * 16);
        const float2 h = ld_shared2(a + kLanes * 32 - lane * 8);
        g[0] = h.x;
        g[1] = lo.x; g[2] = lo.y; g[3] = lo.z; g[4] = lo.w;
        g[5] = hi.x; g[6] = hi.y; g[7] = hi.z; g[8] = hi.w;
        g[9] = h.y;
    }
    __device__ __forceinline__ void gray_put(uint32_t slot, int lane, const float g[10]) const {
        const uint32_t a = gray + slot * kWGraySlot;
        st_shared4(a, g[1], g[2], g[3], g[4]);
        st_shared4(a + kLanes * 16, g[5], g[6], g[7], g[8]);
        st_shared2(a + kLanes * 32 - lane * 8, g[0], g[9]);
    }
    __device__ __forceinline__ void sobel_get(uint32_t slot, float2 I[8]) const {
        const uint32_t a = sobel + slot * kWSobelSlot;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = lds128(a + q * (kLanes * 16));
            I[2 * q] = make_float2(v.x, v.y);
            I[2 * q + 1] = make_float2(v.z, v.w);
        }
    }
    __device__ __forceinline__ void sobel_put(uint32_t slot, const float2 I[8]) const {
        const uint32_t a = sobel + slot * kWSobelSlot;
#pragma unroll
        for (int q = 0; q < 4; ++q) st_shared4(a + q * (kLanes * 16), I[2 * q].x, I[2 * q].y, I[2 * q + 1].x, I[2 * q + 1].y);
    }
    __device__ __forceinline__ void acc_zero() const {
#pragma unroll
        for (int i = 0; i < 5; ++i) st_shared4(acc + 16 * i, 0.0f, 0.0f, 0.0f, 0.0f);
    }
    __device__ __forceinline__ void acc_add(const float v[kParamSlots]) const {
        float t[20];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float4 q = lds128(acc + 16 * i);
            t[4 * i] = q.x; t[4 * i + 1] = q.y; t[4 * i + 2] = q.z; t[4 * i + 3] = q.w;
        }
#pragma unroll
        for (int i = 0; i < kParamSlots; ++i) t[i] += v[i];
#pragma unroll
        for (int i = 0; i < 5; ++i) st_shared4(acc + 16 * i, t[4 * i], t[4 * i + 1], t[4 * i + 2], t[4 * i + 3]);
    }
    __device__ __forceinline__ void acc_get(float v[kParamSlots]) const {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float4 q = lds128(acc + 16 * i);
            const float t[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (4 * i + k < kParamSlots) v[4 * i + k] = t[k];
        }
    }
};

// The lane's 8 cotangent values of a staged row (16-bit or float32).
template <typename TG> struct WideCot { uint4 q[sizeof(TG) == 4 ? 2 : 1]; };
template <typename TG>
__device__ __forceinline__ void cot8(const WideCot<TG>& c, float gv[8]) {
    if constexpr (sizeof(TG) == 4) {
        gv[0] = __uint_as_float(c.q[0].x); gv[1] = __uint_as_float(c.q[0].y);
        gv[2] = __uint_as_float(c.q[0].z); gv[3] = __uint_as_float(c.q[0].w);
        gv[4] = __uint_as_float(c.q[1].x); gv[5] = __uint_as_float(c.q[1].y);
        gv[6] = __uint_as_float(c.q[1].z); gv[7] = __uint_as_float(c.q[1].w);
    } else {
        const uint32_t w[4] = {c.q[0].x, c.q[0].y, c.q[0].z, c.q[0].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            gv[2 * i] = Unpack16<TG>::lo(w[i]);
            gv[2 * i + 1] = Unpack16<TG>::hi(w[i]);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Staging: step s delivers image row y0-4+s (clamped) and cotangent row y0-6+s (zero outside the
// image) of the warp's 256-column span into a ring slot; a slot holds the image span then the
// cotangent span, each lane's pieces side by side.
//   WAdjBulk:  interior segments: lane 0 moves both spans of a row with two bulk copies completing
//              on the slot's mbarrier (bounded waits).
//   WAdjLanes: edge segments: every lane copies its own pieces with cp.async, the pixels outside
//              [0, W) zero-filled; each lane reads back only what it copied.
// ---------------------------------------------------------------------------------------------
template <typename TI, typename TG>
struct WSlot {
    static constexpr uint32_t kImg = kWSegLoad * 3 * sizeof(TI);  // image span bytes
    static constexpr uint32_t kCot = kWSegLoad * sizeof(TG);      // cotangent span bytes
    static constexpr uint32_t kBytes = kImg + kCot;
    static constexpr uint32_t kLaneImg = kWCols * 3 * sizeof(TI);  // 48 or 96
    static constexpr uint32_t kLaneCot = kWCols * sizeof(TG);      // 16 or 32

    // The lane's pieces of a slot (shared address of the slot's start). Pieces of 32 or 96 bytes
    // (float32) put the 8 lanes of a quarter warp on only 4 of the 8 16-byte bank groups; lanes
    // 4..7 of each quarter therefore read the 16-byte chunks of each pair in swapped order (which
    // lands them on the other 4 groups) and swap the pair back in registers.
    __device__ __forceinline__ static uint4 pick(bool swap, const uint4& a, const uint4& b) {
        return make_uint4(swap ? b.x : a.x, swap ? b.y : a.y, swap ? b.z : a.z, swap ? b.w : a.w);
    }
    __device__ __forceinline__ static void read(uint32_t slot, int lane, bool g_in, WideRaw<TI>& r, float gv[8]) {
        constexpr int NQ = kLaneImg / 16;
        constexpr bool kSwizzle = SHINE_WIDE_BWD_SWAP_PAIRS && sizeof(TI) == 4;
        const uint32_t im = slot + lane * kLaneImg;
        const uint32_t flip = kSwizzle ? (uint32_t)(lane >> 2) & 1u : 0u;
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const float4 t = lds128(im + 16 * ((uint32_t)i ^ flip));
            r.q[i] = make_uint4(__float_as_uint(t.x), __float_as_uint(t.y), __float_as_uint(t.z), __float_as_uint(t.w));
        }
        if constexpr (kSwizzle) {
#pragma unroll
            for (int i = 0; i < NQ; i += 2) {
                const uint4 a = r.q[i], b = r.q[i + 1];
                r.q[i] = pick(flip, a, b);
                r.q[i + 1] = pick(flip, b, a);
            }
        }
        if (g_in) {
            WideCot<TG> c;
            const uint32_t co = slot + kImg + lane * kLaneCot;
            constexpr bool kSwizzleG = SHINE_WIDE_BWD_SWAP_PAIRS && sizeof(TG) == 4;
            const uint32_t gflip = kSwizzleG ? (uint32_t)(lane >> 2) & 1u : 0u;
#pragma unroll
            for (int i = 0; i < (int)(kLaneCot / 16); ++i) {
                const float4 t = lds128(co + 16 * ((uint32_t)i ^ gflip));
                c.q[i] = make_uint4(__float_as_uint(t.x), __float_as_uint(t.y), __float_as_uint(t.z), __float_as_uint(t.w));
            }
            if constexpr (kSwizzleG) {
                const uint4 a = c.q[0], b = c.q[1];
                c.q[0] = pick(gflip, a, b);
                c.q[1] = pick(gflip, b, a);
            }
            cot8<TG>(c, gv);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) gv[j] = 0.0f;
        }
    }
};

template <typename TI, typename TG, int NS>
struct WAdjBulk {
    using SL = WSlot<TI, TG>;
    BulkState& bs;
    const int lane, n, H, gho;
    uint32_t slot, phase, bar, dst;  // current slot
    uint32_t bar0, dst0;             // slot 0
    const char* isrc;                // image row of the next copy
    const char* gsrc;                // cotangent row of the next copy
    int64_t ipitch, gpitch;          // bytes
    int fq = 0, fr;                  // next stream row to fetch, its image row (unclamped)
    int last_issued = -1, last_done = -1;

    __device__ __forceinline__ WAdjBulk(BulkState& bs_, const BwdArgs& a, uint32_t ring0, int lane_, int xs, int r_first,
                                        int n_)
        : bs(bs_), lane(lane_), n(n_), H(a.H), gho(a.gho) {
        slot = bs.seq % NS;
        phase = (bs.seq / NS) & 1u;
        bar0 = bs.bars;
        dst0 = ring0;
        bar = bar0 + 8 * slot;
        dst = dst0 + slot * SL::kBytes;
        ipitch = a.img_pitch * (int64_t)sizeof(TI);
        gpitch = a.gout_pitch * (int64_t)sizeof(TG);
        fr = r_first;
        isrc = reinterpret_cast<const char*>(static_cast<const TI*>(a.img) + (int64_t)clampi(r_first, H) * a.img_pitch +
                                             (int64_t)xs * 3);
        const int gy = r_first - 2;
        gsrc = reinterpret_cast<const char*>(static_cast<const TG*>(a.gout) + (int64_t)(gy < 0 ? 0 : gy) * a.gout_pitch +
                                             xs);
        uint32_t b = bar, d = dst, sl = slot;
#pragma unroll 1
        for (int i = 0; i < NS - 1 && fq < n; ++i) {
            issue(b, d);
            if (++sl == NS) { sl = 0; b = bar0; d = dst0; } else { b += 8; d += SL::kBytes; }
        }
    }
    __device__ __forceinline__ void issue(uint32_t b, uint32_t d) {
        const int gy = fr - 2;
        const bool g_in = gy >= 0 && gy < gho;
        if (lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(b, SL::kImg + (g_in ? SL::kCot : 0));
            bulk_copy_g2s(d, isrc, SL::kImg, b);
            if (g_in) bulk_copy_g2s(d + SL::kImg, gsrc, SL::kCot, b);
        }
        last_issued = fq;
        ++fq;
        if (fr >= 0 && fr < H - 1) isrc += ipitch;  // rows beyond the image repeat row H-1
        if (gy >= 0) gsrc += gpitch;
        ++fr;
    }
    template <bool G_IN>
    __device__ __forceinline__ void take(int s, int r, WideRaw<TI>& raw, float gv[8]) {
        const bool ok = __all_sync(kFull, mbar_wait(bar, phase));
        if (ok) last_done = s;
        else bs.failed = true;
        const int gy = r - 2;
        SL::read(dst, lane, G_IN || (gy >= 0 && gy < gho), raw, gv);
        __syncwarp();  // every lane has read the slot that the next copy overwrites
        // row s + NS - 1 goes to the slot of row s - 1 (free since the previous step)
        const uint32_t pb = slot == 0 ? bar0 + 8 * (NS - 1) : bar - 8;
        const uint32_t pd = slot == 0 ? dst0 + (NS - 1) * SL::kBytes : dst - SL::kBytes;
        if (ok && fq < n) issue(pb, pd);
        if (++slot == NS) {
            slot = 0; phase ^= 1u; bar = bar0; dst = dst0;
        } else {
            bar += 8; dst += SL::kBytes;
        }
    }
    __device__ __forceinline__ void finish() {
        if (bs.failed) {
            // Drain the copies issued but not waited for, with bounded waits, so that no bulk
            // copy still writes this warp's shared memory when the kernel returns.
            for (int s2 = last_done + 1; s2 <= last_issued; ++s2) {
                const uint32_t q = bs.seq + s2;
                mbar_wait(bar0 + 8 * (q % NS), (q / NS) & 1u);
            }
        }
        bs.seq += (uint32_t)n;
    }
};

template <typename TI, typename TG, int NS>
struct WAdjLanes {
    using SL = WSlot<TI, TG>;
    const TI* img;
    const TG* gout;
    int64_t ipitch, gpitch;  // elements
    const int lane, H, gho, r_first, n;
    int x, vbytes_img, vbytes_cot;  // lane's first column; bytes of its pieces inside the image
    uint32_t ring0;
    int fq = 0;

    __device__ __forceinline__ WAdjLanes(const BwdArgs& a, uint32_t ring0_, int lane_, int x_, int r_first_, int n_)
        : img(static_cast<const TI*>(a.img)), gout(static_cast<const TG*>(a.gout)), ipitch(a.img_pitch),
          gpitch(a.gout_pitch), lane(lane_), H(a.H), gho(a.gho), r_first(r_first_), n(n_), x(x_), ring0(ring0_) {
        const int npx = x < 0 ? 0 : (a.W - x >= kWCols ? kWCols : (a.W - x > 0 ? a.W - x : 0));
        vbytes_img = npx * 3 * (int)sizeof(TI);
        vbytes_cot = npx * (int)sizeof(TG);
#pragma unroll 1
        for (int i = 0; i < NS - 1; ++i) fetch();
    }
    __device__ __forceinline__ void fetch() {
        if (fq < n) {
            const uint32_t slot = ring0 + (uint32_t)(fq % NS) * SL::kBytes;
            const int r = r_first + fq, gy = r - 2;
            const int xc = x < 0 ? 0 : x;
            const char* isrc = reinterpret_cast<const char*>(img + (int64_t)clampi(r, H) * ipitch + (int64_t)xc * 3);
#pragma unroll
            for (int i = 0; i < (int)(SL::kLaneImg / 16); ++i) {
                int nb = vbytes_img - 16 * i;
                nb = nb < 0 ? 0 : (nb > 16 ? 16 : nb);
                cp_async16(slot + lane * SL::kLaneImg + 16 * i, nb > 0 ? isrc + 16 * i : isrc, nb);
            }
            const bool g_in = gy >= 0 && gy < gho;
            const char* gsrc = reinterpret_cast<const char*>(gout + (int64_t)(g_in ? gy : 0) * gpitch + xc);
#pragma unroll
            for (int i = 0; i < (int)(SL::kLaneCot / 16); ++i) {
                int nb = g_in ? vbytes_cot - 16 * i : 0;
                nb = nb < 0 ? 0 : (nb > 16 ? 16 : nb);
                cp_async16(slot + SL::kImg + lane * SL::kLaneCot + 16 * i, nb > 0 ? gsrc + 16 * i : gsrc, nb);
            }
        }
        cp_async_commit();
        ++fq;
    }
    template <bool G_IN>
    __device__ __forceinline__ void take(int s, int, WideRaw<TI>& raw, float gv[8]) {
        cp_async_wait<NS - 2>();  // the oldest row in flight has landed
        // zero-filled outside the cotangent's rows and columns, so it is read as it is
        SL::read(ring0 + (uint32_t)(s % NS) * SL::kBytes, lane, true, raw, gv);
        fetch();  // row s + NS - 1 goes to the slot read one step earlier
    }
    __device__ __forceinline__ void finish() { cp_async_wait<0>(); }
};

// ---------------------------------------------------------------------------------------------
// The strip: rows y0 .. y1-1 of the segment whose lane-1 column is x + 8 (x = the lane's first
// column). The strip's parameter-cotangent terms are added into the lane's shared-memory sums.
// ---------------------------------------------------------------------------------------------
// WITH_R: also store R (computed anyway in B1) at the rows this warp owns into a.rout when it is
// given, for the fused forward+backward pass (CLAMP: the output has the image's geometry);
// a.rout_vec allows 16-byte stores of a lane's 8 values.
template <typename TI, bool EDGE, bool BULK, bool WITH_R, typename Src>
__device__ __forceinline__ void wide_adj_strip(const BwdArgs& a, const Params& P, int lane, int x, int y0, int y1,
                                               Src& src, const WRings& rg, const bool* failed) {
    const int H = a.H, W = a.W;
    const bool producer = lane >= 1 && lane <= 30;
    const int r_first = y0 - 4;
    const int nrows = y1 - y0 + 8;  // image rows y0-4 .. y1+3, cotangent rows y0-6 .. y1+1

    bool cin[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) cin[j] = !EDGE || (x + j >= 0 && x + j < W);
    const bool full = !EDGE || (x >= 0 && x + kWCols <= W);

    float2 P1[8], P2[8];   // Sobel push partials (rows r and r+1)
    float2 qa[8], qb[8];   // running gS sums of the box adjoint (xx, yy): rows k-1 + k, row k
    float qaq[8], qbq[8];  // the same for xy
    float2 ga1[8], ga2[8]; // d gray of rows u+1 and u+2 so far, x and y weight planes apart
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        P1[j] = P2[j] = qa[j] = qb[j] = ga1[j] = ga2[j] = make_float2(0.0f, 0.0f);
        qaq[j] = qbq[j] = 0.0f;
    }
    TI* gimg = static_cast<TI*>(a.gimg);
    const float kc[3] = {kGrayR, kGrayG, kGrayB};
    constexpr int kFlushRows = 16;
    float2 partw[9];
    float partk = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) partw[i] = make_float2(0.0f, 0.0f);
    auto flush = [&]() {
        float v[kParamSlots];
        v[0] = partk;
#pragma unroll
        for (int i = 0; i < 9; ++i) { v[1 + i] = partw[i].x; v[10 + i] = partw[i].y; }
        rg.acc_add(v);
        partk = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) partw[i] = make_float2(0.0f, 0.0f);
    };

    auto step = [&](auto fast_tag, int s) {
        constexpr bool FAST = decltype(fast_tag)::value;
        const int r = r_first + s;
        // ring slots: gray row r-4 (and then row r) at s & 3, rows r-3, r-2 after it; Sobel row
        // r-1 at (s + 3) & 3, rows r-3, r-2 at (s + 1) & 3, (s + 2) & 3
        const uint32_t s0 = (uint32_t)s & 3u, s1 = (uint32_t)(s + 1) & 3u, s2 = (uint32_t)(s + 2) & 3u,
                       s3 = (uint32_t)(s + 3) & 3u;
        float g10[10], gv[8];
        {
            WideRaw<TI> raw;
            src.template take<FAST && BULK>(s, r, raw, gv);
            float c[8];
            gray8<TI>(raw, c);
            widen10<EDGE>(c, g10, x, W);
        }
        // B1: gray row r completes Sobel row r-1 (push form), which goes to the Sobel ring.
        float2 I2[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float2 sv = P1[j], p1 = P2[j], p2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float2 gg = dup2(g10[j + b]);
                sv = __ffma2_rn(P.w[6 + b], gg, sv);
                p1 = __ffma2_rn(P.w[3 + b], gg, p1);
                p2 = __ffma2_rn(P.w[b], gg, p2);
            }
            I2[j] = sv; P1[j] = p1; P2[j] = p2;
        }
        rg.sobel_put(s3, I2);
        // B1: S at row r-2 from products at rows r-3, r-2, r-1 (clamped at their stage).
        const int sr = r - 2;
        float2 S2[8];  // (Sxx, Syy)
        float Sxy[8];
        {
            float2 v2[8];
            float vxy[8];
            {
                float2 I0[8], I1[8];
                rg.sobel_get(s1, I0);
                rg.sobel_get(s2, I1);
                const bool top = !FAST && sr == 0, bot = !FAST && sr == H - 1;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float2 A = top ? I1[j] : I0[j], B = bot ? I1[j] : I2[j], m = I1[j];
                    v2[j] = __ffma2_rn(B, B, __ffma2_rn(m, m, __fmul2_rn(A, A)));
                    vxy[j] = fmaf(B.x, B.y, fmaf(m.x, m.y, __fmul_rn(A.x, A.y)));
                }
            }
            hbox8<EDGE>(v2, S2, x, W);
            hbox8<EDGE>(vxy, Sxy, x, W);
        }
        const bool own_row = FAST || (sr >= y0 && sr < y1);
        if constexpr (WITH_R) {
            // A5 at row sr, bit-identical to the forward's R (same sums in the same order)
            if (own_row && producer && a.rout != nullptr) {
                float R[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) R[j] = response(S2[j].x, Sxy[j], S2[j].y, P.kappa);
                SHINE_CHECK(a.dbg, sr >= 0 && sr < H && (!full || !a.rout_vec || (x >= 0 && x + kWCols <= W)),
                            kDbgBwdStore);
                TI* orow = static_cast<TI*>(a.rout) + (int64_t)sr * a.rout_pitch;
                if (full && a.rout_vec) {
                    store8(orow + x, R);
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (cin[j]) orow[x + j] = Conv<TI>::st(R[j]);
                }
            }
        }
        // B2: gS at row r-2 and the d kappa terms.
        float2 gsn[8];
        float gqn[8];
        {
            float dk[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float tr = S2[j].x + S2[j].y;
                const float g = gv[j];
                const float k2 = 2.0f * P.kappa * tr;
                gsn[j] = make_float2(g * (S2[j].y - k2), g * (S2[j].x - k2));
                gqn[j] = -2.0f * g * Sxy[j];
                dk[j] = -g * tr * tr;
            }
            if (own_row) partk += ((dk[0] + dk[1]) + (dk[2] + dk[3])) + ((dk[4] + dk[5]) + (dk[6] + dk[7]));
        }
        // B3: gP at row k = r-3 = clamped box sum of gS rows k-1, k, k+1.
        const int k = r - 3;
        float2 gp2[8];
        float gpq[8];
        {
            float2 vg2[8];
            float vgq[8];
            if (!FAST && (k == 0 || k == H - 1)) {
                const bool top = k == 0, bot = k == H - 1;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    vg2[j] = __fadd2_rn(top ? __fadd2_rn(qb[j], qb[j]) : qa[j], bot ? qb[j] : gsn[j]);
                    vgq[j] = (top ? qbq[j] + qbq[j] : qaq[j]) + (bot ? qbq[j] : gqn[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    vg2[j] = __fadd2_rn(qa[j], gsn[j]);
                    vgq[j] = qaq[j] + gqn[j];
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                qa[j] = __fadd2_rn(qb[j], gsn[j]);
                qb[j] = gsn[j];
                qaq[j] = qbq[j] + gqn[j];
                qbq[j] = gqn[j];
            }
            hbox8<EDGE>(vg2, gp2, x, W);
            hbox8<EDGE>(vgq, gpq, x, W);
        }
        // B4: gI at row k (zero outside the image: the padded domain of B5).
        float2 gI[8];
        if (FAST || (k >= 0 && k < H)) {
            float2 I0[8];
            rg.sobel_get(s1, I0);  // Sobel row k
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float2 i0 = I0[j];
                const float vx = fmaf(2.0f * i0.x, gp2[j].x, i0.y * gpq[j]);
                const float vy = fmaf(i0.x, gpq[j], 2.0f * i0.y * gp2[j].y);
                gI[j] = make_float2(cin[j] ? vx : 0.0f, cin[j] ? vy : 0.0f);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) gI[j] = make_float2(0.0f, 0.0f);
        }
        // B5 (weights): (d Wx[a][b], d Wy[a][b]) += gI(k, c) * G(clamp(k + a - 1), clamp(c + b - 1))
        // for the rows this warp owns; gray rows k-1, k, k+1 (image rows r-4 .. r-2) come from
        // the gray ring.
        if (FAST || (k >= y0 && k < y1)) {
            float G[10];
            rg.gray_get(s0, lane, G);  // row k-1 = r-4
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int b = 0; b < 3; ++b) partw[b] = __ffma2_rn(gI[j], dup2(G[j + b]), partw[b]);
            rg.gray_get(s1, lane, G);  // row k
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int b = 0; b < 3; ++b) partw[3 + b] = __ffma2_rn(gI[j], dup2(G[j + b]), partw[3 + b]);
            rg.gray_get(s2, lane, G);  // row k+1
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int b = 0; b < 3; ++b) partw[6 + b] = __ffma2_rn(gI[j], dup2(G[j + b]), partw[6 + b]);
        }
        rg.gray_put(s0, lane, g10);  // row r takes the slot of row r-4
        float2 gin[10];
        widen10<false>(gI, gin, x, W);

        // B5 (image) + B6 at row u = r-4: the transposed stencil in push form.
        const int u = r - 4;
        float2 done[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float2 d = ga1[j], n1 = ga2[j], n2 = make_float2(0.0f, 0.0f);
            const float2 below = ga2[j];  // d gray of row u+1 so far
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const int c = j - b + 2;  // gI column (lane column j) - b + 1 in widened coordinates
                d = __ffma2_rn(P.w[b], gin[c], d);
                n1 = __ffma2_rn(P.w[3 + b], gin[c], n1);
                n2 = __ffma2_rn(P.w[6 + b], gin[c], n2);
            }
            if (!FAST && u == H - 1) d = __fadd2_rn(d, below);
            if (!FAST && k == 0) n1 = __fadd2_rn(n1, d);
            done[j] = d; ga1[j] = n1; ga2[j] = n2;
        }
        if (FAST || u >= y0) {
            float gg[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) gg[j] = done[j].x + done[j].y;
            if constexpr (EDGE) {
                // padded column -1 folds onto column 0, column W onto column W-1
                float r10[10];
                widen10<false>(gg, r10, x, W);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (x + j == 0) gg[j] += r10[j];
                    if (x + j == W - 1) gg[j] += r10[j + 2];
                }
            }
            if (producer) {
                SHINE_CHECK(a.dbg, u >= 0 && u < H && (!full || !a.gimg_vec || (x >= 0 && x + kWCols <= W)), kDbgBwdStore);
                TI* orow = gimg + (int64_t)u * a.gimg_pitch + (int64_t)x * 3;
                float o[24];
#pragma unroll
                for (int j = 0; j < 8; ++j)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) o[3 * j + ch] = kc[ch] * gg[j];
                if (full && a.gimg_vec) {
                    if constexpr (sizeof(TI) == 4) {
                        float4* dd = reinterpret_cast<float4*>(orow);
#pragma unroll
                        for (int i = 0; i < 6; ++i) dd[i] = make_float4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
                    } else {
                        uint32_t w[12];
#pragma unroll
                        for (int i = 0; i < 12; ++i) {
                            TI t2[2] = {Conv<TI>::st(o[2 * i]), Conv<TI>::st(o[2 * i + 1])};
                            w[i] = *reinterpret_cast<const uint32_t*>(t2);
                        }
                        uint4* dd = reinterpret_cast<uint4*>(orow);
#pragma unroll
                        for (int i = 0; i < 3; ++i) dd[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (cin[j])
#pragma unroll
                            for (int ch = 0; ch < 3; ++ch) orow[3 * j + ch] = Conv<TI>::st(o[3 * j + ch]);
                }
            }
        }
    };
    const std::integral_constant<bool, false> general{};
    const std::integral_constant<bool, true> fast{};
    // Fast steps: u = r - 4 >= max(y0, 2) and S row r - 2 <= min(y1 - 1, H - 3).
    const int s_a = 8 + (y0 < 2 ? 2 - y0 : 0);
    const int s_b = (y1 - 3 < H - 5 ? y1 - 3 : H - 5) - y0 + 9;  // exclusive
    int since_flush = 0;
    // Steps 0 and 1 only fill the Sobel push partials and the rings.
#pragma unroll 1
    for (int s = 0; s < nrows; ++s) {
        if (BULK && *failed) break;
        if (s >= s_a && s < s_b) step(fast, s);
        else step(general, s);
        if (s >= 2 && ++since_flush == kFlushRows) { flush(); since_flush = 0; }
    }
    flush();
    src.finish();
}

}  // namespace shine
