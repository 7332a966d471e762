// Forward strip: one warp computes R over one (column segment, row band) of one image.
//
// Per output row y the warp takes one image row out of its staging (loaded several rows
// earlier), makes its gray row, the Sobel row y+1, the three product sums over rows y-1..y+1
// (the slide2D + reduce of A4 done vertically in registers first, then horizontally with two
// shuffles per plane) and R[y]. HBM traffic is the image once and R once; nothing else leaves
// the registers.
#pragma once

#include "harris_common.cuh"
#include "harris_kernels.h"

namespace shine {

// Forward staging state of bulk (TMA) copies, carried by a warp from strip to strip.
struct FwdBulk {
    uint32_t bars;  // shared address of this warp's NS barriers
    uint32_t seq;   // rows staged by this warp so far (row n sits in slot n % NS)
    bool failed;    // a bounded wait gave up
};

// The 6-wide gray row (clamped at the image border on EDGE warps) of the lane's 12 channel values.
template <bool EDGE>
__device__ __forceinline__ void gray_row(const float v[12], float g6[6], int x, int W) {
    float c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) c[j] = gray_of(v[3 * j], v[3 * j + 1], v[3 * j + 2]);
    make_row6(c, g6);
    if constexpr (EDGE) clamp_row6(g6, x, W);
}

template <typename TO>
__device__ __forceinline__ void store4(TO* p, const float R[4]) {
    if constexpr (sizeof(TO) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(R[0], R[1], R[2], R[3]);
    } else {
        TO o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = Conv<TO>::st(R[j]);
        *reinterpret_cast<uint2*>(p) = *reinterpret_cast<uint2*>(o);
    }
}

// The strip walk shared by both staging methods: y0 .. y1-1 are the output rows, take(q, k,
// g6) delivers sequence row q (image row y0 - 2 + q, clamped) as a gray row (k = q mod D, a
// constant in unrolled code), store(y, R) writes R[y], and go() is false once the staging has
// failed. Per output row: one gray row in, one Sobel row completed, one row of product sums
// completed, the horizontal box sums, the response. The running sums are updated in place, so
// the loop keeps no window of rows that would have to be shifted.
template <bool EDGE, int D, typename Take, typename Store, typename Go>
__device__ __forceinline__ void fwd_strip_core(const Params& P, int x, int W, int H, int y0, int y1, Take&& take,
                                               Store&& store, Go&& go) {
    StripRun st;
#pragma unroll
    for (int j = 0; j < 4; ++j) st.P1[j] = st.P2[j] = make_float2(0.0f, 0.0f);
    float g[6];
    take(0, 0 % D, g);
    push_gray(P, g, st);
    take(1, 1 % D, g);
    push_gray(P, g, st);
    take(2, 2 % D, g);
    push_gray(P, g, st);  // S = Sobel row y0-1
    square_S(st);
    take(3, 3 % D, g);
    push_gray(P, g, st);  // S = Sobel row y0
    if (y0 == 0) square_S(st);  // the product row above the image is the clamped copy of row 0
    add_S(st);
    square_S(st);
#pragma unroll 1
    for (int y = y0; y < y1; y += D) {
        if (!go()) break;
#pragma unroll
        for (int u = 0; u < D; ++u) {
            const int yy = y + u;
            if (u == 0 || yy < y1) {
                take(yy - y0 + 4, (4 + u) % D, g);  // gray row yy+2
                // S = Sobel row yy+1; at the bottom image row S stays at row yy, the clamped
                // row below it at the product stage.
                if (yy != H - 1) push_gray(P, g, st);
                float2 v2[4];
                float vxy[4];
                push_products(st, v2, vxy);
                float2 s2[4];
                float sxy[4];
                horizontal_box<EDGE>(v2, s2, x, W);
                horizontal_box<EDGE>(vxy, sxy, x, W);
                float R[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) R[j] = response(s2[j].x, sxy[j], s2[j].y, P.kappa);
                store(yy, R);
            }
        }
    }
}

// Rows y0 .. y1-1 of a strip with register staging (D rows in flight), for every segment kind
// and alignment; store(y, R) receives each row's R at the lane's 4 columns.
template <typename TI, int D, bool EDGE, bool ALIGNED, typename Store>
__device__ __forceinline__ void fwd_rows(const FwdArgs& a, const Params& P, int x, int y0, int y1, Store&& store) {
    const int H = a.H, W = a.W;
    const RegRows<TI, EDGE, ALIGNED> rows(static_cast<const TI*>(a.img), a.img_pitch, x, W);
    const int r_first = y0 - 2;     // sequence row q is image row r_first + q (clamped)
    const int nrows = y1 - y0 + 4;  // gray rows y0-2 .. y1+1
    RawRow<TI> buf[D];              // buf[q % D] holds sequence row q until taken
#pragma unroll
    for (int d = 0; d < D; ++d) rows.load(clampi(r_first + d, H), buf[d]);
    auto take = [&](int q, int k, float g6[6]) {
        float v[12];
        RegRows<TI, EDGE, ALIGNED>::unpack(buf[k], v);
        if (q + D < nrows) rows.load(clampi(r_first + q + D, H), buf[k]);
        gray_row<EDGE>(v, g6, x, W);
    };
    fwd_strip_core<EDGE, D>(P, x, W, H, y0, y1, take, store, [] { return true; });
}

// Bulk (TMA) staging of a warp's stream of gray rows g_first .. g_first+n-1 of an interior
// segment with 16-byte aligned rows: lane 0 moves each row's whole 128-pixel segment into a
// ring of NS shared-memory slots with one copy completing on the slot's mbarrier, so NS rows are
// in flight without holding registers. The ring position and the row pointers are
// strength-reduced: per row the warp does the barrier wait, three shared loads, one copy issue
// and the gray arithmetic. finish() must follow the last take().
template <typename TI, int NS>
struct BulkGray {
    static constexpr int kSlot = kLanes * 12;  // elements per slot
    static constexpr uint32_t kBytes = kSegLoad * 3 * sizeof(TI);
    const FwdArgs& a;
    FwdBulk& bulk;
    const int lane, x, g_first, n;
    const TI* seg;
    uint32_t ring0, lane_ring, seq0, slot, phase, fslot;
    int fq = 0, tq = 0, failed_q = 0;  // next row to fetch; rows taken; first row whose wait gave up

    __device__ __forceinline__ BulkGray(const FwdArgs& a_, FwdBulk& bulk_, const TI* ring, int lane_, int x_,
                                        int g_first_, int n_)
        : a(a_), bulk(bulk_), lane(lane_), x(x_), g_first(g_first_), n(n_) {
        seg = static_cast<const TI*>(a.img) + (int64_t)(x - 4 * lane) * 3;
        ring0 = smem_u32(ring - lane * 12);  // slot 0 of the warp's ring
        lane_ring = smem_u32(ring);          // this lane's 12 elements of slot 0
        seq0 = bulk.seq;
        slot = seq0 % NS;
        phase = (seq0 / NS) & 1u;
        fslot = slot;
#pragma unroll 1
        for (int i = 0; i < NS && fq < n; ++i) fetch();
    }
    // Row fq goes to the slot of row fq - NS.
    __device__ __forceinline__ void fetch() {
        if (lane == 0) {
            const TI* src = seg + (int64_t)clampi(g_first + fq, a.H) * a.img_pitch;
            const uint32_t bar = bulk.bars + 8 * fslot;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, kBytes);
            bulk_copy_g2s(ring0 + fslot * (kSlot * (uint32_t)sizeof(TI)), src, kBytes, bar);
        }
        ++fq;
        fslot = fslot + 1 == NS ? 0 : fslot + 1;
    }
    // The next row as a gray row; its slot is then refilled with the row NS further on.
    __device__ __forceinline__ void take(float g6[6]) {
        const bool ok = warp_mbar_wait(bulk.bars + 8 * slot, phase, lane);
        if (!ok && !bulk.failed) { bulk.failed = true; failed_q = tq; }
        ++tq;
        float v[12];
        const uint32_t src = lane_ring + slot * (kSlot * (uint32_t)sizeof(TI));
        if constexpr (sizeof(TI) == 4) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float4 t = lds128(src + 16 * i);
                v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
            }
        } else {
            RawRow<TI> r;
#pragma unroll
            for (int i = 0; i < 3; ++i) r.q[i] = lds64(src + 8 * i);
            RegRows<TI, false, true>::unpack(r, v);
        }
        __syncwarp();  // every lane has read the slot before the copy that overwrites it
        if (!bulk.failed && fq < n) fetch();
        if (++slot == NS) { slot = 0; phase ^= 1u; }
        gray_row<false>(v, g6, x, 0);
    }
    __device__ __forceinline__ void finish() {
        if (bulk.failed) {
            // Drain the copies issued but not seen complete (bounded waits), so that no bulk copy
            // still writes this warp's shared memory when the kernel returns.
            for (int q = failed_q; q < fq; ++q) {
                const uint32_t m = seq0 + (uint32_t)q;
                mbar_wait(bulk.bars + 8 * (m % NS), (m / NS) & 1u);
            }
        }
        bulk.seq = seq0 + (uint32_t)n;
    }
};

// Forward strip that writes R (register staging; any segment): the batched forward-only mode.
template <typename TI, typename TO, int D, bool EDGE, bool ALIGNED>
__device__ __forceinline__ void fwd_strip(const FwdArgs& a, const Params& P, int lane, int x, int y0, int y1) {
    TO* out = static_cast<TO*>(a.out);
    const bool producer = lane >= 1 && lane <= 30;
    fwd_rows<TI, D, EDGE, ALIGNED>(a, P, x, y0, y1, [&](int y, const float R[4]) {
        if (!producer) return;
        TO* orow = out + (int64_t)(y - a.oy) * a.out_pitch;
        if (!EDGE && a.out_vec) {
            store4(orow + x, R);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = x + j;
                if (c >= a.xlo && c < a.xhi) orow[c - a.ox] = Conv<TO>::st(R[j]);
            }
        }
    });
}

}  // namespace shine
