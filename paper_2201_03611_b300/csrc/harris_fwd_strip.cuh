// Forward strip: one warp computes R over one (column segment, row band) of one image.
//
// Per output row y the warp takes one image row out of its register staging (loaded D rows
// earlier, then refilled with the row D further down), makes its gray row, the Sobel row y+1,
// the three product sums over rows y-1..y+1 (the slide2D + reduce of A4 done vertically in
// registers first, then horizontally with two shuffles per plane) and R[y]. HBM traffic is the
// image once and R once; nothing else leaves the registers.
#pragma once

#include "harris_common.cuh"
#include "harris_kernels.h"

namespace shine {

// Forward staging state of bulk (TMA) copies: see BulkState in harris_bwd_strip.cuh.
struct FwdBulk {
    uint32_t bars;  // shared address of this warp's NS barriers
    uint32_t seq;   // rows staged by this warp so far
    bool failed;    // a bounded wait gave up
};

// TMA = false: rows are staged in registers (D rows in flight). TMA = true (interior segments
// with 16-byte aligned rows): lane 0 moves each row's whole 128-pixel segment into a ring of NS
// shared-memory slots with one bulk copy completing on the slot's mbarrier; NS - 1 rows are in
// flight without holding registers.
template <typename TI, typename TO, int D, bool EDGE, bool ALIGNED, bool TMA = false, int NS = 1>
__device__ __forceinline__ void fwd_strip(const FwdArgs& a, const Params& P, int lane, int x, int y0,
                                          int y1, TI* ring = nullptr, FwdBulk* bulk = nullptr) {
    const int H = a.H, W = a.W;
    const RegRows<TI, EDGE, ALIGNED> rows(static_cast<const TI*>(a.img), a.img_pitch, x, W);
    const int r_first = y0 - 2;         // sequence row q is image row r_first + q (clamped)
    const int nrows = y1 - y0 + 4;      // gray rows y0-2 .. y1+1
    constexpr int kSlot = kLanes * 12;  // elements per shared-memory slot
    constexpr uint32_t kBytes = kSegLoad * 3 * sizeof(TI);
    const uint32_t seq0 = TMA ? bulk->seq : 0u;
    int last_issued = -1, last_done = -1;

    auto bulk_fetch = [&](int q) {
        if constexpr (TMA) {
            if (q < nrows) last_issued = q;
            if (lane == 0 && q < nrows) {
                const uint32_t n = seq0 + q, slot = n % NS, bar = bulk->bars + 8 * slot;
                const TI* src = static_cast<const TI*>(a.img) + (int64_t)clampi(r_first + q, H) * a.img_pitch +
                                (int64_t)(x - 4 * lane) * 3;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, kBytes);
                bulk_copy_g2s(smem_u32(ring - lane * 12 + slot * kSlot), src, kBytes, bar);
            }
        }
    };

    RawRow<TI> buf[TMA ? 1 : D];  // register staging: buf[q % D] holds sequence row q until taken
    if constexpr (TMA) {
#pragma unroll
        for (int q = 0; q < NS - 1; ++q) bulk_fetch(q);
    } else {
#pragma unroll
        for (int d = 0; d < D; ++d) rows.load(clampi(r_first + d, H), buf[d]);
    }

    // Take sequence row q (from its register slot, refilled with row q + D; or from its shared
    // slot, whose copy is then reissued for row q + NS - 1) and make the 6-wide gray row
    // (clamped at the image border).
    auto take = [&](int q, RawRow<TI>& slot, float g6[6]) {
        float v[12];
        if constexpr (TMA) {
            const uint32_t n = seq0 + q, sl = n % NS;
            const bool ok = __all_sync(kFull, mbar_wait(bulk->bars + 8 * sl, (n / NS) & 1u));
            if (ok) last_done = q;
            else bulk->failed = true;
            const TI* src = ring + sl * kSlot;
            if constexpr (sizeof(TI) == 4) {
                const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float4 t = s4[i];
                    v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
                }
            } else {
                RawRow<TI> r;
                const uint2* s2 = reinterpret_cast<const uint2*>(src);
#pragma unroll
                for (int i = 0; i < 3; ++i) r.q[i] = s2[i];
                RegRows<TI, EDGE, ALIGNED>::unpack(r, v);
            }
            __syncwarp();  // every lane has read the slot the next copy overwrites
            if (ok) bulk_fetch(q + NS - 1);
        } else {
            RegRows<TI, EDGE, ALIGNED>::unpack(slot, v);
            if (q + D < nrows) rows.load(clampi(r_first + q + D, H), slot);
        }
        float c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = gray_of(v[3 * j], v[3 * j + 1], v[3 * j + 2]);
        make_row6(c, g6);
        if constexpr (EDGE) clamp_row6(g6, x, W);
    };

    float g0[6], g1[6], g2[6];
    float2 Ia[4], Ib[4], Ic[4];  // Sobel rows y-1, y, y+1
    // Steps per main-loop iteration: D for register staging (constant slot indices); for bulk
    // staging kFwdUnroll, so that the 3-row gray and 2-row Sobel windows rotate by renaming.
    constexpr int DB = TMA ? kFwdUnroll : D;
    take(0, buf[TMA ? 0 : 0 % DB], g0);
    take(1, buf[TMA ? 0 : 1 % DB], g1);
    take(2, buf[TMA ? 0 : 2 % DB], g2);
    sobel(P, g0, g1, g2, Ia);  // row y0-1 (replaced by row y0 at the top border)
    take(3, buf[TMA ? 0 : 3 % DB], g0);
    sobel(P, g1, g2, g0, Ib);  // row y0
#pragma unroll
    for (int i = 0; i < 6; ++i) { float t = g1[i]; g1[i] = g0[i]; g0[i] = g2[i]; g2[i] = t; }
    // now g0 = gray row y0, g1 = gray row y0 + 1 (g2 is scratch)

    TO* out = static_cast<TO*>(a.out);
    const bool producer = lane >= 1 && lane <= 30;

    auto step = [&](int q, RawRow<TI>& slot) {
        const int y = y0 + q - 4;
        take(q, slot, g2);             // gray row y+2
        sobel(P, g0, g1, g2, Ic);      // row y+1 (replaced by row y at the bottom border)
        // A3 + A4: products summed over rows y-1, y, y+1, clamped at their own stage.
        float2 v2[4];
        float vxy[4];
        if (y == 0 || y == H - 1) {
            float2 A[4], B[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                A[j] = (y == 0) ? Ib[j] : Ia[j];
                B[j] = (y == H - 1) ? Ib[j] : Ic[j];
            }
            vertical_products(A, Ib, B, v2, vxy);
        } else {
            vertical_products(Ia, Ib, Ic, v2, vxy);
        }
        float2 s2[4];
        float sxy[4];
        horizontal_box<EDGE>(v2, s2, x, W);
        horizontal_box<EDGE>(vxy, sxy, x, W);
        // A5
        float R[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) R[j] = response(s2[j].x, sxy[j], s2[j].y, P.kappa);
        if (producer) {
            const int yo = y - a.oy;
            TO* orow = out + (int64_t)yo * a.out_pitch;
            if (!EDGE && a.out_vec) {
                if constexpr (sizeof(TO) == 4) {
                    *reinterpret_cast<float4*>(orow + x) = make_float4(R[0], R[1], R[2], R[3]);
                } else {
                    TO o[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) o[j] = Conv<TO>::st(R[j]);
                    *reinterpret_cast<uint2*>(orow + x) = *reinterpret_cast<uint2*>(o);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int c = x + j;
                    if (c >= a.xlo && c < a.xhi) orow[c - a.ox] = Conv<TO>::st(R[j]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) { g0[i] = g1[i]; g1[i] = g2[i]; }
#pragma unroll
        for (int j = 0; j < 4; ++j) { Ia[j] = Ib[j]; Ib[j] = Ic[j]; }
    };

    // Main loop: D steps per iteration so that every register staging slot index is a constant.
#pragma unroll 1
    for (int q0 = 4; q0 < nrows; q0 += DB) {
        if (TMA && bulk->failed) break;
#pragma unroll
        for (int d = 0; d < DB; ++d)
            if (q0 + d < nrows) step(q0 + d, buf[TMA ? 0 : (4 + d) % DB]);
    }
    if constexpr (TMA) {
        if (bulk->failed) {
            // Drain the copies issued but not waited for (bounded), so that no bulk copy still
            // writes this warp's shared memory when the kernel returns.
            for (int q = last_done + 1; q <= last_issued; ++q) {
                const uint32_t n = seq0 + q;
                mbar_wait(bulk->bars + 8 * (n % NS), (n / NS) & 1u);
            }
        }
        bulk->seq = seq0 + (uint32_t)nrows;
    }
}

}  // namespace shine
