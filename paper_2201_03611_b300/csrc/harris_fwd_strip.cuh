// Forward strip: one warp computes R over one (column segment, row band) of one image.
//
// Rows are processed RB at a time: one wait for RB staged image rows, their gray rows and
// Sobel rows, then the RB product/box/response rows. The RB rows' work is independent
// (instruction-level parallelism for a warp that otherwise waits on shuffle and shared-memory
// latency). HBM traffic is the image once and R once; nothing else leaves the registers.
#pragma once

#include "harris_common.cuh"
#include "harris_kernels.h"

namespace shine {

template <typename TI, typename TO, int NS, bool EDGE, bool ALIGNED, int RB = kFwdRowsPerBlock>
__device__ __forceinline__ void fwd_strip(const FwdArgs& a, const Params& P, int lane, int x, int y0,
                                          int y1, TI* ring) {
    // Staging: kFirst rows are put in flight up front; every block then reads RB rows and stages
    // RB more. Before block b, rows up to 3 + RB (b + 1) + (kFirst - 4) have been issued while
    // rows up to 3 + RB (b + 1) are needed, so waiting until at most kFirst - 4 groups are
    // pending leaves that many rows in flight. Rows staged after a block's reads go to slots of
    // rows consumed in earlier blocks (kFirst + 2 RB - 4 <= NS).
    constexpr int kFirst = (NS + 4 - 2 * RB) < NS ? (NS + 4 - 2 * RB) : NS;
    static_assert(kFirst - 4 >= RB, "the ring must hold at least one block in flight");
    const int H = a.H, W = a.W;
    PixelRows<TI, NS, EDGE, ALIGNED> rows(ring, static_cast<const TI*>(a.img), a.img_pitch, x, W);
    const int nblocks = (y1 - y0 + RB - 1) / RB;
    const int nrows = 4 + RB * nblocks;  // gray rows y0-2 .. y0+1+RB*nblocks (clamped)
    const int r_first = y0 - 2;

#pragma unroll
    for (int q = 0; q < kFirst; ++q) {
        if (q < nrows) rows.fetch(q % NS, clampi(r_first + q, H));
        cp_async_commit();
    }
    int next = kFirst;  // next sequence row to stage

    auto gray6 = [&](int q, float g6[6]) {
        float v[12];
        rows.read(q % NS, clampi(r_first + q, H), v);
        float c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = gray_of(v[3 * j], v[3 * j + 1], v[3 * j + 2]);
        make_row6(c, g6);
        if constexpr (EDGE) clamp_row6(g6, x, W);
    };
    auto stage_more = [&]() {
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            if (next < nrows) rows.fetch(next % NS, clampi(r_first + next, H));
            cp_async_commit();
            ++next;
        }
    };

    // g[0], g[1]: gray rows y, y+1 of the coming block; I[0], I[1]: Sobel rows y-1, y.
    float g[RB + 2][6];
    float2 I[RB + 2][4];
    {
        cp_async_wait<kFirst - 4>();  // sequence rows 0..3 landed
        float g0[6], g1[6];
        gray6(0, g0);
        gray6(1, g1);
        gray6(2, g[0]);
        gray6(3, g[1]);
        stage_more();
        sobel(P, g0, g1, g[0], I[0]);  // row y0-1 (replaced by row y0 at the top border)
        sobel(P, g1, g[0], g[1], I[1]);  // row y0
    }

    TO* out = static_cast<TO*>(a.out);
    const bool producer = lane >= 1 && lane <= 30;

    auto emit = [&](int y, const float2 Iu[4], const float2 Im[4], const float2 Id[4]) {
        if (y >= y1) return;
        // A3 + A4: products summed over rows y-1, y, y+1, clamped at their own stage.
        float2 v2[4];
        float vxy[4];
        if (y == 0 || y == H - 1) {
            float2 A[4], B[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                A[j] = (y == 0) ? Im[j] : Iu[j];
                B[j] = (y == H - 1) ? Im[j] : Id[j];
            }
            vertical_products(A, Im, B, v2, vxy);
        } else {
            vertical_products(Iu, Im, Id, v2, vxy);
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
    };

#pragma unroll 1
    for (int b = 0; b < nblocks; ++b) {
        const int q = 4 + RB * b;  // first sequence row of this block (gray row y+2)
        const int y = y0 + RB * b;
        cp_async_wait<kFirst - 4>();  // sequence rows q .. q+RB-1 landed
#pragma unroll
        for (int i = 0; i < RB; ++i) gray6(q + i, g[2 + i]);
        stage_more();
#pragma unroll
        for (int i = 0; i < RB; ++i) sobel(P, g[i], g[i + 1], g[i + 2], I[2 + i]);  // rows y+1 ..
#pragma unroll
        for (int i = 0; i < RB; ++i) emit(y + i, I[i], I[i + 1], I[i + 2]);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
#pragma unroll
            for (int c = 0; c < 6; ++c) g[i][c] = g[RB + i][c];
#pragma unroll
            for (int j = 0; j < 4; ++j) I[i][j] = I[RB + i][j];
        }
    }
    cp_async_wait<0>();
}

}  // namespace shine
