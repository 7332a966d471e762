// Forward strip: one warp computes R over one (column segment, row band) of one image.
//
// Per output row y it stages one new image row, makes its gray row, the Sobel/product row
// y+1, adds the three product rows around y (the slide2D+reduce of A4 done vertically in
// registers first, then horizontally with two shuffles per plane), and stores R[y]. HBM
// traffic is the image once and R once; nothing else leaves the registers.
#pragma once

#include "harris_common.cuh"
#include "harris_kernels.h"

namespace shine {

template <typename TI, typename TO, int NS, bool EDGE, bool ALIGNED>
__device__ __forceinline__ void fwd_strip(const FwdArgs& a, const Params& P, int lane, int x, int y0,
                                          int y1, TI* ring) {
    const int H = a.H, W = a.W;
    PixelRows<TI, NS, EDGE, ALIGNED> rows(ring, static_cast<const TI*>(a.img), a.img_pitch, x, W);
    const int nrows = y1 - y0 + 4;  // gray rows y0-2 .. y1+1 (clamped)
    const int r_first = y0 - 2;

#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
        if (s < nrows) rows.fetch(s, clampi(r_first + s, H));
        cp_async_commit();
    }

    // Gray row number s of the sequence, 6 columns wide, clamped at the image border.
    auto gray_row = [&](int s, float g6[6]) {
        cp_async_wait<NS - 2>();
        float v[12];
        rows.read(s % NS, clampi(r_first + s, H), v);
        float c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = gray_of(v[3 * j], v[3 * j + 1], v[3 * j + 2]);
        int sn = s + NS - 1;
        if (sn < nrows) rows.fetch(sn % NS, clampi(r_first + sn, H));
        cp_async_commit();
        make_row6(c, g6);
        if constexpr (EDGE) clamp_row6(g6, x, W);
    };

    float g0[6], g1[6], g2[6];
    float ixa[4], iya[4], ixb[4], iyb[4], ixc[4], iyc[4];  // Sobel rows y-1, y, y+1
    gray_row(0, g0);
    gray_row(1, g1);
    gray_row(2, g2);
    sobel(P, g0, g1, g2, ixa, iya);  // row y0-1 (replaced by row y0 at the top border)
#pragma unroll
    for (int i = 0; i < 6; ++i) { g0[i] = g1[i]; g1[i] = g2[i]; }
    gray_row(3, g2);
    sobel(P, g0, g1, g2, ixb, iyb);  // row y0

    TO* out = static_cast<TO*>(a.out);
    const bool producer = lane >= 1 && lane <= 30;

#pragma unroll 2
    for (int y = y0; y < y1; ++y) {
#pragma unroll
        for (int i = 0; i < 6; ++i) { g0[i] = g1[i]; g1[i] = g2[i]; }
        gray_row(y - y0 + 4, g2);
        sobel(P, g0, g1, g2, ixc, iyc);  // row y+1 (replaced by row y at the bottom border)

        // A3 + A4: products summed over rows y-1, y, y+1, clamped at their own stage.
        float v[3][4];
        if (y == 0 || y == H - 1) {
            float ax[4], ay[4], bx[4], by[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ax[j] = (y == 0) ? ixb[j] : ixa[j];
                ay[j] = (y == 0) ? iyb[j] : iya[j];
                bx[j] = (y == H - 1) ? ixb[j] : ixc[j];
                by[j] = (y == H - 1) ? iyb[j] : iyc[j];
            }
            vertical_products(ax, ay, ixb, iyb, bx, by, v);
        } else {
            vertical_products(ixa, iya, ixb, iyb, ixc, iyc, v);
        }
        float s3[3][4];
#pragma unroll
        for (int q = 0; q < 3; ++q) horizontal_box<EDGE>(v[q], s3[q], x, W);
        // A5
        float R[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) R[j] = response(s3[0][j], s3[1][j], s3[2][j], P.kappa);
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
        for (int j = 0; j < 4; ++j) {
            ixa[j] = ixb[j]; iya[j] = iyb[j];
            ixb[j] = ixc[j]; iyb[j] = iyc[j];
        }
    }
    cp_async_wait<0>();
}

}  // namespace shine
