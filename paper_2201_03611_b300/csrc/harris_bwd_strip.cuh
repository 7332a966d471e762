// Backward strip: one warp computes the vector-Jacobian product over one (column segment,
// row band) of one image; see harris_bwd.cu for the adjoint chain B1-B6.
#pragma once

#include "harris_common.cuh"
#include "harris_kernels.h"

namespace shine {

// The lane's 4 cotangent values of successive rows (one 16- or 8-byte chunk per row).
template <typename T, int NS, bool EDGE, bool ALIGNED>
struct CotRows {
    static constexpr int kChunk = 4 * sizeof(T);
    T* ring;
    const T* g;
    int64_t pitch;
    int x, ox, oy, gho, gwo;
    int valid_bytes;

    __device__ __forceinline__ CotRows(T* ring_, const T* g_, int64_t pitch_, int x_, int ox_, int oy_,
                                       int gho_, int gwo_)
        : ring(ring_), g(g_), pitch(pitch_), x(x_), ox(ox_), oy(oy_), gho(gho_), gwo(gwo_) {
        int gx = x - ox;
        int npx = gx < 0 ? 0 : (gwo - gx >= 4 ? 4 : (gwo - gx > 0 ? gwo - gx : 0));
        valid_bytes = npx * (int)sizeof(T);
    }

    // Stage the cotangent of image row r (zero outside the cotangent's rows).
    __device__ __forceinline__ void fetch(int slot, int r) const {
        if constexpr (ALIGNED) {
            int gy = r - oy;
            bool row_in = gy >= 0 && gy < gho;
            int nb = row_in ? (EDGE ? valid_bytes : kChunk) : 0;
            const char* src = nb > 0
                ? reinterpret_cast<const char*>(g + (int64_t)gy * pitch + (x - ox))
                : reinterpret_cast<const char*>(g);
            uint32_t dst = smem_u32(ring + slot * 4);
            if constexpr (kChunk == 16) cp_async16(dst, src, nb);
            else cp_async8(dst, src, nb);
        }
    }

    __device__ __forceinline__ void read(int slot, int r, float v[4]) const {
        if constexpr (ALIGNED) {
            if constexpr (sizeof(T) == 4) {
                float4 q = *reinterpret_cast<const float4*>(ring + slot * 4);
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
                uint2 q = *reinterpret_cast<const uint2*>(ring + slot * 4);
                v[0] = Bits16<T>::to_f(q.x & 0xffffu);
                v[1] = Bits16<T>::to_f(q.x >> 16);
                v[2] = Bits16<T>::to_f(q.y & 0xffffu);
                v[3] = Bits16<T>::to_f(q.y >> 16);
            }
        } else {
            int gy = r - oy;
            bool row_in = gy >= 0 && gy < gho;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int gx = x + j - ox;
                v[j] = (row_in && gx >= 0 && gx < gwo) ? Conv<T>::ld(g[(int64_t)gy * pitch + gx]) : 0.0f;
            }
        }
    }
};

__device__ __forceinline__ void copy6(float d[6], const float s[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = s[i];
}
__device__ __forceinline__ void copy4(float d[4], const float s[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = s[i];
}

// WITH_R: also store R (computed anyway in B1) into rout at the rows this warp owns, for the
// fused forward+backward pass; rout has the output geometry of the forward pass.
template <typename TI, typename TG, int NS, bool EDGE, bool ALIGNED, bool GALIGNED, bool WITH_R = false>
__device__ __forceinline__ void bwd_strip(const BwdArgs& a, const Params& P, int lane, int x, int y0,
                                          int y1, TI* ring, TG* gring, float acc[kParamSlots],
                                          TI* rout = nullptr, int64_t rpitch = 0, bool rvec = false) {
    const int H = a.H, W = a.W;
    const bool producer = lane >= 1 && lane <= 30;
    PixelRows<TI, NS, EDGE, ALIGNED> rows(ring, static_cast<const TI*>(a.img), a.img_pitch, x, W);
    CotRows<TG, NS, EDGE, GALIGNED> grows(gring, static_cast<const TG*>(a.gout), a.gout_pitch, x, a.ox,
                                          a.oy, a.gho, a.gwo);
    const int r_first = y0 - 4;
    const int nrows = y1 - y0 + 8;  // image rows y0-4 .. y1+3, cotangent rows y0-6 .. y1+1

    // Column validity of the lane's 4 columns (only EDGE warps can have invalid ones).
    bool cin[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cin[j] = !EDGE || (x + j >= 0 && x + j < W);

#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
        if (s < nrows) {
            rows.fetch(s, clampi(r_first + s, H));
            grows.fetch(s, r_first + s - 2);
        }
        cp_async_commit();
    }

    // Step s: gray row (6 wide, clamped) of image row r_first + s, and its cotangent row
    // (row - 2), staged NS - 1 steps ahead.
    auto stage_in = [&](int s, float g6[6], float gv[4]) {
        cp_async_wait<NS - 2>();
        const int r = r_first + s;
        float v[12];
        rows.read(s % NS, clampi(r, H), v);
        grows.read(s % NS, r - 2, gv);
        float c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = gray_of(v[3 * j], v[3 * j + 1], v[3 * j + 2]);
        const int sn = s + NS - 1;
        if (sn < nrows) {
            rows.fetch(sn % NS, clampi(r_first + sn, H));
            grows.fetch(sn % NS, r_first + sn - 2);
        }
        cp_async_commit();
        make_row6(c, g6);
        if constexpr (EDGE) clamp_row6(g6, x, W);
    };

    // Register windows (row index relative to the lead image row r of the current step).
    float G0[6], G1[6], G2[6], G3[6], G4[6];  // gray rows r-4 .. r
    float ix0[4], iy0[4], ix1[4], iy1[4];       // I rows r-3, r-2 (r-1 computed per step)
    float gs0[3][4], gs1[3][4];                 // gS rows r-4, r-3 (r-2 computed per step)
    float gx0[6], gy0[6], gx1[6], gy1[6];       // gI0 rows r-5, r-4 (6 wide)
    float gv[4];

#pragma unroll
    for (int i = 0; i < 6; ++i) {
        gx0[i] = gy0[i] = gx1[i] = gy1[i] = 0.0f;
        G0[i] = G1[i] = G2[i] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        ix0[j] = iy0[j] = ix1[j] = iy1[j] = 0.0f;
#pragma unroll
        for (int q = 0; q < 3; ++q) gs0[q][j] = gs1[q][j] = 0.0f;
    }
    stage_in(0, G3, gv);  // image rows r_first, r_first + 1; shifted down at every step
    stage_in(1, G4, gv);

    TI* gimg = static_cast<TI*>(a.gimg);
    const float kc[3] = {kGrayR, kGrayG, kGrayB};
    // Two-level sum of the parameter cotangents: `part` collects kFlushRows rows, then is added
    // into `acc`, so no float32 accumulator sees more than ~4 * max(kFlushRows, rows/kFlushRows)
    // terms.
    constexpr int kFlushRows = 16;
    float part[kParamSlots];
#pragma unroll
    for (int i = 0; i < kParamSlots; ++i) part[i] = 0.0f;

#pragma unroll 1
    for (int s = 2; s < nrows; ++s) {
        const int r = r_first + s;
        // shift the gray window down one row and stage row r into G4
        copy6(G0, G1); copy6(G1, G2); copy6(G2, G3); copy6(G3, G4);
        stage_in(s, G4, gv);
        // B1: I at row r-1 (gray rows r-2, r-1, r).
        float ix2[4], iy2[4];
        sobel(P, G2, G3, G4, ix2, iy2);

        // B1: S at row r-2 from products at rows r-3, r-2, r-1 (clamped at their stage).
        const int sr = r - 2;
        float vs[3][4];
        if (sr == 0 || sr == H - 1) {
            float ax[4], ay[4], bx[4], by[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                ax[j] = (sr == 0) ? ix1[j] : ix0[j];
                ay[j] = (sr == 0) ? iy1[j] : iy0[j];
                bx[j] = (sr == H - 1) ? ix1[j] : ix2[j];
                by[j] = (sr == H - 1) ? iy1[j] : iy2[j];
            }
            vertical_products(ax, ay, ix1, iy1, bx, by, vs);
        } else {
            vertical_products(ix0, iy0, ix1, iy1, ix2, iy2, vs);
        }
        // B2: gS at row r-2 (horizontal box sum first, then the response adjoint).
        float gsn[3][4];
        {
            float S[3][4];
#pragma unroll
            for (int q = 0; q < 3; ++q) horizontal_box<EDGE>(vs[q], S[q], x, W);
            const bool own_row = sr >= y0 && sr < y1;
            if constexpr (WITH_R) {
                // R at row sr (A5), for rows this warp owns inside the forward output region
                const int rlo = a.valid ? 2 : 0, rhi = a.valid ? H - 2 : H;
                if (rout != nullptr && own_row && producer && sr >= rlo && sr < rhi) {
                    float R[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) R[j] = response(S[0][j], S[1][j], S[2][j], P.kappa);
                    TI* orow = rout + (int64_t)(sr - rlo) * rpitch;
                    if (!EDGE && rvec && !a.valid) {
                        if constexpr (sizeof(TI) == 4) {
                            *reinterpret_cast<float4*>(orow + x) = make_float4(R[0], R[1], R[2], R[3]);
                        } else {
                            TI o[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) o[j] = Conv<TI>::st(R[j]);
                            *reinterpret_cast<uint2*>(orow + x) = *reinterpret_cast<const uint2*>(o);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int c = x + j;
                            if (c >= rlo && c < W - rlo) orow[c - rlo] = Conv<TI>::st(R[j]);
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float sxx = S[0][j], sxy = S[1][j], syy = S[2][j];
                float tr = sxx + syy;
                float g = gv[j];
                float k2 = 2.0f * P.kappa * tr;
                gsn[0][j] = g * (syy - k2);
                gsn[1][j] = -2.0f * g * sxy;
                gsn[2][j] = g * (sxx - k2);
                float dk = -g * tr * tr;
                part[0] += (own_row && cin[j]) ? dk : 0.0f;
            }
        }
        // B3: gP at row k = r-3 = clamped box sum of gS rows k-1, k, k+1.
        const int k = r - 3;
        float gp[3][4];
        {
            const bool top = k == 0, bot = k == H - 1;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float vg[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float lo = top ? gs1[q][j] : gs0[q][j];
                    float hi = bot ? gs1[q][j] : gsn[q][j];
                    vg[j] = lo + gs1[q][j] + hi;
                }
                float r6[6];
                make_row6(vg, r6);
                if constexpr (EDGE) clamp_row6(r6, x, W);
#pragma unroll
                for (int j = 0; j < 4; ++j) gp[q][j] = r6[j] + r6[j + 1] + r6[j + 2];
            }
        }
        // B4: gI at row k (zero outside the image: the padded domain of B5).
        float gIx[4], gIy[4];
        {
            const bool row_in = k >= 0 && k < H;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float vx = fmaf(2.0f * ix0[j], gp[0][j], iy0[j] * gp[1][j]);
                float vy = fmaf(ix0[j], gp[1][j], 2.0f * iy0[j] * gp[2][j]);
                bool in = row_in && cin[j];
                gIx[j] = in ? vx : 0.0f;
                gIy[j] = in ? vy : 0.0f;
            }
        }
        // B5 (weights): d W[a][b] += gI(k, c) * G(clamp(k + a - 1), clamp(c + b - 1)) for the
        // rows and columns this warp owns. Gray rows k-1, k, k+1 are G0, G1, G2.
        {
            const bool own = k >= y0 && k < y1 && producer;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float ex = own ? gIx[j] : 0.0f, ey = own ? gIy[j] : 0.0f;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    part[1 + b] = fmaf(ex, G0[j + b], part[1 + b]);
                    part[4 + b] = fmaf(ex, G1[j + b], part[4 + b]);
                    part[7 + b] = fmaf(ex, G2[j + b], part[7 + b]);
                    part[10 + b] = fmaf(ey, G0[j + b], part[10 + b]);
                    part[13 + b] = fmaf(ey, G1[j + b], part[13 + b]);
                    part[16 + b] = fmaf(ey, G2[j + b], part[16 + b]);
                }
            }
        }
        float gxn[6], gyn[6];
        make_row6(gIx, gxn);
        make_row6(gIy, gyn);

        // B5 (image) + B6 at row u = r-4: transposed stencil over gI0 rows u-1 (gx0), u (gx1),
        // u+1 (gxn), with the vertical clamp folds, then the horizontal folds, then store.
        const int u = r - 4;
        if (u >= y0 && gimg != nullptr) {
            float gg[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float t = 0.0f;
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int c = j - b + 2;  // gI0 column v - b + 1 in row6 coordinates
                    t = fmaf(P.wx[b], gxn[c], t);
                    t = fmaf(P.wy[b], gyn[c], t);
                    t = fmaf(P.wx[3 + b], gx1[c], t);
                    t = fmaf(P.wy[3 + b], gy1[c], t);
                    t = fmaf(P.wx[6 + b], gx0[c], t);
                    t = fmaf(P.wy[6 + b], gy0[c], t);
                }
                gg[j] = t;
            }
            if (u == 0 || u == H - 1) {
                // padded row -1 (weights row 0) and row H (weights row 2) fold onto row u
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float t = 0.0f;
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const int c = j - b + 2;
                        if (u == 0) {
                            t = fmaf(P.wx[b], gx1[c], t);
                            t = fmaf(P.wy[b], gy1[c], t);
                        }
                        if (u == H - 1) {
                            t = fmaf(P.wx[6 + b], gx1[c], t);
                            t = fmaf(P.wy[6 + b], gy1[c], t);
                        }
                    }
                    gg[j] += t;
                }
            }
            if constexpr (EDGE) {
                // padded column -1 folds onto column 0, column W onto column W-1
                float r6[6];
                make_row6(gg, r6);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (x + j == 0) gg[j] += r6[j];
                    if (x + j == W - 1) gg[j] += r6[j + 2];
                }
            }
            if (producer) {
                TI* orow = gimg + (int64_t)u * a.gimg_pitch + (int64_t)x * 3;
                float o[12];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) o[3 * j + ch] = kc[ch] * gg[j];
                if (!EDGE && a.gimg_vec) {
                    if constexpr (sizeof(TI) == 4) {
                        float4* d = reinterpret_cast<float4*>(orow);
                        d[0] = make_float4(o[0], o[1], o[2], o[3]);
                        d[1] = make_float4(o[4], o[5], o[6], o[7]);
                        d[2] = make_float4(o[8], o[9], o[10], o[11]);
                    } else {
                        TI t[12];
#pragma unroll
                        for (int i = 0; i < 12; ++i) t[i] = Conv<TI>::st(o[i]);
                        uint2* d = reinterpret_cast<uint2*>(orow);
                        const uint2* sv = reinterpret_cast<const uint2*>(t);
                        d[0] = sv[0]; d[1] = sv[1]; d[2] = sv[2];
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (cin[j])
#pragma unroll
                            for (int ch = 0; ch < 3; ++ch) orow[3 * j + ch] = Conv<TI>::st(o[3 * j + ch]);
                }
            }
        }
        if ((s & (kFlushRows - 1)) == 0) {
#pragma unroll
            for (int i = 0; i < kParamSlots; ++i) { acc[i] += part[i]; part[i] = 0.0f; }
        }
        // shift the windows
        copy4(ix0, ix1); copy4(iy0, iy1); copy4(ix1, ix2); copy4(iy1, iy2);
#pragma unroll
        for (int q = 0; q < 3; ++q) { copy4(gs0[q], gs1[q]); copy4(gs1[q], gsn[q]); }
        copy6(gx0, gx1); copy6(gy0, gy1); copy6(gx1, gxn); copy6(gy1, gyn);
    }
#pragma unroll
    for (int i = 0; i < kParamSlots; ++i) acc[i] += part[i];
    cp_async_wait<0>();
}

}  // namespace shine
