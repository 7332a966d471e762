// Backward strip: one warp computes the vector-Jacobian product over one (column segment,
// row band) of one image; see harris_bwd.cu for the adjoint chain B1-B6.
#pragma once

#include <type_traits>

#include "harris_common.cuh"
#include "harris_kernels.h"

namespace shine {

// The lane's 4 cotangent values of successive rows (one 16- or 8-byte chunk per row), staged
// like the image rows: a slot holds the 32 lanes' chunks side by side.
template <typename T, int NS, bool EDGE, bool ALIGNED>
struct CotRows {
    static constexpr int kChunk = 4 * sizeof(T);
    static constexpr int kSlot = kLanes * 4;
    T* ring;  // this lane's 4 elements of slot 0
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
            uint32_t dst = smem_u32(ring + slot * kSlot);
            if constexpr (kChunk == 16) cp_async16(dst, src, nb);
            else cp_async8(dst, src, nb);
        }
    }

    __device__ __forceinline__ void read(int slot, int r, float v[4]) const {
        if constexpr (ALIGNED) {
            if constexpr (sizeof(T) == 4) {
                float4 q = *reinterpret_cast<const float4*>(ring + slot * kSlot);
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
                uint2 q = *reinterpret_cast<const uint2*>(ring + slot * kSlot);
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

// WITH_R: also store R (computed anyway in B1) into rout at the rows this warp owns, for the
// fused forward+backward pass; rout has the output geometry of the forward pass.
//
// acc receives this strip's parameter cotangents: acc[0] = d kappa, acc[1 + t] = d Wx[t],
// acc[10 + t] = d Wy[t] (t = 3a + b), for the rows [y0, y1) and producer columns it owns.
// Staging of the strip's rows. TMA: lane 0 moves each row's whole image segment and cotangent
// segment with two bulk copies completing on the slot's mbarrier (interior segments with
// 16-byte aligned rows); otherwise every lane stages its own chunks with cp.async. Both fill the
// same slot layout (lane stride 12 image / 4 cotangent elements). Bulk staging keeps the copy
// engine streaming at the full HBM rate with few warps; the per-lane path tops out lower.
struct BulkState {
    uint32_t bars;     // shared address of this warp's NS barriers
    uint32_t seq;      // rows staged by this warp so far (slot = seq % NS, phase = seq / NS)
    bool failed;       // a bounded wait gave up
};

template <typename TI, typename TG, int NS, bool EDGE, bool ALIGNED, bool GALIGNED, bool WITH_R = false,
          bool TMA = false>
__device__ __forceinline__ void bwd_strip(const BwdArgs& a, const Params& P, int lane, int x, int y0,
                                          int y1, TI* ring, TG* gring, float acc[kParamSlots],
                                          TI* rout = nullptr, int64_t rpitch = 0, bool rvec = false,
                                          BulkState* bulk = nullptr) {
    const int H = a.H, W = a.W;
    const bool producer = lane >= 1 && lane <= 30;
    PixelRows<TI, NS, EDGE, ALIGNED> rows(ring, static_cast<const TI*>(a.img), a.img_pitch, x, W);
    CotRows<TG, NS, EDGE, GALIGNED> grows(gring, static_cast<const TG*>(a.gout), a.gout_pitch, x, a.ox,
                                          a.oy, a.gho, a.gwo);
    const int r_first = y0 - 4;
    const int nrows = y1 - y0 + 8;  // image rows y0-4 .. y1+3, cotangent rows y0-6 .. y1+1
    const uint32_t seq0 = TMA ? bulk->seq : 0u;

    // Column validity of the lane's 4 columns (only EDGE warps can have invalid ones).
    bool cin[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cin[j] = !EDGE || (x + j >= 0 && x + j < W);

    // Bulk staging: the warp's segment starts 4 columns left of the lane-1 column.
    const int xs = x - 4 * lane;
    if constexpr (TMA) {
        SHINE_CHECK(a.dbg, xs >= 0 && xs + kSegLoad <= W, kDbgBwdStage);
        SHINE_CHECK(a.dbg, xs - a.ox >= 0 && xs - a.ox + kSegLoad <= a.gwo, kDbgBwdStage);
    } else if constexpr (ALIGNED && !EDGE) {
        SHINE_CHECK(a.dbg, x >= 0 && x + kCols <= W, kDbgBwdStage);
    }
    if constexpr (ALIGNED) {
        SHINE_CHECK(a.dbg, smem_in(smem_u32(ring), (uint32_t)((NS - 1) * PixelRows<TI, NS, EDGE, ALIGNED>::kSlot + 12) *
                                                       (uint32_t)sizeof(TI)), kDbgSmem);
    }
    constexpr uint32_t kImgBytes = kSegLoad * 3 * sizeof(TI), kCotBytes = kSegLoad * sizeof(TG);
    int last_issued = -1, last_done = -1;  // bulk staging: rows issued / waited for successfully
    // ring position of the next row to stage, advanced one slot per step (no division per step)
    uint32_t st_slot = TMA ? seq0 % NS : 0u, st_phase = TMA ? (seq0 / NS) & 1u : 0u;
    auto bulk_fetch = [&](int s, uint32_t slot) {
        if constexpr (TMA) {
            if (s < nrows) last_issued = s;
            if (lane == 0 && s < nrows) {
                const uint32_t bar = bulk->bars + 8 * slot;
                const int r = r_first + s, gy = r - 2;
                const bool g_in = gy >= 0 && gy < a.gho;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, kImgBytes + (g_in ? kCotBytes : 0));
                const TI* src = static_cast<const TI*>(a.img) + (int64_t)clampi(r, H) * a.img_pitch + (int64_t)xs * 3;
                bulk_copy_g2s(smem_u32(ring - lane * 12 + slot * PixelRows<TI, NS, EDGE, ALIGNED>::kSlot), src,
                              kImgBytes, bar);
                if (g_in) {
                    const TG* gs = static_cast<const TG*>(a.gout) + (int64_t)gy * a.gout_pitch + xs;
                    bulk_copy_g2s(smem_u32(gring - lane * 4 + slot * CotRows<TG, NS, EDGE, GALIGNED>::kSlot), gs,
                                  kCotBytes, bar);
                }
            }
        }
    };

    if constexpr (TMA) {
#pragma unroll
        for (int s = 0; s < NS - 1; ++s) bulk_fetch(s, (seq0 + s) % NS);
    } else {
#pragma unroll
        for (int s = 0; s < NS - 1; ++s) {
            if (s < nrows) {
                rows.fetch(s, clampi(r_first + s, H));
                grows.fetch(s, r_first + s - 2);
            }
            cp_async_commit();
        }
    }

    // Step s: gray row (6 wide, clamped) of image row r_first + s, and its cotangent row
    // (row - 2), staged NS - 1 steps ahead.
    auto stage_in = [&](auto fast_tag, int s, float g6[6], float gv[4]) {
        constexpr bool FAST_ROW = decltype(fast_tag)::value;
        const int r = r_first + s;
        float v[12];
        if constexpr (TMA) {
            const uint32_t slot = st_slot;
            const bool ok = __all_sync(kFull, mbar_wait(bulk->bars + 8 * slot, st_phase));
            if (++st_slot == (uint32_t)NS) { st_slot = 0; st_phase ^= 1u; }
            if (ok) last_done = s;
            else bulk->failed = true;
            rows.read(slot, clampi(r, H), v);
            const int gy = r - 2;
            // fast steps of a bulk-staged (CLAMP) strip always have their cotangent row
            if (FAST_ROW || (gy >= 0 && gy < a.gho)) {
                grows.read(slot, r - 2, gv);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) gv[j] = 0.0f;
            }
            __syncwarp();  // every lane has read the slot that the next copy overwrites
            if (ok) bulk_fetch(s + NS - 1, slot == 0 ? (uint32_t)NS - 1 : slot - 1);  // row s+NS-1 reuses row s-1's slot
        } else {
            cp_async_wait<NS - 2>();
            rows.read(s % NS, clampi(r, H), v);
            grows.read(s % NS, r - 2, gv);
        }
        float c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = gray_of(v[3 * j], v[3 * j + 1], v[3 * j + 2]);
        if constexpr (!TMA) {
            const int sn = s + NS - 1;
            if (sn < nrows) {
                rows.fetch(sn % NS, clampi(r_first + sn, H));
                grows.fetch(sn % NS, r_first + sn - 2);
            }
            cp_async_commit();
        }
        make_row6(c, g6);
        if constexpr (EDGE) clamp_row6(g6, x, W);
    };

    // Register windows (row index relative to the lead image row r of the current step).
    float G0[6], G1[6], G2[6], G3[6], G4[6];  // gray rows r-4 .. r
    float2 I0[4], I1[4];                       // (Ix, Iy) rows r-3, r-2 (r-1 computed per step)
    // Running sums (push form: each row is added into the sums it belongs to when it arrives):
    float2 qa[4], qb[4];   // (gSxx, gSyy): rows k-1 and k summed, row k alone (k = r-3)
    float qaq[4], qbq[4];  // gSxy likewise
    float2 ga1[4], ga2[4]; // d gray of rows k-1 and k so far, x and y weight planes apart
    float gv[4];

#pragma unroll
    for (int i = 0; i < 6; ++i) G0[i] = G1[i] = G2[i] = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        I0[j] = I1[j] = qa[j] = qb[j] = ga1[j] = ga2[j] = make_float2(0.0f, 0.0f);
        qaq[j] = qbq[j] = 0.0f;
    }
    stage_in(std::false_type{}, 0, G3, gv);  // image rows r_first, r_first + 1; shifted down at every step
    stage_in(std::false_type{}, 1, G4, gv);

    TI* gimg = static_cast<TI*>(a.gimg);
    const float kc[3] = {kGrayR, kGrayG, kGrayB};
    // Two-level sum of the parameter cotangents: the part* accumulators collect kFlushRows
    // rows, then are added into acc, so no float32 accumulator sees more than
    // ~4 * max(kFlushRows, rows / kFlushRows) terms.
    constexpr int kFlushRows = 16;
    float2 partw[9];  // (d Wx[t], d Wy[t])
    float partk = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) partw[i] = make_float2(0.0f, 0.0f);

    // One step: stage image row r = r_first + s and cotangent row r-2, then B1..B6 for the rows
    // whose inputs are complete. FAST steps are those whose rows are all interior to the image
    // and to this strip (no clamp, fold or ownership test is needed).
    auto step = [&](auto fast_tag, int s) {
        constexpr bool FAST = decltype(fast_tag)::value;
        const int r = r_first + s;
        // shift the gray window down one row and stage row r into G4
#pragma unroll
        for (int i = 0; i < 6; ++i) { G0[i] = G1[i]; G1[i] = G2[i]; G2[i] = G3[i]; G3[i] = G4[i]; }
        stage_in(fast_tag, s, G4, gv);

        // B1: I at row r-1 (gray rows r-2, r-1, r).
        float2 I2[4];
        sobel(P, G2, G3, G4, I2);

        // B1: S at row r-2 from products at rows r-3, r-2, r-1 (clamped at their stage).
        const int sr = r - 2;
        float2 v2[4];
        float vxy[4];
        if (!FAST && (sr == 0 || sr == H - 1)) {
            float2 A[4], B[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                A[j] = (sr == 0) ? I1[j] : I0[j];
                B[j] = (sr == H - 1) ? I1[j] : I2[j];
            }
            vertical_products(A, I1, B, v2, vxy);
        } else {
            vertical_products(I0, I1, I2, v2, vxy);
        }
        float2 S2[4];  // (Sxx, Syy)
        float Sxy[4];
        horizontal_box<EDGE>(v2, S2, x, W);
        horizontal_box<EDGE>(vxy, Sxy, x, W);
        const bool own_row = FAST || (sr >= y0 && sr < y1);
        if constexpr (WITH_R) {
            // R at row sr (A5), for rows this warp owns inside the forward output region
            const int rlo = a.valid ? 2 : 0, rhi = a.valid ? H - 2 : H;
            if (rout != nullptr && own_row && producer && (FAST || (sr >= rlo && sr < rhi))) {
                float R[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) R[j] = response(S2[j].x, Sxy[j], S2[j].y, P.kappa);
                SHINE_CHECK(a.dbg, sr >= rlo && sr < rhi && (EDGE || !rvec || a.valid || (x >= 0 && x + kCols <= W)),
                            kDbgBwdStore);
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
        // B2: gS at row r-2 and the d kappa terms (the cotangent is zero outside the image, so
        // only the row needs testing; lanes 0 and 31 are dropped when the warp reduces).
        float2 gsn[4];
        float gqn[4];
        float dk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float tr = S2[j].x + S2[j].y;
            const float g = gv[j];
            const float k2 = 2.0f * P.kappa * tr;
            gsn[j] = make_float2(g * (S2[j].y - k2), g * (S2[j].x - k2));
            gqn[j] = -2.0f * g * Sxy[j];
            dk[j] = -g * tr * tr;
        }
        if (own_row) partk += (dk[0] + dk[1]) + (dk[2] + dk[3]);
        // B3: gP at row k = r-3 = clamped box sum of gS rows k-1, k, k+1 (gS row k+1 arrives
        // now): (k-1 + k) + k+1, with row k counted twice at either clamped image border.
        const int k = r - 3;
        float2 gp2[4];  // (gPxx, gPyy)
        float gpq[4];   // gPxy
        {
            float2 vg2[4];
            float vgq[4];
            if (!FAST && (k == 0 || k == H - 1)) {
                const bool top = k == 0, bot = k == H - 1;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    vg2[j] = __fadd2_rn(top ? __fadd2_rn(qb[j], qb[j]) : qa[j], bot ? qb[j] : gsn[j]);
                    vgq[j] = (top ? qbq[j] + qbq[j] : qaq[j]) + (bot ? qbq[j] : gqn[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    vg2[j] = __fadd2_rn(qa[j], gsn[j]);
                    vgq[j] = qaq[j] + gqn[j];
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                qa[j] = __fadd2_rn(qb[j], gsn[j]);
                qb[j] = gsn[j];
                qaq[j] = qbq[j] + gqn[j];
                qbq[j] = gqn[j];
            }
            horizontal_box<EDGE>(vg2, gp2, x, W);
            horizontal_box<EDGE>(vgq, gpq, x, W);
        }
        // B4: gI at row k (zero outside the image: the padded domain of B5).
        float2 gI[4];
        if (FAST || (k >= 0 && k < H)) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 i0 = I0[j];
                float vx = fmaf(2.0f * i0.x, gp2[j].x, i0.y * gpq[j]);
                float vy = fmaf(i0.x, gpq[j], 2.0f * i0.y * gp2[j].y);
                gI[j] = make_float2(cin[j] ? vx : 0.0f, cin[j] ? vy : 0.0f);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) gI[j] = make_float2(0.0f, 0.0f);
        }
        // B5 (weights): (d Wx[a][b], d Wy[a][b]) += gI(k, c) * G(clamp(k + a - 1), clamp(c + b - 1))
        // for the rows this warp owns (gI is zero outside the image; lanes 0 and 31 are dropped
        // when the warp reduces). Gray rows k-1, k, k+1 are G0, G1, G2.
        if (FAST || (k >= y0 && k < y1)) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    partw[b] = __ffma2_rn(gI[j], dup2(G0[j + b]), partw[b]);
                    partw[3 + b] = __ffma2_rn(gI[j], dup2(G1[j + b]), partw[3 + b]);
                    partw[6 + b] = __ffma2_rn(gI[j], dup2(G2[j + b]), partw[6 + b]);
                }
            }
        }
        float2 gin[6];
        make_row6(gI, gin);

        // B5 (image) + B6 at row u = r-4: the transposed stencil in push form. gI row k = u+1
        // arrives: its taps complete d gray of row u and are added into rows k and k+1. The
        // padded row -1 (complete when row 0 arrives) folds onto row 0, the padded row H
        // (complete once row H-1 has arrived) onto row H-1.
        const int u = r - 4;
        float2 done[4];
        if (gimg != nullptr) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 d = ga1[j], n1 = ga2[j], n2 = make_float2(0.0f, 0.0f);
                const float2 below = ga2[j];  // d gray of row u+1 so far
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int c = j - b + 2;  // gI column (lane column j) - b + 1 in row6 coordinates
                    d = __ffma2_rn(P.w[b], gin[c], d);
                    n1 = __ffma2_rn(P.w[3 + b], gin[c], n1);
                    n2 = __ffma2_rn(P.w[6 + b], gin[c], n2);
                }
                if (!FAST && u == H - 1) d = __fadd2_rn(d, below);
                if (!FAST && k == 0) n1 = __fadd2_rn(n1, d);
                done[j] = d; ga1[j] = n1; ga2[j] = n2;
            }
        }
        if ((FAST || u >= y0) && gimg != nullptr) {
            float gg[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) gg[j] = done[j].x + done[j].y;
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
                SHINE_CHECK(a.dbg, u >= 0 && u < H && (EDGE || !a.gimg_vec || (x >= 0 && x + kCols <= W)), kDbgBwdStore);
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
        // shift the windows
#pragma unroll
        for (int j = 0; j < 4; ++j) { I0[j] = I1[j]; I1[j] = I2[j]; }
    };
    auto flush = [&]() {
        acc[0] += partk;
        partk = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            acc[1 + i] += partw[i].x;
            acc[10 + i] += partw[i].y;
            partw[i] = make_float2(0.0f, 0.0f);
        }
    };
    const std::integral_constant<bool, false> general{};
    const std::integral_constant<bool, true> fast{};
    // Fast steps: u = r - 4 >= max(y0, 2) and S row r - 2 <= min(y1 - 1, H - 3).
    const int s_a = 8 + (y0 < 2 ? 2 - y0 : 0);
    const int s_b = (y1 - 3 < H - 5 ? y1 - 3 : H - 5) - y0 + 9;  // exclusive
    int s = 2, since_flush = 0;
    // One loop with one copy of each step kind (the general steps at the strip's two ends, the
    // fast ones between), to keep the code the warps run small.
#pragma unroll 1
    for (; s < nrows; ++s) {
        if (TMA && bulk->failed) break;
        if (s >= s_a && s < s_b) step(fast, s);
        else step(general, s);
        if (++since_flush == kFlushRows) { flush(); since_flush = 0; }
    }
    acc[0] += partk;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        acc[1 + i] += partw[i].x;
        acc[10 + i] += partw[i].y;
    }
    if constexpr (TMA) {
        if (bulk->failed) {
            // Drain the copies issued but not waited for, with bounded waits, so that no bulk
            // copy still writes this warp's shared memory when the kernel returns.
            for (int s2 = last_done + 1; s2 <= last_issued; ++s2) {
                const uint32_t q = seq0 + s2;
                mbar_wait(bulk->bars + 8 * (q % NS), (q / NS) & 1u);
            }
        }
        bulk->seq = seq0 + (uint32_t)nrows;  // every staged row was waited for and read
    } else {
        cp_async_wait<0>();
    }
}

}  // namespace shine
