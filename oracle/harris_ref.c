/*
 * FP64 reference of the Harris pattern pipeline, written stage by stage with full
 * intermediate arrays (no fusion, no tiling).
 *
 * ORACLE -- test infrastructure only. Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library; the product path never does. It shares no
 * code, header or constant with the CUDA kernels.
 *
 * Stages (the same composition the pattern evaluator in oracle/harris.py spells out):
 *   A1 G[y][x]   = 0.299 r + 0.587 g + 0.114 b                        (map)
 *   A2 I[i][j]   = sum_ab W[a][b] * X(i,a)(j,b)                       (slide2D(3,1) + zip + reduce)
 *   A3 P         = (Ix*Ix, Ix*Iy, Iy*Iy)                              (zip + map)
 *   A4 S[i][j]   = sum_ab P(i,a)(j,b)                                 (slide2D(3,1) + reduce)
 *   A5 R         = Sxx*Syy - Sxy^2 - kappa*(Sxx+Syy)^2                (map)
 * where X(i,a)(j,b) is x[clamp(i+a-1)][clamp(j+b-1)] in CLAMP mode (pad_clamp2D(1) before the
 * slide) and x[i+a][j+b] in VALID mode (no pad; each stage shrinks by 2).
 *
 * The backward pass is reverse mode of the same stages: each stencil's adjoint scatters
 * W[a][b]*gy onto the index it read (overlap-add; with clamp, onto the clamped index), and the
 * weight cotangent is the sum over all windows of gy times the value read.
 *
 * Inputs are double arrays (exact images of the stored bf16/fp16/f32 values); all arithmetic
 * and all outputs are double. Images are H x W x 3, row-major, channel fastest, dense.
 * Return value: 0 on success, -1 on a bad argument, -2 when memory runs out.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double kGray[3] = {0.299, 0.587, 0.114};
static const double kOnes[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};

static int64_t clampi(int64_t i, int64_t n) { return i < 0 ? 0 : (i > n - 1 ? n - 1 : i); }

/* Index of tap t (0..2) of output position i on an axis of input length n. */
static int64_t tap(int64_t i, int t, int64_t n, int clamp) {
    return clamp ? clampi(i + t - 1, n) : i + t;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* A2/A4: y = 3x3 weighted window sum over x (h x w). Output is h x w (clamp) or (h-2)x(w-2). */
static void stencil3(const double* x, int64_t h, int64_t w, int clamp, const double* wt, double* y) {
    int64_t ho = clamp ? h : h - 2, wo = clamp ? w : w - 2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ho; ++i)
        for (int64_t j = 0; j < wo; ++j) {
            double acc = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    acc = acc + wt[a * 3 + b] * x[tap(i, a, h, clamp) * w + tap(j, b, w, clamp)];
            y[i * wo + j] = acc;
        }
}

/* Adjoint of stencil3: gx += scatter of wt*gy, gwt += sum gy * x (gwt may be NULL), and
 * gabs += sum |gy * x|, the magnitude of the terms of that sum (gabs may be NULL). */
static void stencil3_vjp(const double* x, int64_t h, int64_t w, int clamp, const double* wt,
                         const double* gy, double* gx, double* gwt, double* gabs) {
    int64_t ho = clamp ? h : h - 2, wo = clamp ? w : w - 2;
    double gw[9] = {0}, ga[9] = {0};
    for (int64_t i = 0; i < ho; ++i)
        for (int64_t j = 0; j < wo; ++j) {
            double g = gy[i * wo + j];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    int64_t k = tap(i, a, h, clamp) * w + tap(j, b, w, clamp);
                    gx[k] += wt[a * 3 + b] * g;
                    gw[a * 3 + b] += g * x[k];
                    ga[a * 3 + b] += fabs(g * x[k]);
                }
        }
    if (gwt)
        for (int t = 0; t < 9; ++t) gwt[t] += gw[t];
    if (gabs)
        for (int t = 0; t < 9; ++t) gabs[t] += ga[t];
}

typedef struct {
    int64_t h1, w1, h2, w2; /* sizes after the first and the second stencil stage */
    double *G, *Ix, *Iy, *Pxx, *Pxy, *Pyy, *Sxx, *Sxy, *Syy;
} stages_t;

static void free_stages(stages_t* s) {
    free(s->G); free(s->Ix); free(s->Iy); free(s->Pxx); free(s->Pxy); free(s->Pyy);
    free(s->Sxx); free(s->Sxy); free(s->Syy);
}

static int check_args(int64_t H, int64_t W, int border) {
    if (border != 0 && border != 1) return -1;
    if (border == 0 && (H < 5 || W < 5)) return -1;
    if (H < 1 || W < 1) return -1;
    return 0;
}

static int run_stages(const double* img, int64_t H, int64_t W, int border, const double* wx,
                      const double* wy, stages_t* s) {
    int clamp = border == 1;
    memset(s, 0, sizeof(*s));
    s->h1 = clamp ? H : H - 2; s->w1 = clamp ? W : W - 2;
    s->h2 = clamp ? H : H - 4; s->w2 = clamp ? W : W - 4;
    size_t n0 = (size_t)(H * W), n1 = (size_t)(s->h1 * s->w1), n2 = (size_t)(s->h2 * s->w2);
    s->G = malloc(n0 * 8); s->Ix = malloc(n1 * 8); s->Iy = malloc(n1 * 8);
    s->Pxx = malloc(n1 * 8); s->Pxy = malloc(n1 * 8); s->Pyy = malloc(n1 * 8);
    s->Sxx = malloc(n2 * 8); s->Sxy = malloc(n2 * 8); s->Syy = malloc(n2 * 8);
    if (!s->G || !s->Ix || !s->Iy || !s->Pxx || !s->Pxy || !s->Pyy || !s->Sxx || !s->Sxy || !s->Syy) {
        free_stages(s);
        return -2;
    }
    /* A1 */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)n0; ++k) {
        double acc = 0.0;
        for (int c = 0; c < 3; ++c) acc = acc + img[k * 3 + c] * kGray[c];
        s->G[k] = acc;
    }
    /* A2 */
    stencil3(s->G, H, W, clamp, wx, s->Ix);
    stencil3(s->G, H, W, clamp, wy, s->Iy);
    /* A3 */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)n1; ++k) {
        s->Pxx[k] = s->Ix[k] * s->Ix[k];
        s->Pxy[k] = s->Ix[k] * s->Iy[k];
        s->Pyy[k] = s->Iy[k] * s->Iy[k];
    }
    /* A4 */
    stencil3(s->Pxx, s->h1, s->w1, clamp, kOnes, s->Sxx);
    stencil3(s->Pxy, s->h1, s->w1, clamp, kOnes, s->Sxy);
    stencil3(s->Pyy, s->h1, s->w1, clamp, kOnes, s->Syy);
    return 0;
}

/* R (h2 x w2) of one image. border: 0 = VALID (H,W >= 5), 1 = CLAMP. */
int oracle_harris_forward(const double* img, int64_t H, int64_t W, int border, double kappa,
                          const double* wx, const double* wy, double* R, int nthreads) {
    if (!img || !wx || !wy || !R || check_args(H, W, border)) return -1;
    set_threads(nthreads);
    stages_t s;
    int rc = run_stages(img, H, W, border, wx, wy, &s);
    if (rc) return rc;
    int64_t n2 = s.h2 * s.w2;
    /* A5 */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n2; ++k) {
        double tr = s.Sxx[k] + s.Syy[k];
        R[k] = s.Sxx[k] * s.Syy[k] - s.Sxy[k] * s.Sxy[k] - kappa * tr * tr;
    }
    free_stages(&s);
    return 0;
}

/* Cotangents of L = sum(g * R): gimg (H x W x 3), gkappa[1], gwx[9], gwy[9]. g is h2 x w2.
 * absp (nullable, 19 entries: kappa, Wx, Wy) receives the sum of |term| of each parameter
 * cotangent's sum, the scale against which a floating-point evaluation of it is judged. */
int oracle_harris_backward(const double* img, const double* g, int64_t H, int64_t W, int border,
                           double kappa, const double* wx, const double* wy, double* gimg,
                           double* gkappa, double* gwx, double* gwy, double* absp, int nthreads) {
    if (!img || !g || !wx || !wy || !gimg || !gkappa || !gwx || !gwy || check_args(H, W, border))
        return -1;
    set_threads(nthreads);
    int clamp = border == 1;
    stages_t s;
    int rc = run_stages(img, H, W, border, wx, wy, &s);
    if (rc) return rc;
    size_t n0 = (size_t)(H * W), n1 = (size_t)(s.h1 * s.w1), n2 = (size_t)(s.h2 * s.w2);
    double *gSxx = malloc(n2 * 8), *gSxy = malloc(n2 * 8), *gSyy = malloc(n2 * 8);
    double *gPxx = calloc(n1, 8), *gPxy = calloc(n1, 8), *gPyy = calloc(n1, 8);
    double *gIx = malloc(n1 * 8), *gIy = malloc(n1 * 8), *gG = calloc(n0, 8);
    if (!gSxx || !gSxy || !gSyy || !gPxx || !gPxy || !gPyy || !gIx || !gIy || !gG) {
        rc = -2;
        goto done;
    }
    /* A5 adjoint; kappa is shared by every pixel, so its cotangent is the sum. */
    double gk = 0.0, gk_abs = 0.0;
    for (size_t k = 0; k < n2; ++k) {
        double tr = s.Sxx[k] + s.Syy[k], gv = g[k];
        gSxx[k] = gv * (s.Syy[k] - 2.0 * kappa * tr);
        gSyy[k] = gv * (s.Sxx[k] - 2.0 * kappa * tr);
        gSxy[k] = -2.0 * gv * s.Sxy[k];
        gk += -gv * tr * tr;
        gk_abs += fabs(gv * tr * tr);
    }
    *gkappa = gk;
    if (absp)
        for (int t = 0; t < 19; ++t) absp[t] = 0.0;
    if (absp) absp[0] = gk_abs;
    /* A4 adjoint. */
    stencil3_vjp(s.Pxx, s.h1, s.w1, clamp, kOnes, gSxx, gPxx, NULL, NULL);
    stencil3_vjp(s.Pxy, s.h1, s.w1, clamp, kOnes, gSxy, gPxy, NULL, NULL);
    stencil3_vjp(s.Pyy, s.h1, s.w1, clamp, kOnes, gSyy, gPyy, NULL, NULL);
    /* A3 adjoint. */
    for (size_t k = 0; k < n1; ++k) {
        gIx[k] = 2.0 * s.Ix[k] * gPxx[k] + s.Iy[k] * gPxy[k];
        gIy[k] = s.Ix[k] * gPxy[k] + 2.0 * s.Iy[k] * gPyy[k];
    }
    /* A2 adjoint. */
    for (int t = 0; t < 9; ++t) { gwx[t] = 0.0; gwy[t] = 0.0; }
    stencil3_vjp(s.G, H, W, clamp, wx, gIx, gG, gwx, absp ? absp + 1 : NULL);
    stencil3_vjp(s.G, H, W, clamp, wy, gIy, gG, gwy, absp ? absp + 10 : NULL);
    /* A1 adjoint. */
    for (size_t k = 0; k < n0; ++k)
        for (int c = 0; c < 3; ++c) gimg[k * 3 + c] = kGray[c] * gG[k];
done:
    free(gSxx); free(gSxy); free(gSyy); free(gPxx); free(gPxy); free(gPyy);
    free(gIx); free(gIy); free(gG);
    free_stages(&s);
    return rc;
}

/* ---------------------------------------------------------------------------------------------
 * Point forms: the same definitions evaluated for one output at a time, for images too large
 * to hold every FP64 stage. They re-derive each value from the image directly.
 * ------------------------------------------------------------------------------------------- */

static double gray_at(const double* img, int64_t W, int64_t y, int64_t x) {
    double acc = 0.0;
    for (int c = 0; c < 3; ++c) acc = acc + img[(y * W + x) * 3 + c] * kGray[c];
    return acc;
}

/* The local footprint of one output (i, j): the 3x3 stage-2 positions it sums and, for each,
 * Ix, Iy from the 3x3 gray positions they read. Image index of stage-1 read (a2, b2) of
 * stage-2 tap (a, b) is (tap(tap(i,a),a2), tap(tap(j,b),b2)) on the respective input sizes. */
typedef struct {
    double ix[9], iy[9], sxx, sxy, syy;
    int64_t gy[9][9], gx[9][9]; /* [stage-2 tap][stage-1 tap] -> image row / column */
} local_t;

static void local_forward(const double* img, int64_t H, int64_t W, int clamp, const double* wx,
                          const double* wy, int64_t i, int64_t j, local_t* L) {
    int64_t h1 = clamp ? H : H - 2, w1 = clamp ? W : W - 2;
    L->sxx = L->sxy = L->syy = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            int64_t k = tap(i, a, h1, clamp), l = tap(j, b, w1, clamp);
            double ix = 0.0, iy = 0.0;
            for (int a2 = 0; a2 < 3; ++a2)
                for (int b2 = 0; b2 < 3; ++b2) {
                    int64_t yy = tap(k, a2, H, clamp), xx = tap(l, b2, W, clamp);
                    double gv = gray_at(img, W, yy, xx);
                    ix = ix + wx[a2 * 3 + b2] * gv;
                    iy = iy + wy[a2 * 3 + b2] * gv;
                    L->gy[a * 3 + b][a2 * 3 + b2] = yy;
                    L->gx[a * 3 + b][a2 * 3 + b2] = xx;
                }
            L->ix[a * 3 + b] = ix;
            L->iy[a * 3 + b] = iy;
            L->sxx = L->sxx + ix * ix;
            L->sxy = L->sxy + ix * iy;
            L->syy = L->syy + iy * iy;
        }
}

/* R at n output positions pts[2k] = row, pts[2k+1] = column (output coordinates). */
int oracle_harris_forward_points(const double* img, int64_t H, int64_t W, int border,
                                 double kappa, const double* wx, const double* wy,
                                 const int64_t* pts, int64_t n, double* out, int nthreads) {
    if (!img || !wx || !wy || !pts || !out || check_args(H, W, border)) return -1;
    int clamp = border == 1;
    int64_t h2 = clamp ? H : H - 4, w2 = clamp ? W : W - 4;
    for (int64_t k = 0; k < n; ++k)
        if (pts[2 * k] < 0 || pts[2 * k] >= h2 || pts[2 * k + 1] < 0 || pts[2 * k + 1] >= w2) return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; ++k) {
        local_t L;
        local_forward(img, H, W, clamp, wx, wy, pts[2 * k], pts[2 * k + 1], &L);
        double tr = L.sxx + L.syy;
        out[k] = L.sxx * L.syy - L.sxy * L.sxy - kappa * tr * tr;
    }
    return 0;
}

/* Chain rule through one output (i, j) with cotangent gv. Adds d(gv*R[i][j])/dG at image
 * position (qy, qx) to *acc_g, and (if non-NULL) the output's contributions to the parameter
 * cotangents. */
static void local_backward(const double* img, int64_t H, int64_t W, int clamp, double kappa,
                           const double* wx, const double* wy, int64_t i, int64_t j, double gv,
                           int64_t qy, int64_t qx, double* acc_g, double* gk, double* gwx,
                           double* gwy) {
    local_t L;
    local_forward(img, H, W, clamp, wx, wy, i, j, &L);
    double tr = L.sxx + L.syy;
    double gsxx = gv * (L.syy - 2.0 * kappa * tr);
    double gsyy = gv * (L.sxx - 2.0 * kappa * tr);
    double gsxy = -2.0 * gv * L.sxy;
    if (gk) *gk += -gv * tr * tr;
    for (int t = 0; t < 9; ++t) {
        /* the box sum broadcasts gS to each of its 9 products */
        double gix = 2.0 * L.ix[t] * gsxx + L.iy[t] * gsxy;
        double giy = L.ix[t] * gsxy + 2.0 * L.iy[t] * gsyy;
        for (int t2 = 0; t2 < 9; ++t2) {
            int64_t yy = L.gy[t][t2], xx = L.gx[t][t2];
            if (acc_g && yy == qy && xx == qx) *acc_g += wx[t2] * gix + wy[t2] * giy;
            if (gwx) {
                double gval = gray_at(img, W, yy, xx);
                gwx[t2] += gix * gval;
                gwy[t2] += giy * gval;
            }
        }
    }
}

/* d img at n image positions pts (row, column): out[3k + c]. g is the h2 x w2 cotangent. */
int oracle_harris_backward_points(const double* img, const double* g, int64_t H, int64_t W,
                                  int border, double kappa, const double* wx, const double* wy,
                                  const int64_t* pts, int64_t n, double* out, int nthreads) {
    if (!img || !g || !wx || !wy || !pts || !out || check_args(H, W, border)) return -1;
    int clamp = border == 1;
    int64_t h2 = clamp ? H : H - 4, w2 = clamp ? W : W - 4;
    for (int64_t k = 0; k < n; ++k)
        if (pts[2 * k] < 0 || pts[2 * k] >= H || pts[2 * k + 1] < 0 || pts[2 * k + 1] >= W) return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) {
        int64_t qy = pts[2 * k], qx = pts[2 * k + 1];
        /* Outputs that can read image position q: within 2 (clamp) or whose 5x5 footprint
         * [i, i+4] covers q (valid). Clamping only moves reads closer, so this is complete. */
        int64_t i0 = clamp ? qy - 2 : qy - 4, i1 = clamp ? qy + 2 : qy;
        int64_t j0 = clamp ? qx - 2 : qx - 4, j1 = clamp ? qx + 2 : qx;
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > h2 - 1) i1 = h2 - 1;
        if (j1 > w2 - 1) j1 = w2 - 1;
        double acc = 0.0;
        for (int64_t i = i0; i <= i1; ++i)
            for (int64_t j = j0; j <= j1; ++j)
                local_backward(img, H, W, clamp, kappa, wx, wy, i, j, g[i * w2 + j], qy,
                               qx, &acc, NULL, NULL, NULL);
        for (int c = 0; c < 3; ++c) out[3 * k + c] = kGray[c] * acc;
    }
    return 0;
}

/* d kappa, d Wx, d Wy as the sum over every output of its own chain-rule contribution, rows
 * summed in row order. Needs no FP64 stage arrays, so it covers images of any size. */
int oracle_harris_param_grads(const double* img, const double* g, int64_t H, int64_t W, int border,
                              double kappa, const double* wx, const double* wy, double* gkappa,
                              double* gwx, double* gwy, int nthreads) {
    if (!img || !g || !wx || !wy || !gkappa || !gwx || !gwy || check_args(H, W, border)) return -1;
    int clamp = border == 1;
    int64_t h2 = clamp ? H : H - 4, w2 = clamp ? W : W - 4;
    double* rows = calloc((size_t)h2 * 19, 8);
    if (!rows) return -2;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < h2; ++i) {
        double* r = rows + i * 19;
        for (int64_t j = 0; j < w2; ++j)
            local_backward(img, H, W, clamp, kappa, wx, wy, i, j, g[i * w2 + j], -1, -1,
                           NULL, &r[0], &r[1], &r[10]);
    }
    *gkappa = 0.0;
    for (int t = 0; t < 9; ++t) { gwx[t] = 0.0; gwy[t] = 0.0; }
    for (int64_t i = 0; i < h2; ++i) {
        *gkappa += rows[i * 19];
        for (int t = 0; t < 9; ++t) { gwx[t] += rows[i * 19 + 1 + t]; gwy[t] += rows[i * 19 + 10 + t]; }
    }
    free(rows);
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
