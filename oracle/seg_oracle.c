/*
 * seg_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see the
 * header).  Every function follows one passage of the paper and is written
 * for reading, not for speed: whole-image loops, no blocking, no fusion.
 *
 * Paper: J. Spencer, "A Restricted-Domain Dual Formulation for Two-Phase
 * Image Segmentation", arXiv 1807.11534.
 *
 * Readings taken where the paper is silent or garbled:
 *  - The discrete gradient/divergence are those of Chambolle (2004), which
 *    Section 2.1 cites without printing: forward differences set to 0 on the
 *    last row/column, and div = -grad^T.
 *  - The v-step of Section 2.1 prints r(x); Section 3 prints f(x).  f is used.
 *  - Section 3 writes "Fg cap Bg" for where rho = 0; that set is empty, so the
 *    union Fg cup Bg is used (rho = 0 outside RD).
 *  - The initialisation is u0 = H(-f) (Section 1; Section 3 garbles it as
 *    -H(f)), with H(s) = 1 iff s > 0, so f = 0 starts (and, outside RD, stays)
 *    in Bg.  RD = {|f| < q-hat} strictly, Fg = {f < 0} \ RD, Bg = the rest.
 *  - v0 is the v-step applied to u0; p0 = 0 (Section 3: rho initialised to 0).
 *  - n_inner fixed-point sweeps for rho per outer iteration (the paper does
 *    not say how many); the sweeps are Jacobi (all of RD from the same p^n).
 *  - The stopping norm of Section 4 is the Euclidean norm over all pixels.
 *
 * The restricted solution for 0 < q-hat < inf has no closed form.  It is
 * pinned by what it minimises: Section 3's u-step keeps rho = 0 off RD (so
 * only RD's |grad u| terms remain in TV) and evaluates the rho equation at RD
 * points with the fixed v of Fg / Bg, so the converged iterate minimises
 *   E_R(u, v) = sum_RD |grad u| + (1/2 theta) sum_all (u - v)^2
 *               + lambda sum_RD f v,   v = H(-f) off RD, u free everywhere
 * (u off RD is an auxiliary value the method never reports), which the tests
 * compare with an independent minimiser; also by the special cases and
 * invariants (q-hat = 0, q-hat = inf, |p| <= 1, v in [0,1], large lambda, the
 * disk, the 1-D ROF sub-problem, weak duality).
 */
#include "seg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j) ((int64_t)(i) * (int64_t)W + (int64_t)(j))

/* ---------------------------------------------------------------- fitting */

/* Eq. CV: f = (z - c1)^2 - (z - c2)^2 (Section 1).
 * Eq. DS: f = CV + gamma P(x), with P the Euclidean distance to the nearest
 * marker pixel divided by its maximum over the image (the paper takes P from
 * its reference [CDSS] without defining it; this normalised distance is the
 * reading used here).  Computed in FP64 in this fixed order, then rounded once
 * to float32. */
void oracle_fitting(const float* z, int H, int W, double c1, double c2,
                    const int32_t* markers, int n_markers, double gamma,
                    double* f64_out, float* f32_out)
{
    int64_t n = (int64_t)H * W;
    int64_t* d2 = NULL;
    int64_t d2max = 0;
    if (n_markers > 0) {
        d2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                int64_t best = -1;
                for (int k = 0; k < n_markers; ++k) {
                    int64_t dy = (int64_t)i - markers[2 * k];
                    int64_t dx = (int64_t)j - markers[2 * k + 1];
                    int64_t s = dy * dy + dx * dx;
                    if (best < 0 || s < best) best = s;
                }
                d2[IDX(i, j)] = best;
                if (best > d2max) d2max = best;
            }
    }
    double dmax = sqrt((double)d2max);
    for (int64_t x = 0; x < n; ++x) {
        double zz = (double)z[x];
        double t1 = zz - c1;
        double t2 = zz - c2;
        double a = t1 * t1;
        double b = t2 * t2;
        double f = a - b;
        if (n_markers > 0) {
            double P = (d2max > 0) ? sqrt((double)d2[x]) / dmax : 0.0;
            double gp = gamma * P;
            f = f + gp;
        }
        if (f64_out) f64_out[x] = f;
        if (f32_out) f32_out[x] = (float)f;
    }
    free(d2);
}

/* c1, c2 as the average foreground / background intensities (Section 1,
 * below Eq. CV), with the classes given by a label mask. */
void oracle_class_means(const float* z, const uint8_t* label, int64_t n,
                        double* c1, double* c2)
{
    double s1 = 0.0, s0 = 0.0;
    int64_t n1 = 0, n0 = 0;
    for (int64_t x = 0; x < n; ++x) {
        if (label[x]) { s1 += (double)z[x]; ++n1; }
        else          { s0 += (double)z[x]; ++n0; }
    }
    *c1 = n1 ? s1 / (double)n1 : 0.0;
    *c2 = n0 ? s0 / (double)n0 : 0.0;
}

/* Chan-Vese update of the intensities: the alternating step of the
 * piecewise-constant model ([ACWE], cited in Section 1 for Eq. CV) with the
 * relaxed u thresholded.  For fixed u the fitting energy
 * sum (z-c1)^2 [u > thresh] + (z-c2)^2 [u <= thresh] is minimised by the
 * class means; a class without pixels keeps its previous value (c1, c2 are
 * in / out).  Sums in FP64 in index order. */
void oracle_update_means(const float* z, const double* u, int64_t n, double thresh,
                         double* c1, double* c2)
{
    double s1 = 0.0, s0 = 0.0;
    int64_t n1 = 0, n0 = 0;
    for (int64_t x = 0; x < n; ++x) {
        if (u[x] > thresh) { s1 += (double)z[x]; ++n1; }
        else               { s0 += (double)z[x]; ++n0; }
    }
    if (n1) *c1 = s1 / (double)n1;
    if (n0) *c2 = s0 / (double)n0;
}

/* --------------------------------------------------------------- domain */

static int cmp_float(const void* a, const void* b)
{
    float x = *(const float*)a, y = *(const float*)b;
    return (x > y) - (x < y);
}

/* Section 3: q-hat starts at 0 and grows until the fraction of pixels in RD
 * reaches q.  With RD = {|f| < q-hat}: k = ceil(q n); q-hat = 0 for k = 0,
 * else the next float above the k-th smallest |f|. */
float oracle_quantile_delta(const float* f32, int64_t n, double q)
{
    if (n <= 0) return 0.0f;
    int64_t k = (int64_t)ceil(q * (double)n);
    if (k <= 0) return 0.0f;
    if (k > n) k = n;
    float* a = (float*)malloc(sizeof(float) * (size_t)n);
    for (int64_t x = 0; x < n; ++x) a[x] = fabsf(f32[x]);
    qsort(a, (size_t)n, sizeof(float), cmp_float);
    float t = a[k - 1];
    free(a);
    return nextafterf(t, INFINITY);
}

/* Section 3: Fg = {f <= -q-hat}, Bg = {f >= q-hat}, RD = the rest; u0 = H(-f)
 * (Section 1) decides the fixed value, so f = 0 outside RD is Bg. */
void oracle_domain(const float* f32, int64_t n, float delta, uint8_t* region)
{
    for (int64_t x = 0; x < n; ++x) {
        float f = f32[x];
        if (fabsf(f) < delta) region[x] = 2;
        else if (f < 0.0f) region[x] = 1;
        else region[x] = 0;
    }
}

/* Local mean for the robust restriction: the mean of f over the
 * (2r+1) x (2r+1) square around each pixel, clipped to the image, summed in
 * FP64 in row-major window order, divided by the count, rounded to float32. */
void oracle_box_mean(const float* f, int H, int W, int r, float* out)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double sum = 0.0;
            int cnt = 0;
            for (int a = i - r; a <= i + r; ++a)
                for (int b = j - r; b <= j + r; ++b)
                    if (a >= 0 && a < H && b >= 0 && b < W) {
                        sum += (double)f[(int64_t)a * W + b];
                        ++cnt;
                    }
            out[(int64_t)i * W + j] = (float)(sum / (double)cnt);
        }
}

/* Robust partition (the Conclusion's noisy-f case, as read here): RD =
 * {|fbar| < delta} plus the pixels where f and its local mean fbar disagree
 * in sign (their fixed value H(-f) is contradicted by the neighbourhood);
 * outside RD the codes follow the raw f as in oracle_domain. */
void oracle_domain_robust(const float* f32, const float* fbar, int64_t n, float delta,
                          uint8_t* region)
{
    for (int64_t x = 0; x < n; ++x) {
        float f = f32[x], m = fbar[x];
        if (fabsf(m) < delta || ((f < 0.0f) != (m < 0.0f))) region[x] = 2;
        else if (f < 0.0f) region[x] = 1;
        else region[x] = 0;
    }
}

/* Robust restriction (Conclusion: a robust restriction for noisy f is left
 * open; the reading here grows RD by its neighbourhood): a pixel joins RD if
 * some RD pixel lies within Chebyshev distance r, i.e. in the (2r+1) x (2r+1)
 * square around it, clipped to the image.  Other pixels keep their code. */
void oracle_dilate(const uint8_t* region, int H, int W, int r, uint8_t* out)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            uint8_t c = region[(int64_t)i * W + j];
            for (int a = i - r; a <= i + r && c != 2; ++a)
                for (int b = j - r; b <= j + r; ++b)
                    if (a >= 0 && a < H && b >= 0 && b < W && region[(int64_t)a * W + b] == 2) {
                        c = 2;
                        break;
                    }
            out[(int64_t)i * W + j] = c;
        }
}

int64_t oracle_pixel_list(const uint8_t* region, int64_t n, int32_t* list)
{
    int64_t c = 0;
    for (int64_t x = 0; x < n; ++x)
        if (region[x] == 2) {
            if (list) list[c] = (int32_t)x;
            ++c;
        }
    return c;
}

int64_t oracle_tile_list(const uint8_t* region, int H, int W, int th, int tw,
                         int32_t* list)
{
    int nty = (H + th - 1) / th, ntx = (W + tw - 1) / tw;
    int64_t c = 0;
    for (int ty = 0; ty < nty; ++ty)
        for (int tx = 0; tx < ntx; ++tx) {
            int any = 0;
            for (int i = ty * th; i < H && i < (ty + 1) * th && !any; ++i)
                for (int j = tx * tw; j < W && j < (tx + 1) * tw; ++j)
                    if (region[IDX(i, j)] == 2) { any = 1; break; }
            if (any) {
                if (list) list[c] = ty * ntx + tx;
                ++c;
            }
        }
    return c;
}

/* RD pixels numbered tile by tile (tiles in row-major order, then rows, then
 * columns inside a tile): the compact order of the GPU library's state. */
int64_t oracle_pixel_list_tiled(const uint8_t* region, int H, int W, int th, int tw,
                                int32_t* list)
{
    int nty = (H + th - 1) / th, ntx = (W + tw - 1) / tw;
    int64_t c = 0;
    for (int ty = 0; ty < nty; ++ty)
        for (int tx = 0; tx < ntx; ++tx)
            for (int i = ty * th; i < H && i < (ty + 1) * th; ++i)
                for (int j = tx * tw; j < W && j < (tx + 1) * tw; ++j)
                    if (region[IDX(i, j)] == 2) {
                        if (list) list[c] = (int32_t)IDX(i, j);
                        ++c;
                    }
    return c;
}

/* ------------------------------------------------------------ operators */

/* Chambolle (2004) gradient: forward differences, zero on the last row
 * (first component) and last column (second component). */
void oracle_grad(const double* w, int H, int W, double* g1, double* g2)
{
#pragma omp parallel for
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            g1[IDX(i, j)] = (i < H - 1) ? w[IDX(i + 1, j)] - w[IDX(i, j)] : 0.0;
            g2[IDX(i, j)] = (j < W - 1) ? w[IDX(i, j + 1)] - w[IDX(i, j)] : 0.0;
        }
}

/* Chambolle (2004) divergence, the negative adjoint of oracle_grad:
 * (div p) = [i<H-1] p1(i,j) - [i>0] p1(i-1,j) + [j<W-1] p2(i,j) - [j>0] p2(i,j-1). */
void oracle_div(const double* p1, const double* p2, int H, int W, double* d)
{
#pragma omp parallel for
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double a = (i < H - 1 ? p1[IDX(i, j)] : 0.0) - (i > 0 ? p1[IDX(i - 1, j)] : 0.0);
            double b = (j < W - 1 ? p2[IDX(i, j)] : 0.0) - (j > 0 ? p2[IDX(i, j - 1)] : 0.0);
            d[IDX(i, j)] = a + b;
        }
}

/* -------------------------------------------------------------- solver */

static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/* Section 3.  Outside RD: u = v = 1 on Fg, 0 on Bg, rho = 0.  On RD:
 *   rho^{n+1} = (rho^n + tau grad(div rho^n - v/theta))
 *               / (1 + tau |grad(div rho^n - v/theta)|)        (fixed point)
 *   u = v - theta div rho                                     (u-step)
 *   v = min(max(u - theta lambda f, 0), 1)                    (v-step)
 * alternated until the Section 4 criterion
 *   max(||u^l - u^(l-1)||, ||v^l - v^(l-1)||) <= tol
 * holds (tol <= 0: run exactly `iters` iterations). */
int oracle_solve(const float* f32, int H, int W, const uint8_t* region,
                 double lambda, double theta, double tau,
                 int iters, int n_inner, double tol, int warm,
                 double* u, double* v, double* p1, double* p2, double* hist)
{
    int64_t n = (int64_t)H * W;
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    double* w = (double*)malloc(sizeof(double) * (size_t)n);
    double* g1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* g2 = (double*)malloc(sizeof(double) * (size_t)n);
    double* q1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* q2 = (double*)malloc(sizeof(double) * (size_t)n);
    double* row_u = (double*)malloc(sizeof(double) * (size_t)H);
    double* row_v = (double*)malloc(sizeof(double) * (size_t)H);

    if (!warm) {
        for (int64_t x = 0; x < n; ++x) {
            double f = (double)f32[x];
            double h = (f < 0.0) ? 1.0 : 0.0;     /* u0 = H(-f) */
            u[x] = h;
            p1[x] = 0.0;
            p2[x] = 0.0;
            v[x] = (region[x] == 2) ? clamp01(h - theta * lambda * f) : h;
        }
    }
    /* the fixed values outside RD (also enforced on a warm start) */
    for (int64_t x = 0; x < n; ++x)
        if (region[x] != 2) {
            double h = (region[x] == 1) ? 1.0 : 0.0;
            u[x] = h;
            v[x] = h;
            p1[x] = 0.0;
            p2[x] = 0.0;
        }

    int done = 0;
    for (int it = 0; it < iters; ++it) {
        /* fixed-point sweeps for rho with v held fixed */
        for (int s = 0; s < n_inner; ++s) {
            oracle_div(p1, p2, H, W, d);
#pragma omp parallel for
            for (int64_t x = 0; x < n; ++x) w[x] = d[x] - v[x] / theta;
            oracle_grad(w, H, W, g1, g2);
#pragma omp parallel for
            for (int64_t x = 0; x < n; ++x) {
                if (region[x] == 2) {
                    double nrm = sqrt(g1[x] * g1[x] + g2[x] * g2[x]);
                    double den = 1.0 + tau * nrm;
                    q1[x] = (p1[x] + tau * g1[x]) / den;
                    q2[x] = (p2[x] + tau * g2[x]) / den;
                } else {
                    q1[x] = 0.0;
                    q2[x] = 0.0;
                }
            }
#pragma omp parallel for
            for (int64_t x = 0; x < n; ++x) {
                p1[x] = q1[x];
                p2[x] = q2[x];
            }
        }
        /* u-step then v-step on RD; the increments' squared norms are summed
         * per row, then over the rows in order */
        oracle_div(p1, p2, H, W, d);
#pragma omp parallel for
        for (int i = 0; i < H; ++i) {
            double ru = 0.0, rv = 0.0;
            for (int64_t x = IDX(i, 0); x < IDX(i, W); ++x) {
                if (region[x] != 2) continue;
                double un = v[x] - theta * d[x];
                double vn = clamp01(un - theta * lambda * (double)f32[x]);
                ru += (un - u[x]) * (un - u[x]);
                rv += (vn - v[x]) * (vn - v[x]);
                u[x] = un;
                v[x] = vn;
            }
            row_u[i] = ru;
            row_v[i] = rv;
        }
        double su = 0.0, sv = 0.0;
        for (int i = 0; i < H; ++i) {
            su += row_u[i];
            sv += row_v[i];
        }
        double du = sqrt(su), dv = sqrt(sv);
        if (hist) { hist[2 * it] = du; hist[2 * it + 1] = dv; }
        done = it + 1;
        if (tol > 0.0 && (du > dv ? du : dv) <= tol) break;
    }
    free(d); free(w); free(g1); free(g2); free(q1); free(q2); free(row_u); free(row_v);
    return done;
}

/* ------------------------------------------------------- 3-D volumes */

/* The Conclusion names 3-D problems as the next target; the method is the
 * same with a third axis.  Volumes are [D][H][W] (slice z, row i, column j),
 * grad has the components (i, j, z) as forward differences set to 0 on the
 * last row / column / slice, and div = -grad^T (Chambolle's operators with
 * one more axis). */
#define IDX3(z, i, j) (((int64_t)(z) * H + (int64_t)(i)) * (int64_t)W + (int64_t)(j))

void oracle_grad3(const double* w, int D, int H, int W, double* g1, double* g2, double* g3)
{
    for (int z = 0; z < D; ++z)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double c = w[IDX3(z, i, j)];
                g1[IDX3(z, i, j)] = (i < H - 1) ? w[IDX3(z, i + 1, j)] - c : 0.0;
                g2[IDX3(z, i, j)] = (j < W - 1) ? w[IDX3(z, i, j + 1)] - c : 0.0;
                g3[IDX3(z, i, j)] = (z < D - 1) ? w[IDX3(z + 1, i, j)] - c : 0.0;
            }
}

void oracle_div3(const double* p1, const double* p2, const double* p3, int D, int H, int W,
                 double* d)
{
    for (int z = 0; z < D; ++z)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double a = (i < H - 1 ? p1[IDX3(z, i, j)] : 0.0) - (i > 0 ? p1[IDX3(z, i - 1, j)] : 0.0);
                double b = (j < W - 1 ? p2[IDX3(z, i, j)] : 0.0) - (j > 0 ? p2[IDX3(z, i, j - 1)] : 0.0);
                double c = (z < D - 1 ? p3[IDX3(z, i, j)] : 0.0) - (z > 0 ? p3[IDX3(z - 1, i, j)] : 0.0);
                d[IDX3(z, i, j)] = a + b + c;
            }
}

/* Section 3's iteration on a volume: the same steps as oracle_solve with
 * three components of rho; region codes per voxel as oracle_domain gives
 * them for the flattened volume. */
int oracle_solve3(const float* f32, int D, int H, int W, const uint8_t* region,
                  double lambda, double theta, double tau, int iters, double tol, int warm,
                  double* u, double* v, double* p1, double* p2, double* p3, double* hist)
{
    int64_t n = (int64_t)D * H * W;
    size_t sz = sizeof(double) * (size_t)n;
    double* d = (double*)malloc(sz);
    double* w = (double*)malloc(sz);
    double* g1 = (double*)malloc(sz);
    double* g2 = (double*)malloc(sz);
    double* g3 = (double*)malloc(sz);

    for (int64_t x = 0; x < n; ++x) {
        double f = (double)f32[x];
        if (!warm) {
            double h = (f < 0.0) ? 1.0 : 0.0;
            u[x] = h;
            p1[x] = 0.0;
            p2[x] = 0.0;
            p3[x] = 0.0;
            v[x] = (region[x] == 2) ? clamp01(h - theta * lambda * f) : h;
        }
        if (region[x] != 2) {
            double h = (region[x] == 1) ? 1.0 : 0.0;
            u[x] = h;
            v[x] = h;
            p1[x] = 0.0;
            p2[x] = 0.0;
            p3[x] = 0.0;
        }
    }
    int done = 0;
    for (int it = 0; it < iters; ++it) {
        oracle_div3(p1, p2, p3, D, H, W, d);
        for (int64_t x = 0; x < n; ++x) w[x] = d[x] - v[x] / theta;
        oracle_grad3(w, D, H, W, g1, g2, g3);
        for (int64_t x = 0; x < n; ++x) {
            if (region[x] != 2) continue;
            double nrm = sqrt(g1[x] * g1[x] + g2[x] * g2[x] + g3[x] * g3[x]);
            double den = 1.0 + tau * nrm;
            p1[x] = (p1[x] + tau * g1[x]) / den;
            p2[x] = (p2[x] + tau * g2[x]) / den;
            p3[x] = (p3[x] + tau * g3[x]) / den;
        }
        oracle_div3(p1, p2, p3, D, H, W, d);
        double su = 0.0, sv = 0.0;
        for (int64_t x = 0; x < n; ++x) {
            if (region[x] != 2) continue;
            double un = v[x] - theta * d[x];
            double vn = clamp01(un - theta * lambda * (double)f32[x]);
            su += (un - u[x]) * (un - u[x]);
            sv += (vn - v[x]) * (vn - v[x]);
            u[x] = un;
            v[x] = vn;
        }
        double du = sqrt(su), dv = sqrt(sv);
        if (hist) { hist[2 * it] = du; hist[2 * it + 1] = dv; }
        done = it + 1;
        if (tol > 0.0 && (du > dv ? du : dv) <= tol) break;
    }
    free(d); free(w); free(g1); free(g2); free(g3);
    return done;
}

/* ------------------------------------------ restricted primal-dual solver */

/* The Conclusion proposes carrying the restriction over to other solvers of
 * Eq. CR.  This is the first-order primal-dual method of Chambolle and Pock
 * (2011) on the same partition, with the same restriction as Section 3 (the
 * dual variable is 0 outside RD, u fixed to H(-f) there):
 *   p <- P(p + sigma grad ubar)      on RD, P the projection onto |p| <= 1
 *   u' = clip(u + tau (div p - lambda f), 0, 1)                      on RD
 *   ubar = 2 u' - u
 * from u0 = H(-f), ubar0 = u0, p0 = 0 (or the caller's u, p), sigma tau <= 1/8
 * for convergence (||grad||^2 <= 8).  Stopping test (Section 4's, with p in
 * the place of v): max(||u' - u||, ||p' - p||) <= tol, checked every
 * iteration; hist gets the two norms.  Returns the iterations done. */
int oracle_solve_pd(const float* f32, int H, int W, const uint8_t* region,
                    double lambda, double sigma, double tau, int iters, double tol,
                    int warm, double* u, double* p1, double* p2, double* hist)
{
    int64_t n = (int64_t)H * W;
    size_t sz = sizeof(double) * (size_t)n;
    double* ub = (double*)malloc(sz);
    double* g1 = (double*)malloc(sz);
    double* g2 = (double*)malloc(sz);
    double* d = (double*)malloc(sz);

    for (int64_t x = 0; x < n; ++x) {
        if (!warm) {
            u[x] = ((double)f32[x] < 0.0) ? 1.0 : 0.0;
            p1[x] = 0.0;
            p2[x] = 0.0;
        }
        if (region[x] != 2) {
            u[x] = (region[x] == 1) ? 1.0 : 0.0;
            p1[x] = 0.0;
            p2[x] = 0.0;
        }
        ub[x] = u[x];
    }
    int done = 0;
    for (int it = 0; it < iters; ++it) {
        /* dual ascent step and projection */
        oracle_grad(ub, H, W, g1, g2);
        double sp = 0.0;
        for (int64_t x = 0; x < n; ++x) {
            if (region[x] != 2) continue;
            double a = p1[x] + sigma * g1[x];
            double b = p2[x] + sigma * g2[x];
            double nrm = sqrt(a * a + b * b);
            double s = nrm > 1.0 ? nrm : 1.0;
            a /= s;
            b /= s;
            sp += (a - p1[x]) * (a - p1[x]) + (b - p2[x]) * (b - p2[x]);
            p1[x] = a;
            p2[x] = b;
        }
        /* primal descent step, clip, extrapolation */
        oracle_div(p1, p2, H, W, d);
        double su = 0.0;
        for (int64_t x = 0; x < n; ++x) {
            if (region[x] != 2) continue;
            double un = clamp01(u[x] + tau * (d[x] - lambda * (double)f32[x]));
            su += (un - u[x]) * (un - u[x]);
            ub[x] = 2.0 * un - u[x];
            u[x] = un;
        }
        double du = sqrt(su), dp = sqrt(sp);
        if (hist) { hist[2 * it] = du; hist[2 * it + 1] = dp; }
        done = it + 1;
        if (tol > 0.0 && (du > dp ? du : dp) <= tol) break;
    }
    free(ub); free(g1); free(g2); free(d);
    return done;
}

/* ------------------------------------------------------- reverse mode */

/* Gradient of L = <gu, u^K> + <gv, v^K> through the unrolled iteration of
 * oracle_solve (cold start, n_inner = 1, `iters` = K iterations, no stopping
 * test), with respect to f on RD (gf; 0 elsewhere) and lambda (*glam).  The
 * partition is held fixed (no derivative through the threshold), u0 = H(-f)
 * is piecewise constant, and the clip has derivative 1 strictly inside (0,1)
 * and 0 elsewhere; d|g| is taken as 0 at g = 0.  Plain reverse-mode
 * differentiation of the same steps, storing every iterate:
 *   v = clip(s), s = u - theta lambda f:  sbar = vbar [0 < s < 1],
 *       fbar -= theta lambda sbar, lambdabar -= theta sum f sbar
 *   u = v_prev - theta div p:            v_prevbar += ubar, pbar += theta grad ubar
 *   p = (p_prev + tau g) / d, d = 1 + tau |g|:
 *       p_prevbar += pbar / d,  gbar = (tau / d) (pbar - (pbar . p) g/|g|)
 *   g = grad w:                          wbar = -div gbar
 *   w = div p_prev - v_prev / theta:      p_prevbar -= grad wbar, v_prevbar -= wbar / theta
 * (div^T = -grad, so grad^T = -div.) */
void oracle_solve_grad(const float* f32, int H, int W, const uint8_t* region,
                       double lambda, double theta, double tau, int iters,
                       const double* gu, const double* gv, double* gf, double* glam)
{
    int64_t n = (int64_t)H * W;
    size_t sz = sizeof(double) * (size_t)n;
    int K = iters;
    double* P1 = (double*)malloc(sz * (size_t)(K + 1));
    double* P2 = (double*)malloc(sz * (size_t)(K + 1));
    double* V = (double*)malloc(sz * (size_t)(K + 1));
    double* U = (double*)malloc(sz * (size_t)(K + 1));
    double* d = (double*)malloc(sz);
    double* w = (double*)malloc(sz);
    double* g1 = (double*)malloc(sz);
    double* g2 = (double*)malloc(sz);
    double* ub = (double*)malloc(sz);
    double* vb = (double*)malloc(sz);
    double* p1b = (double*)malloc(sz);
    double* p2b = (double*)malloc(sz);
    double* gb1 = (double*)malloc(sz);
    double* gb2 = (double*)malloc(sz);
    double* wb = (double*)malloc(sz);
    double* t1 = (double*)malloc(sz);
    double* t2 = (double*)malloc(sz);

    /* forward, every iterate kept */
    for (int64_t x = 0; x < n; ++x) {
        double f = (double)f32[x];
        double h = (f < 0.0) ? 1.0 : 0.0;
        if (region[x] != 2) h = (region[x] == 1) ? 1.0 : 0.0;
        U[x] = h;
        P1[x] = 0.0;
        P2[x] = 0.0;
        V[x] = (region[x] == 2) ? clamp01(h - theta * lambda * f) : h;
    }
    for (int k = 0; k < K; ++k) {
        double *p1 = P1 + (int64_t)k * n, *p2 = P2 + (int64_t)k * n, *v = V + (int64_t)k * n;
        double *q1 = P1 + (int64_t)(k + 1) * n, *q2 = P2 + (int64_t)(k + 1) * n;
        double *un = U + (int64_t)(k + 1) * n, *vn = V + (int64_t)(k + 1) * n;
        oracle_div(p1, p2, H, W, d);
        for (int64_t x = 0; x < n; ++x) w[x] = d[x] - v[x] / theta;
        oracle_grad(w, H, W, g1, g2);
        for (int64_t x = 0; x < n; ++x) {
            if (region[x] == 2) {
                double den = 1.0 + tau * sqrt(g1[x] * g1[x] + g2[x] * g2[x]);
                q1[x] = (p1[x] + tau * g1[x]) / den;
                q2[x] = (p2[x] + tau * g2[x]) / den;
            } else {
                q1[x] = 0.0;
                q2[x] = 0.0;
            }
        }
        oracle_div(q1, q2, H, W, d);
        for (int64_t x = 0; x < n; ++x) {
            if (region[x] == 2) {
                un[x] = v[x] - theta * d[x];
                vn[x] = clamp01(un[x] - theta * lambda * (double)f32[x]);
            } else {
                un[x] = U[x];
                vn[x] = V[x];
            }
        }
    }

    /* reverse */
    double lb = 0.0;
    for (int64_t x = 0; x < n; ++x) {
        gf[x] = 0.0;
        vb[x] = (region[x] == 2 && gv) ? gv[x] : 0.0;
        p1b[x] = 0.0;
        p2b[x] = 0.0;
    }
    for (int k = K - 1; k >= 0; --k) {
        double *p1 = P1 + (int64_t)k * n, *p2 = P2 + (int64_t)k * n, *v = V + (int64_t)k * n;
        double *q1 = P1 + (int64_t)(k + 1) * n, *q2 = P2 + (int64_t)(k + 1) * n;
        double *un = U + (int64_t)(k + 1) * n;
        /* v^{k+1} = clip(u^{k+1} - theta lambda f) */
        for (int64_t x = 0; x < n; ++x) {
            ub[x] = 0.0;
            if (region[x] != 2) continue;
            double f = (double)f32[x];
            double sv = un[x] - theta * lambda * f;
            double sb = (sv > 0.0 && sv < 1.0) ? vb[x] : 0.0;
            ub[x] = sb + ((k == K - 1) ? gu[x] : 0.0);
            gf[x] -= theta * lambda * sb;
            lb -= theta * f * sb;
        }
        /* u^{k+1} = v^k - theta div p^{k+1}: pbar += theta grad ubar on RD */
        oracle_grad(ub, H, W, t1, t2);
        for (int64_t x = 0; x < n; ++x) {
            if (region[x] != 2) continue;
            p1b[x] += theta * t1[x];
            p2b[x] += theta * t2[x];
        }
        /* p^{k+1} = (p^k + tau g^k) / d */
        oracle_div(p1, p2, H, W, d);
        for (int64_t x = 0; x < n; ++x) w[x] = d[x] - v[x] / theta;
        oracle_grad(w, H, W, g1, g2);
        for (int64_t x = 0; x < n; ++x) {
            gb1[x] = 0.0;
            gb2[x] = 0.0;
            if (region[x] != 2) { p1b[x] = 0.0; p2b[x] = 0.0; continue; }
            double nrm = sqrt(g1[x] * g1[x] + g2[x] * g2[x]);
            double den = 1.0 + tau * nrm;
            double dot = p1b[x] * q1[x] + p2b[x] * q2[x];
            double h1 = nrm > 0.0 ? g1[x] / nrm : 0.0, h2 = nrm > 0.0 ? g2[x] / nrm : 0.0;
            gb1[x] = (tau / den) * (p1b[x] - dot * h1);
            gb2[x] = (tau / den) * (p2b[x] - dot * h2);
            p1b[x] = p1b[x] / den;
            p2b[x] = p2b[x] / den;
        }
        /* g = grad w (zero components carry no adjoint) */
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                if (i == H - 1) gb1[IDX(i, j)] = 0.0;
                if (j == W - 1) gb2[IDX(i, j)] = 0.0;
            }
        oracle_div(gb1, gb2, H, W, d);
        for (int64_t x = 0; x < n; ++x) wb[x] = -d[x];
        /* w = div p^k - v^k / theta */
        oracle_grad(wb, H, W, t1, t2);
        for (int64_t x = 0; x < n; ++x) {
            if (region[x] != 2) { vb[x] = 0.0; continue; }
            p1b[x] -= t1[x];
            p2b[x] -= t2[x];
            vb[x] = ub[x] - wb[x] / theta;
        }
    }
    /* v^0 = clip(u^0 - theta lambda f) */
    for (int64_t x = 0; x < n; ++x) {
        if (region[x] != 2) continue;
        double f = (double)f32[x];
        double sv = U[x] - theta * lambda * f;
        double sb = (sv > 0.0 && sv < 1.0) ? vb[x] : 0.0;
        gf[x] -= theta * lambda * sb;
        lb -= theta * f * sb;
    }
    *glam = lb;
    free(P1); free(P2); free(V); free(U); free(d); free(w); free(g1); free(g2);
    free(ub); free(vb); free(p1b); free(p2b); free(gb1); free(gb2); free(wb); free(t1); free(t2);
}

/* ------------------------------------------------------------- energies */

static double tv(const double* u, int H, int W)
{
    double s = 0.0;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double a = (i < H - 1) ? u[IDX(i + 1, j)] - u[IDX(i, j)] : 0.0;
            double b = (j < W - 1) ? u[IDX(i, j + 1)] - u[IDX(i, j)] : 0.0;
            s += sqrt(a * a + b * b);
        }
    return s;
}

/* Eq. CR energy TV(u) + lambda sum f u; Eq. DF energy (with the exact-penalty
 * term psi(v) = 0 for v in [0,1]); the dual bound
 *   D(p) = sum min(0, lambda f + div p),
 * obtained from TV(u) = max_{|p|<=1} <u, div p> and minimising over u in [0,1]
 * pixel by pixel (valid when |p| <= 1); gap = E_CR(v) - D(p) >= 0. */
void oracle_energy(const double* u, const double* v, const double* p1,
                   const double* p2, const float* f32, int H, int W,
                   double lambda, double theta, double* out)
{
    int64_t n = (int64_t)H * W;
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    oracle_div(p1, p2, H, W, d);
    double tvu = tv(u, H, W), tvv = tv(v, H, W);
    double fu = 0.0, fv = 0.0, quad = 0.0, dual = 0.0;
    for (int64_t x = 0; x < n; ++x) {
        double f = (double)f32[x];
        fu += f * u[x];
        fv += f * v[x];
        quad += (u[x] - v[x]) * (u[x] - v[x]);
        double c = lambda * f + d[x];
        dual += (c < 0.0) ? c : 0.0;
    }
    out[0] = tvu;
    out[1] = tvu + lambda * fu;
    out[2] = tvv + lambda * fv;
    out[3] = tvu + quad / (2.0 * theta) + lambda * fv;
    out[4] = dual;
    out[5] = out[2] - dual;
    free(d);
}

/* Section 4: GT = {u_gt > eps}, Omega* = {u* > eps};
 * E1 = N(GT cap Omega*) / N(GT cup Omega*) (1 when both are empty),
 * E2 = sum (u* - u_gt)^2 (h = 1). */
void oracle_errors(const double* u_star, const double* u_gt, int64_t n,
                   double eps, double* out)
{
    int64_t inter = 0, uni = 0;
    double e2 = 0.0;
    for (int64_t x = 0; x < n; ++x) {
        int a = u_gt[x] > eps, b = u_star[x] > eps;
        inter += a && b;
        uni += a || b;
        e2 += (u_star[x] - u_gt[x]) * (u_star[x] - u_gt[x]);
    }
    out[0] = uni ? (double)inter / (double)uni : 1.0;
    out[1] = e2;
}
