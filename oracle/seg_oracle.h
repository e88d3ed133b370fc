/*
 * seg_oracle.h -- plain, slow FP64 CPU oracle for the restricted-domain dual
 * formulation of two-phase TV segmentation (Spencer, "A Restricted-Domain
 * Dual Formulation for Two-Phase Image Segmentation", arXiv 1807.11534).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this code: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no header, helper or constant with the
 * CUDA library.
 *
 * Conventions: images are row-major [H][W] (no pitch), index i over rows,
 * j over columns, h = 1.  Region codes: 0 = Bg (u fixed at 0), 1 = Fg (u fixed
 * at 1), 2 = RD (restricted domain, where the iteration runs).
 */
#ifndef SEG_ORACLE_H
#define SEG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Fitting term: Eq. CV, and Eq. DS when n_markers > 0 (Section 1). */
void oracle_fitting(const float* z, int H, int W, double c1, double c2,
                    const int32_t* markers, int n_markers, double gamma,
                    double* f64_out, float* f32_out);

/* Class means of z over label==1 (c1, foreground) and label==0 (c2). */
/* Chan-Vese update of c1, c2 from the thresholded relaxed u (in / out). */
void oracle_update_means(const float* z, const double* u, int64_t n, double thresh,
                         double* c1, double* c2);

void oracle_class_means(const float* z, const uint8_t* label, int64_t n,
                        double* c1, double* c2);

/* q -> q-hat (Section 3): smallest threshold whose restricted domain holds at
 * least ceil(q n) pixels, decided on the float32 |f|. */
float oracle_quantile_delta(const float* f32, int64_t n, double q);

/* Fg / Bg / RD partition of Section 3, decided in float32. */
void oracle_domain(const float* f32, int64_t n, float delta, uint8_t* region);

/* Local mean of f over (2r+1)^2 squares clipped to the image (FP64 sum in
 * row-major window order, one rounding to float32). */
void oracle_box_mean(const float* f, int H, int W, int r, float* out);

/* Robust partition: RD = {|fbar| < delta} plus the pixels where f and fbar
 * differ in sign; Fg / Bg from the raw f outside RD. */
void oracle_domain_robust(const float* f32, const float* fbar, int64_t n, float delta,
                          uint8_t* region);

/* Robust restriction (Conclusion): RD grown by every pixel within Chebyshev
 * distance r of an RD pixel; the other codes are kept. */
void oracle_dilate(const uint8_t* region, int H, int W, int r, uint8_t* out);

/* Row-major linear indices of RD pixels; returns the count. */
int64_t oracle_pixel_list(const uint8_t* region, int64_t n, int32_t* list);

/* Linear ids (ty*ntx+tx, ascending) of th x tw tiles holding an RD pixel. */
int64_t oracle_tile_list(const uint8_t* region, int H, int W, int th, int tw,
                         int32_t* list);

/* RD pixel ids in tile-major order (tiles row-major, rows, columns). */
int64_t oracle_pixel_list_tiled(const uint8_t* region, int H, int W, int th, int tw,
                                int32_t* list);

/* Discrete gradient and divergence (forward differences, Neumann; the
 * divergence is minus the adjoint of the gradient). */
void oracle_grad(const double* w, int H, int W, double* g1, double* g2);
void oracle_div(const double* p1, const double* p2, int H, int W, double* d);

/* The restricted dual iteration (Sections 2.1 and 3).  warm = 0 starts from
 * u = H(-f), p = 0, v = v-step(u); warm = 1 continues from the given u, v,
 * p1, p2.  hist (nullable, 2*iters) receives ||u^l - u^(l-1)||, ||v^l - v^(l-1)||
 * for each iteration run.  Returns the number of iterations run. */
int oracle_solve(const float* f32, int H, int W, const uint8_t* region,
                 double lambda, double theta, double tau,
                 int iters, int n_inner, double tol, int warm,
                 double* u, double* v, double* p1, double* p2, double* hist);

/* 3-D volumes [D][H][W]: forward-difference gradient (components along
 * rows, columns, slices; 0 on the last one), div = -grad^T, and Section 3's
 * iteration with three components of rho (region codes per voxel). */
void oracle_grad3(const double* w, int D, int H, int W, double* g1, double* g2, double* g3);
void oracle_div3(const double* p1, const double* p2, const double* p3, int D, int H, int W,
                 double* d);
int oracle_solve3(const float* f32, int D, int H, int W, const uint8_t* region,
                  double lambda, double theta, double tau, int iters, double tol, int warm,
                  double* u, double* v, double* p1, double* p2, double* p3, double* hist);

/* Restricted primal-dual (Chambolle-Pock) solver of Eq. CR on the same
 * partition (the Conclusion's extension to other solvers): p on RD only, u
 * fixed to H(-f) outside RD; u, p1, p2 in/out (warm start when warm != 0);
 * hist[2 it] = ||u' - u||, hist[2 it + 1] = ||p' - p||.  Returns iterations done. */
int oracle_solve_pd(const float* f32, int H, int W, const uint8_t* region,
                    double lambda, double sigma, double tau, int iters, double tol,
                    int warm, double* u, double* p1, double* p2, double* hist);

/* Reverse mode of the unrolled iteration (cold start, n_inner = 1, no stop):
 * gradient of <gu, u^K> + <gv, v^K> (gv nullable) with respect to f (gf,
 * nonzero on RD only) and lambda (*glam), the partition held fixed. */
void oracle_solve_grad(const float* f32, int H, int W, const uint8_t* region,
                       double lambda, double theta, double tau, int iters,
                       const double* gu, const double* gv, double* gf, double* glam);

/* out[0] = TV(u), out[1] = E_CR(u), out[2] = E_CR(v), out[3] = E_DF(u, v),
 * out[4] = D(p) (dual lower bound), out[5] = E_CR(v) - D(p) (duality gap). */
void oracle_energy(const double* u, const double* v, const double* p1,
                   const double* p2, const float* f32, int H, int W,
                   double lambda, double theta, double* out);

/* E1 (Tanimoto of the 0.5-thresholded masks) and E2 (sum of squared
 * differences), Section 4. out[0] = E1, out[1] = E2. */
void oracle_errors(const double* u_star, const double* u_gt, int64_t n,
                   double eps, double* out);

#ifdef __cplusplus
}
#endif
#endif
