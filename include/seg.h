/*
 * seg.h -- C ABI of libseg, a GB300 (sm_103a) implementation of the
 * restricted-domain dual formulation of two-phase TV segmentation
 * (J. Spencer, "A Restricted-Domain Dual Formulation for Two-Phase Image
 * Segmentation", arXiv 1807.11534).
 *
 * The method minimises the convex relaxation (Eq. CR, Section 2)
 *     min_{u in [0,1]}  TV(u) + lambda * sum f u
 * with the dual splitting of Section 2.1 (Eq. DF): a fixed-point step on the
 * dual field p (the paper's rho), u = v - theta div p, and
 * v = clip(u - theta lambda f, 0, 1), run only on the restricted domain
 * RD = {|f| < delta} of Section 3 while u = v = H(-f) elsewhere and p = 0.
 *
 * Conventions (all entry points):
 *  - Images are row-major float32 [H][ld] in device memory; ld (elements) is
 *    a multiple of 32 and ld >= W.  Entries in columns W..ld-1 are ignored on
 *    input and left untouched on output.
 *  - Bit masks are uint32 [H][ld/32]: bit b of word k in row i is pixel
 *    (i, 32k + b); bits beyond W are 0.
 *  - Tiles are 32 columns wide (one mask word) and tile_h rows high
 *    (tile_h in {4, 8, 16, 32}); tile id = ty * ceil(W/32) + tx.
 *  - All pointers are device pointers unless a comment says "host".  The
 *    caller allocates every buffer (through any allocator; PyTorch in the
 *    Python binding); the library never allocates device memory.  Scratch
 *    comes from a caller-provided workspace of seg_workspace_bytes() bytes,
 *    16-byte aligned, zero-filled before its first use, owned by the caller,
 *    used by one call at a time.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) and returns a seg_status for errors found on the host
 *    (arguments, launch failures).  Errors found on the device (non-finite
 *    input, capacity overflow) are recorded in the workspace status word and
 *    returned by seg_read_status(), which synchronises the stream.
 *  - seg_last_error() returns a thread-local message for the last failure.
 */
#ifndef SEG_H
#define SEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int seg_status;
#define SEG_OK 0
#define SEG_ERR_INVALID_ARG 1   /* bad size, null pointer, bad parameter */
#define SEG_ERR_ALIGN 2         /* ld not a multiple of 32, pointer not 16-byte aligned */
#define SEG_ERR_CUDA 3          /* a CUDA runtime call failed (message has the reason) */
#define SEG_ERR_CAPACITY 4      /* an output buffer is smaller than the result */
#define SEG_ERR_TIMEOUT 5       /* a bounded device-side wait ran out */
#define SEG_ERR_NONFINITE 6     /* the fitting term holds NaN or Inf */
#define SEG_ERR_WORKSPACE 7     /* workspace missing or smaller than required */

/* solve modes */
#define SEG_MODE_DENSE 0        /* dense [H][ld] state, tile list of the domain, fused stencil */
#define SEG_MODE_COMPACT 1      /* state stored only for RD pixels (tile-major compact order) */
#define SEG_MODE_TILED 2        /* dense [H][ld] state, several iterations per pass: each
                                   60 x 68 window (own region + a halo as wide as the
                                   iterations it runs) is iterated in shared memory over
                                   its RD pixels; float32 storage only */

/* storage types of the iteration state (p1, p2, v); arithmetic is float32 */
#define SEG_STORE_F32 0
#define SEG_STORE_BF16 1
#define SEG_STORE_F16 2

/* Parameters of one solve (host struct, read during the call only). */
typedef struct seg_params {
    double lambda;      /* weight of the fitting term, Eq. CR */
    double theta;       /* coupling of u and v, Eq. DF (default 0.2) */
    double tau;         /* fixed-point step for p, Section 3 (default 0.125 = 1/8) */
    double tol;         /* stop when max(||du||,||dv||) <= tol (Section 4); <= 0: run `iters` */
    int iters;          /* maximum number of outer iterations */
    int n_inner;        /* fixed-point sweeps for p per outer iteration (>= 1; default 1) */
    int check_every;    /* evaluate the stopping test every this many iterations (>= 1); with
                           tol <= 0 the dense, compact and batch solves test only the last
                           iteration (nothing is decided; stats hold that test's norms) */
    int warm_start;     /* 0: start from u = H(-f), p = 0, v = v-step(u); 1: from the u, v, p1, p2 given */
    int mode;           /* SEG_MODE_DENSE, SEG_MODE_COMPACT or SEG_MODE_TILED */
    int storage;        /* SEG_STORE_*; 16-bit storage is SEG_MODE_COMPACT only */
    int tile_h;         /* tile height used by seg_build_domain for this domain */
    int sweep;          /* SEG_MODE_TILED: outer iterations per window pass (0: 4);
                           sweep * n_inner <= 8.  Ignored by the other modes. */
} seg_params;

/* Library version (major*10000 + minor*100 + patch). */
int seg_version(void);

/* Thread-local message of the last failed call ("" if none). */
const char* seg_last_error(void);

/* Number of kernel launches the library has issued in this process (host
 * counter, for diagnostics and launch accounting). */
unsigned long long seg_launch_count(void);

/* Workspace bytes needed by any call on an H x W image with pitch ld, up to
 * n_tiles_cap active tiles of height tile_h.  Never zero. */
size_t seg_workspace_bytes(int H, int W, int ld, int tile_h);

/* Bytes of iteration state for seg_solve: dense mode 6*H*ld float32
 * (ping-pong p1, p2, v); tiled mode the same planes plus the RD pixel list of
 * every window (about 4 bytes per pixel); compact mode room for `capacity` RD pixels
 * (ping-pong p1, p2, v in the storage type, plus f, u and the pixel list). */
size_t seg_state_bytes(int H, int ld, int64_t capacity, int mode, int storage);

/* Synchronise `stream` and return the device status word of the workspace
 * (SEG_OK or the first device-side error), then clear it. */
seg_status seg_read_status(void* ws, size_t ws_bytes, void* stream);

/* Diagnostics of the device-side waits (no counterpart in the paper).  Every
 * wait inside a kernel -- the grid barriers of the persistent solvers, the
 * TMA completions of the tiled solver -- gives up after a bounded number of
 * SM clock cycles, records SEG_ERR_TIMEOUT in the workspace status word,
 * raises the workspace's done flag and returns, so a lost block never hangs
 * the GPU.  This call sets, for later calls on this workspace:
 *   wait_cycles     the bound (> 0), or 0 for the default of 2e9 cycles
 *                   (about 1 s at the SM clock);
 *   extra_arrivals  0 for normal operation; k > 0 makes every grid barrier
 *                   wait for k arrivals beyond the launch's blocks, arrivals
 *                   that never come, so that every such wait runs out after
 *                   wait_cycles (the way the tests drive the timeout path).
 * The values stay in the workspace header until the next call; a solve that
 * timed out leaves its outputs undefined.  Asynchronous on `stream`.
 * Errors: INVALID_ARG (negative values), WORKSPACE, CUDA. */
seg_status seg_set_wait_limit(void* ws, size_t ws_bytes, long long wait_cycles, int extra_arrivals,
                              void* stream);

/* Fitting term (Section 1): Eq. CV  f = (z - c1)^2 - (z - c2)^2, and when
 * n_markers > 0 Eq. DS  f = CV + gamma P(x), with P the Euclidean distance to
 * the nearest marker pixel divided by its maximum over the image.
 *   z        [H][ld] float32 image.
 *   c1, c2   foreground / background intensities (host doubles), used when
 *            label == NULL; both NaN: the c1, c2 the workspace holds from the
 *            last seg_make_fitting or seg_update_means on it (so a Chan-Vese
 *            loop needs no host round trip).
 *   label    NULL, or uint8 [H][ld] class mask: c1 = mean of z where label != 0,
 *            c2 = mean where label == 0 (FP64 on the device).
 *   markers  NULL or int32 [n_markers][2] (row, col) device array.
 *   f        out [H][ld] float32; computed in FP64 and rounded once.
 *   c_out    NULL or out double[2] (device): the c1, c2 used.
 * Errors: INVALID_ARG (sizes, null z/f, markers NULL with n_markers > 0),
 * ALIGN, WORKSPACE, CUDA. */
seg_status seg_make_fitting(const float* z, int H, int W, int ld,
                            double c1, double c2, const uint8_t* label,
                            const int32_t* markers, int n_markers, double gamma,
                            float* f, double* c_out,
                            void* ws, size_t ws_bytes, void* stream);

/* Chan-Vese update of the intensities of Eq. CV (the alternating step of the
 * piecewise-constant model the fitting term of Section 1 comes from [ACWE],
 * with the relaxed u thresholded): c1 = mean of z over {u > thresh}, c2 =
 * mean of z over {u <= thresh}, in FP64 with a fixed-order reduction.  A
 * class with no pixel keeps the value the workspace held.  The result is
 * stored in the workspace (for seg_make_fitting with c1 = c2 = NaN) and, if
 * c_out is not NULL, in c_out (device double[2]).
 *   z, u     [H][ld] float32 image and relaxed indicator.
 * Errors: INVALID_ARG (sizes, NULL z/u, non-finite thresh), ALIGN, WORKSPACE,
 * CUDA. */
seg_status seg_update_means(const float* z, const float* u, int H, int W, int ld,
                            double thresh, double* c_out,
                            void* ws, size_t ws_bytes, void* stream);

/* Restricted domain (Section 3): RD = {|f| < delta}, Fg = {f < 0} \ RD,
 * Bg = rest (u0 = H(-f), Section 1, with H(0) = 0).  When q >= 0 delta is
 * chosen from q as in Section 3: the smallest threshold whose RD holds at
 * least ceil(q * H * W) pixels, i.e. the float just above the k-th smallest
 * |f| (exact radix select on the float bits); q < 0 uses `delta` as given.
 *   act, fg   out uint32 [H][ld/32]: RD bits, and f < 0 bits (all pixels).
 *   wstart    out int32 [H][ld/32]: compact index of the first RD pixel of
 *             each word in tile-major order (tiles row-major, rows top to
 *             bottom inside a tile, columns left to right).
 *   tiles     out int32 [tiles_cap]: ids of tiles holding an RD pixel, ascending.
 *   pixels    NULL or out int32 [pixels_cap]: linear ids i*W + j of RD pixels
 *             in tile-major compact order.
 *   counts    out int32[4] (device): n_tiles, n_active, n_fg (fixed Fg pixels),
 *             and the k of quantile mode (0 otherwise).
 *   delta_out NULL or out float[1] (device): the threshold used.
 * The lists are bit-exact functions of f.  Overflowing tiles_cap/pixels_cap
 * records SEG_ERR_CAPACITY in the status word; a NaN/Inf in f records
 * SEG_ERR_NONFINITE.  Host-side errors: INVALID_ARG, ALIGN, WORKSPACE, CUDA. */
seg_status seg_build_domain(const float* f, int H, int W, int ld,
                            double delta, double q, int tile_h,
                            uint32_t* act, uint32_t* fg, int32_t* wstart,
                            int32_t* tiles, int tiles_cap,
                            int32_t* pixels, int64_t pixels_cap,
                            int32_t* counts, float* delta_out,
                            void* ws, size_t ws_bytes, void* stream);

/* Robust restriction (the Conclusion leaves open how to restrict the domain
 * robustly when f is noisy; this is the reading used here).  As
 * seg_build_domain, with two optional changes:
 *   fbar     NULL (or f): RD = {|f| < delta}.  Otherwise a device [H][ld]
 *            float32 field, normally the local mean of f from seg_box_mean:
 *            RD = {|fbar| < delta} united with the pixels where f and fbar
 *            have different signs ((f < 0) != (fbar < 0)), i.e. the pixels
 *            whose fixed value H(-f) their neighbourhood contradicts; in
 *            quantile mode delta is the quantile of |fbar|.
 *   radius   RD is then grown by every pixel within Chebyshev distance radius
 *            of an RD pixel (a (2r+1) x (2r+1) square dilation clipped to the
 *            image); 0 = no growth.
 * Fg = {f < 0} outside the final RD (the fixed values stay H(-f) of the raw
 * f), Bg = the rest; counts and lists describe the final RD.  With fbar NULL
 * and radius 0 the outputs equal seg_build_domain's.  wstart is used as
 * scratch before it is written.
 * Errors: as seg_build_domain (NaN/Inf in fbar too), and INVALID_ARG for
 * radius outside [0, 32]. */
seg_status seg_build_domain_robust(const float* f, const float* fbar, int H, int W, int ld,
                                   double delta, double q, int radius, int tile_h,
                                   uint32_t* act, uint32_t* fg, int32_t* wstart,
                                   int32_t* tiles, int tiles_cap,
                                   int32_t* pixels, int64_t pixels_cap,
                                   int32_t* counts, float* delta_out,
                                   void* ws, size_t ws_bytes, void* stream);

/* Local mean for the robust restriction: out[i][j] = the mean of f over the
 * (2r+1) x (2r+1) square around (i, j) clipped to the image, the window's
 * values summed in FP64 in row-major order, divided by their count and
 * rounded once to float32 (a bit-exact function of f).  Columns >= W of out
 * are not written.
 *   f, out   device [H][ld] float32, not aliased.
 * Errors: INVALID_ARG (sizes, NULL, aliasing, radius outside [0, 16]), ALIGN,
 * CUDA. */
seg_status seg_box_mean(const float* f, int H, int W, int ld, int radius, float* out,
                        void* stream);

/* Restricted dual iteration (Sections 2.1 and 3) on the domain built by
 * seg_build_domain for the same f and tile_h:
 *   p <- (p + tau g) / (1 + tau |g|),  g = grad(div p - v/theta)   on RD
 *   u  = v - theta div p,  v = clip(u - theta lambda f, 0, 1)       on RD
 * with p = 0 and u = v = H(-f) outside RD, alternated prm->iters times or
 * until the Section 4 test max(||u^l - u^(l-1)||, ||v^l - v^(l-1)||) <= tol
 * (Euclidean norms over the image, checked every check_every iterations).
 *   u, v, p1, p2  [H][ld] float32: the warm start on input when
 *                 prm->warm_start, and the final iterate on output.
 *   state         seg_state_bytes(H, ld, capacity, mode, storage) bytes
 *                 (compact mode: capacity >= n_active).
 * SEG_MODE_TILED additionally needs f 16-byte aligned (it is read by TMA)
 * and returns INVALID_ARG when sweep * n_inner > 8.
 *   stats         out double[8] (device): [0] iterations run, [1] last
 *                 ||du||, [2] last ||dv|| (from the last check), [3] n_active,
 *                 [4] n_tiles, [5] iteration of the last check, [6] compact
 *                 mode: blocks of the persistent solver that kept their
 *                 pixels' state in shared memory, [7] compact mode: blocks
 *                 that ran one grid barrier per iteration (diagnostics).
 * Errors: INVALID_ARG, ALIGN, WORKSPACE, CUDA on the host; CAPACITY (compact
 * state too small) in the status word. */
seg_status seg_solve(const float* f, int H, int W, int ld,
                     const uint32_t* act, const uint32_t* fg, const int32_t* wstart,
                     const int32_t* tiles, const int32_t* counts,
                     const seg_params* prm,
                     float* u, float* v, float* p1, float* p2,
                     void* state, size_t state_bytes, double* stats,
                     void* ws, size_t ws_bytes, void* stream);

/* 3-D volumes (the Conclusion names 3-D problems as the next target): the
 * same iteration as seg_solve with a third component of p and the slice
 * neighbours.  A volume is [D][H][ld] float32 (slice z, row i, column j; the
 * rows of all slices stacked), so seg_make_fitting (without markers) and
 * seg_build_domain / seg_build_domain_robust apply to it as a (D*H) x W
 * image, and their act, fg, pixels and counts are the partition of the
 * volume; the iteration runs over its RD voxel list (seg_build_domain's
 * `pixels`, linear ids (z*H + i)*W + j in tile-major order).  grad is the
 * forward difference along rows, columns and slices (0
 * on the last one), div = -grad^T:
 *   p <- (p + tau g) / (1 + tau |g|),  g = grad(div p - v/theta)   on RD
 *   u  = v - theta div p,  v = clip(u - theta lambda f, 0, 1)       on RD
 * with p = 0 and u = v = H(-f) outside RD, the Section 4 test as seg_solve.
 *   prm           lambda, theta, tau, tol, iters, check_every, warm_start,
 *                 tile_h (as for seg_build_domain) are used; n_inner must be
 *                 1 and storage SEG_STORE_F32; mode is ignored.
 *   u, v, p1, p2, p3  [D][H][ld] float32: warm start in, result out (p1
 *                 along rows, p2 along columns, p3 along slices).
 *   wstart, voxels  seg_build_domain's compact starts and RD voxel list
 *                 (`pixels`) for the stacked image.
 *   state         seg_state_bytes3d(capacity) bytes, 256-byte aligned: the
 *                 compact state of up to `capacity` RD voxels (92 bytes each).
 *   stats         out double[8] (device), as seg_solve.
 * Errors: INVALID_ARG, ALIGN, WORKSPACE (a workspace for the (D*H) x W
 * image), CUDA on the host; CAPACITY (more RD voxels than the state holds)
 * and TIMEOUT in the status word. */
size_t seg_state_bytes3d(int64_t capacity);
seg_status seg_solve3d(const float* f, int D, int H, int W, int ld,
                       const uint32_t* act, const uint32_t* fg, const int32_t* wstart,
                       const int32_t* voxels,
                       const int32_t* counts, const seg_params* prm,
                       float* u, float* v, float* p1, float* p2, float* p3,
                       void* state, size_t state_bytes, double* stats,
                       void* ws, size_t ws_bytes, void* stream);

/* Parameters of a restricted primal-dual solve (host struct, read during the
 * call only). */
typedef struct seg_pd_params {
    double lambda;      /* weight of the fitting term, Eq. CR */
    double sigma;       /* dual step (default 1/sqrt(8)) */
    double tau;         /* primal step (default 1/sqrt(8)); sigma tau <= 1/8 converges */
    double tol;         /* stop when max(||du||, ||dp||) <= tol; <= 0: run `iters` */
    int iters;          /* maximum number of iterations */
    int check_every;    /* evaluate the stopping test every this many iterations (>= 1); with
                           tol <= 0 only the last iteration is tested */
    int warm_start;     /* 0: start from u = H(-f), p = 0; 1: from the u, p1, p2 given */
    int tile_h;         /* tile height used by seg_build_domain for this domain */
} seg_pd_params;

/* Restricted primal-dual solver of Eq. CR (the Conclusion proposes carrying
 * the restriction over to other solvers of Eq. CR; this is the first-order
 * primal-dual method of Chambolle and Pock, 2011) on the domain built by
 * seg_build_domain, with Section 3's restriction (p = 0 and u = H(-f)
 * outside RD):
 *   p <- P(p + sigma grad ubar),  P the projection onto |p| <= 1    on RD
 *   u' = clip(u + tau (div p - lambda f), 0, 1),  ubar = 2 u' - u    on RD
 * from ubar = u, alternated prm->iters times or until max(||u' - u||,
 * ||p' - p||) <= tol (Section 4's test with p in the place of v, checked every
 * check_every iterations).  Unlike seg_solve it minimises Eq. CR itself (no
 * theta coupling); grad/div are the same discrete operators.
 *   u, p1, p2     [H][ld] float32: warm start in (prm->warm_start; the
 *                 extrapolation restarts there, ubar = u), result out.
 *   state         seg_state_bytes(H, ld, capacity, SEG_MODE_COMPACT,
 *                 SEG_STORE_F32) bytes (capacity >= n_active).
 *   stats         out double[8] (device): as seg_solve, [2] = last ||dp||.
 * Errors: INVALID_ARG, ALIGN, WORKSPACE, CUDA on the host; CAPACITY in the
 * status word. */
seg_status seg_solve_pd(const float* f, int H, int W, int ld,
                        const uint32_t* act, const uint32_t* fg, const int32_t* wstart,
                        const int32_t* counts, const seg_pd_params* prm,
                        float* u, float* p1, float* p2,
                        void* state, size_t state_bytes, double* stats,
                        void* ws, size_t ws_bytes, void* stream);

/* One image of a batch for seg_solve_batch (host struct holding device
 * pointers): the fitting term and the domain of seg_build_domain for it,
 * its u, v, p1, p2 [H][ld] (warm start in, result out) and its lambda. */
typedef struct seg_image {
    const float* f;
    int H, W, ld;
    const uint32_t* act;
    const uint32_t* fg;
    const int32_t* wstart;
    const int32_t* counts;
    float* u;
    float* v;
    float* p1;
    float* p2;
    double lambda;
} seg_image;

/* Workspace bytes for seg_solve_batch (independent of the image sizes). */
size_t seg_batch_workspace_bytes(int n_images, int64_t max_pixels);

/* The iteration of seg_solve for up to 128 images at once, in one persistent
 * launch (Section 3 per image; the images are independent problems whose RD
 * pixels are concatenated).  Compact mode only; theta, tau, the iteration
 * count, n_inner, storage and the stopping test (Euclidean norms over the
 * whole batch) are shared, lambda is per image.  state: seg_state_bytes(0, 0,
 * capacity, SEG_MODE_COMPACT, storage) with capacity >= the total RD pixels
 * (else SEG_ERR_CAPACITY in the status word).  stats as for seg_solve
 * (stats[3] = total RD pixels).  With tol <= 0 and n_inner = 1 the launch
 * may solve the images in consecutive waves of whole images (each small
 * enough for shared memory); the iterates are the same (the images are
 * independent) and stats[1..2] are summed over the waves.
 * Errors: INVALID_ARG, ALIGN, WORKSPACE, CUDA. */
seg_status seg_solve_batch(const seg_image* images, int n_images, const seg_params* prm,
                           void* state, size_t state_bytes, double* stats,
                           void* ws, size_t ws_bytes, void* stream);

/* Bytes of the checkpoints of seg_solve_diff: (p1, p2, v) as float32 for
 * ceil(iters / ckpt_every) iterates, for a state of `capacity` RD pixels. */
size_t seg_ckpt_bytes(int64_t capacity, int iters, int ckpt_every);

/* Scratch bytes of seg_backward (adjoint fields and two segment buffers of
 * ckpt_every + 1 recomputed iterates each: one segment is recomputed while
 * the reverse steps walk back through the next later one). */
size_t seg_backward_scratch_bytes(int64_t capacity, int ckpt_every);

/* Differentiable forward (not in the paper): seg_solve in compact mode with
 * float32 storage, n_inner = 1, cold start and a fixed number of iterations
 * (tol <= 0), which also writes the iterate (p1, p2, v) every ckpt_every
 * iterations into `ckpt` (seg_ckpt_bytes).  Arguments otherwise as
 * seg_solve.  Errors: INVALID_ARG, ALIGN, CAPACITY, WORKSPACE, CUDA. */
seg_status seg_solve_diff(const float* f, int H, int W, int ld,
                          const uint32_t* act, const uint32_t* fg, const int32_t* wstart,
                          const int32_t* tiles, const int32_t* counts,
                          const seg_params* prm,
                          float* u, float* v, float* p1, float* p2,
                          void* state, size_t state_bytes,
                          int ckpt_every, void* ckpt, size_t ckpt_bytes, double* stats,
                          void* ws, size_t ws_bytes, void* stream);

/* seg_solve_diff for a batch of images solved together (not in the paper):
 * the images of seg_solve_batch in one persistent launch, compact mode,
 * float32 storage, n_inner = 1, cold start, a fixed number of iterations
 * (tol <= 0), writing the batch's iterate (p1, p2, v) every ckpt_every
 * iterations into `ckpt` (seg_ckpt_bytes for the batch's capacity).  The
 * images' iterates are those of seg_solve_diff on each image alone.  state
 * as for seg_solve_batch; ws: seg_batch_workspace_bytes bytes.
 * Errors: INVALID_ARG, ALIGN, CAPACITY, WORKSPACE, CUDA. */
seg_status seg_solve_diff_batch(const seg_image* images, int n_images, const seg_params* prm,
                                void* state, size_t state_bytes, int ckpt_every, void* ckpt,
                                size_t ckpt_bytes, double* stats, void* ws, size_t ws_bytes,
                                void* stream);

/* Per-image arguments of seg_backward_batch (host struct holding device
 * pointers), as the arguments of the same names of seg_backward. */
typedef struct seg_adj_image {
    const float* grad_u;   /* dL/du^K, [H][ld] */
    const float* grad_v;   /* NULL or dL/dv^K, [H][ld] */
    const float* z;        /* NULL, or the image z of Eq. CV (then c is required) */
    const double* c;       /* with z: the c1, c2 used, device double[2] */
    float* grad_f;         /* out: dL/df, [H][ld], 0 outside RD */
    double* grad_out;      /* out: device double[3], dL/dlambda, dL/dc1, dL/dc2 */
} seg_adj_image;

/* Reverse mode of seg_solve_diff_batch (not in the paper): the adjoint of
 * every image of the batch in one persistent reverse sweep (the segments
 * are recomputed from the checkpoints as in seg_backward), with the
 * per-image gradients of seg_backward.  images, state, ckpt and prm must be
 * those of the seg_solve_diff_batch call, unmodified; adj holds n_images
 * entries.  scratch: seg_backward_scratch_bytes for the batch's capacity;
 * ws: seg_batch_workspace_bytes bytes (the compact bases are recomputed from
 * the images' domain counts).  The per-image sums for lambda, c1 and c2 are
 * reduced in the same fixed order as seg_backward's, so each image's
 * gradients equal those of seg_backward on that image alone.
 * Errors: INVALID_ARG, ALIGN, CAPACITY, WORKSPACE, CUDA. */
seg_status seg_backward_batch(const seg_image* images, const seg_adj_image* adj, int n_images,
                              const seg_params* prm, const void* state, size_t state_bytes,
                              const void* ckpt, size_t ckpt_bytes, int ckpt_every, void* scratch,
                              size_t scratch_bytes, void* ws, size_t ws_bytes, void* stream);

/* Reverse mode of the unrolled iteration run by seg_solve_diff (not in the
 * paper): given dL/du^K (grad_u, [H][ld]) and optionally dL/dv^K (grad_v),
 * returns dL/df (grad_f, [H][ld], 0 outside RD) and grad_out = {dL/dlambda,
 * dL/dc1, dL/dc2} (device double[3]; the c terms need z and c = {c1, c2},
 * device double[2], else they are 0).  The partition is held fixed; the
 * clip's derivative is 1 strictly inside (0, 1).  The forward iterates are
 * recomputed segment by segment from the checkpoints (state and ckpt must be
 * those of the seg_solve_diff call, unmodified).  scratch:
 * seg_backward_scratch_bytes bytes, caller-owned.  Errors: INVALID_ARG,
 * ALIGN, CAPACITY, WORKSPACE, CUDA. */
seg_status seg_backward(const float* f, int H, int W, int ld,
                        const uint32_t* act, const uint32_t* fg, const int32_t* wstart,
                        const int32_t* counts, const seg_params* prm,
                        const void* state, size_t state_bytes,
                        const void* ckpt, size_t ckpt_bytes, int ckpt_every,
                        const float* grad_u, const float* grad_v, const float* z, const double* c,
                        float* grad_f, double* grad_out, void* scratch, size_t scratch_bytes,
                        void* ws, size_t ws_bytes, void* stream);

/* Energies of an iterate (FP64 reductions over the image):
 *   out[0] TV(u) (isotropic, forward differences), out[1] E_CR(u) = TV(u) +
 *   lambda sum f u (Eq. CR), out[2] E_CR(v), out[3] E_DF(u, v) (Eq. DF with
 *   psi(v) = 0 on [0,1]), out[4] the dual bound D(p) = sum min(0, lambda f +
 *   div p) (valid when |p| <= 1), out[5] the duality gap E_CR(v) - D(p).
 *   out: device double[6].  Errors: INVALID_ARG, ALIGN, WORKSPACE, CUDA. */
seg_status seg_energy(const float* f, int H, int W, int ld,
                      const float* u, const float* v, const float* p1, const float* p2,
                      double lambda, double theta, double* out,
                      void* ws, size_t ws_bytes, void* stream);

/* seg_energy without a workspace, for callers that cannot allocate device
 * memory (code running under stream capture, hosts that forbid further device
 * allocation, loops where an allocation's implicit synchronisation is not
 * acceptable).  The paper has no counterpart: this is a library convenience.
 * Same inputs and output as seg_energy (out: device double[6]); the per-block
 * partial sums live in a fixed 196,672-byte device array inside the library,
 * present on every GPU that loads it until the process exits.  Images above
 * 33,554,432 pixels are rejected with SEG_ERR_CAPACITY.  The first call on a
 * device looks up that array's address (cudaGetSymbolAddress) and caches it,
 * so make the first call before any stream capture.  The cached address
 * belongs to the device's current primary context: after cudaDeviceReset
 * (or anything else that destroys that context) the library is loaded anew
 * at another address and the cached one is stale, so do not call this entry
 * point in a process after resetting the device.  No slot needs clearing
 * (each call writes every slot it reads); all calls share the array, so calls
 * that overlap on the GPU race and may return wrong sums.  It never calls
 * cudaMalloc or cudaFree.  Errors: INVALID_ARG, ALIGN, CAPACITY, CUDA. */
seg_status seg_energy_noalloc(const float* f, int H, int W, int ld,
                              const float* u, const float* v, const float* p1, const float* p2,
                              double lambda, double theta, double* out, void* stream);

/* Error measures of Section 4: out[0] = E1 = N(GT & O*) / N(GT | O*) with
 * GT = {u_gt > eps}, O* = {u_star > eps} (1 when both are empty), out[1] =
 * E2 = sum (u_star - u_gt)^2.  out: device double[2]. */
seg_status seg_errors(const float* u_star, const float* u_gt, int H, int W, int ld,
                      double eps, double* out, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SEG_H */
