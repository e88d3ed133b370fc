// solve.cu -- the restricted dual iteration of Sections 2.1 and 3.
//
// One outer iteration, on RD only (p = 0 and u = v = H(-f) elsewhere):
//   w  = div p - v / theta
//   g  = grad w
//   p' = (p + tau g) / (1 + tau |g|)              fixed-point step for rho
//   u' = v - theta div p'                          u-step
//   v' = min(max(u' - theta lambda f, 0), 1)       v-step
// with Chambolle's discrete operators (forward differences, zero on the last
// row / column; div = -grad^T).  The stopping test of Section 4 compares
// max(||u'-u||, ||v'-v||) with tol every check_every iterations.
//
// Two implementations:
//  * dense   : state in [H][ld] float32 ping-pong images.  One warp walks down
//              a strip of 32 columns with the previous row in registers and
//              its horizontal neighbours from shuffles; one pass per
//              iteration, no shared memory.  RD is given by the RD bit plane
//              (every pixel when RD is the whole image: the original method).
//  * compact : state stored only for RD pixels, in the tile-major compact order
//              of the domain (float32, bf16 or fp16 storage, float32
//              arithmetic).  A neighbour table, built once per solve, holds
//              for each RD pixel the compact index of the six pixels the
//              fixed-point step reads (or a code for a fixed / outside pixel).
//              Each iteration is two fully parallel passes over the RD pixels:
//              the dual step (p') and the primal step (u', v').
// Per-block FP64 partial sums of |du|^2, |dv|^2 feed a fixed-order reduction,
// so the stopping test is deterministic.  Once it fires, a device flag makes
// every later launch of the solve return immediately.
#include <algorithm>
#include <cmath>

#include "seg_internal.cuh"

namespace seg {

struct IterParams {
    float theta, inv_theta, tau, theta_lambda;
    int H, W, ld, nw, ntx, th;
    int check, write_u;
    uint32_t seed;   // per-launch seed of the stochastic rounding of 16-bit stores
};

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

// p' = (p + tau g) / (1 + tau |g|); |g| through the hardware reciprocal square
// root and the quotient through the fast divide (a few ulp; the iteration is
// checked against the FP64 oracle to 1e-4).
__device__ __forceinline__ void chambolle_update(float p1, float p2, float g1, float g2, float tau,
                                                 float& q1, float& q2) {
    const float s = fmaf(g1, g1, g2 * g2);
    const float nrm = s > 0.f ? s * rsqrtf(s) : 0.f;
    const float r = __fdividef(1.0f, fmaf(tau, nrm, 1.0f));
    q1 = fmaf(tau, g1, p1) * r;
    q2 = fmaf(tau, g2, p2) * r;
}

// ============================================================ dense stencil

// One warp walks down a strip of 32 image columns (lanes) and a band of
// kDenseBand output rows, keeping the previous row of p1, p2, v, w and p1' in
// registers.  Per step i it has row i (loaded one step ahead), forms
// w(i) = div p - v/theta, then p'(i-1) from w(i-1), w(i) and w(i-1) one
// column right, then u', v' of row i-1 from p'(i-1), p1'(i-2) and p2'(i-1)
// one column left.  Lane 0 lacks its left neighbour and lane 31 its right
// one, so p' is exact on lanes 1..30 and u', v' on lanes 2..30: strips
// overlap by 3 columns and each warp writes kStripOut = 29 columns.
constexpr int kStripOut = 29;
constexpr int kDenseBand = 32;
constexpr int kDenseWarps = 4;

struct RowVals {
    float p1, p2, v, f, u;
    uint32_t act;
};

template <bool PONLY>
__device__ __forceinline__ void load_row(RowVals& r, bool valid, int off, int moff, int bit,
                                         bool need_u, bool full, const uint32_t* __restrict__ act,
                                         const float* __restrict__ f, const float* __restrict__ p1i,
                                         const float* __restrict__ p2i, const float* __restrict__ vi,
                                         const float* u) {
    if (valid) {
        r.p1 = __ldg(p1i + off);
        r.p2 = __ldg(p2i + off);
        r.v = __ldg(vi + off);
        r.f = PONLY ? 0.f : __ldg(f + off);
        r.u = need_u ? u[off] : 0.f;
        r.act = full ? 1u : ((__ldg(act + moff) >> bit) & 1u);
    } else {
        r.p1 = 0.f; r.p2 = 0.f; r.v = 0.f; r.f = 0.f; r.u = 0.f; r.act = 0u;
    }
}

// PONLY: fixed-point sweep for p only (extra inner sweeps), v unchanged.
template <bool PONLY>
__global__ void __launch_bounds__(kDenseWarps * 32)
k_step_dense(IterParams P, int n_strips, int n_tasks, const int32_t* __restrict__ counts,
             const uint32_t* __restrict__ act, const float* __restrict__ f,
             const float* __restrict__ p1i, const float* __restrict__ p2i, const float* __restrict__ vi,
             float* __restrict__ p1o, float* __restrict__ p2o, float* __restrict__ vo,
             float* __restrict__ u, double* __restrict__ partials, WsHeader* h) {
    if (*(volatile int*)&h->done) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool full = counts[1] == P.H * P.W;     // every pixel in RD: no mask loads
    const bool need_u = !PONLY && P.check;
    for (int task = blockIdx.x * kDenseWarps + warp; task < n_tasks;
         task += gridDim.x * kDenseWarps) {
        const int strip = task % n_strips, band = task / n_strips;
        const int j = strip * kStripOut - 2 + lane;
        const bool jin = j >= 0 && j < P.W;
        const bool notlastc = j < P.W - 1;
        const bool hasleft = j > 0;
        const bool outl = lane >= 2 && lane <= 30 && jin;
        const int rb = band * kDenseBand;
        const int re = min(rb + kDenseBand, P.H);
        const int jc = jin ? j : 0;
        const int bit = jc & 31;
        int off = (rb - 2) * P.ld + jc;          // H * ld < 2^31 (checked by the caller)
        int moff = (rb - 2) * P.nw + (jc >> 5);
        float p1m = 0.f, p2m = 0.f, vm = 0.f, fm = 0.f, um = 0.f, wm = 0.f, q1m = 0.f;
        uint32_t am = 0u;
        float du2 = 0.f, dv2 = 0.f;
        RowVals cur, nxt;
        int i = rb - 2;
        load_row<PONLY>(cur, jin && i >= 0 && i < P.H, off, moff, bit, need_u, full, act, f, p1i,
                        p2i, vi, u);
        for (; i <= re; ++i) {
            const int offn = off + P.ld, moffn = moff + P.nw;
            load_row<PONLY>(nxt, jin && i + 1 >= 0 && i + 1 < P.H && i + 1 <= re, offn, moffn, bit,
                            need_u, full, act, f, p1i, p2i, vi, u);
            // w at row i
            const float a2l = __shfl_up_sync(FULL, cur.p2, 1);
            const float d1 = (i < P.H - 1 ? cur.p1 : 0.f) - p1m;
            const float d2 = (notlastc ? cur.p2 : 0.f) - (hasleft ? a2l : 0.f);
            const float w = (d1 + d2) - cur.v * P.inv_theta;
            // p' at row i-1
            const int im = i - 1;
            const float wr = __shfl_down_sync(FULL, wm, 1);
            float q1 = 0.f, q2 = 0.f;
            if (am) {
                const float g1 = im < P.H - 1 ? w - wm : 0.f;
                const float g2 = notlastc ? wr - wm : 0.f;
                chambolle_update(p1m, p2m, g1, g2, P.tau, q1, q2);
            }
            const float q2l = __shfl_up_sync(FULL, q2, 1);
            // u', v' at row i-1
            if (am && outl && im >= rb) {
                const int o = off - P.ld;
                p1o[o] = q1;
                p2o[o] = q2;
                if (!PONLY) {
                    const float div = ((im < P.H - 1 ? q1 : 0.f) - q1m) +
                                      ((notlastc ? q2 : 0.f) - (hasleft ? q2l : 0.f));
                    const float un = fmaf(-P.theta, div, vm);
                    const float vn = clamp01(fmaf(-P.theta_lambda, fm, un));
                    vo[o] = vn;
                    if (P.check) {
                        const float da = un - um, db = vn - vm;
                        du2 = fmaf(da, da, du2);
                        dv2 = fmaf(db, db, dv2);
                    }
                    if (P.write_u) u[o] = un;
                }
            }
            p1m = cur.p1; p2m = cur.p2; vm = cur.v; fm = cur.f; um = cur.u; am = cur.act;
            wm = w; q1m = q1;
            cur = nxt;
            off = offn;
            moff = moffn;
        }
        if (!PONLY && P.check) {
            double a = du2, b = dv2;
            for (int d = 16; d > 0; d >>= 1) {
                a += __shfl_down_sync(FULL, a, d);
                b += __shfl_down_sync(FULL, b, d);
            }
            if (lane == 0) { partials[2 * task] = a; partials[2 * task + 1] = b; }
        }
    }
}

// Cold or warm start of the dense state: both ping-pong copies get the fixed
// values outside RD; RD pixels get p = 0, u0 = H(-f), v0 = clip(u0 -
// theta lambda f) (cold) or the caller's iterate (warm).
__global__ void k_init_dense(IterParams P, const uint32_t* __restrict__ act,
                             const uint32_t* __restrict__ fgm, const float* __restrict__ f,
                             int warm, const float* __restrict__ wp1, const float* __restrict__ wp2,
                             const float* __restrict__ wv, float* u, float* st) {
    int64_t plane = (int64_t)P.H * P.ld;
    float *P1a = st, *P1b = st + plane, *P2a = st + 2 * plane, *P2b = st + 3 * plane,
          *Va = st + 4 * plane, *Vb = st + 5 * plane;
    int64_t n = (int64_t)P.H * P.W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = x / P.W, j = x - i * P.W;
        int64_t o = i * P.ld + j, wo = i * P.nw + (j >> 5);
        bool a = (act[wo] >> (j & 31)) & 1u;
        float hh = ((fgm[wo] >> (j & 31)) & 1u) ? 1.f : 0.f;
        float p1 = 0.f, p2 = 0.f, v = hh, uu = hh;
        if (a) {
            if (warm) { p1 = wp1[o]; p2 = wp2[o]; v = wv[o]; uu = u[o]; }
            else v = clamp01(fmaf(-P.theta_lambda, f[o], hh));
        }
        P1a[o] = p1; P1b[o] = p1; P2a[o] = p2; P2b[o] = p2; Va[o] = v; Vb[o] = v;
        u[o] = uu;
    }
}

__global__ void k_final_dense(IterParams P, const WsHeader* __restrict__ h, int iters, int n_inner,
                              const float* __restrict__ st, float* v, float* p1, float* p2) {
    int64_t plane = (int64_t)P.H * P.ld;
    int l = h->done ? h->iters_done : iters;
    int vb = l & 1, pb = (int)(((long long)l * n_inner) & 1);
    const float* P1 = st + pb * plane;
    const float* P2 = st + (2 + pb) * plane;
    const float* V = st + (4 + vb) * plane;
    int64_t n = (int64_t)P.H * P.W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = x / P.W, j = x - i * P.W;
        int64_t o = i * P.ld + j;
        p1[o] = P1[o]; p2[o] = P2[o]; v[o] = V[o];
    }
}

// ========================================================== compact stencil

constexpr int kCompactThreads = 256;

// neighbour slots of the table and the codes for pixels that are not in RD
enum { NB_UP = 0, NB_LEFT = 1, NB_DOWN = 2, NB_RIGHT = 3, NB_DOWNLEFT = 4, NB_UPRIGHT = 5, NB_COUNT = 6 };
constexpr int kNbBg = -1;    // fixed background: p = 0, v = 0
constexpr int kNbFg = -2;    // fixed foreground: p = 0, v = 1
constexpr int kNbOut = -3;   // outside the image (the gradient there is 0)

struct CompactState {
    void *p1[2], *p2[2], *v;
    float* f;
    float* u;
    int32_t* nb;     // [NB_COUNT][cap]
    int64_t cap;
};

// Compact index of pixel (i, j) when it is in RD, else its code.
__device__ __forceinline__ int nb_code(const IterParams& P, const uint32_t* __restrict__ act,
                                       const uint32_t* __restrict__ fgm,
                                       const int32_t* __restrict__ wstart, int i, int j) {
    if (i < 0 || i >= P.H || j < 0 || j >= P.W) return kNbOut;
    const int64_t o = (int64_t)i * P.nw + (j >> 5);
    const int b = j & 31;
    const uint32_t a = act[o];
    if ((a >> b) & 1u) return wstart[o] + __popc(a & lanemask_lt(b));
    return ((fgm[o] >> b) & 1u) ? kNbFg : kNbBg;
}

// One warp per mask word (lane b is pixel (i, 32 wx + b)): gathers f and the
// start iterate of every RD pixel into compact order and fills its row of the
// neighbour table.
template <typename T>
__global__ void k_compact_gather(IterParams P, const uint32_t* __restrict__ act,
                                 const uint32_t* __restrict__ fgm, const int32_t* __restrict__ wstart,
                                 const int32_t* __restrict__ counts, const float* __restrict__ f,
                                 int warm, const float* __restrict__ u, const float* __restrict__ v,
                                 const float* __restrict__ p1, const float* __restrict__ p2,
                                 CompactState S, WsHeader* h) {
    if (counts[1] > S.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            record_status(h, SEG_ERR_CAPACITY);
            h->done = 1;
            h->iters_done = 0;
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const int64_t word = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t nwords = (int64_t)P.H * P.ntx;
    if (word >= nwords) return;
    const int i = (int)(word / P.ntx);
    const int wx = (int)(word - (int64_t)i * P.ntx);
    const int j = wx * 32 + lane;
    const int64_t wo = (int64_t)i * P.nw + wx;
    const uint32_t a = act[wo];
    if (!((a >> lane) & 1u)) return;
    const int64_t idx = wstart[wo] + __popc(a & lanemask_lt(lane));
    const int64_t o = (int64_t)i * P.ld + j;
    const float fv = f[o];
    const float hh = ((fgm[wo] >> lane) & 1u) ? 1.f : 0.f;
    S.f[idx] = fv;
    T* P1 = static_cast<T*>(S.p1[0]);
    T* P2 = static_cast<T*>(S.p2[0]);
    T* V = static_cast<T*>(S.v);
    if (warm) {
        // p1 on the last row and p2 on the last column never enter div p;
        // they are held at 0 (where a cold start keeps them)
        Store<T>::st(P1, idx, i < P.H - 1 ? p1[o] : 0.f);
        Store<T>::st(P2, idx, j < P.W - 1 ? p2[o] : 0.f);
        Store<T>::st(V, idx, v[o]);
        S.u[idx] = u[o];
    } else {
        Store<T>::st(P1, idx, 0.f);
        Store<T>::st(P2, idx, 0.f);
        Store<T>::st(V, idx, clamp01(fmaf(-P.theta_lambda, fv, hh)));
        S.u[idx] = hh;
    }
    int32_t* nb = S.nb;
    const int64_t cap = S.cap;
    nb[NB_UP * cap + idx] = nb_code(P, act, fgm, wstart, i - 1, j);
    nb[NB_LEFT * cap + idx] = nb_code(P, act, fgm, wstart, i, j - 1);
    nb[NB_DOWN * cap + idx] = nb_code(P, act, fgm, wstart, i + 1, j);
    nb[NB_RIGHT * cap + idx] = nb_code(P, act, fgm, wstart, i, j + 1);
    nb[NB_DOWNLEFT * cap + idx] = nb_code(P, act, fgm, wstart, i + 1, j - 1);
    nb[NB_UPRIGHT * cap + idx] = nb_code(P, act, fgm, wstart, i - 1, j + 1);
}

template <typename T>
__device__ __forceinline__ float nb_ld(const T* __restrict__ X, int n) {
    return n >= 0 ? Store<T>::ld(X, n) : 0.f;
}
__device__ __forceinline__ float nb_vfix(int n) { return n == kNbFg ? 1.f : 0.f; }

// Dual step on every RD pixel a (grid-stride):
//   w(y) = (p1(y) - p1(y-e1)) + (p2(y) - p2(y-e2)) - v(y)/theta at y = x,
//   x+e1, x+e2; g = (w(x+e1) - w(x), w(x+e2) - w(x)) (0 across the image
//   border); p'(x) = (p(x) + tau g) / (1 + tau |g|).
// p1 vanishes on the last row and p2 on the last column (their gradient
// component is 0 there and they start at 0), so no border masks are needed
// in w.
template <typename T>
__global__ void __launch_bounds__(kCompactThreads)
k_dual_compact(IterParams P, const int32_t* __restrict__ counts, const int32_t* __restrict__ nb,
               int64_t cap, const T* __restrict__ P1i, const T* __restrict__ P2i,
               const T* __restrict__ Vi, T* __restrict__ P1o, T* __restrict__ P2o, WsHeader* h) {
    if (*(volatile int*)&h->done) return;
    const int n = counts[1];
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const int n_up = __ldg(nb + NB_UP * cap + a);
        const int n_left = __ldg(nb + NB_LEFT * cap + a);
        const int n_down = __ldg(nb + NB_DOWN * cap + a);
        const int n_right = __ldg(nb + NB_RIGHT * cap + a);
        const int n_dl = __ldg(nb + NB_DOWNLEFT * cap + a);
        const int n_ur = __ldg(nb + NB_UPRIGHT * cap + a);
        const float p1 = Store<T>::ld(P1i, a), p2 = Store<T>::ld(P2i, a), v = Store<T>::ld(Vi, a);
        const float p1_up = nb_ld(P1i, n_up);
        const float p2_left = nb_ld(P2i, n_left);
        const float p1_d = nb_ld(P1i, n_down), p2_d = nb_ld(P2i, n_down);
        const float v_d = n_down >= 0 ? Store<T>::ld(Vi, n_down) : nb_vfix(n_down);
        const float p1_r = nb_ld(P1i, n_right), p2_r = nb_ld(P2i, n_right);
        const float v_r = n_right >= 0 ? Store<T>::ld(Vi, n_right) : nb_vfix(n_right);
        const float p2_dl = nb_ld(P2i, n_dl);
        const float p1_ur = nb_ld(P1i, n_ur);
        const float w0 = (p1 - p1_up) + (p2 - p2_left) - v * P.inv_theta;
        const float g1 = n_down != kNbOut ? ((p1_d - p1) + (p2_d - p2_dl) - v_d * P.inv_theta) - w0 : 0.f;
        const float g2 = n_right != kNbOut ? ((p1_r - p1_ur) + (p2_r - p2) - v_r * P.inv_theta) - w0 : 0.f;
        float q1, q2;
        chambolle_update(p1, p2, g1, g2, P.tau, q1, q2);
        const uint32_t rnd = mix32((uint32_t)a * 3u + P.seed);
        Store<T>::st_sr(P1o, a, q1, rnd);
        Store<T>::st_sr(P2o, a, q2, mix32(rnd ^ 0x9e3779b9u));
    }
}

// Primal step on every RD pixel: u' = v - theta div p', v' = clip(u' - theta
// lambda f) (v updated in place), with per-block FP64 partials of |du|^2 and
// |dv|^2 for the stopping test.
template <typename T>
__global__ void __launch_bounds__(kCompactThreads)
k_primal_compact(IterParams P, const int32_t* __restrict__ counts, const int32_t* __restrict__ nb,
                 int64_t cap, const T* __restrict__ P1n, const T* __restrict__ P2n, T* __restrict__ V,
                 const float* __restrict__ F, float* __restrict__ U, double* __restrict__ partials,
                 WsHeader* h) {
    __shared__ double s_red[2 * (kCompactThreads / 32)];
    if (*(volatile int*)&h->done) return;
    const int n = counts[1];
    float du2 = 0.f, dv2 = 0.f;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const int n_up = __ldg(nb + NB_UP * cap + a);
        const int n_left = __ldg(nb + NB_LEFT * cap + a);
        const float q1 = Store<T>::ld(P1n, a), q2 = Store<T>::ld(P2n, a);
        const float q1u = nb_ld(P1n, n_up), q2l = nb_ld(P2n, n_left);
        const float div = (q1 - q1u) + (q2 - q2l);
        const float vv = Store<T>::ld_rw(V, a);
        const float un = fmaf(-P.theta, div, vv);
        const float vn = clamp01(fmaf(-P.theta_lambda, __ldg(F + a), un));
        Store<T>::st_sr(V, a, vn, mix32((uint32_t)a * 5u + P.seed));
        if (P.check) {
            const float da = un - U[a], db = vn - vv;
            du2 = fmaf(da, da, du2);
            dv2 = fmaf(db, db, dv2);
        }
        if (P.write_u) U[a] = un;
    }
    if (P.check) {
        double a = du2, b = dv2;
        for (int d = 16; d > 0; d >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, d);
            b += __shfl_down_sync(0xffffffffu, b, d);
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) { s_red[2 * wid] = a; s_red[2 * wid + 1] = b; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double x = 0.0, y = 0.0;
            for (int w = 0; w < kCompactThreads / 32; ++w) { x += s_red[2 * w]; y += s_red[2 * w + 1]; }
            partials[2 * blockIdx.x] = x;
            partials[2 * blockIdx.x + 1] = y;
        }
    }
}

// Dense u, v, p1, p2 of the final iterate: compact values on RD, the fixed
// values elsewhere.
template <typename T>
__global__ void k_compact_scatter(IterParams P, const uint32_t* __restrict__ act,
                                  const uint32_t* __restrict__ fgm, const int32_t* __restrict__ wstart,
                                  const int32_t* __restrict__ counts, int iters, int n_inner,
                                  CompactState S, const WsHeader* __restrict__ h, float* u, float* v,
                                  float* p1, float* p2) {
    const int lane = threadIdx.x & 31;
    const int64_t word = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t nwords = (int64_t)P.H * P.ntx;
    if (word >= nwords) return;
    const int64_t i = word / P.ntx;
    const int wx = (int)(word - i * P.ntx);
    const int j = wx * 32 + lane;
    if (j >= P.W) return;
    const int64_t wo = i * P.nw + wx;
    const int64_t o = i * P.ld + j;
    const uint32_t a = act[wo];
    const float hh = ((fgm[wo] >> lane) & 1u) ? 1.f : 0.f;
    const bool ok = counts[1] <= S.cap;
    if (ok && ((a >> lane) & 1u)) {
        const int l = h->done ? h->iters_done : iters;
        const int pb = (int)(((long long)l * n_inner) & 1);
        const int64_t idx = wstart[wo] + __popc(a & lanemask_lt(lane));
        u[o] = S.u[idx];
        v[o] = Store<T>::ld_rw(static_cast<const T*>(S.v), idx);
        p1[o] = Store<T>::ld_rw(static_cast<const T*>(S.p1[pb]), idx);
        p2[o] = Store<T>::ld_rw(static_cast<const T*>(S.p2[pb]), idx);
    } else {
        u[o] = hh; v[o] = hh; p1[o] = 0.f; p2[o] = 0.f;
    }
}

// =================================================== stopping test, stats

__global__ void k_solve_begin(WsHeader* h) {
    h->done = 0;
    h->iters_done = 0;
    h->last_check = 0;
    h->du = 0.0;
    h->dv = 0.0;
}

// Section 4 stopping test after iteration l: sums the n partial pairs in a
// fixed order (thread t owns pairs t, t+1024, ...; then a fixed tree),
// records the norms and raises the done flag when both are <= tol.
constexpr int kCheckThreads = 1024;
__global__ void __launch_bounds__(kCheckThreads)
k_check(const double* __restrict__ partials, int n, int l, double tol, WsHeader* h) {
    __shared__ double sa[kCheckThreads], sb[kCheckThreads];
    if (*(volatile int*)&h->done) return;
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < n; k += kCheckThreads) { a += partials[2 * k]; b += partials[2 * k + 1]; }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = kCheckThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) { sa[threadIdx.x] += sa[threadIdx.x + w]; sb[threadIdx.x] += sb[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double du = sqrt(sa[0]), dv = sqrt(sb[0]);
        h->du = du;
        h->dv = dv;
        h->last_check = l;
        if (tol > 0.0 && fmax(du, dv) <= tol) {
            h->iters_done = l;
            h->done = 1;
        }
    }
}

__global__ void k_solve_end(const WsHeader* __restrict__ h, const int32_t* __restrict__ counts,
                            int iters, double* stats) {
    stats[0] = h->done ? h->iters_done : iters;
    stats[1] = h->du;
    stats[2] = h->dv;
    stats[3] = counts[1];
    stats[4] = counts[0];
    stats[5] = h->last_check;
    stats[6] = 0.0;
    stats[7] = 0.0;
}

// ================================================================== host

static uint32_t mix32_host(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352du;
    x ^= x >> 15; x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <typename K>
static int grid_for(K kernel, int threads, int64_t max_blocks) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (per_sm <= 0) per_sm = 1;
    int64_t g = (int64_t)per_sm * sm_count();
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, max_blocks));
}

struct CompactLayout {
    size_t off[8];
    int64_t cap;
};

// compact state: p1[2], p2[2], v (storage type), f, u (float32), neighbour
// table (int32 x 6), each array 256-byte aligned
constexpr int kCompactArrays = 8;
static CompactLayout compact_layout(size_t state_bytes, int storage) {
    CompactLayout C{};
    size_t sz = storage_size(storage);
    size_t per = 5 * sz + 8 + 4 * NB_COUNT;
    C.cap = state_bytes > kCompactArrays * 256 ? (int64_t)((state_bytes - kCompactArrays * 256) / per) : 0;
    size_t o = 0;
    for (int a = 0; a < 5; ++a) { C.off[a] = o; o = align_up(o + sz * (size_t)C.cap, 256); }
    C.off[5] = o; o = align_up(o + 4 * (size_t)C.cap, 256);   // f
    C.off[6] = o; o = align_up(o + 4 * (size_t)C.cap, 256);   // u
    C.off[7] = o;                                             // neighbour table
    return C;
}

static seg_status run_dense(const IterParams& P0, const seg_params* prm, const int32_t* counts,
                            const uint32_t* act, const float* f, float* u, float* st,
                            double* partials, WsHeader* h, cudaStream_t s) {
    int64_t plane = (int64_t)P0.H * P0.ld;
    float* P1[2] = {st, st + plane};
    float* P2[2] = {st + 2 * plane, st + 3 * plane};
    float* V[2] = {st + 4 * plane, st + 5 * plane};
    auto kfull = k_step_dense<false>;
    auto kp = k_step_dense<true>;
    const int n_strips = (P0.W + kStripOut - 1) / kStripOut;
    const int n_tasks = n_strips * ((P0.H + kDenseBand - 1) / kDenseBand);
    const int64_t max_blocks = (n_tasks + kDenseWarps - 1) / kDenseWarps;
    const int grid = grid_for(kfull, kDenseWarps * 32, max_blocks);
    const int gridp = grid_for(kp, kDenseWarps * 32, max_blocks);
    int pb = 0, vb = 0;
    const int C = std::max(1, prm->check_every);
    for (int it = 0; it < prm->iters; ++it) {
        const int l = it + 1;
        for (int sw = 1; sw < prm->n_inner; ++sw) {
            IterParams P = P0;
            P.check = 0; P.write_u = 0;
            kp<<<gridp, kDenseWarps * 32, 0, s>>>(P, n_strips, n_tasks, counts, act, f, P1[pb], P2[pb],
                                                  V[vb], P1[pb ^ 1], P2[pb ^ 1], V[vb], u, partials, h);
            SEG_LAUNCHED("k_step_dense<p-only>");
            pb ^= 1;
        }
        IterParams P = P0;
        P.check = (l % C == 0) || l == prm->iters;
        P.write_u = P.check || ((l + 1) % C == 0) || l == prm->iters;
        kfull<<<grid, kDenseWarps * 32, 0, s>>>(P, n_strips, n_tasks, counts, act, f, P1[pb], P2[pb],
                                                V[vb], P1[pb ^ 1], P2[pb ^ 1], V[vb ^ 1], u, partials, h);
        SEG_LAUNCHED("k_step_dense");
        pb ^= 1;
        vb ^= 1;
        if (P.check) {
            k_check<<<1, kCheckThreads, 0, s>>>(partials, n_tasks, l, prm->tol, h);
            SEG_LAUNCHED("k_check");
        }
    }
    return SEG_OK;
}

template <typename T>
static seg_status solve_compact_typed(const IterParams& P0, const seg_params* prm, const float* f,
                                      const uint32_t* act, const uint32_t* fgm, const int32_t* wstart,
                                      const int32_t* counts, float* u, float* v, float* p1, float* p2,
                                      void* state, size_t state_bytes, double* partials,
                                      int64_t max_partials, WsHeader* h, cudaStream_t s) {
    CompactLayout C = compact_layout(state_bytes, prm->storage);
    CompactState S{};
    char* base = static_cast<char*>(state);
    S.p1[0] = base + C.off[0];
    S.p1[1] = base + C.off[1];
    S.p2[0] = base + C.off[2];
    S.p2[1] = base + C.off[3];
    S.v = base + C.off[4];
    S.f = reinterpret_cast<float*>(base + C.off[5]);
    S.u = reinterpret_cast<float*>(base + C.off[6]);
    S.nb = reinterpret_cast<int32_t*>(base + C.off[7]);
    S.cap = C.cap;
    const int64_t nwords = (int64_t)P0.H * P0.ntx;
    const unsigned gblocks = (unsigned)((nwords + 7) / 8);
    k_compact_gather<T><<<gblocks, 256, 0, s>>>(P0, act, fgm, wstart, counts, f, prm->warm_start, u, v,
                                                p1, p2, S, h);
    SEG_LAUNCHED("k_compact_gather");

    T* P1[2] = {static_cast<T*>(S.p1[0]), static_cast<T*>(S.p1[1])};
    T* P2[2] = {static_cast<T*>(S.p2[0]), static_cast<T*>(S.p2[1])};
    T* V = static_cast<T*>(S.v);
    auto kd = k_dual_compact<T>;
    auto kq = k_primal_compact<T>;
    // the grids are fixed for the whole solve (the RD size stays on the
    // device); the primal grid is also the number of stopping-test partials
    const int64_t most = std::max<int64_t>(1, std::min<int64_t>(C.cap, (int64_t)P0.H * P0.W));
    const int64_t need = (most + kCompactThreads - 1) / kCompactThreads;
    const int gd = grid_for(kd, kCompactThreads, need);
    const int gq = (int)std::min<int64_t>(grid_for(kq, kCompactThreads, need), max_partials);
    int pb = 0;
    const int Cc = std::max(1, prm->check_every);
    for (int it = 0; it < prm->iters; ++it) {
        const int l = it + 1;
        for (int sw = 0; sw < prm->n_inner; ++sw) {
            IterParams P = P0;
            P.seed = mix32_host(0x51ed270bu ^ (uint32_t)(it * 131 + sw));
            kd<<<gd, kCompactThreads, 0, s>>>(P, counts, S.nb, S.cap, P1[pb], P2[pb], V, P1[pb ^ 1],
                                              P2[pb ^ 1], h);
            SEG_LAUNCHED("k_dual_compact");
            pb ^= 1;
        }
        IterParams P = P0;
        P.check = (l % Cc == 0) || l == prm->iters;
        P.write_u = P.check || ((l + 1) % Cc == 0) || l == prm->iters;
        P.seed = mix32_host(0x2545f491u ^ (uint32_t)it);
        kq<<<gq, kCompactThreads, 0, s>>>(P, counts, S.nb, S.cap, P1[pb], P2[pb], V, S.f, S.u,
                                          partials, h);
        SEG_LAUNCHED("k_primal_compact");
        if (P.check) {
            k_check<<<1, kCheckThreads, 0, s>>>(partials, gq, l, prm->tol, h);
            SEG_LAUNCHED("k_check");
        }
    }
    k_compact_scatter<T><<<gblocks, 256, 0, s>>>(P0, act, fgm, wstart, counts, prm->iters,
                                                 std::max(1, prm->n_inner), S, h, u, v, p1, p2);
    SEG_LAUNCHED("k_compact_scatter");
    return SEG_OK;
}

}  // namespace seg

using namespace seg;

extern "C" size_t seg_state_bytes(int H, int ld, int64_t capacity, int mode, int storage) {
    if (mode == SEG_MODE_DENSE) return 6 * 4 * (size_t)std::max(H, 0) * (size_t)std::max(ld, 0) + 256;
    size_t sz = storage_size(storage);
    return kCompactArrays * 256 + (size_t)std::max<int64_t>(capacity, 1) * (5 * sz + 8 + 4 * NB_COUNT);
}

extern "C" seg_status seg_solve(const float* f, int H, int W, int ld, const uint32_t* act,
                                const uint32_t* fgm, const int32_t* wstart, const int32_t* tiles,
                                const int32_t* counts, const seg_params* prm, float* u, float* v,
                                float* p1, float* p2, void* state, size_t state_bytes, double* stats,
                                void* ws, size_t ws_bytes, void* stream) {
    clear_error();
    if (!prm) return fail(SEG_ERR_INVALID_ARG, "params must be non-NULL");
    if (!f || !act || !fgm || !wstart || !tiles || !counts || !u || !v || !p1 || !p2 || !state || !stats)
        return fail(SEG_ERR_INVALID_ARG, "a required pointer is NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * ld >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d (H*ld < 2^31)", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    const int th = prm->tile_h;
    if (th != 4 && th != 8 && th != 16 && th != 32)
        return fail(SEG_ERR_INVALID_ARG, "tile_h=%d not in {4, 8, 16, 32}", th);
    if (prm->iters < 0 || prm->n_inner < 1 || prm->check_every < 1)
        return fail(SEG_ERR_INVALID_ARG, "iters >= 0, n_inner >= 1, check_every >= 1 required");
    if (!(prm->theta > 0) || !(prm->tau > 0) || !std::isfinite(prm->lambda) || std::isnan(prm->tol))
        return fail(SEG_ERR_INVALID_ARG, "theta, tau must be > 0 and lambda finite");
    if (prm->mode != SEG_MODE_DENSE && prm->mode != SEG_MODE_COMPACT)
        return fail(SEG_ERR_INVALID_ARG, "unknown mode %d", prm->mode);
    if (prm->storage < 0 || prm->storage > 2)
        return fail(SEG_ERR_INVALID_ARG, "unknown storage %d", prm->storage);
    if (prm->mode == SEG_MODE_DENSE && prm->storage != SEG_STORE_F32)
        return fail(SEG_ERR_INVALID_ARG, "16-bit storage needs SEG_MODE_COMPACT");
    if (reinterpret_cast<uintptr_t>(state) % 16)
        return fail(SEG_ERR_ALIGN, "state buffer not 16-byte aligned");
    WsLayout L = ws_layout(H, W, th);
    SEG_TRY(check_ws(ws, ws_bytes, L));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    double* partials = ws_at<double>(ws, L.partials);

    IterParams P{};
    P.theta = (float)prm->theta;
    P.inv_theta = (float)(1.0 / prm->theta);
    P.tau = (float)prm->tau;
    P.theta_lambda = (float)(prm->theta * prm->lambda);
    P.H = H; P.W = W; P.ld = ld; P.nw = ld / 32; P.ntx = (W + 31) / 32; P.th = th;

    k_solve_begin<<<1, 1, 0, s>>>(h);
    SEG_LAUNCHED("k_solve_begin");
    if (prm->mode == SEG_MODE_DENSE) {
        if (state_bytes < seg_state_bytes(H, ld, 0, SEG_MODE_DENSE, SEG_STORE_F32))
            return fail(SEG_ERR_CAPACITY, "dense state needs %zu bytes, got %zu",
                        seg_state_bytes(H, ld, 0, SEG_MODE_DENSE, SEG_STORE_F32), state_bytes);
        float* st = static_cast<float*>(state);
        int64_t n = (int64_t)H * W;
        int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
        k_init_dense<<<blocks, 256, 0, s>>>(P, act, fgm, f, prm->warm_start, p1, p2, v, u, st);
        SEG_LAUNCHED("k_init_dense");
        SEG_TRY(run_dense(P, prm, counts, act, f, u, st, partials, h, s));
        k_final_dense<<<blocks, 256, 0, s>>>(P, h, prm->iters, prm->n_inner, st, v, p1, p2);
        SEG_LAUNCHED("k_final_dense");
    } else {
        switch (prm->storage) {
            case SEG_STORE_F32:
                SEG_TRY(solve_compact_typed<float>(P, prm, f, act, fgm, wstart, counts, u, v, p1, p2,
                                                   state, state_bytes, partials, L.npartials, h, s));
                break;
            case SEG_STORE_BF16:
                SEG_TRY(solve_compact_typed<__nv_bfloat16>(P, prm, f, act, fgm, wstart, counts, u, v, p1,
                                                           p2, state, state_bytes, partials,
                                                           L.npartials, h, s));
                break;
            default:
                SEG_TRY(solve_compact_typed<__half>(P, prm, f, act, fgm, wstart, counts, u, v, p1, p2,
                                                    state, state_bytes, partials, L.npartials, h, s));
                break;
        }
    }
    k_solve_end<<<1, 1, 0, s>>>(h, counts, prm->iters, stats);
    SEG_LAUNCHED("k_solve_end");
    return SEG_OK;
}
