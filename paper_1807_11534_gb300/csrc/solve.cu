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
// Two implementations (SEG_MODE_TILED, temporal blocking, is in tiled.cu):
//  * dense   : state in [H][ld] float32 ping-pong images.  One warp walks down
//              a strip of 64 columns (two per lane) with the previous row in
//              registers and its horizontal neighbours from shuffles; one pass
//              per iteration, no shared memory.  RD is given by the RD bit
//              plane (every pixel when RD is the whole image: the original
//              method).
//  * compact : state stored only for RD pixels, in the tile-major compact order
//              of the domain (float32, bf16 or fp16 storage, float32
//              arithmetic).  A neighbour table, built once per solve, holds
//              for each RD pixel the compact index of the eight pixels the
//              iteration reads (or a code for a fixed / outside pixel).  One
//              persistent cooperative launch runs every iteration: a dual
//              phase (p') and a primal phase (u', v', and w = div p - v/theta
//              for the next dual phase) separated by grid barriers, or one
//              fused phase per iteration when each block holds at most one
//              pixel; each block keeps what it can of its pixels' state in
//              shared memory (see the persistent compact solver below).
// Per-block FP64 partial sums of |du|^2, |dv|^2 feed a fixed-order reduction,
// so the stopping test is deterministic.  Once it fires, a device flag makes
// every later launch of the solve return immediately.
#include <algorithm>
#include <climits>
#include <cmath>

#include "iterate.cuh"

namespace seg {

// ============================================================ dense stencil

// One warp walks down a strip of 64 image columns (two per lane, loaded as
// float2) and a band of band_h output rows, keeping the previous row of
// p1, p2, v, f, u, w and p1' in registers.  Per step i it has row i (loaded
// one step ahead), forms w(i) = div p - v/theta, then p'(i-1) from w(i-1),
// w(i) and w(i-1) one column right, then u', v' of row i-1 from p'(i-1),
// p1'(i-2) and p2'(i-1) one column left; neighbours across the lane pair come
// from warp shuffles.  Lane 0 lacks a left and lane 31 a right neighbour, so
// lanes 1..30 write: strips overlap by 4 columns and each warp writes
// kStripOut = 60 columns.  No shared memory, no block barriers.
constexpr int kStripOut = 60;
constexpr int kDenseWarps = 4;

struct RowVals {
    float2 p1, p2, v, f, u;
    uint32_t act;   // bit 0: column a in RD, bit 1: column b in RD
};

template <bool PONLY, bool CHECK>
__device__ __forceinline__ void load_row(RowVals& r, bool valid, int off, int moff, int bit,
                                         uint32_t inimg, bool full, const uint32_t* __restrict__ act,
                                         const float* __restrict__ f, const float* __restrict__ p1i,
                                         const float* __restrict__ p2i, const float* __restrict__ vi,
                                         const float* u) {
    const float2 z = make_float2(0.f, 0.f);
    if (valid) {
        r.p1 = __ldg(reinterpret_cast<const float2*>(p1i + off));
        r.p2 = __ldg(reinterpret_cast<const float2*>(p2i + off));
        r.v = __ldg(reinterpret_cast<const float2*>(vi + off));
        r.f = PONLY ? z : __ldg(reinterpret_cast<const float2*>(f + off));
        r.u = CHECK ? *reinterpret_cast<const float2*>(u + off) : z;
        r.act = full ? inimg : ((__ldg(act + moff) >> bit) & inimg);
    } else {
        r.p1 = z; r.p2 = z; r.v = z; r.f = z; r.u = z; r.act = 0u;
    }
}

// PONLY: fixed-point sweep for p only (extra inner sweeps), v unchanged.
// CHECK: accumulate |du|^2, |dv|^2 for the stopping test.  WRITEU: store u'.
template <bool PONLY, bool CHECK, bool WRITEU>
__global__ void __launch_bounds__(kDenseWarps * 32)
k_step_dense(IterParams P, int n_strips, int n_tasks, int band_h, const int32_t* __restrict__ counts,
             const uint32_t* __restrict__ act, const float* __restrict__ f,
             const float* __restrict__ p1i, const float* __restrict__ p2i, const float* __restrict__ vi,
             float* __restrict__ p1o, float* __restrict__ p2o, float* __restrict__ vo,
             float* __restrict__ u, double* __restrict__ partials, WsHeader* h) {
    if (*(volatile int*)&h->done) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool full = counts[1] == P.H * P.W;     // every pixel in RD: no mask loads
    for (int task = blockIdx.x * kDenseWarps + warp; task < n_tasks;
         task += gridDim.x * kDenseWarps) {
        const int strip = task % n_strips, band = task / n_strips;
        const int ja = strip * kStripOut - 2 + 2 * lane;   // columns ja, ja + 1 (ja even)
        const int jb = ja + 1;
        const bool lvalid = ja >= 0 && ja < P.ld;           // the float2 lies inside the pitch
        const uint32_t inimg = (ja >= 0 && ja < P.W ? 1u : 0u) | (jb >= 0 && jb < P.W ? 2u : 0u);
        const bool a_nl = ja < P.W - 1, b_nl = jb < P.W - 1;   // not on the last column
        const bool a_hl = ja > 0;                               // has a left neighbour
        const bool outl = lane >= 1 && lane <= 30;
        const int rb = band * band_h;
        const int re = min(rb + band_h, P.H);
        const int jc = lvalid ? ja : 0;
        const int bit = jc & 31;                                // ja even: bits ja, ja+1 in one word
        int off = (rb - 2) * P.ld + jc;          // H * ld < 2^31 (checked by the caller)
        int moff = (rb - 2) * P.nw + (jc >> 5);
        float2 p1m = make_float2(0.f, 0.f), p2m = p1m, vm = p1m, fm = p1m, um = p1m, wm = p1m, q1m = p1m;
        uint32_t am = 0u;
        float du2 = 0.f, dv2 = 0.f;
        RowVals cur, nxt;
        int i = rb - 2;
        load_row<PONLY, CHECK>(cur, lvalid && i >= 0 && i < P.H, off, moff, bit, inimg, full, act, f,
                               p1i, p2i, vi, u);
        for (; i <= re; ++i) {
            const int offn = off + P.ld, moffn = moff + P.nw;
            load_row<PONLY, CHECK>(nxt, lvalid && i + 1 >= 0 && i + 1 < P.H && i + 1 <= re, offn,
                                   moffn, bit, inimg, full, act, f, p1i, p2i, vi, u);
            const bool rl = i < P.H - 1;         // row i is not the last row
            // w at row i (columns a, b)
            const float p2_la = __shfl_up_sync(FULL, cur.p2.y, 1);
            float2 w;
            w.x = ((rl ? cur.p1.x : 0.f) - p1m.x) + ((a_nl ? cur.p2.x : 0.f) - (a_hl ? p2_la : 0.f)) -
                  cur.v.x * P.inv_theta;
            w.y = ((rl ? cur.p1.y : 0.f) - p1m.y) + ((b_nl ? cur.p2.y : 0.f) - cur.p2.x) -
                  cur.v.y * P.inv_theta;
            // p' at row i-1
            const bool rlm = i - 1 < P.H - 1;
            const float w_rb = __shfl_down_sync(FULL, wm.x, 1);
            float2 q1, q2;
            chambolle_update(p1m.x, p2m.x, rlm ? w.x - wm.x : 0.f, a_nl ? wm.y - wm.x : 0.f, P.tau,
                             q1.x, q2.x);
            chambolle_update(p1m.y, p2m.y, rlm ? w.y - wm.y : 0.f, b_nl ? w_rb - wm.y : 0.f, P.tau,
                             q1.y, q2.y);
            if (!(am & 1u)) { q1.x = 0.f; q2.x = 0.f; }
            if (!(am & 2u)) { q1.y = 0.f; q2.y = 0.f; }
            const float q2_la = __shfl_up_sync(FULL, q2.y, 1);
            // u', v' at row i-1
            if (outl && i - 1 >= rb && am) {
                const int o = off - P.ld;
                float2 un, vn;
                un.x = fmaf(-P.theta, ((rlm ? q1.x : 0.f) - q1m.x) + ((a_nl ? q2.x : 0.f) - (a_hl ? q2_la : 0.f)), vm.x);
                un.y = fmaf(-P.theta, ((rlm ? q1.y : 0.f) - q1m.y) + ((b_nl ? q2.y : 0.f) - q2.x), vm.y);
                vn.x = clamp01(fmaf(-P.theta_lambda, fm.x, un.x));
                vn.y = clamp01(fmaf(-P.theta_lambda, fm.y, un.y));
                if (am == 3u) {
                    *reinterpret_cast<float2*>(p1o + o) = q1;
                    *reinterpret_cast<float2*>(p2o + o) = q2;
                    if (!PONLY) *reinterpret_cast<float2*>(vo + o) = vn;
                    if (!PONLY && WRITEU) *reinterpret_cast<float2*>(u + o) = un;
                } else if (am & 1u) {
                    p1o[o] = q1.x; p2o[o] = q2.x;
                    if (!PONLY) vo[o] = vn.x;
                    if (!PONLY && WRITEU) u[o] = un.x;
                } else {
                    p1o[o + 1] = q1.y; p2o[o + 1] = q2.y;
                    if (!PONLY) vo[o + 1] = vn.y;
                    if (!PONLY && WRITEU) u[o + 1] = un.y;
                }
                if (!PONLY && CHECK) {
                    const float dax = (am & 1u) ? un.x - um.x : 0.f, day = (am & 2u) ? un.y - um.y : 0.f;
                    const float dbx = (am & 1u) ? vn.x - vm.x : 0.f, dby = (am & 2u) ? vn.y - vm.y : 0.f;
                    du2 = fmaf(dax, dax, fmaf(day, day, du2));
                    dv2 = fmaf(dbx, dbx, fmaf(dby, dby, dv2));
                }
            }
            p1m = cur.p1; p2m = cur.p2; vm = cur.v; fm = cur.f; um = cur.u; am = cur.act;
            wm = w; q1m = q1;
            cur = nxt;
            off = offn;
            moff = moffn;
        }
        if (!PONLY && CHECK) {
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
        int64_t i = (int64_t)((uint32_t)x / (uint32_t)P.W), j = x - i * P.W;   // x < 2^31
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
        int64_t i = (int64_t)((uint32_t)x / (uint32_t)P.W), j = x - i * P.W;   // x < 2^31
        int64_t o = i * P.ld + j;
        p1[o] = P1[o]; p2[o] = P2[o]; v[o] = V[o];
    }
}

// ========================================================== compact stencil

// neighbour slots of the table and the codes for pixels that are not in RD
// (NB_UUR = (i-2, j+1) and NB_LLD = (i+1, j-2) are the neighbours of x - e1
// and x - e2 that the fused iteration needs when it redoes their dual step)
enum { NB_UP = 0, NB_LEFT = 1, NB_DOWN = 2, NB_RIGHT = 3, NB_DOWNLEFT = 4, NB_UPRIGHT = 5, NB_UUR = 6,
       NB_LLD = 7, NB_COUNT = 8 };
constexpr int kNbBg = -1;    // fixed background: p = 0, v = 0
constexpr int kNbFg = -2;    // fixed foreground: p = 0, v = 1
constexpr int kNbOut = -3;   // outside the image (the gradient there is 0)

struct CompactState {
    void *p1[2], *p2[2], *v;
    float* f;
    float* u;
    float* w;        // div p - v/theta of the current iterate
    int32_t* nb;     // [NB_COUNT][stride]
    float* w2;       // the other w buffer of the fused iteration
    float* up;       // u of the iteration before a stopping test
    int64_t cap;
    int64_t stride;
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

// A batch of images solved together in compact form: their RD pixels are
// concatenated (image k's compact index i becomes base[k] + i), the
// neighbour table holds concatenated indices, and f is stored premultiplied
// by theta * lambda_k, so the persistent solver needs no per-image data.  A
// single image is a batch of one.
constexpr int kMaxBatch = 128;

struct BatchImage {
    const float* f;
    const uint32_t* act;
    const uint32_t* fg;
    const int32_t* wstart;
    const int32_t* counts;
    float *u, *v, *p1, *p2;
    long long word_off;      // first flattened word of this image
    int H, W, ld, nw, ntx;
    float theta_lambda;      // theta * lambda of this image
};

struct BatchDesc {
    int n;
    long long total_words;   // sum over images of H * ceil(W/32)
    BatchImage img[kMaxBatch];
};

// Image of a flattened word index (binary search over the word offsets).
__device__ __forceinline__ int batch_image_of(const BatchDesc& B, long long word) {
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.img[mid].word_off <= word) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Compact bases of the images (exclusive prefix of their RD counts) and the
// batch total; a total above the capacity records SEG_ERR_CAPACITY and stops
// the solve before it starts.
__global__ void k_batch_bases(BatchDesc B, int32_t* base, int32_t* totals, int64_t cap, WsHeader* h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long run = 0, tiles = 0;
    for (int k = 0; k < B.n; ++k) {
        base[k] = (int32_t)run;
        run += B.img[k].counts[1];
        tiles += B.img[k].counts[0];
    }
    base[B.n] = (int32_t)run;
    totals[0] = (int32_t)tiles;
    totals[1] = run > cap ? 0 : (int32_t)run;
    if (run > cap) {
        record_status(h, SEG_ERR_CAPACITY);
        h->done = 1;
        h->iters_done = 0;
    }
}

// One warp per mask word of the batch (lane b is pixel (i, 32 wx + b) of its
// image): gathers f (times theta lambda) and the start iterate of every RD
// pixel into compact order and fills its row of the neighbour table.
template <typename T>
__global__ void k_compact_gather(IterParams P, BatchDesc B, const int32_t* __restrict__ base,
                                 int warm, CompactState S, const WsHeader* __restrict__ h,
                                 const int32_t* __restrict__ totals, long long rm_above) {
    if (*(volatile const int*)&h->done) return;
    if (totals[1] > rm_above) return;   // the row-major solve of wide.cu takes this image
    const int lane = threadIdx.x & 31;
    const long long word = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (word >= B.total_words) return;
    const int k = batch_image_of(B, word);
    const BatchImage& I = B.img[k];
    const long long lw = word - I.word_off;
    const int i = (int)(lw / I.ntx);
    const int wx = (int)(lw - (long long)i * I.ntx);
    const int j = wx * 32 + lane;
    const int64_t wo = (int64_t)i * I.nw + wx;
    const uint32_t a = I.act[wo];
    if (!((a >> lane) & 1u)) return;
    const int b0 = base[k];
    const int64_t idx = b0 + I.wstart[wo] + __popc(a & lanemask_lt(lane));
    const int64_t o = (int64_t)i * I.ld + j;
    const float fv = I.f[o];
    const float hh = ((I.fg[wo] >> lane) & 1u) ? 1.f : 0.f;
    S.f[idx] = I.theta_lambda * fv;
    T* P1 = static_cast<T*>(S.p1[0]);
    T* P2 = static_cast<T*>(S.p2[0]);
    T* V = static_cast<T*>(S.v);
    if (warm) {
        // p1 on the last row and p2 on the last column never enter div p;
        // they are held at 0 (where a cold start keeps them)
        Store<T>::st(P1, idx, i < I.H - 1 ? I.p1[o] : 0.f);
        Store<T>::st(P2, idx, j < I.W - 1 ? I.p2[o] : 0.f);
        Store<T>::st(V, idx, I.v[o] - Store<T>::vbias);
        S.u[idx] = I.u[o];
        S.up[idx] = I.u[o];
    } else {
        Store<T>::st(P1, idx, 0.f);
        Store<T>::st(P2, idx, 0.f);
        Store<T>::st(V, idx, clamp01(fmaf(-I.theta_lambda, fv, hh)) - Store<T>::vbias);
        S.u[idx] = hh;
        S.up[idx] = hh;
    }
    // w = div p - v/theta; with p = 0 (cold start) it is -v/theta, else the
    // solver forms it once the table is complete
    S.w[idx] = warm ? 0.f : -(Store<T>::ld_rw(V, idx) + Store<T>::vbias) * P.inv_theta;
    IterParams Q = P;
    Q.H = I.H; Q.W = I.W; Q.nw = I.nw;
    auto code = [&](int ii, int jj) {
        const int c = nb_code(Q, I.act, I.fg, I.wstart, ii, jj);
        return c >= 0 ? c + b0 : c;
    };
    int32_t* nb = S.nb;
    const int64_t st = S.stride;
    nb[NB_UP * st + idx] = code(i - 1, j);
    nb[NB_LEFT * st + idx] = code(i, j - 1);
    nb[NB_DOWN * st + idx] = code(i + 1, j);
    nb[NB_RIGHT * st + idx] = code(i, j + 1);
    nb[NB_DOWNLEFT * st + idx] = code(i + 1, j - 1);
    nb[NB_UPRIGHT * st + idx] = code(i - 1, j + 1);
    nb[NB_UUR * st + idx] = code(i - 2, j + 1);
    nb[NB_LLD * st + idx] = code(i + 1, j - 2);
}

template <typename T>
__device__ __forceinline__ float to_f(T x) { return (float)x; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float to_f<__half>(__half x) { return __half2float(x); }

// w written by other blocks earlier in a persistent solve (see Store::ldc)
__device__ __forceinline__ float ldw(const float* p) { return *p; }

// state at a neighbour (0 where it is fixed or outside); the state is
// rewritten by other blocks between the phases of a persistent solve
template <typename T>
__device__ __forceinline__ float nb_ld(const T* X, int n) {
    return n >= 0 ? Store<T>::ldc(X, n) : 0.f;
}

// w at a fixed (non-RD) neighbour y: p(y) = 0, so div p(y) is minus the two
// p components that flow into y, and v(y) is its fixed value.
__device__ __forceinline__ float w_fixed(float p_in_1, float p_in_2, int code, float inv_theta) {
    return -(p_in_1 + p_in_2) - (code == kNbFg ? inv_theta : 0.f);
}

// One component of g = grad w at x toward the neighbour with code n: wn is w
// there when it is in RD, pa and pb the p components that flow into it when
// it is fixed, 0 across the image border.  Selects, not branches (the same
// values as the branching form).
__device__ __forceinline__ float g_comp(int n, float wn, float pa, float pb, float w0, float inv_theta) {
    const float w = n >= 0 ? wn : w_fixed(pa, pb, n, inv_theta);
    return n == kNbOut ? 0.f : w - w0;
}

// ------------------------------------------------ persistent compact solver
//
// All iterations of a compact solve run in one cooperative launch: every
// block owns a contiguous range of compact indices for the whole solve and
// the passes are separated by grid-wide barriers (all blocks are resident, as
// the cooperative launch guarantees).  One iteration:
//   dual phase   p'(x) from w at x, x+e1, x+e2           -> barrier
//   primal phase u', v', w', stop-test partials          -> barrier
//   (check iterations) block 0 sums the partials in a fixed order and raises
//   the done flag, which every block reads after the next barrier.
// The grid takes one of these (the same in every block):
//  * fused (n_inner = 1, at most one pixel per block: very sparse domains,
//    where the ring set-up below costs more than it saves): one phase and one barrier
//    per iteration; the thread of x also redoes the dual steps of x - e1 and
//    x - e2 (same inputs, same arithmetic, same rounding as their owners),
//    which is all the v-step of x needs, and w is ping-ponged.  The iterates
//    are bit-identical to the two-phase ones.
//  * one barrier with shared-memory state and a ring (n_inner = 1, every
//    block's state fits, by a grid-wide vote): see compact_iterations_h1.
// Otherwise each block takes the first of these that applies (blocks may
// differ; all keep the same two-barrier protocol and the same global arrays
// current):
//  * shared-memory state (n_inner = 1, the block's pixels fit): see
//    compact_iterations_gh below.
//  * neighbour-table rows and v in shared memory, neighbour values from the
//    global arrays (only the owner reads a pixel's rows and v).
//  * everything in global memory.
constexpr int kBackwardThreads = 1024;  // block size of the persistent reverse sweep (tables in global memory)
constexpr int kBackwardThreadsSm = 512;  // block size of the sweep with its tables in shared memory
constexpr int kBackwardMinBlocks = 2;   // resident blocks per SM the registers are sized for (global tables)
constexpr int kBackwardMinBlocksSm = 2;   // the same, tables in shared memory
constexpr int kBackwardUnroll = 1;      // pixels per thread whose loads are in flight together
// dynamic shared memory of the persistent solver: one or two blocks per SM
constexpr size_t compact_smem(int nt) { return nt == 1024 ? 226 * 1024 : 112 * 1024; }
constexpr int kCompactThreads = 512;   // two blocks per SM: one block's block barriers overlap the other's work
constexpr int kCompactWideUnroll = 2;   // pixels per thread in flight in k_solve_compact_wide
constexpr int kCompactUnroll = 4;       // pixels per thread in flight in the two-phase iteration
// the fused iteration for blocks of at most this many pixels (the one-barrier
// ring path measured faster at every size tried above it, 0.6 to 5 pixels
// per thread)
constexpr int kFuseMaxPerBlock = 1;

// Own-pixel arrays (neighbour-table rows, v) of the pixels a block updates:
// SH, copies in shared memory indexed from the block's first pixel a0; else
// the global arrays (a0 = 0).  theta lambda f is read from its global array.
template <typename T, bool SH>
struct Own {
    const int32_t* nb;   // [NB_COUNT][ns]
    int64_t ns;
    T* v;
    const float* f;      // global, indexed by a
    int a0;
    __device__ __forceinline__ int nbr(int k, int a) const {
        const int64_t i = (int64_t)k * ns + (a - a0);
        return SH ? nb[i] : __ldg(nb + i);
    }
    __device__ __forceinline__ float fv(int a) const { return __ldg(f + a); }
    __device__ __forceinline__ int vi(int a) const { return a - a0; }
};

// Dual step on one RD pixel:
//   g = (w(x+e1) - w(x), w(x+e2) - w(x))   (a component is 0 across the
//       image border), p'(x) = (p(x) + tau g) / (1 + tau |g|),
// with w = div p - v/theta taken from the primal step's output where the
// neighbour is in RD, and formed from p(x) and p(x+e1-e2) (resp. p(x+e2-e1))
// where it is fixed.  p1 vanishes on the last row and p2 on the last column
// (their gradient component is 0 there and they start at 0).
template <typename T, bool SH>
__device__ __forceinline__ void dual_one(const IterParams& P, int a, const Own<T, SH>& O, const T* P1i,
                                         const T* P2i, const float* Wc, T* P1o, T* P2o, uint32_t seed) {
    const int n_down = O.nbr(NB_DOWN, a);
    const int n_right = O.nbr(NB_RIGHT, a);
    const int n_dl = O.nbr(NB_DOWNLEFT, a);
    const int n_ur = O.nbr(NB_UPRIGHT, a);
    const float p1 = Store<T>::ldc(P1i, a), p2 = Store<T>::ldc(P2i, a);
    const float w0 = ldw(Wc + a);
    const float wd = n_down >= 0 ? ldw(Wc + n_down) : 0.f;
    const float wr = n_right >= 0 ? ldw(Wc + n_right) : 0.f;
    const float p2dl = nb_ld(P2i, n_dl);
    const float p1ur = nb_ld(P1i, n_ur);
    // (branches, not g_comp's selects: the neighbour loads above are
    // conditional, and this form measured faster on this path)
    float g1 = 0.f, g2 = 0.f;
    if (n_down != kNbOut) g1 = (n_down >= 0 ? wd : w_fixed(p1, p2dl, n_down, P.inv_theta)) - w0;
    if (n_right != kNbOut) g2 = (n_right >= 0 ? wr : w_fixed(p1ur, p2, n_right, P.inv_theta)) - w0;
    float q1, q2;
    chambolle_update(p1, p2, g1, g2, P.tau, q1, q2);
    const uint32_t rnd = mix32((uint32_t)a * 3u + seed);
    Store<T>::st_sr(P1o, a, q1, rnd);
    Store<T>::st_sr(P2o, a, q2, mix32(rnd ^ 0x9e3779b9u));
}

// Primal step on one RD pixel: u' = v - theta div p', v' = clip(u' - theta
// lambda f) (v updated in place), w' = div p' - v'/theta for the next dual
// step.  wonly: just w = div p' - v/theta (between extra fixed-point sweeps,
// or for a warm start).
template <typename T, bool SH>
__device__ __forceinline__ void primal_one(const IterParams& P, int a, const Own<T, SH>& O, const T* P1n,
                                           const T* P2n, float* U, float* Up, float* Wc, bool wonly,
                                           bool check, bool write_u, bool write_prev, uint32_t seed,
                                           float& du2, float& dv2) {
    const int n_up = O.nbr(NB_UP, a);
    const int n_left = O.nbr(NB_LEFT, a);
    const float q1 = Store<T>::ldc(P1n, a), q2 = Store<T>::ldc(P2n, a);
    const float vv = Store<T>::ld_rw(O.v, O.vi(a)) + Store<T>::vbias;
    const float q1u = nb_ld(P1n, n_up), q2l = nb_ld(P2n, n_left);
    const float div = (q1 - q1u) + (q2 - q2l);
    if (wonly) {
        Wc[a] = div - vv * P.inv_theta;
        return;
    }
    const float un = fmaf(-P.theta, div, vv);
    const float vn = clamp01(un - O.fv(a));   // F = theta lambda f
    const float vs = Store<T>::st_sr(O.v, O.vi(a), vn - Store<T>::vbias, mix32((uint32_t)a * 5u + seed)) +
                     Store<T>::vbias;
    Wc[a] = div - vs * P.inv_theta;
    if (check) {
        const float da = un - Up[a], db = vn - vv;
        du2 = fmaf(da, da, du2);
        dv2 = fmaf(db, db, dv2);
    }
    if (write_prev) Up[a] = un;
    if (write_u) U[a] = un;
}

// One fused iteration at one RD pixel (n_inner = 1): p'(x) as the dual step
// computes it, p1'(x - e1) and p2'(x - e2) as the dual steps of x - e1 and
// x - e2 compute them (their neighbours below / right are x, x - e1 + e2 and
// x + e1 - e2, x; a fixed one of those needs p at (i-2, j+1) resp.
// (i+1, j-2)), each rounded as its owner stores it; then the primal step of
// x.  Reads p, w of the current iterate (P1i, P2i, Wi), writes p', w' to the
// other buffers and v in place.
template <typename T, bool SH>
__device__ __forceinline__ void fused_one(const IterParams& P, int a, const Own<T, SH>& O, const T* P1i,
                                          const T* P2i, const float* Wi, T* P1o, T* P2o, float* Wo, float* U,
                                          float* Up, bool check, bool write_u, bool write_prev, uint32_t seed_d,
                                          uint32_t seed_p, float& du2, float& dv2) {
    const int n_up = O.nbr(NB_UP, a), n_left = O.nbr(NB_LEFT, a);
    const int n_down = O.nbr(NB_DOWN, a), n_right = O.nbr(NB_RIGHT, a);
    const int n_dl = O.nbr(NB_DOWNLEFT, a), n_ur = O.nbr(NB_UPRIGHT, a);
    const int n_uur = n_up >= 0 ? O.nbr(NB_UUR, a) : kNbOut;
    const int n_lld = n_left >= 0 ? O.nbr(NB_LLD, a) : kNbOut;
    // every load of the step, independent of one another
    const float p1 = Store<T>::ldc(P1i, a), p2 = Store<T>::ldc(P2i, a);
    const float w0 = ldw(Wi + a);
    const float wd = n_down >= 0 ? ldw(Wi + n_down) : 0.f;
    const float wr = n_right >= 0 ? ldw(Wi + n_right) : 0.f;
    const float p2dl = nb_ld(P2i, n_dl), p1ur = nb_ld(P1i, n_ur);
    const float p1U = nb_ld(P1i, n_up), p2U = nb_ld(P2i, n_up);
    const float wU = n_up >= 0 ? ldw(Wi + n_up) : 0.f;
    const float wur = n_ur >= 0 ? ldw(Wi + n_ur) : 0.f;
    const float p1uur = nb_ld(P1i, n_uur);
    const float p1L = nb_ld(P1i, n_left), p2L = nb_ld(P2i, n_left);
    const float wL = n_left >= 0 ? ldw(Wi + n_left) : 0.f;
    const float wdl = n_dl >= 0 ? ldw(Wi + n_dl) : 0.f;
    const float p2lld = nb_ld(P2i, n_lld);
    // p'(x)
    const float g1 = g_comp(n_down, wd, p1, p2dl, w0, P.inv_theta);
    const float g2 = g_comp(n_right, wr, p1ur, p2, w0, P.inv_theta);
    float q1, q2;
    chambolle_update(p1, p2, g1, g2, P.tau, q1, q2);
    const uint32_t rnd = mix32((uint32_t)a * 3u + seed_d);
    q1 = Store<T>::st_sr(P1o, a, q1, rnd);
    q2 = Store<T>::st_sr(P2o, a, q2, mix32(rnd ^ 0x9e3779b9u));
    // p1'(x - e1)
    float q1u = 0.f;
    if (n_up >= 0) {
        const float gu2 = g_comp(n_ur, wur, p1uur, p2U, wU, P.inv_theta);
        float b1, b2;
        chambolle_update(p1U, p2U, w0 - wU, gu2, P.tau, b1, b2);
        q1u = Store<T>::sr(b1, mix32((uint32_t)n_up * 3u + seed_d));
    }
    // p2'(x - e2)
    float q2l = 0.f;
    if (n_left >= 0) {
        const float gl1 = g_comp(n_dl, wdl, p1L, p2lld, wL, P.inv_theta);
        float b1, b2;
        chambolle_update(p1L, p2L, gl1, w0 - wL, P.tau, b1, b2);
        q2l = Store<T>::sr(b2, mix32(mix32((uint32_t)n_left * 3u + seed_d) ^ 0x9e3779b9u));
    }
    // primal step of x
    const float div = (q1 - q1u) + (q2 - q2l);
    const float vv = Store<T>::ld_rw(O.v, O.vi(a)) + Store<T>::vbias;
    const float un = fmaf(-P.theta, div, vv);
    const float vn = clamp01(un - O.fv(a));   // F = theta lambda f
    const float vs = Store<T>::st_sr(O.v, O.vi(a), vn - Store<T>::vbias, mix32((uint32_t)a * 5u + seed_p)) +
                     Store<T>::vbias;
    Wo[a] = div - vs * P.inv_theta;
    if (check) {
        const float da = un - Up[a], db = vn - vv;
        du2 = fmaf(da, da, du2);
        dv2 = fmaf(db, db, dv2);
    }
    if (write_prev) Up[a] = un;
    if (write_u) U[a] = un;
}

// The iterations of one block of the persistent compact solver (see above);
// false when a grid barrier timed out.
template <typename T, bool SH, int NT, int UNROLL>
__device__ __forceinline__ bool compact_iterations(const IterParams& P, const Own<T, SH>& O, int a0, int a1,
                                                   int iters, int n_inner, int check_every, double tol, int warm,
                                                   int64_t stride, T* P1a, T* P1b, T* P2a, T* P2b, float* Uu,
                                                   float* Up, float* Wc, float* Wc2, double* partials, WsHeader* h,
                                                   float* ckpt, int ckpt_every, double* s_red, int fuse,
                                                   unsigned& gen) {
    // gen: barriers passed (the arrival counter starts at 0 each solve and
    // runs on across the waves of a batch)
    const unsigned nblocks = gridDim.x;
    const int tid = threadIdx.x, nt = NT;
    int pb = 0;
    // the block's pixels, UNROLL per thread in flight (one in the fused
    // step, which keeps about three times as many values live)
    auto each = [&](auto&& op) {
        int a = a0 + tid;
        for (; a + (UNROLL - 1) * nt < a1; a += UNROLL * nt) {
#pragma unroll
            for (int k = 0; k < UNROLL; ++k) op(a + k * nt);
        }
        for (; a < a1; a += nt) op(a);
    };
    auto each1 = [&](auto&& op) {
        for (int a = a0 + tid; a < a1; a += nt) op(a);
    };
    float dummy0 = 0.f, dummy1 = 0.f;
    // current / other ping-pong buffers of p, selected without indexing
    auto p1c = [&]() { return pb ? P1b : P1a; };
    auto p2c = [&]() { return pb ? P2b : P2a; };
    auto p1o = [&]() { return pb ? P1a : P1b; };
    auto p2o = [&]() { return pb ? P2a : P2b; };
    if (warm) {   // w of the warm-start iterate
        for (int a = a0 + tid; a < a1; a += nt)
            primal_one(P, a, O, P1a, P2a, Uu, Up, Wc, true, false, false, false, 0u, dummy0, dummy1);
        if (!grid_sync(h, nblocks, gen)) return false;
    }
    const int C = check_every;
    // checkpoint m holds (p1, p2, v) of iterate m * ckpt_every, as float32
    auto save = [&](int m) {
        float* c = ckpt + (int64_t)m * 3 * stride;
        const T* q1 = p1c();
        const T* q2 = p2c();
        for (int a = a0 + tid; a < a1; a += nt) {
            c[a] = to_f(q1[a]);
            c[stride + a] = to_f(q2[a]);
            c[2 * stride + a] = to_f(O.v[O.vi(a)]) + Store<T>::vbias;
        }
    };
    if (ckpt) save(0);
    if (fuse) {   // fused: one phase and one barrier per iteration
        int wb = 0, chk = 0;
        for (int it = 0; it < iters; ++it) {
            const int l = it + 1;
            const bool check = (l % C == 0) || l == iters;
            const bool write_u = check;   // the output u and the stopped iterate
        const bool write_prev = l < iters && ((l + 1) % C == 0 || l + 1 == iters);
            const uint32_t seed_d = mix32(0x51ed270bu ^ (uint32_t)(it * 131));
            const uint32_t seed_p = mix32(0x2545f491u ^ (uint32_t)it);
            const T* pi1 = p1c(); const T* pi2 = p2c();
            T* po1 = p1o(); T* po2 = p2o();
            const float* wi = wb ? Wc2 : Wc;
            float* wo = wb ? Wc : Wc2;
            float du2 = 0.f, dv2 = 0.f;
            if (!check && !write_prev)
                each1([&](int a) {
                    fused_one(P, a, O, pi1, pi2, wi, po1, po2, wo, Uu, Up, false, false, false, seed_d, seed_p, du2,
                              dv2);
                });
            else
                each1([&](int a) {
                    fused_one(P, a, O, pi1, pi2, wi, po1, po2, wo, Uu, Up, check, write_u, write_prev, seed_d,
                              seed_p, du2, dv2);
                });
            pb ^= 1;
            wb ^= 1;
            if (ckpt && l % ckpt_every == 0 && l < iters) save(l / ckpt_every);   // own pixels: no barrier
            // stopping-test partials, double-buffered by check so that a fast
            // block cannot overwrite those a slow block is still summing
            double* part = partials + 2 * (int64_t)nblocks * (chk & 1);
            if (check) {
                float x = du2, y = dv2;
                block_sum2f<NT>(x, y, reinterpret_cast<float*>(s_red));
                if (tid == 0) {
                    part[2 * blockIdx.x] = x;
                    part[2 * blockIdx.x + 1] = y;
                }
            }
            if (!grid_sync(h, nblocks, gen)) return false;
            if (check) {
                // Section 4 stopping test: every block sums the block partials
                // in the same fixed order, so all stop at the same iteration
                // (squared norms against tol^2: the square roots are taken
                // once, for the stats)
                if (tid < 32) {
                    double sx, sy;
                    sum_partials_warp0(part, (int)nblocks, sx, sy);
                    if (tid == 0) {
                        const bool stop = tol > 0.0 && fmax(sx, sy) <= tol * tol;
                        s_red[0] = stop ? 1.0 : 0.0;
                        if (blockIdx.x == 0) {
                            h->du2 = sx;
                            h->dv2 = sy;
                            h->last_check = l;
                            if (stop) {
                                h->iters_done = l;
                                h->done = 1;
                            }
                        }
                    }
                }
                __syncthreads();
                const bool stop = s_red[0] != 0.0;
                ++chk;
                __syncthreads();
                if (stop) return true;
            }
        }
        return true;
    }
    for (int it = 0; it < iters; ++it) {
        const int l = it + 1;
        for (int sw = 0; sw < n_inner; ++sw) {
            const uint32_t seed = mix32(0x51ed270bu ^ (uint32_t)(it * 131 + sw));
            const T* pi1 = p1c(); const T* pi2 = p2c();
            T* po1 = p1o(); T* po2 = p2o();
            each([&](int a) { dual_one(P, a, O, pi1, pi2, Wc, po1, po2, seed); });
            pb ^= 1;
            bool done;
            if (!grid_sync_poll(h, nblocks, gen, sw == 0 && it > 0 && (it % C == 0), done)) return false;
            if (done) return true;   // the previous iteration's stopping test fired
            if (sw + 1 < n_inner) {
                for (int b = a0 + tid; b < a1; b += nt)
                    primal_one(P, b, O, p1c(), p2c(), Uu, Up, Wc, true, false, false, false, 0u, dummy0, dummy1);
                if (!grid_sync(h, nblocks, gen)) return false;
            }
        }
        const bool check = (l % C == 0) || l == iters;
        const bool write_u = check;   // the output u and the stopped iterate
        const bool write_prev = l < iters && ((l + 1) % C == 0 || l + 1 == iters);
        const uint32_t seed = mix32(0x2545f491u ^ (uint32_t)it);
        float du2 = 0.f, dv2 = 0.f;
        const T* q1s = p1c(); const T* q2s = p2c();
        if (!check && !write_prev)
            each([&](int a) { primal_one(P, a, O, q1s, q2s, Uu, Up, Wc, false, false, false, false, seed, du2, dv2); });
        else
            each([&](int a) {
                primal_one(P, a, O, q1s, q2s, Uu, Up, Wc, false, check, write_u, write_prev, seed, du2, dv2);
            });
        if (ckpt && l % ckpt_every == 0 && l < iters) save(l / ckpt_every);
        if (check) {
            float x = du2, y = dv2;
            block_sum2f<NT>(x, y, reinterpret_cast<float*>(s_red));
            if (tid == 0) {
                partials[2 * blockIdx.x] = x;
                partials[2 * blockIdx.x + 1] = y;
            }
        }
        if (!grid_sync(h, nblocks, gen)) return false;
        if (check && blockIdx.x == 0) {
            // Section 4 stopping test: fixed-order FP64 sum of the block partials,
            // squared norms against tol^2 (square roots taken once, for the stats)
            double sx = 0.0, sy = 0.0;
            if (tid < 32) sum_partials_warp0(partials, (int)nblocks, sx, sy);
            if (tid == 0) {
                h->du2 = sx;
                h->dv2 = sy;
                h->last_check = l;
                if (tol > 0.0 && fmax(sx, sy) <= tol * tol) {
                    h->iters_done = l;
                    __threadfence();
                    h->done = 1;
                }
            }
            __syncthreads();
        }
    }
    return true;
}

// ---- shared-memory-resident block state (two-phase iteration, n_inner = 1)
//
// When a block's pixels fit, the whole state of its own pixels lives in
// shared memory for the solve, as float words:
//   P1, P2   two regions each (the ping-pong buffers b = 0, 1) of
//            [own pixels | one zero word | ghost words]
//   W        [own pixels | zero word | ghost words], V [own pixels]
// and every neighbour read is one shared-memory load at a word offset fixed
// at the start: a neighbour the block owns is its own word, a fixed (or
// outside) one the zero word, and one another block owns a ghost word, which
// the block refills from the global arrays (an L2 read) at the start of the
// phase that reads it.  The dual step reads w below x when that neighbour is
// in RD and p2 at x + e1 - e2 when it is fixed (never both), so one offset
// slot serves the two; likewise w right of x and p1 at x - e1 + e2.  p of buffer b is at offset + b x (region size), so
// the ping-pong needs no branch.  A per-pixel byte holds the class of the
// neighbours below and right (RD / fixed background / fixed foreground /
// outside), whether other blocks read the pixel (then its p' and w' are also
// written to the global arrays), and is otherwise the same arithmetic and
// rounding as dual_one / primal_one.  The barrier and stopping-test protocol
// is the one of compact_iterations, so blocks on either path interleave.
// ghost kinds: below (w, or p2 at x + e1 - e2 when below is fixed), right (w,
// or p1 at x - e1 + e2), above (p1'), left (p2')
enum { GK_D = 0, GK_R, GK_UP, GK_LEFT, GK_KINDS };
constexpr uint8_t kFlExport = 16;       // other blocks read this pixel
constexpr uint8_t kFlDualGhost = 32;    // its dual step reads a ghost word
constexpr uint8_t kFlPrimalGhost = 64;  // its primal step reads a ghost word
constexpr uint8_t kFlLate = kFlDualGhost | kFlExport;   // one-barrier path: dual step after the ghost refill
constexpr int kGhostRegs = 2;           // ghosts per thread carried in registers while the interior runs

struct GhostLayout {
    int n;                 // own pixels
    int ns1, ns2, nsw;     // region sizes (words) of P1, P2 (per buffer) and W
    int p1, p2, w, v;      // word offsets of the regions
    int gd, gp;            // ghosts read by the dual / by the primal
    int nbd, nbp;          // pixels whose dual / primal step reads a ghost
    size_t off16, offfl, offgs, offgd, offbd, offbp, bytes;   // byte offsets of the tables
};

template <typename T>
struct GhostState {
    float* sm;             // the shared-memory words
    const uint16_t* off;   // [4][n] word offsets of the kinds D, R, UP, LEFT (p words: buffer 0)
    const uint8_t* fl;     // [n]
    const int32_t* gsrc;   // [gd + gp] compact index of each ghost's pixel
    const uint16_t* gdst;  // [gd + gp] word offset of each ghost (buffer 0 for p kinds)
    const uint16_t* bd;    // [nbd] pixels whose dual step reads a ghost
    const uint16_t* bp;    // [nbp] pixels whose primal step reads a ghost
    GhostLayout L;
    __device__ __forceinline__ T* v() const { return reinterpret_cast<T*>(sm + L.v); }
};

// The source pixel and region (0 W, 1 P1, 2 P2) of the ghost-path read of
// kind k at compact pixel a; a source < 0 reads the zero word.
__device__ __forceinline__ int gk_src(const int32_t* __restrict__ nb, int64_t stride, int a, int k, int& reg) {
    if (k == GK_D || k == GK_R) {
        const int m = __ldg(nb + (k == GK_D ? NB_DOWN : NB_RIGHT) * stride + a);
        if (m >= 0) { reg = 0; return m; }
        reg = k == GK_D ? 2 : 1;
        if (m == kNbOut) return -1;
        return __ldg(nb + (k == GK_D ? NB_DOWNLEFT : NB_UPRIGHT) * stride + a);
    }
    reg = k == GK_UP ? 1 : 2;
    return __ldg(nb + (k == GK_UP ? NB_UP : NB_LEFT) * stride + a);
}

// The class byte of the neighbours below and right of pixel a (bits 0-1 and
// 2-3: 0 RD, 1 fixed Bg, 2 fixed Fg, 3 outside).
__device__ __forceinline__ uint8_t gk_codes(const int32_t* __restrict__ nb, int64_t stride, int a) {
    const int md = __ldg(nb + NB_DOWN * stride + a), mr = __ldg(nb + NB_RIGHT * stride + a);
    return (uint8_t)((md >= 0 ? 0 : md == kNbBg ? 1 : md == kNbFg ? 2 : 3) |
                     ((mr >= 0 ? 0 : mr == kNbBg ? 1 : mr == kNbFg ? 2 : 3) << 2));
}

// Per-phase views of the shared-memory state (pointers fixed for a phase).
struct DualView {
    const float *p1, *p2, *w;     // own p (buffer pb) and w, by own index
    float *q1, *q2;               // own p' (the other buffer)
    const float* sm;              // all shared words (offsets: p words of buffer 0)
    int sh1, sh2;                 // shift of buffer pb in the P1 / P2 regions
    const uint16_t *od, *orr;     // offsets of the kinds D and R
};
struct PrimalView {
    const float *q1, *q2;         // own p' (buffer pb)
    const float *n1, *n2;         // neighbour p' words of buffer pb
    float* w;                     // own w
    const uint16_t *ou, *ol;      // offsets of the neighbours above, left
};

template <typename T>
__device__ __forceinline__ void dual_gh(const IterParams& P, int i, int a, uint8_t fl, const DualView& D,
                                        T* P1o, T* P2o, uint32_t seed) {
    const float p1 = D.p1[i], p2 = D.p2[i], w0 = D.w[i];
    const int cd = fl & 3, cr = (fl >> 2) & 3;   // 0 RD, 1 fixed Bg, 2 fixed Fg, 3 outside
    // w below (RD) or p2 at x + e1 - e2 (below fixed; a p word of buffer pb)
    const float xd = D.sm[D.od[i] + (cd ? D.sh2 : 0)];
    const float xr = D.sm[D.orr[i] + (cr ? D.sh1 : 0)];
    // selects, not branches (the values of g_comp)
    const float wd = cd == 0 ? xd : -(p1 + xd) - (cd == 2 ? P.inv_theta : 0.f);
    const float wr = cr == 0 ? xr : -(xr + p2) - (cr == 2 ? P.inv_theta : 0.f);
    const float g1 = cd == 3 ? 0.f : wd - w0;
    const float g2 = cr == 3 ? 0.f : wr - w0;
    float q1, q2;
    chambolle_update(p1, p2, g1, g2, P.tau, q1, q2);
    const uint32_t rnd = mix32((uint32_t)a * 3u + seed);
    const uint32_t rnd2 = mix32(rnd ^ 0x9e3779b9u);
    if (fl & kFlExport) {
        q1 = Store<T>::st_sr(P1o, a, q1, rnd);
        q2 = Store<T>::st_sr(P2o, a, q2, rnd2);
    } else {
        q1 = Store<T>::sr(q1, rnd);
        q2 = Store<T>::sr(q2, rnd2);
    }
    D.q1[i] = q1;
    D.q2[i] = q2;
}

// Primal step of own pixel i (compact index a) with fa = theta lambda f(a).
template <typename T>
__device__ __forceinline__ void primal_gh_f(const IterParams& P, int i, int a, uint8_t fl, const PrimalView& Q,
                                            T* V, float fa, float* U, float* Up, float* Wg, bool check,
                                            bool write_u, bool write_prev, uint32_t seed, float& du2,
                                            float& dv2) {
    const float q1 = Q.q1[i], q2 = Q.q2[i];
    const float q1u = Q.n1[Q.ou[i]], q2l = Q.n2[Q.ol[i]];
    const float vv = Store<T>::ld_rw(V, i) + Store<T>::vbias;
    const float div = (q1 - q1u) + (q2 - q2l);
    const float un = fmaf(-P.theta, div, vv);
    const float vn = clamp01(un - fa);   // fa = theta lambda f at a
    const float vs = Store<T>::st_sr(V, i, vn - Store<T>::vbias, mix32((uint32_t)a * 5u + seed)) +
                     Store<T>::vbias;
    const float wv = div - vs * P.inv_theta;
    Q.w[i] = wv;
    if (fl & kFlExport) Wg[a] = wv;
    if (check) {
        const float da = un - Up[a], db = vn - vv;
        du2 = fmaf(da, da, du2);
        dv2 = fmaf(db, db, dv2);
    }
    if (write_prev) Up[a] = un;
    if (write_u) U[a] = un;
}

// The same with theta lambda f read from F.
template <typename T>
__device__ __forceinline__ void primal_gh(const IterParams& P, int i, int a, uint8_t fl, const PrimalView& Q,
                                          T* V, const float* F, float* U, float* Up, float* Wg, bool check,
                                          bool write_u, bool write_prev, uint32_t seed, float& du2,
                                          float& dv2) {
    primal_gh_f<T>(P, i, a, fl, Q, V, __ldg(F + a), U, Up, Wg, check, write_u, write_prev, seed, du2, dv2);
}

// Refills ghosts [g0, g1) from the global arrays: w for the neighbours below /
// right, p of buffer pb for the others.
template <typename T>
__device__ __forceinline__ void fill_ghosts(const GhostState<T>& S, int g0, int g1, int pb, const T* P1g,
                                            const T* P2g, const float* Wg, int nt) {
    const GhostLayout& L = S.L;
    for (int g = g0 + (int)threadIdx.x; g < g1; g += nt) {
        const int src = S.gsrc[g], dst = S.gdst[g];
        if (dst >= L.w) S.sm[dst] = ldw(Wg + src);
        else if (dst >= L.p2) S.sm[dst + pb * L.ns2] = Store<T>::ldc(P2g, src);
        else S.sm[dst + pb * L.ns1] = Store<T>::ldc(P1g, src);
    }
}

// Overlapped refill: each thread loads up to kGhostRegs ghosts of [g0, g1)
// into registers (the loads stay in flight), and stores them once the
// interior pixels are done.
template <typename T>
struct GhostRegs {
    float x[kGhostRegs];
    __device__ __forceinline__ void load(const GhostState<T>& S, int g0, int g1, int pb, const T* P1g,
                                         const T* P2g, const float* Wg, int nt) {
        const GhostLayout& L = S.L;
#pragma unroll
        for (int j = 0; j < kGhostRegs; ++j) {
            const int g = g0 + (int)threadIdx.x + j * nt;
            x[j] = 0.f;
            if (g < g1) {
                const int src = S.gsrc[g], dst = S.gdst[g];
                x[j] = dst >= L.w ? ldw(Wg + src) : dst >= L.p2 ? Store<T>::ldc(P2g, src) : Store<T>::ldc(P1g, src);
            }
        }
    }
    __device__ __forceinline__ void store(const GhostState<T>& S, int g0, int g1, int pb, int nt) const {
        const GhostLayout& L = S.L;
#pragma unroll
        for (int j = 0; j < kGhostRegs; ++j) {
            const int g = g0 + (int)threadIdx.x + j * nt;
            if (g < g1) {
                const int dst = S.gdst[g];
                S.sm[dst >= L.w ? dst : dst >= L.p2 ? dst + pb * L.ns2 : dst + pb * L.ns1] = x[j];
            }
        }
    }
};

// The iterations with shared-memory-resident state; returns false when a
// barrier timed out, else the final iterate's buffer in *fb and iteration
// count in *lf.
template <typename T, int NT, int UNROLL>
__device__ __forceinline__ bool compact_iterations_gh(const IterParams& P, const GhostState<T>& S, int a0, int a1,
                                                      int iters, int check_every, double tol, int64_t stride,
                                                      T* P1a, T* P1b, T* P2a, T* P2b, const float* F,
                                                      float* U, float* Up, float* Wc, double* partials,
                                                      WsHeader* h, float* ckpt, int ckpt_every, double* s_red,
                                                      unsigned& gen, int* fb, int* lf) {
    const unsigned nblocks = gridDim.x;
    const int tid = threadIdx.x, nt = NT;
    const GhostLayout& L = S.L;
    // every ghost of a phase fits in the threads' registers (uniform in the block)
    const bool overlap = L.gd <= kGhostRegs * NT && L.gp <= kGhostRegs * NT;
    int pb = 0;
    auto each = [&](auto&& op) {
        int a = a0 + tid;
        for (; a + (UNROLL - 1) * nt < a1; a += UNROLL * nt) {
#pragma unroll
            for (int k = 0; k < UNROLL; ++k) op(a + k * nt);
        }
        for (; a < a1; a += nt) op(a);
    };
    auto save = [&](int m) {
        float* c = ckpt + (int64_t)m * 3 * stride;
        const T* V = S.v();
        for (int a = a0 + tid; a < a1; a += nt) {
            const int i = a - a0;
            c[a] = S.sm[L.p1 + pb * L.ns1 + i];
            c[stride + a] = S.sm[L.p2 + pb * L.ns2 + i];
            c[2 * stride + a] = to_f(V[i]) + Store<T>::vbias;
        }
    };
    if (ckpt) save(0);
    const int C = check_every;
    *fb = 0;
    *lf = iters;
    for (int it = 0; it < iters; ++it) {
        const int l = it + 1;
        {
            const uint32_t seed = mix32(0x51ed270bu ^ (uint32_t)(it * 131));
            T* o1 = pb ? P1a : P1b;
            T* o2 = pb ? P2a : P2b;
            DualView D;
            D.p1 = S.sm + L.p1 + pb * L.ns1;
            D.p2 = S.sm + L.p2 + pb * L.ns2;
            D.w = S.sm + L.w;
            D.q1 = S.sm + L.p1 + (1 - pb) * L.ns1;
            D.q2 = S.sm + L.p2 + (1 - pb) * L.ns2;
            D.sm = S.sm;
            D.sh1 = pb * L.ns1;
            D.sh2 = pb * L.ns2;
            D.od = S.off + GK_D * L.n;
            D.orr = S.off + GK_R * L.n;
            if (overlap) {   // ghosts in flight while the interior pixels update
                GhostRegs<T> R;
                R.load(S, 0, L.gd, pb, pb ? P1b : P1a, pb ? P2b : P2a, Wc, nt);
                each([&](int a) {
                    const uint8_t f = S.fl[a - a0];
                    if (!(f & kFlDualGhost)) dual_gh(P, a - a0, a, f, D, o1, o2, seed);
                });
                R.store(S, 0, L.gd, pb, nt);
                __syncthreads();
                for (int e = tid; e < L.nbd; e += nt) {
                    const int i = S.bd[e];
                    dual_gh(P, i, a0 + i, S.fl[i], D, o1, o2, seed);
                }
            } else {
                fill_ghosts(S, 0, L.gd, pb, pb ? P1b : P1a, pb ? P2b : P2a, Wc, nt);
                __syncthreads();
                each([&](int a) { dual_gh(P, a - a0, a, S.fl[a - a0], D, o1, o2, seed); });
            }
            pb ^= 1;
            bool done;
            if (!grid_sync_poll(h, nblocks, gen, it > 0 && (it % C == 0), done)) return false;
            if (done) {
                *fb = pb ^ 1;   // the dual step after the stopping test wrote the other buffer
                *lf = it;
                return true;
            }
        }
        const bool check = (l % C == 0) || l == iters;
        const bool write_u = check;   // the output u and the stopped iterate
        const bool write_prev = l < iters && ((l + 1) % C == 0 || l + 1 == iters);
        const uint32_t seed = mix32(0x2545f491u ^ (uint32_t)it);
        float du2 = 0.f, dv2 = 0.f;
        PrimalView Q;
        Q.q1 = S.sm + L.p1 + pb * L.ns1;
        Q.q2 = S.sm + L.p2 + pb * L.ns2;
        Q.n1 = S.sm + pb * L.ns1;
        Q.n2 = S.sm + pb * L.ns2;
        Q.w = S.sm + L.w;
        Q.ou = S.off + GK_UP * L.n;
        Q.ol = S.off + GK_LEFT * L.n;
        T* Vs = S.v();
        if (overlap) {
            GhostRegs<T> R;
            R.load(S, L.gd, L.gd + L.gp, pb, pb ? P1b : P1a, pb ? P2b : P2a, Wc, nt);
            if (!check && !write_prev)
                each([&](int a) {
                    const uint8_t f = S.fl[a - a0];
                    if (!(f & kFlPrimalGhost))
                        primal_gh(P, a - a0, a, f, Q, Vs, F, U, Up, Wc, false, false, false, seed, du2, dv2);
                });
            else
                each([&](int a) {
                    const uint8_t f = S.fl[a - a0];
                    if (!(f & kFlPrimalGhost))
                        primal_gh(P, a - a0, a, f, Q, Vs, F, U, Up, Wc, check, write_u, write_prev, seed, du2, dv2);
                });
            R.store(S, L.gd, L.gd + L.gp, pb, nt);
            __syncthreads();
            for (int e = tid; e < L.nbp; e += nt) {
                const int i = S.bp[e];
                primal_gh(P, i, a0 + i, S.fl[i], Q, Vs, F, U, Up, Wc, check, write_u, write_prev, seed, du2, dv2);
            }
        } else {
            fill_ghosts(S, L.gd, L.gd + L.gp, pb, pb ? P1b : P1a, pb ? P2b : P2a, Wc, nt);
            __syncthreads();
            each([&](int a) {
                primal_gh(P, a - a0, a, S.fl[a - a0], Q, Vs, F, U, Up, Wc, check, write_u, write_prev, seed, du2, dv2);
            });
        }
        if (ckpt && l % ckpt_every == 0 && l < iters) {
            __syncthreads();   // boundary pixels were updated by other threads
            save(l / ckpt_every);
        }
        if (check) {
            float x = du2, y = dv2;
            block_sum2f<NT>(x, y, reinterpret_cast<float*>(s_red));
            if (tid == 0) {
                partials[2 * blockIdx.x] = x;
                partials[2 * blockIdx.x + 1] = y;
            }
        }
        if (!grid_sync(h, nblocks, gen)) return false;
        if (check && blockIdx.x == 0) {
            // Section 4 stopping test: fixed-order FP64 sum of the block partials,
            // squared norms against tol^2 (square roots taken once, for the stats)
            double sx = 0.0, sy = 0.0;
            if (tid < 32) sum_partials_warp0(partials, (int)nblocks, sx, sy);
            if (tid == 0) {
                h->du2 = sx;
                h->dv2 = sy;
                h->last_check = l;
                if (tol > 0.0 && fmax(sx, sy) <= tol * tol) {
                    h->iters_done = l;
                    __threadfence();
                    h->done = 1;
                }
            }
            __syncthreads();
        }
    }
    *fb = pb;
    return true;
}

// ---- one grid barrier per iteration
//
// The two-phase iteration needs its second grid barrier only because the
// primal step of x reads p' at x - e1 and x - e2, which another block may
// compute.  When every block's state fits with it, a block also runs the dual
// step of its ring -- the pixels other blocks own directly above or left of
// its own -- from the same inputs and with the same arithmetic and rounding
// as their owners, so its primal step follows its dual step after a block
// barrier, and one grid barrier ends the iteration.  What the dual steps read
// that the block does not compute (w below / right, or p at the diagonal
// neighbour, of its pixels and of its ring, and w of the ring) are ghost
// words refilled at the start of each iteration from the previous iterate,
// whose p and w the global arrays hold in ping-pong buffers, written for the
// pixels some other block reads (marked once, before the iterations).  p' of
// the ring stays in the block's own words, so the ring's p is read once.
// The iterates are bit-identical to the two-barrier ones.
struct H1Layout {
    int n, r, nE;          // own pixels, ring pixels, n + r
    int ns1, ns2, nsw;     // region sizes (words) of P1, P2 (per buffer) and W: [own | ring | zero | ghosts]
    int p1, p2, w, v;      // word offsets of the regions
    int ng, nbd;           // ghost words refilled per iteration; late own pixels
    size_t off16, offfl, offr1, offgs, offgd, offbd, bytes;   // byte offsets of the tables
};

template <typename T>
struct H1State {
    float* sm;             // the shared-memory words
    const uint16_t* off;   // [D: nE][R: nE][UP: n][LEFT: n] word offsets (p words: buffer 0)
    const uint8_t* fl;     // [nE]
    const int32_t* r1;     // [r] compact index of each ring pixel
    const int32_t* gsrc;   // [ng] compact index of each ghost's pixel
    const uint16_t* gdst;  // [ng] word offset of each ghost (p words: buffer 0)
    const uint16_t* bd;    // [nbd] late own pixels (kFlLate)
    H1Layout L;
    __device__ __forceinline__ T* v() const { return reinterpret_cast<T*>(sm + L.v); }
};

// The iterations; returns false when a barrier timed out, else the final
// iterate's count in *lf (its p is in buffer lf & 1).
//
// The grid barrier is split: a block arrives once its primal step is done
// and, unless the iteration ends with a stopping test, runs the next
// iteration's dual steps of its first UNROLL x NT "interior" pixels -- those
// that read no ghost word and that no other block reads, so they touch only
// the block's own words -- before it waits; the rest of the interior runs
// while the ghost loads are in flight, and the "late" pixels (that read a
// ghost or that another block reads: their global p must not change before
// every block has read it) and the ring after the ghost words are stored.
template <typename T, int NT, int UNROLL>
__device__ __forceinline__ bool compact_iterations_h1(const IterParams& P, const H1State<T>& S, int a0, int a1,
                                                      int iters, int check_every, double tol, int64_t stride,
                                                      T* P1a, T* P1b, T* P2a, T* P2b, const float* F,
                                                      float* U, float* Up, float* Wc, float* Wc2,
                                                      double* partials, WsHeader* h, float* ckpt, int ckpt_every,
                                                      double* s_red, unsigned& gen, int* lf) {
    const unsigned nblocks = gridDim.x;
    const int tid = threadIdx.x, nt = NT;
    const H1Layout& L = S.L;
    int pb = 0, chk = 0;
    auto each = [&](auto&& op) {
        int a = a0 + tid;
        for (; a + (UNROLL - 1) * nt < a1; a += UNROLL * nt) {
#pragma unroll
            for (int k = 0; k < UNROLL; ++k) op(a + k * nt);
        }
        for (; a < a1; a += nt) op(a);
    };
    auto save = [&](int m) {
        float* c = ckpt + (int64_t)m * 3 * stride;
        const T* V = S.v();
        for (int a = a0 + tid; a < a1; a += nt) {
            const int i = a - a0;
            c[a] = S.sm[L.p1 + pb * L.ns1 + i];
            c[stride + a] = S.sm[L.p2 + pb * L.ns2 + i];
            c[2 * stride + a] = to_f(V[i]) + Store<T>::vbias;
        }
    };
    // the dual-step view of iteration it (p of buffer b)
    auto dual_view = [&](int b) {
        DualView D;
        D.p1 = S.sm + L.p1 + b * L.ns1;
        D.p2 = S.sm + L.p2 + b * L.ns2;
        D.w = S.sm + L.w;
        D.q1 = S.sm + L.p1 + (1 - b) * L.ns1;
        D.q2 = S.sm + L.p2 + (1 - b) * L.ns2;
        D.sm = S.sm;
        D.sh1 = b * L.ns1;
        D.sh2 = b * L.ns2;
        D.od = S.off;
        D.orr = S.off + L.nE;
        return D;
    };
    auto dual_seed = [](int it) { return mix32(0x51ed270bu ^ (uint32_t)(it * 131)); };
    // dual steps of the interior pixels among own pixels [i0, i1) (no ghost
    // read, no global store)
    const int iA = min(L.n, UNROLL * NT);
    auto interior = [&](const DualView& D, uint32_t seed, int i0, int i1) {
        int a = a0 + i0 + tid;
        const int ae = a0 + i1;
        auto op = [&](int b) {
            const uint8_t f = S.fl[b - a0];
            if (!(f & kFlLate)) dual_gh<T>(P, b - a0, b, f, D, nullptr, nullptr, seed);
        };
        for (; a + (UNROLL - 1) * nt < ae; a += UNROLL * nt) {
#pragma unroll
            for (int k = 0; k < UNROLL; ++k) op(a + k * nt);
        }
        for (; a < ae; a += nt) op(a);
    };
    if (ckpt) save(0);
    const int C = check_every;
    *lf = iters;
    bool early = false;   // this iteration's first interior pixels ran before the barrier
    // theta lambda f of the thread's pixels (at most kFSlots), in registers
    // for the whole solve: the primal step then reads no global memory
    constexpr int kFSlots = 6;
    const bool fslots = L.n <= kFSlots * NT;
    float fr[kFSlots];
    auto load_f = [&]() {
#pragma unroll
        for (int k = 0; k < kFSlots; ++k) {
            const int a = a0 + tid + k * nt;
            fr[k] = (fslots && a < a1) ? __ldg(F + a) : 0.f;
        }
    };
    load_f();
    for (int it = 0; it < iters; ++it) {
        const int l = it + 1;
        const float* Wi = (it & 1) ? Wc2 : Wc;   // w of iterate it
        float* Wo = (it & 1) ? Wc : Wc2;         // w of iterate l (pixels other blocks read)
        {
            const uint32_t seed = dual_seed(it);
            T* o1 = pb ? P1a : P1b;
            T* o2 = pb ? P2a : P2b;
            const T* i1 = pb ? P1b : P1a;
            const T* i2 = pb ? P2b : P2a;
            const DualView D = dual_view(pb);
            if (early && !grid_wait(h, nblocks, gen)) return false;
            // ghosts in flight (kGhostRegs per thread) while interior pixels update
            float x[kGhostRegs];
#pragma unroll
            for (int j = 0; j < kGhostRegs; ++j) {
                const int g = tid + j * nt;
                x[j] = 0.f;
                if (g < L.ng) {
                    const int src = S.gsrc[g], dst = S.gdst[g];
                    x[j] = dst >= L.w ? ldw(Wi + src) : dst >= L.p2 ? Store<T>::ldc(i2, src) : Store<T>::ldc(i1, src);
                }
            }
            interior(D, seed, early ? iA : 0, L.n);
#pragma unroll
            for (int j = 0; j < kGhostRegs; ++j) {
                const int g = tid + j * nt;
                if (g < L.ng) {
                    const int dst = S.gdst[g];
                    S.sm[dst >= L.w ? dst : dst >= L.p2 ? dst + D.sh2 : dst + D.sh1] = x[j];
                }
            }
            __syncthreads();
            // late own pixels, then the ring
            for (int e = tid; e < L.nbd + L.r; e += nt) {
                const bool own = e < L.nbd;
                const int i = own ? S.bd[e] : L.n + (e - L.nbd);
                const int a = own ? a0 + i : S.r1[e - L.nbd];
                dual_gh(P, i, a, S.fl[i], D, o1, o2, seed);
            }
            pb ^= 1;
            __syncthreads();
        }
        const bool check = (l % C == 0) || l == iters;
        const bool write_u = check;   // the output u and the stopped iterate
        const bool write_prev = l < iters && ((l + 1) % C == 0 || l + 1 == iters);
        const uint32_t seed = mix32(0x2545f491u ^ (uint32_t)it);
        float du2 = 0.f, dv2 = 0.f;
        PrimalView Q;
        Q.q1 = S.sm + L.p1 + pb * L.ns1;
        Q.q2 = S.sm + L.p2 + pb * L.ns2;
        Q.n1 = S.sm + pb * L.ns1;
        Q.n2 = S.sm + pb * L.ns2;
        Q.w = S.sm + L.w;
        Q.ou = S.off + 2 * L.nE;
        Q.ol = S.off + 2 * L.nE + L.n;
        T* Vs = S.v();
        if (fslots) {
            if (!check && !write_prev) {
#pragma unroll
                for (int k = 0; k < kFSlots; ++k) {
                    const int a = a0 + tid + k * nt;
                    if (a < a1)
                        primal_gh_f(P, a - a0, a, S.fl[a - a0], Q, Vs, fr[k], U, Up, Wo, false, false, false, seed,
                                    du2, dv2);
                }
            } else {
#pragma unroll
                for (int k = 0; k < kFSlots; ++k) {
                    const int a = a0 + tid + k * nt;
                    if (a < a1)
                        primal_gh_f(P, a - a0, a, S.fl[a - a0], Q, Vs, fr[k], U, Up, Wo, check, write_u, write_prev,
                                    seed, du2, dv2);
                }
            }
        } else if (!check && !write_prev)
            each([&](int a) {
                primal_gh(P, a - a0, a, S.fl[a - a0], Q, Vs, F, U, Up, Wo, false, false, false, seed, du2, dv2);
            });
        else
            each([&](int a) {
                primal_gh(P, a - a0, a, S.fl[a - a0], Q, Vs, F, U, Up, Wo, check, write_u, write_prev, seed, du2,
                          dv2);
            });
        if (ckpt && l % ckpt_every == 0 && l < iters) save(l / ckpt_every);   // own pixels, same threads
        // stopping-test partials, double-buffered by check so that a fast
        // block cannot overwrite those a slow block is still summing
        double* part = partials + 2 * (int64_t)nblocks * (chk & 1);
        if (check) {
            float x = du2, y = dv2;
            block_sum2f<NT>(x, y, reinterpret_cast<float*>(s_red));
            if (tid == 0) {
                part[2 * blockIdx.x] = x;
                part[2 * blockIdx.x + 1] = y;
            }
        }
        grid_arrive(h, gen);
        early = !check;   // (the last iteration is a check)
        if (early) {
            // the next iteration's first interior pixels, on the block's own words
            interior(dual_view(pb), dual_seed(l), 0, iA);
            continue;
        }
        if (!grid_wait(h, nblocks, gen)) return false;
        // Section 4 stopping test: with a tolerance every block sums the
        // block partials in the same fixed order, so all stop after the same
        // iteration (squared norms against tol^2); block 0 records the norms
        if (tol > 0.0 || blockIdx.x == 0) {
            if (tid < 32) {
                double sx, sy;
                sum_partials_warp0(part, (int)nblocks, sx, sy);
                if (tid == 0) {
                    const bool stop = tol > 0.0 && fmax(sx, sy) <= tol * tol;
                    s_red[0] = stop ? 1.0 : 0.0;
                    if (blockIdx.x == 0) {
                        h->du2 = sx;
                        h->dv2 = sy;
                        h->last_check = l;
                        if (stop) {
                            h->iters_done = l;
                            h->done = 1;
                        }
                    }
                }
            }
            __syncthreads();
            const bool stop = s_red[0] != 0.0;
            __syncthreads();
            if (stop) {
                *lf = l;
                return true;
            }
        }
        ++chk;
    }
    return true;
}

// Sets up and runs the one-barrier iteration when every block's state fits
// (a grid-wide vote; `votes`, the vote count seen so far, runs on across the
// waves of a batch).  Returns 1 when it ran the solve, 0 when some block does
// not fit (nothing changed; the caller takes the two-barrier paths), -1 when
// a barrier timed out.
template <typename T, int NT, int UNROLL>
__device__ __forceinline__ int compact_solve_h1(
    const IterParams& P, int iters, int check_every, double tol, int a0, int a1,
    const int32_t* __restrict__ nb, int64_t stride, T* P1a, T* P1b, T* P2a, T* P2b, T* V,
    const float* __restrict__ F, float* U, float* Up, float* Wc, float* Wc2, double* partials, WsHeader* h,
    float* ckpt, int ckpt_every, unsigned& gen, unsigned& votes, double* s_red, unsigned char* c_smem) {
    const unsigned nblocks = gridDim.x;
    const int tid = threadIdx.x, nt = NT;
    const int nown = max(a1 - a0, 0);
    auto other = [&](int m) { return m >= 0 && (m < a0 || m >= a1); };
    // counts: [0] ring pixels, [1..3] ghost words of the W / P1 / P2 areas,
    // [4] ghosts read by own pixels' dual steps; then running slots
    __shared__ int s_h[8];
    if (tid < 8) s_h[tid] = 0;
    __syncthreads();
    {
        int r = 0, gw = 0, g1 = 0, g2 = 0, go = 0;
        for (int i = tid; i < nown; i += nt) {
            const int a = a0 + i;
#pragma unroll
            for (int k = GK_D; k <= GK_R; ++k) {
                int reg;
                const int m = gk_src(nb, stride, a, k, reg);
                if (other(m)) {
                    ++go;
                    gw += reg == 0; g1 += reg == 1; g2 += reg == 2;
                }
            }
#pragma unroll
            for (int k = GK_UP; k <= GK_LEFT; ++k) {
                int reg;
                const int y = gk_src(nb, stride, a, k, reg);
                if (!other(y)) continue;
                ++r;
#pragma unroll
                for (int k2 = GK_D; k2 <= GK_R; ++k2) {
                    int reg2;
                    const int m = gk_src(nb, stride, y, k2, reg2);
                    if (other(m)) { gw += reg2 == 0; g1 += reg2 == 1; g2 += reg2 == 2; }
                }
            }
        }
        if (r) atomicAdd(&s_h[0], r);
        if (gw) atomicAdd(&s_h[1], gw);
        if (g1) atomicAdd(&s_h[2], g1);
        if (g2) atomicAdd(&s_h[3], g2);
        if (go) atomicAdd(&s_h[4], go);
    }
    __syncthreads();
    H1Layout L{};
    L.n = nown;
    L.r = s_h[0];
    L.nE = nown + L.r;
    const int gwx = s_h[1], g1x = s_h[2], g2x = s_h[3];
    L.ng = gwx + g1x + g2x + L.r;   // plus w of every ring pixel
    L.ns1 = L.nE + 1 + g1x;
    L.ns2 = L.nE + 1 + g2x;
    L.nsw = L.nE + 1 + gwx;
    L.p1 = 0;
    L.p2 = 2 * L.ns1;
    L.w = L.p2 + 2 * L.ns2;
    L.v = L.w + L.nsw;
    const int words = L.v + (int)((sizeof(T) * nown + 3) / 4);
    L.off16 = (size_t)4 * words;
    L.offfl = L.off16 + (size_t)2 * (2 * L.nE + 2 * nown);
    L.offr1 = (L.offfl + L.nE + 3) & ~(size_t)3;
    L.offgs = L.offr1 + (size_t)4 * L.r;
    L.offgd = L.offgs + (size_t)4 * L.ng;
    L.offbd = L.offgd + (size_t)2 * L.ng;
    L.bytes = L.offbd + (size_t)2 * nown;
    const bool fits = L.bytes <= compact_smem(NT) && words < 65536 && L.ng <= kGhostRegs * NT;
    // the vote: every block adds 1 when it does not fit
    __shared__ unsigned s_vote;
    if (tid == 0 && !fits) atomicAdd(&h->h1_vote, 1u);
    if (!grid_sync(h, nblocks, gen)) return -1;
    if (tid == 0) s_vote = *(volatile unsigned*)&h->h1_vote;
    __syncthreads();
    const bool all_fit = s_vote == votes;
    votes = s_vote;
    __syncthreads();   // s_vote and s_h are read by every thread before they change
    if (!all_fit) return 0;

    // export marks (1 = another block reads the pixel), cleared before any block marks
    unsigned* mark = reinterpret_cast<unsigned*>(Wc2);
    for (int i = tid; i < nown; i += nt) mark[a0 + i] = 0u;
    float* sm = reinterpret_cast<float*>(c_smem);
    uint16_t* off = reinterpret_cast<uint16_t*>(c_smem + L.off16);
    uint8_t* flg = reinterpret_cast<uint8_t*>(c_smem + L.offfl);
    int32_t* r1 = reinterpret_cast<int32_t*>(c_smem + L.offr1);
    int32_t* gsrc = reinterpret_cast<int32_t*>(c_smem + L.offgs);
    uint16_t* gdst = reinterpret_cast<uint16_t*>(c_smem + L.offgd);
    uint16_t* lbd = reinterpret_cast<uint16_t*>(c_smem + L.offbd);
    if (tid < 8) s_h[tid] = 0;   // [0] ring slots, [1..3] area words, [4] ghost slots
    if (tid == 0) {
        sm[L.p1 + L.nE] = 0.f; sm[L.p1 + L.ns1 + L.nE] = 0.f;
        sm[L.p2 + L.nE] = 0.f; sm[L.p2 + L.ns2 + L.nE] = 0.f;
        sm[L.w + L.nE] = 0.f;
    }
    __syncthreads();
    // the offset of a D / R read of pixel a (a ghost word when another block owns its source)
    auto dr_off = [&](int a, int k, bool& ghost) {
        int reg;
        const int m = gk_src(nb, stride, a, k, reg);
        const int base = reg == 0 ? L.w : reg == 1 ? L.p1 : L.p2;
        ghost = false;
        if (m >= a0 && m < a1) return base + (m - a0);
        if (m < 0) return base + L.nE;   // the zero word
        ghost = true;
        const int gi = atomicAdd(&s_h[1 + reg], 1);
        const int o = base + L.nE + 1 + gi;
        const int slot = atomicAdd(&s_h[4], 1);
        gsrc[slot] = m;
        gdst[slot] = (uint16_t)o;
        return o;
    };
    T* Vs = reinterpret_cast<T*>(sm + L.v);
    for (int i = tid; i < nown; i += nt) {
        const int a = a0 + i;
        bool gd = false, g;
        off[i] = (uint16_t)dr_off(a, GK_D, g);
        gd |= g;
        off[L.nE + i] = (uint16_t)dr_off(a, GK_R, g);
        gd |= g;
        flg[i] = (uint8_t)(gk_codes(nb, stride, a) | (gd ? kFlDualGhost : 0));
#pragma unroll
        for (int k = GK_UP; k <= GK_LEFT; ++k) {
            int reg;
            const int y = gk_src(nb, stride, a, k, reg);
            const int base = k == GK_UP ? L.p1 : L.p2;
            int o;
            if (y >= a0 && y < a1) {
                o = base + (y - a0);
            } else if (y < 0) {
                o = base + L.nE;
            } else {   // a ring pixel: its own words, p read once, w a ghost
                const int j = atomicAdd(&s_h[0], 1);
                const int e = nown + j;
                o = base + e;
                r1[j] = y;
                off[e] = (uint16_t)dr_off(y, GK_D, g);
                off[L.nE + e] = (uint16_t)dr_off(y, GK_R, g);
                flg[e] = gk_codes(nb, stride, y);
                sm[L.p1 + e] = Store<T>::ldc(P1a, y);
                sm[L.p2 + e] = Store<T>::ldc(P2a, y);
                const int slot = atomicAdd(&s_h[4], 1);
                gsrc[slot] = y;
                gdst[slot] = (uint16_t)(L.w + e);
            }
            off[2 * L.nE + (k - GK_UP) * nown + i] = (uint16_t)o;
        }
        sm[L.p1 + i] = Store<T>::ldc(P1a, a);
        sm[L.p2 + i] = Store<T>::ldc(P2a, a);
        sm[L.w + i] = ldw(Wc + a);
        Vs[i] = V[a];
    }
    if (!grid_sync(h, nblocks, gen)) return -1;   // every mark cleared, every table built
    for (int g = tid; g < L.ng; g += nt) mark[gsrc[g]] = 1u;
    if (!grid_sync(h, nblocks, gen)) return -1;   // every mark set
    for (int i = tid; i < nown; i += nt)
        if (__ldcg(mark + a0 + i)) flg[i] |= kFlExport;
    __syncthreads();
    // stable list of the late own pixels
    __shared__ int s_nbd;
    if (tid < 32) {
        int cd = 0;
        for (int b = 0; b < nown; b += 32) {
            const int i = b + tid;
            const unsigned f = i < nown ? flg[i] : 0u;
            const unsigned md = __ballot_sync(0xffffffffu, f & kFlLate);
            if (f & kFlLate) lbd[cd + __popc(md & lanemask_lt(tid))] = (uint16_t)i;
            cd += __popc(md);
        }
        if (tid == 0) {
            s_nbd = cd;
            atomicAdd(&h->n_smem_blocks, 1);
            atomicAdd(&h->n_h1_blocks, 1);
        }
    }
    __syncthreads();
    L.nbd = s_nbd;
    const H1State<T> S{sm, off, flg, r1, gsrc, gdst, lbd, L};
    int lf = iters;
    if (!compact_iterations_h1<T, NT, UNROLL>(P, S, a0, a1, iters, check_every, tol, stride, P1a, P1b, P2a, P2b,
                                              F, U, Up, Wc, Wc2, partials, h, ckpt, ckpt_every, s_red, gen, &lf))
        return -1;
    __syncthreads();
    // the final iterate: v, and p of every own pixel
    const int fb = lf & 1;
    T* G1 = fb ? P1b : P1a;
    T* G2 = fb ? P2b : P2a;
    for (int i = tid; i < nown; i += nt) {
        V[a0 + i] = Vs[i];
        Store<T>::st(G1, a0 + i, sm[L.p1 + fb * L.ns1 + i]);
        Store<T>::st(G2, a0 + i, sm[L.p2 + fb * L.ns2 + i]);
    }
    return 1;
}

// Which of the two persistent compact kernels runs a solve (both are
// launched; the other returns at once).  The shared-memory kernel (two
// 512-thread blocks per SM, grid1 blocks) unless even its table rows would
// not fit in shared memory -- then every block would take the global-memory
// path, and k_solve_compact_wide, the same path at four 512-thread blocks
// per SM (twice the warps to hide the latency of the table and neighbour
// loads), runs instead.
template <typename T>
__device__ __forceinline__ bool compact_wide(int n, int grid1) {
    const int64_t per1 = ((int64_t)n + grid1 - 1) / grid1;
    return (size_t)per1 * (4 * NB_UUR + sizeof(T)) > compact_smem(kCompactThreads);
}

// All iterations of the compact solve over the RD pixels [w0, w0 + n) (the
// whole problem, or one wave of whole images of a batch); false when a grid
// barrier timed out.  gen: barriers passed so far in the launch.
template <typename T, int NT, int UNROLL>
__device__ __forceinline__ bool compact_solve_range(
    const IterParams& P, int iters, int n_inner, int check_every, double tol, int warm, int w0, int n,
    const int32_t* __restrict__ nb, int64_t stride, T* P1a, T* P1b, T* P2a, T* P2b, T* V,
    const float* __restrict__ F, float* U, float* Up, float* Wc, float* Wc2, double* partials, WsHeader* h,
    float* ckpt, int ckpt_every, unsigned& gen, unsigned& votes, double* s_red, unsigned char* c_smem) {
    const unsigned nblocks = gridDim.x;
    const int per = (n + (int)nblocks - 1) / (int)nblocks;
    const int a0 = w0 + (int)blockIdx.x * per, a1 = min(w0 + n, a0 + per);
    const int tid = threadIdx.x, nt = NT;
    // the fused iteration (eight table rows) up to kFuseMaxPerBlock pixels
    // per block; the other paths read six
    const int fuse = n_inner == 1 && per <= kFuseMaxPerBlock;
    const int rows = fuse ? NB_COUNT : NB_UUR;
    if (n_inner == 1 && !fuse) {
        // w of the warm-start iterate first, from the global arrays (every
        // path below then starts from it)
        if (warm) {
            float d0 = 0.f, d1 = 0.f;
            const Own<T, false> O{nb, stride, V, F, 0};
            for (int a = a0 + tid; a < a1; a += nt)
                primal_one(P, a, O, P1a, P2a, U, Up, Wc, true, false, false, false, 0u, d0, d1);
            warm = 0;   // the vote's barrier below orders these writes before any read
        }
        const int h1 = compact_solve_h1<T, NT, UNROLL>(P, iters, check_every, tol, a0, a1, nb, stride, P1a, P1b,
                                                      P2a, P2b, V, F, U, Up, Wc, Wc2, partials, h, ckpt,
                                                      ckpt_every, gen, votes, s_red, c_smem);
        if (h1 != 0) return h1 > 0;
        // shared-memory-resident state if this block's pixels and its ghosts
        // fit (decided per block: both paths keep the global arrays that
        // other blocks read current and pass the same barriers)
        __shared__ int s_cnt[8];   // ghosts per kind, then running slots; ghosts per region
        if (tid < 8) s_cnt[tid] = 0;
        __syncthreads();
        const int nown = max(a1 - a0, 0);
        {
            int c[GK_KINDS] = {0, 0, 0, 0}, c_w = 0, c_p1 = 0, c_p2 = 0;
            for (int i = tid; i < nown; i += nt)
#pragma unroll
                for (int k = 0; k < GK_KINDS; ++k) {
                    int reg;
                    const int m = gk_src(nb, stride, a0 + i, k, reg);
                    const int g = (m >= 0 && (m < a0 || m >= a1)) ? 1 : 0;
                    c[k] += g;
                    c_w += reg == 0 ? g : 0;
                    c_p1 += reg == 1 ? g : 0;
                    c_p2 += reg == 2 ? g : 0;
                }
#pragma unroll
            for (int k = 0; k < GK_KINDS; ++k)
                if (c[k]) atomicAdd(&s_cnt[k], c[k]);
            if (c_w) atomicAdd(&s_cnt[4], c_w);
            if (c_p1) atomicAdd(&s_cnt[5], c_p1);
            if (c_p2) atomicAdd(&s_cnt[6], c_p2);
        }
        __syncthreads();
        GhostLayout L{};
        L.n = nown;
        const int g_w = s_cnt[4], g_p1 = s_cnt[5], g_p2 = s_cnt[6];
        L.gd = s_cnt[GK_D] + s_cnt[GK_R];
        L.gp = s_cnt[GK_UP] + s_cnt[GK_LEFT];
        L.ns1 = nown + 1 + g_p1;
        L.ns2 = nown + 1 + g_p2;
        L.nsw = nown + 1 + g_w;
        L.p1 = 0;
        L.p2 = 2 * L.ns1;
        L.w = L.p2 + 2 * L.ns2;
        L.v = L.w + L.nsw;
        const int words = L.v + (int)((sizeof(T) * nown + 3) / 4);
        L.off16 = (size_t)4 * words;
        L.offfl = L.off16 + (size_t)2 * GK_KINDS * nown;
        L.offgs = (L.offfl + nown + 3) & ~(size_t)3;
        L.offgd = L.offgs + (size_t)4 * (L.gd + L.gp);
        // pixels whose dual / primal step reads a ghost: at most one per ghost
        L.offbd = L.offgd + (size_t)2 * (L.gd + L.gp);
        L.offbp = L.offbd + (size_t)2 * L.gd;
        L.bytes = L.offbp + (size_t)2 * L.gp;
        __syncthreads();   // every thread has read the counts before they become slot cursors
        if (L.bytes <= compact_smem(NT) && words < 65536) {
            float* sm = reinterpret_cast<float*>(c_smem);
            uint16_t* off = reinterpret_cast<uint16_t*>(c_smem + L.off16);
            uint8_t* flg = reinterpret_cast<uint8_t*>(c_smem + L.offfl);
            int32_t* gsrc = reinterpret_cast<int32_t*>(c_smem + L.offgs);
            uint16_t* gdst = reinterpret_cast<uint16_t*>(c_smem + L.offgd);
            uint16_t* lbd = reinterpret_cast<uint16_t*>(c_smem + L.offbd);
            uint16_t* lbp = reinterpret_cast<uint16_t*>(c_smem + L.offbp);
            if (warm) {   // w of the warm-start iterate, from the global arrays (as the other path)
                float d0 = 0.f, d1 = 0.f;
                const Own<T, false> O{nb, stride, V, F, 0};
                for (int a = a0 + tid; a < a1; a += nt)
                    primal_one(P, a, O, P1a, P2a, U, Up, Wc, true, false, false, false, 0u, d0, d1);
                if (!grid_sync(h, nblocks, gen)) return false;
            }
            // ghost slots: dual kinds first (D, R), then primal (up, left)
            if (tid == 0) {
                int acc = 0;
                for (int k = 0; k < GK_KINDS; ++k) { const int c = s_cnt[k]; s_cnt[k] = acc; acc += c; }
            }
            // zero words
            if (tid == 0) {
                sm[L.p1 + nown] = 0.f; sm[L.p1 + L.ns1 + nown] = 0.f;
                sm[L.p2 + nown] = 0.f; sm[L.p2 + L.ns2 + nown] = 0.f;
                sm[L.w + nown] = 0.f;
            }
            __syncthreads();
            // per-kind region base (buffer 0) and running ghost index within the region
            __shared__ int s_reg[3];   // ghosts placed so far in the W, P1, P2 ghost areas
            if (tid < 3) s_reg[tid] = 0;
            __syncthreads();
            T* Vs = reinterpret_cast<T*>(sm + L.v);
            for (int i = tid; i < nown; i += nt) {
                const int a = a0 + i;
                uint8_t f = 0;
                bool exported = false, gdual = false, gprimal = false;
                // other blocks read this pixel if one of its neighbours is theirs
                {
                    const int sl[6] = {NB_UP, NB_LEFT, NB_DOWN, NB_RIGHT, NB_DOWNLEFT, NB_UPRIGHT};
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        const int m = __ldg(nb + sl[k] * stride + a);
                        if (m >= 0 && (m < a0 || m >= a1)) exported = true;
                    }
                }
#pragma unroll
                for (int k = 0; k < GK_KINDS; ++k) {
                    int reg;
                    const int m = gk_src(nb, stride, a, k, reg);
                    const int base = reg == 0 ? L.w : reg == 1 ? L.p1 : L.p2;
                    int o;
                    if (m >= a0 && m < a1) {
                        o = base + (m - a0);
                    } else if (m >= 0) {
                        if (k < GK_UP) gdual = true; else gprimal = true;
                        const int slot = atomicAdd(&s_cnt[k], 1);          // position in the ghost lists
                        const int gi = atomicAdd(&s_reg[reg], 1);          // word in the region's ghost area
                        o = base + nown + 1 + gi;
                        gsrc[slot] = m;
                        gdst[slot] = (uint16_t)o;
                    } else {
                        o = base + nown;                                   // the zero word
                    }
                    off[k * nown + i] = (uint16_t)o;
                }
                f |= gk_codes(nb, stride, a);
                flg[i] = (uint8_t)(f | (exported ? kFlExport : 0) | (gdual ? kFlDualGhost : 0) |
                                   (gprimal ? kFlPrimalGhost : 0));
                sm[L.p1 + i] = Store<T>::ldc(P1a, a);
                sm[L.p2 + i] = Store<T>::ldc(P2a, a);
                sm[L.w + i] = ldw(Wc + a);
                Vs[i] = V[a];
            }
            __syncthreads();
            // stable lists of the pixels that read ghosts
            __shared__ int s_nb[2];
            if (tid < 32) {
                int cd = 0, cp = 0;
                for (int b = 0; b < nown; b += 32) {
                    const int i = b + tid;
                    const unsigned f = i < nown ? flg[i] : 0u;
                    const unsigned md = __ballot_sync(0xffffffffu, f & kFlDualGhost);
                    const unsigned mp = __ballot_sync(0xffffffffu, f & kFlPrimalGhost);
                    if (f & kFlDualGhost) lbd[cd + __popc(md & lanemask_lt(tid))] = (uint16_t)i;
                    if (f & kFlPrimalGhost) lbp[cp + __popc(mp & lanemask_lt(tid))] = (uint16_t)i;
                    cd += __popc(md);
                    cp += __popc(mp);
                }
                if (tid == 0) {
                    s_nb[0] = cd;
                    s_nb[1] = cp;
                    atomicAdd(&h->n_smem_blocks, 1);
                }
            }
            __syncthreads();
            L.nbd = s_nb[0];
            L.nbp = s_nb[1];
            const GhostState<T> S{sm, off, flg, gsrc, gdst, lbd, lbp, L};
            int fb = 0, lf = iters;
            // the barrier generation continues from the warm-start barrier
            if (!compact_iterations_gh<T, NT, UNROLL>(P, S, a0, a1, iters, check_every, tol, stride, P1a, P1b,
                                                       P2a, P2b, F, U, Up, Wc, partials, h, ckpt, ckpt_every,
                                                       s_red, gen, &fb, &lf))
                return false;
            __syncthreads();
            // the final iterate: v, and p of every own pixel (only exported
            // pixels were kept current in the global arrays)
            T* G1 = (lf & 1) ? P1b : P1a;
            T* G2 = (lf & 1) ? P2b : P2a;
            for (int i = tid; i < nown; i += nt) {
                V[a0 + i] = Vs[i];
                Store<T>::st(G1, a0 + i, sm[L.p1 + fb * L.ns1 + i]);
                Store<T>::st(G2, a0 + i, sm[L.p2 + fb * L.ns2 + i]);
            }
            return true;
        }
    }
    if ((size_t)per * (4 * rows + sizeof(T)) <= compact_smem(NT)) {   // the same in every block
        int32_t* nb_s = reinterpret_cast<int32_t*>(c_smem);
        T* v_s = reinterpret_cast<T*>(c_smem + (size_t)4 * rows * per);
        for (int i = tid; i < a1 - a0; i += nt) {
            for (int k = 0; k < rows; ++k) nb_s[k * per + i] = __ldg(nb + k * stride + a0 + i);
            v_s[i] = V[a0 + i];
        }
        __syncthreads();
        const Own<T, true> O{nb_s, per, v_s, F, a0};
        if (!compact_iterations<T, true, NT, UNROLL>(P, O, a0, a1, iters, n_inner, check_every, tol, warm,
                                                     stride, P1a, P1b, P2a, P2b, U, Up, Wc, Wc2, partials, h,
                                                     ckpt, ckpt_every, s_red, fuse, gen))
            return false;
        for (int i = tid; i < a1 - a0; i += nt) V[a0 + i] = v_s[i];
        return true;
    }
    const Own<T, false> O{nb, stride, V, F, 0};
    return compact_iterations<T, false, NT, UNROLL>(P, O, a0, a1, iters, n_inner, check_every, tol, warm,
                                                    stride, P1a, P1b, P2a, P2b, U, Up, Wc, Wc2, partials, h,
                                                    ckpt, ckpt_every, s_red, fuse, gen);
}

// Batches solved in waves: with a fixed iteration count (tol <= 0, so no
// test decides anything across images) and n_inner = 1, a batch larger than
// the shared-memory paths hold is solved as consecutive waves of whole
// images, each at most kWavePerBlock pixels per block (images are
// independent problems, so their iterates do not depend on the grouping);
// stats then hold the norms of the last test summed over the waves, i.e.
// over the whole batch, as without waves.
constexpr int kWavePerBlock = 3000;

inline bool compact_waves(int nimg, double tol, int n_inner, const float* ckpt) {
    return nimg > 1 && !(tol > 0.0) && n_inner == 1 && ckpt == nullptr;
}

// WAVES: the batch's images in waves (see above); otherwise one range, and
// this kernel returns at once when k_solve_compact_wide is the one to run.
template <typename T, int NT, int UNROLL, bool WAVES>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_solve_compact(IterParams P, int iters, int n_inner, int check_every, double tol, int warm,
                const int32_t* __restrict__ counts, const int32_t* __restrict__ nb, int64_t stride,
                T* P1a, T* P1b, T* P2a, T* P2b, T* V, const float* __restrict__ F, float* U,
                float* Up, float* Wc, float* Wc2, double* partials, WsHeader* h, float* ckpt,
                int ckpt_every, int grid1, const int32_t* __restrict__ base, int nimg) {
    __shared__ double s_red[66];   // block_sum2f (as floats), stop flag
    extern __shared__ __align__(16) unsigned char c_smem[];
    // set before the launch (capacity overflow): the same for every block
    if (*(volatile int*)&h->done) return;
    const int n = counts[1];
    unsigned gen = 0u, votes = 0u;
    if (!WAVES) {
        if (compact_wide<T>(n, grid1)) return;
        compact_solve_range<T, NT, UNROLL>(P, iters, n_inner, check_every, tol, warm, 0, n, nb, stride, P1a, P1b,
                                           P2a, P2b, V, F, U, Up, Wc, Wc2, partials, h, ckpt, ckpt_every, gen,
                                           votes, s_red, c_smem);
        return;
    }
    const int cap = (int)gridDim.x * kWavePerBlock;
    double su = 0.0, sv = 0.0;   // block 0, thread 0: the last test's sums over the waves
    for (int k0 = 0; k0 < nimg;) {
        int k1 = k0 + 1;
        while (k1 < nimg && __ldg(base + k1 + 1) - __ldg(base + k0) <= cap) ++k1;
        const int w0 = __ldg(base + k0), wn = __ldg(base + k1) - w0;
        k0 = k1;
        if (wn == 0) continue;
        if (!compact_solve_range<T, NT, UNROLL>(P, iters, n_inner, check_every, tol, warm, w0, wn, nb, stride,
                                                P1a, P1b, P2a, P2b, V, F, U, Up, Wc, Wc2, partials, h, ckpt,
                                                ckpt_every, gen, votes, s_red, c_smem))
            return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            su += h->du2;
            sv += h->dv2;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        h->du2 = su;
        h->dv2 = sv;
    }
}

// The global-memory path of k_solve_compact at twice its blocks per SM (32
// registers a thread), for solves too large for the shared-memory paths.
template <typename T, int NT, int UNROLL>
__global__ void __launch_bounds__(NT, 2048 / NT)
k_solve_compact_wide(IterParams P, int iters, int n_inner, int check_every, double tol, int warm,
                     const int32_t* __restrict__ counts, const int32_t* __restrict__ nb, int64_t stride,
                     T* P1a, T* P1b, T* P2a, T* P2b, T* V, const float* __restrict__ F, float* U,
                     float* Up, float* Wc, float* Wc2, double* partials, WsHeader* h, float* ckpt,
                     int ckpt_every, int grid1, const int32_t* __restrict__ base, int nimg) {
    __shared__ double s_red[66];   // block_sum2f (as floats), stop flag
    if (*(volatile int*)&h->done) return;
    const int n = counts[1];
    if (!compact_wide<T>(n, grid1)) return;
    const unsigned nblocks = gridDim.x;
    const int per = (n + (int)nblocks - 1) / (int)nblocks;
    const int a0 = (int)blockIdx.x * per, a1 = min(n, a0 + per);
    // (never the fused iteration: this kernel runs only when the one-block
    // kernel's blocks would hold more than 8,000 pixels each, so with at
    // most twice its blocks each block holds more than 3 x NT)
    const Own<T, false> O{nb, stride, V, F, 0};
    unsigned gen = 0u;
    compact_iterations<T, false, NT, UNROLL>(P, O, a0, a1, iters, n_inner, check_every, tol, warm, stride, P1a,
                                             P1b, P2a, P2b, U, Up, Wc, Wc2, partials, h, ckpt, ckpt_every,
                                             s_red, 0, gen);
}

// Dense u, v, p1, p2 of the final iterate of every image of the batch:
// compact values on RD, the fixed values elsewhere.
template <typename T>
__global__ void k_compact_scatter(BatchDesc B, const int32_t* __restrict__ base,
                                  const int32_t* __restrict__ totals, int iters, int n_inner,
                                  CompactState S, const WsHeader* __restrict__ h, long long rm_above) {
    if (totals[1] > rm_above) return;   // scattered by wide.cu
    const int lane = threadIdx.x & 31;
    const long long word = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (word >= B.total_words) return;
    const int k = batch_image_of(B, word);
    const BatchImage& I = B.img[k];
    const long long lw = word - I.word_off;
    const int i = (int)(lw / I.ntx);
    const int wx = (int)(lw - (long long)i * I.ntx);
    const int j = wx * 32 + lane;
    if (j >= I.W) return;
    const int64_t wo = (int64_t)i * I.nw + wx;
    const int64_t o = (int64_t)i * I.ld + j;
    const uint32_t a = I.act[wo];
    const float hh = ((I.fg[wo] >> lane) & 1u) ? 1.f : 0.f;
    const bool ok = base[B.n] <= S.cap && totals[1] == base[B.n];
    if (ok && ((a >> lane) & 1u)) {
        const int l = h->done ? h->iters_done : iters;
        const int pb = (int)(((long long)l * n_inner) & 1);
        const int64_t idx = base[k] + I.wstart[wo] + __popc(a & lanemask_lt(lane));
        I.u[o] = S.u[idx];
        I.v[o] = Store<T>::ld_rw(static_cast<const T*>(S.v), idx) + Store<T>::vbias;
        I.p1[o] = Store<T>::ld_rw(static_cast<const T*>(S.p1[pb]), idx);
        I.p2[o] = Store<T>::ld_rw(static_cast<const T*>(S.p2[pb]), idx);
    } else {
        I.u[o] = hh; I.v[o] = hh; I.p1[o] = 0.f; I.p2[o] = 0.f;
    }
}

// =================================================== stopping test, stats

__global__ void k_solve_begin(WsHeader* h) {
    h->bar_count = 0u - h->bar_extra;   // 0 unless the timeout path is under test
    h->done = 0;
    h->iters_done = 0;
    h->last_check = 0;
    h->du2 = 0.0;
    h->dv2 = 0.0;
    for (int k = 0; k < 4; ++k) h->tb_ticket[k] = 0;
    h->tb_buf = 0;
    h->n_smem_blocks = 0;
    h->n_h1_blocks = 0;
    h->h1_vote = 0u;
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
        h->du2 = sa[0];
        h->dv2 = sb[0];
        h->last_check = l;
        if (tol > 0.0 && fmax(sa[0], sb[0]) <= tol * tol) {
            h->iters_done = l;
            h->done = 1;
        }
    }
}

__global__ void k_solve_end(const WsHeader* __restrict__ h, const int32_t* __restrict__ counts,
                            int iters, double* stats) {
    stats[0] = h->done ? h->iters_done : iters;
    stats[1] = sqrt(h->du2);
    stats[2] = sqrt(h->dv2);
    stats[3] = counts[1];
    stats[4] = counts[0];
    stats[5] = h->last_check;
    stats[6] = h->n_smem_blocks;
    stats[7] = h->n_h1_blocks;
}

// ================================================================== host

seg_status launch_solve_begin(WsHeader* h, cudaStream_t s) {
    k_solve_begin<<<1, 1, 0, s>>>(h);
    SEG_LAUNCHED("k_solve_begin");
    return SEG_OK;
}

seg_status launch_solve_end(const WsHeader* h, const int32_t* counts, int iters, double* stats,
                            cudaStream_t s) {
    k_solve_end<<<1, 1, 0, s>>>(h, counts, iters, stats);
    SEG_LAUNCHED("k_solve_end");
    return SEG_OK;
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
    size_t off[11];
    int64_t cap;       // RD pixels the state can hold
    int64_t stride;    // elements allocated per array (cap + a chunk of slack, multiple of 64)
};

// compact state: p1[2], p2[2], v (storage type), f, u, w (float32),
// neighbour table (int32 x NB_COUNT rows), w2, up (float32), each array
// 256-byte aligned and `stride` elements long
constexpr int kCompactArrays = 11;
constexpr int kSlack = 256;   // spare elements past the capacity in every array
constexpr size_t compact_per_element(size_t sz) { return 5 * sz + 20 + 4 * NB_COUNT; }
static int64_t compact_stride(int64_t capacity) {
    return (int64_t)align_up((size_t)std::max<int64_t>(capacity, 1) + kSlack, 64);
}
static CompactLayout compact_layout(size_t state_bytes, int storage) {
    CompactLayout C{};
    const size_t sz = storage_size(storage);
    const size_t per = compact_per_element(sz);
    int64_t stride = state_bytes > kCompactArrays * 256
                         ? (int64_t)((state_bytes - kCompactArrays * 256) / per) / 64 * 64 : 0;
    C.stride = stride;
    C.cap = std::max<int64_t>(0, stride - kSlack);
    size_t o = 0;
    for (int a = 0; a < 5; ++a) { C.off[a] = o; o = align_up(o + sz * (size_t)stride, 256); }
    C.off[5] = o; o = align_up(o + 4 * (size_t)stride, 256);   // f
    C.off[6] = o; o = align_up(o + 4 * (size_t)stride, 256);   // u
    C.off[7] = o; o = align_up(o + 4 * (size_t)stride, 256);   // w
    C.off[8] = o; o = align_up(o + 4 * (size_t)NB_COUNT * stride, 256);   // neighbour table
    C.off[9] = o; o = align_up(o + 4 * (size_t)stride, 256);   // w2
    C.off[10] = o;                                             // up
    return C;
}

using DenseKernel = void (*)(IterParams, int, int, int, const int32_t*, const uint32_t*, const float*,
                             const float*, const float*, const float*, float*, float*, float*, float*,
                             double*, WsHeader*);

static seg_status run_dense(const IterParams& P0, const seg_params* prm, const int32_t* counts,
                            const uint32_t* act, const float* f, float* u, float* st,
                            double* partials, WsHeader* h, cudaStream_t s) {
    int64_t plane = (int64_t)P0.H * P0.ld;
    float* P1[2] = {st, st + plane};
    float* P2[2] = {st + 2 * plane, st + 3 * plane};
    float* V[2] = {st + 4 * plane, st + 5 * plane};
    // variants: [check][write_u]; p-only sweeps neither check nor write u
    DenseKernel kv[2][2] = {{k_step_dense<false, false, false>, k_step_dense<false, false, true>},
                            {k_step_dense<false, true, false>, k_step_dense<false, true, true>}};
    DenseKernel kp = k_step_dense<true, false, false>;
    // band height: 32 rows (3 halo rows per band) unless that leaves fewer
    // than ~48 warps per SM of work, then 16 or 8
    const int n_strips = (P0.W + kStripOut - 1) / kStripOut;
    int band_h = 32;
    while (band_h > 8 && (int64_t)n_strips * ((P0.H + band_h - 1) / band_h) < 48LL * sm_count())
        band_h /= 2;
    const int n_tasks = n_strips * ((P0.H + band_h - 1) / band_h);
    const int64_t max_blocks = (n_tasks + kDenseWarps - 1) / kDenseWarps;
    const int grid = grid_for(kv[1][1], kDenseWarps * 32, max_blocks);
    int pb = 0, vb = 0;
    const int C = test_interval(prm->tol, prm->check_every, prm->iters);
    for (int it = 0; it < prm->iters; ++it) {
        const int l = it + 1;
        for (int sw = 1; sw < prm->n_inner; ++sw) {
            kp<<<grid, kDenseWarps * 32, 0, s>>>(P0, n_strips, n_tasks, band_h, counts, act, f, P1[pb], P2[pb],
                                                 V[vb], P1[pb ^ 1], P2[pb ^ 1], V[vb], u, partials, h);
            SEG_LAUNCHED("k_step_dense<p-only>");
            pb ^= 1;
        }
        const bool check = (l % C == 0) || l == prm->iters;
        const bool write_u = check || ((l + 1) % C == 0) || l == prm->iters;
        kv[check][write_u]<<<grid, kDenseWarps * 32, 0, s>>>(P0, n_strips, n_tasks, band_h, counts, act, f,
                                                             P1[pb], P2[pb], V[vb], P1[pb ^ 1],
                                                             P2[pb ^ 1], V[vb ^ 1], u, partials, h);
        SEG_LAUNCHED("k_step_dense");
        pb ^= 1;
        vb ^= 1;
        if (check) {
            k_check<<<1, kCheckThreads, 0, s>>>(partials, n_tasks, l, prm->tol, h);
            SEG_LAUNCHED("k_check");
        }
    }
    return SEG_OK;
}

// Compact solve of a batch (a single image is a batch of one): bases of the
// images, gather + neighbour table, one cooperative launch for all the
// iterations, scatter.
template <typename T>
static seg_status solve_compact_batch(const IterParams& P0, const seg_params* prm, const BatchDesc& B,
                                      int64_t max_pixels, void* state, size_t state_bytes,
                                      int32_t* base, int32_t* totals, double* partials,
                                      int64_t max_partials, WsHeader* h, cudaStream_t s,
                                      float* ckpt = nullptr, int ckpt_every = 1) {
    CompactLayout C = compact_layout(state_bytes, prm->storage);
    CompactState S{};
    char* sb = static_cast<char*>(state);
    S.p1[0] = sb + C.off[0];
    S.p1[1] = sb + C.off[1];
    S.p2[0] = sb + C.off[2];
    S.p2[1] = sb + C.off[3];
    S.v = sb + C.off[4];
    S.f = reinterpret_cast<float*>(sb + C.off[5]);
    S.u = reinterpret_cast<float*>(sb + C.off[6]);
    S.w = reinterpret_cast<float*>(sb + C.off[7]);
    S.nb = reinterpret_cast<int32_t*>(sb + C.off[8]);
    S.w2 = reinterpret_cast<float*>(sb + C.off[9]);
    S.up = reinterpret_cast<float*>(sb + C.off[10]);
    S.cap = C.cap;
    S.stride = C.stride;
    k_batch_bases<<<1, 1, 0, s>>>(B, base, totals, C.cap, h);
    SEG_LAUNCHED("k_batch_bases");
    const unsigned gblocks = (unsigned)std::max<long long>(1, (B.total_words + 7) / 8);
    // one image without checkpoints, its columns within 16 bits: when its RD
    // is too large for the shared-memory paths, the row-major solve of
    // wide.cu runs instead of the tile-major global-memory kernel (decided
    // on the device from the RD count, like the choice between the two
    // tile-major kernels); wide_above is that count's threshold
    const int NTs = kCompactThreads;
    const bool rm = B.n == 1 && std::max(1, prm->n_inner) == 1 && ckpt == nullptr && B.img[0].W <= 65535 &&
                    B.img[0].H <= 65535;
    const int grid1_pre = [&] {
        int ps = 0;
        const void* k1 = compact_waves(B.n, prm->tol, std::max(1, prm->n_inner), ckpt)
                             ? (const void*)k_solve_compact<T, kCompactThreads, kCompactUnroll, true>
                             : (const void*)k_solve_compact<T, kCompactThreads, kCompactUnroll, false>;
        cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)compact_smem(NTs));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k1, NTs, compact_smem(NTs));
        const int64_t most = std::max<int64_t>(1, std::min<int64_t>(C.cap, max_pixels));
        int g = (int)std::min<int64_t>((int64_t)std::max(ps, 1) * sm_count(),
                                       std::max<int64_t>(1, (most + NTs - 1) / NTs));
        return (int)std::min<int64_t>(g, max_partials / 2);
    }();
    const long long wide_above = (long long)grid1_pre *
                                 (long long)(compact_smem(kCompactThreads) / (4 * NB_UUR + sizeof(T)));
    const long long rm_above = rm ? wide_above : LLONG_MAX;
    k_compact_gather<T><<<gblocks, 256, 0, s>>>(P0, B, base, prm->warm_start, S, h, totals, rm_above);
    SEG_LAUNCHED("k_compact_gather");

    T* P1a = static_cast<T*>(S.p1[0]);
    T* P1b = static_cast<T*>(S.p1[1]);
    T* P2a = static_cast<T*>(S.p2[0]);
    T* P2b = static_cast<T*>(S.p2[1]);
    T* V = static_cast<T*>(S.v);
    const bool waves = compact_waves(B.n, prm->tol, std::max(1, prm->n_inner), ckpt);
    const void* kern = waves ? (const void*)k_solve_compact<T, kCompactThreads, kCompactUnroll, true>
                             : (const void*)k_solve_compact<T, kCompactThreads, kCompactUnroll, false>;
    const size_t smem = compact_smem(NTs);
    // one cooperative launch for the whole solve: the grid is what can be
    // resident at once (at most one block per NT RD pixels of capacity)
    SEG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTs, smem));
    if (per_sm <= 0) return fail(SEG_ERR_CUDA, "k_solve_compact cannot be resident");
    const int64_t most = std::max<int64_t>(1, std::min<int64_t>(C.cap, max_pixels));
    int grid = (int)std::min<int64_t>((int64_t)per_sm * sm_count(),
                                      std::max<int64_t>(1, (most + NTs - 1) / NTs));
    grid = (int)std::min<int64_t>(grid, max_partials / 2);   // partials are double-buffered
    int iters = prm->iters, n_inner = std::max(1, prm->n_inner);
    int check_every = test_interval(prm->tol, prm->check_every, prm->iters);
    double tol = prm->tol;
    int warm = prm->warm_start;
    int64_t stride = S.stride;
    const int32_t* nbp = S.nb;
    const int32_t* cnt = totals;
    float* F = S.f;
    float* U = S.u;
    float* Up = S.up;
    float* Wc = S.w;
    float* Wc2 = S.w2;
    IterParams P = P0;
    // the global-memory kernel for solves too large for shared memory (the
    // kernels decide on the device which of them runs)
    const void* kern2 = (const void*)k_solve_compact_wide<T, kCompactThreads, kCompactWideUnroll>;
    int per_sm2 = 0;
    SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, kern2, NTs, 0));
    if (per_sm2 <= 0) return fail(SEG_ERR_CUDA, "k_solve_compact_wide cannot be resident");
    int grid2 = (int)std::min<int64_t>((int64_t)per_sm2 * sm_count(),
                                       std::max<int64_t>(1, (most + NTs - 1) / NTs));
    grid2 = (int)std::min<int64_t>(grid2, max_partials / 2);
    int grid1 = grid;
    const int32_t* bases = base;
    int nimg = B.n;
    void* args[] = {&P, &iters, &n_inner, &check_every, &tol, &warm, (void*)&cnt, (void*)&nbp, &stride,
                    &P1a, &P1b, &P2a, &P2b, &V, &F, &U, &Up, &Wc, &Wc2, &partials, &h, &ckpt,
                    &ckpt_every, &grid1, &bases, &nimg};
    if (grid != grid1_pre) return fail(SEG_ERR_CUDA, "k_solve_compact: inconsistent grid");
    if (iters > 0 || warm) {
        SEG_TRY_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(NTs), args, smem, s));
        count_launch();
        if (debug_mode()) SEG_TRY(after_launch("k_solve_compact"));
        if (!waves && !rm) {
            SEG_TRY_CUDA(cudaLaunchCooperativeKernel(kern2, dim3(grid2), dim3(NTs), args, 0, s));
            count_launch();
            if (debug_mode()) SEG_TRY(after_launch("k_solve_compact_wide"));
        }
    }
    if (rm) {
        const BatchImage& I = B.img[0];
        RowMajorArgs R{};
        R.act = I.act; R.fg = I.fg; R.f = I.f;
        R.u = I.u; R.v = I.v; R.p1 = I.p1; R.p2 = I.p2;
        R.counts = totals; R.h = h;
        R.H = I.H; R.W = I.W; R.ld = I.ld; R.nw = I.nw; R.ntx = I.ntx;
        R.theta_lambda = I.theta_lambda; R.inv_theta = P0.inv_theta;
        R.wide_above = wide_above;
        RowMajorArrays A{};
        A.p1[0] = S.p1[0]; A.p1[1] = S.p1[1]; A.p2[0] = S.p2[0]; A.p2[1] = S.p2[1]; A.v = S.v;
        A.F = S.f; A.U = S.u; A.Up = S.up; A.Wc = S.w;
        A.dd = reinterpret_cast<uint16_t*>(S.nb);
        A.du = A.dd + S.stride;
        A.fl = A.du + S.stride;
        R.rowstart = reinterpret_cast<int32_t*>(A.fl + S.stride);   // H + 1 <= the rest of the table region
        A.cap = S.cap;
        IterParams Pi = P0;
        Pi.H = I.H; Pi.W = I.W; Pi.ld = I.ld; Pi.nw = I.nw; Pi.ntx = I.ntx;
        SEG_TRY(run_wide_rm(R, A, Pi, prm, partials, max_partials / 2, s));
    }
    k_compact_scatter<T><<<gblocks, 256, 0, s>>>(B, base, totals, prm->iters, std::max(1, prm->n_inner),
                                                 S, h, rm_above);
    SEG_LAUNCHED("k_compact_scatter");
    return SEG_OK;
}

static seg_status solve_compact_any(const IterParams& P, const seg_params* prm, const BatchDesc& B,
                                    int64_t max_pixels, void* state, size_t state_bytes, int32_t* base,
                                    int32_t* totals, double* partials, int64_t max_partials, WsHeader* h,
                                    cudaStream_t s) {
    switch (prm->storage) {
        case SEG_STORE_F32:
            return solve_compact_batch<float>(P, prm, B, max_pixels, state, state_bytes, base, totals,
                                              partials, max_partials, h, s);
        case SEG_STORE_BF16:
            return solve_compact_batch<__nv_bfloat16>(P, prm, B, max_pixels, state, state_bytes, base,
                                                      totals, partials, max_partials, h, s);
        default:
            return solve_compact_batch<__half>(P, prm, B, max_pixels, state, state_bytes, base, totals,
                                               partials, max_partials, h, s);
    }
}

static seg_status check_params(const seg_params* prm) {
    if (!prm) return fail(SEG_ERR_INVALID_ARG, "params must be non-NULL");
    const int th = prm->tile_h;
    if (th != 4 && th != 8 && th != 16 && th != 32)
        return fail(SEG_ERR_INVALID_ARG, "tile_h=%d not in {4, 8, 16, 32}", th);
    if (prm->iters < 0 || prm->n_inner < 1 || prm->check_every < 1)
        return fail(SEG_ERR_INVALID_ARG, "iters >= 0, n_inner >= 1, check_every >= 1 required");
    if (!(prm->theta > 0) || !(prm->tau > 0) || !std::isfinite(prm->lambda) || std::isnan(prm->tol))
        return fail(SEG_ERR_INVALID_ARG, "theta, tau must be > 0 and lambda finite");
    if (prm->mode != SEG_MODE_DENSE && prm->mode != SEG_MODE_COMPACT && prm->mode != SEG_MODE_TILED)
        return fail(SEG_ERR_INVALID_ARG, "unknown mode %d", prm->mode);
    if (prm->storage < 0 || prm->storage > 2)
        return fail(SEG_ERR_INVALID_ARG, "unknown storage %d", prm->storage);
    if (prm->mode != SEG_MODE_COMPACT && prm->storage != SEG_STORE_F32)
        return fail(SEG_ERR_INVALID_ARG, "16-bit storage needs SEG_MODE_COMPACT");
    if (prm->sweep < 0) return fail(SEG_ERR_INVALID_ARG, "sweep must be >= 0");
    return SEG_OK;
}

static IterParams iter_params(const seg_params* prm, int H, int W, int ld) {
    IterParams P{};
    P.theta = (float)prm->theta;
    P.inv_theta = (float)(1.0 / prm->theta);
    P.tau = (float)prm->tau;
    P.theta_lambda = (float)(prm->theta * prm->lambda);
    P.H = H; P.W = W; P.ld = ld; P.nw = ld / 32; P.ntx = (W + 31) / 32; P.th = prm->tile_h;
    return P;
}

// ============================================================ adjoint
//
// Reverse mode of the unrolled compact iteration (float32 state, n_inner =
// 1, a fixed number of iterations), for L with given dL/du^K (and dL/dv^K):
// the partition is held fixed, u0 = H(-f) is piecewise constant, the clip has
// derivative 1 strictly inside (0, 1) -- i.e. where the clipped value lies in
// (0, 1) -- and 0 elsewhere, and d|g| is 0 at g = 0.  For each segment of C
// iterations, from the last to the first, the forward iterates are recomputed
// from the segment's checkpoint into a segment buffer, then the adjoint walks
// back through them:
//   A  sbar = vbar [0 < v^{n+1} < 1];  ubar = sbar (+ dL/du^K at n+1 = K);
//      Fbar -= sbar  (F = theta lambda f)
//   B  qbar = pbar + theta grad ubar;  with d = 1 + tau |g^n|, q = p^{n+1}:
//      gbar = (tau / d) (qbar - (qbar . q) g/|g|),  pbar_direct = qbar / d
//   C  wbar = -div gbar at x, x+e1, x+e2;  pbar = pbar_direct - grad wbar;
//      vbar = ubar - wbar / theta
// (div^T = -grad), then the v0 = clip(u0 - F) term.  Finally df = theta
// lambda Fbar, dlambda = theta sum f Fbar, dc1 = sum df (-2)(z - c1),
// dc2 = sum df 2 (z - c2).

struct AdjArrays {
    float *p1b, *p2b, *vb, *ub, *gb1, *gb2, *pd1, *pd2, *fb, *gu, *gv;   // [stride] each
    float *seg, *seg2;   // two segment buffers: [(C + 1)][4][stride]  (p1, p2, v, w)
};

// gathers dL/du^K, dL/dv^K into compact order and clears the adjoint
__global__ void k_adj_gather(IterParams P, const uint32_t* __restrict__ act,
                             const int32_t* __restrict__ wstart, const int32_t* __restrict__ base,
                             const float* __restrict__ grad_u, const float* __restrict__ grad_v,
                             AdjArrays A) {
    const int lane = threadIdx.x & 31;
    const int64_t word = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t nwords = (int64_t)P.H * P.ntx;
    if (word >= nwords) return;
    const int i = (int)(word / P.ntx);
    const int wx = (int)(word - (int64_t)i * P.ntx);
    const int64_t wo = (int64_t)i * P.nw + wx;
    const uint32_t a = act[wo];
    if (!((a >> lane) & 1u)) return;
    const int64_t idx = (base ? *base : 0) + wstart[wo] + __popc(a & lanemask_lt(lane));
    const int64_t o = (int64_t)i * P.ld + wx * 32 + lane;
    A.gu[idx] = grad_u[o];
    A.gv[idx] = grad_v ? grad_v[o] : 0.f;
}

template <int NT>
__device__ __forceinline__ double block_sum1(double x, double* s_red) {
    for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(0xffffffffu, x, d);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[wid] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t += s_red[w];
    return t;
}

// Where the reverse sweep reads its pixels' neighbour-table rows (up, left,
// down, right, down-left, up-right) and theta lambda f, which nothing
// writes: SM, copies in shared memory made at the start of the launch
// (indexed from the block's first pixel a0), so that the first load of each
// phase's dependent chain is a shared-memory load; else the global table.
enum { ADJ_U = 0, ADJ_L, ADJ_D, ADJ_R, ADJ_DL, ADJ_UR, ADJ_ROWS };
// pixels a block can keep (28 bytes each) at kBackwardMinBlocksSm blocks per SM
constexpr int kAdjSmemPixels = (225 * 1024 / kBackwardMinBlocksSm - 2048) / 28 / 32 * 32;
__host__ __device__ constexpr int adj_table_row(int k) {
    return k == ADJ_U ? NB_UP : k == ADJ_L ? NB_LEFT : k == ADJ_D ? NB_DOWN : k == ADJ_R ? NB_RIGHT
         : k == ADJ_DL ? NB_DOWNLEFT : NB_UPRIGHT;
}
template <bool SM>
struct AdjNb;
template <>
struct AdjNb<true> {   // rows of kAdjSmemPixels words, then theta lambda f
    const int32_t* t;
    int a0;
    __device__ __forceinline__ int nb(int k, int a) const { return t[k * kAdjSmemPixels + (a - a0)]; }
    __device__ __forceinline__ float tlf(int a) const {
        return reinterpret_cast<const float*>(t + ADJ_ROWS * kAdjSmemPixels)[a - a0];
    }
};
template <>
struct AdjNb<false> {   // the rows of the global table
    const int32_t* r[ADJ_ROWS];
    const float* F;
    __device__ __forceinline__ int nb(int k, int a) const { return __ldg(r[k] + a); }
    __device__ __forceinline__ float tlf(int a) const { return __ldg(F + a); }
};

// The replay's steps and phases B and C of a reverse step for U pixels of a
// thread at a time: every load of all U (neighbour-table entries, then the
// values they name) is issued before the first store.  No phase stores into
// an array it loads from other pixels, and a pixel's own words are read
// before they are written, so the U pixels' chains of dependent loads
// overlap.  Every product that meets a sum is written as fmaf or __fmul_rn,
// so that a pixel's rounding does not depend on which copy of the code (the
// U-wide loop or the remainder) took it, and a batch and its images one by
// one give the same bits.

// Replay dual step (dual_one's arithmetic at float32): p' of iterate m + 1
// from p, w of iterate m.
template <bool SM, int U>
__device__ __forceinline__ void adj_replay_dual(const int (&a)[U], const AdjNb<SM>& N, const float* __restrict__ P1,
                                                const float* __restrict__ P2, const float* __restrict__ Wm,
                                                float* __restrict__ Q1, float* __restrict__ Q2, float tau,
                                                float inv_theta) {
    int nd[U], nr[U], ndl[U], nur[U];
    float p1[U], p2[U], w0[U], wd[U], wr[U], p2dl[U], p1ur[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        nd[k] = N.nb(ADJ_D, a[k]);
        nr[k] = N.nb(ADJ_R, a[k]);
        ndl[k] = N.nb(ADJ_DL, a[k]);
        nur[k] = N.nb(ADJ_UR, a[k]);
        p1[k] = P1[a[k]];
        p2[k] = P2[a[k]];
        w0[k] = Wm[a[k]];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        wd[k] = nd[k] >= 0 ? Wm[nd[k]] : 0.f;
        wr[k] = nr[k] >= 0 ? Wm[nr[k]] : 0.f;
        p2dl[k] = ndl[k] >= 0 ? P2[ndl[k]] : 0.f;
        p1ur[k] = nur[k] >= 0 ? P1[nur[k]] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        float g1 = 0.f, g2 = 0.f;
        if (nd[k] != kNbOut) g1 = (nd[k] >= 0 ? wd[k] : w_fixed(p1[k], p2dl[k], nd[k], inv_theta)) - w0[k];
        if (nr[k] != kNbOut) g2 = (nr[k] >= 0 ? wr[k] : w_fixed(p1ur[k], p2[k], nr[k], inv_theta)) - w0[k];
        float q1, q2;
        chambolle_update(p1[k], p2[k], g1, g2, tau, q1, q2);
        Q1[a[k]] = q1;
        Q2[a[k]] = q2;
    }
}

// Replay primal step (primal_one's arithmetic and rounding, v read from
// iterate m and written to iterate m + 1 with w).
template <bool SM, int U>
__device__ __forceinline__ void adj_replay_primal(const int (&a)[U], const AdjNb<SM>& N, const float* __restrict__ P1,
                                                  const float* __restrict__ P2, const float* __restrict__ Vm,
                                                  float* Vn, float* Wn, float theta, float inv_theta) {
    int nu[U], nl[U];
    float q1[U], q2[U], vm[U], ff[U], xu[U], xl[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        nu[k] = N.nb(ADJ_U, a[k]);
        nl[k] = N.nb(ADJ_L, a[k]);
        q1[k] = P1[a[k]];
        q2[k] = P2[a[k]];
        vm[k] = Vm[a[k]];
        ff[k] = N.tlf(a[k]);
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        xu[k] = nu[k] >= 0 ? P1[nu[k]] : 0.f;
        xl[k] = nl[k] >= 0 ? P2[nl[k]] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const float div = (q1[k] - xu[k]) + (q2[k] - xl[k]);
        const float un = fmaf(-theta, div, vm[k]);
        const float vn = clamp01(un - ff[k]);
        Vn[a[k]] = vn;
        Wn[a[k]] = fmaf(-vn, inv_theta, div);
    }
}

// Phase B: qbar = pbar + theta grad ubar, then the adjoint of the
// fixed-point step p' = (p + tau g) / (1 + tau |g|) at iterate m (p, w) with
// p' of iterate m + 1: gbar (to gb1, gb2) and qbar / d (to pd1, pd2).
template <bool SM, int U>
__device__ __forceinline__ void adj_phase_b(const int (&a)[U], const AdjNb<SM>& N, const float* __restrict__ ub,
                                            const float* __restrict__ P1, const float* __restrict__ P2,
                                            const float* __restrict__ Wm, const float* __restrict__ Q1,
                                            const float* __restrict__ Q2, const float* __restrict__ p1b,
                                            const float* __restrict__ p2b, float* __restrict__ gb1,
                                            float* __restrict__ gb2, float* __restrict__ pd1,
                                            float* __restrict__ pd2, float theta, float tau, float inv_theta) {
    int nd[U], nr[U], ndl[U], nur[U];
    float ua[U], p1[U], p2[U], w0[U], q1[U], q2[U], pb1[U], pb2[U];
    float ud[U], ur[U], wd[U], wr[U], p2dl[U], p1ur[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        nd[k] = N.nb(ADJ_D, a[k]);
        nr[k] = N.nb(ADJ_R, a[k]);
        ndl[k] = N.nb(ADJ_DL, a[k]);
        nur[k] = N.nb(ADJ_UR, a[k]);
        ua[k] = ub[a[k]];
        p1[k] = P1[a[k]];
        p2[k] = P2[a[k]];
        w0[k] = Wm[a[k]];
        q1[k] = Q1[a[k]];
        q2[k] = Q2[a[k]];
        pb1[k] = p1b[a[k]];
        pb2[k] = p2b[a[k]];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        ud[k] = nd[k] >= 0 ? ub[nd[k]] : 0.f;
        ur[k] = nr[k] >= 0 ? ub[nr[k]] : 0.f;
        wd[k] = nd[k] >= 0 ? Wm[nd[k]] : 0.f;
        wr[k] = nr[k] >= 0 ? Wm[nr[k]] : 0.f;
        p2dl[k] = ndl[k] >= 0 ? P2[ndl[k]] : 0.f;
        p1ur[k] = nur[k] >= 0 ? P1[nur[k]] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const bool dn = nd[k] != kNbOut, rt = nr[k] != kNbOut;
        const float qb1 = dn ? fmaf(theta, ud[k] - ua[k], pb1[k]) : pb1[k];
        const float qb2 = rt ? fmaf(theta, ur[k] - ua[k], pb2[k]) : pb2[k];
        // g^n as in the forward dual step
        const float g1 = dn ? (nd[k] >= 0 ? wd[k] : w_fixed(p1[k], p2dl[k], nd[k], inv_theta)) - w0[k] : 0.f;
        const float g2 = rt ? (nr[k] >= 0 ? wr[k] : w_fixed(p1ur[k], p2[k], nr[k], inv_theta)) - w0[k] : 0.f;
        const float s2 = fmaf(g1, g1, g2 * g2);
        const float inv_nrm = s2 > 0.f ? rsqrtf(s2) : 0.f;
        const float r = __fdividef(1.0f, fmaf(tau, s2 * inv_nrm, 1.0f));   // 1 / (1 + tau |g|)
        // gbar = (tau / d) (qbar - (qbar . q) g / |g|), d = 1 + tau |g|
        const float dot = fmaf(qb1, q1[k], __fmul_rn(qb2, q2[k])) * inv_nrm;
        const float tr = tau * r;
        gb1[a[k]] = dn ? tr * fmaf(-dot, g1, qb1) : 0.f;
        gb2[a[k]] = rt ? tr * fmaf(-dot, g2, qb2) : 0.f;
        pd1[a[k]] = qb1 * r;
        pd2[a[k]] = qb2 * r;
    }
}

// Phase C: wbar = -div gbar at x, x + e1, x + e2; pbar, vbar of iterate m;
// then (m > 0) the next step's phase A: the clip's adjoint at v of iterate m
// into ubar and fbar.
template <bool SM, int U>
__device__ __forceinline__ void adj_phase_c(const int (&a)[U], const AdjNb<SM>& N, const float* __restrict__ gb1,
                                            const float* __restrict__ gb2, const float* __restrict__ pd1,
                                            const float* __restrict__ pd2, const float* __restrict__ Vm,
                                            float* __restrict__ p1b, float* __restrict__ p2b,
                                            float* __restrict__ vb, float* ub, float* fb, bool phase_a,
                                            float inv_theta) {
    int nu[U], nl[U], nd[U], nr[U], ndl[U], nur[U];
    float g1[U], g2[U], d1[U], d2[U], ua[U], vm[U], fbv[U];
    float g1u[U], g2l[U], g1d[U], g2d[U], g2dl[U], g1r[U], g2r[U], g1ur[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        nu[k] = N.nb(ADJ_U, a[k]);
        nl[k] = N.nb(ADJ_L, a[k]);
        nd[k] = N.nb(ADJ_D, a[k]);
        nr[k] = N.nb(ADJ_R, a[k]);
        ndl[k] = N.nb(ADJ_DL, a[k]);
        nur[k] = N.nb(ADJ_UR, a[k]);
        g1[k] = gb1[a[k]];
        g2[k] = gb2[a[k]];
        d1[k] = pd1[a[k]];
        d2[k] = pd2[a[k]];
        ua[k] = ub[a[k]];
        vm[k] = phase_a ? Vm[a[k]] : 0.f;
        fbv[k] = phase_a ? fb[a[k]] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        g1u[k] = nu[k] >= 0 ? gb1[nu[k]] : 0.f;
        g2l[k] = nl[k] >= 0 ? gb2[nl[k]] : 0.f;
        g1d[k] = nd[k] >= 0 ? gb1[nd[k]] : 0.f;
        g2d[k] = nd[k] >= 0 ? gb2[nd[k]] : 0.f;
        g2dl[k] = ndl[k] >= 0 ? gb2[ndl[k]] : 0.f;
        g1r[k] = nr[k] >= 0 ? gb1[nr[k]] : 0.f;
        g2r[k] = nr[k] >= 0 ? gb2[nr[k]] : 0.f;
        g1ur[k] = nur[k] >= 0 ? gb1[nur[k]] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const float wb0 = -((g1[k] - g1u[k]) + (g2[k] - g2l[k]));
        const float wbd = -((g1d[k] - g1[k]) + (g2d[k] - g2dl[k]));
        const float wbr = -((g1r[k] - g1ur[k]) + (g2r[k] - g2[k]));
        p1b[a[k]] = d1[k] - (nd[k] != kNbOut ? wbd - wb0 : 0.f);
        p2b[a[k]] = d2[k] - (nr[k] != kNbOut ? wbr - wb0 : 0.f);
        const float v_b = fmaf(-wb0, inv_theta, ua[k]);
        vb[a[k]] = v_b;
        if (phase_a) {
            const float sb = (vm[k] > 0.f && vm[k] < 1.f) ? v_b : 0.f;
            ub[a[k]] = sb;
            fb[a[k]] = fbv[k] - sb;
        }
    }
}

// The reverse sweep of a block that owns the compact pixels [a0, a1).
template <bool SM>
__device__ __forceinline__ void adj_sweep(const IterParams& P, int iters, int ckpt_every, int n, int a0, int a1,
                                          const int32_t* __restrict__ nb, int64_t stride,
                                          const float* __restrict__ F, const float* __restrict__ ckpt,
                                          const AdjArrays& A, WsHeader* h, const AdjNb<SM>& N) {
    const unsigned nblocks = gridDim.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    unsigned gen = 0u;
    // the planes of recomputed iterate m in segment buffer `buf` (two: the
    // replay of one segment fills one while the reverse steps of the next
    // later segment read the other)
    struct Planes { float *p1, *p2, *v, *w; };
    auto seg_at = [&](int buf, int m) {
        float* b = (buf ? A.seg2 : A.seg) + (int64_t)m * 4 * stride;
        return Planes{b, b + stride, b + 2 * stride, b + 3 * stride};
    };
    const float theta = P.theta, tau = P.tau, inv_theta = P.inv_theta;
    // op(pixels[U]) over this block's range, U = kBackwardUnroll pixels a
    // thread at a time (stride nt), then the rest one by one
    auto each = [&](auto&& op) {
        int a = a0 + tid;
        for (; a + (kBackwardUnroll - 1) * nt < a1; a += kBackwardUnroll * nt) {
            int b[kBackwardUnroll];
#pragma unroll
            for (int k = 0; k < kBackwardUnroll; ++k) b[k] = a + k * nt;
            op(b);
        }
        for (; a < a1; a += nt) {
            const int b[1] = {a};
            op(b);
        }
    };
    // adjoint of the final iterate
    for (int a = a0 + tid; a < a1; a += nt) {
        A.p1b[a] = 0.f; A.p2b[a] = 0.f; A.vb[a] = A.gv[a]; A.fb[a] = 0.f;
    }
    const int nseg = (iters + ckpt_every - 1) / ckpt_every;
    auto seg_len = [&](int k) { return min(ckpt_every, iters - k * ckpt_every); };
    // Phase j of the replay of segment k into buffer buf: 0, the checkpoint
    // and its w (formed from the checkpoint's own planes); then the dual and
    // the primal step of each iteration m (the forward's steps and rounding:
    // dual_one, then primal_one's primal step with v read from iterate m and
    // written to iterate m + 1).
    auto replay_phase = [&](int k, int buf, int j) {
        if (j == 0) {
            const float* c = ckpt + (int64_t)k * 3 * stride;
            const Planes S0 = seg_at(buf, 0);
            float d0 = 0.f, d1 = 0.f;
            const Own<float, false> Oc{nb, stride, const_cast<float*>(c + 2 * stride), F, 0};
            for (int a = a0 + tid; a < a1; a += nt) {
                S0.p1[a] = c[a]; S0.p2[a] = c[stride + a]; S0.v[a] = c[2 * stride + a];
                primal_one(P, a, Oc, c, c + stride, nullptr, nullptr, S0.w, true, false, false, false, 0u, d0, d1);
            }
            return;
        }
        const int m = (j - 1) >> 1;
        const Planes Sm = seg_at(buf, m), Sn = seg_at(buf, m + 1);
        if (((j - 1) & 1) == 0)
            each([&](const auto& b) { adj_replay_dual(b, N, Sm.p1, Sm.p2, Sm.w, Sn.p1, Sn.p2, tau, inv_theta); });
        else
            each([&](const auto& b) {
                adj_replay_primal(b, N, Sn.p1, Sn.p2, Sm.v, Sn.v, Sn.w, theta, inv_theta);
            });
    };
    // Phase j of the walk back through segment k in buffer buf: 0, phase A
    // of its last step (clip, u^{n+1}; phase A only touches the pixel itself,
    // so for the other steps it runs at the end of phase C of the step
    // after); then phases B and C of each step m, last to first.
    //   B: qbar = pbar + theta grad ubar, the fixed-point step;
    //   C: wbar = -div gbar at x, x+e1, x+e2; pbar, vbar of iterate m; then
    //      the next step's phase A (no other pixel's phase C reads ub).
    auto reverse_phase = [&](int k, int buf, int j) {
        const int M = seg_len(k);
        if (j == 0) {
            const bool last = k * ckpt_every + M == iters;
            const float* vM = seg_at(buf, M).v;
            for (int a = a0 + tid; a < a1; a += nt) {
                const float vn = vM[a];
                const float sb = (vn > 0.f && vn < 1.f) ? A.vb[a] : 0.f;
                A.ub[a] = sb + (last ? A.gu[a] : 0.f);
                A.fb[a] -= sb;
            }
            return;
        }
        const int m = M - 1 - ((j - 1) >> 1);
        const Planes Sm = seg_at(buf, m), Sn = seg_at(buf, m + 1);
        if (((j - 1) & 1) == 0)
            each([&](const auto& b) {
                adj_phase_b(b, N, A.ub, Sm.p1, Sm.p2, Sm.w, Sn.p1, Sn.p2, A.p1b, A.p2b, A.gb1, A.gb2, A.pd1,
                            A.pd2, theta, tau, inv_theta);
            });
        else
            each([&](const auto& b) {
                adj_phase_c(b, N, A.gb1, A.gb2, A.pd1, A.pd2, Sm.v, A.p1b, A.p2b, A.vb, A.ub, A.fb, m > 0,
                            inv_theta);
            });
    };
    const int lastk = nseg - 1;
    if constexpr (SM) {
        // The replay of segment k - 1 runs in step with the walk back
        // through segment k (the two touch disjoint arrays: the other
        // segment buffer and the checkpoints; the adjoint arrays), so each
        // grid barrier serves one phase of each; the last segment's replay
        // runs alone first.
        for (int j = 0; j < 2 * seg_len(lastk) + 1; ++j) {
            replay_phase(lastk, lastk & 1, j);
            if (!grid_sync(h, nblocks, gen)) return;
        }
        for (int k = lastk; k >= 0; --k) {
            const int lr = 2 * seg_len(k) + 1, lp = k > 0 ? 2 * seg_len(k - 1) + 1 : 0;
            for (int j = 0; j < max(lr, lp); ++j) {
                if (j < lr) reverse_phase(k, k & 1, j);
                if (j < lp) replay_phase(k - 1, (k - 1) & 1, j);
                if (!grid_sync(h, nblocks, gen)) return;
            }
        }
    } else {
        // one segment at a time: its replay, then the walk back through it
        // (with the tables in global memory, two phases' loads between
        // barriers cost more than the barriers saved)
        for (int k = lastk; k >= 0; --k) {
            const int M = seg_len(k);
            replay_phase(k, 0, 0);
            if (!grid_sync(h, nblocks, gen)) return;
            for (int m = 0; m < M; ++m) {
                const Planes Sm = seg_at(0, m), Sn = seg_at(0, m + 1);
                each([&](const auto& b) {
                    adj_replay_dual(b, N, Sm.p1, Sm.p2, Sm.w, Sn.p1, Sn.p2, tau, inv_theta);
                });
                if (!grid_sync(h, nblocks, gen)) return;
                each([&](const auto& b) {
                    adj_replay_primal(b, N, Sn.p1, Sn.p2, Sm.v, Sn.v, Sn.w, theta, inv_theta);
                });
                if (!grid_sync(h, nblocks, gen)) return;
            }
            reverse_phase(k, 0, 0);
            if (!grid_sync(h, nblocks, gen)) return;
            for (int m = M - 1; m >= 0; --m) {
                const Planes Sm = seg_at(0, m), Sn = seg_at(0, m + 1);
                each([&](const auto& b) {
                    adj_phase_b(b, N, A.ub, Sm.p1, Sm.p2, Sm.w, Sn.p1, Sn.p2, A.p1b, A.p2b, A.gb1, A.gb2,
                                A.pd1, A.pd2, theta, tau, inv_theta);
                });
                if (!grid_sync(h, nblocks, gen)) return;
                each([&](const auto& b) {
                    adj_phase_c(b, N, A.gb1, A.gb2, A.pd1, A.pd2, Sm.v, A.p1b, A.p2b, A.vb, A.ub, A.fb, m > 0,
                                inv_theta);
                });
                if (!grid_sync(h, nblocks, gen)) return;
            }
        }
    }
    // v0 = clip(u0 - F): its clipped value is in checkpoint 0
    for (int a = a0 + tid; a < a1; a += nt) {
        const float v0 = ckpt[2 * stride + a];
        if (v0 > 0.f && v0 < 1.f) A.fb[a] -= A.vb[a];
    }
}

// Shared memory of one block: the six neighbour-table rows and theta lambda
// f of up to kAdjSmemPixels pixels, sized for kBackwardMinBlocksSm blocks per
// SM.
constexpr size_t kAdjSmemBytes = (size_t)kAdjSmemPixels * (4 * ADJ_ROWS + 4);

// SM: the block's neighbour-table rows and theta lambda f are copied into
// shared memory first (the launch gives kAdjSmemBytes, and every block's
// share of the largest possible RD fits), the replay of one segment runs in
// step with the walk back through the next later one, and blocks have
// kBackwardThreadsSm threads; else the tables are read from the global
// table, one segment at a time, in kBackwardThreads-thread blocks.  Two
// kernels, so that each gets its own register allocation.
template <bool SM>
__global__ void __launch_bounds__(SM ? kBackwardThreadsSm : kBackwardThreads, SM ? kBackwardMinBlocksSm : kBackwardMinBlocks)
k_backward_compact(IterParams P, int iters, int ckpt_every, const int32_t* __restrict__ counts,
                   const int32_t* __restrict__ nb, int64_t stride, const float* __restrict__ F,
                   const float* __restrict__ ckpt, AdjArrays A, WsHeader* h) {
    extern __shared__ __align__(16) unsigned char adj_smem[];
    if (*(volatile int*)&h->done) return;
    const unsigned nblocks = gridDim.x;
    const int n = counts[1];
    const int per = (n + (int)nblocks - 1) / (int)nblocks;
    const int a0 = (int)blockIdx.x * per, a1 = min(n, a0 + per);
    if constexpr (SM) {
        int32_t* sr = reinterpret_cast<int32_t*>(adj_smem);
        float* sF = reinterpret_cast<float*>(sr + ADJ_ROWS * kAdjSmemPixels);
        for (int i = threadIdx.x; i < a1 - a0; i += blockDim.x) {
#pragma unroll
            for (int k = 0; k < ADJ_ROWS; ++k)
                sr[k * kAdjSmemPixels + i] = __ldg(nb + adj_table_row(k) * stride + a0 + i);
            sF[i] = __ldg(F + a0 + i);
        }
        __syncthreads();
        adj_sweep<true>(P, iters, ckpt_every, n, a0, a1, nb, stride, F, ckpt, A, h, AdjNb<true>{sr, a0});
    } else {
        const AdjNb<false> N{{nb + NB_UP * stride, nb + NB_LEFT * stride, nb + NB_DOWN * stride,
                              nb + NB_RIGHT * stride, nb + NB_DOWNLEFT * stride, nb + NB_UPRIGHT * stride},
                             F};
        adj_sweep<false>(P, iters, ckpt_every, n, a0, a1, nb, stride, F, ckpt, A, h, N);
    }
}

// dL/df on the image (0 outside RD) and the FP64 sums for lambda, c1, c2
// (fixed grid of kReduceBlocks blocks: deterministic).
__global__ void __launch_bounds__(256)
k_adj_scatter(IterParams P, const float* __restrict__ f, const uint32_t* __restrict__ act,
              const int32_t* __restrict__ wstart, const int32_t* __restrict__ base,
              const float* __restrict__ Fbar, const float* __restrict__ z, const double* __restrict__ c,
              float theta_lambda, float* __restrict__ grad_f, double* __restrict__ red) {
    __shared__ double s_red[8];
    if (base) Fbar += *base;   // the image's compact range within a batch
    double sl = 0.0, s1 = 0.0, s2 = 0.0;
    const int64_t n = (int64_t)P.H * P.W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)((uint32_t)x / (uint32_t)P.W), j = x - i * P.W;   // x < 2^31
        const int64_t wo = i * P.nw + (j >> 5);
        const int64_t o = i * P.ld + j;
        const uint32_t a = act[wo];
        float gfv = 0.f;
        if ((a >> (j & 31)) & 1u) {
            const int64_t idx = wstart[wo] + __popc(a & lanemask_lt((int)(j & 31)));
            const double fb = Fbar[idx];
            gfv = (float)(theta_lambda * fb);
            sl += (double)P.theta * (double)f[o] * fb;
            if (z) {
                const double zz = z[o];
                s1 += (double)gfv * (-2.0 * (zz - c[0]));
                s2 += (double)gfv * (2.0 * (zz - c[1]));
            }
        }
        grad_f[o] = gfv;
    }
    const double a = block_sum1<256>(sl, s_red);
    const double b = block_sum1<256>(s1, s_red);
    const double d = block_sum1<256>(s2, s_red);
    if (threadIdx.x == 0) {
        red[3 * blockIdx.x] = a;
        red[3 * blockIdx.x + 1] = b;
        red[3 * blockIdx.x + 2] = d;
    }
}

static size_t adj_float_arrays() { return 11; }

}  // namespace seg

using namespace seg;

extern "C" size_t seg_state_bytes(int H, int ld, int64_t capacity, int mode, int storage) {
    if (mode == SEG_MODE_DENSE) return 6 * 4 * (size_t)std::max(H, 0) * (size_t)std::max(ld, 0) + 256;
    if (mode == SEG_MODE_TILED) return tiled_state_bytes(H, ld);
    size_t sz = storage_size(storage);
    return kCompactArrays * 256 + (size_t)compact_stride(capacity) * compact_per_element(sz);
}

extern "C" seg_status seg_solve(const float* f, int H, int W, int ld, const uint32_t* act,
                                const uint32_t* fgm, const int32_t* wstart, const int32_t* tiles,
                                const int32_t* counts, const seg_params* prm, float* u, float* v,
                                float* p1, float* p2, void* state, size_t state_bytes, double* stats,
                                void* ws, size_t ws_bytes, void* stream) {
    clear_error();
    PhaseScope _scope("seg_solve", stream, ws);
    SEG_TRY(check_params(prm));
    if (!f || !act || !fgm || !wstart || !tiles || !counts || !u || !v || !p1 || !p2 || !state || !stats)
        return fail(SEG_ERR_INVALID_ARG, "a required pointer is NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * ld >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d (H*ld < 2^31)", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    if (reinterpret_cast<uintptr_t>(state) % 16)
        return fail(SEG_ERR_ALIGN, "state buffer not 16-byte aligned");
    if (prm->mode == SEG_MODE_TILED) {
        int nwin = 0;
        SEG_TRY(tiled_geometry(H, W, prm->sweep, prm->n_inner, &nwin));
        if (reinterpret_cast<uintptr_t>(f) % 16) return fail(SEG_ERR_ALIGN, "f not 16-byte aligned");
    }
    WsLayout L = ws_layout(H, W, prm->tile_h);
    SEG_TRY(check_ws(ws, ws_bytes, L));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    double* partials = ws_at<double>(ws, L.partials);
    IterParams P = iter_params(prm, H, W, ld);

    k_solve_begin<<<1, 1, 0, s>>>(h);
    SEG_LAUNCHED("k_solve_begin");
    if (prm->mode == SEG_MODE_DENSE || prm->mode == SEG_MODE_TILED) {
        const size_t need = seg_state_bytes(H, ld, 0, prm->mode, SEG_STORE_F32);
        if (state_bytes < need)
            return fail(SEG_ERR_CAPACITY, "dense state needs %zu bytes, got %zu", need, state_bytes);
        float* st = static_cast<float*>(state);
        int64_t n = (int64_t)H * W;
        int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
        k_init_dense<<<blocks, 256, 0, s>>>(P, act, fgm, f, prm->warm_start, p1, p2, v, u, st);
        SEG_LAUNCHED("k_init_dense");
        if (prm->mode == SEG_MODE_TILED) {
            SEG_TRY(run_tiled(P, prm, act, f, u, v, p1, p2, st, partials, L.npartials, h, s));
        } else {
            SEG_TRY(run_dense(P, prm, counts, act, f, u, st, partials, h, s));
            k_final_dense<<<blocks, 256, 0, s>>>(P, h, prm->iters, prm->n_inner, st, v, p1, p2);
            SEG_LAUNCHED("k_final_dense");
        }
    } else {
        BatchDesc B{};
        B.n = 1;
        B.total_words = (long long)H * P.ntx;
        BatchImage& I = B.img[0];
        I.f = f; I.act = act; I.fg = fgm; I.wstart = wstart; I.counts = counts;
        I.u = u; I.v = v; I.p1 = p1; I.p2 = p2;
        I.word_off = 0; I.H = H; I.W = W; I.ld = ld; I.nw = ld / 32; I.ntx = P.ntx;
        I.theta_lambda = P.theta_lambda;
        int32_t* base = ws_at<int32_t>(ws, kWsBatchOff);
        SEG_TRY(solve_compact_any(P, prm, B, (int64_t)H * W, state, state_bytes, base, base + kMaxBatch + 2,
                                  partials, L.npartials, h, s));
        k_solve_end<<<1, 1, 0, s>>>(h, base + kMaxBatch + 2, prm->iters, stats);
        SEG_LAUNCHED("k_solve_end");
        return SEG_OK;
    }
    k_solve_end<<<1, 1, 0, s>>>(h, counts, prm->iters, stats);
    SEG_LAUNCHED("k_solve_end");
    return SEG_OK;
}

extern "C" size_t seg_batch_workspace_bytes(int n_images, int64_t max_pixels) {
    (void)n_images;
    // the fixed regions plus stopping-test partials for the persistent grid
    return align_up(kWsFixedBytes, 256) + 2 * 8 * (size_t)(4096 + 1) + 256 + 0 * (size_t)max_pixels;
}

extern "C" seg_status seg_solve_batch(const seg_image* images, int n_images, const seg_params* prm,
                                      void* state, size_t state_bytes, double* stats, void* ws,
                                      size_t ws_bytes, void* stream) {
    clear_error();
    PhaseScope _scope("seg_solve_batch", stream, ws);
    SEG_TRY(check_params(prm));
    if (prm->mode != SEG_MODE_COMPACT)
        return fail(SEG_ERR_INVALID_ARG, "seg_solve_batch runs SEG_MODE_COMPACT only");
    if (!images || n_images <= 0 || n_images > kMaxBatch)
        return fail(SEG_ERR_INVALID_ARG, "n_images=%d not in [1, %d]", n_images, kMaxBatch);
    if (!state || !stats) return fail(SEG_ERR_INVALID_ARG, "state and stats must be non-NULL");
    if (reinterpret_cast<uintptr_t>(state) % 16 || reinterpret_cast<uintptr_t>(ws) % 16)
        return fail(SEG_ERR_ALIGN, "state / workspace not 16-byte aligned");
    if (!ws || ws_bytes < seg_batch_workspace_bytes(n_images, 0))
        return fail(SEG_ERR_WORKSPACE, "batch workspace needs %zu bytes", seg_batch_workspace_bytes(n_images, 0));
    BatchDesc B{};
    B.n = n_images;
    long long words = 0, pixels = 0;
    for (int k = 0; k < n_images; ++k) {
        const seg_image& X = images[k];
        if (!X.f || !X.act || !X.fg || !X.wstart || !X.counts || !X.u || !X.v || !X.p1 || !X.p2)
            return fail(SEG_ERR_INVALID_ARG, "image %d: a required pointer is NULL", k);
        if (X.H <= 0 || X.W <= 0 || X.ld < X.W || (int64_t)X.H * X.ld >= (1ll << 31))
            return fail(SEG_ERR_INVALID_ARG, "image %d: bad size H=%d W=%d ld=%d", k, X.H, X.W, X.ld);
        if (X.ld % 32) return fail(SEG_ERR_ALIGN, "image %d: ld=%d is not a multiple of 32", k, X.ld);
        if (!std::isfinite(X.lambda)) return fail(SEG_ERR_INVALID_ARG, "image %d: lambda not finite", k);
        BatchImage& I = B.img[k];
        I.f = X.f; I.act = X.act; I.fg = X.fg; I.wstart = X.wstart; I.counts = X.counts;
        I.u = X.u; I.v = X.v; I.p1 = X.p1; I.p2 = X.p2;
        I.word_off = words; I.H = X.H; I.W = X.W; I.ld = X.ld; I.nw = X.ld / 32; I.ntx = (X.W + 31) / 32;
        I.theta_lambda = (float)(prm->theta * X.lambda);
        words += (long long)X.H * I.ntx;
        pixels += (long long)X.H * X.W;
    }
    B.total_words = words;
    if (pixels >= (1ll << 31)) return fail(SEG_ERR_INVALID_ARG, "batch holds %lld pixels (< 2^31)", pixels);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, kWsHeaderOff);
    int32_t* base = ws_at<int32_t>(ws, kWsBatchOff);
    double* partials = ws_at<double>(ws, align_up(kWsFixedBytes, 256));
    IterParams P = iter_params(prm, images[0].H, images[0].W, images[0].ld);
    k_solve_begin<<<1, 1, 0, s>>>(h);
    SEG_LAUNCHED("k_solve_begin");
    SEG_TRY(solve_compact_any(P, prm, B, pixels, state, state_bytes, base, base + kMaxBatch + 2, partials,
                              4096, h, s));
    k_solve_end<<<1, 1, 0, s>>>(h, base + kMaxBatch + 2, prm->iters, stats);
    SEG_LAUNCHED("k_solve_end");
    return SEG_OK;
}


// ----------------------------------------------------- differentiable solve

extern "C" size_t seg_ckpt_bytes(int64_t capacity, int iters, int ckpt_every) {
    if (ckpt_every < 1 || iters < 0) return 0;
    const int64_t m = std::max(1, (iters + ckpt_every - 1) / ckpt_every);
    return (size_t)m * 3 * 4 * (size_t)compact_stride(capacity) + 256;
}

extern "C" size_t seg_backward_scratch_bytes(int64_t capacity, int ckpt_every) {
    const int64_t st = compact_stride(capacity);
    return (adj_float_arrays() + 8 * (size_t)(std::max(ckpt_every, 1) + 1)) * 4 * (size_t)st + 16 * 256;
}

extern "C" seg_status seg_solve_diff(const float* f, int H, int W, int ld, const uint32_t* act,
                                     const uint32_t* fgm, const int32_t* wstart, const int32_t* tiles,
                                     const int32_t* counts, const seg_params* prm, float* u, float* v,
                                     float* p1, float* p2, void* state, size_t state_bytes,
                                     int ckpt_every, void* ckpt, size_t ckpt_bytes, double* stats,
                                     void* ws, size_t ws_bytes, void* stream) {
    clear_error();
    PhaseScope _scope("seg_solve_diff", stream, ws);
    SEG_TRY(check_params(prm));
    if (prm->mode != SEG_MODE_COMPACT || prm->storage != SEG_STORE_F32 || prm->n_inner != 1 ||
        prm->warm_start || prm->tol > 0)
        return fail(SEG_ERR_INVALID_ARG,
                    "seg_solve_diff: compact mode, float32 storage, n_inner = 1, cold start, tol <= 0");
    if (!f || !act || !fgm || !wstart || !tiles || !counts || !u || !v || !p1 || !p2 || !state || !stats ||
        !ckpt)
        return fail(SEG_ERR_INVALID_ARG, "a required pointer is NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * ld >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    if (ckpt_every < 1) return fail(SEG_ERR_INVALID_ARG, "ckpt_every must be >= 1");
    CompactLayout C = compact_layout(state_bytes, prm->storage);
    if (ckpt_bytes < seg_ckpt_bytes(C.cap, prm->iters, ckpt_every))
        return fail(SEG_ERR_CAPACITY, "checkpoints need %zu bytes", seg_ckpt_bytes(C.cap, prm->iters, ckpt_every));
    WsLayout L = ws_layout(H, W, prm->tile_h);
    SEG_TRY(check_ws(ws, ws_bytes, L));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    double* partials = ws_at<double>(ws, L.partials);
    IterParams P = iter_params(prm, H, W, ld);
    BatchDesc B{};
    B.n = 1;
    B.total_words = (long long)H * P.ntx;
    BatchImage& I = B.img[0];
    I.f = f; I.act = act; I.fg = fgm; I.wstart = wstart; I.counts = counts;
    I.u = u; I.v = v; I.p1 = p1; I.p2 = p2;
    I.word_off = 0; I.H = H; I.W = W; I.ld = ld; I.nw = ld / 32; I.ntx = P.ntx;
    I.theta_lambda = P.theta_lambda;
    int32_t* base = ws_at<int32_t>(ws, kWsBatchOff);
    k_solve_begin<<<1, 1, 0, s>>>(h);
    SEG_LAUNCHED("k_solve_begin");
    SEG_TRY(solve_compact_batch<float>(P, prm, B, (int64_t)H * W, state, state_bytes, base,
                                       base + kMaxBatch + 2, partials, L.npartials, h, s,
                                       static_cast<float*>(ckpt), ckpt_every));
    k_solve_end<<<1, 1, 0, s>>>(h, base + kMaxBatch + 2, prm->iters, stats);
    SEG_LAUNCHED("k_solve_end");
    return SEG_OK;
}

// The adjoint of a batch of images solved together by the differentiable
// forward (a single image is a batch of one): gathers dL/du^K, dL/dv^K of
// every image into compact order, one persistent reverse sweep over the
// whole compact range (the images' iterations are independent and lambda
// only enters through F = theta lambda_k f, so the sweep needs no per-image
// data), then dL/df and the FP64 sums of every image.  base: device array
// of the images' compact bases (base[k], and the total RD pixels in
// totals[1]); launched on stream s after the header's reset.
static seg_status backward_batch(const seg_params* prm, const BatchDesc& B, const seg_adj_image* adj,
                                 const int32_t* base, const int32_t* totals, const void* state,
                                 size_t state_bytes, const void* ckpt, int ckpt_every, void* scratch,
                                 double* red, WsHeader* h, cudaStream_t s) {
    CompactLayout C = compact_layout(state_bytes, prm->storage);
    const char* sb = static_cast<const char*>(state);
    const float* F = reinterpret_cast<const float*>(sb + C.off[5]);
    const int32_t* nbp = reinterpret_cast<const int32_t*>(sb + C.off[8]);
    int64_t stride = C.stride;
    AdjArrays A{};
    float* sc = static_cast<float*>(scratch);
    float** fields[] = {&A.p1b, &A.p2b, &A.vb, &A.ub, &A.gb1, &A.gb2, &A.pd1, &A.pd2, &A.fb, &A.gu, &A.gv};
    for (size_t k = 0; k < adj_float_arrays(); ++k) *fields[k] = sc + k * stride;
    A.seg = sc + adj_float_arrays() * stride;
    A.seg2 = A.seg + 4 * (int64_t)(ckpt_every + 1) * stride;
    int64_t pixels = 0;
    for (int k = 0; k < B.n; ++k) {
        const BatchImage& I = B.img[k];
        IterParams Pk = iter_params(prm, I.H, I.W, I.ld);
        const int64_t nwords = (int64_t)I.H * Pk.ntx;
        const unsigned gblocks = (unsigned)((nwords + 7) / 8);
        k_adj_gather<<<gblocks, 256, 0, s>>>(Pk, I.act, I.wstart, B.n > 1 ? base + k : nullptr, adj[k].grad_u,
                                             adj[k].grad_v, A);
        SEG_LAUNCHED("k_adj_gather");
        pixels += (int64_t)I.H * I.W;
    }
    // the tables in shared memory when every block's share of the largest
    // possible RD fits (otherwise no shared memory: the L1 keeps it for the
    // global path)
    const int64_t most = std::max<int64_t>(1, std::min<int64_t>(C.cap, pixels));
    const void* ks = (const void*)k_backward_compact<true>;
    SEG_TRY_CUDA(cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmemBytes));
    int per_sm = 0;
    SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks, kBackwardThreadsSm, kAdjSmemBytes));
    if (per_sm <= 0) return fail(SEG_ERR_CUDA, "k_backward_compact cannot be resident");
    int grid = (int)std::min<int64_t>((int64_t)per_sm * sm_count(),
                                      std::max<int64_t>(1, (most + kBackwardThreadsSm - 1) / kBackwardThreadsSm));
    const bool use_smem = (most + grid - 1) / grid <= kAdjSmemPixels;
    const void* kern = use_smem ? ks : (const void*)k_backward_compact<false>;
    const int threads = use_smem ? kBackwardThreadsSm : kBackwardThreads;
    if (!use_smem) {
        int pg = 0;
        SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pg, kern, kBackwardThreads, 0));
        if (pg <= 0) return fail(SEG_ERR_CUDA, "k_backward_compact cannot be resident");
        grid = (int)std::min<int64_t>((int64_t)pg * sm_count(),
                                      std::max<int64_t>(1, (most + kBackwardThreads - 1) / kBackwardThreads));
    }
    const size_t smem = use_smem ? kAdjSmemBytes : 0;
    IterParams P = iter_params(prm, B.img[0].H, B.img[0].W, B.img[0].ld);
    int iters = prm->iters, ce = ckpt_every;
    const float* ck = static_cast<const float*>(ckpt);
    const int32_t* cnt = totals;
    void* args[] = {&P, &iters, &ce, (void*)&cnt, (void*)&nbp, &stride, (void*)&F, (void*)&ck, &A, &h};
    if (iters > 0) {
        SEG_TRY_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, smem, s));
        count_launch();
        if (debug_mode()) SEG_TRY(after_launch("persistent solve"));
    }
    for (int k = 0; k < B.n; ++k) {
        const BatchImage& I = B.img[k];
        IterParams Pk = iter_params(prm, I.H, I.W, I.ld);
        k_adj_scatter<<<kReduceBlocks, 256, 0, s>>>(Pk, I.f, I.act, I.wstart, B.n > 1 ? base + k : nullptr, A.fb,
                                                    adj[k].z, adj[k].c, I.theta_lambda, adj[k].grad_f, red);
        SEG_LAUNCHED("k_adj_scatter");
        SEG_TRY(reduce_partials(red, kReduceBlocks, 3, adj[k].grad_out, s));
    }
    return SEG_OK;
}

static seg_status check_diff_params(const seg_params* prm, const char* who) {
    SEG_TRY(check_params(prm));
    if (prm->mode != SEG_MODE_COMPACT || prm->storage != SEG_STORE_F32 || prm->n_inner != 1 ||
        prm->warm_start || prm->tol > 0)
        return fail(SEG_ERR_INVALID_ARG, "%s: compact mode, float32 storage, n_inner = 1, cold start, tol <= 0",
                    who);
    return SEG_OK;
}

extern "C" seg_status seg_backward(const float* f, int H, int W, int ld, const uint32_t* act,
                                   const uint32_t* fgm, const int32_t* wstart, const int32_t* counts,
                                   const seg_params* prm, const void* state, size_t state_bytes,
                                   const void* ckpt, size_t ckpt_bytes, int ckpt_every,
                                   const float* grad_u, const float* grad_v, const float* z,
                                   const double* c, float* grad_f, double* grad_out, void* scratch,
                                   size_t scratch_bytes, void* ws, size_t ws_bytes, void* stream) {
    clear_error();
    PhaseScope _scope("seg_backward", stream, ws);
    SEG_TRY(check_params(prm));
    if (prm->mode != SEG_MODE_COMPACT || prm->storage != SEG_STORE_F32 || prm->n_inner != 1)
        return fail(SEG_ERR_INVALID_ARG, "seg_backward: compact mode, float32 storage, n_inner = 1");
    if (!f || !act || !fgm || !wstart || !counts || !state || !ckpt || !grad_u || !grad_f || !grad_out ||
        !scratch || (z && !c))
        return fail(SEG_ERR_INVALID_ARG, "a required pointer is NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * ld >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    if (ckpt_every < 1) return fail(SEG_ERR_INVALID_ARG, "ckpt_every must be >= 1");
    CompactLayout C = compact_layout(state_bytes, prm->storage);
    if (ckpt_bytes < seg_ckpt_bytes(C.cap, prm->iters, ckpt_every))
        return fail(SEG_ERR_CAPACITY, "checkpoint buffer smaller than the forward wrote");
    if (scratch_bytes < seg_backward_scratch_bytes(C.cap, ckpt_every))
        return fail(SEG_ERR_WORKSPACE, "backward scratch needs %zu bytes",
                    seg_backward_scratch_bytes(C.cap, ckpt_every));
    if (reinterpret_cast<uintptr_t>(scratch) % 16)
        return fail(SEG_ERR_ALIGN, "scratch not 16-byte aligned");
    WsLayout L = ws_layout(H, W, prm->tile_h);
    SEG_TRY(check_ws(ws, ws_bytes, L));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    BatchDesc B{};
    B.n = 1;
    BatchImage& I = B.img[0];
    I.f = f; I.act = act; I.fg = fgm; I.wstart = wstart; I.counts = counts;
    I.H = H; I.W = W; I.ld = ld; I.nw = ld / 32; I.ntx = (W + 31) / 32;
    I.theta_lambda = (float)(prm->theta * prm->lambda);
    seg_adj_image adj{grad_u, grad_v, z, c, grad_f, grad_out};
    k_solve_begin<<<1, 1, 0, s>>>(h);
    SEG_LAUNCHED("k_solve_begin");
    return backward_batch(prm, B, &adj, nullptr, counts, state, state_bytes, ckpt, ckpt_every, scratch,
                          ws_at<double>(ws, kWsRedOff), h, s);
}

// The images of a batch as BatchDesc (checks of seg_solve_batch).
static seg_status batch_desc(const seg_image* images, int n_images, const seg_params* prm, BatchDesc& B,
                             long long& pixels) {
    if (!images || n_images <= 0 || n_images > kMaxBatch)
        return fail(SEG_ERR_INVALID_ARG, "n_images=%d not in [1, %d]", n_images, kMaxBatch);
    B = BatchDesc{};
    B.n = n_images;
    long long words = 0;
    pixels = 0;
    for (int k = 0; k < n_images; ++k) {
        const seg_image& X = images[k];
        if (!X.f || !X.act || !X.fg || !X.wstart || !X.counts || !X.u || !X.v || !X.p1 || !X.p2)
            return fail(SEG_ERR_INVALID_ARG, "image %d: a required pointer is NULL", k);
        if (X.H <= 0 || X.W <= 0 || X.ld < X.W || (int64_t)X.H * X.ld >= (1ll << 31))
            return fail(SEG_ERR_INVALID_ARG, "image %d: bad size H=%d W=%d ld=%d", k, X.H, X.W, X.ld);
        if (X.ld % 32) return fail(SEG_ERR_ALIGN, "image %d: ld=%d is not a multiple of 32", k, X.ld);
        if (!std::isfinite(X.lambda)) return fail(SEG_ERR_INVALID_ARG, "image %d: lambda not finite", k);
        BatchImage& I = B.img[k];
        I.f = X.f; I.act = X.act; I.fg = X.fg; I.wstart = X.wstart; I.counts = X.counts;
        I.u = X.u; I.v = X.v; I.p1 = X.p1; I.p2 = X.p2;
        I.word_off = words; I.H = X.H; I.W = X.W; I.ld = X.ld; I.nw = X.ld / 32; I.ntx = (X.W + 31) / 32;
        I.theta_lambda = (float)(prm->theta * X.lambda);
        words += (long long)X.H * I.ntx;
        pixels += (long long)X.H * X.W;
    }
    B.total_words = words;
    if (pixels >= (1ll << 31)) return fail(SEG_ERR_INVALID_ARG, "batch holds %lld pixels (< 2^31)", pixels);
    return SEG_OK;
}

extern "C" seg_status seg_solve_diff_batch(const seg_image* images, int n_images, const seg_params* prm,
                                           void* state, size_t state_bytes, int ckpt_every, void* ckpt,
                                           size_t ckpt_bytes, double* stats, void* ws, size_t ws_bytes,
                                           void* stream) {
    clear_error();
    PhaseScope _scope("seg_solve_diff_batch", stream, ws);
    SEG_TRY(check_diff_params(prm, "seg_solve_diff_batch"));
    if (!state || !stats || !ckpt) return fail(SEG_ERR_INVALID_ARG, "state, ckpt and stats must be non-NULL");
    if (reinterpret_cast<uintptr_t>(state) % 16 || reinterpret_cast<uintptr_t>(ws) % 16 ||
        reinterpret_cast<uintptr_t>(ckpt) % 16)
        return fail(SEG_ERR_ALIGN, "state / ckpt / workspace not 16-byte aligned");
    if (!ws || ws_bytes < seg_batch_workspace_bytes(n_images, 0))
        return fail(SEG_ERR_WORKSPACE, "batch workspace needs %zu bytes", seg_batch_workspace_bytes(n_images, 0));
    if (ckpt_every < 1) return fail(SEG_ERR_INVALID_ARG, "ckpt_every must be >= 1");
    BatchDesc B;
    long long pixels = 0;
    SEG_TRY(batch_desc(images, n_images, prm, B, pixels));
    CompactLayout C = compact_layout(state_bytes, prm->storage);
    if (ckpt_bytes < seg_ckpt_bytes(C.cap, prm->iters, ckpt_every))
        return fail(SEG_ERR_CAPACITY, "checkpoints need %zu bytes", seg_ckpt_bytes(C.cap, prm->iters, ckpt_every));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, kWsHeaderOff);
    int32_t* base = ws_at<int32_t>(ws, kWsBatchOff);
    double* partials = ws_at<double>(ws, align_up(kWsFixedBytes, 256));
    IterParams P = iter_params(prm, images[0].H, images[0].W, images[0].ld);
    k_solve_begin<<<1, 1, 0, s>>>(h);
    SEG_LAUNCHED("k_solve_begin");
    SEG_TRY(solve_compact_batch<float>(P, prm, B, pixels, state, state_bytes, base, base + kMaxBatch + 2,
                                       partials, 4096, h, s, static_cast<float*>(ckpt), ckpt_every));
    k_solve_end<<<1, 1, 0, s>>>(h, base + kMaxBatch + 2, prm->iters, stats);
    SEG_LAUNCHED("k_solve_end");
    return SEG_OK;
}

extern "C" seg_status seg_backward_batch(const seg_image* images, const seg_adj_image* adj, int n_images,
                                         const seg_params* prm, const void* state, size_t state_bytes,
                                         const void* ckpt, size_t ckpt_bytes, int ckpt_every, void* scratch,
                                         size_t scratch_bytes, void* ws, size_t ws_bytes, void* stream) {
    clear_error();
    PhaseScope _scope("seg_backward_batch", stream, ws);
    SEG_TRY(check_params(prm));
    if (prm->mode != SEG_MODE_COMPACT || prm->storage != SEG_STORE_F32 || prm->n_inner != 1)
        return fail(SEG_ERR_INVALID_ARG, "seg_backward_batch: compact mode, float32 storage, n_inner = 1");
    if (!adj || !state || !ckpt || !scratch) return fail(SEG_ERR_INVALID_ARG, "a required pointer is NULL");
    BatchDesc B;
    long long pixels = 0;
    SEG_TRY(batch_desc(images, n_images, prm, B, pixels));
    for (int k = 0; k < n_images; ++k)
        if (!adj[k].grad_u || !adj[k].grad_f || !adj[k].grad_out || (adj[k].z && !adj[k].c))
            return fail(SEG_ERR_INVALID_ARG, "image %d: a required adjoint pointer is NULL", k);
    if (ckpt_every < 1) return fail(SEG_ERR_INVALID_ARG, "ckpt_every must be >= 1");
    if (!ws || ws_bytes < seg_batch_workspace_bytes(n_images, 0))
        return fail(SEG_ERR_WORKSPACE, "batch workspace needs %zu bytes", seg_batch_workspace_bytes(n_images, 0));
    if (reinterpret_cast<uintptr_t>(scratch) % 16 || reinterpret_cast<uintptr_t>(ws) % 16)
        return fail(SEG_ERR_ALIGN, "scratch / workspace not 16-byte aligned");
    CompactLayout C = compact_layout(state_bytes, prm->storage);
    if (ckpt_bytes < seg_ckpt_bytes(C.cap, prm->iters, ckpt_every))
        return fail(SEG_ERR_CAPACITY, "checkpoint buffer smaller than the forward wrote");
    if (scratch_bytes < seg_backward_scratch_bytes(C.cap, ckpt_every))
        return fail(SEG_ERR_WORKSPACE, "backward scratch needs %zu bytes",
                    seg_backward_scratch_bytes(C.cap, ckpt_every));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, kWsHeaderOff);
    int32_t* base = ws_at<int32_t>(ws, kWsBatchOff);
    k_solve_begin<<<1, 1, 0, s>>>(h);
    SEG_LAUNCHED("k_solve_begin");
    // the compact bases of the forward, recomputed from the domains' counts
    k_batch_bases<<<1, 1, 0, s>>>(B, base, base + kMaxBatch + 2, C.cap, h);
    SEG_LAUNCHED("k_batch_bases");
    return backward_batch(prm, B, adj, base, base + kMaxBatch + 2, state, state_bytes, ckpt, ckpt_every,
                          scratch, ws_at<double>(ws, kWsRedOff), h, s);
}

// ================================================== restricted primal-dual
//
// The Conclusion proposes carrying the domain restriction over to other
// solvers of Eq. CR.  This is the primal-dual method of Chambolle and Pock
// (2011) on the same compact RD machinery, with Section 3's restriction (p =
// 0 outside RD, u fixed to H(-f) there):
//   dual    p <- P(p + sigma grad ubar),  P the projection onto |p| <= 1
//   primal  u' = clip(u + tau div p - tau lambda f, 0, 1),  ubar = 2 u' - u
// from u0 = H(-f) (or the caller's u, p), ubar0 = u0.  Every step reads its
// own pixel's old value from one buffer and writes the new value to the
// other (p and u are ping-ponged; ubar is written only by the primal step
// and read only by the dual one), two grid barriers per iteration, and the
// Section 4 test on max(||u' - u||, ||p' - p||) every check_every iterations.
// The neighbour table, f (premultiplied by tau lambda) and the start
// iterate come from k_compact_gather; the state is the compact state's
// arrays: p1[0..1], p2[0..1], u (U0), w (U1), up (ubar), f.

constexpr int kPdThreads = 1024;   // two blocks per SM (32 registers): latency-bound loads
constexpr int kPdSmThreads = 512;  // the shared-memory kernel: two blocks per SM, 112 KB each

__device__ __forceinline__ float pd_fixed(int code) { return code == kNbFg ? 1.f : 0.f; }

// The primal-dual iteration on the global arrays (two grid barriers per
// iteration); gen: barriers passed so far.
template <int NT>
__device__ __forceinline__ void pd_iterations(int iters, int check_every, double tol, float sigma, float tau,
                                              int n, const int32_t* __restrict__ nb, int64_t stride,
                                              float* P1a, float* P1b, float* P2a, float* P2b, float* U0,
                                              float* U1, float* Ub, const float* __restrict__ F,
                                              double* partials, WsHeader* h, double* s_red, unsigned& gen) {
    const unsigned nblocks = gridDim.x;
    const int per = (n + (int)nblocks - 1) / (int)nblocks;
    const int a0 = (int)blockIdx.x * per, a1 = min(n, a0 + per);
    const int tid = threadIdx.x;
    const int C = check_every;
    int chk = 0;
    for (int l = 1; l <= iters; ++l) {
        const bool check = (l % C == 0) || l == iters;
        // iterate l - 1 lives in buffer (l - 1) & 1
        const float* P1i = (l & 1) ? P1a : P1b;
        const float* P2i = (l & 1) ? P2a : P2b;
        float* P1o = (l & 1) ? P1b : P1a;
        float* P2o = (l & 1) ? P2b : P2a;
        const float* Ui = (l & 1) ? U0 : U1;
        float* Uo = (l & 1) ? U1 : U0;
        float du2 = 0.f, dp2 = 0.f;
        for (int a = a0 + tid; a < a1; a += NT) {
            const int nd = __ldg(nb + NB_DOWN * stride + a), nr = __ldg(nb + NB_RIGHT * stride + a);
            const float ub = Ub[a];
            float g1 = 0.f, g2 = 0.f;
            if (nd != kNbOut) g1 = (nd >= 0 ? Ub[nd] : pd_fixed(nd)) - ub;
            if (nr != kNbOut) g2 = (nr >= 0 ? Ub[nr] : pd_fixed(nr)) - ub;
            const float p1 = P1i[a], p2 = P2i[a];
            float q1 = fmaf(sigma, g1, p1), q2 = fmaf(sigma, g2, p2);
            const float s2 = fmaf(q1, q1, q2 * q2);
            if (s2 > 1.f) {
                const float r = rsqrtf(s2);
                q1 *= r;
                q2 *= r;
            }
            P1o[a] = q1;
            P2o[a] = q2;
            if (check) {
                const float d1 = q1 - p1, d2 = q2 - p2;
                dp2 = fmaf(d1, d1, fmaf(d2, d2, dp2));
            }
        }
        if (!grid_sync(h, nblocks, gen)) return;
        for (int a = a0 + tid; a < a1; a += NT) {
            const int nu = __ldg(nb + NB_UP * stride + a), nl = __ldg(nb + NB_LEFT * stride + a);
            const float q1 = P1o[a], q2 = P2o[a];
            const float q1u = nu >= 0 ? P1o[nu] : 0.f, q2l = nl >= 0 ? P2o[nl] : 0.f;
            const float div = (q1 - q1u) + (q2 - q2l);
            const float uo = Ui[a];
            const float un = clamp01(fmaf(tau, div, uo) - __ldg(F + a));   // F = tau lambda f
            Uo[a] = un;
            Ub[a] = fmaf(2.f, un, -uo);
            if (check) {
                const float d = un - uo;
                du2 = fmaf(d, d, du2);
            }
        }
        double* part = partials + 2 * (int64_t)nblocks * (chk & 1);
        if (check) {
            float x = du2, y = dp2;
            block_sum2f<NT>(x, y, reinterpret_cast<float*>(s_red));
            if (tid == 0) {
                part[2 * blockIdx.x] = x;
                part[2 * blockIdx.x + 1] = y;
            }
        }
        if (!grid_sync(h, nblocks, gen)) return;
        if (check) {
            // every block sums the partials in the same order and stops at
            // the same iteration
            if (tid < 32) {
                double sx, sy;
                sum_partials_warp0(part, (int)nblocks, sx, sy);
                if (tid == 0) {
                    const bool stop = tol > 0.0 && fmax(sx, sy) <= tol * tol;
                    s_red[0] = stop ? 1.0 : 0.0;
                    if (blockIdx.x == 0) {
                        h->du2 = sx;
                        h->dv2 = sy;
                        h->last_check = l;
                        if (stop) {
                            h->iters_done = l;
                            h->done = 1;
                        }
                    }
                }
            }
            __syncthreads();
            const bool stop = s_red[0] != 0.0;
            ++chk;
            __syncthreads();
            if (stop) return;
        }
    }
}

// ---- the primal-dual iteration with shared-memory state and one grid barrier
//
// The layout and protocol of the one-barrier dual iteration (compact_solve_h1)
// with u-bar in the part of w and u in that of v: each block keeps p (both
// buffers), u-bar and u of its pixels and of its ring (the pixels other
// blocks own directly above or left of its own; u of its own pixels only) in
// shared memory and runs the ring's dual steps too, so the primal step
// follows after a block barrier.  The dual step reads p only at its own
// pixel (a fixed neighbour contributes its fixed u, not p flowing into it),
// so the ring's p is read once, at the start, and p has no ghost words; the
// ghost words are u-bar below / right of the block's pixels and of its ring,
// and u-bar of the ring, refilled each iteration from the previous iterate,
// which the global arrays keep in ping-pong buffers (written for the pixels
// other blocks read).  The grid barrier is split as in
// compact_iterations_h1; every block takes the Section 4 decision.  The
// iterates are bit-identical to pd_iterations'.
struct PdLayout {
    int n, r, nE;          // own pixels, ring pixels, n + r
    int nsp, nsu;          // region sizes (words): P1 / P2 per buffer [own | ring | zero], UB [own | ring | zero | ghosts]
    int p1, p2, ub, u;     // word offsets of the regions (U: own pixels)
    int ng, nbd;           // ghost words refilled per iteration; own pixels whose dual step reads one
    size_t off16, offfl, offr1, offgs, offgd, offbd, bytes;
};

struct PdSmem {
    float* sm;
    const uint16_t* off;   // [D: nE][R: nE][UP: n][LEFT: n] word offsets (p words: buffer 0)
    const uint8_t* fl;     // [nE]: classes below / right (bits 0-3), kFlExport, kFlDualGhost
    const int32_t* r1;     // [r] compact index of each ring pixel
    const int32_t* gsrc;   // [ng] compact index of each ghost's pixel
    const uint16_t* gdst;  // [ng] word offset of each ghost
    const uint16_t* bd;    // [nbd] own pixels whose dual step reads a ghost
    PdLayout L;
};

// Dual step of entry i: p' = P(p + sigma grad u-bar), the fixed neighbours'
// u-bar their fixed u (selects, the values of pd_iterations' branches); dp2
// accumulates |p' - p|^2 when acc.
__device__ __forceinline__ void pd_dual_sm(const PdSmem& S, int i, uint8_t fl, const float* P1, const float* P2,
                                           float* Q1, float* Q2, float sigma, bool acc, float& dp2) {
    const float ub0 = S.sm[S.L.ub + i];
    const float xd = S.sm[S.off[i]], xr = S.sm[S.off[S.L.nE + i]];
    const int cd = fl & 3, cr = (fl >> 2) & 3;   // 0 RD, 1 fixed Bg, 2 fixed Fg, 3 outside
    const float ud = cd == 0 ? xd : (cd == 2 ? 1.f : 0.f);
    const float ur = cr == 0 ? xr : (cr == 2 ? 1.f : 0.f);
    const float g1 = cd == 3 ? 0.f : ud - ub0;
    const float g2 = cr == 3 ? 0.f : ur - ub0;
    const float p1 = P1[i], p2 = P2[i];
    float q1 = fmaf(sigma, g1, p1), q2 = fmaf(sigma, g2, p2);
    const float s2 = fmaf(q1, q1, q2 * q2);
    const float r = s2 > 1.f ? rsqrtf(s2) : 1.f;
    q1 *= r;
    q2 *= r;
    Q1[i] = q1;
    Q2[i] = q2;
    if (acc) {
        const float d1 = q1 - p1, d2 = q2 - p2;
        dp2 = fmaf(d1, d1, fmaf(d2, d2, dp2));
    }
}

// Primal step of own pixel i (compact index a): u' = clip(u + tau div p' -
// tau lambda f), u-bar' = 2u' - u (exported when other blocks read it); fa
// = tau lambda f(a).
__device__ __forceinline__ void pd_primal_sm(const PdSmem& S, int i, int a, const float* Q1, const float* Q2,
                                             int sh, float tau, float fa, float* Ubo, bool check, float& du2) {
    const float q1 = Q1[i], q2 = Q2[i];
    const float q1u = S.sm[S.off[2 * S.L.nE + i] + sh], q2l = S.sm[S.off[2 * S.L.nE + S.L.n + i] + sh];
    const float div = (q1 - q1u) + (q2 - q2l);
    float* U = S.sm + S.L.u;
    const float uo = U[i];
    const float un = clamp01(fmaf(tau, div, uo) - fa);   // fa = tau lambda f at a
    U[i] = un;
    const float ubn = fmaf(2.f, un, -uo);
    S.sm[S.L.ub + i] = ubn;
    if (S.fl[i] & kFlExport) Ubo[a] = ubn;
    if (check) {
        const float d = un - uo;
        du2 = fmaf(d, d, du2);
    }
}

// Sets up and runs the shared-memory primal-dual iteration when every block's
// state fits (a grid-wide vote).  Returns 1 when it ran the solve, 0 when
// some block does not fit (nothing changed), -1 when a barrier timed out.
template <int NT>
__device__ __forceinline__ int pd_solve_sm(int iters, int check_every, double tol, float sigma, float tau, int n,
                                           const int32_t* __restrict__ nb, int64_t stride, float* P1a,
                                           float* P1b, float* P2a, float* P2b, float* U0, float* U1, float* Ub,
                                           float* Ub2, const float* __restrict__ F, double* partials,
                                           WsHeader* h, double* s_red, unsigned char* c_smem, unsigned& gen) {
    const unsigned nblocks = gridDim.x;
    const int tid = threadIdx.x, nt = NT;
    const int per = (n + (int)nblocks - 1) / (int)nblocks;
    const int a0 = (int)blockIdx.x * per, a1 = min(n, a0 + per);
    const int nown = max(a1 - a0, 0);
    auto other = [&](int m) { return m >= 0 && (m < a0 || m >= a1); };
    auto dr_src = [&](int a, int k) { return __ldg(nb + (k == GK_D ? NB_DOWN : NB_RIGHT) * stride + a); };
    // counts: [0] ring pixels, [1] u-bar ghost words past the ring's, [2] ghosts own pixels read
    __shared__ int s_h[4];
    if (tid < 4) s_h[tid] = 0;
    __syncthreads();
    {
        int r = 0, gu = 0, go = 0;
        for (int i = tid; i < nown; i += nt) {
            const int a = a0 + i;
#pragma unroll
            for (int k = GK_D; k <= GK_R; ++k)
                if (other(dr_src(a, k))) { ++gu; ++go; }
#pragma unroll
            for (int k = GK_UP; k <= GK_LEFT; ++k) {
                const int y = __ldg(nb + (k == GK_UP ? NB_UP : NB_LEFT) * stride + a);
                if (!other(y)) continue;
                ++r;
#pragma unroll
                for (int k2 = GK_D; k2 <= GK_R; ++k2)
                    if (other(dr_src(y, k2))) ++gu;
            }
        }
        if (r) atomicAdd(&s_h[0], r);
        if (gu) atomicAdd(&s_h[1], gu);
        if (go) atomicAdd(&s_h[2], go);
    }
    __syncthreads();
    PdLayout L{};
    L.n = nown;
    L.r = s_h[0];
    L.nE = nown + L.r;
    const int gux = s_h[1];
    L.ng = gux + L.r;   // plus u-bar of every ring pixel
    L.nsp = L.nE + 1;
    L.nsu = L.nE + 1 + gux;
    L.p1 = 0;
    L.p2 = 2 * L.nsp;
    L.ub = L.p2 + 2 * L.nsp;
    L.u = L.ub + L.nsu;
    const int words = L.u + nown;
    L.off16 = (size_t)4 * words;
    L.offfl = L.off16 + (size_t)2 * (2 * L.nE + 2 * nown);
    L.offr1 = (L.offfl + L.nE + 3) & ~(size_t)3;
    L.offgs = L.offr1 + (size_t)4 * L.r;
    L.offgd = L.offgs + (size_t)4 * L.ng;
    L.offbd = L.offgd + (size_t)2 * L.ng;
    L.bytes = L.offbd + (size_t)2 * min(nown, s_h[2]);
    const bool fits = L.bytes <= compact_smem(NT) && words < 65536 && L.ng <= kGhostRegs * NT;
    __shared__ unsigned s_vote;
    if (tid == 0 && !fits) atomicAdd(&h->h1_vote, 1u);
    if (!grid_sync(h, nblocks, gen)) return -1;
    if (tid == 0) s_vote = *(volatile unsigned*)&h->h1_vote;
    __syncthreads();
    const bool all_fit = s_vote == 0u;
    __syncthreads();
    if (!all_fit) return 0;

    unsigned* mark = reinterpret_cast<unsigned*>(Ub2);   // export marks, before Ub2 holds u-bar
    for (int i = tid; i < nown; i += nt) mark[a0 + i] = 0u;
    float* sm = reinterpret_cast<float*>(c_smem);
    uint16_t* off = reinterpret_cast<uint16_t*>(c_smem + L.off16);
    uint8_t* flg = reinterpret_cast<uint8_t*>(c_smem + L.offfl);
    int32_t* r1 = reinterpret_cast<int32_t*>(c_smem + L.offr1);
    int32_t* gsrc = reinterpret_cast<int32_t*>(c_smem + L.offgs);
    uint16_t* gdst = reinterpret_cast<uint16_t*>(c_smem + L.offgd);
    uint16_t* lbd = reinterpret_cast<uint16_t*>(c_smem + L.offbd);
    if (tid < 4) s_h[tid] = 0;   // [0] ring slots, [1] ghost area words, [2] ghost slots
    if (tid == 0) {
        sm[L.p1 + L.nE] = 0.f; sm[L.p1 + L.nsp + L.nE] = 0.f;
        sm[L.p2 + L.nE] = 0.f; sm[L.p2 + L.nsp + L.nE] = 0.f;
        sm[L.ub + L.nE] = 0.f;
    }
    __syncthreads();
    // the u-bar word a D / R read of pixel a uses (a ghost word when another block owns it)
    auto dr_off = [&](int a, int k, bool& ghost) {
        const int m = dr_src(a, k);
        ghost = false;
        if (m >= a0 && m < a1) return L.ub + (m - a0);
        if (m < 0) return L.ub + L.nE;   // fixed or outside: the class is in the flags
        ghost = true;
        const int o = L.ub + L.nE + 1 + atomicAdd(&s_h[1], 1);
        const int slot = atomicAdd(&s_h[2], 1);
        gsrc[slot] = m;
        gdst[slot] = (uint16_t)o;
        return o;
    };
    for (int i = tid; i < nown; i += nt) {
        const int a = a0 + i;
        bool gd = false, g;
        off[i] = (uint16_t)dr_off(a, GK_D, g);
        gd |= g;
        off[L.nE + i] = (uint16_t)dr_off(a, GK_R, g);
        gd |= g;
        flg[i] = (uint8_t)(gk_codes(nb, stride, a) | (gd ? kFlDualGhost : 0));
#pragma unroll
        for (int k = GK_UP; k <= GK_LEFT; ++k) {
            const int y = __ldg(nb + (k == GK_UP ? NB_UP : NB_LEFT) * stride + a);
            const int base = k == GK_UP ? L.p1 : L.p2;
            int o;
            if (y >= a0 && y < a1) {
                o = base + (y - a0);
            } else if (y < 0) {
                o = base + L.nE;
            } else {   // a ring pixel: p read once, u-bar a ghost
                const int j = atomicAdd(&s_h[0], 1);
                const int e = nown + j;
                o = base + e;
                r1[j] = y;
                off[e] = (uint16_t)dr_off(y, GK_D, g);
                off[L.nE + e] = (uint16_t)dr_off(y, GK_R, g);
                flg[e] = gk_codes(nb, stride, y);
                sm[L.p1 + e] = P1a[y];
                sm[L.p2 + e] = P2a[y];
                const int slot = atomicAdd(&s_h[2], 1);
                gsrc[slot] = y;
                gdst[slot] = (uint16_t)(L.ub + e);
            }
            off[2 * L.nE + (k - GK_UP) * nown + i] = (uint16_t)o;
        }
        sm[L.p1 + i] = P1a[a];
        sm[L.p2 + i] = P2a[a];
        sm[L.ub + i] = Ub[a];
        sm[L.u + i] = U0[a];
    }
    if (!grid_sync(h, nblocks, gen)) return -1;   // every mark cleared, every table built
    for (int g = tid; g < L.ng; g += nt) mark[gsrc[g]] = 1u;
    __shared__ int s_nbd;
    if (tid < 32) {   // stable list of the own pixels whose dual step reads a ghost
        int cd = 0;
        for (int b = 0; b < nown; b += 32) {
            const int i = b + tid;
            const unsigned f = i < nown ? flg[i] : 0u;
            const unsigned md = __ballot_sync(0xffffffffu, f & kFlDualGhost);
            if (f & kFlDualGhost) lbd[cd + __popc(md & lanemask_lt(tid))] = (uint16_t)i;
            cd += __popc(md);
        }
        if (tid == 0) {
            s_nbd = cd;
            atomicAdd(&h->n_smem_blocks, 1);
            atomicAdd(&h->n_h1_blocks, 1);
        }
    }
    if (!grid_sync(h, nblocks, gen)) return -1;   // every mark set
    for (int i = tid; i < nown; i += nt)
        if (__ldcg(mark + a0 + i)) flg[i] |= kFlExport;
    __syncthreads();
    L.nbd = s_nbd;
    const PdSmem S{sm, off, flg, r1, gsrc, gdst, lbd, L};

    // ---- iterations
    const int C = check_every;
    const int iA = min(nown, 4 * NT);
    int pb = 0, chk = 0, lf = iters;
    float dp2 = 0.f;
    bool early = false;
    // tau lambda f of the thread's pixels (at most kFSlots), in registers for
    // the whole solve
    constexpr int kFSlots = 6;
    const bool fslots = nown <= kFSlots * NT;
    float fr[kFSlots];
#pragma unroll
    for (int k = 0; k < kFSlots; ++k) {
        const int i = tid + k * nt;
        fr[k] = (fslots && i < nown) ? __ldg(F + a0 + i) : 0.f;
    }
    // interior dual steps (no ghost read) of own pixels [i0, i1)
    auto interior = [&](int b, bool acc, int i0, int i1) {
        const float* P1 = sm + L.p1 + b * L.nsp;
        const float* P2 = sm + L.p2 + b * L.nsp;
        float* Q1 = sm + L.p1 + (1 - b) * L.nsp;
        float* Q2 = sm + L.p2 + (1 - b) * L.nsp;
        for (int i = i0 + tid; i < i1; i += nt) {
            const uint8_t f = flg[i];
            if (!(f & kFlDualGhost)) pd_dual_sm(S, i, f, P1, P2, Q1, Q2, sigma, acc, dp2);
        }
    };
    for (int it = 0; it < iters; ++it) {
        const int l = it + 1;
        const bool check = (l % C == 0) || l == iters;
        const float* Ubi = (it & 1) ? Ub2 : Ub;   // u-bar of iterate it
        float* Ubo = (it & 1) ? Ub : Ub2;         // u-bar of iterate l (pixels other blocks read)
        if (!early) dp2 = 0.f;
        else if (!grid_wait(h, nblocks, gen)) return -1;
        float x[kGhostRegs];
#pragma unroll
        for (int j = 0; j < kGhostRegs; ++j) {
            const int g = tid + j * nt;
            x[j] = g < L.ng ? Ubi[gsrc[g]] : 0.f;
        }
        interior(pb, check, early ? iA : 0, nown);
#pragma unroll
        for (int j = 0; j < kGhostRegs; ++j) {
            const int g = tid + j * nt;
            if (g < L.ng) sm[gdst[g]] = x[j];
        }
        __syncthreads();
        {
            const float* P1 = sm + L.p1 + pb * L.nsp;
            const float* P2 = sm + L.p2 + pb * L.nsp;
            float* Q1 = sm + L.p1 + (1 - pb) * L.nsp;
            float* Q2 = sm + L.p2 + (1 - pb) * L.nsp;
            for (int e = tid; e < L.nbd + L.r; e += nt) {
                const bool own = e < L.nbd;
                const int i = own ? lbd[e] : nown + (e - L.nbd);
                pd_dual_sm(S, i, flg[i], P1, P2, Q1, Q2, sigma, check && own, dp2);
            }
        }
        pb ^= 1;
        __syncthreads();
        float du2 = 0.f;
        {
            const float* Q1 = sm + L.p1 + pb * L.nsp;
            const float* Q2 = sm + L.p2 + pb * L.nsp;
            const int sh = pb * L.nsp;
            if (fslots) {
                if (check) {
#pragma unroll
                    for (int k = 0; k < kFSlots; ++k) {
                        const int i = tid + k * nt;
                        if (i < nown) pd_primal_sm(S, i, a0 + i, Q1, Q2, sh, tau, fr[k], Ubo, true, du2);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < kFSlots; ++k) {
                        const int i = tid + k * nt;
                        if (i < nown) pd_primal_sm(S, i, a0 + i, Q1, Q2, sh, tau, fr[k], Ubo, false, du2);
                    }
                }
            } else if (check) {
                for (int i = tid; i < nown; i += nt)
                    pd_primal_sm(S, i, a0 + i, Q1, Q2, sh, tau, __ldg(F + a0 + i), Ubo, true, du2);
            } else {
                for (int i = tid; i < nown; i += nt)
                    pd_primal_sm(S, i, a0 + i, Q1, Q2, sh, tau, __ldg(F + a0 + i), Ubo, false, du2);
            }
        }
        double* part = partials + 2 * (int64_t)nblocks * (chk & 1);
        if (check) {
            float px = du2, py = dp2;
            block_sum2f<NT>(px, py, reinterpret_cast<float*>(s_red));
            if (tid == 0) {
                part[2 * blockIdx.x] = px;
                part[2 * blockIdx.x + 1] = py;
            }
        }
        grid_arrive(h, gen);
        early = !check;   // (the last iteration is a check)
        if (early) {
            dp2 = 0.f;
            interior(pb, (l + 1) % C == 0 || l + 1 == iters, 0, iA);
            continue;
        }
        if (!grid_wait(h, nblocks, gen)) return -1;
        if (tol > 0.0 || blockIdx.x == 0) {
            if (tid < 32) {
                double sx, sy;
                sum_partials_warp0(part, (int)nblocks, sx, sy);
                if (tid == 0) {
                    const bool stop = tol > 0.0 && fmax(sx, sy) <= tol * tol;
                    s_red[0] = stop ? 1.0 : 0.0;
                    if (blockIdx.x == 0) {
                        h->du2 = sx;
                        h->dv2 = sy;
                        h->last_check = l;
                        if (stop) {
                            h->iters_done = l;
                            h->done = 1;
                        }
                    }
                }
            }
            __syncthreads();
            const bool stop = s_red[0] != 0.0;
            __syncthreads();
            if (stop) {
                lf = l;
                break;
            }
        }
        ++chk;
    }
    __syncthreads();
    // the final iterate: u and p of every own pixel, in the buffers of iterate lf
    float* Uf = (lf & 1) ? U1 : U0;
    float* G1 = (lf & 1) ? P1b : P1a;
    float* G2 = (lf & 1) ? P2b : P2a;
    const int fb = lf & 1;
    for (int i = tid; i < nown; i += nt) {
        Uf[a0 + i] = sm[L.u + i];
        G1[a0 + i] = sm[L.p1 + fb * L.nsp + i];
        G2[a0 + i] = sm[L.p2 + fb * L.nsp + i];
    }
    return 1;
}

// Which primal-dual kernel runs a solve (both are launched; the other returns
// at once): the shared-memory one (two blocks per SM, grid1 blocks) while its
// blocks' pixels are few enough for their state to fit, else k_solve_pd.
constexpr int kPdSmemPerBlock = 3000;
__device__ __forceinline__ bool pd_smem(int n, int grid1) {
    return (n + grid1 - 1) / grid1 <= kPdSmemPerBlock;
}

__global__ void __launch_bounds__(kPdThreads, 2)
k_solve_pd(int iters, int check_every, double tol, float sigma, float tau,
           const int32_t* __restrict__ counts, const int32_t* __restrict__ nb, int64_t stride,
           float* P1a, float* P1b, float* P2a, float* P2b, float* U0, float* U1, float* Ub, float* Ub2,
           const float* __restrict__ F, double* partials, WsHeader* h, int grid1) {
    __shared__ double s_red[66];   // block_sum2f (as floats), stop flag
    if (*(volatile int*)&h->done) return;
    const int n = counts[1];
    if (pd_smem(n, grid1)) return;
    unsigned gen = 0;
    pd_iterations<kPdThreads>(iters, check_every, tol, sigma, tau, n, nb, stride, P1a, P1b, P2a, P2b, U0, U1,
                              Ub, F, partials, h, s_red, gen);
}

__global__ void __launch_bounds__(kPdSmThreads, 2)
k_solve_pd_sm(int iters, int check_every, double tol, float sigma, float tau,
              const int32_t* __restrict__ counts, const int32_t* __restrict__ nb, int64_t stride,
              float* P1a, float* P1b, float* P2a, float* P2b, float* U0, float* U1, float* Ub, float* Ub2,
              const float* __restrict__ F, double* partials, WsHeader* h, int grid1) {
    __shared__ double s_red[66];
    extern __shared__ __align__(16) unsigned char c_smem[];
    if (*(volatile int*)&h->done) return;
    const int n = counts[1];
    if (!pd_smem(n, grid1)) return;
    unsigned gen = 0;
    const int r = pd_solve_sm<kPdSmThreads>(iters, check_every, tol, sigma, tau, n, nb, stride, P1a, P1b, P2a,
                                          P2b, U0, U1, Ub, Ub2, F, partials, h, s_red, c_smem, gen);
    if (r == 0)   // some block's state does not fit: the global-memory iteration, in this grid
        pd_iterations<kPdSmThreads>(iters, check_every, tol, sigma, tau, n, nb, stride, P1a, P1b, P2a, P2b, U0,
                                  U1, Ub, F, partials, h, s_red, gen);
}

// Dense u, p1, p2 of the final primal-dual iterate (fixed values outside RD).
__global__ void k_pd_scatter(BatchDesc B, const int32_t* __restrict__ base,
                             const int32_t* __restrict__ totals, int iters, CompactState S,
                             const WsHeader* __restrict__ h) {
    const int lane = threadIdx.x & 31;
    const long long word = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (word >= B.total_words) return;
    const BatchImage& I = B.img[0];
    const int i = (int)(word / I.ntx);
    const int wx = (int)(word - (long long)i * I.ntx);
    const int j = wx * 32 + lane;
    if (j >= I.W) return;
    const int64_t wo = (int64_t)i * I.nw + wx;
    const int64_t o = (int64_t)i * I.ld + j;
    const uint32_t a = I.act[wo];
    const float hh = ((I.fg[wo] >> lane) & 1u) ? 1.f : 0.f;
    const bool ok = base[1] <= S.cap && totals[1] == base[1];
    if (ok && ((a >> lane) & 1u)) {
        const int l = h->done ? h->iters_done : iters;
        const int pb = l & 1;
        const int64_t idx = I.wstart[wo] + __popc(a & lanemask_lt(lane));
        I.u[o] = pb ? S.w[idx] : S.u[idx];
        I.p1[o] = static_cast<const float*>(S.p1[pb])[idx];
        I.p2[o] = static_cast<const float*>(S.p2[pb])[idx];
    } else {
        I.u[o] = hh;
        I.p1[o] = 0.f;
        I.p2[o] = 0.f;
    }
}

extern "C" seg_status seg_solve_pd(const float* f, int H, int W, int ld, const uint32_t* act,
                                   const uint32_t* fgm, const int32_t* wstart, const int32_t* counts,
                                   const seg_pd_params* prm, float* u, float* p1, float* p2,
                                   void* state, size_t state_bytes, double* stats, void* ws,
                                   size_t ws_bytes, void* stream) {
    clear_error();
    PhaseScope _scope("seg_solve_pd", stream, ws);
    if (!prm) return fail(SEG_ERR_INVALID_ARG, "params must be non-NULL");
    if (!f || !act || !fgm || !wstart || !counts || !u || !p1 || !p2 || !state || !stats)
        return fail(SEG_ERR_INVALID_ARG, "a required pointer is NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * ld >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d (H*ld < 2^31)", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    if (reinterpret_cast<uintptr_t>(state) % 16)
        return fail(SEG_ERR_ALIGN, "state buffer not 16-byte aligned");
    const int th = prm->tile_h;
    if (th != 4 && th != 8 && th != 16 && th != 32)
        return fail(SEG_ERR_INVALID_ARG, "tile_h=%d not in {4, 8, 16, 32}", th);
    if (prm->iters < 0 || prm->check_every < 1)
        return fail(SEG_ERR_INVALID_ARG, "iters >= 0 and check_every >= 1 required");
    if (!(prm->sigma > 0) || !(prm->tau > 0) || !std::isfinite(prm->sigma) || !std::isfinite(prm->tau) ||
        !std::isfinite(prm->lambda) || std::isnan(prm->tol))
        return fail(SEG_ERR_INVALID_ARG, "sigma, tau must be finite and > 0, lambda finite");
    WsLayout L = ws_layout(H, W, th);
    SEG_TRY(check_ws(ws, ws_bytes, L));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    double* partials = ws_at<double>(ws, L.partials);

    // the compact state of the DF solver, float32 storage, gathered with
    // F = tau lambda f
    IterParams P{};
    P.theta = 1.f;
    P.inv_theta = 1.f;
    P.tau = (float)prm->tau;
    P.theta_lambda = (float)(prm->tau * prm->lambda);
    P.H = H; P.W = W; P.ld = ld; P.nw = ld / 32; P.ntx = (W + 31) / 32; P.th = th;
    BatchDesc B{};
    B.n = 1;
    B.total_words = (long long)H * P.ntx;
    BatchImage& I = B.img[0];
    I.f = f; I.act = act; I.fg = fgm; I.wstart = wstart; I.counts = counts;
    I.u = u; I.v = u; I.p1 = p1; I.p2 = p2;
    I.word_off = 0; I.H = H; I.W = W; I.ld = ld; I.nw = ld / 32; I.ntx = P.ntx;
    I.theta_lambda = P.theta_lambda;
    int32_t* base = ws_at<int32_t>(ws, kWsBatchOff);
    int32_t* totals = base + kMaxBatch + 2;

    CompactLayout C = compact_layout(state_bytes, SEG_STORE_F32);
    CompactState S{};
    char* sb = static_cast<char*>(state);
    S.p1[0] = sb + C.off[0];
    S.p1[1] = sb + C.off[1];
    S.p2[0] = sb + C.off[2];
    S.p2[1] = sb + C.off[3];
    S.v = sb + C.off[4];
    S.f = reinterpret_cast<float*>(sb + C.off[5]);
    S.u = reinterpret_cast<float*>(sb + C.off[6]);
    S.w = reinterpret_cast<float*>(sb + C.off[7]);
    S.nb = reinterpret_cast<int32_t*>(sb + C.off[8]);
    S.w2 = reinterpret_cast<float*>(sb + C.off[9]);
    S.up = reinterpret_cast<float*>(sb + C.off[10]);
    S.cap = C.cap;
    S.stride = C.stride;

    k_solve_begin<<<1, 1, 0, s>>>(h);
    SEG_LAUNCHED("k_solve_begin");
    k_batch_bases<<<1, 1, 0, s>>>(B, base, totals, C.cap, h);
    SEG_LAUNCHED("k_batch_bases");
    const unsigned gblocks = (unsigned)std::max<long long>(1, (B.total_words + 7) / 8);
    k_compact_gather<float><<<gblocks, 256, 0, s>>>(P, B, base, prm->warm_start, S, h, totals, LLONG_MAX);
    SEG_LAUNCHED("k_compact_gather");

    const void* kern = (const void*)k_solve_pd;
    const void* kern1 = (const void*)k_solve_pd_sm;
    SEG_TRY_CUDA(cudaFuncSetAttribute(kern1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)compact_smem(kPdSmThreads)));
    int per_sm = 0, per_sm1 = 0;
    SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPdThreads, 0));
    SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, kern1, kPdSmThreads,
                                                               compact_smem(kPdSmThreads)));
    if (per_sm <= 0 || per_sm1 <= 0) return fail(SEG_ERR_CUDA, "k_solve_pd cannot be resident");
    const int64_t most = std::max<int64_t>(1, std::min<int64_t>(C.cap, (int64_t)H * W));
    int grid = (int)std::min<int64_t>((int64_t)per_sm * sm_count(),
                                      std::max<int64_t>(1, (most + kPdThreads - 1) / kPdThreads));
    grid = (int)std::min<int64_t>(grid, L.npartials / 2);
    // the shared-memory kernel: two blocks per SM (at most), the same decision
    // (pd_smem) in both kernels from grid1
    int grid1 = (int)std::min<int64_t>((int64_t)per_sm1 * sm_count(), L.npartials / 2);
    int iters = prm->iters, ce = test_interval(prm->tol, prm->check_every, prm->iters);
    double tol = prm->tol;
    float sigma = (float)prm->sigma, tau = (float)prm->tau;
    const int32_t* cnt = totals;
    const int32_t* nbp = S.nb;
    int64_t stride = S.stride;
    float* P1a = static_cast<float*>(S.p1[0]);
    float* P1b = static_cast<float*>(S.p1[1]);
    float* P2a = static_cast<float*>(S.p2[0]);
    float* P2b = static_cast<float*>(S.p2[1]);
    float* U0 = S.u;
    float* U1 = S.w;
    float* Ub = S.up;
    float* Ub2 = S.w2;   // the second u-bar buffer of the shared-memory kernel
    const float* F = S.f;
    void* args[] = {&iters, &ce, &tol, &sigma, &tau, (void*)&cnt, (void*)&nbp, &stride, &P1a, &P1b,
                    &P2a, &P2b, &U0, &U1, &Ub, &Ub2, (void*)&F, &partials, &h, &grid1};
    if (iters > 0) {
        SEG_TRY_CUDA(cudaLaunchCooperativeKernel(kern1, dim3(grid1), dim3(kPdSmThreads), args,
                                                 compact_smem(kPdSmThreads), s));
        count_launch();
        if (debug_mode()) SEG_TRY(after_launch("persistent solve"));
        SEG_TRY_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kPdThreads), args, 0, s));
        count_launch();
        if (debug_mode()) SEG_TRY(after_launch("persistent solve"));
    }
    k_pd_scatter<<<gblocks, 256, 0, s>>>(B, base, totals, prm->iters, S, h);
    SEG_LAUNCHED("k_pd_scatter");
    k_solve_end<<<1, 1, 0, s>>>(h, totals, prm->iters, stats);
    SEG_LAUNCHED("k_solve_end");
    return SEG_OK;
}
