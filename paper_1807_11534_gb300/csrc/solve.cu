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
// Two fused single-pass stencils implement one iteration each:
//  * dense   : state in [H][ld] float32 ping-pong images; one CTA per 32 x TH
//              tile of the tile list, with its halo staged in shared memory;
//              p' is recomputed on the one-pixel halo above / left so u', v'
//              need no second pass.  RD is the tile list plus the RD bits
//              (delta = inf makes it the original full-domain method).
//  * compact : state stored only for RD pixels, in tile-major compact order
//              (float32, bf16 or fp16 storage, float32 arithmetic).  One CTA
//              per active tile enumerates its RD pixels (and the RD pixels of
//              the halo row above / column left), computes p' for them into
//              shared memory, then u', v' for its own pixels.  Neighbours are
//              found through the RD bit planes: the compact index of pixel
//              (i, j) is wstart[i][j/32] + popc(act & lanemask_lt(j%32)).
// Per-tile FP64 partial sums of |du|^2, |dv|^2 feed a fixed-order reduction,
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
};

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

// p' = (p + tau g) / (1 + tau |g|)
__device__ __forceinline__ void chambolle_update(float p1, float p2, float g1, float g2, float tau,
                                                 float& q1, float& q2) {
    float nrm = sqrtf(fmaf(g1, g1, g2 * g2));
    float r = __frcp_rn(fmaf(tau, nrm, 1.0f));
    q1 = fmaf(tau, g1, p1) * r;
    q2 = fmaf(tau, g2, p2) * r;
}

// Deterministic block reduction of two FP64 values; returns the sums in
// thread 0.  All threads of the block must call it.
template <int NT>
__device__ __forceinline__ void block_sum2(double a, double b, double* s_red, double& ra, double& rb) {
    for (int d = 16; d > 0; d >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, d);
        b += __shfl_down_sync(0xffffffffu, b, d);
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { s_red[2 * wid] = a; s_red[2 * wid + 1] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int w = 0; w < NT / 32; ++w) { x += s_red[2 * w]; y += s_red[2 * w + 1]; }
        ra = x;
        rb = y;
    }
    __syncthreads();
}

// ============================================================ dense stencil

constexpr int kDenseThreads = 256;
constexpr int kSW = 36;   // shared row stride: columns c0-2 .. c0+33

// MASKED: RD given by the act bit plane (restricted); else every pixel of the
// image is in RD (the unrestricted method).  PONLY: fixed-point sweep for p
// only (extra inner sweeps), v unchanged.
template <int TH, bool MASKED, bool PONLY>
__global__ void __launch_bounds__(kDenseThreads)
k_step_dense(IterParams P, const int32_t* __restrict__ tiles, const int32_t* __restrict__ counts,
             const uint32_t* __restrict__ act, const float* __restrict__ f,
             const float* __restrict__ p1i, const float* __restrict__ p2i, const float* __restrict__ vi,
             float* __restrict__ p1o, float* __restrict__ p2o, float* __restrict__ vo,
             float* __restrict__ u, double* __restrict__ partials, WsHeader* h) {
    __shared__ float s1[(TH + 3) * kSW], s2[(TH + 3) * kSW], sv[(TH + 3) * kSW];
    __shared__ float sw[(TH + 2) * kSW];
    __shared__ float q1[(TH + 1) * kSW], q2[(TH + 1) * kSW];
    __shared__ uint32_t sm[TH + 1][2];
    __shared__ double s_red[2 * (kDenseThreads / 32)];
    if (*(volatile int*)&h->done) return;
    const int n_tiles = counts[0];
    const int tid = threadIdx.x;
    for (int k = blockIdx.x; k < n_tiles; k += gridDim.x) {
        const int t = tiles[k];
        const int ty = t / P.ntx, tx = t - ty * P.ntx;
        const int r0 = ty * TH, c0 = tx * 32;
        // ---- stage p1, p2, v on rows r0-2..r0+TH, columns c0-2..c0+33
        for (int e = tid; e < (TH + 3) * kSW; e += kDenseThreads) {
            int r = e / kSW - 2, c = e % kSW - 2;
            int i = r0 + r, j = c0 + c;
            float a = 0.f, b = 0.f, d = 0.f;
            if (i >= 0 && i < P.H && j >= 0 && j < P.W) {
                int64_t o = (int64_t)i * P.ld + j;
                a = p1i[o]; b = p2i[o]; d = vi[o];
            }
            s1[e] = a; s2[e] = b; sv[e] = d;
        }
        if (MASKED && tid < (TH + 1) * 2) {
            int r = tid / 2 - 1, wsel = tid & 1;     // wsel 0: left word, 1: own word
            int i = r0 + r, wx = tx - 1 + wsel;
            sm[r + 1][wsel] = (i >= 0 && i < P.H && wx >= 0) ? act[(int64_t)i * P.nw + wx] : 0u;
        }
        __syncthreads();
        // ---- w = div p - v/theta on rows -1..TH, columns -1..32
        for (int e = tid; e < (TH + 2) * 34; e += kDenseThreads) {
            int r = e / 34 - 1, c = e % 34 - 1;
            int i = r0 + r, j = c0 + c;
            int o = (r + 2) * kSW + (c + 2);
            float w = 0.f;
            if (i >= 0 && i < P.H && j >= 0 && j < P.W) {
                float d1 = (i < P.H - 1 ? s1[o] : 0.f) - s1[o - kSW];
                float d2 = (j < P.W - 1 ? s2[o] : 0.f) - s2[o - 1];
                w = (d1 + d2) - sv[o] * P.inv_theta;
            }
            sw[(r + 1) * kSW + (c + 1)] = w;
        }
        __syncthreads();
        // ---- p' on rows -1..TH-1, columns -1..31 (RD pixels only)
        const int prow0 = PONLY ? 0 : -1, pcol0 = PONLY ? 0 : -1;
        const int npr = TH - prow0, npc = 32 - pcol0;
        for (int e = tid; e < npr * npc; e += kDenseThreads) {
            int r = e / npc + prow0, c = e % npc + pcol0;
            int i = r0 + r, j = c0 + c;
            float a = 0.f, b = 0.f;
            bool in = i >= 0 && i < P.H && j >= 0 && j < P.W;
            if (MASKED && in) {
                uint32_t wd = c < 0 ? sm[r + 1][0] : sm[r + 1][1];
                in = (wd >> (c & 31)) & 1u;
            }
            if (in) {
                int ow = (r + 1) * kSW + (c + 1);
                float g1 = i < P.H - 1 ? sw[ow + kSW] - sw[ow] : 0.f;
                float g2 = j < P.W - 1 ? sw[ow + 1] - sw[ow] : 0.f;
                int o = (r + 2) * kSW + (c + 2);
                chambolle_update(s1[o], s2[o], g1, g2, P.tau, a, b);
            }
            q1[(r + 1) * kSW + (c + 1)] = a;
            q2[(r + 1) * kSW + (c + 1)] = b;
        }
        __syncthreads();
        // ---- u', v' on the tile
        double du2 = 0.0, dv2 = 0.0;
        for (int e = tid; e < TH * 32; e += kDenseThreads) {
            int r = e >> 5, c = e & 31;
            int i = r0 + r, j = c0 + c;
            bool in = i < P.H && j < P.W;
            if (MASKED && in) in = (sm[r + 1][1] >> c) & 1u;
            if (in) {
                int64_t og = (int64_t)i * P.ld + j;
                int oq = (r + 1) * kSW + (c + 1);
                p1o[og] = q1[oq];
                p2o[og] = q2[oq];
                if (!PONLY) {
                    float div = (i < P.H - 1 ? q1[oq] : 0.f) - q1[oq - kSW] +
                                (j < P.W - 1 ? q2[oq] : 0.f) - q2[oq - 1];
                    float vv = sv[(r + 2) * kSW + (c + 2)];
                    float un = fmaf(-P.theta, div, vv);
                    float vn = clamp01(fmaf(-P.theta_lambda, f[og], un));
                    vo[og] = vn;
                    if (P.check) {
                        float a = un - u[og], b = vn - vv;
                        du2 += (double)(a * a);
                        dv2 += (double)(b * b);
                    }
                    if (P.write_u) u[og] = un;
                }
            }
        }
        if (!PONLY && P.check) {
            double ra, rb;
            block_sum2<kDenseThreads>(du2, dv2, s_red, ra, rb);
            if (tid == 0) { partials[2 * k] = ra; partials[2 * k + 1] = rb; }
        } else {
            __syncthreads();
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

constexpr int kCompactThreads = 128;

struct CompactState {
    void *p1[2], *p2[2], *v[2];
    float* f;
    float* u;
    int64_t cap;
};

// Shared-memory view of the rows r0-2..r0+TH of the three word columns
// tx-1, tx, tx+1 around a tile: RD bits, f<0 bits and compact starts.
template <int TH>
struct TileMeta {
    uint32_t act[TH + 3][3];
    uint32_t fg[TH + 3][3];
    int ws[TH + 3][3];
};

// (active, compact index, fixed v) of local pixel (r, c), r in [-2, TH],
// c in [-32, 63] relative to the tile origin.
template <int TH>
__device__ __forceinline__ bool meta_lookup(const TileMeta<TH>& M, int r, int c, int& idx, float& vfix) {
    int wc = (c + 32) >> 5;
    int b = c & 31;
    uint32_t a = M.act[r + 2][wc];
    if ((a >> b) & 1u) {
        idx = M.ws[r + 2][wc] + __popc(a & lanemask_lt(b));
        return true;
    }
    vfix = ((M.fg[r + 2][wc] >> b) & 1u) ? 1.f : 0.f;
    return false;
}

template <typename T, int TH>
__device__ __forceinline__ void nb_p1(const TileMeta<TH>& M, const T* P1, int r, int c, float& p1) {
    int idx; float vf;
    p1 = meta_lookup<TH>(M, r, c, idx, vf) ? Store<T>::ld(P1, idx) : 0.f;
}
template <typename T, int TH>
__device__ __forceinline__ void nb_p2(const TileMeta<TH>& M, const T* P2, int r, int c, float& p2) {
    int idx; float vf;
    p2 = meta_lookup<TH>(M, r, c, idx, vf) ? Store<T>::ld(P2, idx) : 0.f;
}
template <typename T, int TH>
__device__ __forceinline__ void nb_all(const TileMeta<TH>& M, const T* P1, const T* P2, const T* V,
                                       int r, int c, float& p1, float& p2, float& v) {
    int idx; float vf;
    if (meta_lookup<TH>(M, r, c, idx, vf)) {
        p1 = Store<T>::ld(P1, idx); p2 = Store<T>::ld(P2, idx); v = Store<T>::ld(V, idx);
    } else {
        p1 = 0.f; p2 = 0.f; v = vf;
    }
}

// item encoding: local row r in [-1, TH-1], column c in [-1, 31]
__device__ __forceinline__ uint16_t pack_rc(int r, int c) { return (uint16_t)(((r + 2) << 8) | (c + 2)); }
__device__ __forceinline__ void unpack_rc(uint16_t e, int& r, int& c) { r = (e >> 8) - 2; c = (e & 255) - 2; }

template <typename T, int TH, bool PONLY>
__global__ void __launch_bounds__(kCompactThreads)
k_step_compact(IterParams P, const int32_t* __restrict__ tiles, const int32_t* __restrict__ counts,
               const uint32_t* __restrict__ act, const uint32_t* __restrict__ fgm,
               const int32_t* __restrict__ wstart, const T* __restrict__ P1i,
               const T* __restrict__ P2i, const T* __restrict__ Vi, T* __restrict__ P1o,
               T* __restrict__ P2o, T* __restrict__ Vo, const float* __restrict__ F,
               float* __restrict__ U, double* __restrict__ partials, WsHeader* h) {
    constexpr int kMaxItems = TH * 32 + 32 + TH;
    __shared__ TileMeta<TH> M;
    __shared__ int s_lp[TH + 1];       // exclusive prefix of RD counts of the tile rows
    __shared__ int s_hcp[TH + 1];      // exclusive prefix of the halo-column RD bits
    __shared__ int s_cnt[3];           // n_own, halo-row count, halo-column count
    __shared__ uint16_t s_item[kMaxItems];
    __shared__ float s_q1[kMaxItems], s_q2[kMaxItems];
    __shared__ double s_red[2 * (kCompactThreads / 32)];
    if (*(volatile int*)&h->done) return;
    const int n_tiles = counts[0];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int k = blockIdx.x; k < n_tiles; k += gridDim.x) {
        const int t = tiles[k];
        const int ty = t / P.ntx, tx = t - ty * P.ntx;
        const int r0 = ty * TH, c0 = tx * 32;
        // ---- word metadata of rows r0-2..r0+TH, word columns tx-1..tx+1
        for (int e = tid; e < (TH + 3) * 3; e += kCompactThreads) {
            int rr = e / 3, wc = e - rr * 3;
            int i = r0 + rr - 2, wx = tx - 1 + wc;
            uint32_t a = 0u, g = 0u;
            int s = 0;
            if (i >= 0 && i < P.H && wx >= 0 && wx < P.ntx) {
                int64_t o = (int64_t)i * P.nw + wx;
                a = act[o]; g = fgm[o]; s = wstart[o];
            }
            M.act[rr][wc] = a; M.fg[rr][wc] = g; M.ws[rr][wc] = s;
        }
        __syncthreads();
        if (wid == 0) {
            uint32_t a = lane < TH ? M.act[lane + 2][1] : 0u;
            int c = __popc(a);
            int hb = lane < TH ? (int)(M.act[lane + 2][0] >> 31) : 0;
            int ic = c, ih = hb;
            for (int d = 1; d < 32; d <<= 1) {
                int o1 = __shfl_up_sync(0xffffffffu, ic, d);
                int o2 = __shfl_up_sync(0xffffffffu, ih, d);
                if (lane >= d) { ic += o1; ih += o2; }
            }
            if (lane < TH) { s_lp[lane] = ic - c; s_hcp[lane] = ih - hb; }
            if (lane == TH - 1) { s_lp[TH] = ic; s_hcp[TH] = ih; s_cnt[0] = ic; s_cnt[2] = PONLY ? 0 : ih; }
            if (lane == 0) s_cnt[1] = PONLY ? 0 : __popc(M.act[1][1]);
        }
        __syncthreads();
        const int n_own = s_cnt[0], n_hr = s_cnt[1], n_hc = s_cnt[2];
        const int n_items = n_own + n_hr + n_hc;
        const int tstart = M.ws[2][1];   // compact index of the tile's first RD pixel
        // ---- enumerate items: own pixels (row-major), halo row, halo column
        for (int rr = wid; rr < TH + (PONLY ? 0 : 1); rr += kCompactThreads / 32) {
            if (rr < TH) {
                uint32_t a = M.act[rr + 2][1];
                if ((a >> lane) & 1u) s_item[s_lp[rr] + __popc(a & lanemask_lt(lane))] = pack_rc(rr, lane);
            } else {
                uint32_t a = M.act[1][1];
                if ((a >> lane) & 1u) s_item[n_own + __popc(a & lanemask_lt(lane))] = pack_rc(-1, lane);
            }
        }
        if (!PONLY && tid < TH && ((M.act[tid + 2][0] >> 31) & 1u))
            s_item[n_own + n_hr + s_hcp[tid]] = pack_rc(tid, -1);
        __syncthreads();
        // ---- phase 1: p' at every item
        for (int e = tid; e < n_items; e += kCompactThreads) {
            int r, c;
            unpack_rc(s_item[e], r, c);
            const int i = r0 + r, j = c0 + c;
            float p1y, p2y, vy;
            if (e < n_own) {
                int idx = tstart + e;
                p1y = Store<T>::ld(P1i, idx); p2y = Store<T>::ld(P2i, idx); vy = Store<T>::ld(Vi, idx);
            } else {
                nb_all<T, TH>(M, P1i, P2i, Vi, r, c, p1y, p2y, vy);
            }
            float p1_um, p2_lm, p1_d, p2_d, v_d, p1_r, p2_r, v_r, p2_dl, p1_ur;
            nb_p1<T, TH>(M, P1i, r - 1, c, p1_um);        // y - e1
            nb_p2<T, TH>(M, P2i, r, c - 1, p2_lm);        // y - e2
            nb_all<T, TH>(M, P1i, P2i, Vi, r + 1, c, p1_d, p2_d, v_d);   // y + e1
            nb_all<T, TH>(M, P1i, P2i, Vi, r, c + 1, p1_r, p2_r, v_r);   // y + e2
            nb_p2<T, TH>(M, P2i, r + 1, c - 1, p2_dl);    // y + e1 - e2
            nb_p1<T, TH>(M, P1i, r - 1, c + 1, p1_ur);    // y + e2 - e1
            const bool lr = i < P.H - 1, lc = j < P.W - 1;
            float w0 = ((lr ? p1y : 0.f) - p1_um) + ((lc ? p2y : 0.f) - p2_lm) - vy * P.inv_theta;
            float g1 = 0.f, g2 = 0.f;
            if (lr) {
                float wd = ((i + 1 < P.H - 1 ? p1_d : 0.f) - p1y) + ((lc ? p2_d : 0.f) - p2_dl) -
                           v_d * P.inv_theta;
                g1 = wd - w0;
            }
            if (lc) {
                float wr = ((lr ? p1_r : 0.f) - p1_ur) + ((j + 1 < P.W - 1 ? p2_r : 0.f) - p2y) -
                           v_r * P.inv_theta;
                g2 = wr - w0;
            }
            float a, b;
            chambolle_update(p1y, p2y, g1, g2, P.tau, a, b);
            s_q1[e] = a;
            s_q2[e] = b;
        }
        __syncthreads();
        // ---- phase 2: u', v' for own pixels, write back
        double du2 = 0.0, dv2 = 0.0;
        for (int e = tid; e < n_own; e += kCompactThreads) {
            int r, c;
            unpack_rc(s_item[e], r, c);
            const int i = r0 + r, j = c0 + c;
            const int idx = tstart + e;
            float q1 = s_q1[e], q2 = s_q2[e];
            Store<T>::st(P1o, idx, q1);
            Store<T>::st(P2o, idx, q2);
            if (PONLY) continue;
            float q1u = 0.f, q2l = 0.f;
            if (r > 0) {
                uint32_t a = M.act[r + 1][1];
                if ((a >> c) & 1u) q1u = s_q1[s_lp[r - 1] + __popc(a & lanemask_lt(c))];
            } else {
                uint32_t a = M.act[1][1];
                if ((a >> c) & 1u) q1u = s_q1[n_own + __popc(a & lanemask_lt(c))];
            }
            if (c > 0) {
                if ((M.act[r + 2][1] >> (c - 1)) & 1u) q2l = s_q2[e - 1];
            } else {
                if ((M.act[r + 2][0] >> 31) & 1u) q2l = s_q2[n_own + n_hr + s_hcp[r]];
            }
            float div = ((i < P.H - 1 ? q1 : 0.f) - q1u) + ((j < P.W - 1 ? q2 : 0.f) - q2l);
            float vv = Store<T>::ld(Vi, idx);
            float un = fmaf(-P.theta, div, vv);
            float vn = clamp01(fmaf(-P.theta_lambda, __ldg(F + idx), un));
            Store<T>::st(Vo, idx, vn);
            if (P.check) {
                float da = un - U[idx], db = vn - vv;
                du2 += (double)(da * da);
                dv2 += (double)(db * db);
            }
            if (P.write_u) U[idx] = un;
        }
        if (!PONLY && P.check) {
            double ra, rb;
            block_sum2<kCompactThreads>(du2, dv2, s_red, ra, rb);
            if (tid == 0) { partials[2 * k] = ra; partials[2 * k + 1] = rb; }
        } else {
            __syncthreads();
        }
    }
}

// One warp per mask word: lane b is pixel (i, 32 wx + b).
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
    int lane = threadIdx.x & 31;
    int64_t word = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    int64_t nwords = (int64_t)P.H * P.ntx;
    if (word >= nwords) return;
    int64_t i = word / P.ntx;
    int wx = (int)(word - i * P.ntx);
    int64_t wo = i * P.nw + wx;
    uint32_t a = act[wo];
    if (!((a >> lane) & 1u)) return;
    int64_t idx = wstart[wo] + __popc(a & lanemask_lt(lane));
    int64_t o = i * P.ld + wx * 32 + lane;
    float fv = f[o];
    float hh = ((fgm[wo] >> lane) & 1u) ? 1.f : 0.f;
    S.f[idx] = fv;
    T* P1 = static_cast<T*>(S.p1[0]);
    T* P2 = static_cast<T*>(S.p2[0]);
    T* V = static_cast<T*>(S.v[0]);
    if (warm) {
        Store<T>::st(P1, idx, p1[o]); Store<T>::st(P2, idx, p2[o]); Store<T>::st(V, idx, v[o]);
        S.u[idx] = u[o];
    } else {
        Store<T>::st(P1, idx, 0.f); Store<T>::st(P2, idx, 0.f);
        Store<T>::st(V, idx, clamp01(fmaf(-P.theta_lambda, fv, hh)));
        S.u[idx] = hh;
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
    int lane = threadIdx.x & 31;
    int64_t word = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    int64_t nwords = (int64_t)P.H * P.ntx;
    if (word >= nwords) return;
    int64_t i = word / P.ntx;
    int wx = (int)(word - i * P.ntx);
    int j = wx * 32 + lane;
    if (j >= P.W) return;
    int64_t wo = i * P.nw + wx;
    int64_t o = i * P.ld + j;
    uint32_t a = act[wo];
    float hh = ((fgm[wo] >> lane) & 1u) ? 1.f : 0.f;
    bool ok = counts[1] <= S.cap;
    if (ok && ((a >> lane) & 1u)) {
        int l = h->done ? h->iters_done : iters;
        int vb = l & 1, pb = (int)(((long long)l * n_inner) & 1);
        int64_t idx = wstart[wo] + __popc(a & lanemask_lt(lane));
        u[o] = S.u[idx];
        v[o] = Store<T>::ld_rw(static_cast<const T*>(S.v[vb]), idx);
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

// Section 4 stopping test after iteration l: sums the per-tile partials in a
// fixed order, records the norms and raises the done flag when both are <= tol.
__global__ void k_check(const double* __restrict__ partials, const int32_t* __restrict__ counts,
                        int l, double tol, WsHeader* h) {
    __shared__ double sa[256], sb[256];
    if (*(volatile int*)&h->done) return;
    int n = counts[0];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) { a += partials[2 * k]; b += partials[2 * k + 1]; }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
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
static int grid_for(K kernel, int threads, int64_t max_tiles) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (per_sm <= 0) per_sm = 1;
    int64_t g = (int64_t)per_sm * sm_count();
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, max_tiles));
}

struct CompactLayout {
    size_t off[8];
    int64_t cap;
};

static CompactLayout compact_layout(size_t state_bytes, int storage) {
    CompactLayout C{};
    size_t sz = storage_size(storage);
    size_t per = 6 * sz + 8;
    C.cap = state_bytes > 8 * 256 ? (int64_t)((state_bytes - 8 * 256) / per) : 0;
    size_t o = 0;
    for (int a = 0; a < 6; ++a) { C.off[a] = o; o = align_up(o + sz * (size_t)C.cap, 256); }
    C.off[6] = o; o = align_up(o + 4 * (size_t)C.cap, 256);
    C.off[7] = o;
    return C;
}

template <int TH, bool MASKED>
static seg_status run_dense(const IterParams& P0, const seg_params* prm, const int32_t* tiles,
                            const int32_t* counts, const uint32_t* act, const float* f, float* u,
                            float* st, double* partials, WsHeader* h, int64_t max_tiles,
                            cudaStream_t s) {
    int64_t plane = (int64_t)P0.H * P0.ld;
    float* P1[2] = {st, st + plane};
    float* P2[2] = {st + 2 * plane, st + 3 * plane};
    float* V[2] = {st + 4 * plane, st + 5 * plane};
    auto kfull = k_step_dense<TH, MASKED, false>;
    auto kp = k_step_dense<TH, MASKED, true>;
    int grid = grid_for(kfull, kDenseThreads, max_tiles);
    int gridp = grid_for(kp, kDenseThreads, max_tiles);
    int pb = 0, vb = 0;
    const int C = std::max(1, prm->check_every);
    for (int it = 0; it < prm->iters; ++it) {
        const int l = it + 1;
        for (int sw = 1; sw < prm->n_inner; ++sw) {
            IterParams P = P0;
            P.check = 0; P.write_u = 0;
            kp<<<gridp, kDenseThreads, 0, s>>>(P, tiles, counts, act, f, P1[pb], P2[pb], V[vb],
                                               P1[pb ^ 1], P2[pb ^ 1], V[vb], u, partials, h);
            SEG_LAUNCHED("k_step_dense<p-only>");
            pb ^= 1;
        }
        IterParams P = P0;
        P.check = (l % C == 0) || l == prm->iters;
        P.write_u = P.check || ((l + 1) % C == 0) || l == prm->iters;
        kfull<<<grid, kDenseThreads, 0, s>>>(P, tiles, counts, act, f, P1[pb], P2[pb], V[vb],
                                             P1[pb ^ 1], P2[pb ^ 1], V[vb ^ 1], u, partials, h);
        SEG_LAUNCHED("k_step_dense");
        pb ^= 1;
        vb ^= 1;
        if (P.check) {
            k_check<<<1, 256, 0, s>>>(partials, counts, l, prm->tol, h);
            SEG_LAUNCHED("k_check");
        }
    }
    return SEG_OK;
}

template <typename T, int TH>
static seg_status run_compact(const IterParams& P0, const seg_params* prm, const int32_t* tiles,
                              const int32_t* counts, const uint32_t* act, const uint32_t* fgm,
                              const int32_t* wstart, const CompactState& S, double* partials,
                              WsHeader* h, int64_t max_tiles, cudaStream_t s) {
    T* P1[2] = {static_cast<T*>(S.p1[0]), static_cast<T*>(S.p1[1])};
    T* P2[2] = {static_cast<T*>(S.p2[0]), static_cast<T*>(S.p2[1])};
    T* V[2] = {static_cast<T*>(S.v[0]), static_cast<T*>(S.v[1])};
    auto kfull = k_step_compact<T, TH, false>;
    auto kp = k_step_compact<T, TH, true>;
    int grid = grid_for(kfull, kCompactThreads, max_tiles);
    int gridp = grid_for(kp, kCompactThreads, max_tiles);
    int pb = 0, vb = 0;
    const int C = std::max(1, prm->check_every);
    for (int it = 0; it < prm->iters; ++it) {
        const int l = it + 1;
        for (int sw = 1; sw < prm->n_inner; ++sw) {
            IterParams P = P0;
            P.check = 0; P.write_u = 0;
            kp<<<gridp, kCompactThreads, 0, s>>>(P, tiles, counts, act, fgm, wstart, P1[pb], P2[pb],
                                                 V[vb], P1[pb ^ 1], P2[pb ^ 1], V[vb], S.f, S.u,
                                                 partials, h);
            SEG_LAUNCHED("k_step_compact<p-only>");
            pb ^= 1;
        }
        IterParams P = P0;
        P.check = (l % C == 0) || l == prm->iters;
        P.write_u = P.check || ((l + 1) % C == 0) || l == prm->iters;
        kfull<<<grid, kCompactThreads, 0, s>>>(P, tiles, counts, act, fgm, wstart, P1[pb], P2[pb],
                                               V[vb], P1[pb ^ 1], P2[pb ^ 1], V[vb ^ 1], S.f, S.u,
                                               partials, h);
        SEG_LAUNCHED("k_step_compact");
        pb ^= 1;
        vb ^= 1;
        if (P.check) {
            k_check<<<1, 256, 0, s>>>(partials, counts, l, prm->tol, h);
            SEG_LAUNCHED("k_check");
        }
    }
    return SEG_OK;
}

template <typename T>
static seg_status solve_compact_typed(const IterParams& P, const seg_params* prm, const float* f,
                                      const uint32_t* act, const uint32_t* fgm, const int32_t* wstart,
                                      const int32_t* tiles, const int32_t* counts, float* u, float* v,
                                      float* p1, float* p2, void* state, size_t state_bytes,
                                      double* partials, WsHeader* h, int64_t max_tiles, cudaStream_t s) {
    CompactLayout C = compact_layout(state_bytes, prm->storage);
    CompactState S{};
    char* base = static_cast<char*>(state);
    for (int b = 0; b < 2; ++b) {
        S.p1[b] = base + C.off[0 + b];
        S.p2[b] = base + C.off[2 + b];
        S.v[b] = base + C.off[4 + b];
    }
    S.f = reinterpret_cast<float*>(base + C.off[6]);
    S.u = reinterpret_cast<float*>(base + C.off[7]);
    S.cap = C.cap;
    int64_t nwords = (int64_t)P.H * P.ntx;
    unsigned gblocks = (unsigned)((nwords + 7) / 8);
    k_compact_gather<T><<<gblocks, 256, 0, s>>>(P, act, fgm, wstart, counts, f, prm->warm_start, u, v,
                                                p1, p2, S, h);
    SEG_LAUNCHED("k_compact_gather");
    switch (prm->tile_h) {
        case 4:  SEG_TRY((run_compact<T, 4>(P, prm, tiles, counts, act, fgm, wstart, S, partials, h, max_tiles, s))); break;
        case 8:  SEG_TRY((run_compact<T, 8>(P, prm, tiles, counts, act, fgm, wstart, S, partials, h, max_tiles, s))); break;
        case 16: SEG_TRY((run_compact<T, 16>(P, prm, tiles, counts, act, fgm, wstart, S, partials, h, max_tiles, s))); break;
        default: SEG_TRY((run_compact<T, 32>(P, prm, tiles, counts, act, fgm, wstart, S, partials, h, max_tiles, s))); break;
    }
    k_compact_scatter<T><<<gblocks, 256, 0, s>>>(P, act, fgm, wstart, counts, prm->iters,
                                                 std::max(1, prm->n_inner), S, h, u, v, p1, p2);
    SEG_LAUNCHED("k_compact_scatter");
    return SEG_OK;
}

}  // namespace seg

using namespace seg;

extern "C" size_t seg_state_bytes(int H, int ld, int64_t capacity, int mode, int storage) {
    if (mode == SEG_MODE_DENSE) return 6 * 4 * (size_t)std::max(H, 0) * (size_t)std::max(ld, 0) + 256;
    size_t sz = storage_size(storage);
    return 8 * 256 + (size_t)std::max<int64_t>(capacity, 1) * (6 * sz + 8);
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
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * W >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d", H, W, ld);
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
        switch (th) {
            case 4:  SEG_TRY((run_dense<4, true>(P, prm, tiles, counts, act, f, u, st, partials, h, L.ntiles, s))); break;
            case 8:  SEG_TRY((run_dense<8, true>(P, prm, tiles, counts, act, f, u, st, partials, h, L.ntiles, s))); break;
            case 16: SEG_TRY((run_dense<16, true>(P, prm, tiles, counts, act, f, u, st, partials, h, L.ntiles, s))); break;
            default: SEG_TRY((run_dense<32, true>(P, prm, tiles, counts, act, f, u, st, partials, h, L.ntiles, s))); break;
        }
        k_final_dense<<<blocks, 256, 0, s>>>(P, h, prm->iters, prm->n_inner, st, v, p1, p2);
        SEG_LAUNCHED("k_final_dense");
    } else {
        switch (prm->storage) {
            case SEG_STORE_F32:
                SEG_TRY(solve_compact_typed<float>(P, prm, f, act, fgm, wstart, tiles, counts, u, v, p1, p2,
                                                   state, state_bytes, partials, h, L.ntiles, s));
                break;
            case SEG_STORE_BF16:
                SEG_TRY(solve_compact_typed<__nv_bfloat16>(P, prm, f, act, fgm, wstart, tiles, counts, u, v,
                                                           p1, p2, state, state_bytes, partials, h, L.ntiles, s));
                break;
            default:
                SEG_TRY(solve_compact_typed<__half>(P, prm, f, act, fgm, wstart, tiles, counts, u, v, p1, p2,
                                                    state, state_bytes, partials, h, L.ntiles, s));
                break;
        }
    }
    k_solve_end<<<1, 1, 0, s>>>(h, counts, prm->iters, stats);
    SEG_LAUNCHED("k_solve_end");
    return SEG_OK;
}
