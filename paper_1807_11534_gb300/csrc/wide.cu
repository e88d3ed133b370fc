// wide.cu -- the restricted iteration of Sections 2.1 and 3 for one image
// whose RD is too large for the shared-memory paths of solve.cu, on a
// compact state in row-major order.
//
// RD pixels are numbered row by row (rowstart[i] + the RD pixels before
// column j in row i), so that in the compact arrays
//   * the neighbours left and right of pixel a, when in RD, are a - 1 and
//     a + 1;
//   * the RD pixels of row i + 1 at columns >= j start at D0 = a + dD, and
//     those of row i - 1 at columns >= j at U0 = a - dU, with 0 <= dD, dU
//     <= W (the RD pixels of at most one row lie in between), so x + e1 is
//     D0 and x + e1 - e2 is D0 - 1, x - e1 is U0 and x - e1 + e2 is U0 + 1
//     (or U0 when x - e1 is fixed), whenever those pixels are in RD;
// and the whole neighbourhood of a pixel is two 16-bit offsets and a 16-bit
// word of flags (6 bytes, against the 24 of the six-row int32 table of the
// tile-major order).  Each block keeps its pixels' neighbourhoods (and theta
// lambda f, while they fit with it) in shared memory for the whole launch,
// and the rest of the iteration's arrays (both p buffers, w, v) stay in L2
// for images like the 4096^2 precision workload, so the two phases of an
// iteration (dual step, grid barrier, primal step, grid barrier) take one L2
// round trip each.  The arithmetic and rounding of every step are those of
// dual_one / primal_one in solve.cu (the 16-bit stores' random words are
// drawn from the compact index, as there, and at bf16 both components of p'
// take halves of one word, so 16-bit results differ in the rounding noise
// only); the stopping test, the header fields and the stats are those of the
// other compact paths.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "iterate.cuh"

namespace seg {

enum : uint16_t {
    RM_DOWN_RD = 1u << 0,    // x + e1 in RD (at D0)
    RM_DOWN_FG = 1u << 1,    // x + e1 fixed foreground (else background)
    RM_DOWN_OUT = 1u << 2,   // x on the last row
    RM_RIGHT_RD = 1u << 3,   // x + e2 in RD (at a + 1)
    RM_RIGHT_FG = 1u << 4,
    RM_RIGHT_OUT = 1u << 5,  // x on the last column
    RM_DL_RD = 1u << 6,      // x + e1 - e2 in RD (at D0 - 1)
    RM_UR_RD = 1u << 7,      // x - e1 + e2 in RD (at U0 + [x - e1 in RD])
    RM_UP_RD = 1u << 8,      // x - e1 in RD (at U0)
    RM_LEFT_RD = 1u << 9,    // x - e2 in RD (at a - 1)
};

template <typename T>
struct RowMajorState {
    T* p1[2];
    T* p2[2];
    T* v;
    float *F, *U, *Up, *Wc;
    uint16_t *dd, *du, *fl;
};

template <typename T>
RowMajorState<T> rm_state(const RowMajorArrays& A) {
    return RowMajorState<T>{{static_cast<T*>(A.p1[0]), static_cast<T*>(A.p1[1])},
                            {static_cast<T*>(A.p2[0]), static_cast<T*>(A.p2[1])},
                            static_cast<T*>(A.v), A.F, A.U, A.Up, A.Wc, A.dd, A.du, A.fl};
}

// w at a fixed neighbour: p there is 0, so div p is minus the two
// components that flow into it, and v is its fixed value (as w_fixed)
__device__ __forceinline__ float rm_w_fixed(float p_in_1, float p_in_2, bool fg, float inv_theta) {
    return -(p_in_1 + p_in_2) - (fg ? inv_theta : 0.f);
}

// ------------------------------------------------------------ setup

// RD pixels per row (one warp per row).
__global__ void k_rm_rowcount(RowMajorArgs R) {
    if (*(volatile const int*)&R.h->done || R.counts[1] <= R.wide_above) return;
    const int lane = threadIdx.x & 31;
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= R.H) return;
    int c = 0;
    for (int k = lane; k < R.ntx; k += 32) c += __popc(__ldg(R.act + (int64_t)i * R.nw + k));
    for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
    if (lane == 0) R.rowstart[i] = c;
}

// Exclusive scan of the row counts in place (one block), rowstart[H] = total.
__global__ void k_rm_rowscan(RowMajorArgs R) {
    if (*(volatile const int*)&R.h->done || R.counts[1] <= R.wide_above) return;
    __shared__ int s[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < R.H; base += 1024) {
        const int i = base + (int)threadIdx.x;
        const int x = i < R.H ? R.rowstart[i] : 0;
        s[threadIdx.x] = x;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {   // inclusive Hillis-Steele scan
            const int t = threadIdx.x >= (unsigned)d ? s[threadIdx.x - d] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < R.H) R.rowstart[i] = carry + s[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) R.rowstart[R.H] = carry;
}

// The row-major position of pixel (r, j): rowstart[r] plus the RD pixels of
// row r before column j, from the warp's running word prefix `pre` of row r
// (RD pixels in the words before word k) and word `w` of row r.
__device__ __forceinline__ int rm_pos(const int32_t* rowstart, int r, int pre, uint32_t w, int b) {
    return rowstart[r] + pre + __popc(w & lanemask_lt(b));
}

// One warp per row: the compact state of every RD pixel of the row in
// row-major order (f times theta lambda, the start iterate, w for a cold
// start), its offsets and flags.  Lane l takes word k = 32 c + l of the
// chunk c, with the same word of the rows above and below.
template <typename T>
__global__ void k_rm_gather(RowMajorArgs R, RowMajorState<T> S, int warm) {
    if (*(volatile const int*)&R.h->done || R.counts[1] <= R.wide_above) return;
    const int lane = threadIdx.x & 31;
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= R.H) return;
    const unsigned FULL = 0xffffffffu;
    int pre_u = 0, pre_c = 0, pre_d = 0;   // RD pixels of rows i-1, i, i+1 before this chunk
    for (int c0 = 0; c0 < R.ntx; c0 += 32) {
        const int k = c0 + lane;
        const bool in = k < R.ntx;
        const int64_t o = (int64_t)i * R.nw + k;
        const uint32_t wc = in ? __ldg(R.act + o) : 0u;
        const uint32_t fc = in ? __ldg(R.fg + o) : 0u;
        const uint32_t wu = in && i > 0 ? __ldg(R.act + o - R.nw) : 0u;
        const uint32_t wd = in && i + 1 < R.H ? __ldg(R.act + o + R.nw) : 0u;
        const uint32_t fd = in && i + 1 < R.H ? __ldg(R.fg + o + R.nw) : 0u;
        // the next word of this row (for the right neighbour of bit 31) and
        // of the row above (for x - e1 + e2 of bit 31); the previous word of
        // this row and of the row below (for bit 0)
        const uint32_t wcn = k + 1 < R.ntx ? __ldg(R.act + o + 1) : 0u;
        const uint32_t fcn = k + 1 < R.ntx ? __ldg(R.fg + o + 1) : 0u;
        const uint32_t wun = k + 1 < R.ntx && i > 0 ? __ldg(R.act + o - R.nw + 1) : 0u;
        const uint32_t wcp = in && k > 0 ? __ldg(R.act + o - 1) : 0u;
        const uint32_t wdp = in && k > 0 && i + 1 < R.H ? __ldg(R.act + o + R.nw - 1) : 0u;
        // exclusive prefix of the three rows' word counts across the lanes
        int cu = __popc(wu), cc = __popc(wc), cd = __popc(wd);
        int su = cu, sc = cc, sd = cd;
        for (int d = 1; d < 32; d <<= 1) {
            const int tu = __shfl_up_sync(FULL, su, d), tc = __shfl_up_sync(FULL, sc, d),
                      td = __shfl_up_sync(FULL, sd, d);
            if (lane >= d) { su += tu; sc += tc; sd += td; }
        }
        const int wpre_u = pre_u + su - cu, wpre_c = pre_c + sc - cc, wpre_d = pre_d + sd - cd;
        for (uint32_t bits = wc; bits; bits &= bits - 1) {
            const int b = __ffs(bits) - 1;
            const int j = 32 * k + b;
            const int a = rm_pos(R.rowstart, i, wpre_c, wc, b);
            uint16_t fl = 0;
            const bool last_row = i + 1 >= R.H, last_col = j + 1 >= R.W;
            if (last_row) fl |= RM_DOWN_OUT;
            else {
                if ((wd >> b) & 1u) fl |= RM_DOWN_RD;
                else if ((fd >> b) & 1u) fl |= RM_DOWN_FG;
                const bool dl = b > 0 ? ((wd >> (b - 1)) & 1u) : (j > 0 && (wdp >> 31));
                if (dl) fl |= RM_DL_RD;
            }
            if (last_col) fl |= RM_RIGHT_OUT;
            else {
                const bool r_rd = b < 31 ? ((wc >> (b + 1)) & 1u) : (wcn & 1u);
                const bool r_fg = b < 31 ? ((fc >> (b + 1)) & 1u) : (fcn & 1u);
                if (r_rd) fl |= RM_RIGHT_RD;
                else if (r_fg) fl |= RM_RIGHT_FG;
                const bool ur = i > 0 && (b < 31 ? ((wu >> (b + 1)) & 1u) : (wun & 1u));
                if (ur) fl |= RM_UR_RD;
            }
            if (i > 0 && ((wu >> b) & 1u)) fl |= RM_UP_RD;
            if (j > 0 && (b > 0 ? ((wc >> (b - 1)) & 1u) : (wcp >> 31))) fl |= RM_LEFT_RD;
            const int d0 = last_row ? a : rm_pos(R.rowstart, i + 1, wpre_d, wd, b);
            const int u0 = i > 0 ? rm_pos(R.rowstart, i - 1, wpre_u, wu, b) : a;
            S.dd[a] = (uint16_t)(d0 - a);
            S.du[a] = (uint16_t)(a - u0);
            S.fl[a] = fl;
            const int64_t off = (int64_t)i * R.ld + j;
            const float fv = R.f[off];
            const float hh = ((fc >> b) & 1u) ? 1.f : 0.f;
            S.F[a] = R.theta_lambda * fv;
            if (warm) {
                Store<T>::st(S.p1[0], a, i < R.H - 1 ? R.p1[off] : 0.f);
                Store<T>::st(S.p2[0], a, j < R.W - 1 ? R.p2[off] : 0.f);
                Store<T>::st(S.v, a, R.v[off] - Store<T>::vbias);
                S.U[a] = R.u[off];
                S.Up[a] = R.u[off];
                S.Wc[a] = 0.f;   // formed by the solve from the whole state
            } else {
                Store<T>::st(S.p1[0], a, 0.f);
                Store<T>::st(S.p2[0], a, 0.f);
                Store<T>::st(S.v, a, clamp01(fmaf(-R.theta_lambda, fv, hh)) - Store<T>::vbias);
                S.U[a] = hh;
                S.Up[a] = hh;
                S.Wc[a] = -(Store<T>::ld_rw(S.v, a) + Store<T>::vbias) * R.inv_theta;
            }
        }
        pre_u = __shfl_sync(FULL, wpre_u + cu, 31);
        pre_c = __shfl_sync(FULL, wpre_c + cc, 31);
        pre_d = __shfl_sync(FULL, wpre_d + cd, 31);
    }
}

// ------------------------------------------------------------ iteration

constexpr int kRmThreads = 768;   // threads per block
constexpr int kRmMinBlocks = 2;   // resident blocks per SM the registers are sized for
constexpr int kRmUnroll = 2;      // pixels per thread whose loads are in flight together

// The two phases below take U pixels of a thread at a time and issue every
// load of all U before the first store: the stores go to other arrays than
// the loads of the same phase (p' to the other buffers in the dual step; v
// and w of the pixel itself in the primal step), so nothing orders a later
// pixel's loads after an earlier pixel's stores, and U pixels' chains of two
// dependent loads (the neighbourhood, then the neighbours) overlap.  Loads
// whose use depends on a flag are issued unconditionally where the index is
// always valid (w at a + 1, p2 at a - 1, clamped into [0, n)) and selected
// afterwards.

// Where a block reads its pixels' neighbourhoods and theta lambda f, which no
// step writes.  The neighbourhoods from copies in shared memory made at the
// start of the launch (indexed from the block's first pixel a0) when SM, so
// that the first load of each step's chain of two is a shared-memory load and
// only the neighbours' values come from L2; theta lambda f from shared memory
// too when SMF (an independent load: worth the 4 bytes only while they
// leave the block's pixels room); else from the global arrays.
template <bool SM, bool SMF>
struct RmNbh {
    const uint16_t *fl, *dd, *du;
    const float* F;
    int a0;
    __device__ __forceinline__ uint32_t flags(int a) const { return SM ? fl[a - a0] : __ldg(fl + a); }
    __device__ __forceinline__ int down(int a) const { return SM ? dd[a - a0] : __ldg(dd + a); }
    __device__ __forceinline__ int up(int a) const { return SM ? du[a - a0] : __ldg(du + a); }
    __device__ __forceinline__ float tlf(int a) const { return SMF ? F[a - a0] : __ldg(F + a); }
};

// Dual step (dual_one's arithmetic) at pixels a[0..U): reads p, w of the
// current iterate, writes p' to the other buffers.
template <typename T, bool SM, bool SMF, int U>
__device__ __forceinline__ void rm_dual(const IterParams& P, const RowMajorState<T>& S, const RmNbh<SM, SMF>& N,
                                        const int (&a)[U], int n, const T* __restrict__ P1i,
                                        const T* __restrict__ P2i, T* __restrict__ P1o, T* __restrict__ P2o,
                                        uint32_t seed) {
    const float* __restrict__ Wc = S.Wc;
    uint32_t fl[U];
    int dd[U], du[U];
    float p1[U], p2[U], w0[U], wr[U], xd[U], xr[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        fl[k] = N.flags(a[k]);
        dd[k] = N.down(a[k]);
        du[k] = N.up(a[k]);
        p1[k] = Store<T>::ldc(P1i, a[k]);
        p2[k] = Store<T>::ldc(P2i, a[k]);
        w0[k] = Wc[a[k]];
        wr[k] = Wc[min(a[k] + 1, n - 1)];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        // x + e1: w there when in RD, else p2 at x + e1 - e2 (0 unless in RD);
        // x + e2 fixed: p1 at x - e1 + e2 (0 unless in RD)
        const int d0 = a[k] + dd[k];
        const int ur = a[k] - du[k] + ((fl[k] & RM_UP_RD) ? 1 : 0);
        xd[k] = (fl[k] & RM_DOWN_RD) ? Wc[d0] : (fl[k] & RM_DL_RD) ? Store<T>::ldc(P2i, d0 - 1) : 0.f;
        xr[k] = (fl[k] & (RM_RIGHT_RD | RM_UR_RD)) == RM_UR_RD ? Store<T>::ldc(P1i, ur) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const uint32_t f = fl[k];
        float g1 = 0.f, g2 = 0.f;
        if (!(f & RM_DOWN_OUT))
            g1 = ((f & RM_DOWN_RD) ? xd[k] : rm_w_fixed(p1[k], xd[k], f & RM_DOWN_FG, P.inv_theta)) - w0[k];
        if (!(f & RM_RIGHT_OUT))
            g2 = ((f & RM_RIGHT_RD) ? wr[k] : rm_w_fixed(xr[k], p2[k], f & RM_RIGHT_FG, P.inv_theta)) - w0[k];
        float q1, q2;
        chambolle_update(p1[k], p2[k], g1, g2, P.tau, q1, q2);
        const uint32_t rnd = mix32((uint32_t)a[k] * 3u + seed);
        // bf16 rounding takes the low 16 bits of its word, so one hash serves
        // both components there (its high half for p2)
        const uint32_t rnd2 = std::is_same<T, __nv_bfloat16>::value ? rnd >> 16 : mix32(rnd ^ 0x9e3779b9u);
        Store<T>::st_sr(P1o, a[k], q1, rnd);
        Store<T>::st_sr(P2o, a[k], q2, rnd2);
    }
}

// Primal step (primal_one's arithmetic) at pixels a[0..U): u' = v - theta
// div p', v' = clip(u' - theta lambda f) in place, w' for the next dual step;
// wonly: just w = div p - v/theta (a warm start).
template <typename T, bool SM, bool SMF, int U>
__device__ __forceinline__ void rm_primal(const IterParams& P, const RowMajorState<T>& S, const RmNbh<SM, SMF>& N,
                                          const int (&a)[U], const T* __restrict__ P1n,
                                          const T* __restrict__ P2n, bool wonly, bool check, bool write_u,
                                          bool write_prev, uint32_t seed, float& du2, float& dv2) {
    uint32_t fl[U];
    int du[U];
    float q1[U], q2[U], vv[U], ff[U], q2l[U], q1u[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        fl[k] = N.flags(a[k]);
        du[k] = N.up(a[k]);
        q1[k] = Store<T>::ldc(P1n, a[k]);
        q2[k] = Store<T>::ldc(P2n, a[k]);
        vv[k] = Store<T>::ld_rw(S.v, a[k]) + Store<T>::vbias;
        ff[k] = N.tlf(a[k]);   // theta lambda f
        q2l[k] = Store<T>::ldc(P2n, max(a[k] - 1, 0));
    }
#pragma unroll
    for (int k = 0; k < U; ++k) q1u[k] = (fl[k] & RM_UP_RD) ? Store<T>::ldc(P1n, a[k] - du[k]) : 0.f;
#pragma unroll
    for (int k = 0; k < U; ++k) {
        const float div = (q1[k] - q1u[k]) + (q2[k] - ((fl[k] & RM_LEFT_RD) ? q2l[k] : 0.f));
        if (wonly) {
            S.Wc[a[k]] = div - vv[k] * P.inv_theta;
            continue;
        }
        const float un = fmaf(-P.theta, div, vv[k]);
        const float vn = clamp01(un - ff[k]);
        const float vs = Store<T>::st_sr(S.v, a[k], vn - Store<T>::vbias, mix32((uint32_t)a[k] * 5u + seed)) +
                         Store<T>::vbias;
        S.Wc[a[k]] = div - vs * P.inv_theta;
        if (check) {
            const float da = un - S.Up[a[k]], db = vn - vv[k];
            du2 = fmaf(da, da, du2);
            dv2 = fmaf(db, db, dv2);
        }
        if (write_prev) S.Up[a[k]] = un;
        if (write_u) S.U[a[k]] = un;
    }
}

// All iterations of one launch for a block that owns the pixels [a0, a1) of
// the row-major compact order: dual phase, grid barrier, primal phase (and
// the Section 4 partials), grid barrier; the stopping test as in the other
// compact paths.  Each barrier is split into arrival and wait around the
// block's interior pixels of the next phase, which read only what this block
// wrote: the primal steps of the pixels whose up and left neighbours are the
// block's own ([ep, a1)), and the next iteration's dual steps of the pixels
// whose right and lower neighbours' w are the block's own ([a0, bd)).  The
// rest (the first and last row or so of the range) waits for the barrier.
// A dual step done after the stopping test fired writes only the p buffer
// that is not the result's.
template <typename T, bool SM, bool SMF>
__device__ __forceinline__ void rm_iterations(const IterParams& P, const RowMajorState<T>& S,
                                              const RmNbh<SM, SMF>& N,
                                              int n, int a0, int a1, int iters, int check_every, double tol,
                                              int warm, double* partials, WsHeader* h, double* s_red) {
    const unsigned nblocks = gridDim.x;
    const int tid = threadIdx.x, nt = kRmThreads;
    unsigned gen = 0u;
    // the split points: bd = the first pixel whose dual step reads w of
    // another block (x + e1 or x + e2 in RD at or beyond a1; the lower
    // neighbours' positions grow with a, so every later pixel is treated
    // alike), ep = one past the last pixel whose primal step reads p' of
    // another block (x - e1 or x - e2 in RD before a0)
    __shared__ int s_split[2];
    if (tid == 0) {
        s_split[0] = a1;
        s_split[1] = a0;
    }
    __syncthreads();
    {
        int bd = a1, ep = a0;
        for (int a = a0 + tid; a < a1; a += nt) {
            const uint32_t f = N.flags(a);
            if (((f & RM_DOWN_RD) && a + N.down(a) >= a1) || ((f & RM_RIGHT_RD) && a + 1 >= a1)) bd = min(bd, a);
            if (((f & RM_UP_RD) && a - N.up(a) < a0) || ((f & RM_LEFT_RD) && a - 1 < a0)) ep = max(ep, a + 1);
        }
        if (bd < a1) atomicMin(&s_split[0], bd);
        if (ep > a0) atomicMax(&s_split[1], ep);
    }
    __syncthreads();
    const int bd = s_split[0], ep = s_split[1];
    // op(pixels[U]) over [b0, b1), U = kRmUnroll pixels a thread at a time
    // (stride nt), then the rest one by one
    auto each = [&](int b0, int b1, auto&& op) {
        int a = b0 + tid;
        for (; a + (kRmUnroll - 1) * nt < b1; a += kRmUnroll * nt) {
            int b[kRmUnroll];
#pragma unroll
            for (int k = 0; k < kRmUnroll; ++k) b[k] = a + k * nt;
            op(b);
        }
        for (; a < b1; a += nt) {
            const int b[1] = {a};
            op(b);
        }
    };
    float d0 = 0.f, d1 = 0.f;
    if (warm) {
        for (int a = a0 + tid; a < a1; a += nt) {
            const int b[1] = {a};
            rm_primal(P, S, N, b, S.p1[0], S.p2[0], true, false, false, false, 0u, d0, d1);
        }
        if (!grid_sync(h, nblocks, gen)) return;
    }
    // dual steps of iteration `it` over [b0, b1): p of buffer it & 1 into the
    // other (the buffers picked by the parity in two copies, so that every
    // array base stays a kernel parameter)
    auto dual = [&](int it, int b0, int b1) {
        const uint32_t seed_d = mix32(0x51ed270bu ^ (uint32_t)(it * 131));
        if (it & 1)
            each(b0, b1, [&](const auto& b) { rm_dual(P, S, N, b, n, S.p1[1], S.p2[1], S.p1[0], S.p2[0], seed_d); });
        else
            each(b0, b1, [&](const auto& b) { rm_dual(P, S, N, b, n, S.p1[0], S.p2[0], S.p1[1], S.p2[1], seed_d); });
    };
    const int C = check_every;
    if (iters > 0) dual(0, a0, a1);
    for (int it = 0; it < iters; ++it) {
        const int l = it + 1;
        // p' of this iteration is in buffer l & 1
        grid_arrive(h, gen);
        const bool check = (l % C == 0) || l == iters;
        const bool write_prev = l < iters && ((l + 1) % C == 0 || l + 1 == iters);
        const uint32_t seed = mix32(0x2545f491u ^ (uint32_t)it);
        float du2 = 0.f, dv2 = 0.f;
        // primal steps over [b0, b1) with p' of buffer l & 1
        auto primal = [&](int b0, int b1) {
            if (l & 1) {
                if (!check && !write_prev)
                    each(b0, b1, [&](const auto& b) {
                        rm_primal(P, S, N, b, S.p1[1], S.p2[1], false, false, false, false, seed, du2, dv2);
                    });
                else
                    each(b0, b1, [&](const auto& b) {
                        rm_primal(P, S, N, b, S.p1[1], S.p2[1], false, check, check, write_prev, seed, du2, dv2);
                    });
            } else {
                if (!check && !write_prev)
                    each(b0, b1, [&](const auto& b) {
                        rm_primal(P, S, N, b, S.p1[0], S.p2[0], false, false, false, false, seed, du2, dv2);
                    });
                else
                    each(b0, b1, [&](const auto& b) {
                        rm_primal(P, S, N, b, S.p1[0], S.p2[0], false, check, check, write_prev, seed, du2, dv2);
                    });
            }
        };
        // after a stopping test the barrier may end the solve, so no primal
        // step runs before it there
        const bool poll = it > 0 && (it % C == 0);
        const bool early = !(poll && tol > 0.0);
        if (early) primal(ep, a1);
        bool done;
        if (!grid_wait(h, nblocks, gen, poll, done)) return;
        if (done) return;   // the previous iteration's stopping test fired
        if (early)
            primal(a0, ep);
        else
            primal(a0, a1);
        if (check) {
            float x = du2, y = dv2;
            block_sum2f<kRmThreads>(x, y, reinterpret_cast<float*>(s_red));
            if (tid == 0) {
                partials[2 * blockIdx.x] = x;
                partials[2 * blockIdx.x + 1] = y;
            }
        }
        grid_arrive(h, gen);
        if (l < iters) dual(l, a0, bd);
        if (!grid_wait(h, nblocks, gen)) return;
        if (check && blockIdx.x == 0) {
            // Section 4 stopping test: fixed-order FP64 sum of the block
            // partials, squared norms against tol^2
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
        if (l < iters) dual(l, bd, a1);
    }
}

// Shared memory of one block, sized for kRmMinBlocks blocks per SM: the
// neighbourhood (three 16-bit words) and theta lambda f of up to
// kRmSmemPixelsF pixels, or the neighbourhood alone of up to kRmSmemPixels.
constexpr size_t kRmSmemBytes = (225 * 1024 / kRmMinBlocks - 2048) / 60 * 60;
constexpr int kRmSmemPixelsF = (int)(kRmSmemBytes / 10);
constexpr int kRmSmemPixels = (int)(kRmSmemBytes / 6);

// All iterations in one cooperative launch: each block owns a contiguous
// range of the row-major compact order.  SMEM (launched with kRmSmemBytes of
// shared memory, for RD counts up to smem_above): each block keeps its
// pixels' neighbourhoods, and theta lambda f, in shared memory as far as they
// fit (the same choice in every block: the ranges differ by at most one
// pixel).  Else (launched without, so that the L1 keeps the whole of its
// on-chip memory for the global arrays; above smem_above) everything is read
// from the global arrays.  Both are launched when the RD count is not known
// on the host; the one that does not apply returns at once.
template <typename T, bool SMEM>
__global__ void __launch_bounds__(kRmThreads, kRmMinBlocks)
k_solve_wide_rm(IterParams P, RowMajorState<T> S, const int32_t* __restrict__ counts, long long wide_above,
                long long smem_above, int iters, int check_every, double tol, int warm, double* partials,
                WsHeader* h) {
    __shared__ double s_red[66];   // block_sum2f (as floats), stop flag
    extern __shared__ __align__(16) unsigned char rm_smem[];
    if (*(volatile int*)&h->done) return;
    const int n = counts[1];
    if (n <= wide_above) return;
    if (SMEM ? n > smem_above : n <= smem_above) return;   // the other launch's
    const unsigned nblocks = gridDim.x;
    const int per = (n + (int)nblocks - 1) / (int)nblocks;
    const int a0 = (int)blockIdx.x * per, a1 = min(n, a0 + per);
    if (!SMEM) {
        rm_iterations<T, false, false>(P, S, RmNbh<false, false>{S.fl, S.dd, S.du, S.F, 0}, n, a0, a1, iters,
                                       check_every, tol, warm, partials, h, s_red);
    } else if (per <= kRmSmemPixelsF) {   // the same choice in every block
        float* sF = reinterpret_cast<float*>(rm_smem);
        uint16_t* sfl = reinterpret_cast<uint16_t*>(sF + kRmSmemPixelsF);
        uint16_t* sdd = sfl + kRmSmemPixelsF;
        uint16_t* sdu = sdd + kRmSmemPixelsF;
        for (int i = threadIdx.x; i < a1 - a0; i += kRmThreads) {
            sF[i] = __ldg(S.F + a0 + i);
            sfl[i] = __ldg(S.fl + a0 + i);
            sdd[i] = __ldg(S.dd + a0 + i);
            sdu[i] = __ldg(S.du + a0 + i);
        }
        __syncthreads();
        rm_iterations<T, true, true>(P, S, RmNbh<true, true>{sfl, sdd, sdu, sF, a0}, n, a0, a1, iters,
                                     check_every, tol, warm, partials, h, s_red);
    } else if (per <= kRmSmemPixels) {
        uint16_t* sfl = reinterpret_cast<uint16_t*>(rm_smem);
        uint16_t* sdd = sfl + kRmSmemPixels;
        uint16_t* sdu = sdd + kRmSmemPixels;
        for (int i = threadIdx.x; i < a1 - a0; i += kRmThreads) {
            sfl[i] = __ldg(S.fl + a0 + i);
            sdd[i] = __ldg(S.dd + a0 + i);
            sdu[i] = __ldg(S.du + a0 + i);
        }
        __syncthreads();
        rm_iterations<T, true, false>(P, S, RmNbh<true, false>{sfl, sdd, sdu, S.F, a0}, n, a0, a1, iters,
                                      check_every, tol, warm, partials, h, s_red);
    }
}

// ------------------------------------------------------------ scatter

// Dense u, v, p1, p2 of the final iterate (one warp per row): compact values
// on RD, the fixed values elsewhere.
template <typename T>
__global__ void k_rm_scatter(RowMajorArgs R, RowMajorState<T> S, int iters, long long cap) {
    if (R.counts[1] <= R.wide_above) return;
    const int lane = threadIdx.x & 31;
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= R.H) return;
    const bool ok = R.counts[1] <= cap && R.rowstart[R.H] == R.counts[1];
    const int l = R.h->done ? R.h->iters_done : iters;
    const int pb = l & 1;
    const T* P1 = pb ? S.p1[1] : S.p1[0];
    const T* P2 = pb ? S.p2[1] : S.p2[0];
    int pre = 0;
    for (int c0 = 0; c0 < R.ntx; c0 += 32) {
        const int k = c0 + lane;
        const bool in = k < R.ntx;
        const int64_t o = (int64_t)i * R.nw + k;
        const uint32_t wc = in ? __ldg(R.act + o) : 0u;
        const uint32_t fc = in ? __ldg(R.fg + o) : 0u;
        const int cc = __popc(wc);
        int sc = cc;
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, sc, d);
            if (lane >= d) sc += t;
        }
        const int wpre = pre + sc - cc;
        if (in) {
            for (int b = 0; b < 32; ++b) {
                const int j = 32 * k + b;
                if (j >= R.W) break;
                const int64_t off = (int64_t)i * R.ld + j;
                if (ok && ((wc >> b) & 1u)) {
                    const int a = rm_pos(R.rowstart, i, wpre, wc, b);
                    R.u[off] = S.U[a];
                    R.v[off] = Store<T>::ld_rw(S.v, a) + Store<T>::vbias;
                    R.p1[off] = Store<T>::ld_rw(P1, a);
                    R.p2[off] = Store<T>::ld_rw(P2, a);
                } else {
                    const float hh = ((fc >> b) & 1u) ? 1.f : 0.f;
                    R.u[off] = hh; R.v[off] = hh; R.p1[off] = 0.f; R.p2[off] = 0.f;
                }
            }
        }
        pre = __shfl_sync(0xffffffffu, wpre + cc, 31);
    }
}

// ------------------------------------------------------------ host

template <typename T>
static seg_status run_wide_rm_t(const RowMajorArgs& R, const RowMajorArrays& A, const IterParams& P,
                                const seg_params* prm, double* partials, long long max_partials,
                                cudaStream_t s) {
    const RowMajorState<T> S = rm_state<T>(A);
    const unsigned row_blocks = (unsigned)std::max(1, (R.H * 32 + 255) / 256);
    k_rm_rowcount<<<row_blocks, 256, 0, s>>>(R);
    SEG_LAUNCHED("k_rm_rowcount");
    k_rm_rowscan<<<1, 1024, 0, s>>>(R);
    SEG_LAUNCHED("k_rm_rowscan");
    k_rm_gather<T><<<row_blocks, 256, 0, s>>>(R, S, prm->warm_start);
    SEG_LAUNCHED("k_rm_gather");
    const long long most = std::max<long long>(1, std::min<long long>(A.cap, (long long)R.H * R.W));
    auto grid_of = [&](const void* k, size_t smem, int& grid) -> seg_status {
        int per_sm = 0;
        SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kRmThreads, smem));
        if (per_sm <= 0) return fail(SEG_ERR_CUDA, "k_solve_wide_rm cannot be resident");
        grid = (int)std::min<long long>((long long)per_sm * sm_count(), (most + kRmThreads - 1) / kRmThreads);
        grid = std::max(1, (int)std::min<long long>(grid, max_partials));
        return SEG_OK;
    };
    const void* ks = (const void*)k_solve_wide_rm<T, true>;
    const void* kg = (const void*)k_solve_wide_rm<T, false>;
    SEG_TRY_CUDA(cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRmSmemBytes));
    int grid_s = 1, grid_g = 1;
    SEG_TRY(grid_of(ks, kRmSmemBytes, grid_s));
    SEG_TRY(grid_of(kg, 0, grid_g));
    IterParams Pk = P;
    RowMajorState<T> Sk = S;
    const int32_t* counts = R.counts;
    long long above = R.wide_above;
    long long smem_above = (long long)kRmSmemPixels * grid_s;   // per <= kRmSmemPixels in every block
    int iters = prm->iters, ce = test_interval(prm->tol, prm->check_every, prm->iters);
    double tol = prm->tol;
    int warm = prm->warm_start;
    WsHeader* h = R.h;
    void* args[] = {&Pk, &Sk, (void*)&counts, &above, &smem_above, &iters, &ce, &tol, &warm, &partials, &h};
    if (iters > 0 || warm) {
        SEG_TRY_CUDA(cudaLaunchCooperativeKernel(ks, dim3(grid_s), dim3(kRmThreads), args, kRmSmemBytes, s));
        count_launch();
        if (debug_mode()) SEG_TRY(after_launch("k_solve_wide_rm (shared memory)"));
        if (most > smem_above) {   // an RD count beyond the shared-memory launch is possible
            SEG_TRY_CUDA(cudaLaunchCooperativeKernel(kg, dim3(grid_g), dim3(kRmThreads), args, 0, s));
            count_launch();
            if (debug_mode()) SEG_TRY(after_launch("k_solve_wide_rm (global memory)"));
        }
    }
    k_rm_scatter<T><<<row_blocks, 256, 0, s>>>(R, S, prm->iters, A.cap);
    SEG_LAUNCHED("k_rm_scatter");
    return SEG_OK;
}

seg_status run_wide_rm(const RowMajorArgs& R, const RowMajorArrays& A, const IterParams& P,
                       const seg_params* prm, double* partials, long long max_partials, cudaStream_t s) {
    switch (prm->storage) {
        case SEG_STORE_F32: return run_wide_rm_t<float>(R, A, P, prm, partials, max_partials, s);
        case SEG_STORE_BF16: return run_wide_rm_t<__nv_bfloat16>(R, A, P, prm, partials, max_partials, s);
        default: return run_wide_rm_t<__half>(R, A, P, prm, partials, max_partials, s);
    }
}

}  // namespace seg
