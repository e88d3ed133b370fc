// tiled.cu -- temporally blocked solve (SEG_MODE_TILED).
//
// The iteration of Sections 2.1 and 3, with the same arithmetic as the dense
// and compact solvers, on the dense [H][ld] ping-pong state, several outer
// iterations per pass over the image.
//
// The image is cut into own regions of Ro x Co pixels.  A window adds a halo
// of hb + 1 rows / columns above and left and hb below and right, where hb =
// iterations per sweep x fixed-point sweeps per iteration.  For p'(x) one
// fixed-point sweep reads p at x and its six stencil neighbours and v at x,
// x+e1, x+e2; the v-step reads p' at x, x-e1, x-e2.  So every pixel whose
// inputs lie in the window computes exactly the value of the unblocked
// iteration, and the set of such pixels shrinks by one pixel on every side
// per fixed-point sweep, and for v by one more row / column above and left.
// After kk <= hb / n_inner iterations the own region is still exact.  Each
// window is therefore loaded once per sweep by TMA (its zero fill outside the
// image gives p = 0 there, and the gradient components across the last row /
// column are zeroed explicitly), iterated kk times in shared memory over the
// list of its RD pixels (fixed pixels keep p = 0 and v = H(-f) as loaded), and
// its own region is written to the other ping-pong buffer.
//
// One persistent cooperative launch runs all the sweeps, separated by the
// bounded grid barrier.  Windows are handed out by an atomic ticket per
// sweep; the stopping test of Section 4 sums per-window partials in window
// order, and every block computes that sum itself, so results and the
// iteration at which the solve stops do not depend on the schedule.
#include <cuda.h>

#include <algorithm>
#include <cstdlib>

#include "iterate.cuh"

namespace seg {

constexpr int kTbCols = 68;              // window width = shared-memory row pitch (floats)
constexpr int kTbRows = 60;              // window height
constexpr int kTbPix = kTbRows * kTbCols;
constexpr int kTbFront = 96;             // floats before each plane's window
constexpr int kTbPlane = 4288;           // floats per plane: front guard, window, back guard
static_assert(kTbFront >= kTbCols + 1 && (kTbFront * 4) % 128 == 0, "front guard: one row, TMA alignment");
static_assert(kTbPlane - kTbFront - kTbPix >= kTbCols + 1 && (kTbPlane * 4) % 128 == 0, "back guard");
constexpr int kTbMaxHalo = 8;            // largest hb = sweep x n_inner
constexpr int kTbDefaultSweep = 4;
constexpr size_t kTbListBytes = ((size_t)kTbPix * 2 + 127) / 128 * 128;
static_assert((kTbPix * 2) % 16 == 0, "list slots must keep bulk copies 16-byte aligned");
// shared memory: NBUF input buffers {p1, p2, v, f, RD list}, two scratch p
// planes, a little scratch.  NBUF = 2 (one block of 1024 threads per SM)
// loads the next window while the current one is iterated; NBUF = 1 (two
// blocks of 512 threads per SM) overlaps one block's loads with the other's
// iterations.
constexpr size_t kTbBufBytes = 4 * (size_t)kTbPlane * 4 + kTbListBytes;
constexpr size_t tb_scratch_off(int nbuf) { return nbuf * kTbBufBytes; }
constexpr size_t tb_misc_off(int nbuf) { return tb_scratch_off(nbuf) + 2 * (size_t)kTbPlane * 4; }
constexpr size_t tb_smem(int nbuf) { return tb_misc_off(nbuf) + 1024 + 128; }   // + 128: base alignment
constexpr int tb_threads(int nbuf) { return nbuf == 2 ? 1024 : 512; }

struct TbGeom {
    int hb;          // halo budget: iterations per sweep x fixed-point sweeps
    int T, L;        // halo above / left of the own region (L a multiple of 4)
    int Ro, Co;      // own region (Co a multiple of 4)
    int nwx, nwin;   // windows per row of windows, windows in all
};

// TMA descriptors of the ping-pong state planes and of f (kernel parameters)
struct TbMaps {
    CUtensorMap p1[2], p2[2], v[2], f;
};

// Per-window RD lists, built once per solve: the RD pixels of window w as
// (row << 7) | column in row-major order at lists[w * kTbPix], their number
// and the number inside the own region in counts[w], and the ascending list
// of windows whose own region holds an RD pixel (the only ones a sweep
// visits) with its length in *nact.
__global__ void k_tb_lists(IterParams P, TbGeom G, const uint32_t* __restrict__ act,
                           uint16_t* __restrict__ lists, int2* __restrict__ counts) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= G.nwin) return;
    const int wy = w / G.nwx, wx = w - wy * G.nwx;
    const int i0 = wy * G.Ro - G.T, j0 = wx * G.Co - G.L;
    uint16_t* out = lists + (int64_t)w * kTbPix;
    int n = 0, n_own = 0;
    for (int r = 0; r < kTbRows; ++r) {
        const int gi = i0 + r;
        const bool row_in = gi >= 0 && gi < P.H;
        const bool row_own = r >= G.T && r < G.T + G.Ro;
        for (int k = 0; k < 3; ++k) {
            const int c = 32 * k + lane, gj = j0 + c;
            bool a = false;
            if (row_in && c < kTbCols && gj >= 0 && gj < P.W)
                a = (__ldg(act + (int64_t)gi * P.nw + (gj >> 5)) >> (gj & 31)) & 1u;
            const unsigned m = __ballot_sync(FULL, a);
            if (a) out[n + __popc(m & lanemask_lt(lane))] = (uint16_t)((r << 7) | c);
            n += __popc(m);
            n_own += __popc(__ballot_sync(FULL, a && row_own && c >= G.L && c < G.L + G.Co));
        }
    }
    if (lane == 0) counts[w] = make_int2(n, n_own);
}

// Ascending list of the windows with an RD pixel in their own region.
__global__ void __launch_bounds__(1024)
k_tb_active(TbGeom G, const int2* __restrict__ counts, int* __restrict__ active, int* __restrict__ nact) {
    __shared__ int s_warp[32];
    __shared__ int s_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < G.nwin; c0 += 1024) {
        const int w = c0 + tid;
        const bool on = w < G.nwin && counts[w].y > 0;
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (lane == 0) s_warp[wid] = __popc(m);
        __syncthreads();
        int pre = s_base;
        for (int k = 0; k < wid; ++k) pre += s_warp[k];
        if (on) active[pre + __popc(m & lanemask_lt(lane))] = w;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int k = 0; k < 32; ++k) t += s_warp[k];
            s_base += t;
        }
        __syncthreads();
    }
    if (tid == 0) *nact = s_base;
}

// Fixed-point step for p at one RD pixel of the window (packed (row << 7) |
// column), from p and v in shared memory:
//   w(y) = div p(y) - v(y)/theta at y = x, x+e1, x+e2,
//   g = (w(x+e1) - w(x), w(x+e2) - w(x)), zero across the last row / column,
//   p'(x) = (p(x) + tau g) / (1 + tau |g|).
__device__ __forceinline__ void tb_dual(const IterParams& P, int rc, int rlim, int clim,
                                        const float* p1, const float* p2, const float* V,
                                        float* q1, float* q2) {
    const int r = rc >> 7, c = rc & 127, o = r * kTbCols + c;
    const float p1x = p1[o], p1u = p1[o - kTbCols], p1d = p1[o + kTbCols];
    const float p1r = p1[o + 1], p1ur = p1[o + 1 - kTbCols];
    const float p2x = p2[o], p2l = p2[o - 1], p2d = p2[o + kTbCols];
    const float p2dl = p2[o + kTbCols - 1], p2r = p2[o + 1];
    const float w0 = ((p1x - p1u) + (p2x - p2l)) - V[o] * P.inv_theta;
    const float wd = ((p1d - p1x) + (p2d - p2dl)) - V[o + kTbCols] * P.inv_theta;
    const float wr = ((p1r - p1ur) + (p2r - p2x)) - V[o + 1] * P.inv_theta;
    const float g1 = r < rlim ? wd - w0 : 0.f;
    const float g2 = c < clim ? wr - w0 : 0.f;
    float a, b;
    chambolle_update(p1x, p2x, g1, g2, P.tau, a, b);
    q1[o] = a;
    q2[o] = b;
}

template <int NBUF>
struct TbSmem {
    unsigned char* base;
    __device__ float* p1(int b) const { return reinterpret_cast<float*>(base + b * kTbBufBytes) + kTbFront; }
    __device__ float* p2(int b) const { return p1(b) + kTbPlane; }
    __device__ float* v(int b) const { return p1(b) + 2 * kTbPlane; }
    __device__ float* f(int b) const { return p1(b) + 3 * kTbPlane; }
    __device__ uint16_t* list(int b) const {
        return reinterpret_cast<uint16_t*>(base + b * kTbBufBytes + 4 * (size_t)kTbPlane * 4);
    }
    __device__ float* s1() const { return reinterpret_cast<float*>(base + tb_scratch_off(NBUF)) + kTbFront; }
    __device__ float* s2() const { return s1() + kTbPlane; }
};

template <int NBUF>
__global__ void __launch_bounds__(tb_threads(NBUF), 2 / NBUF)
k_solve_tiled(IterParams P, TbGeom G, int iters, int n_inner, int kmax, int check_every, double tol,
              const __grid_constant__ TbMaps maps, const uint16_t* __restrict__ lists,
              const int2* __restrict__ counts, const int* __restrict__ active,
              const int* __restrict__ nact_p, float* st, float* u, double* partials, WsHeader* h) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int kTbThreads = tb_threads(NBUF);
    TbSmem<NBUF> S{reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                    ~static_cast<uintptr_t>(127))};
    unsigned char* const misc = S.base + tb_misc_off(NBUF);
    uint64_t* const bar = reinterpret_cast<uint64_t*>(misc);             // [2]
    int* const s_a = reinterpret_cast<int*>(misc + 16);                  // [2] active index per buffer
    int* const s_w = reinterpret_cast<int*>(misc + 24);                  // [2] window per buffer
    int* const s_n = reinterpret_cast<int*>(misc + 32);                  // [2] RD pixels per buffer
    int* const s_first = reinterpret_cast<int*>(misc + 40);              // first ticket of a sweep
    int* const s_next = reinterpret_cast<int*>(misc + 44);               // next ticket (NBUF = 1)
    double* const s_red = reinterpret_cast<double*>(misc + 64);          // [66]: block_sum2f (as floats), stop flag

    if (*(volatile int*)&h->done) return;
    const int tid = threadIdx.x;
    const unsigned nblocks = gridDim.x;
    const int64_t plane = (int64_t)P.H * P.ld;
    const int nact = *nact_p;
    // guards and the scratch planes start at zero (fixed pixels hold p = 0)
    for (int k = tid; k < (int)(tb_misc_off(NBUF) / 4); k += kTbThreads) reinterpret_cast<float*>(S.base)[k] = 0.f;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
        *s_first = atomicAdd(&h->tb_ticket[0], 1);
    }
    __syncthreads();

    // thread 0: loads of active window `a` into buffer b (planes by tiled TMA,
    // the RD list by a bulk copy), all completing on bar[b]
    auto issue = [&](int a, int b, int cur_g) {
        const int w = active[a];
        const int n = counts[w].x;
        const int wy = w / G.nwx, wx = w - wy * G.nwx;
        const int i0 = wy * G.Ro - G.T, j0 = wx * G.Co - G.L;
        const uint32_t lb = (uint32_t)((2 * n + 15) & ~15);
        s_w[b] = w;
        s_n[b] = n;
        fence_proxy_async_global();
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar + b, 4u * kTbPix * 4u + lb);
        tma_load_2d(S.p1(b), &maps.p1[cur_g], j0, i0, bar + b);
        tma_load_2d(S.p2(b), &maps.p2[cur_g], j0, i0, bar + b);
        tma_load_2d(S.v(b), &maps.v[cur_g], j0, i0, bar + b);
        tma_load_2d(S.f(b), &maps.f, j0, i0, bar + b);
        if (lb) bulk_g2s(S.list(b), lists + (int64_t)w * kTbPix, lb, bar + b);
    };

    unsigned gen = 0u;
    uint32_t ph0 = 0u, ph1 = 0u;
    int l0 = 0, sweep = 0, chk = 0, cur_g = 0;
    const int C = check_every;
    while (l0 < iters) {
        const int bnd = min(iters, (l0 / C + 1) * C);
        const int kk = min(kmax, bnd - l0);
        const int l1 = l0 + kk;
        const bool is_check = (l1 % C == 0) || l1 == iters;
        // the ticket of sweep + 2 was last used two barriers ago
        if (blockIdx.x == 0 && tid == 0) h->tb_ticket[(sweep + 2) & 3] = 0;
        float* const N1 = st + (int64_t)(cur_g ^ 1) * plane;
        float* const N2 = st + (int64_t)(2 + (cur_g ^ 1)) * plane;
        float* const NV = st + (int64_t)(4 + (cur_g ^ 1)) * plane;
        double* const part = partials + 2 * (int64_t)(chk & 1) * G.nwin;
        if (tid == 0) {
            const int a = *s_first;
            s_a[0] = a;
            if (a < nact) issue(a, 0, cur_g);
        }
        int b = 0;
        for (;;) {
            __syncthreads();
            const int a = s_a[b];
            if (a >= nact) break;
            if (tid == 0) {
                const int an = atomicAdd(&h->tb_ticket[sweep & 3], 1);
                if (NBUF == 2) {   // the next window goes to the other buffer, freed by the last sync
                    s_a[b ^ 1] = an;
                    if (an < nact) issue(an, b ^ 1, cur_g);
                } else {
                    *s_next = an;
                }
            }
            const bool ok = mbar_wait_bounded(bar + b, b ? ph1 : ph0, h);
            if (b) ph1 ^= 1u; else ph0 ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {   // copies may still be in flight
                    mbar_wait_bounded(bar, ph0, h);
                    if (NBUF == 2) mbar_wait_bounded(bar + 1, ph1, h);
                }
                h->done = 1;
                return;
            }
            const int w = s_w[b], n = s_n[b];
            const int wy = w / G.nwx, wx = w - wy * G.nwx;
            const int i0 = wy * G.Ro - G.T, j0 = wx * G.Co - G.L;
            const uint16_t* list = S.list(b);
            float* const V = S.v(b);
            const float* const F = S.f(b);
            float du2 = 0.f, dv2 = 0.f;
            {
                const int rlim = P.H - 1 - i0, clim = P.W - 1 - j0;
                const int rT = G.T, rE = G.T + G.Ro, cL = G.L, cE = G.L + G.Co;
                int cur = 0;   // 0: p in buffer b, 1: p in the scratch planes
                for (int it = 0; it < kk; ++it) {
                    for (int sw = 0; sw < n_inner; ++sw) {
                        const float* p1 = cur ? S.s1() : S.p1(b);
                        const float* p2 = cur ? S.s2() : S.p2(b);
                        float* q1 = cur ? S.p1(b) : S.s1();
                        float* q2 = cur ? S.p2(b) : S.s2();
                        int e = tid;
                        for (; e + kTbThreads < n; e += 2 * kTbThreads) {
                            tb_dual(P, list[e], rlim, clim, p1, p2, V, q1, q2);
                            tb_dual(P, list[e + kTbThreads], rlim, clim, p1, p2, V, q1, q2);
                        }
                        if (e < n) tb_dual(P, list[e], rlim, clim, p1, p2, V, q1, q2);
                        __syncthreads();
                        cur ^= 1;
                    }
                    // v-step on the RD pixels; u of the own region is written
                    // at the end of the sweep, and one iteration earlier when
                    // the sweep ends with a stopping test (the test reads it)
                    const bool last = it == kk - 1;
                    const bool wu = last || (is_check && it == kk - 2);
                    const bool test = is_check && last;
                    const float* q1 = cur ? S.s1() : S.p1(b);
                    const float* q2 = cur ? S.s2() : S.p2(b);
                    for (int e = tid; e < n; e += kTbThreads) {
                        const int rc = list[e];
                        const int r = rc >> 7, c = rc & 127, o = r * kTbCols + c;
                        const float div = (q1[o] - q1[o - kTbCols]) + (q2[o] - q2[o - 1]);
                        const float vv = V[o];
                        const float un = fmaf(-P.theta, div, vv);
                        const float vn = clamp01(fmaf(-P.theta_lambda, F[o], un));
                        V[o] = vn;
                        if (wu && r >= rT && r < rE && c >= cL && c < cE) {
                            float* up = u + (int64_t)(i0 + r) * P.ld + (j0 + c);
                            if (test) {
                                const float da = un - __ldcg(up), db = vn - vv;
                                du2 = fmaf(da, da, du2);
                                dv2 = fmaf(db, db, dv2);
                            }
                            __stcg(up, un);
                        }
                    }
                    __syncthreads();
                }
                // own region -> the other ping-pong buffer (fixed pixels are
                // written back unchanged; columns past W stay zero)
                const int c4 = G.Co >> 2;
                const float* s1 = cur ? S.s1() : S.p1(b);
                const float* s2 = cur ? S.s2() : S.p2(b);
                for (int k = tid; k < G.Ro * c4; k += kTbThreads) {
                    const int rr = k / c4, cc = k - rr * c4;
                    const int r = G.T + rr, c = G.L + 4 * cc;
                    const int gi = i0 + r, gj = j0 + c;
                    if (gi < P.H && gj < P.ld) {
                        const int o = r * kTbCols + c;
                        const int64_t go = (int64_t)gi * P.ld + gj;
                        __stcg(reinterpret_cast<float4*>(N1 + go), *reinterpret_cast<const float4*>(s1 + o));
                        __stcg(reinterpret_cast<float4*>(N2 + go), *reinterpret_cast<const float4*>(s2 + o));
                        __stcg(reinterpret_cast<float4*>(NV + go), *reinterpret_cast<const float4*>(V + o));
                    }
                }
                // the scratch planes are shared by both buffers: clear the RD
                // values this window left there, which may sit on fixed pixels
                // (p = 0) of the next window
                __syncthreads();
                float* z1 = S.s1();
                float* z2 = S.s2();
                for (int e = tid; e < n; e += kTbThreads) {
                    const int rc = list[e];
                    const int o = (rc >> 7) * kTbCols + (rc & 127);
                    z1[o] = 0.f;
                    z2[o] = 0.f;
                }
            }
            if (is_check) {   // per-window partials of the stopping test, fixed order
                float x = du2, y = dv2;
                block_sum2f<kTbThreads>(x, y, reinterpret_cast<float*>(s_red));
                if (tid == 0) {
                    __stcg(part + 2 * a, (double)x);
                    __stcg(part + 2 * a + 1, (double)y);
                }
            }
            if (NBUF == 1) {   // the buffer is free again: load the next window
                __syncthreads();
                if (tid == 0) {
                    const int an = *s_next;
                    s_a[0] = an;
                    if (an < nact) issue(an, 0, cur_g);
                }
            } else {
                b ^= 1;
            }
        }
        // the first ticket of the next sweep (its counter was reset two
        // barriers ago); its loads wait for the barrier
        if (tid == 0) *s_first = atomicAdd(&h->tb_ticket[(sweep + 1) & 3], 1);
        if (!grid_sync(h, nblocks, gen)) return;
        l0 = l1;
        cur_g ^= 1;
        ++sweep;
        if (is_check) {
            // every block sums the window partials in window order (squared
            // norms against tol^2; the square roots are taken once, for the stats)
            if (tid < 32) {
                double x, y;
                sum_partials_warp0(part, nact, x, y);
                if (tid == 0) {
                    const bool stop = tol > 0.0 && fmax(x, y) <= tol * tol;
                    s_red[0] = stop ? 1.0 : 0.0;
                    if (blockIdx.x == 0) {
                        h->du2 = x;
                        h->dv2 = y;
                        h->last_check = l0;
                        if (stop) {
                            h->iters_done = l0;
                            h->done = 1;
                        }
                    }
                }
            }
            __syncthreads();
            const bool stop = s_red[0] != 0.0;
            ++chk;
            __syncthreads();
            if (stop) break;
        }
    }
    if (blockIdx.x == 0 && tid == 0) h->tb_buf = cur_g;
}

// p1, p2, v of the final iterate from the ping-pong buffer the solve ended in.
__global__ void k_final_tiled(IterParams P, const WsHeader* __restrict__ h, const float* __restrict__ st,
                              float* v, float* p1, float* p2) {
    const int64_t plane = (int64_t)P.H * P.ld;
    const int b = h->tb_buf;
    const float* S1 = st + b * plane;
    const float* S2 = st + (2 + b) * plane;
    const float* SV = st + (4 + b) * plane;
    const int64_t n = (int64_t)P.H * P.W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)((uint32_t)x / (uint32_t)P.W), j = x - i * P.W;   // x < 2^31
        const int64_t o = i * P.ld + j;
        p1[o] = S1[o];
        p2[o] = S2[o];
        v[o] = SV[o];
    }
}

// ------------------------------------------------------------------ host

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Descriptor of an H x W float32 image with pitch ld, loaded as kTbCols x
// kTbRows boxes; elements outside the image read as zero.
static seg_status tb_map(CUtensorMap* m, const float* base, int H, int W, int ld) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(SEG_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (reinterpret_cast<uintptr_t>(base) % 16) return fail(SEG_ERR_ALIGN, "TMA source not 16-byte aligned");
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kTbCols, (cuuint32_t)kTbRows};
    const cuuint32_t es[2] = {1u, 1u};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
                           es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SEG_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return SEG_OK;
}

static int round4(int x) { return (x + 3) / 4 * 4; }

// Input buffers per block of the tiled solver (1 or 2; SEG_TILED_BUFFERS
// overrides the default of 1 for experiments).
static int tb_buffers() {
    static int nb = 0;
    if (!nb) {
        const char* e = getenv("SEG_TILED_BUFFERS");
        nb = (e && atoi(e) == 2) ? 2 : 1;
    }
    return nb;
}

static TbGeom tb_geom(int H, int W, int hb) {
    TbGeom G{};
    G.hb = hb;
    G.T = hb + 1;
    G.L = round4(hb + 1);
    G.Ro = kTbRows - G.T - hb;
    G.Co = kTbCols - G.L - round4(hb);
    G.nwx = (W + G.Co - 1) / G.Co;
    G.nwin = G.nwx * ((H + G.Ro - 1) / G.Ro);
    return G;
}

// Bytes after the six state planes: per-window RD lists, counts, the list of
// active windows and its length, for up to nwin windows.
static size_t tb_lists_bytes(int64_t nwin) {
    return align_up((size_t)nwin * kTbPix * 2, 256) + align_up((size_t)nwin * 8, 256) +
           align_up((size_t)nwin * 4 + 4, 256);
}

size_t tiled_state_bytes(int H, int ld) {
    // the most windows any sweep length gives (the smallest own region) on an
    // H x ld image
    const TbGeom G = tb_geom(std::max(H, 1), std::max(ld, 1), kTbMaxHalo);
    return align_up(6 * 4 * (size_t)std::max(H, 0) * (size_t)std::max(ld, 0), 256) + tb_lists_bytes(G.nwin) + 256;
}

seg_status tiled_geometry(int H, int W, int sweep, int n_inner, int* nwin) {
    const int k = sweep > 0 ? sweep : kTbDefaultSweep;
    const int hb = k * std::max(1, n_inner);
    if (hb > kTbMaxHalo)
        return fail(SEG_ERR_INVALID_ARG, "sweep (%d) x n_inner (%d) must be <= %d", k, n_inner, kTbMaxHalo);
    *nwin = tb_geom(H, W, hb).nwin;
    return SEG_OK;
}

seg_status run_tiled(const IterParams& P, const seg_params* prm, const uint32_t* act, const float* f,
                     float* u, float* v, float* p1, float* p2, float* st, double* partials, int64_t npartials,
                     WsHeader* h, cudaStream_t s) {
    const int n_inner = std::max(1, prm->n_inner);
    const int k = prm->sweep > 0 ? prm->sweep : kTbDefaultSweep;
    int nwin = 0;
    SEG_TRY(tiled_geometry(P.H, P.W, prm->sweep, n_inner, &nwin));
    TbGeom G = tb_geom(P.H, P.W, k * n_inner);
    if (2 * (int64_t)G.nwin > npartials)
        return fail(SEG_ERR_WORKSPACE, "workspace holds %lld partial pairs, the tiled solve needs %d",
                    (long long)npartials, 2 * G.nwin);
    const int64_t plane = (int64_t)P.H * P.ld;
    // per-window lists after the planes (the state was sized for the most windows)
    char* lb = reinterpret_cast<char*>(st) + align_up(6 * sizeof(float) * (size_t)plane, 256);
    uint16_t* lists = reinterpret_cast<uint16_t*>(lb);
    int2* counts = reinterpret_cast<int2*>(lb + align_up((size_t)G.nwin * kTbPix * 2, 256));
    int* active = reinterpret_cast<int*>(reinterpret_cast<char*>(counts) + align_up((size_t)G.nwin * 8, 256));
    int* nact = active + G.nwin;
    TbMaps M;
    for (int b = 0; b < 2; ++b) {
        SEG_TRY(tb_map(&M.p1[b], st + b * plane, P.H, P.W, P.ld));
        SEG_TRY(tb_map(&M.p2[b], st + (2 + b) * plane, P.H, P.W, P.ld));
        SEG_TRY(tb_map(&M.v[b], st + (4 + b) * plane, P.H, P.W, P.ld));
    }
    SEG_TRY(tb_map(&M.f, f, P.H, P.W, P.ld));
    k_tb_lists<<<(G.nwin + 3) / 4, 128, 0, s>>>(P, G, act, lists, counts);
    SEG_LAUNCHED("k_tb_lists");
    k_tb_active<<<1, 1024, 0, s>>>(G, counts, active, nact);
    SEG_LAUNCHED("k_tb_active");
    const int nbuf = tb_buffers();
    const void* kern = nbuf == 2 ? (const void*)k_solve_tiled<2> : (const void*)k_solve_tiled<1>;
    const int threads = tb_threads(nbuf);
    const size_t smem = tb_smem(nbuf);
    SEG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm <= 0) return fail(SEG_ERR_CUDA, "k_solve_tiled cannot be resident");
    const int grid = (int)std::min<int64_t>((int64_t)per_sm * sm_count(), G.nwin);
    IterParams Pk = P;
    int iters = prm->iters, check_every = std::max(1, prm->check_every);
    int kmax = k;
    int ni = n_inner;
    double tol = prm->tol;
    const uint16_t* lc = lists;
    const int2* cc = counts;
    const int* ac = active;
    const int* nc = nact;
    void* args[] = {&Pk, &G, &iters, &ni, &kmax, &check_every, &tol, &M, (void*)&lc, (void*)&cc, (void*)&ac,
                    (void*)&nc, &st, &u, &partials, &h};
    if (iters > 0) {
        SEG_TRY_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(threads), args, smem, s));
        count_launch();
    }
    const int64_t n = (int64_t)P.H * P.W;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
    k_final_tiled<<<blocks, 256, 0, s>>>(P, h, st, v, p1, p2);
    SEG_LAUNCHED("k_final_tiled");
    return SEG_OK;
}

}  // namespace seg
