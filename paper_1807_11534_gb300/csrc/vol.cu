// vol.cu -- Section 3's restricted dual iteration on 3-D volumes (the
// Conclusion names 3-D problems as a case where restricting the domain pays
// off most).
//
// A volume is [D][H][ld] float32 (slice z, row i, column j; the rows of all
// slices stacked), so the fitting term and the partition of
// seg_make_fitting / seg_build_domain apply to it unchanged as a (D*H) x W
// image: RD bits, f<0 bits, the compact starts of every mask word and the
// RD voxel list in tile-major order.  The iteration is the 2-D one with a
// third component of p and the slice neighbours (grad: forward differences
// along rows, columns and slices, 0 on the last one; div = -grad^T):
//   w = div p - v/theta,  p <- (p + tau grad w) / (1 + tau |grad w|)   on RD
//   u = v - theta div p,  v = clip(u - theta lambda f, 0, 1)           on RD
//
// The state is compact: one element per RD voxel in list order (p in two
// ping-pong buffers, w, v, theta lambda f, u of the iteration before a
// stopping test, the voxel's dense offset) plus a neighbour table of 12
// entries per voxel (compact index, or a code for fixed background /
// foreground / outside): the six axis neighbours, and for each forward
// neighbour y the two backward neighbours of y other than the voxel itself,
// which w at a fixed y needs (p(y) = 0 and v(y) = H(-f(y)), so w(y) is minus
// the sum of those neighbours' previous p components, minus v(y)/theta).
// Consecutive threads take consecutive voxels, so the voxel's own state is
// read and written in full sectors however scattered RD is in the volume.
// One persistent cooperative launch runs every iteration: two grid barriers
// per iteration, the Section 4 test every check_every iterations.
#include <algorithm>
#include <cmath>

#include "iterate.cuh"
#include "seg_internal.cuh"

namespace seg {

struct VolGeom {
    int D, H, W, ld, nw;
    int R;              // rows of the stacked volume, D * H
    float theta, inv_theta, tau, theta_lambda;
};

// neighbour slots: the six axis neighbours, then for y = x + e1, x + e2,
// x + e3 (in that order) the two backward neighbours of y other than x
enum {
    VN_UP = 0, VN_DOWN, VN_LEFT, VN_RIGHT, VN_BACK, VN_FRONT,
    VN_DOWN_LEFT, VN_DOWN_BACK,     // (x + e1) - e2, (x + e1) - e3
    VN_RIGHT_UP, VN_RIGHT_BACK,     // (x + e2) - e1, (x + e2) - e3
    VN_FRONT_UP, VN_FRONT_LEFT,     // (x + e3) - e1, (x + e3) - e2
    VN_COUNT
};
constexpr int kVBg = -1;    // fixed background: p = 0, v = 0
constexpr int kVFg = -2;    // fixed foreground: p = 0, v = 1
constexpr int kVOut = -3;   // outside the volume

struct VolState {           // compact arrays, `stride` elements each
    float* p[2][3];         // buffer b, component k (along rows, columns, slices)
    float *w, *v, *f, *up;  // w = div p - v/theta; f premultiplied by theta lambda
    int32_t* off;           // dense offset (z*H + i)*ld + j of each RD voxel
    int32_t* nb;            // [VN_COUNT][stride]
    int64_t cap, stride;
};

// one p buffer (selected without indexing the state's array by a runtime
// value, which would put it in local memory)
struct VolBuf {
    float *p1, *p2, *p3;
};

__device__ __forceinline__ VolBuf vol_buf(const VolState& S, int b) {
    return b ? VolBuf{S.p[1][0], S.p[1][1], S.p[1][2]} : VolBuf{S.p[0][0], S.p[0][1], S.p[0][2]};
}

constexpr int kVolThreads = 512;   // threads per block
constexpr int kVolMinBlocks = 2;   // resident blocks per SM of the staged solve (64 registers)
constexpr int kVolUnroll = 2;      // voxels per thread whose loads are in flight together (staged solve)
constexpr int kVolArrays = 11 + VN_COUNT;
constexpr int64_t kVolSlack = 256;

inline int64_t vol_stride(int64_t capacity) {
    return (std::max<int64_t>(capacity, 1) + kVolSlack + 63) / 64 * 64;
}

__device__ __forceinline__ uint32_t plane_bit(const uint32_t* __restrict__ plane, int nw, int64_t r,
                                              int j) {
    return (__ldg(plane + r * nw + (j >> 5)) >> (j & 31)) & 1u;
}

// Compact index of voxel (z, i, j) if it is in RD, else its code.
__device__ __forceinline__ int vol_code(const VolGeom& G, const uint32_t* __restrict__ act,
                                        const uint32_t* __restrict__ fgm, const int32_t* __restrict__ wstart,
                                        int z, int i, int j) {
    if (z < 0 || z >= G.D || i < 0 || i >= G.H || j < 0 || j >= G.W) return kVOut;
    const int64_t wo = ((int64_t)z * G.H + i) * G.nw + (j >> 5);
    const uint32_t a = __ldg(act + wo);
    const int b = j & 31;
    if ((a >> b) & 1u) return __ldg(wstart + wo) + __popc(a & lanemask_lt(b));
    return ((__ldg(fgm + wo) >> b) & 1u) ? kVFg : kVBg;
}

// Fixed voxels of the dense outputs (u = v = H(-f), p = 0); RD voxels are
// written by the solve and the scatter.
__global__ void k_vol_fixed(VolGeom G, const uint32_t* __restrict__ act, const uint32_t* __restrict__ fgm,
                            float* u, float* v, float* p1, float* p2, float* p3) {
    const int64_t n = (int64_t)G.R * G.W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(x / G.W), j = (int)(x - (int64_t)r * G.W);
        if (plane_bit(act, G.nw, r, j)) continue;
        const int64_t o = (int64_t)r * G.ld + j;
        const float hh = plane_bit(fgm, G.nw, r, j) ? 1.f : 0.f;
        u[o] = hh;
        v[o] = hh;
        p1[o] = 0.f;
        p2[o] = 0.f;
        p3[o] = 0.f;
    }
}

// Compact state and neighbour table of every RD voxel (list entry k is
// compact index k): start iterate u0 = H(-f) and v0 = clip(u0 - theta lambda
// f) (or the caller's u, v, p, with the p components that never enter div
// -- last row / column / slice -- held at 0), w = -v/theta for a cold start.
__global__ void k_vol_setup(VolGeom G, const int32_t* __restrict__ vox, const int32_t* __restrict__ counts,
                            const uint32_t* __restrict__ act, const uint32_t* __restrict__ fgm,
                            const int32_t* __restrict__ wstart, const float* __restrict__ f, int warm,
                            const float* u, const float* v, const float* p1in, const float* p2in,
                            const float* p3in, VolState S, WsHeader* h) {
    const int n = counts[1];
    if (n > S.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            record_status(h, SEG_ERR_CAPACITY);
            h->done = 1;
            h->iters_done = 0;
        }
        return;
    }
    const int64_t st = S.stride;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int id = __ldg(vox + k);   // r * W + j
        const int r = id / G.W, j = id - r * G.W;
        const int z = r / G.H, i = r - z * G.H;
        const int64_t o = (int64_t)r * G.ld + j;
        int32_t* nb = S.nb + k;
        nb[VN_UP * st] = vol_code(G, act, fgm, wstart, z, i - 1, j);
        nb[VN_DOWN * st] = vol_code(G, act, fgm, wstart, z, i + 1, j);
        nb[VN_LEFT * st] = vol_code(G, act, fgm, wstart, z, i, j - 1);
        nb[VN_RIGHT * st] = vol_code(G, act, fgm, wstart, z, i, j + 1);
        nb[VN_BACK * st] = vol_code(G, act, fgm, wstart, z - 1, i, j);
        nb[VN_FRONT * st] = vol_code(G, act, fgm, wstart, z + 1, i, j);
        nb[VN_DOWN_LEFT * st] = vol_code(G, act, fgm, wstart, z, i + 1, j - 1);
        nb[VN_DOWN_BACK * st] = vol_code(G, act, fgm, wstart, z - 1, i + 1, j);
        nb[VN_RIGHT_UP * st] = vol_code(G, act, fgm, wstart, z, i - 1, j + 1);
        nb[VN_RIGHT_BACK * st] = vol_code(G, act, fgm, wstart, z - 1, i, j + 1);
        nb[VN_FRONT_UP * st] = vol_code(G, act, fgm, wstart, z + 1, i - 1, j);
        nb[VN_FRONT_LEFT * st] = vol_code(G, act, fgm, wstart, z + 1, i, j - 1);
        S.off[k] = (int32_t)o;
        const float fv = f[o];
        S.f[k] = G.theta_lambda * fv;
        const float hh = plane_bit(fgm, G.nw, r, j) ? 1.f : 0.f;
        float uu = hh, vv, q1 = 0.f, q2 = 0.f, q3 = 0.f;
        if (warm) {
            uu = u[o];
            vv = v[o];
            q1 = i < G.H - 1 ? p1in[o] : 0.f;
            q2 = j < G.W - 1 ? p2in[o] : 0.f;
            q3 = z < G.D - 1 ? p3in[o] : 0.f;
        } else {
            vv = clamp01(uu - G.theta_lambda * fv);
        }
        S.p[0][0][k] = q1;
        S.p[0][1][k] = q2;
        S.p[0][2][k] = q3;
        S.v[k] = vv;
        S.up[k] = uu;
        S.w[k] = -vv * G.inv_theta;   // div p = 0 (cold start); k_vol_warm_w otherwise
    }
}

// p component at a table entry (0 at fixed and outside voxels)
__device__ __forceinline__ float vol_pat(const float* P, int c) { return c >= 0 ? P[c] : 0.f; }

__device__ __forceinline__ float vol_div(const VolState& S, const VolBuf& B, int k) {
    const int64_t st = S.stride;
    const int nu = __ldg(S.nb + VN_UP * st + k), nl = __ldg(S.nb + VN_LEFT * st + k);
    const int nbk = __ldg(S.nb + VN_BACK * st + k);
    return (B.p1[k] - vol_pat(B.p1, nu)) + (B.p2[k] - vol_pat(B.p2, nl)) + (B.p3[k] - vol_pat(B.p3, nbk));
}

// w = div p - v/theta of a warm start (after the whole table exists).
__global__ void k_vol_warm_w(const int32_t* __restrict__ counts, VolGeom G, VolState S) {
    const int n = counts[1];
    if (n > S.cap) return;
    const VolBuf B = vol_buf(S, 0);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        S.w[k] = vol_div(S, B, k) - S.v[k] * G.inv_theta;
}

// The two phases take U voxels of a thread at a time and issue every load of
// all U before the first store, stage by stage (the table entries, then what
// they name): the stores of a phase go to other arrays than its loads (p' to
// the other buffers; v and w of the voxel itself), so the U voxels' chains of
// dependent loads overlap instead of queueing behind each other's stores.

// Dual (fixed-point) step at compact voxels k[0..U) from the previous p (Bi)
// into Bo.
template <int U>
__device__ __forceinline__ void vol_dual(const VolGeom& G, const VolState& S, const VolBuf& Bi, const VolBuf& Bo,
                                         const int (&k)[U]) {
    const int64_t st = S.stride;
    const float* __restrict__ W = S.w;
    const float* __restrict__ I1 = Bi.p1;
    const float* __restrict__ I2 = Bi.p2;
    const float* __restrict__ I3 = Bi.p3;
    int nd[U], nr[U], nf[U];
    float w0[U], p1[U], p2[U], p3[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int* nb = S.nb + k[u];
        nd[u] = __ldg(nb + VN_DOWN * st);
        nr[u] = __ldg(nb + VN_RIGHT * st);
        nf[u] = __ldg(nb + VN_FRONT * st);
        w0[u] = W[k[u]];
        p1[u] = I1[k[u]];
        p2[u] = I2[k[u]];
        p3[u] = I3[k[u]];
    }
    // per forward neighbour y: w(y) when y is in RD; when y is fixed, the
    // table entries of its other backward neighbours, then their p
    // components (0 where those are not in RD)
    float xd[U], xr[U], xf[U];
    int s1[U][3], s2[U][3];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int* nb = S.nb + k[u];
        const bool fd = nd[u] < 0 && nd[u] != kVOut, fr = nr[u] < 0 && nr[u] != kVOut,
                   ff = nf[u] < 0 && nf[u] != kVOut;
        xd[u] = nd[u] >= 0 ? W[nd[u]] : 0.f;
        xr[u] = nr[u] >= 0 ? W[nr[u]] : 0.f;
        xf[u] = nf[u] >= 0 ? W[nf[u]] : 0.f;
        s1[u][0] = fd ? __ldg(nb + VN_DOWN_LEFT * st) : -1;
        s2[u][0] = fd ? __ldg(nb + VN_DOWN_BACK * st) : -1;
        s1[u][1] = fr ? __ldg(nb + VN_RIGHT_UP * st) : -1;
        s2[u][1] = fr ? __ldg(nb + VN_RIGHT_BACK * st) : -1;
        s1[u][2] = ff ? __ldg(nb + VN_FRONT_UP * st) : -1;
        s2[u][2] = ff ? __ldg(nb + VN_FRONT_LEFT * st) : -1;
    }
    float a1[U][3], a2[U][3];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        a1[u][0] = vol_pat(I2, s1[u][0]);
        a2[u][0] = vol_pat(I3, s2[u][0]);
        a1[u][1] = vol_pat(I1, s1[u][1]);
        a2[u][1] = vol_pat(I3, s2[u][1]);
        a1[u][2] = vol_pat(I1, s1[u][2]);
        a2[u][2] = vol_pat(I2, s2[u][2]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        float g1 = 0.f, g2 = 0.f, g3 = 0.f;
        if (nd[u] >= 0) {
            g1 = xd[u] - w0[u];
        } else if (nd[u] != kVOut) {   // w at a fixed y = x + e1: its p1 backward neighbour is x itself
            const float sm = p1[u] + a1[u][0] + a2[u][0];
            g1 = (-sm - (nd[u] == kVFg ? G.inv_theta : 0.f)) - w0[u];
        }
        if (nr[u] >= 0) {
            g2 = xr[u] - w0[u];
        } else if (nr[u] != kVOut) {
            const float sm = a1[u][1] + p2[u] + a2[u][1];
            g2 = (-sm - (nr[u] == kVFg ? G.inv_theta : 0.f)) - w0[u];
        }
        if (nf[u] >= 0) {
            g3 = xf[u] - w0[u];
        } else if (nf[u] != kVOut) {
            const float sm = a1[u][2] + a2[u][2] + p3[u];
            g3 = (-sm - (nf[u] == kVFg ? G.inv_theta : 0.f)) - w0[u];
        }
        const float s2n = fmaf(g1, g1, fmaf(g2, g2, g3 * g3));
        const float nrm = s2n > 0.f ? s2n * rsqrtf(s2n) : 0.f;
        const float rc = __fdividef(1.0f, fmaf(G.tau, nrm, 1.0f));
        Bo.p1[k[u]] = fmaf(G.tau, g1, p1[u]) * rc;
        Bo.p2[k[u]] = fmaf(G.tau, g2, p2[u]) * rc;
        Bo.p3[k[u]] = fmaf(G.tau, g3, p3[u]) * rc;
    }
}

// Primal step at compact voxels k[0..U) with the new p (Bo): v in place, w
// for the next dual step, u to the dense output on a stopping-test iteration.
template <int U>
__device__ __forceinline__ void vol_primal(const VolGeom& G, float* U_out, const VolState& S, const VolBuf& Bo,
                                           const int (&k)[U], bool check, bool write_u, bool write_prev,
                                           float& du2, float& dv2) {
    const int64_t st = S.stride;
    const float* __restrict__ Q1 = Bo.p1;
    const float* __restrict__ Q2 = Bo.p2;
    const float* __restrict__ Q3 = Bo.p3;
    int nu[U], nl[U], nbk[U];
    float q1[U], q2[U], q3[U], vv[U], ff[U], xu[U], xl[U], xb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        nu[u] = __ldg(S.nb + VN_UP * st + k[u]);
        nl[u] = __ldg(S.nb + VN_LEFT * st + k[u]);
        nbk[u] = __ldg(S.nb + VN_BACK * st + k[u]);
        q1[u] = Q1[k[u]];
        q2[u] = Q2[k[u]];
        q3[u] = Q3[k[u]];
        vv[u] = S.v[k[u]];
        ff[u] = __ldg(S.f + k[u]);   // f premultiplied by theta lambda
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        xu[u] = vol_pat(Q1, nu[u]);
        xl[u] = vol_pat(Q2, nl[u]);
        xb[u] = vol_pat(Q3, nbk[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const float div = (q1[u] - xu[u]) + (q2[u] - xl[u]) + (q3[u] - xb[u]);
        const float un = fmaf(-G.theta, div, vv[u]);
        const float vn = clamp01(un - ff[u]);
        S.v[k[u]] = vn;
        S.w[k[u]] = div - vn * G.inv_theta;
        if (check) {
            const float da = un - S.up[k[u]], db = vn - vv[u];
            du2 = fmaf(da, da, du2);
            dv2 = fmaf(db, db, dv2);
        }
        if (write_prev) S.up[k[u]] = un;
        if (write_u) U_out[__ldg(S.off + k[u])] = un;
    }
}

// One voxel at a time (the solve of dense volumes, where every neighbour is
// in RD and more warps hide the two-load chain better than staging).
// Dual (fixed-point) step at compact voxel k from the previous p (Bi) into Bo.
__device__ __forceinline__ void vol_dual1(const VolGeom& G, const VolState& S, const VolBuf& Bi, const VolBuf& Bo,
                                          int k) {
    const int64_t st = S.stride;
    const int* nb = S.nb + k;
    const int nd = __ldg(nb + VN_DOWN * st), nr = __ldg(nb + VN_RIGHT * st), nf = __ldg(nb + VN_FRONT * st);
    const float w0 = S.w[k];
    const float p1 = Bi.p1[k], p2 = Bi.p2[k], p3 = Bi.p3[k];
    float g1 = 0.f, g2 = 0.f, g3 = 0.f;
    if (nd >= 0) {
        g1 = S.w[nd] - w0;
    } else if (nd != kVOut) {   // w at a fixed y = x + e1: its p1 backward neighbour is x itself
        const float s = p1 + vol_pat(Bi.p2, __ldg(nb + VN_DOWN_LEFT * st)) +
                        vol_pat(Bi.p3, __ldg(nb + VN_DOWN_BACK * st));
        g1 = (-s - (nd == kVFg ? G.inv_theta : 0.f)) - w0;
    }
    if (nr >= 0) {
        g2 = S.w[nr] - w0;
    } else if (nr != kVOut) {
        const float s = vol_pat(Bi.p1, __ldg(nb + VN_RIGHT_UP * st)) + p2 +
                        vol_pat(Bi.p3, __ldg(nb + VN_RIGHT_BACK * st));
        g2 = (-s - (nr == kVFg ? G.inv_theta : 0.f)) - w0;
    }
    if (nf >= 0) {
        g3 = S.w[nf] - w0;
    } else if (nf != kVOut) {
        const float s = vol_pat(Bi.p1, __ldg(nb + VN_FRONT_UP * st)) +
                        vol_pat(Bi.p2, __ldg(nb + VN_FRONT_LEFT * st)) + p3;
        g3 = (-s - (nf == kVFg ? G.inv_theta : 0.f)) - w0;
    }
    const float s = fmaf(g1, g1, fmaf(g2, g2, g3 * g3));
    const float nrm = s > 0.f ? s * rsqrtf(s) : 0.f;
    const float rc = __fdividef(1.0f, fmaf(G.tau, nrm, 1.0f));
    Bo.p1[k] = fmaf(G.tau, g1, p1) * rc;
    Bo.p2[k] = fmaf(G.tau, g2, p2) * rc;
    Bo.p3[k] = fmaf(G.tau, g3, p3) * rc;
}

// Primal step at compact voxel k with the new p (Bo): v in place, w for the
// next dual step, u to the dense output on a stopping-test iteration.
__device__ __forceinline__ void vol_primal1(const VolGeom& G, float* U, const VolState& S, const VolBuf& Bo, int k,
                                            bool check, bool write_u, bool write_prev, float& du2, float& dv2) {
    const float div = vol_div(S, Bo, k);
    const float vv = S.v[k];
    const float un = fmaf(-G.theta, div, vv);
    const float vn = clamp01(un - __ldg(S.f + k));   // f premultiplied by theta lambda
    S.v[k] = vn;
    S.w[k] = div - vn * G.inv_theta;
    if (check) {
        const float da = un - S.up[k], db = vn - vv;
        du2 = fmaf(da, da, du2);
        dv2 = fmaf(db, db, dv2);
    }
    if (write_prev) S.up[k] = un;
    if (write_u) U[__ldg(S.off + k)] = un;
}

// STAGED: kVolUnroll voxels a thread, staged loads, kVolMinBlocks blocks per
// SM, for RD counts up to staged_upto (restricted volumes); else one voxel
// at a time at four blocks per SM (dense volumes).  Both are launched (the
// RD count is on the device); the one that does not apply returns at once.
template <bool STAGED>
__global__ void __launch_bounds__(kVolThreads, STAGED ? kVolMinBlocks : 4)
k_solve_vol(VolGeom G, int iters, int check_every, double tol, const int32_t* __restrict__ counts, float* U,
            VolState S, double* partials, WsHeader* h, long long staged_upto) {
    __shared__ double s_red[66];   // block_sum2f (as floats), stop flag
    if (*(volatile int*)&h->done) return;
    const unsigned nblocks = gridDim.x;
    const int n = counts[1];
    if (STAGED ? n > staged_upto : n <= staged_upto) return;   // the other launch's
    const int tid = threadIdx.x;
    const int k0 = (int)blockIdx.x * kVolThreads + tid, stride = (int)nblocks * kVolThreads;
    const int C = check_every;
    unsigned gen = 0;
    int chk = 0;
    // op(voxels[U]) over this thread's voxels k0, k0 + stride, ..., U =
    // kVolUnroll at a time, then the rest one by one
    constexpr int UN = STAGED ? kVolUnroll : 1;
    auto each = [&](auto&& op) {
        int k = k0;
        for (; k + (UN - 1) * stride < n; k += UN * stride) {
            int b[UN];
#pragma unroll
            for (int u = 0; u < UN; ++u) b[u] = k + u * stride;
            op(b);
        }
        for (; k < n; k += stride) {
            const int b[1] = {k};
            op(b);
        }
    };
    for (int l = 1; l <= iters; ++l) {
        const bool check = (l % C == 0) || l == iters;
        const bool write_prev = l < iters && ((l + 1) % C == 0 || l + 1 == iters);
        const VolBuf Bi = vol_buf(S, (l - 1) & 1), Bo = vol_buf(S, l & 1);
        if constexpr (STAGED)
            each([&](const auto& ks) { vol_dual(G, S, Bi, Bo, ks); });
        else
            for (int k = k0; k < n; k += stride) vol_dual1(G, S, Bi, Bo, k);
        if (!grid_sync(h, nblocks, gen)) return;
        float du2 = 0.f, dv2 = 0.f;
        if constexpr (STAGED)
            each([&](const auto& ks) { vol_primal(G, U, S, Bo, ks, check, check, write_prev, du2, dv2); });
        else
            for (int k = k0; k < n; k += stride) vol_primal1(G, U, S, Bo, k, check, check, write_prev, du2, dv2);
        double* part = partials + 2 * (int64_t)nblocks * (chk & 1);
        if (check) {
            float x = du2, y = dv2;
            block_sum2f<kVolThreads>(x, y, reinterpret_cast<float*>(s_red));
            if (tid == 0) {
                part[2 * blockIdx.x] = x;
                part[2 * blockIdx.x + 1] = y;
            }
        }
        if (!grid_sync(h, nblocks, gen)) return;
        if (check) {
            // Section 4 test: every block sums the partials in the same order
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

// v and p of the final iterate (p from the buffer of its parity) to the dense
// outputs; u too when no iteration ran (iterations write it themselves).
__global__ void k_vol_scatter(const int32_t* __restrict__ counts, const WsHeader* __restrict__ h, int iters,
                              VolState S, float* u, float* v, float* p1, float* p2, float* p3) {
    const int n = counts[1];
    if (n > S.cap) return;
    const int l = h->done ? h->iters_done : iters;
    const VolBuf B = vol_buf(S, l & 1);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int64_t o = S.off[k];
        v[o] = S.v[k];
        p1[o] = B.p1[k];
        p2[o] = B.p2[k];
        p3[o] = B.p3[k];
        if (l == 0) u[o] = S.up[k];
    }
}

}  // namespace seg

using namespace seg;

extern "C" size_t seg_state_bytes3d(int64_t capacity) {
    return (size_t)kVolArrays * align_up(4 * (size_t)vol_stride(capacity), 256) + 256;
}

extern "C" seg_status seg_solve3d(const float* f, int D, int H, int W, int ld, const uint32_t* act,
                                  const uint32_t* fgm, const int32_t* wstart, const int32_t* voxels,
                                  const int32_t* counts, const seg_params* prm, float* u, float* v, float* p1,
                                  float* p2, float* p3, void* state, size_t state_bytes, double* stats, void* ws,
                                  size_t ws_bytes, void* stream) {
    clear_error();
    PhaseScope _scope("seg_solve3d", stream, ws);
    if (!prm) return fail(SEG_ERR_INVALID_ARG, "params must be non-NULL");
    if (!f || !act || !fgm || !wstart || !voxels || !counts || !u || !v || !p1 || !p2 || !p3 || !state || !stats)
        return fail(SEG_ERR_INVALID_ARG, "a required pointer is NULL");
    if (D <= 0 || H <= 0 || W <= 0 || ld < W || (int64_t)D * H * ld >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad volume size D=%d H=%d W=%d ld=%d (D*H*ld < 2^31)", D, H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    const int th = prm->tile_h;
    if (th != 4 && th != 8 && th != 16 && th != 32)
        return fail(SEG_ERR_INVALID_ARG, "tile_h=%d not in {4, 8, 16, 32}", th);
    if (prm->iters < 0 || prm->n_inner != 1 || prm->check_every < 1)
        return fail(SEG_ERR_INVALID_ARG, "iters >= 0, n_inner = 1 and check_every >= 1 required");
    if (!(prm->theta > 0) || !(prm->tau > 0) || !std::isfinite(prm->lambda) || std::isnan(prm->tol))
        return fail(SEG_ERR_INVALID_ARG, "theta, tau must be > 0 and lambda finite");
    if (prm->storage != SEG_STORE_F32) return fail(SEG_ERR_INVALID_ARG, "volumes use float32 storage");
    if (reinterpret_cast<uintptr_t>(state) % 256) return fail(SEG_ERR_ALIGN, "state not 256-byte aligned");
    const int R = D * H;
    WsLayout L = ws_layout(R, W, th);
    SEG_TRY(check_ws(ws, ws_bytes, L));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    double* partials = ws_at<double>(ws, L.partials);

    VolGeom G{};
    G.D = D; G.H = H; G.W = W; G.ld = ld; G.nw = ld / 32; G.R = R;
    G.theta = (float)prm->theta;
    G.inv_theta = (float)(1.0 / prm->theta);
    G.tau = (float)prm->tau;
    G.theta_lambda = (float)(prm->theta * prm->lambda);
    // the largest array length (a multiple of 64) whose arrays fit in state_bytes
    VolState S{};
    const size_t per_array = state_bytes > 256 ? (state_bytes - 256) / kVolArrays / 256 * 256 : 0;
    S.stride = (int64_t)(per_array / 4) / 64 * 64;
    S.cap = std::max<int64_t>(0, S.stride - kVolSlack);
    char* sb = static_cast<char*>(state);
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 3; ++k) S.p[b][k] = reinterpret_cast<float*>(sb + (size_t)(3 * b + k) * per_array);
    S.w = reinterpret_cast<float*>(sb + 6 * per_array);
    S.v = reinterpret_cast<float*>(sb + 7 * per_array);
    S.f = reinterpret_cast<float*>(sb + 8 * per_array);
    S.up = reinterpret_cast<float*>(sb + 9 * per_array);
    S.off = reinterpret_cast<int32_t*>(sb + 10 * per_array);
    S.nb = reinterpret_cast<int32_t*>(sb + 11 * per_array);   // VN_COUNT arrays of stride

    SEG_TRY(launch_solve_begin(h, s));
    const int64_t nvox = (int64_t)R * W;
    const int eblocks = (int)std::min<int64_t>((nvox + 255) / 256, (int64_t)sm_count() * 16);
    k_vol_setup<<<eblocks, 256, 0, s>>>(G, voxels, counts, act, fgm, wstart, f, prm->warm_start, u, v, p1, p2,
                                        p3, S, h);
    SEG_LAUNCHED("k_vol_setup");
    if (prm->warm_start) {
        k_vol_warm_w<<<eblocks, 256, 0, s>>>(counts, G, S);
        SEG_LAUNCHED("k_vol_warm_w");
    }
    k_vol_fixed<<<eblocks, 256, 0, s>>>(G, act, fgm, u, v, p1, p2, p3);
    SEG_LAUNCHED("k_vol_fixed");
    auto grid_of = [&](const void* k, int& grid) -> seg_status {
        int per_sm = 0;
        SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kVolThreads, 0));
        if (per_sm <= 0) return fail(SEG_ERR_CUDA, "k_solve_vol cannot be resident");
        grid = (int)std::min<int64_t>((int64_t)per_sm * sm_count(), L.npartials / 2);
        grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, (std::max<int64_t>(S.cap, 1) + kVolThreads - 1) /
                                                                      kVolThreads));
        return SEG_OK;
    };
    const void* ks = (const void*)k_solve_vol<true>;
    const void* kd = (const void*)k_solve_vol<false>;
    int grid_s = 1, grid_d = 1;
    SEG_TRY(grid_of(ks, grid_s));
    SEG_TRY(grid_of(kd, grid_d));
    // the staged solve for RD up to half the volume, the plain one above
    long long staged_upto = nvox / 2;
    int iters = prm->iters, ce = test_interval(prm->tol, prm->check_every, prm->iters);
    double tol = prm->tol;
    void* args[] = {&G, &iters, &ce, &tol, (void*)&counts, &u, &S, &partials, &h, &staged_upto};
    if (iters > 0) {
        SEG_TRY_CUDA(cudaLaunchCooperativeKernel(ks, dim3(grid_s), dim3(kVolThreads), args, 0, s));
        count_launch();
        if (debug_mode()) SEG_TRY(after_launch("persistent solve (staged)"));
        if (std::min<int64_t>(S.cap, nvox) > staged_upto) {
            SEG_TRY_CUDA(cudaLaunchCooperativeKernel(kd, dim3(grid_d), dim3(kVolThreads), args, 0, s));
            count_launch();
            if (debug_mode()) SEG_TRY(after_launch("persistent solve (plain)"));
        }
    }
    k_vol_scatter<<<eblocks, 256, 0, s>>>(counts, h, prm->iters, S, u, v, p1, p2, p3);
    SEG_LAUNCHED("k_vol_scatter");
    SEG_TRY(launch_solve_end(h, counts, prm->iters, stats, s));
    return SEG_OK;
}
