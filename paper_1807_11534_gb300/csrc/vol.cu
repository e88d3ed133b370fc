// vol.cu -- Section 3's restricted dual iteration on 3-D volumes (the
// Conclusion names 3-D problems as a case where restricting the domain pays
// off most).
//
// A volume is [D][H][ld] float32 (slice z, row i, column j; the rows of all
// slices stacked), so the fitting term and the partition of
// seg_make_fitting / seg_build_domain apply to it unchanged as a (D*H) x W
// image: RD bits, f<0 bits and the list of 32-column x tile_h-row tiles that
// hold an RD voxel.  The iteration is the 2-D one with a third component of
// p and the slice neighbours (grad: forward differences along rows, columns
// and slices, 0 on the last one; div = -grad^T):
//   w = div p - v/theta,  p <- (p + tau grad w) / (1 + tau |grad w|)   on RD
//   u = v - theta div p,  v = clip(u - theta lambda f, 0, 1)           on RD
// The state is dense ([D][H][ld] planes, p = 0 outside RD), ping-pong for p
// so that w at a fixed neighbour y (p(y) = 0, v(y) = H(-f(y))) can be formed
// from the previous p of y's backward neighbours.  One persistent
// cooperative launch runs every iteration over the RD voxel list of
// seg_build_domain (linear ids in tile-major order, so consecutive threads
// take neighbouring voxels and no lane idles on a fixed voxel), two grid
// barriers per iteration, the Section 4 test every check_every iterations.
#include <algorithm>
#include <cmath>

#include "iterate.cuh"
#include "seg_internal.cuh"

namespace seg {

struct VolGeom {
    int D, H, W, ld, nw, ntx, th;
    int R;              // rows of the stacked volume, D * H
    int64_t slice;      // H * ld
    float theta, inv_theta, tau, theta_lambda;
};

struct VolState {
    float* p[2][3];     // buffer b, component k (along rows, columns, slices)
    float* w;           // div p - v/theta of the current iterate (RD voxels)
    float* up;          // u of the iteration before a stopping test
    int32_t* off;       // per RD voxel (list order): its offset (z*H + i)*ld + j
    uint16_t* flg;      // per RD voxel: kVf* bits below
};

// Per-voxel flags, computed once per solve: which backward / forward
// neighbours exist, and the state of the three forward neighbours (2 bits
// each: RD, fixed background, fixed foreground).
enum : uint16_t {
    kVfUp = 1, kVfDown = 2, kVfLeft = 4, kVfRight = 8, kVfBack = 16, kVfFront = 32,
    kVfShiftDown = 6, kVfShiftRight = 8, kVfShiftFront = 10   // 2-bit neighbour codes
};
enum { kVnRd = 0, kVnBg = 1, kVnFg = 2 };

// one p buffer (selected without indexing the state's array by a runtime
// value, which would put it in local memory)
struct VolBuf {
    float *p1, *p2, *p3;
};

__device__ __forceinline__ VolBuf vol_buf(const VolState& S, int b) {
    return b ? VolBuf{S.p[1][0], S.p[1][1], S.p[1][2]} : VolBuf{S.p[0][0], S.p[0][1], S.p[0][2]};
}

constexpr int kVolThreads = 1024;   // one block per SM
constexpr int kVolPlanes = 10;      // p[2][3], w, up, off, flg

__device__ __forceinline__ uint32_t plane_bit(const uint32_t* __restrict__ plane, int nw, int64_t r,
                                              int j) {
    return (__ldg(plane + r * nw + (j >> 5)) >> (j & 31)) & 1u;
}

// Start iterate: u0 = H(-f) (or the caller's u) and v0 = clip(u0 - theta
// lambda f) on RD, the fixed values outside; p = 0 outside RD and on the
// components that never enter div (last row / column / slice).
__global__ void k_vol_init(VolGeom G, const uint32_t* __restrict__ act, const uint32_t* __restrict__ fgm,
                           const float* __restrict__ f, int warm, float* u, float* v,
                           const float* __restrict__ p1in, const float* __restrict__ p2in,
                           const float* __restrict__ p3in, VolState S) {
    const int64_t n = (int64_t)G.R * G.W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(x / G.W), j = (int)(x - (int64_t)r * G.W);
        const int z = r / G.H, i = r - z * G.H;
        const int64_t o = (int64_t)r * G.ld + j;
        const float hh = plane_bit(fgm, G.nw, r, j) ? 1.f : 0.f;
        float uu = hh, vv = hh, q1 = 0.f, q2 = 0.f, q3 = 0.f, ww = 0.f;
        if (plane_bit(act, G.nw, r, j)) {
            if (warm) {
                uu = u[o];
                vv = v[o];
                q1 = i < G.H - 1 ? p1in[o] : 0.f;
                q2 = j < G.W - 1 ? p2in[o] : 0.f;
                q3 = z < G.D - 1 ? p3in[o] : 0.f;
            } else {
                vv = clamp01(uu - G.theta_lambda * f[o]);
                ww = -vv * G.inv_theta;   // div p = 0
            }
        }
        u[o] = uu;
        v[o] = vv;
        S.p[0][0][o] = q1; S.p[0][1][o] = q2; S.p[0][2][o] = q3;
        S.p[1][0][o] = 0.f; S.p[1][1][o] = 0.f; S.p[1][2][o] = 0.f;
        S.w[o] = ww;
        S.up[o] = uu;
    }
}

__device__ __forceinline__ float vol_div(const VolGeom& G, const float* Q1, const float* Q2, const float* Q3,
                                         int64_t o, int z, int i, int j) {
    const float a = (i < G.H - 1 ? Q1[o] : 0.f) - (i > 0 ? Q1[o - G.ld] : 0.f);
    const float b = (j < G.W - 1 ? Q2[o] : 0.f) - (j > 0 ? Q2[o - 1] : 0.f);
    const float c = (z < G.D - 1 ? Q3[o] : 0.f) - (z > 0 ? Q3[o - G.slice] : 0.f);
    return a + b + c;
}

// w of a warm start (the caller's p): div p - v/theta on RD.
__global__ void k_vol_w(VolGeom G, const uint32_t* __restrict__ act, const float* __restrict__ v, VolState S) {
    const int64_t n = (int64_t)G.R * G.W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(x / G.W), j = (int)(x - (int64_t)r * G.W);
        if (!plane_bit(act, G.nw, r, j)) continue;
        const int z = r / G.H, i = r - z * G.H;
        const int64_t o = (int64_t)r * G.ld + j;
        S.w[o] = vol_div(G, S.p[0][0], S.p[0][1], S.p[0][2], o, z, i, j) - v[o] * G.inv_theta;
    }
}

// Offsets and flags of the RD voxels (one pass over the voxel list).
__global__ void k_vol_setup(VolGeom G, const int32_t* __restrict__ vox, const int32_t* __restrict__ counts,
                            const uint32_t* __restrict__ act, const uint32_t* __restrict__ fgm, VolState S) {
    const int n = counts[1];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int id = vox[k];   // r * W + j
        const int r = id / G.W, j = id - r * G.W;
        const int z = r / G.H, i = r - z * G.H;
        auto code = [&](int64_t rr, int jj) -> uint16_t {
            if (plane_bit(act, G.nw, rr, jj)) return kVnRd;
            return plane_bit(fgm, G.nw, rr, jj) ? kVnFg : kVnBg;
        };
        uint16_t fl = 0;
        if (i > 0) fl |= kVfUp;
        if (j > 0) fl |= kVfLeft;
        if (z > 0) fl |= kVfBack;
        if (i + 1 < G.H) fl |= kVfDown | (uint16_t)(code(r + 1, j) << kVfShiftDown);
        if (j + 1 < G.W) fl |= kVfRight | (uint16_t)(code(r, j + 1) << kVfShiftRight);
        if (z + 1 < G.D) fl |= kVfFront | (uint16_t)(code(r + G.H, j) << kVfShiftFront);
        S.off[k] = (int32_t)((int64_t)r * G.ld + j);
        S.flg[k] = fl;
    }
}

// w at a fixed voxel y: p(y) = 0, so div p(y) is minus the backward
// neighbours' components along the axes where y has one; v(y) = H(-f(y)).
// hu, hl, hb: whether y has a neighbour above / left / behind.
__device__ __forceinline__ float vol_wfixed(const VolGeom& G, const VolBuf& B, int64_t y, bool hu, bool hl,
                                            bool hb, unsigned code) {
    const float s = (hu ? B.p1[y - G.ld] : 0.f) + (hl ? B.p2[y - 1] : 0.f) + (hb ? B.p3[y - G.slice] : 0.f);
    return -s - (code == kVnFg ? G.inv_theta : 0.f);
}

// The voxels of a thread are taken kVolUnroll at a time: first every load of
// the group, then the arithmetic and the stores (loads ahead of the stores
// let the compiler keep them in flight together).  One voxel at a time with
// this order measured fastest (256^3 volume: 270 us per full-volume
// iteration at 1, 326 at 2, 517 at 4 with 512 threads).
constexpr int kVolUnroll = 1;

// Dual (fixed-point) step at RD voxels (list entries k0 + u * stride) from the
// previous p (Bi) into Bo.
__device__ __forceinline__ void vol_dual(const VolGeom& G, const VolState& S, const VolBuf& Bi, const VolBuf& Bo,
                                         int n, int k0, int stride) {
    int64_t o[kVolUnroll];
    unsigned fl[kVolUnroll];
    float w0[kVolUnroll], wy[kVolUnroll][3], pp[kVolUnroll][3];
#pragma unroll
    for (int u = 0; u < kVolUnroll; ++u) {
        const int k = k0 + u * stride;
        o[u] = k < n ? (int64_t)__ldg(S.off + k) : 0;
        fl[u] = k < n ? (unsigned)__ldg(S.flg + k) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kVolUnroll; ++u) {
        if (k0 + u * stride >= n) continue;
        const int64_t x = o[u];
        const unsigned f = fl[u];
        const bool hu = f & kVfUp, hl = f & kVfLeft, hb = f & kVfBack;
        w0[u] = S.w[x];
        pp[u][0] = Bi.p1[x];
        pp[u][1] = Bi.p2[x];
        pp[u][2] = Bi.p3[x];
        wy[u][0] = wy[u][1] = wy[u][2] = 0.f;
        if (f & kVfDown) {
            const unsigned c = (f >> kVfShiftDown) & 3u;
            wy[u][0] = c == kVnRd ? S.w[x + G.ld] : vol_wfixed(G, Bi, x + G.ld, true, hl, hb, c);
        }
        if (f & kVfRight) {
            const unsigned c = (f >> kVfShiftRight) & 3u;
            wy[u][1] = c == kVnRd ? S.w[x + 1] : vol_wfixed(G, Bi, x + 1, hu, true, hb, c);
        }
        if (f & kVfFront) {
            const unsigned c = (f >> kVfShiftFront) & 3u;
            wy[u][2] = c == kVnRd ? S.w[x + G.slice] : vol_wfixed(G, Bi, x + G.slice, hu, hl, true, c);
        }
    }
#pragma unroll
    for (int u = 0; u < kVolUnroll; ++u) {
        if (k0 + u * stride >= n) continue;
        const unsigned f = fl[u];
        const float g1 = (f & kVfDown) ? wy[u][0] - w0[u] : 0.f;
        const float g2 = (f & kVfRight) ? wy[u][1] - w0[u] : 0.f;
        const float g3 = (f & kVfFront) ? wy[u][2] - w0[u] : 0.f;
        const float s = fmaf(g1, g1, fmaf(g2, g2, g3 * g3));
        const float nrm = s > 0.f ? s * rsqrtf(s) : 0.f;
        const float rc = __fdividef(1.0f, fmaf(G.tau, nrm, 1.0f));
        Bo.p1[o[u]] = fmaf(G.tau, g1, pp[u][0]) * rc;
        Bo.p2[o[u]] = fmaf(G.tau, g2, pp[u][1]) * rc;
        Bo.p3[o[u]] = fmaf(G.tau, g3, pp[u][2]) * rc;
    }
}

// Primal step at RD voxels (list entries k0 + u * stride) with the new p
// (Bo): u, v in place, w for the next dual step, the stopping-test sums.
__device__ __forceinline__ void vol_primal(const VolGeom& G, const float* __restrict__ f, float* U, float* V,
                                           const VolState& S, const VolBuf& Bo, int n, int k0, int stride,
                                           bool check, bool write_u, bool write_prev, float& du2, float& dv2) {
    int64_t o[kVolUnroll];
    unsigned fl[kVolUnroll];
    float dv[kVolUnroll], vv[kVolUnroll], ff[kVolUnroll], uo[kVolUnroll];
#pragma unroll
    for (int u = 0; u < kVolUnroll; ++u) {
        const int k = k0 + u * stride;
        o[u] = k < n ? (int64_t)__ldg(S.off + k) : 0;
        fl[u] = k < n ? (unsigned)__ldg(S.flg + k) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kVolUnroll; ++u) {
        if (k0 + u * stride >= n) continue;
        const int64_t x = o[u];
        const unsigned b = fl[u];
        const float a1 = ((b & kVfDown) ? Bo.p1[x] : 0.f) - ((b & kVfUp) ? Bo.p1[x - G.ld] : 0.f);
        const float a2 = ((b & kVfRight) ? Bo.p2[x] : 0.f) - ((b & kVfLeft) ? Bo.p2[x - 1] : 0.f);
        const float a3 = ((b & kVfFront) ? Bo.p3[x] : 0.f) - ((b & kVfBack) ? Bo.p3[x - G.slice] : 0.f);
        dv[u] = a1 + a2 + a3;
        vv[u] = V[x];
        ff[u] = __ldg(f + x);
        uo[u] = check ? S.up[x] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kVolUnroll; ++u) {
        if (k0 + u * stride >= n) continue;
        const int64_t x = o[u];
        const float un = fmaf(-G.theta, dv[u], vv[u]);
        const float vn = clamp01(un - G.theta_lambda * ff[u]);
        V[x] = vn;
        S.w[x] = dv[u] - vn * G.inv_theta;
        if (check) {
            const float da = un - uo[u], db = vn - vv[u];
            du2 = fmaf(da, da, du2);
            dv2 = fmaf(db, db, dv2);
        }
        if (write_prev) S.up[x] = un;
        if (write_u) U[x] = un;
    }
}

template <typename Fn>
__device__ __forceinline__ void vol_each(int n, Fn fn) {
    const int stride = (int)gridDim.x * kVolThreads;
    for (int k0 = (int)blockIdx.x * kVolThreads + (int)threadIdx.x; k0 < n; k0 += kVolUnroll * stride)
        fn(k0, stride);
}

__global__ void __launch_bounds__(kVolThreads, 1)
k_solve_vol(VolGeom G, int iters, int check_every, double tol, const uint32_t* __restrict__ act,
            const uint32_t* __restrict__ fgm, const int32_t* __restrict__ vox,
            const int32_t* __restrict__ counts, const float* __restrict__ f, float* U, float* V, VolState S,
            double* partials, WsHeader* h) {
    __shared__ double s_red[66];   // block_sum2f (as floats), stop flag
    if (*(volatile int*)&h->done) return;
    const unsigned nblocks = gridDim.x;
    const int n = counts[1];
    const int tid = threadIdx.x;
    const int C = check_every;
    unsigned gen = 0;
    int chk = 0;
    for (int l = 1; l <= iters; ++l) {
        const bool check = (l % C == 0) || l == iters;
        const bool write_prev = l < iters && ((l + 1) % C == 0 || l + 1 == iters);
        const VolBuf Bi = vol_buf(S, (l - 1) & 1), Bo = vol_buf(S, l & 1);
        vol_each(n, [&](int k0, int stride) { vol_dual(G, S, Bi, Bo, n, k0, stride); });
        if (!grid_sync(h, nblocks, gen)) return;
        float du2 = 0.f, dv2 = 0.f;
        vol_each(n, [&](int k0, int stride) {
            vol_primal(G, f, U, V, S, Bo, n, k0, stride, check, check, write_prev, du2, dv2);
        });
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

// p of the final iterate (buffer of its parity) to the caller's planes.
__global__ void k_vol_final(VolGeom G, const WsHeader* __restrict__ h, int iters, VolState S, float* p1,
                            float* p2, float* p3) {
    const int l = h->done ? h->iters_done : iters;
    const VolBuf B = vol_buf(S, l & 1);
    const int64_t n = (int64_t)G.R * G.W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(x / G.W), j = (int)(x - (int64_t)r * G.W);
        const int64_t o = (int64_t)r * G.ld + j;
        p1[o] = B.p1[o];
        p2[o] = B.p2[o];
        p3[o] = B.p3[o];
    }
}

}  // namespace seg

using namespace seg;

extern "C" size_t seg_state_bytes3d(int D, int H, int ld) {
    const size_t plane = (size_t)std::max(D, 0) * (size_t)std::max(H, 0) * (size_t)std::max(ld, 0);
    return kVolPlanes * align_up(4 * plane, 256) + 256;
}

extern "C" seg_status seg_solve3d(const float* f, int D, int H, int W, int ld, const uint32_t* act,
                                  const uint32_t* fgm, const int32_t* voxels, const int32_t* counts,
                                  const seg_params* prm, float* u, float* v, float* p1, float* p2, float* p3,
                                  void* state, size_t state_bytes, double* stats, void* ws,
                                  size_t ws_bytes, void* stream) {
    clear_error();
    if (!prm) return fail(SEG_ERR_INVALID_ARG, "params must be non-NULL");
    if (!f || !act || !fgm || !voxels || !counts || !u || !v || !p1 || !p2 || !p3 || !state || !stats)
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
    const size_t need = seg_state_bytes3d(D, H, ld);
    if (state_bytes < need) return fail(SEG_ERR_CAPACITY, "volume state needs %zu bytes, got %zu", need, state_bytes);
    if (reinterpret_cast<uintptr_t>(state) % 256) return fail(SEG_ERR_ALIGN, "state not 256-byte aligned");
    const int R = D * H;
    WsLayout L = ws_layout(R, W, th);
    SEG_TRY(check_ws(ws, ws_bytes, L));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    double* partials = ws_at<double>(ws, L.partials);

    VolGeom G{};
    G.D = D; G.H = H; G.W = W; G.ld = ld; G.nw = ld / 32; G.ntx = (W + 31) / 32; G.th = th; G.R = R;
    G.slice = (int64_t)H * ld;
    G.theta = (float)prm->theta;
    G.inv_theta = (float)(1.0 / prm->theta);
    G.tau = (float)prm->tau;
    G.theta_lambda = (float)(prm->theta * prm->lambda);
    VolState S{};
    const size_t plane = align_up(4 * (size_t)R * ld, 256);
    char* sb = static_cast<char*>(state);
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 3; ++k) S.p[b][k] = reinterpret_cast<float*>(sb + (size_t)(3 * b + k) * plane);
    S.w = reinterpret_cast<float*>(sb + 6 * plane);
    S.up = reinterpret_cast<float*>(sb + 7 * plane);
    S.off = reinterpret_cast<int32_t*>(sb + 8 * plane);
    S.flg = reinterpret_cast<uint16_t*>(sb + 9 * plane);

    SEG_TRY(launch_solve_begin(h, s));
    const int64_t n = (int64_t)R * W;
    const int eblocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
    k_vol_init<<<eblocks, 256, 0, s>>>(G, act, fgm, f, prm->warm_start, u, v, p1, p2, p3, S);
    SEG_LAUNCHED("k_vol_init");
    if (prm->warm_start) {
        k_vol_w<<<eblocks, 256, 0, s>>>(G, act, v, S);
        SEG_LAUNCHED("k_vol_w");
    }
    k_vol_setup<<<eblocks, 256, 0, s>>>(G, voxels, counts, act, fgm, S);
    SEG_LAUNCHED("k_vol_setup");
    const void* kern = (const void*)k_solve_vol;
    int per_sm = 0;
    SEG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kVolThreads, 0));
    if (per_sm <= 0) return fail(SEG_ERR_CUDA, "k_solve_vol cannot be resident");
    int grid = (int)std::min<int64_t>((int64_t)per_sm * sm_count(), L.npartials / 2);
    int iters = prm->iters, ce = prm->check_every;
    double tol = prm->tol;
    void* args[] = {&G, &iters, &ce, &tol, (void*)&act, (void*)&fgm, (void*)&voxels, (void*)&counts,
                    (void*)&f, &u, &v, &S, &partials, &h};
    if (iters > 0) {
        SEG_TRY_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kVolThreads), args, 0, s));
        count_launch();
    }
    k_vol_final<<<eblocks, 256, 0, s>>>(G, h, prm->iters, S, p1, p2, p3);
    SEG_LAUNCHED("k_vol_final");
    SEG_TRY(launch_solve_end(h, counts, prm->iters, stats, s));
    return SEG_OK;
}
