// energy.cu -- energies and error measures, FP64 reductions over the image.
//
//   TV(u)   = sum |grad u| (isotropic, forward differences, zero on the last
//             row / column)
//   E_CR(u) = TV(u) + lambda sum f u                      (Eq. CR, Section 2)
//   E_DF    = TV(u) + sum (u - v)^2 / (2 theta) + lambda sum f v   (Eq. DF,
//             whose penalty psi(v) vanishes for v in [0, 1])
//   D(p)    = sum min(0, lambda f + div p): writing TV(u) = max_{|p|<=1}
//             <u, div p> and minimising lambda <f, u> + <u, div p> over
//             u in [0, 1] pixel by pixel gives this lower bound on Eq. CR
//   gap     = E_CR(v) - D(p) >= 0 for v in [0, 1], |p| <= 1
//   E1, E2  : Section 4 (Tanimoto of the eps-thresholded masks; sum of
//             squared differences)
// Each block accumulates its pixels in FP64 in a fixed order; a fixed grid and
// a fixed-order final reduction make the sums deterministic.
#include "seg_internal.cuh"

namespace seg {

constexpr int kEnThreads = kEnergyBlockThreads;

template <int NTERMS>
__device__ __forceinline__ void block_store_terms(double (&acc)[NTERMS], double* red) {
    __shared__ double s[NTERMS][kEnThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < NTERMS; ++t) {
        double a = acc[t];
        for (int d = 16; d > 0; d >>= 1) a += __shfl_down_sync(0xffffffffu, a, d);
        if (lane == 0) s[t][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < NTERMS) {
        double x = 0;
        for (int w = 0; w < kEnThreads / 32; ++w) x += s[threadIdx.x][w];
        red[(int64_t)blockIdx.x * NTERMS + threadIdx.x] = x;
    }
}

// terms: 0 TV(u), 1 TV(v), 2 sum f u, 3 sum f v, 4 sum (u-v)^2, 5 sum min(0, lambda f + div p)
__global__ void k_energy_terms(const float* __restrict__ f, int H, int W, int ld,
                               const float* __restrict__ u, const float* __restrict__ v,
                               const float* __restrict__ p1, const float* __restrict__ p2,
                               double lambda, double* __restrict__ red) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    int64_t n = (int64_t)H * W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = x / W, j = x - i * W;
        int64_t o = i * ld + j;
        double uu = u[o], vv = v[o], ff = f[o];
        double au = i < H - 1 ? (double)u[o + ld] - uu : 0.0;
        double bu = j < W - 1 ? (double)u[o + 1] - uu : 0.0;
        double av = i < H - 1 ? (double)v[o + ld] - vv : 0.0;
        double bv = j < W - 1 ? (double)v[o + 1] - vv : 0.0;
        acc[0] += sqrt(au * au + bu * bu);
        acc[1] += sqrt(av * av + bv * bv);
        acc[2] += ff * uu;
        acc[3] += ff * vv;
        acc[4] += (uu - vv) * (uu - vv);
        double d = (i < H - 1 ? (double)p1[o] : 0.0) - (i > 0 ? (double)p1[o - ld] : 0.0) +
                   (j < W - 1 ? (double)p2[o] : 0.0) - (j > 0 ? (double)p2[o - 1] : 0.0);
        double c = lambda * ff + d;
        acc[5] += c < 0.0 ? c : 0.0;
    }
    block_store_terms<6>(acc, red);
}

__global__ void k_energy_final(const double* __restrict__ sums, double lambda, double theta,
                               double* out) {
    double tvu = sums[0], tvv = sums[1], fu = sums[2], fv = sums[3], quad = sums[4], dual = sums[5];
    out[0] = tvu;
    out[1] = tvu + lambda * fu;
    out[2] = tvv + lambda * fv;
    out[3] = tvu + quad / (2.0 * theta) + lambda * fv;
    out[4] = dual;
    out[5] = out[2] - dual;
}

// terms: 0 N(GT & O*), 1 N(GT | O*), 2 sum (u* - u_gt)^2
__global__ void k_error_terms(const float* __restrict__ us, const float* __restrict__ ug, int H, int W,
                              int ld, float eps, double* __restrict__ red) {
    double acc[3] = {0, 0, 0};
    int64_t n = (int64_t)H * W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = x / W, j = x - i * W;
        int64_t o = i * ld + j;
        float a = us[o], b = ug[o];
        bool A = b > eps, B = a > eps;
        acc[0] += (A && B) ? 1.0 : 0.0;
        acc[1] += (A || B) ? 1.0 : 0.0;
        double d = (double)a - (double)b;
        acc[2] += d * d;
    }
    block_store_terms<3>(acc, red);
}

__global__ void k_error_final(const double* __restrict__ sums, double* out) {
    out[0] = sums[1] > 0 ? sums[0] / sums[1] : 1.0;
    out[1] = sums[2];
}

}  // namespace seg

using namespace seg;

static seg_status check_image(const void* a, int H, int W, int ld) {
    if (!a) return fail(SEG_ERR_INVALID_ARG, "image pointer is NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * W >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    return SEG_OK;
}

extern "C" seg_status seg_energy(const float* f, int H, int W, int ld, const float* u, const float* v,
                                 const float* p1, const float* p2, double lambda, double theta,
                                 double* out, void* ws, size_t ws_bytes, void* stream) {
    clear_error();
    SEG_TRY(check_image(f, H, W, ld));
    if (!u || !v || !p1 || !p2 || !out) return fail(SEG_ERR_INVALID_ARG, "a required pointer is NULL");
    if (!(theta > 0)) return fail(SEG_ERR_INVALID_ARG, "theta must be > 0");
    if (!ws || ws_bytes < kWsFixedBytes) return fail(SEG_ERR_WORKSPACE, "workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* red = ws_at<double>(ws, kWsRedOff);
    double* sums = red + (size_t)kReduceBlocks * 6;
    k_energy_terms<<<kReduceBlocks, kEnThreads, 0, s>>>(f, H, W, ld, u, v, p1, p2, lambda, red);
    SEG_LAUNCHED("k_energy_terms");
    SEG_TRY(reduce_partials(red, kReduceBlocks, 6, sums, s));
    k_energy_final<<<1, 1, 0, s>>>(sums, lambda, theta, out);
    SEG_LAUNCHED("k_energy_final");
    return SEG_OK;
}

extern "C" seg_status seg_errors(const float* u_star, const float* u_gt, int H, int W, int ld,
                                 double eps, double* out, void* ws, size_t ws_bytes, void* stream) {
    clear_error();
    SEG_TRY(check_image(u_star, H, W, ld));
    SEG_TRY(check_image(u_gt, H, W, ld));
    if (!out) return fail(SEG_ERR_INVALID_ARG, "out is NULL");
    if (!ws || ws_bytes < kWsFixedBytes) return fail(SEG_ERR_WORKSPACE, "workspace too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* red = ws_at<double>(ws, kWsRedOff);
    double* sums = red + (size_t)kReduceBlocks * 3;
    k_error_terms<<<kReduceBlocks, kEnThreads, 0, s>>>(u_star, u_gt, H, W, ld, (float)eps, red);
    SEG_LAUNCHED("k_error_terms");
    SEG_TRY(reduce_partials(red, kReduceBlocks, 3, sums, s));
    k_error_final<<<1, 1, 0, s>>>(sums, out);
    SEG_LAUNCHED("k_error_final");
    return SEG_OK;
}
