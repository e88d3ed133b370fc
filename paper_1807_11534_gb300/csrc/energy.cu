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
// The energy terms are accumulated per thread in double-float arithmetic
// (below) and combined across threads and blocks in FP64; the error terms
// in FP64.  A fixed grid and fixed-order reductions make the sums
// deterministic.
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

// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2 (Dekker 1971).  The error-free sum is
// Knuth's TwoSum, the error-free product uses the FMA, and the square root
// takes one correction step of the float root (Karp and Markstein).  About 48
// significant bits, all on the float pipes: the per-pixel energy terms cost a
// handful of float operations instead of FP64 ones, which this part runs at a
// small fraction of the float rate.
struct DF {
    float hi, lo;
};

// (explicitly rounded operations: the compiler must not fuse a product into
// a following sum here, which would break the error-free steps)
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {   // |a| >= |b| or a = 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = df_two_sum(a.hi, b.hi);
    const DF t = df_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return df_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_sqrt(DF a) {
    if (!(a.hi > 0.f)) return {0.f, 0.f};
    const float r = __fsqrt_rn(a.hi);
    const float rr = __fmul_rn(r, r);
    // a - r^2 with r^2 split exactly by the FMA
    const float e = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, rr), __fmaf_rn(r, r, -rr)), a.lo);
    return df_fast_two_sum(r, __fdiv_rn(e, __fmul_rn(2.f, r)));
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// |(a, b)| for a, b exact double-float differences
__device__ __forceinline__ DF df_hypot(DF a, DF b) { return df_sqrt(df_add(df_mul(a, a), df_mul(b, b))); }

// terms: 0 TV(u), 1 TV(v), 2 sum f u, 3 sum f v, 4 sum (u-v)^2, 5 sum min(0, lambda f + div p)
// Differences of two floats and products of two floats are exact in
// double-float; the rest carries ~2^-48 relative error per operation, and
// each thread's sums are double-float too, so no FP64 work happens per pixel.
__global__ void k_energy_terms(const float* __restrict__ f, int H, int W, int ld,
                               const float* __restrict__ u, const float* __restrict__ v,
                               const float* __restrict__ p1, const float* __restrict__ p2,
                               double lambda, double* __restrict__ red) {
    const DF zero{0.f, 0.f};
    DF acc[6] = {zero, zero, zero, zero, zero, zero};
    const float lam_hi = (float)lambda;
    const DF lam{lam_hi, (float)(lambda - (double)lam_hi)};
    const unsigned n = (unsigned)H * (unsigned)W;   // < 2^31 (checked by the callers)
    for (unsigned x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const unsigned i = x / (unsigned)W, j = x - i * (unsigned)W;
        const int64_t o = (int64_t)i * ld + j;
        const float uu = u[o], vv = v[o], ff = f[o];
        const bool dn = i + 1 < (unsigned)H, rt = j + 1 < (unsigned)W;
        const DF au = dn ? df_two_sum(u[o + ld], -uu) : zero;
        const DF bu = rt ? df_two_sum(u[o + 1], -uu) : zero;
        const DF av = dn ? df_two_sum(v[o + ld], -vv) : zero;
        const DF bv = rt ? df_two_sum(v[o + 1], -vv) : zero;
        acc[0] = df_add(acc[0], df_hypot(au, bu));
        acc[1] = df_add(acc[1], df_hypot(av, bv));
        acc[2] = df_add(acc[2], df_mul({ff, 0.f}, {uu, 0.f}));
        acc[3] = df_add(acc[3], df_mul({ff, 0.f}, {vv, 0.f}));
        const DF d = df_two_sum(uu, -vv);
        acc[4] = df_add(acc[4], df_mul(d, d));
        // div p (Chambolle): the components that never enter it are skipped
        DF dp = zero;
        if (dn) dp = df_add(dp, {p1[o], 0.f});
        if (i > 0) dp = df_add(dp, {-p1[o - ld], 0.f});
        if (rt) dp = df_add(dp, {p2[o], 0.f});
        if (j > 0) dp = df_add(dp, {-p2[o - 1], 0.f});
        const DF c = df_add(df_mul(lam, {ff, 0.f}), dp);
        if (c.hi < 0.f || (c.hi == 0.f && c.lo < 0.f)) acc[5] = df_add(acc[5], c);
    }
    double out[6];
#pragma unroll
    for (int t = 0; t < 6; ++t) out[t] = df_to_double(acc[t]);
    block_store_terms<6>(out, red);
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
        int64_t i = (int64_t)((uint32_t)x / (uint32_t)W), j = x - i * W;   // x < 2^31
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
    PhaseScope _scope("seg_energy", stream, ws);
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
    PhaseScope _scope("seg_errors", stream, ws);
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
