// fit.cu -- the fitting term of Section 1: Eq. CV f = (z-c1)^2 - (z-c2)^2 and
// Eq. DS f = CV + gamma P(x), with P the distance to the nearest marker pixel
// normalised by its maximum.  f is evaluated in FP64 with one IEEE rounding
// per operation (explicit _rn intrinsics: no contraction into FMA) and
// rounded once to float32, so it is a bit-exact function of z, c1, c2,
// markers and gamma.  c1, c2 may come from a label mask (class means, FP64,
// fixed-order reduction).
#include <algorithm>
#include <cmath>

#include "seg_internal.cuh"

namespace seg {

constexpr int kFitThreads = 256;
constexpr int kMarkerChunk = 1024;

// Per-block FP64 sums of z over label != 0 / label == 0 and their counts;
// red[b*4 + {0,1,2,3}] = {sum1, sum0, n1, n0}.
__global__ void k_label_sums(const float* __restrict__ z, const uint8_t* __restrict__ label,
                             int H, int W, int ld, double* __restrict__ red) {
    __shared__ double s[4][kFitThreads];
    double s1 = 0, s0 = 0;
    unsigned c1 = 0, c0 = 0;
    int64_t n = (int64_t)H * W;
    // both sums take an addition per pixel (0 for the other class: exact, so
    // the sums are those of the class's pixels in the same order), with no
    // divergence between the classes
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = (int64_t)((uint32_t)x / (uint32_t)W), j = x - i * W;   // x < 2^31
        const double zz = (double)z[i * ld + j];
        const bool in = label[i * ld + j] != 0;
        s1 = __dadd_rn(s1, in ? zz : 0.0);
        s0 = __dadd_rn(s0, in ? 0.0 : zz);
        c1 += in ? 1u : 0u;
        c0 += in ? 0u : 1u;
    }
    s[0][threadIdx.x] = s1; s[1][threadIdx.x] = s0; s[2][threadIdx.x] = (double)c1; s[3][threadIdx.x] = (double)c0;
    __syncthreads();
    for (int w = kFitThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int t = 0; t < 4; ++t) s[t][threadIdx.x] = __dadd_rn(s[t][threadIdx.x], s[t][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 4) red[(int64_t)blockIdx.x * 4 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_label_means(const double* __restrict__ sums, WsHeader* h, double* c_out) {
    double c1 = sums[2] > 0 ? __ddiv_rn(sums[0], sums[2]) : 0.0;
    double c2 = sums[3] > 0 ? __ddiv_rn(sums[1], sums[3]) : 0.0;
    h->c[0] = c1;
    h->c[1] = c2;
    if (c_out) { c_out[0] = c1; c_out[1] = c2; }
}

__global__ void k_set_c(WsHeader* h, double c1, double c2, double* c_out) {
    h->c[0] = c1;
    h->c[1] = c2;
    h->d2max = 0ull;
    if (c_out) { c_out[0] = c1; c_out[1] = c2; }
}

// Keeps the c1, c2 already in the header (set by the last fitting term or
// class-mean update).
__global__ void k_keep_c(WsHeader* h, double* c_out) {
    h->d2max = 0ull;
    if (c_out) { c_out[0] = h->c[0]; c_out[1] = h->c[1]; }
}

// Per-block FP64 sums of z over u > thresh (foreground) and u <= thresh and
// their counts; red[b*4 + {0,1,2,3}] = {sum1, sum0, n1, n0}.
__global__ void k_class_sums(const float* __restrict__ z, const float* __restrict__ u, float thresh,
                             int H, int W, int ld, double* __restrict__ red) {
    __shared__ double s[4][kFitThreads];
    double s1 = 0, s0 = 0;
    unsigned c1 = 0, c0 = 0;
    int64_t n = (int64_t)H * W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = (int64_t)((uint32_t)x / (uint32_t)W), j = x - i * W;   // x < 2^31
        const double zz = (double)z[i * ld + j];
        const bool in = u[i * ld + j] > thresh;   // as k_label_sums: branch-free, exact
        s1 = __dadd_rn(s1, in ? zz : 0.0);
        s0 = __dadd_rn(s0, in ? 0.0 : zz);
        c1 += in ? 1u : 0u;
        c0 += in ? 0u : 1u;
    }
    s[0][threadIdx.x] = s1; s[1][threadIdx.x] = s0; s[2][threadIdx.x] = (double)c1; s[3][threadIdx.x] = (double)c0;
    __syncthreads();
    for (int w = kFitThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int t = 0; t < 4; ++t) s[t][threadIdx.x] = __dadd_rn(s[t][threadIdx.x], s[t][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 4) red[(int64_t)blockIdx.x * 4 + threadIdx.x] = s[threadIdx.x][0];
}

// c1, c2 = the class means; a class without pixels keeps its previous value.
__global__ void k_update_means(const double* __restrict__ sums, WsHeader* h, double* c_out) {
    if (sums[2] > 0) h->c[0] = __ddiv_rn(sums[0], sums[2]);
    if (sums[3] > 0) h->c[1] = __ddiv_rn(sums[1], sums[3]);
    if (c_out) { c_out[0] = h->c[0]; c_out[1] = h->c[1]; }
}

// Smallest squared distance (exact integer) from pixel (i, j) to a marker.
__device__ __forceinline__ unsigned long long min_d2(const int2* sm, int m, int i, int j,
                                                     unsigned long long best) {
    for (int k = 0; k < m; ++k) {
        long long dy = (long long)i - sm[k].x, dx = (long long)j - sm[k].y;
        unsigned long long d = (unsigned long long)(dy * dy + dx * dx);
        best = d < best ? d : best;
    }
    return best;
}

// The same in 32-bit integers, exact when both image sides are at most
// kSmallSide and every marker lies inside the image (every squared distance
// is then below 2^31).
constexpr int kSmallSide = 32767;

// Whether every marker lies inside the H x W image (the same answer in every
// block; all threads of the block must call it).
__device__ __forceinline__ bool markers_inside(const int32_t* __restrict__ markers, int n_markers, int H, int W) {
    int ok = 1;
    for (int k = threadIdx.x; k < n_markers; k += blockDim.x) {
        const int my = markers[2 * k], mx = markers[2 * k + 1];
        ok &= (my >= 0 && my < H && mx >= 0 && mx < W) ? 1 : 0;
    }
    return __syncthreads_and(ok) != 0;
}
__device__ __forceinline__ unsigned min_d2_32(const int2* sm, int m, int i, int j, unsigned best) {
    for (int k = 0; k < m; ++k) {
        const int dy = i - sm[k].x, dx = j - sm[k].y;
        const unsigned d = (unsigned)(dy * dy + dx * dx);
        best = d < best ? d : best;
    }
    return best;
}

// Maximum over the image of the squared distance to the nearest marker.
// SMALL (both sides <= kSmallSide) with every marker inside the image:
// 32-bit distances, and each pixel's nearest squared distance is left in its
// f word (as uint32 bits) for k_fitting<true>, which then skips the marker
// loop.
template <bool SMALL>
__global__ void k_marker_dmax(const int32_t* __restrict__ markers, int n_markers, int H, int W, int ld,
                              WsHeader* h, float* __restrict__ f) {
    __shared__ int2 sm[kMarkerChunk];
    __shared__ unsigned long long s_max[kFitThreads / 32];
    int64_t n = (int64_t)H * W;
    unsigned long long local = 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t x0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // every thread of the block walks the same number of rounds so the
    // marker chunks can be staged with __syncthreads
    int64_t rounds = (n + stride - 1) / stride;
    const bool small = SMALL && markers_inside(markers, n_markers, H, W);
    for (int64_t r = 0; r < rounds; ++r) {
        int64_t x = x0 + r * stride;
        const int i = (int)((uint32_t)x / (uint32_t)W), j = (int)(x - (int64_t)i * W);   // x < 2^31
        unsigned long long best = ~0ull;
        unsigned best32 = ~0u;
        for (int c0 = 0; c0 < n_markers; c0 += kMarkerChunk) {
            int m = min(kMarkerChunk, n_markers - c0);
            __syncthreads();
            for (int k = threadIdx.x; k < m; k += blockDim.x)
                sm[k] = make_int2(markers[2 * (c0 + k)], markers[2 * (c0 + k) + 1]);
            __syncthreads();
            if (x < n) {
                if (small) best32 = min_d2_32(sm, m, i, j, best32);
                else best = min_d2(sm, m, i, j, best);
            }
        }
        if (small && x < n) {
            best = best32;
            reinterpret_cast<unsigned*>(f)[(int64_t)i * ld + j] = best32;
        }
        if (x < n && best > local) local = best;
    }
    for (int d = 16; d > 0; d >>= 1) {
        unsigned long long o = __shfl_down_sync(0xffffffffu, local, d);
        local = o > local ? o : local;
    }
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int w = 0; w < kFitThreads / 32; ++w) m = s_max[w] > m ? s_max[w] : m;
        atomicMax(&h->d2max, m);
    }
}

// f = ((z-c1)^2 - (z-c2)^2) [+ gamma * sqrt(d2) / sqrt(d2max)], FP64, one
// rounding per operation in this order, then rounded to float32.  CACHED:
// d2 is read from the pixel's f word where k_marker_dmax<true> left it
// (every marker inside the image; else the marker loop runs here).
template <bool CACHED>
__global__ void k_fitting(const float* __restrict__ z, int H, int W, int ld,
                          const int32_t* __restrict__ markers, int n_markers, double gamma,
                          const WsHeader* __restrict__ h, float* __restrict__ f) {
    __shared__ int2 sm[kMarkerChunk];
    const double c1 = h->c[0], c2 = h->c[1];
    const unsigned long long d2max = h->d2max;
    const double dmax = __dsqrt_rn((double)d2max);
    int64_t n = (int64_t)H * W;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t x0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t rounds = (n + stride - 1) / stride;
    const bool cached = CACHED && markers_inside(markers, n_markers, H, W);
    for (int64_t r = 0; r < rounds; ++r) {
        int64_t x = x0 + r * stride;
        const int i = (int)((uint32_t)x / (uint32_t)W), j = (int)(x - (int64_t)i * W);   // x < 2^31
        unsigned long long best = ~0ull;
        if (cached) {
            if (x < n) best = reinterpret_cast<const unsigned*>(f)[(int64_t)i * ld + j];
        } else {
            for (int c0 = 0; c0 < n_markers; c0 += kMarkerChunk) {
                int m = min(kMarkerChunk, n_markers - c0);
                __syncthreads();
                for (int k = threadIdx.x; k < m; k += blockDim.x)
                    sm[k] = make_int2(markers[2 * (c0 + k)], markers[2 * (c0 + k) + 1]);
                __syncthreads();
                if (x < n) best = min_d2(sm, m, i, j, best);
            }
        }
        if (x >= n) continue;
        double zz = (double)z[(int64_t)i * ld + j];
        double t1 = __dsub_rn(zz, c1);
        double t2 = __dsub_rn(zz, c2);
        double a = __dmul_rn(t1, t1);
        double b = __dmul_rn(t2, t2);
        double fv = __dsub_rn(a, b);
        if (n_markers > 0) {
            double P = d2max > 0 ? __ddiv_rn(__dsqrt_rn((double)best), dmax) : 0.0;
            double gp = __dmul_rn(gamma, P);
            fv = __dadd_rn(fv, gp);
        }
        f[(int64_t)i * ld + j] = __double2float_rn(fv);
    }
}

}  // namespace seg

using namespace seg;

extern "C" seg_status seg_make_fitting(const float* z, int H, int W, int ld, double c1, double c2,
                                       const uint8_t* label, const int32_t* markers, int n_markers,
                                       double gamma, float* f, double* c_out, void* ws,
                                       size_t ws_bytes, void* stream) {
    clear_error();
    PhaseScope _scope("seg_make_fitting", stream, ws);
    if (!z || !f) return fail(SEG_ERR_INVALID_ARG, "z and f must be non-NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * W >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    if (n_markers < 0 || (n_markers > 0 && !markers))
        return fail(SEG_ERR_INVALID_ARG, "markers NULL with n_markers=%d", n_markers);
    // the fitting term only needs the header and the reduction scratch
    if (!ws || ws_bytes < kWsFixedBytes)
        return fail(SEG_ERR_WORKSPACE, "workspace too small for seg_make_fitting");
    if (reinterpret_cast<uintptr_t>(ws) % 16) return fail(SEG_ERR_ALIGN, "workspace not 16-byte aligned");
    WsLayout L = ws_layout(H, W, 32);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    if (!label && std::isnan(c1) && std::isnan(c2)) {   // the c1, c2 already in the workspace
        k_keep_c<<<1, 1, 0, s>>>(h, c_out);
        SEG_LAUNCHED("k_keep_c");
    } else {
        k_set_c<<<1, 1, 0, s>>>(h, c1, c2, label ? nullptr : c_out);
        SEG_LAUNCHED("k_set_c");
    }
    if (label) {
        double* red = ws_at<double>(ws, L.red);
        k_label_sums<<<kReduceBlocks, kFitThreads, 0, s>>>(z, label, H, W, ld, red);
        SEG_LAUNCHED("k_label_sums");
        double* sums = red + (size_t)kReduceBlocks * 4;
        SEG_TRY(reduce_partials(red, kReduceBlocks, 4, sums, s));
        k_label_means<<<1, 1, 0, s>>>(sums, h, c_out);
        SEG_LAUNCHED("k_label_means");
    }
    int64_t n = (int64_t)H * W;
    int blocks = (int)std::min<int64_t>((n + kFitThreads - 1) / kFitThreads, 152 * 8);
    const bool small = H <= kSmallSide && W <= kSmallSide;
    if (n_markers > 0 && small) {
        k_marker_dmax<true><<<blocks, kFitThreads, 0, s>>>(markers, n_markers, H, W, ld, h, f);
        SEG_LAUNCHED("k_marker_dmax");
        k_fitting<true><<<blocks, kFitThreads, 0, s>>>(z, H, W, ld, markers, n_markers, gamma, h, f);
        SEG_LAUNCHED("k_fitting");
    } else {
        if (n_markers > 0) {
            k_marker_dmax<false><<<blocks, kFitThreads, 0, s>>>(markers, n_markers, H, W, ld, h, f);
            SEG_LAUNCHED("k_marker_dmax");
        }
        k_fitting<false><<<blocks, kFitThreads, 0, s>>>(z, H, W, ld, markers, n_markers, gamma, h, f);
        SEG_LAUNCHED("k_fitting");
    }
    return SEG_OK;
}

// Chan-Vese update of the intensities (the alternating step of the
// piecewise-constant model of Section 1's [ACWE] fitting term, with the
// relaxed u thresholded): c1 = mean of z over u > thresh, c2 = mean over
// u <= thresh, FP64 with a fixed-order reduction, stored in the workspace for
// the next seg_make_fitting (called with c1 = c2 = NaN) and in c_out.
extern "C" seg_status seg_update_means(const float* z, const float* u, int H, int W, int ld, double thresh,
                                       double* c_out, void* ws, size_t ws_bytes, void* stream) {
    using namespace seg;
    clear_error();
    PhaseScope _scope("seg_update_means", stream, ws);
    if (!z || !u) return fail(SEG_ERR_INVALID_ARG, "z and u must be non-NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * W >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    if (!std::isfinite(thresh)) return fail(SEG_ERR_INVALID_ARG, "thresh must be finite");
    if (!ws || ws_bytes < kWsFixedBytes)
        return fail(SEG_ERR_WORKSPACE, "workspace too small for seg_update_means");
    if (reinterpret_cast<uintptr_t>(ws) % 16) return fail(SEG_ERR_ALIGN, "workspace not 16-byte aligned");
    WsLayout L = ws_layout(H, W, 32);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    double* red = ws_at<double>(ws, L.red);
    k_class_sums<<<kReduceBlocks, kFitThreads, 0, s>>>(z, u, (float)thresh, H, W, ld, red);
    SEG_LAUNCHED("k_class_sums");
    double* sums = red + (size_t)kReduceBlocks * 4;
    SEG_TRY(reduce_partials(red, kReduceBlocks, 4, sums, s));
    k_update_means<<<1, 1, 0, s>>>(sums, h, c_out);
    SEG_LAUNCHED("k_update_means");
    return SEG_OK;
}
