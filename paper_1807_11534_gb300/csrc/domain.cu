// domain.cu -- the Fg / Bg / RD partition of Section 3 and its bit-exact
// stream compaction.
//
//   RD = {|f| < delta}, Fg = {f < 0} \ RD, Bg = the rest (u0 = H(-f), H(0) = 0)
//
// The partition is stored as two bit planes (RD bits, f<0 bits) of one
// uint32 per 32 pixels.  Tiles of 32 columns x tile_h rows holding an RD
// pixel are compacted into an ascending tile list; RD pixels are numbered in
// tile-major order (tiles row-major, then rows, then columns), and every mask
// word gets the compact index of its first RD pixel, so the compact index of
// pixel (i, j) is wstart[i][j/32] + popc(act[i][j/32] & lanemask_lt(j%32)).
// Integer scans only: the outputs are bit-exact functions of f and delta.
//
// Robust restriction (the Conclusion's open point for noisy f): RD may be
// grown by every pixel within Chebyshev distance r of an RD pixel (a square
// dilation of the RD bit plane, rows then columns), before the lists are
// built; the grown pixels start from u0 = H(-f) like any RD pixel.
//
// Quantile mode (Section 3: q-hat grows from 0 until |RD| / n reaches q):
// delta is the float just above the k-th smallest |f|, k = ceil(q n), found
// by an exact 4-pass radix select on the bit patterns of |f| (for
// non-negative floats the bit order is the numeric order).
#include <algorithm>
#include <cmath>

#include "seg_internal.cuh"

namespace seg {

constexpr int kDomThreads = 256;

__global__ void k_set_delta(WsHeader* h, float delta) {
    h->delta = delta;
    h->n_fg = 0;
    h->qk0 = 0;
}

__global__ void k_q_init(WsHeader* h, long long k) {
    h->qprefix = 0u;
    h->qk = k;
    h->qk0 = k;
    h->n_fg = 0;
}

// Histogram of digit (key >> shift) & 255 over the keys whose higher digits
// equal the prefix found so far.
__global__ void k_q_hist(const float* __restrict__ f, int H, int W, int ld, int shift,
                         const WsHeader* __restrict__ h, unsigned* __restrict__ hist) {
    __shared__ unsigned sh[kHistBins];
    for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const unsigned prefix = h->qprefix;
    const int hi = shift + 8;
    int64_t n = (int64_t)H * W;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = (int64_t)((uint32_t)x / (uint32_t)W), j = x - i * W;   // x < 2^31
        unsigned key = __float_as_uint(f[i * ld + j]) & 0x7fffffffu;
        bool match = hi >= 32 ? true : ((key >> hi) == (prefix >> hi));
        if (match) atomicAdd(&sh[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kHistBins; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

__global__ void k_q_select(WsHeader* h, const unsigned* __restrict__ hist, int shift) {
    long long need = h->qk;
    long long cum = 0;
    int b = 0;
    for (; b < kHistBins; ++b) {
        if (cum + (long long)hist[b] >= need) break;
        cum += hist[b];
    }
    if (b == kHistBins) b = kHistBins - 1;   // unreachable for 1 <= k <= n
    h->qprefix |= (unsigned)b << shift;
    h->qk = need - cum;
}

__global__ void k_q_finish(WsHeader* h) {
    unsigned t = h->qprefix;   // bit pattern of the k-th smallest |f|
    if (t >= 0x7f800000u) {    // Inf or NaN: no finite threshold above it
        record_status(h, SEG_ERR_NONFINITE);
        h->delta = __uint_as_float(0x7f800000u);
    } else {
        h->delta = __uint_as_float(t + 1u);   // next float above t
    }
}

// One warp per mask word: lane b classifies pixel (i, 32k + b).
// fsel: the field thresholded (f, or its local mean fbar for the robust
// restriction, which also admits the pixels whose sign differs from fbar's).
__global__ void k_classify(const float* __restrict__ f, const float* __restrict__ fsel, int H,
                           int W, int ld, int nw, WsHeader* h, uint32_t* __restrict__ act,
                           uint32_t* __restrict__ fg) {
    __shared__ int s_fg[kDomThreads / 32];
    const float delta = h->delta;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t word = (int64_t)blockIdx.x * (blockDim.x / 32) + wid;
    int64_t nwords = (int64_t)H * nw;
    int cnt = 0;
    if (word < nwords) {
        int64_t i = word / nw;
        int j = (int)(word - i * nw) * 32 + lane;
        bool a = false, g = false, bad = false;
        if (j < W) {
            const float fv = f[i * ld + j];
            const float fs = fsel[i * ld + j];
            bad = !isfinite(fv) || !isfinite(fs);
            a = fabsf(fs) < delta || ((fv < 0.0f) != (fs < 0.0f));
            g = fv < 0.0f;
        }
        unsigned wa = __ballot_sync(0xffffffffu, a);
        unsigned wg = __ballot_sync(0xffffffffu, g);
        unsigned wb = __ballot_sync(0xffffffffu, bad);
        if (lane == 0) {
            act[word] = wa;
            fg[word] = wg;
            if (wb) record_status(h, SEG_ERR_NONFINITE);
            cnt = __popc(wg & ~wa);
        }
    }
    if (lane == 0) s_fg[wid] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kDomThreads / 32; ++w) t += s_fg[w];
        if (t) atomicAdd(&h->n_fg, t);
    }
}

// Square dilation, horizontal half: one thread per word; bit b of word k is
// column 32k + b, and a column joins if a column within r of it is in RD
// (r <= 32: the neighbour words suffice).  Columns >= W stay clear.
__global__ void k_dilate_rows(const uint32_t* __restrict__ act, int H, int W, int nw, int r,
                              uint32_t* __restrict__ out, WsHeader* h) {
    const int64_t word = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (word == 0) h->n_fg = 0;   // recounted by k_dilate_cols
    if (word >= (int64_t)H * nw) return;
    const int64_t i = word / nw;
    const int k = (int)(word - i * nw);
    const int ntx = (W + 31) / 32;
    if (k >= ntx) {
        out[word] = 0u;
        return;
    }
    const uint32_t c = act[word];
    const uint32_t pv = k > 0 ? act[word - 1] : 0u;
    const uint32_t nx = k + 1 < ntx ? act[word + 1] : 0u;
    uint32_t d = c;
    for (int s = 1; s <= r; ++s) {
        if (s < 32) d |= (c >> s) | (nx << (32 - s)) | (c << s) | (pv >> (32 - s));
        else d |= nx | pv;
    }
    const int rem = W - 32 * k;
    if (rem < 32) d &= (1u << rem) - 1u;
    out[word] = d;
}

// Square dilation, vertical half: OR of the rows within r; recounts the
// fixed foreground pixels (f < 0 outside the grown RD).
__global__ void k_dilate_cols(const uint32_t* __restrict__ rows, int H, int nw, int r,
                              const uint32_t* __restrict__ fg, uint32_t* __restrict__ act,
                              WsHeader* h) {
    __shared__ int s_fg[kDomThreads / 32];
    const int64_t word = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (word < (int64_t)H * nw) {
        const int i = (int)(word / nw);
        const int k = (int)(word - (int64_t)i * nw);
        const int i0 = i - r < 0 ? 0 : i - r, i1 = i + r >= H ? H - 1 : i + r;
        uint32_t d = 0u;
        for (int ii = i0; ii <= i1; ++ii) d |= rows[(int64_t)ii * nw + k];
        act[word] = d;
        cnt = __popc(fg[word] & ~d);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) s_fg[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kDomThreads / 32; ++w) t += s_fg[w];
        if (t) atomicAdd(&h->n_fg, t);
    }
}

// Local mean of f over the (2r+1) x (2r+1) square clipped to the image: the
// window's values summed in FP64 in row-major order, divided by the count
// and rounded once to float32 (the rounding order is fixed, so the result is
// a bit-exact function of f).
__global__ void k_box_mean(const float* __restrict__ f, int H, int W, int ld, int r,
                           float* __restrict__ out) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= (int64_t)H * W) return;
    const int i = (int)((uint32_t)x / (uint32_t)W), j = (int)(x - (int64_t)i * W);   // x < 2^31
    const int i0 = max(i - r, 0), i1 = min(i + r, H - 1), j0 = max(j - r, 0), j1 = min(j + r, W - 1);
    double sum = 0.0;
    for (int a = i0; a <= i1; ++a)
        for (int b = j0; b <= j1; ++b) sum = __dadd_rn(sum, (double)f[(int64_t)a * ld + b]);
    const double cnt = (double)((i1 - i0 + 1) * (j1 - j0 + 1));
    out[(int64_t)i * ld + j] = __double2float_rn(__ddiv_rn(sum, cnt));
}

__global__ void k_tile_count(const uint32_t* __restrict__ act, int H, int nw, int ntx, int th,
                             int64_t ntiles, int* __restrict__ cnt, int* __restrict__ flag) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int64_t ty = t / ntx, tx = t - ty * ntx;
    int c = 0;
    for (int r = 0; r < th; ++r) {
        int64_t i = ty * th + r;
        if (i >= H) break;
        c += __popc(act[i * nw + tx]);
    }
    cnt[t] = c;
    flag[t] = c > 0;
}

// One warp per tile: wstart of its words, its slot in the tile list and the
// linear ids of its RD pixels.
__global__ void k_tile_emit(const uint32_t* __restrict__ act, int H, int W, int nw, int ntx,
                            int th, int64_t ntiles, const int* __restrict__ tstart,
                            const int* __restrict__ tflag, const int* __restrict__ tpos,
                            int32_t* __restrict__ wstart, int32_t* __restrict__ tiles,
                            int tiles_cap, int32_t* __restrict__ pixels, int64_t pixels_cap,
                            WsHeader* h) {
    int lane = threadIdx.x & 31;
    int64_t t = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (t >= ntiles) return;
    int64_t ty = t / ntx, tx = t - ty * ntx;
    int64_t i = ty * th + lane;
    bool row = lane < th && i < H;
    uint32_t w = row ? act[i * nw + tx] : 0u;
    int c = __popc(w);
    int inc = c;
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    int base = tstart[t] + inc - c;
    if (row) wstart[i * nw + tx] = base;
    if (lane == 0 && tflag[t]) {
        int p = tpos[t];
        if (p < tiles_cap) tiles[p] = (int32_t)t;
        else record_status(h, SEG_ERR_CAPACITY);
    }
    if (pixels && row) {
        int k = 0;
        while (w) {
            int b = __ffs(w) - 1;
            int64_t idx = (int64_t)base + k;
            if (idx < pixels_cap) pixels[idx] = (int32_t)(i * W + tx * 32 + b);
            else record_status(h, SEG_ERR_CAPACITY);
            w &= w - 1;
            ++k;
        }
    }
}

__global__ void k_domain_finish(const WsHeader* __restrict__ h, int32_t* counts, float* delta_out,
                                const int* __restrict__ n_tiles_dev, const int* __restrict__ n_act_dev) {
    counts[0] = *n_tiles_dev;
    counts[1] = *n_act_dev;
    counts[2] = h->n_fg;
    counts[3] = (int32_t)h->qk0;
    if (delta_out) *delta_out = h->delta;
}

}  // namespace seg

using namespace seg;

static seg_status build_domain(const float* f, const float* fbar, int H, int W, int ld,
                               double delta, double q, int radius, int tile_h, uint32_t* act, uint32_t* fg,
                               int32_t* wstart, int32_t* tiles, int tiles_cap, int32_t* pixels,
                               int64_t pixels_cap, int32_t* counts, float* delta_out, void* ws,
                               size_t ws_bytes, void* stream) {
    clear_error();
    if (radius < 0 || radius > 32)
        return fail(SEG_ERR_INVALID_ARG, "radius=%d not in [0, 32]", radius);
    if (!f || !act || !fg || !wstart || !tiles || !counts)
        return fail(SEG_ERR_INVALID_ARG, "f, act, fg, wstart, tiles and counts must be non-NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * W >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    if (tile_h != 4 && tile_h != 8 && tile_h != 16 && tile_h != 32)
        return fail(SEG_ERR_INVALID_ARG, "tile_h=%d not in {4, 8, 16, 32}", tile_h);
    if (tiles_cap < 0 || pixels_cap < 0) return fail(SEG_ERR_INVALID_ARG, "negative capacity");
    if (std::isnan(delta) && q < 0) return fail(SEG_ERR_INVALID_ARG, "delta is NaN");
    if (!(q <= 1.0)) return fail(SEG_ERR_INVALID_ARG, "q=%g > 1", q);
    WsLayout L = ws_layout(H, W, tile_h);
    SEG_TRY(check_ws(ws, ws_bytes, L));
    const float* fsel = fbar ? fbar : f;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader* h = ws_at<WsHeader>(ws, L.header);
    int64_t n = (int64_t)H * W;
    int nw = ld / 32, ntx = (W + 31) / 32;

    if (q >= 0) {
        long long k = (long long)std::ceil(q * (double)n);
        if (k > n) k = n;
        if (k <= 0) {
            k_set_delta<<<1, 1, 0, s>>>(h, 0.0f);
            SEG_LAUNCHED("k_set_delta");
        } else {
            k_q_init<<<1, 1, 0, s>>>(h, k);
            SEG_LAUNCHED("k_q_init");
            unsigned* hist = ws_at<unsigned>(ws, L.hist);
            int blocks = (int)std::min<int64_t>((n + kDomThreads - 1) / kDomThreads, 152 * 8);
            for (int shift = 24; shift >= 0; shift -= 8) {
                SEG_TRY_CUDA(cudaMemsetAsync(hist, 0, 4 * kHistBins, s));
                k_q_hist<<<blocks, kDomThreads, 0, s>>>(fsel, H, W, ld, shift, h, hist);
                SEG_LAUNCHED("k_q_hist");
                k_q_select<<<1, 1, 0, s>>>(h, hist, shift);
                SEG_LAUNCHED("k_q_select");
            }
            k_q_finish<<<1, 1, 0, s>>>(h);
            SEG_LAUNCHED("k_q_finish");
        }
    } else {
        float d = (float)delta;   // +inf stays +inf: the unrestricted problem
        k_set_delta<<<1, 1, 0, s>>>(h, d);
        SEG_LAUNCHED("k_set_delta");
    }

    int64_t nwords = (int64_t)H * nw;
    k_classify<<<(unsigned)((nwords + 7) / 8), kDomThreads, 0, s>>>(f, fsel, H, W, ld, nw, h, act,
                                                                    fg);
    SEG_LAUNCHED("k_classify");
    if (radius > 0) {   // wstart (same shape, written later) holds the row pass
        uint32_t* rows = reinterpret_cast<uint32_t*>(wstart);
        const unsigned nb = (unsigned)((nwords + kDomThreads - 1) / kDomThreads);
        k_dilate_rows<<<nb, kDomThreads, 0, s>>>(act, H, W, nw, radius, rows, h);
        SEG_LAUNCHED("k_dilate_rows");
        k_dilate_cols<<<nb, kDomThreads, 0, s>>>(rows, H, nw, radius, fg, act, h);
        SEG_LAUNCHED("k_dilate_cols");
    }

    int* cnt = ws_at<int>(ws, L.tile_cnt);
    int* flag = ws_at<int>(ws, L.tile_flag);
    int* tstart = ws_at<int>(ws, L.tile_start);
    int* tpos = ws_at<int>(ws, L.tile_pos);
    int* tmp = ws_at<int>(ws, L.scan_tmp);
    int* n_act_dev = cnt + L.ntiles;     // spare slot after each array
    int* n_tiles_dev = flag + L.ntiles;
    k_tile_count<<<(unsigned)((L.ntiles + 255) / 256), 256, 0, s>>>(act, H, nw, ntx, tile_h,
                                                                    L.ntiles, cnt, flag);
    SEG_LAUNCHED("k_tile_count");
    SEG_TRY(scan_exclusive(cnt, tstart, L.ntiles, n_act_dev, tmp, s));
    SEG_TRY(scan_exclusive(flag, tpos, L.ntiles, n_tiles_dev, tmp, s));
    k_tile_emit<<<(unsigned)((L.ntiles + 7) / 8), 256, 0, s>>>(act, H, W, nw, ntx, tile_h, L.ntiles,
                                                              tstart, flag, tpos, wstart, tiles,
                                                              tiles_cap, pixels, pixels_cap, h);
    SEG_LAUNCHED("k_tile_emit");
    k_domain_finish<<<1, 1, 0, s>>>(h, counts, delta_out, n_tiles_dev, n_act_dev);
    SEG_LAUNCHED("k_domain_finish");
    return SEG_OK;
}

extern "C" seg_status seg_build_domain(const float* f, int H, int W, int ld, double delta, double q,
                                       int tile_h, uint32_t* act, uint32_t* fg, int32_t* wstart,
                                       int32_t* tiles, int tiles_cap, int32_t* pixels,
                                       int64_t pixels_cap, int32_t* counts, float* delta_out,
                                       void* ws, size_t ws_bytes, void* stream) {
    PhaseScope _scope("seg_build_domain", stream, ws);
    return build_domain(f, nullptr, H, W, ld, delta, q, 0, tile_h, act, fg, wstart, tiles,
                        tiles_cap, pixels, pixels_cap, counts, delta_out, ws, ws_bytes, stream);
}

extern "C" seg_status seg_build_domain_robust(const float* f, const float* fbar, int H, int W,
                                              int ld, double delta, double q, int radius,
                                              int tile_h, uint32_t* act, uint32_t* fg,
                                              int32_t* wstart, int32_t* tiles, int tiles_cap,
                                              int32_t* pixels, int64_t pixels_cap,
                                              int32_t* counts, float* delta_out, void* ws,
                                              size_t ws_bytes, void* stream) {
    PhaseScope _scope("seg_build_domain_robust", stream, ws);
    if (fbar == f) fbar = nullptr;
    return build_domain(f, fbar, H, W, ld, delta, q, radius, tile_h, act, fg, wstart, tiles,
                        tiles_cap, pixels, pixels_cap, counts, delta_out, ws, ws_bytes, stream);
}

extern "C" seg_status seg_box_mean(const float* f, int H, int W, int ld, int radius, float* out,
                                   void* stream) {
    clear_error();
    PhaseScope _scope("seg_box_mean", stream, nullptr);
    if (!f || !out) return fail(SEG_ERR_INVALID_ARG, "f and out must be non-NULL");
    if (H <= 0 || W <= 0 || ld < W || (int64_t)H * W >= (1ll << 31))
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    if (radius < 0 || radius > 16)
        return fail(SEG_ERR_INVALID_ARG, "radius=%d not in [0, 16]", radius);
    if (f == out) return fail(SEG_ERR_INVALID_ARG, "out must not alias f");
    const int64_t n = (int64_t)H * W;
    k_box_mean<<<(unsigned)((n + kDomThreads - 1) / kDomThreads), kDomThreads, 0,
                 static_cast<cudaStream_t>(stream)>>>(f, H, W, ld, radius, out);
    SEG_LAUNCHED("k_box_mean");
    return SEG_OK;
}
