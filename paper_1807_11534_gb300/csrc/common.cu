// common.cu -- error reporting, workspace queries, the deterministic integer
// scan and FP64 partial-sum reduction shared by the other units.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "seg_internal.cuh"

namespace seg {

static thread_local char g_err[512] = "";

seg_status fail(seg_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

void clear_error() { g_err[0] = 0; }

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0, m = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
        n = m > 0 ? m : 1;
    }
    return n;
}

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---------------------------------------------------------- tracing, debug

static thread_local cudaStream_t t_stream = nullptr;
static thread_local void* t_ws = nullptr;
static thread_local int t_depth = 0;

bool debug_mode() {
    static const bool on = [] {
        const char* e = std::getenv("SEG_DEBUG");
        return e && e[0] && std::strcmp(e, "0") != 0;
    }();
    return on;
}

PhaseScope::PhaseScope(const char* name, void* stream, void* ws) {
    nvtxRangePushA(name);
    if (t_depth++ == 0) {
        t_stream = static_cast<cudaStream_t>(stream);
        t_ws = ws;
    }
}

PhaseScope::~PhaseScope() {
    if (--t_depth == 0) {
        t_stream = nullptr;
        t_ws = nullptr;
    }
    nvtxRangePop();
}

seg_status after_launch(const char* name) {
    if (!debug_mode()) return SEG_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(t_stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return SEG_OK;   // nothing may synchronise a stream under capture
    cudaError_t e = cudaStreamSynchronize(t_stream);
    if (e != cudaSuccess)
        return fail(SEG_ERR_CUDA, "%s: %s (debug check after the launch)", name, cudaGetErrorString(e));
    if (t_ws) {
        int st = 0;
        e = cudaMemcpy(&st, t_ws, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return fail(SEG_ERR_CUDA, "%s: reading the status word: %s", name, cudaGetErrorString(e));
        if (st != SEG_OK) {
            cudaMemsetAsync(t_ws, 0, sizeof(int), t_stream);
            return fail(st, "%s: device-side status %d after the launch (debug check)", name, st);
        }
    }
    return SEG_OK;
}

seg_status check_ws(void* ws, size_t ws_bytes, const WsLayout& L) {
    if (!ws) return fail(SEG_ERR_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 16) return fail(SEG_ERR_ALIGN, "workspace not 16-byte aligned");
    if (ws_bytes < L.total)
        return fail(SEG_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);
    return SEG_OK;
}

// ------------------------------------------------------------------- scan

constexpr int kScanThreads = 256;
constexpr int kScanPer = kScanItems / kScanThreads;

// Block-level exclusive scan of kScanItems consecutive items; block totals to
// sums[blockIdx.x].
__global__ void k_scan_block(const int* __restrict__ in, int* __restrict__ out, int64_t n,
                             int* __restrict__ sums) {
    __shared__ int s_warp[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanItems + (int64_t)threadIdx.x * kScanPer;
    int v[kScanPer];
    int loc = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        loc += v[k];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = loc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int x = (lane < kScanThreads / 32) ? s_warp[lane] : 0;
        int y = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, y, d);
            if (lane >= d) y += t;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = y - x;   // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1) sums[blockIdx.x] = y;
    }
    __syncthreads();
    int run = s_warp[wid] + inc - loc;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

__global__ void k_scan_add(int* __restrict__ out, int64_t n, const int* __restrict__ offs) {
    int64_t base = (int64_t)blockIdx.x * kScanItems;
    int add = offs[blockIdx.x];
    for (int k = threadIdx.x; k < kScanItems; k += blockDim.x)
        if (base + k < n) out[base + k] += add;
}

__global__ void k_copy_total(const int* __restrict__ sums, int* __restrict__ total) {
    *total = sums[0];
}

seg_status scan_exclusive(const int* in, int* out, int64_t n, int* total, int* tmp,
                          cudaStream_t s) {
    if (n <= 0) {
        SEG_TRY_CUDA(cudaMemsetAsync(total, 0, sizeof(int), s));
        return SEG_OK;
    }
    int64_t nb = (n + kScanItems - 1) / kScanItems;
    int* sums = tmp;
    k_scan_block<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    SEG_LAUNCHED("k_scan_block");
    if (nb == 1) {
        k_copy_total<<<1, 1, 0, s>>>(sums, total);
        SEG_LAUNCHED("k_copy_total");
        return SEG_OK;
    }
    // scan the block sums in place, then add them back
    SEG_TRY(scan_exclusive(sums, sums, nb, total, tmp + nb + 1, s));
    k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, sums);
    SEG_LAUNCHED("k_scan_add");
    return SEG_OK;
}

// ------------------------------------------------------- FP64 reductions

__global__ void k_reduce_partials(const double* __restrict__ red, int nblk, int terms,
                                  double* __restrict__ out) {
    // one block; thread t owns blocks t, t+256, ... (fixed order), then a
    // fixed binary tree in shared memory
    __shared__ double s[256];
    for (int term = 0; term < terms; ++term) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblk; b += 256) acc += red[(int64_t)b * terms + term];
        s[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[term] = s[0];
        __syncthreads();
    }
}

seg_status reduce_partials(const double* red, int nblk, int terms, double* out, cudaStream_t s) {
    k_reduce_partials<<<1, 256, 0, s>>>(red, nblk, terms, out);
    SEG_LAUNCHED("k_reduce_partials");
    return SEG_OK;
}

}  // namespace seg

// ---------------------------------------------------------------- C ABI

extern "C" int seg_version(void) { return 100; }

extern "C" const char* seg_last_error(void) { return seg::g_err; }

extern "C" unsigned long long seg_launch_count(void) { return seg::g_launches.load(); }

extern "C" size_t seg_workspace_bytes(int H, int W, int ld, int tile_h) {
    (void)ld;
    if (H <= 0 || W <= 0 || tile_h <= 0) return 256;
    return seg::ws_layout(H, W, tile_h).total;
}

namespace seg {
__global__ void k_set_wait_limit(WsHeader* h, long long wait_cycles, unsigned extra) {
    h->wait_cycles = wait_cycles;
    h->bar_extra = extra;
}
}  // namespace seg

extern "C" seg_status seg_set_wait_limit(void* ws, size_t ws_bytes, long long wait_cycles,
                                         int extra_arrivals, void* stream) {
    seg::clear_error();
    seg::PhaseScope _scope("seg_set_wait_limit", stream, ws);
    if (!ws || ws_bytes < 256) return seg::fail(SEG_ERR_WORKSPACE, "workspace missing");
    if (wait_cycles < 0 || extra_arrivals < 0)
        return seg::fail(SEG_ERR_INVALID_ARG, "wait_cycles and extra_arrivals must be >= 0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    seg::k_set_wait_limit<<<1, 1, 0, s>>>(static_cast<seg::WsHeader*>(ws), wait_cycles,
                                           (unsigned)extra_arrivals);
    SEG_LAUNCHED("k_set_wait_limit");
    return SEG_OK;
}

extern "C" seg_status seg_read_status(void* ws, size_t ws_bytes, void* stream) {
    seg::clear_error();
    if (!ws || ws_bytes < 256) return seg::fail(SEG_ERR_WORKSPACE, "workspace missing");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = 0;
    SEG_TRY_CUDA(cudaMemcpyAsync(&st, ws, sizeof(int), cudaMemcpyDeviceToHost, s));
    SEG_TRY_CUDA(cudaStreamSynchronize(s));
    SEG_TRY_CUDA(cudaMemsetAsync(ws, 0, sizeof(int), s));
    if (st != SEG_OK) {
        const char* what = st == SEG_ERR_NONFINITE ? "fitting term holds NaN or Inf"
                         : st == SEG_ERR_CAPACITY  ? "an output buffer overflowed"
                         : st == SEG_ERR_TIMEOUT   ? "a device-side wait timed out"
                                                   : "device-side error";
        return seg::fail(st, "%s", what);
    }
    return SEG_OK;
}
