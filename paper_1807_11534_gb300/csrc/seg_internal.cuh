// seg_internal.cuh -- internals shared by the libseg translation units:
// error reporting, the workspace layout, storage-type converters and small
// device helpers.  Nothing here is visible through the C ABI (include/seg.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "seg.h"

namespace seg {

// ------------------------------------------------------------------ errors

// Records `msg` as the thread-local last error and returns `st`.
seg_status fail(seg_status st, const char* fmt, ...);
void clear_error();

#define SEG_TRY_CUDA(expr)                                                           \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess)                                                       \
            return ::seg::fail(SEG_ERR_CUDA, "%s: %s (%s:%d)", #expr,                \
                               cudaGetErrorString(_e), __FILE__, __LINE__);          \
    } while (0)

#define SEG_TRY(expr)                                                                \
    do {                                                                             \
        seg_status _s = (expr);                                                      \
        if (_s != SEG_OK) return _s;                                                 \
    } while (0)

// Host-side count of kernel launches issued by the library (diagnostics).
void count_launch();

// Streaming multiprocessors of the current device (queried once).
int sm_count();

// One public call: an NVTX range named after it for its launches, and the
// stream and workspace that the debug mode's checks use (see after_launch).
struct PhaseScope {
    PhaseScope(const char* name, void* stream, void* ws);
    ~PhaseScope();
    PhaseScope(const PhaseScope&) = delete;
    PhaseScope& operator=(const PhaseScope&) = delete;
};

// Debug mode (SEG_DEBUG=1 in the environment, read once): after every launch
// of a public call, unless its stream is being captured into a graph, the
// stream is synchronised, and a CUDA error or a device-side status recorded
// in the call's workspace is returned by that call, with the name of the
// launch that raised it.  Off: returns SEG_OK at once.
seg_status after_launch(const char* name);
bool debug_mode();

// Checks the launch that was just issued.
#define SEG_LAUNCHED(name)                                                           \
    do {                                                                             \
        ::seg::count_launch();                                                       \
        cudaError_t _e = cudaGetLastError();                                         \
        if (_e != cudaSuccess)                                                       \
            return ::seg::fail(SEG_ERR_CUDA, "launch of %s failed: %s", name,        \
                               cudaGetErrorString(_e));                              \
        if (::seg::debug_mode()) SEG_TRY(::seg::after_launch(name));                \
    } while (0)

// -------------------------------------------------------------- workspace

// Device-side header at the start of every workspace.
struct WsHeader {
    int status;          // first device-side error (SEG_OK when none)
    int done;            // set by the stopping test; step kernels then return at once
    int iters_done;      // iteration at which the stopping test fired
    int last_check;      // iteration of the last stopping test
    double c[2];         // c1, c2 used by the fitting term
    double du2, dv2;     // last ||u^l - u^(l-1)||^2, ||v^l - v^(l-1)||^2
    unsigned long long d2max;   // largest squared marker distance (Eq. DS)
    float delta;         // domain threshold in use
    unsigned int qprefix;       // radix-select prefix (quantile mode)
    long long qk;        // rank still to find (quantile mode)
    long long qk0;       // rank asked for, k = ceil(q n)
    int n_fg;            // fixed foreground pixels
    // temporally blocked solver: window tickets of the last four sweeps and
    // the ping-pong buffer that holds the final state
    int tb_ticket[4];
    int tb_buf;
    int n_smem_blocks;   // compact solver: blocks that held their state in shared memory
    int n_h1_blocks;     // compact solver: blocks that ran one grid barrier per iteration
    unsigned h1_vote;    // compact solver: blocks whose one-barrier state did not fit (a vote)
    long long wait_cycles;   // bound of every device-side wait, SM clock cycles (0: kWaitCycles);
                             // set by seg_set_wait_limit, kept across solves
    // grid barrier of the persistent solvers: monotonic arrival counter, on
    // its own cache line
    alignas(128) unsigned bar_count;
    unsigned bar_extra;  // arrivals a grid barrier waits for beyond the launch's blocks: 0,
                         // except to test the timeout path (seg_set_wait_limit); the
                         // counter starts at -bar_extra instead of 0
};
static_assert(sizeof(WsHeader) <= 256, "header must fit its slot");

__device__ __forceinline__ unsigned atom_add_release_gpu(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr int kScanItems = 1024;        // items per block of the exclusive scan
constexpr int kHistBins = 256;          // radix-select digit bins (8 bits per pass)
constexpr int kReduceBlocks = 1024;     // fixed grid of deterministic FP64 reductions
constexpr int kEnergyTerms = 8;
constexpr int kEnergyBlockThreads = 256;  // block size of the energy / error kernels

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The stopping-test interval a solve runs with.  Without a tolerance
// (tol <= 0) no test decides anything and only the last test's norms are
// reported, so only the last iteration is tested.
inline int test_interval(double tol, int check_every, int iters) {
    return tol > 0.0 ? (check_every > 1 ? check_every : 1) : (iters > 1 ? iters : 1);
}

// Byte offsets of the workspace regions for one image geometry.
struct WsLayout {
    size_t header, tile_cnt, tile_flag, tile_start, tile_pos, scan_tmp, partials,
        hist, red, total;
    int64_t ntiles;
    int64_t scan_tmp_items;
    int64_t npartials;      // stopping-test partial pairs the workspace holds
};

inline int64_t scan_tmp_items_for(int64_t n) {
    int64_t tot = 0;
    while (n > 1) {
        n = (n + kScanItems - 1) / kScanItems;
        tot += n + 1;
    }
    return tot + 2;
}

// Geometry-independent regions come first so that calls that need only
// them (fitting, energy) accept any workspace sized for the image.
constexpr size_t kWsHeaderOff = 0;
constexpr size_t kWsRedOff = 256;
constexpr size_t kWsHistOff = kWsRedOff + 8 * (size_t)kReduceBlocks * kEnergyTerms;
constexpr size_t kWsBatchOff = kWsHistOff + 4 * (size_t)kHistBins;   // compact bases of a batch
constexpr size_t kWsFixedBytes = kWsBatchOff + 4 * (size_t)(128 + 2 + 2);

inline WsLayout ws_layout(int H, int W, int tile_h) {
    WsLayout L{};
    int64_t nty = (H + tile_h - 1) / tile_h, ntx = (W + 31) / 32;
    L.ntiles = nty * ntx;
    L.scan_tmp_items = scan_tmp_items_for(L.ntiles);
    L.header = kWsHeaderOff;
    L.red = kWsRedOff;
    L.hist = kWsHistOff;
    size_t o = align_up(kWsFixedBytes, 256);
    L.tile_cnt = o;   o = align_up(o + 4 * (size_t)(L.ntiles + 1), 256);
    L.tile_flag = o;  o = align_up(o + 4 * (size_t)(L.ntiles + 1), 256);
    L.tile_start = o; o = align_up(o + 4 * (size_t)(L.ntiles + 1), 256);
    L.tile_pos = o;   o = align_up(o + 4 * (size_t)(L.ntiles + 1), 256);
    L.scan_tmp = o;   o = align_up(o + 4 * (size_t)L.scan_tmp_items, 256);
    // stopping-test partials: one pair per 60-column x (8 or more)-row warp
    // task (dense mode) or per block of the primal step (compact mode, at
    // most 4096 blocks)
    int64_t dense_tasks = (int64_t)((W + 59) / 60) * ((H + 7) / 8);
    L.npartials = dense_tasks > 4096 ? dense_tasks : 4096;
    L.partials = o;   o = align_up(o + 2 * 8 * (size_t)(L.npartials + 1), 256);
    L.total = o;
    return L;
}

template <typename T>
inline T* ws_at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

// Validates a workspace pointer/size for a geometry.
seg_status check_ws(void* ws, size_t ws_bytes, const WsLayout& L);

// ------------------------------------------------------ device utilities

__device__ __forceinline__ void record_status(WsHeader* h, int st) {
    atomicCAS(&h->status, SEG_OK, st);
}

__device__ __forceinline__ unsigned lanemask_lt(int b) { return (1u << b) - 1u; }

// 32-bit integer hash (the "lowbias32" finaliser of C. Wellons' hash-prospector,
// a published xorshift-multiply mixer); used as a counter-based generator.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352du;
    x ^= x >> 15; x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// storage-type converters (arithmetic is always float32).  16-bit stores use
// unbiased stochastic rounding with the random word `r`: a round-to-nearest
// store would drop every update smaller than half a unit in the last place,
// which stalls the fixed-point iteration long before it converges.
//
// vbias: v in [0, 1] is stored as v - vbias.  For the 16-bit types vbias = 0.5
// maps v to [-0.5, 0.5], where the unit in the last place is at most 2^-9
// (bf16) instead of up to 2^-7 near v = 1, and 0 and 1 stay exact.
template <typename T> struct Store;
template <> struct Store<float> {
    static constexpr float vbias = 0.0f;
    static __device__ __forceinline__ float ld(const float* p, int64_t i) { return __ldg(p + i); }
    // load of state that other blocks write during the kernel: a plain
    // (not read-only-path) load, ordered after their writes by the grid
    // barrier's acquire, which also discards stale L1 lines
    static __device__ __forceinline__ float ldc(const float* p, int64_t i) { return p[i]; }
    static __device__ __forceinline__ float ld_rw(const float* p, int64_t i) { return p[i]; }
    static __device__ __forceinline__ void st(float* p, int64_t i, float x) { p[i] = x; }
    // x rounded to the storage type (stochastically for 16-bit types, with
    // the random word r), as a float
    static __device__ __forceinline__ float sr(float x, uint32_t) { return x; }
    // stores x (stochastically rounded for 16-bit types) and returns the
    // value stored
    static __device__ __forceinline__ float st_sr(float* p, int64_t i, float x, uint32_t) { p[i] = x; return x; }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr float vbias = 0.5f;
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(__ldg(p + i)); }
    static __device__ __forceinline__ float ldc(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }
    static __device__ __forceinline__ float ld_rw(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, int64_t i, float x) { p[i] = __float2bfloat16_rn(x); }
    // bf16 keeps the top 16 bits of the float: adding a uniform 16-bit word to
    // the discarded bits before truncating rounds up with probability equal
    // to the discarded fraction (finite values; |x| <= 1 here)
    static __device__ __forceinline__ __nv_bfloat16 sr_t(float x, uint32_t r) {
        uint32_t b = __float_as_uint(x);
        b += r & 0xffffu;
        return __ushort_as_bfloat16((unsigned short)(b >> 16));
    }
    static __device__ __forceinline__ float sr(float x, uint32_t r) { return __bfloat162float(sr_t(x, r)); }
    static __device__ __forceinline__ float st_sr(__nv_bfloat16* p, int64_t i, float x, uint32_t r) {
        const __nv_bfloat16 y = sr_t(x, r);
        p[i] = y;
        return __bfloat162float(y);
    }
};
template <> struct Store<__half> {
    static constexpr float vbias = 0.5f;
    static __device__ __forceinline__ float ld(const __half* p, int64_t i) { return __half2float(__ldg(p + i)); }
    static __device__ __forceinline__ float ldc(const __half* p, int64_t i) { return __half2float(p[i]); }
    static __device__ __forceinline__ float ld_rw(const __half* p, int64_t i) { return __half2float(p[i]); }
    static __device__ __forceinline__ void st(__half* p, int64_t i, float x) { p[i] = __float2half_rn(x); }
    // round to one of the two neighbouring halves with probabilities given by
    // the distance to each
    static __device__ __forceinline__ __half sr_t(float x, uint32_t r) {
        __half lo = __float2half_rd(x), hi = __float2half_ru(x);
        float fl = __half2float(lo), fh = __half2float(hi);
        float u = (float)(r >> 8) * (1.0f / 16777216.0f);
        const bool up = fh > fl && u * (fh - fl) < x - fl;
        return up ? hi : lo;
    }
    static __device__ __forceinline__ float sr(float x, uint32_t r) { return __half2float(sr_t(x, r)); }
    static __device__ __forceinline__ float st_sr(__half* p, int64_t i, float x, uint32_t r) {
        const __half y = sr_t(x, r);
        p[i] = y;
        return __half2float(y);
    }
};

inline size_t storage_size(int storage) { return storage == SEG_STORE_F32 ? 4 : 2; }

// ------------------------------------------- TMA bulk copies and mbarriers

// Shared-memory address of a generic pointer into this CTA's shared memory.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the barrier initialisation visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic shared-memory accesses before later
// asynchronous-proxy accesses (a bulk copy refilling a buffer).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival on `bar` that also expects `bytes` of transaction completions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// Bulk (non-tensor) TMA copy global -> shared, completing on `bar`.  dst, src
// and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// Tiled TMA load of one 2-D box at (x, y) = (column, row) of the tensor
// described by `map` (a kernel parameter or global-memory descriptor) into
// shared memory, completing on `bar`.  x times the element size must be a
// multiple of 16 bytes; coordinates outside the tensor read as zero.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar)) : "memory");
}

// Orders this thread's earlier generic-proxy global accesses (and those it
// has acquired from other threads) before its later TMA accesses.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Default bound of a device-side wait: ~1 s of SM clock.  A workspace can
// set its own (WsHeader::wait_cycles).
constexpr long long kWaitCycles = 2000000000LL;
__device__ __forceinline__ long long wait_budget(const WsHeader* h) {
    const long long c = h->wait_cycles;
    return c > 0 ? c : kWaitCycles;
}

// Waits for phase `parity` of `bar` for at most the workspace's wait bound;
// returns false (after recording SEG_ERR_TIMEOUT) when the wait runs out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, WsHeader* h) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64(), budget = wait_budget(h);
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) {
            record_status(h, SEG_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// ---------------------------------------------------- internal launchers

// Exclusive scan of n int32 values (in may equal out); writes the total to
// *total (device).  Deterministic (integer adds in a fixed tree).
seg_status scan_exclusive(const int* in, int* out, int64_t n, int* total, int* tmp,
                          cudaStream_t s);

// Energy kernels (energy.cu), written for blocks of kEnergyBlockThreads
// threads: per-block FP64 partials of the six energy
// terms over a grid-stride loop, and the combination of their sums.
__global__ void k_energy_terms(const float* __restrict__ f, int H, int W, int ld,
                               const float* __restrict__ u, const float* __restrict__ v,
                               const float* __restrict__ p1, const float* __restrict__ p2,
                               double lambda, double* __restrict__ red);
__global__ void k_energy_final(const double* __restrict__ sums, double lambda, double theta,
                               double* out);

// Deterministic FP64 sum of `terms` interleaved partial arrays written by
// `nblk` blocks (red[k * terms + t]); writes sums to out[t].
seg_status reduce_partials(const double* red, int nblk, int terms, double* out, cudaStream_t s);

}  // namespace seg
