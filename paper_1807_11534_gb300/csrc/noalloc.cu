// noalloc.cu -- seg_energy_noalloc: the energy / duality-gap evaluation of
// seg_energy for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc or any allocating
// routine: code that runs while a CUDA stream is being captured into a graph
// (allocation is not a capturable operation), host applications that hand
// the library a fixed memory budget and forbid further device allocation,
// and latency-critical loops where an allocation would synchronise the
// device.  Such callers cannot provide the workspace seg_energy needs for its
// per-block partial sums.  This entry point takes the same inputs and output
// and keeps its scratch in a file-scope device array instead.
//
// Scratch: g_energy_scratch holds the per-block FP64 partials of the six
// energy terms for up to kNoAllocMaxBlocks blocks plus their sums, 196,672
// bytes in all.  Every GPU that loads the library holds this array until the
// process exits.  Each block covers at most kNoAllocPixPerBlock pixels, so
// the largest image accepted is kNoAllocMaxBlocks * kNoAllocPixPerBlock =
// 33,554,432 pixels (e.g. 5792 x 5792); larger images are rejected with
// SEG_ERR_CAPACITY.  Every slot the call reads is written earlier in the same
// call, so nothing has to be cleared between calls; the array keeps the last
// call's partials.  All calls share the one array: calls whose kernels
// overlap on the GPU (on different streams, or from different threads without
// ordering) race on it and may return wrong sums.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress while that device is current and caches it; that
// first call should therefore be made before any stream capture begins.  The
// name g_energy_scratch in host code is only a host-side stand-in, never a
// device address, which is why the looked-up address is what the kernels get.
#include <mutex>

#include "seg_internal.cuh"

namespace seg {

constexpr int kNoAllocMaxBlocks = 4096;
constexpr int64_t kNoAllocPixPerBlock = 8192;
constexpr int kNoAllocTerms = 6;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_energy_scratch[kNoAllocMaxBlocks * kNoAllocTerms + 8];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of g_energy_scratch on the current device (looked up once).
static seg_status noalloc_scratch(double** out) {
    int dev = 0;
    SEG_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(SEG_ERR_INVALID_ARG, "device %d beyond the %d devices supported", dev,
                    kNoAllocMaxDevices);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_energy_scratch);
        if (e != cudaSuccess || !p)
            return fail(SEG_ERR_CUDA, "cudaGetSymbolAddress(g_energy_scratch) on device %d: %s", dev,
                        cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return SEG_OK;
}

}  // namespace seg

using namespace seg;

extern "C" seg_status seg_energy_noalloc(const float* f, int H, int W, int ld, const float* u,
                                         const float* v, const float* p1, const float* p2,
                                         double lambda, double theta, double* out, void* stream) {
    clear_error();
    PhaseScope _scope("seg_energy_noalloc", stream, nullptr);
    if (!f || !u || !v || !p1 || !p2 || !out)
        return fail(SEG_ERR_INVALID_ARG, "a required pointer is NULL");
    if (H <= 0 || W <= 0 || ld < W)
        return fail(SEG_ERR_INVALID_ARG, "bad image size H=%d W=%d ld=%d", H, W, ld);
    if (ld % 32) return fail(SEG_ERR_ALIGN, "ld=%d is not a multiple of 32", ld);
    if (!(theta > 0)) return fail(SEG_ERR_INVALID_ARG, "theta must be > 0");
    const int64_t n = (int64_t)H * W;
    const int64_t max_pixels = (int64_t)kNoAllocMaxBlocks * kNoAllocPixPerBlock;
    if (n > max_pixels)
        return fail(SEG_ERR_CAPACITY,
                    "seg_energy_noalloc: %lld pixels exceed its fixed scratch limit of %lld pixels "
                    "(use seg_energy with a workspace)",
                    (long long)n, (long long)max_pixels);
    double* scratch = nullptr;
    SEG_TRY(noalloc_scratch(&scratch));
    const int blocks = (int)((n + kNoAllocPixPerBlock - 1) / kNoAllocPixPerBlock);
    double* red = scratch;
    double* sums = scratch + (size_t)kNoAllocMaxBlocks * kNoAllocTerms;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_energy_terms<<<blocks, kEnergyBlockThreads, 0, s>>>(f, H, W, ld, u, v, p1, p2, lambda, red);
    SEG_LAUNCHED("k_energy_terms");
    SEG_TRY(reduce_partials(red, blocks, kNoAllocTerms, sums, s));
    k_energy_final<<<1, 1, 0, s>>>(sums, lambda, theta, out);
    SEG_LAUNCHED("k_energy_final");
    return SEG_OK;
}
