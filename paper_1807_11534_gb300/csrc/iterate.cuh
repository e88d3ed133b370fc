// iterate.cuh -- pieces of one outer iteration of Sections 2.1 and 3 shared
// by the solvers of solve.cu (dense, compact) and tiled.cu (temporally
// blocked): the scalar parameters, the fixed-point update of p, and the
// bounded grid-wide barrier of the persistent kernels.
#pragma once

#include "seg_internal.cuh"

namespace seg {

struct IterParams {
    float theta, inv_theta, tau, theta_lambda;
    int H, W, ld, nw, ntx, th;
    uint32_t seed;   // per-launch seed of the stochastic rounding of 16-bit stores
};

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

// p' = (p + tau g) / (1 + tau |g|); |g| through the hardware reciprocal square
// root and the quotient through the fast divide (a few ulp; the iteration is
// checked against the FP64 oracle to 1e-4).
__device__ __forceinline__ void chambolle_update(float p1, float p2, float g1, float g2, float tau,
                                                 float& q1, float& q2) {
    const float s = fmaf(g1, g1, g2 * g2);
    const float nrm = s > 0.f ? s * rsqrtf(s) : 0.f;
    const float r = __fdividef(1.0f, fmaf(tau, nrm, 1.0f));
    q1 = fmaf(tau, g1, p1) * r;
    q2 = fmaf(tau, g2, p2) * r;
}

// ------------------------------------------------ persistent kernels

// Grid-wide barrier on a monotonic arrival counter, with a bounded wait:
// thread 0 of each block adds 1 with a release reduction (no round trip) and
// polls the counter with acquire loads until it reaches nblocks x `gen` (the
// block's count of barriers passed, tracked in a register; the counter is
// reset before each persistent launch).  Returns false after recording
// SEG_ERR_TIMEOUT (and raising the done flag) if the others do not arrive
// within the workspace's wait bound (~1 s by default).
__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Split form of the barrier: grid_arrive after the block's writes (a block
// barrier, then thread 0's release reduction; returns the new generation),
// grid_wait before reading what other blocks wrote.  Work that only reads
// this block's own writes may run in between.
__device__ __forceinline__ void grid_arrive(WsHeader* h, unsigned& gen) {
    __syncthreads();
    ++gen;
    if (threadIdx.x == 0) red_add_release_gpu(&h->bar_count, 1u);
}

// poll: thread 0 also reads the done flag after the barrier and the block
// gets it in `done` (one load per block instead of one per warp on a single
// line).
__device__ __forceinline__ bool grid_wait(WsHeader* h, unsigned nblocks, unsigned gen, bool poll,
                                          bool& done) {
    __shared__ int s_ok, s_done;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = nblocks * gen;
        // the wait bound is read only when the first poll fails, so the
        // block that completes the barrier pays no extra load
        if ((int)(ld_acquire_gpu(&h->bar_count) - target) < 0) {
            const long long t0 = clock64(), budget = wait_budget(h);
            while ((int)(ld_acquire_gpu(&h->bar_count) - target) < 0) {
                if (clock64() - t0 > budget) {
                    record_status(h, SEG_ERR_TIMEOUT);
                    h->done = 1;
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
        if (poll) s_done = *(volatile int*)&h->done;
    }
    __syncthreads();
    done = poll && s_done != 0;
    return s_ok != 0;
}

__device__ __forceinline__ bool grid_wait(WsHeader* h, unsigned nblocks, unsigned gen) {
    bool d;
    return grid_wait(h, nblocks, gen, false, d);
}

__device__ __forceinline__ bool grid_sync(WsHeader* h, unsigned nblocks, unsigned& gen) {
    grid_arrive(h, gen);
    return grid_wait(h, nblocks, gen);
}

__device__ __forceinline__ bool grid_sync_poll(WsHeader* h, unsigned nblocks, unsigned& gen, bool poll,
                                               bool& done) {
    grid_arrive(h, gen);
    return grid_wait(h, nblocks, gen, poll, done);
}

// Stopping-test sums (Section 4), deterministic and with no FP64 work in the
// block (FP64 is a narrow pipe on this part, and every block reduces at every
// test):
//  * block_sum2f: the FP32 sums of (x, y) over a block of NT threads, a warp
//    shuffle tree, the warp sums staged in shared memory (s_red, 64 floats),
//    then one shuffle tree over them; the totals land in every thread;
//  * sum_partials_warp0: the FP64 sum of n (x, y) pairs written by the
//    blocks, in a fixed order by warp 0 (lane l adds pairs l, l + 32, ...,
//    then a shuffle tree); returns the totals in lane 0 of warp 0.
// All threads of the block must call block_sum2f.
template <int NT>
__device__ __forceinline__ void block_sum2f(float& x, float& y, float* s_red) {
    const unsigned FULL = 0xffffffffu;
    for (int d = 16; d > 0; d >>= 1) {
        x += __shfl_down_sync(FULL, x, d);
        y += __shfl_down_sync(FULL, y, d);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();   // s_red may still be read from an earlier use
    if (lane == 0) { s_red[2 * wid] = x; s_red[2 * wid + 1] = y; }
    __syncthreads();
    if (wid == 0) {
        x = lane < NT / 32 ? s_red[2 * lane] : 0.f;
        y = lane < NT / 32 ? s_red[2 * lane + 1] : 0.f;
        for (int d = 16; d > 0; d >>= 1) {
            x += __shfl_down_sync(FULL, x, d);
            y += __shfl_down_sync(FULL, y, d);
        }
        if (lane == 0) { s_red[64] = x; s_red[65] = y; }
    }
    __syncthreads();
    x = s_red[64];
    y = s_red[65];
}

__device__ __forceinline__ void sum_partials_warp0(const double* part, int n, double& x, double& y) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    x = 0.0;
    y = 0.0;
    for (int k = lane; k < n; k += 32) {
        x += __ldcg(part + 2 * k);
        y += __ldcg(part + 2 * k + 1);
    }
    for (int d = 16; d > 0; d >>= 1) {
        x += __shfl_down_sync(FULL, x, d);
        y += __shfl_down_sync(FULL, y, d);
    }
}

// ------------------------------------------------ host helpers of solve.cu

// Reset of the solve's header words before a persistent solve, and the
// stats of the finished solve (see seg_solve): launched on stream s.
seg_status launch_solve_begin(WsHeader* h, cudaStream_t s);
seg_status launch_solve_end(const WsHeader* h, const int32_t* counts, int iters, double* stats,
                            cudaStream_t s);

// ------------------------------------------------ host entry of tiled.cu

// Temporally blocked solve on the dense ping-pong state `st` (initialised by
// the dense init kernel): all iterations in one cooperative launch, then the
// final p1, p2, v copied out (u is written by the solve itself).
seg_status run_tiled(const IterParams& P, const seg_params* prm, const uint32_t* act, const float* f,
                     float* u, float* v, float* p1, float* p2, float* st, double* partials, int64_t npartials,
                     WsHeader* h, cudaStream_t s);

// ------------------------------------------------ host entry of wide.cu

// One image solved in row-major compact order when its RD is too large for
// the shared-memory paths (wide.cu).  Every kernel of run_wide_rm returns at
// once unless counts[1] > wide_above, the condition under which the
// tile-major kernels of solve.cu return at once instead, so the choice is
// made on the device and survives graph capture.
struct RowMajorArgs {
    const uint32_t* act;     // RD bit plane [H][nw]
    const uint32_t* fg;      // f < 0 bit plane
    const float* f;          // [H][ld]
    float *u, *v, *p1, *p2;  // [H][ld]: warm-start input, result output
    const int32_t* counts;   // counts[1] = |RD|
    WsHeader* h;
    int H, W, ld, nw, ntx;
    float theta_lambda, inv_theta;
    long long wide_above;
    int32_t* rowstart;       // [H + 1] scratch: RD pixels before each row
};
struct RowMajorArrays {      // `cap` elements each, p and v in the storage type
    void *p1[2], *p2[2], *v;
    float *F, *U, *Up, *Wc;  // theta lambda f, u, u of the iteration before a test, w
    uint16_t *dd, *du, *fl;  // offsets to the rows below / above, neighbour flags
    long long cap;
};
seg_status run_wide_rm(const RowMajorArgs& R, const RowMajorArrays& A, const IterParams& P,
                       const seg_params* prm, double* partials, long long max_partials, cudaStream_t s);

// Number of windows of the tiled solve for an H x W image (validates sweep
// and n_inner).
seg_status tiled_geometry(int H, int W, int sweep, int n_inner, int* nwin);

// State bytes of the tiled solve: the six dense planes and the per-window
// RD lists.
size_t tiled_state_bytes(int H, int ld);

}  // namespace seg
