// Fault-detection probes: bounded device waits that are made to run out on
// purpose, so tests can check that a wait which never completes ends with
// DSG_ETIMEOUT and leaves the context usable.  Nothing here faults, traps or
// spins without a limit.
#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace dsg {

struct DebugCtl {
    uint32_t bar;
    uint32_t err;
    uint32_t flag;   // never set by anyone
    uint32_t passed; // blocks that got through
};

__global__ void debug_wait_flag_kernel(DebugCtl* c, uint64_t limit_ns) {
    if (threadIdx.x == 0 && wait_flag(&c->flag, &c->err, limit_ns)) atomicAdd(&c->passed, 1u);
}

// Every block but the last one enters a grid barrier; the last one leaves
// early, so the barrier can never complete and the waiters must time out.
__global__ void debug_straggler_kernel(DebugCtl* c, uint64_t limit_ns) {
    if (blockIdx.x == gridDim.x - 1) return;
    if (grid_barrier(&c->bar, &c->err, limit_ns) && threadIdx.x == 0) atomicAdd(&c->passed, 1u);
}

static dsg_status run_debug(int which, uint64_t limit_ns) {
    cudaStream_t s = nullptr;
    Scratch sc(s);
    DebugCtl* c;
    DSG_TRY_CUDA(sc.get(&c, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(c, 0, sizeof(DebugCtl), s));
    if (which == 0) {
        debug_wait_flag_kernel<<<1, 32, 0, s>>>(c, limit_ns);
        DSG_TRY_CUDA(cudaGetLastError());
    } else {
        void* params[] = {&c, &limit_ns};
        DSG_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)debug_straggler_kernel, dim3(2), dim3(32), params, 0, s));
    }
    DebugCtl h;
    DSG_TRY_CUDA(cudaMemcpyAsync(&h, c, sizeof(h), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    if (h.passed) {
        set_error("debug wait: a wait that cannot complete reported success");
        return DSG_ECUDA;
    }
    return status_from_err(h.err, which == 0 ? "debug flag wait" : "debug straggler barrier");
}

// Random 4-byte accesses over a words-long array: mode 0 plain loads, 1
// reductions (no return), 2 atomics returning the old value.  Addresses come
// from a multiplicative hash of the op index.
__global__ void random_access_kernel(uint32_t* a, uint32_t words, uint64_t ops, int mode, uint32_t* sink) {
    uint32_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ops; i += stride) {
        uint32_t h = (uint32_t)((i * 0x9E3779B97F4A7C15ull) >> 32);
        uint32_t idx = (uint32_t)(((uint64_t)h * words) >> 32);
        if (mode == 0) acc += a[idx];
        else if (mode == 1) atomicAdd(&a[idx], 1u);
        else acc += atomicAdd(&a[idx], 1u);
    }
    if (acc == 0x12345678u) *sink = acc;
}

__global__ void barrier_loop_kernel(DebugCtl* c, uint32_t iters, uint64_t limit_ns) {
    for (uint32_t i = 0; i < iters; ++i)
        if (!grid_barrier(&c->bar, &c->err, limit_ns)) return;
}

}  // namespace dsg

using namespace dsg;

// Throughput (10^9 ops/s) of random 4-byte accesses to a `words`-long array.
extern "C" dsg_status dsg_debug_random_access(uint32_t words, uint64_t ops, int mode, double* gops) {
    clear_error();
    DSG_CHECK_ARG(gops && words > 0 && mode >= 0 && mode <= 2, "arguments");
    cudaStream_t s = nullptr;
    Scratch sc(s);
    uint32_t *a, *sink;
    DSG_TRY_CUDA(sc.get(&a, words));
    DSG_TRY_CUDA(sc.get(&sink, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(a, 0, (size_t)words * 4, s));
    uint32_t grid = (uint32_t)dev_info().sms * 8;
    random_access_kernel<<<grid, 256, 0, s>>>(a, words, ops / 8, mode, sink);  // warm-up
    cudaEvent_t e0, e1;
    DSG_TRY_CUDA(cudaEventCreate(&e0));
    DSG_TRY_CUDA(cudaEventCreate(&e1));
    DSG_TRY_CUDA(cudaEventRecord(e0, s));
    random_access_kernel<<<grid, 256, 0, s>>>(a, words, ops, mode, sink);
    DSG_TRY_CUDA(cudaEventRecord(e1, s));
    DSG_TRY_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *gops = (double)ops / ((double)ms * 1e6);
    return DSG_OK;
}

// Grid-barrier latency of a co-resident grid of `block`-thread blocks,
// blocks_per_sm per SM (0 = as many as fit): average ns per barrier over
// `iters` barriers, timed with CUDA events.
extern "C" dsg_status dsg_debug_barrier_ns(uint32_t block, uint32_t blocks_per_sm, uint32_t iters, double* ns,
                                           uint32_t* grid_out) {
    clear_error();
    DSG_CHECK_ARG(ns && iters > 0 && iters <= 1000000, "ns / iters");
    DSG_CHECK_ARG(block >= 32 && block <= 1024 && block % 32 == 0, "block");
    cudaStream_t s = nullptr;
    Scratch sc(s);
    DebugCtl* c;
    DSG_TRY_CUDA(sc.get(&c, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(c, 0, sizeof(DebugCtl), s));
    int per_sm = 0;
    DSG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_loop_kernel, (int)block, 0));
    if (blocks_per_sm && (int)blocks_per_sm < per_sm) per_sm = (int)blocks_per_sm;
    uint32_t grid = (uint32_t)per_sm * (uint32_t)dev_info().sms;
    uint64_t lim = wait_limit_ns();
    void* params[] = {&c, &iters, &lim};
    cudaEvent_t e0, e1;
    DSG_TRY_CUDA(cudaEventCreate(&e0));
    DSG_TRY_CUDA(cudaEventCreate(&e1));
    DSG_TRY_CUDA(cudaEventRecord(e0, s));
    DSG_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)barrier_loop_kernel, dim3(grid), dim3(block), params, 0, s));
    DSG_TRY_CUDA(cudaEventRecord(e1, s));
    DSG_TRY_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    DebugCtl h;
    DSG_TRY_CUDA(cudaMemcpy(&h, c, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.err) return status_from_err(h.err, "barrier loop");
    *ns = (double)ms * 1e6 / iters;
    if (grid_out) *grid_out = grid;
    return DSG_OK;
}

extern "C" dsg_status dsg_debug_wait_timeout(uint32_t which, uint64_t limit_ns) {
    clear_error();
    DSG_CHECK_ARG(which <= 1, "which must be 0 (flag) or 1 (barrier)");
    DSG_CHECK_ARG(limit_ns > 0 && limit_ns <= 10ull * 1000 * 1000 * 1000, "limit_ns must be in (0, 10 s]");
    return run_debug((int)which, limit_ns);
}
