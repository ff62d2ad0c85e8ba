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

}  // namespace dsg

using namespace dsg;

extern "C" dsg_status dsg_debug_wait_timeout(uint32_t which, uint64_t limit_ns) {
    clear_error();
    DSG_CHECK_ARG(which <= 1, "which must be 0 (flag) or 1 (barrier)");
    DSG_CHECK_ARG(limit_ns > 0 && limit_ns <= 10ull * 1000 * 1000 * 1000, "limit_ns must be in (0, 10 s]");
    return run_debug((int)which, limit_ns);
}
