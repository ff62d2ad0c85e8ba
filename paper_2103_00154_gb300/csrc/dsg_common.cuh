// Internal helpers of libdsg: status plumbing, device-memory pool, warp/block
// primitives and a bounded grid barrier for the persistent round loops.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/dsg.h"

// ---------------------------------------------------------------- host side

namespace dsg {

// Thread-local message of the last failing call.
void set_error(const char* fmt, ...);
void clear_error();

#define DSG_TRY_CUDA(expr)                                                                        \
    do {                                                                                          \
        cudaError_t _e = (expr);                                                                  \
        if (_e != cudaSuccess) {                                                                  \
            ::dsg::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__,   \
                             __LINE__);                                                           \
            return _e == cudaErrorMemoryAllocation ? DSG_ENOMEM : DSG_ECUDA;                      \
        }                                                                                         \
    } while (0)

#define DSG_CHECK_ARG(cond, msg)                   \
    do {                                           \
        if (!(cond)) {                             \
            ::dsg::set_error("invalid argument: %s", msg); \
            return DSG_EINVAL;                     \
        }                                          \
    } while (0)

// Stream-ordered allocation from a per-device pool that keeps its memory
// between calls (release threshold = max), so repeated solves do not go back
// to the driver.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t dev_free(void* p, cudaStream_t s);

// True when p is device (or managed) memory of the current device.
bool is_device_ptr(const void* p);

// Copy that works for any host/device combination (UVA).
cudaError_t copy_any(void* dst, const void* src, size_t bytes, cudaStream_t s);

// Device properties cached per device.
struct DevInfo {
    int device = -1;
    int sms = 0;
    size_t l2_bytes = 0;
};
const DevInfo& dev_info();

// Upper bound on device-side waits (ns); 0 = library default.
uint64_t wait_limit_ns();

// Error bits written by kernels into their control block.
enum : uint32_t {
    ERR_TIMEOUT = 1u,   // a bounded wait ran out
    ERR_RANGE = 2u,     // an index out of range was seen (input validation)
    ERR_CAPACITY = 4u,  // an internal list would have overflowed
};

dsg_status status_from_err(uint32_t err, const char* what);

// RAII list of stream-ordered allocations released on scope exit.
struct Scratch {
    cudaStream_t s;
    void* ptrs[32];
    int n = 0;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (int i = 0; i < n; ++i) dev_free(ptrs[i], s);
    }
    template <class T>
    cudaError_t get(T** p, size_t count) {
        void* q = nullptr;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        cudaError_t e = dev_alloc(&q, (bytes + 255) & ~size_t(255), s);
        if (e != cudaSuccess) return e;
        ptrs[n++] = q;
        *p = static_cast<T*>(q);
        return cudaSuccess;
    }
};

}  // namespace dsg

// The graph object behind the opaque handle.
struct dsg_graph {
    uint32_t n = 0;
    uint64_t m = 0;          // undirected edges; off[n] == 2m
    uint64_t* off = nullptr; // device, n+1
    uint32_t* adj = nullptr; // device, 2m
    bool owns = true;        // library allocated off/adj
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t max_blocks = 0; // cap on the grid of persistent kernels for this handle (0: whole GPU)
    uint32_t force_block = 0; // block size of those kernels regardless of tuning (0: tuned)
    bool no_tail = false;     // core numbers: keep every level in the grid-wide kernel
};

// -------------------------------------------------------------- device side

namespace dsg {

constexpr uint32_t kFullMask = 0xffffffffu;

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t warp_id() { return threadIdx.x >> 5; }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFullMask, v, o));
    return v;
}

// Inclusive warp scan.
template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(kFullMask, v, o);
        if (lane_id() >= (uint32_t)o) v += t;
    }
    return v;
}

// Block-wide exclusive scan; every thread of the block must call it.
// `tmp` needs 33 slots of shared memory.  Returns the thread's exclusive
// prefix; *total receives the block sum.
template <class T>
__device__ __forceinline__ T block_excl_scan(T v, T* tmp, T* total) {
    T inc = warp_incl_scan(v);
    if (lane_id() == 31) tmp[warp_id()] = inc;
    __syncthreads();
    if (warp_id() == 0) {
        uint32_t nw = (blockDim.x + 31) >> 5;
        T w = lane_id() < nw ? tmp[lane_id()] : T(0);
        T wi = warp_incl_scan(w);
        tmp[lane_id()] = wi - w;  // exclusive warp offsets
        if (lane_id() == 31) tmp[32] = wi;
    }
    __syncthreads();
    T res = tmp[warp_id()] + inc - v;
    *total = tmp[32];
    __syncthreads();
    return res;
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T* tmp) {
    v = warp_sum(v);
    if (lane_id() == 0) tmp[warp_id()] = v;
    __syncthreads();
    T r = 0;
    if (warp_id() == 0) {
        uint32_t nw = (blockDim.x + 31) >> 5;
        r = lane_id() < nw ? tmp[lane_id()] : T(0);
        r = warp_sum(r);
        if (lane_id() == 0) tmp[32] = r;
    }
    __syncthreads();
    r = tmp[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t block_min_u32(uint32_t v, uint32_t* tmp) {
    v = warp_min(v);
    if (lane_id() == 0) tmp[warp_id()] = v;
    __syncthreads();
    if (warp_id() == 0) {
        uint32_t nw = (blockDim.x + 31) >> 5;
        uint32_t r = lane_id() < nw ? tmp[lane_id()] : 0xffffffffu;
        r = warp_min(r);
        if (lane_id() == 0) tmp[32] = r;
    }
    __syncthreads();
    uint32_t r = tmp[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const unsigned long long* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
    return *reinterpret_cast<const volatile uint64_t*>(p);
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a co-resident (cooperative) grid.  One counter word,
// zero at launch.  Block 0 adds 2^31 - (nblocks - 1), every other block adds
// 1, so the top bit flips exactly when the last block arrives and the low
// bits return to zero -- no reset is needed between uses.  The wait is
// bounded: after `limit_ns` the block records ERR_TIMEOUT in *err and the
// call returns false (all blocks then leave the kernel).  A block that sees
// *err already set stops waiting too.
__device__ __forceinline__ bool grid_barrier(uint32_t* bar, uint32_t* err, uint64_t limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t add = blockIdx.x == 0 ? (0x80000000u - (gridDim.x - 1)) : 1u;
        __threadfence();
        uint32_t old = atomicAdd(bar, add);
        int ok = 1;
        const uint64_t t0 = global_ns();
        uint32_t polls = 0;
        while (((old ^ ld_acquire_u32(bar)) & 0x80000000u) == 0) {
            if ((++polls & 31u) == 0) {
                if (global_ns() - t0 > limit_ns) { atomicOr(err, ERR_TIMEOUT); ok = 0; break; }
                if (ld_volatile_u32(err) & ERR_TIMEOUT) { ok = 0; break; }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Wait (one thread) until *flag != 0, at most limit_ns; on time-out record
// ERR_TIMEOUT in *err and return false.
__device__ __forceinline__ bool wait_flag(const uint32_t* flag, uint32_t* err, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    uint32_t polls = 0;
    while (ld_acquire_u32(flag) == 0) {
        if ((++polls & 31u) == 0 && global_ns() - t0 > limit_ns) {
            atomicOr(err, ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Mask of the lanes below this one.
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace dsg
