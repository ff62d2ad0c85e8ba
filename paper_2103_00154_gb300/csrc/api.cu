// Host side of the C ABI: status strings, last-error text, the device memory
// pool, and graph handles built from a CSR.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <unordered_map>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace dsg {

static thread_local char g_err[512];

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];
static bool g_pool_ready[64];

static cudaError_t pool_for(int dev, cudaMemPool_t* out) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_pool_ready[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t thr = UINT64_MAX;
        e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr);
        if (e != cudaSuccess) return e;
        g_pool_ready[dev] = true;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

// Caller-installed allocator (dsg_set_allocator); pointers it handed out are
// remembered so each goes back to the allocator that made it.
struct HookAlloc {
    dsg_alloc_fn alloc = nullptr;
    dsg_free_fn free = nullptr;
    void* ctx = nullptr;
};
static std::mutex g_hook_mu;
static HookAlloc g_hook;
static std::unordered_map<void*, HookAlloc>* g_hook_ptrs = nullptr;

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    HookAlloc h;
    {
        std::lock_guard<std::mutex> lk(g_hook_mu);
        h = g_hook;
    }
    if (h.alloc) {
        void* q = h.alloc(bytes, h.ctx, (void*)s);
        if (!q) return cudaErrorMemoryAllocation;
        std::lock_guard<std::mutex> lk(g_hook_mu);
        if (!g_hook_ptrs) g_hook_ptrs = new std::unordered_map<void*, HookAlloc>();
        (*g_hook_ptrs)[q] = h;
        *p = q;
        return cudaSuccess;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool;
    e = pool_for(dev, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t dev_free(void* p, cudaStream_t s) {
    if (!p) return cudaSuccess;
    HookAlloc h;
    {
        std::lock_guard<std::mutex> lk(g_hook_mu);
        if (g_hook_ptrs) {
            auto it = g_hook_ptrs->find(p);
            if (it != g_hook_ptrs->end()) {
                h = it->second;
                g_hook_ptrs->erase(it);
            }
        }
    }
    if (h.free) {
        h.free(p, h.ctx, (void*)s);
        return cudaSuccess;
    }
    return cudaFreeAsync(p, s);
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaError_t copy_any(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
}

const DevInfo& dev_info() {
    static thread_local DevInfo cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    DevInfo& d = cache[dev & 63];
    if (d.device != dev) {
        cudaDeviceProp pr;
        if (cudaGetDeviceProperties(&pr, dev) == cudaSuccess) {
            d.sms = pr.multiProcessorCount;
            d.l2_bytes = pr.l2CacheSize;
        } else {
            d.sms = 1;
        }
        d.device = dev;
    }
    return d;
}

static uint64_t g_wait_ns = 0;

uint64_t wait_limit_ns() {
    if (g_wait_ns) return g_wait_ns;
    const char* e = getenv("DSG_WAIT_LIMIT_NS");
    if (e && *e) {
        uint64_t v = strtoull(e, nullptr, 10);
        if (v) return v;
    }
    return 10ull * 1000 * 1000 * 1000;  // 10 s: far above any barrier wait of a healthy run
}

dsg_status status_from_err(uint32_t err, const char* what) {
    if (err == 0) return DSG_OK;
    if (err & ERR_TIMEOUT) {
        set_error("%s: a bounded device wait ran out", what);
        return DSG_ETIMEOUT;
    }
    if (err & ERR_RANGE) {
        set_error("%s: vertex id out of range", what);
        return DSG_EINVAL;
    }
    set_error("%s: internal capacity exceeded (err=0x%x)", what, err);
    return DSG_ECUDA;
}

}  // namespace dsg

using namespace dsg;

extern "C" {

const char* dsg_status_string(dsg_status s) {
    switch (s) {
        case DSG_OK: return "ok";
        case DSG_EINVAL: return "invalid argument";
        case DSG_ENOMEM: return "out of memory";
        case DSG_ECUDA: return "CUDA error";
        case DSG_ETIMEOUT: return "device wait timed out";
        case DSG_EBUSY: return "busy";
        case DSG_EAGAIN: return "not ready";
        case DSG_ENOTFOUND: return "not found";
        case DSG_EOVERFLOW: return "output capacity too small";
    }
    return "unknown status";
}

const char* dsg_last_error(void) { return g_err; }

const char* dsg_version(void) { return "dsg 0.1 (sm_103a)"; }

void dsg_set_wait_limit_ns(uint64_t ns) { g_wait_ns = ns; }

uint64_t dsg_round_bound(uint32_t n, uint32_t p, uint32_t q) {
    if (n == 0) return 1;
    if (p == 0 || q == 0) return (uint64_t)n + 1;
    double b = ceil(log((double)n) / log1p((double)p / (double)q)) + 2.0;
    if (b > (double)n + 1.0) return (uint64_t)n + 1;
    return (uint64_t)b;
}

dsg_status dsg_graph_info(const dsg_graph* g, uint32_t* n, uint64_t* m) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return DSG_OK;
}

dsg_status dsg_graph_set_stream(dsg_graph* g, void* stream) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    g->stream = (cudaStream_t)stream;
    return DSG_OK;
}

dsg_status dsg_graph_view(const dsg_graph* g, void* stream, dsg_graph** out) {
    clear_error();
    DSG_CHECK_ARG(g && out, "graph or out is NULL");
    dsg_graph* v = new dsg_graph(*g);
    v->owns = false;
    v->stream = (cudaStream_t)stream;
    v->max_blocks = 0;
    v->force_block = 0;
    *out = v;
    return DSG_OK;
}

dsg_status dsg_graph_set_max_blocks(dsg_graph* g, uint32_t max_blocks) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    g->max_blocks = max_blocks;
    return DSG_OK;
}

dsg_status dsg_graph_csr(const dsg_graph* g, uint64_t* off, uint32_t* adj) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    if (off) DSG_TRY_CUDA(copy_any(off, g->off, ((size_t)g->n + 1) * sizeof(uint64_t), g->stream));
    if (adj) DSG_TRY_CUDA(copy_any(adj, g->adj, (size_t)(2 * g->m) * sizeof(uint32_t), g->stream));
    DSG_TRY_CUDA(cudaStreamSynchronize(g->stream));
    return DSG_OK;
}

void dsg_graph_free(dsg_graph* g) {
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->owns) {
        cudaStreamSynchronize(g->stream);
        dev_free(g->off, g->stream);
        dev_free(g->adj, g->stream);
        cudaStreamSynchronize(g->stream);
    }
    delete g;
}

dsg_status dsg_graph_from_csr(uint32_t n, const uint64_t* off, const uint32_t* adj, uint32_t flags, void* stream,
                              dsg_graph** out) {
    clear_error();
    DSG_CHECK_ARG(out, "out is NULL");
    DSG_CHECK_ARG(n < 0x80000000u, "n must be below 2^31");
    DSG_CHECK_ARG(off, "off is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    DSG_TRY_CUDA(cudaGetDevice(&dev));
    // total adjacency length
    uint64_t total = 0;
    if (is_device_ptr(off)) {
        DSG_TRY_CUDA(cudaMemcpyAsync(&total, off + n, sizeof(uint64_t), cudaMemcpyDefault, s));
        DSG_TRY_CUDA(cudaStreamSynchronize(s));
    } else {
        total = off[n];
    }
    DSG_CHECK_ARG(total == 0 || adj, "adj is NULL");
    if (flags & DSG_CSR_CANONICALIZE) {
        // Treat every CSR entry (v, adj[j]) as a raw pair and run the ingest.
        return ingest_from_csr_entries(n, off, adj, total, flags, s, out);
    }
    DSG_CHECK_ARG(total % 2 == 0, "off[n] must be even for a symmetric CSR");
    dsg_graph* g = new dsg_graph();
    g->n = n;
    g->m = total / 2;
    g->device = dev;
    g->stream = s;
    if ((flags & DSG_PTRS_DEVICE) && is_device_ptr(off) && (total == 0 || is_device_ptr(adj))) {
        g->owns = false;
        g->off = const_cast<uint64_t*>(off);
        g->adj = const_cast<uint32_t*>(adj);
    } else {
        DSG_CHECK_ARG(!(flags & DSG_PTRS_DEVICE), "DSG_PTRS_DEVICE given with host pointers");
        cudaError_t e = dev_alloc((void**)&g->off, ((size_t)n + 1) * sizeof(uint64_t), s);
        if (e == cudaSuccess) e = dev_alloc((void**)&g->adj, (size_t)(total ? total : 1) * sizeof(uint32_t), s);
        if (e == cudaSuccess) e = copy_any(g->off, off, ((size_t)n + 1) * sizeof(uint64_t), s);
        if (e == cudaSuccess) e = copy_any(g->adj, adj, (size_t)total * sizeof(uint32_t), s);
        if (e != cudaSuccess) {
            set_error("graph_from_csr: %s", cudaGetErrorString(e));
            dsg_graph_free(g);
            return e == cudaErrorMemoryAllocation ? DSG_ENOMEM : DSG_ECUDA;
        }
    }
    if (flags & DSG_CSR_VALIDATE) {
        dsg_status st = validate_csr(g);
        if (st != DSG_OK) {
            dsg_graph_free(g);
            return st;
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("graph_from_csr: %s", cudaGetErrorString(e));
        dsg_graph_free(g);
        return DSG_ECUDA;
    }
    *out = g;
    return DSG_OK;
}

}  // extern "C"

extern "C" void dsg_set_allocator(dsg_alloc_fn alloc, dsg_free_fn free_fn, void* ctx) {
    std::lock_guard<std::mutex> lk(g_hook_mu);
    if (alloc && free_fn) {
        g_hook.alloc = alloc;
        g_hook.free = free_fn;
        g_hook.ctx = ctx;
    } else {
        g_hook = HookAlloc();
    }
}
