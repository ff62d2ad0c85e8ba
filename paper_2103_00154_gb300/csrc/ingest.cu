// CSR ingest: raw undirected pairs -> canonical CSR (Def. 1: a simple graph,
// E a set of edges between distinct vertices).
//
//   1. count   every non-loop pair adds one to the row of each endpoint
//   2. scan    row starts of the (still repeated) entries
//   3. scatter each pair is written into both rows
//   4. sort    each row sorted and de-duplicated in place; rows are binned by
//              length: <= 32 entries one warp (register bitonic network),
//              <= kMidMax one block (shared-memory bitonic), longer rows one
//              block each (shared-memory sorted runs + merge-path passes)
//   5. scan    final row lengths -> off
//   6. copy    unique entries into adj
// The result is byte-identical to sorting the (min, max) keys and removing
// repeats, because a canonical CSR of a given edge set is unique.
#include <cooperative_groups.h>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace cg = cooperative_groups;

namespace dsg {

constexpr uint32_t kPad = 0xffffffffu;
constexpr uint32_t kMidMax = 4096;   // longest row sorted in one shared-memory pass
constexpr uint32_t kMidThreads = 512;
constexpr uint32_t kScanTile = 2048;

__global__ void validate_off_kernel(uint32_t n, const uint64_t* __restrict__ off, uint32_t* bad);

struct IngestCtl {
    uint32_t err;
    uint32_t n_mid;
    uint32_t n_big;
    uint32_t pad;
};

// ----------------------------------------------------------- device scan

__global__ void scan_tile_sums(const uint32_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ sums) {
    __shared__ uint64_t tmp[33];
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t s = 0;
    for (uint32_t j = threadIdx.x; j < kScanTile; j += blockDim.x)
        if (base + j < n) s += in[base + j];
    s = block_sum<uint64_t>(s, tmp);
    if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

// One block: exclusive scan of the tile sums in place; *total = grand total.
__global__ void scan_sums_single(uint64_t* __restrict__ sums, uint64_t nt, uint64_t* __restrict__ total) {
    __shared__ uint64_t tmp[33];
    uint64_t carry = 0;
    for (uint64_t b = 0; b < nt; b += blockDim.x) {
        uint64_t i = b + threadIdx.x;
        uint64_t v = i < nt ? sums[i] : 0;
        uint64_t tot;
        uint64_t pre = block_excl_scan<uint64_t>(v, tmp, &tot);
        if (i < nt) sums[i] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_tile_apply(const uint32_t* __restrict__ in, uint64_t n, const uint64_t* __restrict__ sums,
                                uint64_t* __restrict__ out) {
    __shared__ uint64_t tmp[33];
    const uint32_t per = kScanTile / 1024;  // blockDim == 1024
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * per;
    uint64_t vals[kScanTile / 1024];
    uint64_t loc = 0;
#pragma unroll
    for (uint32_t j = 0; j < per; ++j) {
        vals[j] = base + j < n ? in[base + j] : 0;
        loc += vals[j];
    }
    uint64_t tot;
    uint64_t pre = block_excl_scan<uint64_t>(loc, tmp, &tot);
    uint64_t run = sums[blockIdx.x] + pre;
#pragma unroll
    for (uint32_t j = 0; j < per; ++j) {
        if (base + j < n) out[base + j] = run;
        run += vals[j];
    }
}

// out[0..n) = exclusive prefix of in, out[n] = total.  `sums` needs
// ceil(n / kScanTile) + 1 slots.
static cudaError_t device_scan(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* sums, cudaStream_t s) {
    uint64_t nt = (n + kScanTile - 1) / kScanTile;
    if (nt == 0) return cudaMemsetAsync(out, 0, sizeof(uint64_t), s);
    { LaunchScope ls_("ingest_scan_tile_sums", s); scan_tile_sums<<<(uint32_t)nt, 256, 0, s>>>(in, n, sums); }
    { LaunchScope ls_("ingest_scan_sums_single", s); scan_sums_single<<<1, 1024, 0, s>>>(sums, nt, out + n); }
    { LaunchScope ls_("ingest_scan_tile_apply", s); scan_tile_apply<<<(uint32_t)nt, 1024, 0, s>>>(in, n, sums, out); }
    return cudaGetLastError();
}

// ----------------------------------------------------------- count / scatter

__global__ void count_kernel(uint32_t n, uint64_t m_raw, const uint32_t* __restrict__ src,
                             const uint32_t* __restrict__ dst, uint32_t* __restrict__ cnt, IngestCtl* ctl) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_raw;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = src[i], v = dst[i];
        if (u >= n || v >= n) {
            atomicOr(&ctl->err, ERR_RANGE);
            continue;
        }
        if (u == v) continue;
        atomicAdd(&cnt[u], 1u);
        atomicAdd(&cnt[v], 1u);
    }
}

__global__ void scatter_kernel(uint32_t n, uint64_t m_raw, const uint32_t* __restrict__ src,
                               const uint32_t* __restrict__ dst, const uint64_t* __restrict__ start,
                               uint32_t* __restrict__ fill, uint32_t* __restrict__ tmp) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_raw;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = src[i], v = dst[i];
        if (u >= n || v >= n || u == v) continue;
        tmp[start[u] + atomicAdd(&fill[u], 1u)] = v;
        tmp[start[v] + atomicAdd(&fill[v], 1u)] = u;
    }
}

// ----------------------------------------------------------- row sort

// Rows of <= 32 entries: one warp per row, register bitonic sort, dedup by
// neighbour compare; longer rows are appended to the mid / big lists.
__global__ void sort_small_rows(uint32_t n, const uint64_t* __restrict__ start, const uint32_t* __restrict__ cnt,
                                uint32_t* __restrict__ tmp, uint32_t* __restrict__ newlen,
                                uint32_t* __restrict__ mid_list, uint32_t* __restrict__ big_list, IngestCtl* ctl) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = gw; v < n; v += nw) {
        uint32_t len = cnt[v];
        if (len > 32) {
            if (lane == 0) {
                if (len <= kMidMax) mid_list[atomicAdd(&ctl->n_mid, 1u)] = (uint32_t)v;
                else big_list[atomicAdd(&ctl->n_big, 1u)] = (uint32_t)v;
            }
            continue;
        }
        if (len == 0) {
            if (lane == 0) newlen[v] = 0;
            continue;
        }
        uint64_t b = start[v];
        uint32_t x = lane < len ? tmp[b + lane] : kPad;
#pragma unroll
        for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                uint32_t y = __shfl_xor_sync(kFullMask, x, j);
                bool up = (lane & k) == 0;
                bool lower = (lane & j) == 0;
                // lower lane keeps min when ascending, max when descending
                x = (lower == up) ? min(x, y) : max(x, y);
            }
        }
        uint32_t prev = __shfl_up_sync(kFullMask, x, 1);
        bool keep = x != kPad && (lane == 0 || x != prev);
        uint32_t bal = __ballot_sync(kFullMask, keep);
        if (keep) tmp[b + __popc(bal & lanemask_lt())] = x;
        if (lane == 0) newlen[v] = __popc(bal);
    }
}

// Bitonic sort of `len` values in shared memory padded to a power of two `p2`.
__device__ void smem_bitonic(uint32_t* s, uint32_t p2) {
    for (uint32_t k = 2; k <= p2; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < p2; i += blockDim.x) {
                uint32_t l = i ^ j;
                if (l > i) {
                    uint32_t a = s[i], b = s[l];
                    bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        s[i] = b;
                        s[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Keep the first of each run of equal values of sorted s[0, len) (no kPad
// inside), writing them compacted to out; returns the kept count.
__device__ uint32_t smem_unique_write(const uint32_t* s, uint32_t len, uint32_t* out, uint32_t* scan_tmp) {
    uint32_t kept = 0;
    for (uint32_t t = 0; t < len; t += blockDim.x) {
        uint32_t i = t + threadIdx.x;
        bool keep = i < len && (i == 0 || s[i] != s[i - 1]);
        uint32_t tot;
        uint32_t pre = block_excl_scan<uint32_t>(keep ? 1u : 0u, scan_tmp, &tot);
        if (keep) out[kept + pre] = s[i];
        kept += tot;
    }
    return kept;
}

__global__ void __launch_bounds__(kMidThreads) sort_mid_rows(const uint32_t* __restrict__ list,
                                                             const IngestCtl* __restrict__ ctl,
                                                             const uint64_t* __restrict__ start,
                                                             const uint32_t* __restrict__ cnt,
                                                             uint32_t* __restrict__ tmp,
                                                             uint32_t* __restrict__ newlen) {
    __shared__ uint32_t s[kMidMax];
    __shared__ uint32_t scan_tmp[33];
    const uint32_t nmid = ctl->n_mid;
    for (uint32_t r = blockIdx.x; r < nmid; r += gridDim.x) {
        uint32_t v = list[r];
        uint32_t len = cnt[v];
        uint64_t b = start[v];
        uint32_t p2 = 64;
        while (p2 < len) p2 <<= 1;
        for (uint32_t i = threadIdx.x; i < p2; i += blockDim.x) s[i] = i < len ? tmp[b + i] : kPad;
        __syncthreads();
        smem_bitonic(s, p2);
        uint32_t kept = smem_unique_write(s, len, tmp + b, scan_tmp);
        if (threadIdx.x == 0) newlen[v] = kept;
        __syncthreads();
    }
}

// Rows longer than kMidMax: one block per row.  Runs of kMidMax entries are
// sorted in shared memory, then merged pairwise (merge path: each thread
// binary-searches its diagonal and merges its share sequentially) between
// tmp and the spare buffer until one run remains; finally de-duplicated.
__device__ void merge_path_block(const uint32_t* A, uint32_t la, const uint32_t* B, uint32_t lb, uint32_t* out) {
    uint32_t total = la + lb;
    uint32_t per = (total + blockDim.x - 1) / blockDim.x;
    uint32_t d0 = min(total, threadIdx.x * per), d1 = min(total, d0 + per);
    // split of diagonal d: i from A, d - i from B, with A[i-1] <= B[d-i] and B[d-i-1] < A[i]
    auto split = [&](uint32_t d) {
        uint32_t lo = d > lb ? d - lb : 0, hi = min(d, la);
        while (lo < hi) {
            uint32_t i = (lo + hi) >> 1;
            if (A[i] <= B[d - i - 1]) lo = i + 1; else hi = i;
        }
        return lo;
    };
    uint32_t i = split(d0), j = d0 - i;
    for (uint32_t d = d0; d < d1; ++d) {
        if (j >= lb || (i < la && A[i] <= B[j])) out[d] = A[i++];
        else out[d] = B[j++];
    }
}

__global__ void __launch_bounds__(kMidThreads) sort_big_rows(const uint32_t* __restrict__ list,
                                                             const IngestCtl* __restrict__ ctl,
                                                             const uint64_t* __restrict__ start,
                                                             const uint32_t* __restrict__ cnt,
                                                             uint32_t* __restrict__ tmp, uint32_t* __restrict__ spare,
                                                             uint32_t* __restrict__ newlen) {
    __shared__ uint32_t s[kMidMax];
    __shared__ uint32_t scan_tmp[33];
    const uint32_t nbig = ctl->n_big;
    for (uint32_t r = blockIdx.x; r < nbig; r += gridDim.x) {
        uint32_t v = list[r];
        uint32_t len = cnt[v];
        uint64_t b = start[v];
        uint32_t* src = tmp + b;
        uint32_t* dst = spare + b;
        // sorted runs of kMidMax
        for (uint32_t r0 = 0; r0 < len; r0 += kMidMax) {
            uint32_t l = min(kMidMax, len - r0);
            for (uint32_t i = threadIdx.x; i < kMidMax; i += blockDim.x) s[i] = i < l ? src[r0 + i] : kPad;
            __syncthreads();
            smem_bitonic(s, kMidMax);
            for (uint32_t i = threadIdx.x; i < l; i += blockDim.x) src[r0 + i] = s[i];
            __syncthreads();
        }
        // merge passes
        for (uint32_t run = kMidMax; run < len; run <<= 1) {
            for (uint32_t a0 = 0; a0 < len; a0 += 2 * run) {
                uint32_t la = min(run, len - a0);
                uint32_t lb = a0 + run < len ? min(run, len - a0 - run) : 0;
                merge_path_block(src + a0, la, src + a0 + la, lb, dst + a0);
                __syncthreads();
            }
            uint32_t* t = src; src = dst; dst = t;
        }
        // unique, in tiles, into tmp (src may be tmp or spare; writes trail reads)
        uint32_t kept = 0;
        for (uint32_t t0 = 0; t0 < len; t0 += blockDim.x) {
            uint32_t i = t0 + threadIdx.x;
            uint32_t x = i < len ? src[i] : 0;
            bool keep = i < len && (i == 0 || x != src[i - 1]);
            uint32_t tot;
            uint32_t pre = block_excl_scan<uint32_t>(keep ? 1u : 0u, scan_tmp, &tot);
            __syncthreads();
            if (keep) tmp[b + kept + pre] = x;
            kept += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) newlen[v] = kept;
        __syncthreads();
    }
}

__global__ void copy_rows(uint32_t n, const uint64_t* __restrict__ start, const uint32_t* __restrict__ tmp,
                          const uint64_t* __restrict__ off, uint32_t* __restrict__ adj) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = gw; v < n; v += nw) {
        uint64_t b = start[v], o = off[v], len = off[v + 1] - o;
        for (uint64_t j = lane; j < len; j += 32) adj[o + j] = tmp[b + j];
    }
}

// owner of each CSR entry (to ingest a CSR as raw pairs)
__global__ void expand_rows(uint32_t n, const uint64_t* __restrict__ off, uint32_t* __restrict__ src) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = gw; v < n; v += nw)
        for (uint64_t j = off[v] + lane; j < off[v + 1]; j += 32) src[j] = (uint32_t)v;
}

static uint32_t grid_for(uint64_t work, uint32_t block) {
    uint64_t g = (work + block - 1) / block;
    uint64_t cap = (uint64_t)dev_info().sms * 16;
    if (g > cap) g = cap;
    return (uint32_t)(g ? g : 1);
}

// Core ingest on device arrays src/dst (m_raw pairs).  Allocates the graph.
static dsg_status ingest_device(uint32_t n, uint64_t m_raw, const uint32_t* src, const uint32_t* dst,
                                cudaStream_t s, dsg_graph** out) {
    int dev = 0;
    DSG_TRY_CUDA(cudaGetDevice(&dev));
    Scratch sc(s);
    uint32_t *cnt, *tmp, *spare, *newlen, *mid_list, *big_list;
    uint64_t *start, *sums;
    IngestCtl* ctl;
    const uint64_t nt = (uint64_t)n / kScanTile + 2;
    DSG_TRY_CUDA(sc.get(&cnt, (size_t)n + 1));
    DSG_TRY_CUDA(sc.get(&start, (size_t)n + 1));
    DSG_TRY_CUDA(sc.get(&sums, nt));
    DSG_TRY_CUDA(sc.get(&newlen, (size_t)n + 1));
    DSG_TRY_CUDA(sc.get(&mid_list, (size_t)n + 1));
    DSG_TRY_CUDA(sc.get(&big_list, (size_t)n + 1));
    DSG_TRY_CUDA(sc.get(&ctl, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)n + 1) * 4, s));
    DSG_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(IngestCtl), s));
    { LaunchScope ls_("ingest_count_kernel", s); count_kernel<<<grid_for(m_raw, 256), 256, 0, s>>>(n, m_raw, src, dst, cnt, ctl); }
    DSG_TRY_CUDA(cudaGetLastError());
    DSG_TRY_CUDA(device_scan(cnt, n, start, sums, s));
    IngestCtl hc;
    uint64_t total = 0;
    DSG_TRY_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaMemcpyAsync(&total, start + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    if (hc.err & ERR_RANGE) {
        set_error("graph_from_edges: a vertex id is >= n");
        return DSG_EINVAL;
    }
    DSG_TRY_CUDA(sc.get(&tmp, total ? total : 1));
    DSG_TRY_CUDA(sc.get(&spare, total ? total : 1));
    DSG_TRY_CUDA(cudaMemsetAsync(newlen, 0, ((size_t)n + 1) * 4, s));  // reused as the fill counter
    { LaunchScope ls_("ingest_scatter_kernel", s); scatter_kernel<<<grid_for(m_raw, 256), 256, 0, s>>>(n, m_raw, src, dst, start, newlen, tmp); }
    DSG_TRY_CUDA(cudaGetLastError());
    {
        LaunchScope ls_("ingest_sort_small_rows", s);
        sort_small_rows<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(n, start, cnt, tmp, newlen, mid_list,
                                                                         big_list, ctl);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    { LaunchScope ls_("ingest_sort_mid_rows", s); sort_mid_rows<<<dev_info().sms * 4, kMidThreads, 0, s>>>(mid_list, ctl, start, cnt, tmp, newlen); }
    DSG_TRY_CUDA(cudaGetLastError());
    { LaunchScope ls_("ingest_sort_big_rows", s); sort_big_rows<<<dev_info().sms * 2, kMidThreads, 0, s>>>(big_list, ctl, start, cnt, tmp, spare, newlen); }
    DSG_TRY_CUDA(cudaGetLastError());
    dsg_graph* g = new dsg_graph();
    g->n = n;
    g->device = dev;
    g->stream = s;
    cudaError_t e = dev_alloc((void**)&g->off, ((size_t)n + 1) * sizeof(uint64_t), s);
    if (e == cudaSuccess) e = device_scan(newlen, n, g->off, sums, s);
    uint64_t total2 = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total2, g->off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = dev_alloc((void**)&g->adj, (size_t)(total2 ? total2 : 1) * sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        { LaunchScope ls_("ingest_copy_rows", s); copy_rows<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(n, start, tmp, g->off, g->adj); }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("graph_from_edges: %s", cudaGetErrorString(e));
        g->owns = true;
        dsg_graph_free(g);
        return e == cudaErrorMemoryAllocation ? DSG_ENOMEM : DSG_ECUDA;
    }
    g->m = total2 / 2;
    *out = g;
    return DSG_OK;
}

dsg_status ingest_from_csr_entries(uint32_t n, const uint64_t* off, const uint32_t* adj, uint64_t total,
                                   uint32_t flags, cudaStream_t s, dsg_graph** out) {
    Scratch sc(s);
    const uint64_t* doff = off;
    const uint32_t* dadj = adj;
    if (!is_device_ptr(off)) {
        uint64_t* t;
        DSG_TRY_CUDA(sc.get(&t, (size_t)n + 1));
        DSG_TRY_CUDA(copy_any(t, off, ((size_t)n + 1) * 8, s));
        doff = t;
    }
    if (total && !is_device_ptr(adj)) {
        uint32_t* t;
        DSG_TRY_CUDA(sc.get(&t, total));
        DSG_TRY_CUDA(copy_any(t, adj, total * 4, s));
        dadj = t;
    }
    {
        // offsets must start at 0 and never decrease before rows are expanded
        uint32_t* bad;
        DSG_TRY_CUDA(sc.get(&bad, 1));
        DSG_TRY_CUDA(cudaMemsetAsync(bad, 0, 4, s));
        { LaunchScope ls_("ingest_validate_off_kernel", s); validate_off_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, doff, bad); }
        DSG_TRY_CUDA(cudaGetLastError());
        uint32_t hb = 0;
        DSG_TRY_CUDA(cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, s));
        DSG_TRY_CUDA(cudaStreamSynchronize(s));
        if (hb) {
            set_error("graph_from_csr: offsets must start at 0 and be non-decreasing");
            return DSG_EINVAL;
        }
    }
    uint32_t* src;
    DSG_TRY_CUDA(sc.get(&src, total ? total : 1));
    { LaunchScope ls_("ingest_expand_rows", s); expand_rows<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(n, doff, src); }
    DSG_TRY_CUDA(cudaGetLastError());
    dsg_status st = ingest_device(n, total, src, dadj, s, out);
    if (st == DSG_OK && (flags & DSG_CSR_VALIDATE)) {
        st = validate_csr(*out);
        if (st != DSG_OK) {
            dsg_graph_free(*out);
            *out = nullptr;
        }
    }
    return st;
}

// ----------------------------------------------------------- validation

__global__ void validate_kernel(uint32_t n, const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj,
                                uint32_t* bad) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t total = off[n];
    for (uint64_t v = gw; v < n; v += nw) {
        uint64_t b = off[v], e = off[v + 1];
        if (e < b || e > total) {
            if (lane == 0) atomicOr(bad, 1u);  // offsets not monotone
            continue;
        }
        for (uint64_t j = b + lane; j < e; j += 32) {
            uint32_t u = adj[j];
            if (u >= n) { atomicOr(bad, 2u); continue; }        // id out of range
            if (u == v) { atomicOr(bad, 4u); continue; }        // self-loop
            if (j > b && adj[j - 1] >= u) atomicOr(bad, 8u);    // unsorted or repeated
            // symmetric: v must appear in row u
            uint64_t lo = off[u], hi = off[u + 1];
            if (hi < lo || hi > total) { atomicOr(bad, 1u); continue; }
            while (lo < hi) {
                uint64_t mid = (lo + hi) >> 1;
                if (adj[mid] < v) lo = mid + 1; else hi = mid;
            }
            if (lo >= off[u + 1] || adj[lo] != v) atomicOr(bad, 16u);
        }
    }
}

__global__ void validate_off_kernel(uint32_t n, const uint64_t* __restrict__ off, uint32_t* bad) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && off[0] != 0) atomicOr(bad, 1u);
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        if (off[v + 1] < off[v]) atomicOr(bad, 1u);
}

dsg_status validate_csr(const dsg_graph* g) {
    cudaStream_t s = g->stream;
    Scratch sc(s);
    uint32_t* bad;
    DSG_TRY_CUDA(sc.get(&bad, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(bad, 0, 4, s));
    { LaunchScope ls_("ingest_validate_off_kernel", s); validate_off_kernel<<<grid_for(g->n, 256), 256, 0, s>>>(g->n, g->off, bad); }
    uint32_t hb = 0;
    DSG_TRY_CUDA(cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    if (hb == 0) {
        { LaunchScope ls_("ingest_validate_kernel", s); validate_kernel<<<grid_for((uint64_t)g->n * 32, 256), 256, 0, s>>>(g->n, g->off, g->adj, bad); }
        DSG_TRY_CUDA(cudaGetLastError());
        DSG_TRY_CUDA(cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, s));
        DSG_TRY_CUDA(cudaStreamSynchronize(s));
    }
    if (hb) {
        set_error("CSR is not canonical (%s%s%s%s%s)", hb & 1 ? "offsets " : "", hb & 2 ? "id>=n " : "",
                  hb & 4 ? "self-loop " : "", hb & 8 ? "unsorted/repeated " : "", hb & 16 ? "asymmetric" : "");
        return DSG_EINVAL;
    }
    return DSG_OK;
}

}  // namespace dsg

using namespace dsg;

extern "C" dsg_status dsg_graph_from_edges(uint32_t n, uint64_t m_raw, const uint32_t* src, const uint32_t* dst,
                                           uint32_t flags, void* stream, dsg_graph** out) {
    clear_error();
    DSG_CHECK_ARG(out, "out is NULL");
    DSG_CHECK_ARG(n < 0x80000000u, "n must be below 2^31");
    DSG_CHECK_ARG(m_raw == 0 || (src && dst), "src/dst is NULL");
    DSG_CHECK_ARG(m_raw < (1ull << 32), "m_raw must be below 2^32");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t* dsrc = src;
    const uint32_t* ddst = dst;
    Scratch sc(s);
    bool on_dev = m_raw == 0 || (is_device_ptr(src) && is_device_ptr(dst));
    if (flags & DSG_PTRS_DEVICE) DSG_CHECK_ARG(on_dev, "DSG_PTRS_DEVICE given with host pointers");
    if (!on_dev) {
        uint32_t *a, *b;
        DSG_TRY_CUDA(sc.get(&a, m_raw));
        DSG_TRY_CUDA(sc.get(&b, m_raw));
        DSG_TRY_CUDA(copy_any(a, src, m_raw * 4, s));
        DSG_TRY_CUDA(copy_any(b, dst, m_raw * 4, s));
        dsrc = a;
        ddst = b;
    }
    dsg_status st = ingest_device(n, m_raw, dsrc, ddst, s, out);
    if (st == DSG_OK && (flags & DSG_CSR_VALIDATE)) {
        st = validate_csr(*out);
        if (st != DSG_OK) {
            dsg_graph_free(*out);
            *out = nullptr;
        }
    }
    return st;
}
