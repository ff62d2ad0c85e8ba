// Densest k-core and the vertex augmentation of CBDS-P (Algorithm 2).
//
// Phase 1 of Algorithm 2 leaves every vertex's core number (PKC, kcore.cu).
// The densest core is the k-core {v : core(v) >= k} of highest density
// |E_k| / |V_k| (Sec. 3.2; the densest core is a 2-approximation of the
// densest subgraph).  It is found here exactly, with one pass over the
// adjacency:
//   hV[c] = #{v : core(v) = c}
//   hE[c] = #{edges {u, v} : min(core(u), core(v)) = c}
// so that V_k and E_k are suffix sums of hV and hE, and the smallest k of
// highest density wins (strict comparison with increasing k, Algorithm 2's
// maximum update).  Label k goes with the k-core {core >= k} (Algorithm 2
// measures a level's density once its vertices joined `visited`, but its
// second phase compares against the labelled core, so label and set are
// taken to be the same core).
//
// Phase 2 of Algorithm 2 then grows the densest core by vertices outside it:
//   eligible v: core(v) lies strictly between the core's density E_k/V_k and k*
//   cnt(v)    : neighbours of v inside the densest core
//   legit v   : eligible and cnt(v) > E_k/V_k; each adds cnt(v) edges and one vertex
//   pairs     : every edge between two legit vertices is added once
// giving m_e = E_k + sum cnt + pairs and m_v = V_k + #legit.  All density
// tests are exact: an integer x exceeds E/V iff x * V > E.
//
// Kernels (all plain grid-stride launches on the graph's stream, no host
// synchronisation between them):
//   core_max      max core number (sizes the shared-memory histograms)
//   core_hist     hV and hE in one edge-balanced pass over the adjacency
//   densest_pick  suffix sums and the argmax, one block
//   core_mask     out_set[v] = core(v) >= k*
//   elig_items    eligible vertices -> row chunks (v << 32 | c) to count
//   elig_count    one warp per chunk: neighbours with core >= k*
//   legit_mark    legit test, totals, legit row chunks
//   legit_pairs   one warp per legit chunk: legit neighbours u > v
#include <stdio.h>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace dsg {

namespace {

constexpr uint32_t kHistTB = 512;
constexpr uint32_t kShBins = 4096;  // per histogram; shared memory path when k_max < kShBins
constexpr uint32_t kPickTB = 1024;
constexpr uint32_t kRowChunk = 1024;  // entries per phase-2 work item

struct __align__(128) CbdsCtl {
    uint32_t kmax;
    uint32_t pad0;
    uint64_t kstar, Ek, Vk;  // densest core
    uint64_t inter;          // sum cnt(v) over legit v + legit pairs
    uint64_t nleg;
    uint64_t n_elig_items, n_legit_items;
};

// Warp-aggregated histogram increment: lanes holding the same key combine
// their counts before one atomic.  key == ~0u means "no increment".
__device__ __forceinline__ void hist_add_shared(uint32_t* h, uint32_t key) {
    const uint32_t peers = __match_any_sync(kFullMask, key);
    const uint32_t leader = __ffs(peers) - 1;
    if (key != ~0u && (threadIdx.x & 31u) == leader) atomicAdd(&h[key], (uint32_t)__popc(peers));
}

__device__ __forceinline__ void hist_add_global(unsigned long long* h, uint32_t key) {
    const uint32_t peers = __match_any_sync(kFullMask, key);
    const uint32_t leader = __ffs(peers) - 1;
    if (key != ~0u && (threadIdx.x & 31u) == leader) atomicAdd(&h[key], (unsigned long long)__popc(peers));
}

__global__ void core_max_kernel(const uint32_t* __restrict__ core, uint32_t n, CbdsCtl* ctl) {
    uint32_t mx = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        mx = max(mx, core[v]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFullMask, mx, o));
    if ((threadIdx.x & 31u) == 0 && mx) atomicMax(&ctl->kmax, mx);
}

struct HistShared {
    uint32_t hv[kShBins];
    uint32_t he[kShBins];
};

__global__ void __launch_bounds__(kHistTB, 3) core_hist_kernel(const uint64_t* __restrict__ off,
                                                             const uint32_t* __restrict__ adj,
                                                             const uint32_t* __restrict__ core, uint32_t n,
                                                             const CbdsCtl* __restrict__ ctl,
                                                             unsigned long long* __restrict__ hV,
                                                             unsigned long long* __restrict__ hE) {
    __shared__ HistShared sh;
    const bool use_sh = ctl->kmax < kShBins;
    if (use_sh) {
        for (uint32_t i = threadIdx.x; i < kShBins; i += blockDim.x) sh.hv[i] = sh.he[i] = 0;
        __syncthreads();
    }
    // vertices: hV[core(v)]
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v0 = tid - (threadIdx.x & 31u); v0 < n; v0 += nth) {
        const uint64_t v = v0 + (threadIdx.x & 31u);
        const uint32_t key = v < n ? core[v] : ~0u;
        if (use_sh) hist_add_shared(sh.hv, key); else hist_add_global(hV, key);
    }
    // edges, each once (entry (v, u) with u > v): hE[min(core(v), core(u))]
    auto pre = [&](uint64_t j) { return adj[j]; };
    auto visit = [&](const uint32_t* v, const uint64_t*, const uint32_t* u, uint32_t valid) {
        uint32_t cv[kWalkU], cu[kWalkU];
#pragma unroll
        for (uint32_t t = 0; t < kWalkU; ++t) {
            const bool take = (valid >> t & 1u) && u[t] > v[t];
            cv[t] = take ? core[v[t]] : ~0u;
            cu[t] = take ? core[u[t]] : ~0u;
        }
#pragma unroll
        for (uint32_t t = 0; t < kWalkU; ++t) {
            const uint32_t key = min(cv[t], cu[t]);
            if (use_sh) hist_add_shared(sh.he, key); else hist_add_global(hE, key);
        }
    };
    walk_all_entries(off, n, pre, visit);
    if (use_sh) {
        __syncthreads();
        const uint32_t kmax = ctl->kmax;
        for (uint32_t i = threadIdx.x; i <= kmax; i += blockDim.x) {
            if (sh.hv[i]) atomicAdd(&hV[i], (unsigned long long)sh.hv[i]);
            if (sh.he[i]) atomicAdd(&hE[i], (unsigned long long)sh.he[i]);
        }
    }
}

// (E, V, k) candidates: a beats b when E_a / V_a > E_b / V_b, or equal and k_a < k_b.
struct Cand {
    uint64_t E, V, k;
};
__device__ __forceinline__ bool beats(const Cand& a, const Cand& b) {
    if (a.V == 0) return false;
    if (b.V == 0) return true;
    const unsigned __int128 l = (unsigned __int128)a.E * b.V, r = (unsigned __int128)b.E * a.V;
    return l > r || (l == r && a.k < b.k);
}

__global__ void __launch_bounds__(kPickTB) densest_pick_kernel(const unsigned long long* __restrict__ hV,
                                                                const unsigned long long* __restrict__ hE,
                                                                CbdsCtl* ctl) {
    __shared__ uint64_t tmp[33];
    __shared__ Cand red[kPickTB / 32];
    const uint32_t kmax = ctl->kmax;
    uint64_t carryV = 0, carryE = 0;
    Cand best{0, 0, 0};
    // chunks of kPickTB bins from the top down; thread t takes k = top - t
    for (int64_t top = kmax; top >= 0; top -= kPickTB) {
        const int64_t k = top - (int64_t)threadIdx.x;
        const uint64_t xv = k >= 0 ? hV[k] : 0, xe = k >= 0 ? hE[k] : 0;
        uint64_t totV, totE;
        const uint64_t pv = block_excl_scan<uint64_t>(xv, tmp, &totV);
        __syncthreads();
        const uint64_t pe = block_excl_scan<uint64_t>(xe, tmp, &totE);
        __syncthreads();
        if (k >= 0) {
            const Cand c{carryE + pe + xe, carryV + pv + xv, (uint64_t)k};
            if (beats(c, best)) best = c;
        }
        carryV += totV;
        carryE += totE;
    }
    // block argmax
    for (int o = 16; o > 0; o >>= 1) {
        Cand c{__shfl_xor_sync(kFullMask, best.E, o), __shfl_xor_sync(kFullMask, best.V, o),
               __shfl_xor_sync(kFullMask, best.k, o)};
        if (beats(c, best)) best = c;
    }
    if ((threadIdx.x & 31u) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        Cand b = red[0];
        for (uint32_t i = 1; i < blockDim.x / 32; ++i)
            if (beats(red[i], b)) b = red[i];
        ctl->kstar = b.k;
        ctl->Ek = b.E;
        ctl->Vk = b.V;
    }
}

__global__ void core_mask_kernel(const uint32_t* __restrict__ core, const uint8_t* __restrict__ legit, uint32_t n,
                                 const CbdsCtl* __restrict__ ctl, uint8_t* __restrict__ out) {
    const uint64_t ks = ctl->kstar;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        out[v] = (uint8_t)(core[v] >= ks || (legit && legit[v]));
}

__device__ __forceinline__ bool is_eligible(uint64_t dv, const CbdsCtl& c) {
    return (unsigned __int128)dv * c.Vk > c.Ek && dv < c.kstar;
}

// Warp-aggregated reservation of `want` slots on *counter.
__device__ __forceinline__ uint64_t warp_reserve(unsigned long long* counter, uint32_t want) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t inc = warp_incl_scan(want);
    const uint32_t tot = __shfl_sync(kFullMask, inc, 31);
    unsigned long long base = 0;
    if (lane == 31 && tot) base = atomicAdd(counter, (unsigned long long)tot);
    base = __shfl_sync(kFullMask, base, 31);
    return base + inc - want;
}

__device__ __forceinline__ void emit_chunks(uint64_t* items, uint64_t at, uint32_t v, uint32_t cnt) {
    for (uint32_t c = 0; c < cnt; ++c) items[at + c] = (uint64_t)v << 32 | c;
}

__global__ void elig_items_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ core, uint32_t n,
                                  CbdsCtl* ctl, uint32_t* __restrict__ cnt, uint64_t* __restrict__ items) {
    const CbdsCtl c = *ctl;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - (threadIdx.x & 31u); v0 < n; v0 += nth) {
        const uint64_t v = v0 + (threadIdx.x & 31u);
        uint32_t want = 0;
        if (v < n && is_eligible(core[v], c)) {
            cnt[v] = 0;
            const uint64_t len = off[v + 1] - off[v];
            want = (uint32_t)((len + kRowChunk - 1) / kRowChunk);
        }
        const uint64_t at = warp_reserve((unsigned long long*)&ctl->n_elig_items, want);
        emit_chunks(items, at, (uint32_t)v, want);
    }
}

// One warp per item: counts the entries of the item's row chunk that pass
// `test`, adds the count to acc (per-vertex or global).
template <bool PAIRS>
__global__ void row_chunk_count_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj,
                                       const uint32_t* __restrict__ core, const uint8_t* __restrict__ legit,
                                       CbdsCtl* ctl, const uint64_t* __restrict__ items,
                                       uint32_t* __restrict__ cnt) {
    const uint64_t nitems = PAIRS ? ctl->n_legit_items : ctl->n_elig_items;
    const uint64_t ks = ctl->kstar;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t pairs = 0;
    for (uint64_t it = gw; it < nitems; it += nw) {
        const uint64_t item = items[it];
        const uint32_t v = (uint32_t)(item >> 32), ci = (uint32_t)item;
        const uint64_t b = off[v] + (uint64_t)ci * kRowChunk;
        const uint64_t e = min(off[v + 1], b + kRowChunk);
        uint32_t s = 0;
        for (uint64_t j = b + lane; j < e; j += 32) {
            const uint32_t u = adj[j];
            if (PAIRS) s += (u > v && legit[u]) ? 1u : 0u;
            else s += core[u] >= ks ? 1u : 0u;
        }
        s = warp_sum(s);
        if (PAIRS) pairs += s;
        else if (lane == 0 && s) atomicAdd(&cnt[v], s);
    }
    if (PAIRS && lane == 0 && pairs) atomicAdd((unsigned long long*)&ctl->inter, (unsigned long long)pairs);
}

__global__ void legit_mark_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ core, uint32_t n,
                                  CbdsCtl* ctl, const uint32_t* __restrict__ cnt, uint8_t* __restrict__ legit,
                                  uint64_t* __restrict__ items) {
    const CbdsCtl c = *ctl;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    uint64_t inter = 0, nleg = 0;
    for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x - (threadIdx.x & 31u); v0 < n; v0 += nth) {
        const uint64_t v = v0 + (threadIdx.x & 31u);
        uint32_t want = 0;
        if (v < n) {
            bool lg = false;
            if (is_eligible(core[v], c)) {
                const uint64_t x = cnt[v];
                lg = (unsigned __int128)x * c.Vk > c.Ek;
                if (lg) {
                    inter += x;
                    ++nleg;
                    const uint64_t len = off[v + 1] - off[v];
                    want = (uint32_t)((len + kRowChunk - 1) / kRowChunk);
                }
            }
            legit[v] = lg ? 1 : 0;
        }
        const uint64_t at = warp_reserve((unsigned long long*)&ctl->n_legit_items, want);
        emit_chunks(items, at, (uint32_t)v, want);
    }
    inter = warp_sum(inter);
    nleg = warp_sum(nleg);
    if ((threadIdx.x & 31u) == 0) {
        if (inter) atomicAdd((unsigned long long*)&ctl->inter, (unsigned long long)inter);
        if (nleg) atomicAdd((unsigned long long*)&ctl->nleg, (unsigned long long)nleg);
    }
}

uint32_t grid_for(uint32_t per_sm) { return (uint32_t)dev_info().sms * per_sm; }

// Full-occupancy grid for a kernel of kHistTB threads (at least one block per SM).
template <class K>
uint32_t occ_grid(K kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kHistTB, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return grid_for((uint32_t)per_sm);
}

}  // namespace

// Densest core (and, with phase2, the augmentation) of g for the core
// numbers core_dev (device, n).  Launches only; the caller synchronises.
// set_dev (nullable, device, n): densest core [+ legit vertices].
static dsg_status run_cbds(const dsg_graph* g, const uint32_t* core_dev, bool phase2, uint8_t* set_dev,
                           dsg_cbds_result* res) {
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    Scratch sc(s);
    CbdsCtl* ctl;
    DSG_TRY_CUDA(sc.get(&ctl, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(CbdsCtl), s));
    const uint32_t grid = grid_for(2);
    {
        LaunchScope ls("cbds_core_max", s);
        core_max_kernel<<<grid, kHistTB, 0, s>>>(core_dev, n, ctl);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    // the histograms are sized by the largest core number (a core number is below n)
    uint32_t kmax = 0;
    DSG_TRY_CUDA(cudaMemcpyAsync(&kmax, &ctl->kmax, 4, cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    if (kmax >= n) {
        set_error("invalid argument: core value %u is not below n = %u", kmax, n);
        return DSG_EINVAL;
    }
    const uint64_t K = (uint64_t)kmax + 1;
    unsigned long long *hV, *hE;
    DSG_TRY_CUDA(sc.get(&hV, K));
    DSG_TRY_CUDA(sc.get(&hE, K));
    DSG_TRY_CUDA(cudaMemsetAsync(hV, 0, K * 8, s));
    DSG_TRY_CUDA(cudaMemsetAsync(hE, 0, K * 8, s));
    {
        LaunchScope ls("cbds_core_hist", s);
        core_hist_kernel<<<occ_grid(core_hist_kernel), kHistTB, 0, s>>>(g->off, g->adj, core_dev, n, ctl, hV, hE);
    }
    {
        LaunchScope ls("cbds_densest_pick", s);
        densest_pick_kernel<<<1, kPickTB, 0, s>>>(hV, hE, ctl);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    uint8_t* legit = nullptr;
    if (phase2) {
        const uint64_t item_cap = (uint64_t)n + 2 * g->m / kRowChunk + 1;
        uint32_t* cnt;
        uint64_t* items;
        DSG_TRY_CUDA(sc.get(&cnt, n));
        DSG_TRY_CUDA(sc.get(&legit, n));
        DSG_TRY_CUDA(sc.get(&items, item_cap));
        {
            LaunchScope ls("cbds_elig_items", s);
            elig_items_kernel<<<grid, kHistTB, 0, s>>>(g->off, core_dev, n, ctl, cnt, items);
        }
        {
            LaunchScope ls("cbds_elig_count", s);
            row_chunk_count_kernel<false><<<grid, kHistTB, 0, s>>>(g->off, g->adj, core_dev, nullptr, ctl, items, cnt);
        }
        {
            LaunchScope ls("cbds_legit_mark", s);
            legit_mark_kernel<<<grid, kHistTB, 0, s>>>(g->off, core_dev, n, ctl, cnt, legit, items);
        }
        {
            LaunchScope ls("cbds_legit_pairs", s);
            row_chunk_count_kernel<true><<<grid, kHistTB, 0, s>>>(g->off, g->adj, core_dev, legit, ctl, items, nullptr);
        }
        DSG_TRY_CUDA(cudaGetLastError());
    }
    if (set_dev) {
        LaunchScope ls("cbds_set", s);
        core_mask_kernel<<<grid, kHistTB, 0, s>>>(core_dev, legit, n, ctl, set_dev);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    CbdsCtl c;
    DSG_TRY_CUDA(cudaMemcpyAsync(&c, ctl, sizeof(CbdsCtl), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    res->k_star = c.kstar;
    res->E_core = c.Ek;
    res->V_core = c.Vk;
    res->E = phase2 ? c.Ek + c.inter : c.Ek;
    res->V = phase2 ? c.Vk + c.nleg : c.Vk;
    res->n_legit = phase2 ? c.nleg : 0;
    return DSG_OK;
}

}  // namespace dsg

using namespace dsg;

static dsg_status cbds_entry(const dsg_graph* g, const uint32_t* core_in, uint32_t* out_core, uint8_t* out_set,
                             bool phase2, dsg_cbds_result* res) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    DSG_CHECK_ARG(res, "result is NULL");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    memset(res, 0, sizeof(*res));
    const uint32_t n = g->n;
    if (n == 0) return DSG_OK;
    cudaStream_t s = g->stream;
    Scratch sc(s);
    uint32_t* core = nullptr;
    if (core_in && is_device_ptr(core_in)) {
        core = const_cast<uint32_t*>(core_in);
    } else if (out_core && is_device_ptr(out_core) && !core_in) {
        core = out_core;
    } else {
        DSG_TRY_CUDA(sc.get(&core, n));
    }
    if (core_in) {
        if (core != core_in) DSG_TRY_CUDA(copy_any(core, core_in, (size_t)n * 4, s));
    } else {
        dsg_status st = run_kcore(g, core, nullptr, 0);
        if (st != DSG_OK) return st;
    }
    uint8_t* set_dev = nullptr;
    const bool set_direct = out_set && is_device_ptr(out_set);
    if (out_set) {
        if (set_direct) set_dev = out_set;
        else DSG_TRY_CUDA(sc.get(&set_dev, n));
    }
    dsg_cbds_result r;
    dsg_status st = run_cbds(g, core, phase2, set_dev, &r);
    if (st != DSG_OK) return st;
    if (out_set && !set_direct) DSG_TRY_CUDA(copy_any(out_set, set_dev, n, s));
    if (out_core && core != out_core) DSG_TRY_CUDA(copy_any(out_core, core, (size_t)n * 4, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    *res = r;
    return DSG_OK;
}

extern "C" dsg_status dsg_densest_core(const dsg_graph* g, const uint32_t* core, uint32_t* out_core,
                                       uint8_t* out_set, dsg_cbds_result* res) {
    return cbds_entry(g, core, out_core, out_set, false, res);
}

extern "C" dsg_status dsg_cbds(const dsg_graph* g, const uint32_t* core, uint32_t* out_core, uint8_t* out_set,
                               dsg_cbds_result* res) {
    return cbds_entry(g, core, out_core, out_set, true, res);
}
