// Batched solve: many independent graphs in one persistent launch.
//
// The graphs are packed as one concatenated CSR: graph g owns global vertex
// slots [vtx_base[g], vtx_base[g+1]); its row for local vertex v is
// adj[off[vtx_base[g] + v] .. off[vtx_base[g] + v + 1]) and holds LOCAL ids.
// Each block pulls the next graph from a device counter (graphs are queued
// largest first, so the long ones start early) and solves it alone: the
// Bahmani peel of Algorithm 1 and, when asked, the core numbers of
// Algorithm 2's first phase.  A round's (or level's) barrier is the block's
// __syncthreads, so a graph costs no grid-wide synchronisation; per-graph
// state lives in the concatenated scratch arrays at the graph's vertex slots.
#include <algorithm>
#include <vector>

#include "dsg_batch.cuh"
#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace dsg {

constexpr uint32_t kDeadB = 0x80000000u;

template <int TB>
struct BatchSmem {
    BlockTile<TB> tile;
    TileSmem<TB> red;
    uint64_t u64[4];
    uint32_t u32[4];
    uint32_t item;
};

__device__ __forceinline__ uint32_t b_threshold(uint64_t p, uint64_t q, uint64_t E, uint64_t S) {
    unsigned __int128 num = (unsigned __int128)2 * (unsigned __int128)(p + q) * (unsigned __int128)E;
    unsigned __int128 den = (unsigned __int128)q * (unsigned __int128)S;
    unsigned __int128 t = num / den;
    return t > (unsigned __int128)0xffffffffu ? 0xffffffffu : (uint32_t)t;
}

// Algorithm 1 on one graph by one block.
template <int TB>
__device__ void peel_block(const BatchArgs& a, uint32_t g, BatchSmem<TB>& sm) {
    const uint32_t tid = threadIdx.x;
    const uint64_t vb = a.slot[g];
    const uint32_t n = a.gn[g];
    const uint64_t* off = a.goff[g];
    const uint32_t* adj = a.gadj[g];
    uint32_t* st = a.st + vb;
    uint32_t* alive_a = a.la + vb;
    uint32_t* alive_b = a.lb + vb;
    uint32_t* failed = a.lf + vb;
    const uint64_t p = a.p[g], q = a.q[g];
    uint64_t S = n, E = n ? (off[n] - off[0]) / 2 : 0;
    uint64_t best_E = E, best_V = S, best_round = 0, r = 0;
    uint64_t sum_S = 0, ndec = 0;  // byte-model counters (thread-local; summed at the end)
    const uint32_t* alive = nullptr;
    uint32_t* next = alive_a;
    while (S > 0) {
        const uint32_t T = b_threshold(p, q, E, S);
        const uint32_t mark = kDeadB | (uint32_t)(r + 1);
        uint32_t nf = 0, ns = 0;
        if (tid == 0) sum_S += S;
        // part 1: test every alive vertex against the round-start degrees
        for (uint64_t t = 0; t < S; t += TB) {
            uint64_t i = t + tid;
            bool valid = i < S, fail = false;
            uint32_t v = 0;
            if (valid) {
                uint32_t d;
                if (r == 0) {
                    v = (uint32_t)i;
                    d = (uint32_t)(off[v + 1] - off[v]);
                } else {
                    v = alive[i];
                    d = st[v];
                }
                fail = d <= T;
                if (fail) st[v] = mark;
                else if (r == 0) st[v] = d;
            }
            uint64_t tot;
            uint64_t pk = (uint64_t)(valid && fail) | ((uint64_t)(valid && !fail) << 32);
            uint64_t pre = block_excl_scan<uint64_t>(pk, sm.red.scan_tmp64, &tot);
            if (valid && fail) failed[nf + (uint32_t)pre] = v;
            if (valid && !fail) next[ns + (uint32_t)(pre >> 32)] = v;
            nf += (uint32_t)tot;
            ns += (uint32_t)(tot >> 32);
        }
        __syncthreads();
        // part 2: remove the failed vertices' edges
        uint64_t dE = 0;
        auto visit = [&](const uint32_t* u, const uint32_t* v, uint32_t valid) {
            uint32_t w[kBatch];
#pragma unroll
            for (uint32_t j = 0; j < kBatch; ++j) w[j] = (valid >> j & 1u) ? st[u[j]] : kDeadB;
#pragma unroll
            for (uint32_t j = 0; j < kBatch; ++j) {
                if (!(valid >> j & 1u)) continue;
                if (!(w[j] & kDeadB)) {
                    atomicSub(&st[u[j]], 1u);
                    ++dE;
                    ++ndec;
                } else if (w[j] == mark && u[j] > v[j]) {
                    ++dE;
                }
            }
        };
        scan_block_list<TB>(off, adj, failed, 0, nf, sm.tile, visit);
        dE = block_sum<uint64_t>(dE, sm.red.scan_tmp64);
        ++r;
        S -= nf;
        E -= dE;
        if (S > 0 && (unsigned __int128)E * best_V > (unsigned __int128)best_E * S) {
            best_round = r;
            best_E = E;
            best_V = S;
        }
        alive = next;
        next = (next == alive_a) ? alive_b : alive_a;
    }
    if (a.stats) {
        ndec = warp_sum(ndec);
        if ((tid & 31u) == 0 && ndec) atomicAdd(&a.stats[1], (unsigned long long)ndec);
        if (tid == 0) {
            atomicAdd(&a.stats[0], (unsigned long long)sum_S);
            atomicAdd(&a.stats[2], (unsigned long long)(n ? off[n] - off[0] : 0));
        }
    }
    if (tid == 0) {
        a.res[4 * (uint64_t)g + 0] = n ? best_E : 0;
        a.res[4 * (uint64_t)g + 1] = n ? best_V : 0;
        a.res[4 * (uint64_t)g + 2] = r;
        a.res[4 * (uint64_t)g + 3] = best_round;
    }
    if (a.out_set)
        for (uint32_t v = tid; v < n; v += TB) a.out_set[vb + v] = (st[v] & ~kDeadB) > best_round ? 1 : 0;
    __syncthreads();
}

// Algorithm 2, first phase, on one graph by one block: level k collects the
// remaining vertices of degree k, then drains them (atomicSub on every
// neighbour; a == k+1 joins the level; a <= k is undone, so a vertex already
// at or below k never reads k+1 again); the level's frontier is one FIFO in
// global memory with a shared-memory cursor.
template <int TB>
__device__ void kcore_block(const BatchArgs& a, uint32_t g, BatchSmem<TB>& sm) {
    const uint32_t tid = threadIdx.x;
    const uint64_t vb = a.slot[g];
    const uint32_t n = a.gn[g];
    const uint64_t* off = a.goff[g];
    const uint32_t* adj = a.gadj[g];
    uint32_t* deg = a.core + vb;
    uint32_t* rem_a = a.la + vb;
    uint32_t* rem_b = a.lb + vb;
    uint32_t* Q = a.lf + vb;
    if (n == 0) return;
    uint32_t mn = 0xffffffffu;
    for (uint32_t v = tid; v < n; v += TB) {
        uint32_t d = (uint32_t)(off[v + 1] - off[v]);
        deg[v] = d;
        mn = min(mn, d);
    }
    uint32_t k = block_min_u32(mn, sm.red.scan_tmp);
    const uint32_t* rem = nullptr;
    uint32_t* rem_next = rem_a;
    uint32_t rem_n = n, visited = 0;
    if (tid == 0) sm.u32[0] = 0;  // FIFO cursor
    __syncthreads();
    for (;;) {
        uint32_t kept = 0, mnext = 0xffffffffu;
        for (uint32_t t = 0; t < rem_n; t += TB) {
            uint32_t i = t + tid;
            bool keep = false;
            uint32_t v = 0;
            if (i < rem_n) {
                v = rem ? rem[i] : i;
                uint32_t d = deg[v];
                if (d == k) Q[atomicAdd(&sm.u32[0], 1u)] = v;
                else if (d > k) {
                    keep = true;
                    mnext = min(mnext, d);
                }
            }
            uint32_t tot;
            uint32_t pre = block_excl_scan<uint32_t>(keep ? 1u : 0u, sm.red.scan_tmp, &tot);
            if (keep) rem_next[kept + pre] = v;
            kept += tot;
        }
        __syncthreads();
        uint32_t q_lo = visited, q_hi = sm.u32[0];
        __syncthreads();
        while (q_lo < q_hi) {
            // every neighbour loses one degree at once (no read first); one
            // already at or below k gets it back
            auto visit = [&](const uint32_t* u, const uint32_t* v, uint32_t valid) {
                uint32_t need = 0, old[kBatch];
#pragma unroll
                for (uint32_t j = 0; j < kBatch; ++j) {
                    if (!(valid >> j & 1u) || u[j] == v[j]) continue;
                    old[j] = atomicSub(&deg[u[j]], 1u);
                    need |= 1u << j;
                }
#pragma unroll
                for (uint32_t j = 0; j < kBatch; ++j) {
                    if (!(need >> j & 1u)) continue;
                    if (old[j] == k + 1) Q[atomicAdd(&sm.u32[0], 1u)] = u[j];
                    else if (old[j] <= k) atomicAdd(&deg[u[j]], 1u);
                    else mnext = min(mnext, old[j] - 1);
                }
            };
            scan_block_list<TB>(off, adj, Q, q_lo, q_hi, sm.tile, visit);
            q_lo = q_hi;
            q_hi = sm.u32[0];
            __syncthreads();
        }
        visited = q_hi;
        if (visited >= n) break;
        k = block_min_u32(mnext, sm.red.scan_tmp);
        if (k == 0xffffffffu) break;
        rem_n = kept;
        rem = rem_next;
        rem_next = (rem_next == rem_a) ? rem_b : rem_a;
    }
    __syncthreads();
}

template <int TB>
__global__ void __launch_bounds__(TB) batch_kernel(BatchArgs a) {
    __shared__ BatchSmem<TB> sm;
    for (;;) {
        if (threadIdx.x == 0) sm.item = (uint32_t)atomicAdd(a.next, 1ull);
        __syncthreads();
        const uint32_t item = sm.item;
        __syncthreads();
        if (item >= a.G) break;
        const uint32_t g = a.order[item];
        peel_block<TB>(a, g, sm);
        if (a.core && (!a.want_core || a.want_core[g])) kcore_block<TB>(a, g, sm);
    }
}

template <int TB>
static cudaError_t batch_launch_tb(const BatchArgs& a, cudaStream_t s, uint32_t max_grid) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<TB>, TB, 0);
    if (e != cudaSuccess) return e;
    uint32_t slots = (uint32_t)(per_sm > 0 ? per_sm : 1) * (uint32_t)dev_info().sms;
    if (max_grid && slots > max_grid) slots = max_grid;
    uint32_t grid = slots < a.G ? slots : a.G;
    LaunchScope ls("batch_solve", s);
    batch_kernel<TB><<<grid, TB, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t batch_launch(const BatchArgs& a, cudaStream_t s, uint32_t block, uint32_t max_grid) {
    if (a.G == 0) return cudaSuccess;
    switch (block) {
        case 256: return batch_launch_tb<256>(a, s, max_grid);
        case 1024: return batch_launch_tb<1024>(a, s, max_grid);
        default: return batch_launch_tb<512>(a, s, max_grid);
    }
}

// Block slots of the block-per-graph kernel at `block` threads.
static uint32_t batch_slots(uint32_t block) {
    int per_sm = 0;
    cudaError_t e;
    switch (block) {
        case 256: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<256>, 256, 0); break;
        case 1024: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<1024>, 1024, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<512>, 512, 0); break;
    }
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return (uint32_t)per_sm * (uint32_t)dev_info().sms;
}

uint32_t batch_slots_for(uint32_t block) { return batch_slots(block); }

// want_core[g] read from host or device memory.
static bool host_want_core(const uint8_t* want_core, uint32_t g, cudaStream_t s) {
    uint8_t w = 1;
    if (copy_any(&w, want_core + g, 1, s) != cudaSuccess) return true;
    cudaStreamSynchronize(s);
    return w != 0;
}

template <class T>
static cudaError_t to_device(Scratch& sc, const T* src, size_t count, cudaStream_t s, const T** out) {
    if (!src || count == 0) {
        *out = src;
        return cudaSuccess;
    }
    if (is_device_ptr(src)) {
        *out = src;
        return cudaSuccess;
    }
    T* d;
    cudaError_t e = sc.get(&d, count);
    if (e != cudaSuccess) return e;
    e = copy_any(d, src, count * sizeof(T), s);
    *out = d;
    return e;
}

// ends[g] = off[vb[g]] for g = 0..G: every graph's first adjacency offset
// (and the batch's end), gathered for one copy to the host.
__global__ void gather_ends_kernel(const uint64_t* __restrict__ off, const uint64_t* __restrict__ vb, uint32_t G1,
                                   uint64_t* __restrict__ ends) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < G1) ends[g] = off[vb[g]];
}

}  // namespace dsg

using namespace dsg;

extern "C" dsg_status dsg_batch_solve(const dsg_batch* b, dsg_batch_result* r, void* stream) {
    clear_error();
    DSG_CHECK_ARG(b && r, "batch / result is NULL");
    DSG_CHECK_ARG(b->vtx_base && b->off && b->eps_num && b->eps_den, "batch arrays are NULL");
    const uint32_t G = b->num_graphs;
    cudaStream_t s = (cudaStream_t)stream;
    if (G == 0) return DSG_OK;
    // host copies of the small per-graph arrays (ordering, checks)
    std::vector<uint64_t> vb(G + 1);
    std::vector<uint32_t> hp(G), hq(G);
    DSG_TRY_CUDA(copy_any(vb.data(), b->vtx_base, (G + 1) * sizeof(uint64_t), s));
    DSG_TRY_CUDA(copy_any(hp.data(), b->eps_num, G * sizeof(uint32_t), s));
    DSG_TRY_CUDA(copy_any(hq.data(), b->eps_den, G * sizeof(uint32_t), s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    DSG_CHECK_ARG(vb[0] == 0, "vtx_base[0] must be 0");
    for (uint32_t g = 0; g < G; ++g) {
        DSG_CHECK_ARG(vb[g + 1] >= vb[g], "vtx_base must not decrease");
        DSG_CHECK_ARG(vb[g + 1] - vb[g] < 0x80000000ull, "a graph has 2^31 vertices or more");
        DSG_CHECK_ARG(hq[g] != 0, "eps_den must be positive");
    }
    const uint64_t N = vb[G];
    uint64_t total = 0;
    DSG_TRY_CUDA(copy_any(&total, b->off + N, sizeof(uint64_t), s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    DSG_CHECK_ARG(total == 0 || b->adj, "adj is NULL");
    Scratch sc(s);
    const uint64_t* d_off;
    DSG_TRY_CUDA(to_device(sc, b->off, N + 1, s, &d_off));
    // largest first (by adjacency length, then vertices): every graph's first offset, gathered
    // on the device and copied in one piece
    std::vector<uint64_t> hoff_ends(G + 1);
    {
        const uint64_t* d_vb;
        DSG_TRY_CUDA(to_device(sc, vb.data(), G + 1, s, &d_vb));
        uint64_t* d_ends;
        DSG_TRY_CUDA(sc.get(&d_ends, G + 1));
        {
            LaunchScope ls("batch_ends", s);
            gather_ends_kernel<<<(G + 1 + 255) / 256, 256, 0, s>>>(d_off, d_vb, G + 1, d_ends);
        }
        DSG_TRY_CUDA(cudaGetLastError());
        DSG_TRY_CUDA(cudaMemcpyAsync(hoff_ends.data(), d_ends, (G + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        DSG_TRY_CUDA(cudaStreamSynchronize(s));
    }
    std::vector<uint32_t> order(G);
    for (uint32_t g = 0; g < G; ++g) order[g] = g;
    auto work = [&](uint32_t x) { return (hoff_ends[x + 1] - hoff_ends[x]) + (vb[x + 1] - vb[x]); };
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return work(x) > work(y); });
    BatchArgs a;
    a.G = G;
    const uint32_t* d_adj;
    DSG_TRY_CUDA(to_device(sc, b->adj, total, s, &d_adj));
    DSG_TRY_CUDA(to_device(sc, b->eps_num, G, s, &a.p));
    DSG_TRY_CUDA(to_device(sc, b->eps_den, G, s, &a.q));
    DSG_TRY_CUDA(to_device(sc, b->want_core, b->want_core ? G : 0, s, &a.want_core));
    {
        std::vector<const uint64_t*> hoffp(G);
        std::vector<const uint32_t*> hadjp(G);
        std::vector<uint32_t> hn(G);
        for (uint32_t g = 0; g < G; ++g) {
            hoffp[g] = d_off + vb[g];
            hadjp[g] = d_adj;
            hn[g] = (uint32_t)(vb[g + 1] - vb[g]);
        }
        const uint64_t** t_off;
        const uint32_t** t_adj;
        uint64_t* t_slot;
        uint32_t* t_n;
        DSG_TRY_CUDA(sc.get(&t_off, G));
        DSG_TRY_CUDA(sc.get(&t_adj, G));
        DSG_TRY_CUDA(sc.get(&t_slot, G));
        DSG_TRY_CUDA(sc.get(&t_n, G));
        DSG_TRY_CUDA(copy_any(t_off, hoffp.data(), G * sizeof(void*), s));
        DSG_TRY_CUDA(copy_any(t_adj, hadjp.data(), G * sizeof(void*), s));
        DSG_TRY_CUDA(copy_any(t_slot, vb.data(), G * sizeof(uint64_t), s));
        DSG_TRY_CUDA(copy_any(t_n, hn.data(), G * sizeof(uint32_t), s));
        a.goff = t_off;
        a.gadj = t_adj;
        a.slot = t_slot;
        a.gn = t_n;
        // the tables live in stream-ordered scratch: keep the host vectors alive until the copies ran
        DSG_TRY_CUDA(cudaStreamSynchronize(s));
    }
    uint32_t* d_order;
    DSG_TRY_CUDA(sc.get(&d_order, G));
    DSG_TRY_CUDA(copy_any(d_order, order.data(), G * sizeof(uint32_t), s));
    a.order = d_order;
    DSG_TRY_CUDA(sc.get(&a.st, N ? N : 1));
    DSG_TRY_CUDA(sc.get(&a.la, N ? N : 1));
    DSG_TRY_CUDA(sc.get(&a.lb, N ? N : 1));
    DSG_TRY_CUDA(sc.get(&a.lf, N ? N : 1));
    bool core_direct = r->core && is_device_ptr(r->core);
    bool set_direct = r->out_set && is_device_ptr(r->out_set);
    a.core = nullptr;
    if (r->core) {
        if (core_direct) {
            a.core = r->core;
        } else {
            // start from the caller's values so graphs without core numbers stay untouched
            DSG_TRY_CUDA(sc.get(&a.core, N ? N : 1));
            DSG_TRY_CUDA(copy_any(a.core, r->core, N * sizeof(uint32_t), s));
        }
    }
    a.out_set = nullptr;
    if (r->out_set) {
        if (set_direct) a.out_set = r->out_set;
        else DSG_TRY_CUDA(sc.get(&a.out_set, N ? N : 1));
    }
    DSG_TRY_CUDA(sc.get(&a.res, 4 * (size_t)G));
    DSG_TRY_CUDA(sc.get(&a.next, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(a.next, 0, sizeof(unsigned long long), s));
    // Scheduling: a graph whose work is well above one block's share of the
    // batch would alone set the batch's makespan, so it is solved first by
    // the grid-wide kernels; the rest share one block-per-graph launch.
    uint64_t total_work = 0;
    for (uint32_t g = 0; g < G; ++g) total_work += work(g);
    const Tuning tu = tuning_for_batch(G, total_work);
    a.hot_deg = tu.hot_deg;
    const uint32_t block = tu.batch_block ? tu.batch_block : 512;
    const uint32_t slots = batch_slots(block);
    unsigned long long* d_stats = nullptr;
    if (r->stats) {
        DSG_TRY_CUDA(sc.get(&d_stats, 3));
        DSG_TRY_CUDA(cudaMemsetAsync(d_stats, 0, 3 * sizeof(unsigned long long), s));
    }
    a.stats = d_stats;
    uint64_t big_sum_S = 0, big_dec = 0, big_entries = 0;
    const uint64_t share = total_work / slots;
    uint32_t nbig = 0;
    if (tu.batch_split)
        while (nbig < G && work(order[nbig]) > tu.batch_split) ++nbig;
    else
        while (nbig < G && work(order[nbig]) > 2 * share && work(order[nbig]) > (1u << 20)) ++nbig;
    std::vector<uint64_t> res(4 * (size_t)G, 0);
    for (uint32_t i = 0; i < nbig; ++i) {
        const uint32_t g = order[i];
        dsg_graph view;
        view.n = (uint32_t)(vb[g + 1] - vb[g]);
        view.m = (hoff_ends[g + 1] - hoff_ends[g]) / 2;
        view.off = const_cast<uint64_t*>(d_off) + vb[g];
        view.adj = const_cast<uint32_t*>(d_adj);
        view.owns = false;
        DSG_TRY_CUDA(cudaGetDevice(&view.device));
        view.stream = s;
        uint64_t extra[2] = {0, 0};
        dsg_status st = peel_into(&view, hp[g], hq[g], a.out_set ? a.out_set + vb[g] : nullptr, &res[4 * (size_t)g],
                                  r->stats ? extra : nullptr);
        if (st != DSG_OK) return st;
        big_sum_S += extra[0];
        big_dec += extra[1];
        big_entries += 2 * view.m;
        bool want = a.core && (!b->want_core || host_want_core(b->want_core, g, s));
        if (want) {
            st = run_kcore(&view, a.core + vb[g], nullptr, 0);
            if (st != DSG_OK) return st;
        }
    }
    const uint32_t nsmall = G - nbig;
    a.order = d_order + nbig;
    a.G = nsmall;
    if (nsmall) DSG_TRY_CUDA(batch_launch(a, s, block));
    DSG_TRY_CUDA(cudaGetLastError());
    std::vector<uint64_t> res_dev(4 * (size_t)G);
    DSG_TRY_CUDA(cudaMemcpyAsync(res_dev.data(), a.res, res_dev.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    if (r->core && !core_direct) DSG_TRY_CUDA(copy_any(r->core, a.core, N * sizeof(uint32_t), s));
    if (r->out_set && !set_direct) DSG_TRY_CUDA(copy_any(r->out_set, a.out_set, N, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    for (uint32_t i = nbig; i < G; ++i) {
        const uint32_t g = order[i];
        for (int k = 0; k < 4; ++k) res[4 * (size_t)g + k] = res_dev[4 * (size_t)g + k];
    }
    for (uint32_t g = 0; g < G; ++g) {
        if (r->E) r->E[g] = res[4 * (size_t)g + 0];
        if (r->V) r->V[g] = res[4 * (size_t)g + 1];
        if (r->rounds) r->rounds[g] = res[4 * (size_t)g + 2];
        if (r->best_round) r->best_round[g] = res[4 * (size_t)g + 3];
    }
    if (r->stats) {
        unsigned long long h[3] = {0, 0, 0};
        DSG_TRY_CUDA(cudaMemcpy(h, d_stats, sizeof(h), cudaMemcpyDeviceToHost));
        r->stats[0] = h[0] + big_sum_S;
        r->stats[1] = h[1] + big_dec;
        r->stats[2] = h[2] + big_entries;
        r->stats[3] = nbig;
    }
    return DSG_OK;
}
