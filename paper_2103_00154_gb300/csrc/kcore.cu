// Core numbers by the level-synchronous peel of Algorithm 2's first phase
// (PKC), as one persistent cooperative kernel.
//
// Level k (Alg. 2 first phase):
//   phase A: scan the remaining vertices; degree == k joins the level's
//     frontier (Alg. 2 "if v.deg = k: buff[end++] <- v"), degree > k stays in
//     the (compacted) remaining list, degree < k was finished at an earlier
//     level and drops out;
//   grid barrier;
//   drain, in sub-rounds separated by grid barriers: for every frontier vertex
//     v and neighbour u with deg[u] > k, a = atomicSub(deg[u], 1); a == k+1
//     puts u in the frontier (it just reached k); a <= k is undone with
//     atomicAdd (another thread got there first) -- Alg. 2's drain loop;
//   the level ends when a sub-round adds nothing; "visited" grows by the
//   frontier size (Alg. 2 "atomicAdd(visited, end)").
// Empty levels are skipped: the next k is the least degree above k among the
// remaining vertices, tracked with atomicMin during the scan and the drain
// (never above the true minimum, so no level with work is skipped).
// When visited == n, deg[v] is the core number of v.
//
// Counter discipline (no barrier is wasted, yet no block reads a counter that
// a faster block may already be changing): the scan's frontier, push count
// and remaining-list cursor are written only in scans and read right after the
// scan's barrier; the drain's are written only in drains and read right after
// a drain barrier.  Every level runs at least one drain sub-round, so a scan
// and the next scan are always separated by a barrier.
#include <cooperative_groups.h>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace cg = cooperative_groups;

namespace dsg {

struct __align__(128) CoreCtl {
    uint32_t bar;
    uint32_t pad0[31];
    uint32_t err;
    uint32_t pad1[31];
    // Counters written in the level scan (phase A) and read only after the
    // scan's barrier, and counters written in the drain and read only after a
    // drain barrier: each is stable between its barrier and the next phase
    // that writes it, which is always at least one barrier later.
    unsigned long long qa_tail;  // scan frontier, short rows (all levels)
    unsigned long long pad2[15];
    unsigned long long ca_tail;  // scan frontier, chunk items (all levels)
    unsigned long long pad3[15];
    unsigned long long pushedA;  // vertices put in a frontier by scans
    unsigned long long pad4[15];
    unsigned long long qtail;    // drain frontier, short rows (all levels)
    unsigned long long pad8[15];
    unsigned long long ctail;    // drain frontier, chunk items (all levels)
    unsigned long long pad9[15];
    unsigned long long pushedD;  // vertices put in a frontier by drains
    unsigned long long pad10[15];
    unsigned long long keep;     // remaining-list writes (all levels)
    unsigned long long pad5[15];
    uint32_t next_min[2];
    uint32_t pad6[30];
    unsigned long long atomics;  // degree atomics (decrements + undos)
    unsigned long long pad7[15];
    unsigned long long levels, subrounds, rem_scanned, rem_written;
    unsigned long long dbg[4];   // bounds-check builds: first bad access (site, index, capacity, level)
    unsigned long long stamps;
};

// Bounds checks of the debug build (DSG_DEBUG_BOUNDS): a bad index is
// recorded once in ctl->dbg and the access is skipped.
#ifdef DSG_DEBUG_BOUNDS
#define DSG_BOUND(ctl, site, idx, cap, lvl, skip)                                                      \
    do {                                                                                              \
        if ((uint64_t)(idx) >= (uint64_t)(cap)) {                                                     \
            if (atomicOr(&(ctl)->err, ERR_RANGE) == 0 || true) {                                      \
                if (atomicCAS(&(ctl)->dbg[0], 0ull, (unsigned long long)(site)) == 0) {               \
                    (ctl)->dbg[1] = (idx);                                                            \
                    (ctl)->dbg[2] = (cap);                                                            \
                    (ctl)->dbg[3] = (lvl);                                                            \
                }                                                                                     \
            }                                                                                         \
            skip;                                                                                     \
        }                                                                                             \
    } while (0)
#else
#define DSG_BOUND(ctl, site, idx, cap, lvl, skip) do { } while (0)
#endif

struct CoreArgs {
    uint32_t n;
    const uint64_t* off;
    const uint32_t* adj;
    uint32_t* deg;
    uint32_t* remA;
    uint32_t* remB;
    uint32_t* QA;   // frontier found by the level scans
    uint64_t* CA;
    uint32_t* Q;    // frontier found while draining
    uint64_t* C;
    CoreCtl* ctl;
    uint64_t limit_ns;
    uint32_t short_max;
    uint32_t chunk_len;
    uint32_t hot_deg;
    uint32_t local_max;   // rows up to this length found while draining stay in the block
    uint32_t local_work;  // ... while the block's local entries this sub-round stay within this
    uint64_t chunk_cap;
    uint64_t* trace;      // nullable: block 0 stamps (%globaltimer, kind) after every barrier
    uint64_t trace_cap;
};

// Block-local frontier: vertices that reach k while this block drains are
// drained by the same block in the same sub-round (PKC's thread-local buff,
// Algorithm 2), so a chain of degree-k vertices costs no grid barrier per
// link.  Overflow goes to the global frontier of the next sub-round.
constexpr uint32_t kLocalQ = 1024;

template <int TB>
struct CoreSmem {
    TileSmem<TB> tile;
    BlockTile<TB> btile;
    AggTable agg;
    uint32_t lq[kLocalQ];
    uint32_t lq_tail;
    uint32_t lq_work;  // row entries this block has taken on locally in this sub-round
    uint64_t bases[4];
    uint64_t red[33];
    uint32_t redm[33];
};

// Put v (row length len) into a frontier: short rows by id into Q (cursor
// *qt), long rows as chunk items into C (cursor *ct).  Called by any subset of
// lanes; short pushes are aggregated over the lanes that take this path
// together.
__device__ __forceinline__ void push_frontier(const CoreArgs& a, uint32_t* Q, unsigned long long* qt, uint64_t* C,
                                              unsigned long long* ct, uint32_t v, uint64_t len) {
    if (len <= a.short_max) {
        cg::coalesced_group g = cg::coalesced_threads();
        unsigned long long base = 0;
        if (g.thread_rank() == 0) base = atomicAdd(qt, (unsigned long long)g.size());
        base = g.shfl(base, 0);
        DSG_BOUND(a.ctl, 1, base + g.thread_rank(), a.n, 0, return);
        Q[base + g.thread_rank()] = v;
    } else {
        uint64_t nch = (len + a.chunk_len - 1) / a.chunk_len;
        unsigned long long c0 = atomicAdd(ct, (unsigned long long)nch);
        DSG_BOUND(a.ctl, 2, c0 + nch - 1, a.chunk_cap, 0, return);
        for (uint64_t c = 0; c < nch; ++c) C[c0 + c] = ((uint64_t)v << 32) | c;
    }
}

template <int TB>
__global__ void __launch_bounds__(TB) kcore_kernel(CoreArgs a) {
    __shared__ CoreSmem<TB> sm;
    CoreCtl* ctl = a.ctl;
    const uint32_t tid = threadIdx.x;
    const uint32_t n = a.n;
    uint64_t nstamp = 0;
    // trace entries: 2 words each, (time, kind << 32 | k); kind 0 start, 1 init, 2 scan, 3 drain
    auto stamp = [&](uint32_t kind, uint32_t kk) {
        if (a.trace && blockIdx.x == 0 && tid == 0 && 2 * nstamp + 1 < a.trace_cap) {
            a.trace[2 * nstamp] = global_ns();
            a.trace[2 * nstamp + 1] = ((uint64_t)kind << 32) | kk;
        }
        ++nstamp;
    };
    stamp(0, 0);
    agg_clear(sm.agg);
    const uint32_t hot = hot_threshold(a.hot_deg);
    // ---- init: deg = row length; least degree -> first level
    {
        uint32_t mn = 0xffffffffu;
        for (uint64_t v = (uint64_t)blockIdx.x * TB + tid; v < n; v += (uint64_t)gridDim.x * TB) {
            uint32_t d = (uint32_t)(a.off[v + 1] - a.off[v]);
            a.deg[v] = d;
            mn = min(mn, d);
        }
        mn = block_min_u32(mn, sm.redm);
        if (tid == 0 && mn != 0xffffffffu) atomicMin(&ctl->next_min[0], mn);
    }
    if (!grid_barrier(&ctl->bar, &ctl->err, a.limit_ns)) return;
    stamp(1, 0);
    uint32_t k = ld_relaxed_u32(&ctl->next_min[0]);
    uint64_t rem_n = n, keep_base = 0;
    const uint32_t* rem = nullptr;  // level 0: identity
    uint32_t* rem_next = a.remA;
    uint64_t q_lo = 0, c_lo = 0, qa_lo = 0, ca_lo = 0;
    uint64_t level = 0, subrounds = 0, rem_scanned = 0, rem_written = 0;
    for (;;) {
        rem_scanned += rem_n;
        const uint32_t par_next = (uint32_t)((level + 1) & 1);
        // ------------------------------------------ phase A: level scan
        uint32_t mn = 0xffffffffu;
        uint64_t pushed = 0;
        for (uint64_t t = (uint64_t)blockIdx.x * TB; t < rem_n; t += (uint64_t)gridDim.x * TB) {
            uint64_t i = t + tid;
            bool keep = false;
            uint32_t v = 0;
            if (i < rem_n) {
                v = rem ? rem[i] : (uint32_t)i;
                uint32_t d = a.deg[v];
                if (d == k) {
                    push_frontier(a, a.QA, &ctl->qa_tail, a.CA, &ctl->ca_tail, v, a.off[v + 1] - a.off[v]);
                    ++pushed;
                } else if (d > k) {
                    keep = true;
                    mn = min(mn, d);
                }
            }
            uint32_t tot;
            uint32_t pre = block_excl_scan<uint32_t>(keep ? 1u : 0u, sm.tile.scan_tmp, &tot);
            if (tid == 0) sm.bases[0] = tot ? atomicAdd(&ctl->keep, (unsigned long long)tot) : 0;
            __syncthreads();
            if (keep) {
                DSG_BOUND(ctl, 3, sm.bases[0] - keep_base + pre, n, level, keep = false);
                if (keep) rem_next[sm.bases[0] - keep_base + pre] = v;
            }
            __syncthreads();
        }
        uint32_t bmn = block_min_u32(mn, sm.redm);
        if (tid == 0 && bmn != 0xffffffffu) atomicMin(&ctl->next_min[par_next], bmn);
        uint64_t bp = block_sum<uint64_t>(pushed, sm.red);
        if (tid == 0 && bp) atomicAdd(&ctl->pushedA, (unsigned long long)bp);
        if (!grid_barrier(&ctl->bar, &ctl->err, a.limit_ns)) return;
        stamp(2, k);
        // the level's k has been read by every block: recycle its slot
        if (blockIdx.x == 0 && tid == 0) ctl->next_min[level & 1] = 0xffffffffu;
        // scan-written counters: stable until the next level's scan, which is
        // at least one drain barrier away
        const uint64_t kept = ld_relaxed_u64(&ctl->keep) - keep_base;
        const uint64_t qa_hi = ld_relaxed_u64(&ctl->qa_tail);
        const uint64_t ca_hi = ld_relaxed_u64(&ctl->ca_tail);
        const uint64_t pushedA = ld_relaxed_u64(&ctl->pushedA);
        uint64_t q_hi = q_lo, c_hi = c_lo;
        // ------------------------------------------ drain in sub-rounds
        // sub-round 0 walks the scan frontier (always run, so every level has a
        // barrier between its scan and the next); later ones walk the drain's
        for (bool first = true; first || q_lo < q_hi || c_lo < c_hi; first = false) {
            uint32_t dmn = 0xffffffffu;
            uint64_t dpushed = 0, natom = 0;
            uint32_t* deg = a.deg;
            // u reached k: drain it in this block if there is room, else globally
            auto reach_k = [&](uint32_t u) {
                uint64_t len = a.off[u + 1] - a.off[u];
                ++dpushed;
                // keep it in the block while the block's own share stays small:
                // past local_work entries a grid-wide sub-round is cheaper
                if (len <= a.local_max && atomicAdd(&sm.lq_work, (uint32_t)len) + len <= a.local_work) {
                    uint32_t pos = atomicAdd(&sm.lq_tail, 1u);
                    if (pos < kLocalQ) {
                        sm.lq[pos] = u;
                        return;
                    }
                }
                push_frontier(a, a.Q, &ctl->qtail, a.C, &ctl->ctail, u, len);
            };
            // c was just taken from u's degree, which was old: keep what brings
            // it down to k, give back the rest (Algorithm 2's undo, for c units),
            // and report the crossing into k
            auto settle = [&](uint32_t u, uint32_t old, uint32_t c) {
                if (old <= k) {
                    atomicAdd(&deg[u], c);
                    ++natom;
                    return;
                }
                uint32_t legit = min(c, old - k);
                if (legit < c) {
                    atomicAdd(&deg[u], c - legit);
                    ++natom;
                }
                uint32_t nv = old - legit;
                if (nv == k) reach_k(u);
                else dmn = min(dmn, nv);
            };
            auto visit = [&](const uint32_t* u, const uint32_t* v, uint32_t valid) {
                uint32_t d[kBatch], old[kBatch], need = 0;
#pragma unroll
                for (uint32_t j = 0; j < kBatch; ++j) {
                    if (!(valid >> j & 1u)) continue;
#ifdef DSG_DEBUG_BOUNDS
                    if (u[j] >= n) {
                        DSG_BOUND(ctl, 4, u[j], n, level, (void)0);
                        continue;
                    }
#endif
                    if (u[j] == v[j]) continue;
                    d[j] = deg[u[j]];
                    need |= 1u << j;
                }
#pragma unroll
                for (uint32_t j = 0; j < kBatch; ++j) {
                    if (!(need >> j & 1u)) continue;
                    if (d[j] <= k || (d[j] >= hot && agg_add(sm.agg, u[j]))) {
                        need &= ~(1u << j);  // already at k, or settled at the flush
                        continue;
                    }
                    old[j] = atomicSub(&deg[u[j]], 1u);
                    ++natom;
                }
#pragma unroll
                for (uint32_t j = 0; j < kBatch; ++j)
                    if (need >> j & 1u) settle(u[j], old[j], 1u);
            };
            auto flush = [&]() {
                __syncthreads();
                for (uint32_t i = tid; i < kAggSlots; i += TB) {
                    uint32_t key = sm.agg.key[i];
                    if (key != kAggEmpty) {
                        uint32_t c = sm.agg.cnt[i];
                        sm.agg.key[i] = kAggEmpty;
                        sm.agg.cnt[i] = 0;
                        uint32_t old = atomicSub(&deg[key], c);
                        ++natom;
                        settle(key, old, c);
                    }
                }
                __syncthreads();
            };
            if (tid == 0) {
                sm.lq_tail = 0;
                sm.lq_work = 0;
            }
            __syncthreads();
            if (first)
                scan_frontier<TB>(a.off, a.adj, a.QA, qa_lo, qa_hi, a.CA, ca_lo, ca_hi, a.chunk_len, visit, n);
            else
                scan_frontier<TB>(a.off, a.adj, a.Q, q_lo, q_hi, a.C, c_lo, c_hi, a.chunk_len, visit, n);
            flush();
            // drain what this block found, until it finds nothing more
            for (uint32_t lq_lo = 0;;) {
                uint32_t lq_hi = min(sm.lq_tail, kLocalQ);
                __syncthreads();
                if (lq_lo >= lq_hi) break;
                scan_block_list<TB>(a.off, a.adj, sm.lq, lq_lo, lq_hi, sm.btile, visit);
                flush();
                lq_lo = lq_hi;
            }
            uint32_t b2 = block_min_u32(dmn, sm.redm);
            if (tid == 0 && b2 != 0xffffffffu) atomicMin(&ctl->next_min[par_next], b2);
            uint64_t bp2 = block_sum<uint64_t>(dpushed, sm.red);
            if (tid == 0 && bp2) atomicAdd(&ctl->pushedD, (unsigned long long)bp2);
            uint64_t ba = block_sum<uint64_t>(natom, sm.red);
            if (tid == 0 && ba) atomicAdd(&ctl->atomics, (unsigned long long)ba);
            if (!grid_barrier(&ctl->bar, &ctl->err, a.limit_ns)) return;
            stamp(3, k);
            ++subrounds;
            q_lo = q_hi;
            c_lo = c_hi;
            q_hi = ld_relaxed_u64(&ctl->qtail);
            c_hi = ld_relaxed_u64(&ctl->ctail);
        }
        ++level;
        qa_lo = qa_hi;
        ca_lo = ca_hi;
        // drain-written counter: stable until the next level's drain
        const uint64_t visited = pushedA + ld_relaxed_u64(&ctl->pushedD);
        if (visited >= n) break;
        k = ld_relaxed_u32(&ctl->next_min[par_next]);
        if (k == 0xffffffffu) {  // nothing left above k yet visited < n: cannot happen on valid input
            if (blockIdx.x == 0 && tid == 0) atomicOr(&ctl->err, ERR_CAPACITY);
            break;
        }
        keep_base += kept;
        rem_written += kept;
        rem_n = kept;
        rem = rem_next;
        rem_next = (rem_next == a.remA) ? a.remB : a.remA;
    }
    if (blockIdx.x == 0 && tid == 0) {
        ctl->stamps = nstamp;
        ctl->levels = level;
        ctl->subrounds = subrounds;
        ctl->rem_scanned = rem_scanned;
        ctl->rem_written = rem_written;
    }
}

template <int TB>
static cudaError_t launch_kcore(CoreArgs& a, uint32_t blocks_per_sm, cudaStream_t s) {
    uint32_t grid = 1;
    cudaError_t e = coop_grid(kcore_kernel<TB>, TB, 0, a.n, blocks_per_sm, &grid);
    if (e != cudaSuccess) return e;
    void* params[] = {&a};
    LaunchScope ls("kcore_levels", s);
    return cudaLaunchCooperativeKernel((const void*)kcore_kernel<TB>, dim3(grid), dim3(TB), params, 0, s);
}

dsg_status run_kcore(const dsg_graph* g, uint32_t* core_out, uint64_t* stats, uint32_t nstats,
                     uint64_t* trace_dev, uint64_t trace_cap, uint64_t* stamps) {
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    if (n == 0) return DSG_OK;
    const Tuning tu = tuning_for(g, 1);
    const uint64_t chunk_cap = (uint64_t)n + (2 * g->m) / tu.chunk_len + 1;
    Scratch sc(s);
    CoreArgs a;
    a.n = n;
    a.off = g->off;
    a.adj = g->adj;
    a.limit_ns = wait_limit_ns();
    a.short_max = tu.short_max;
    a.chunk_len = tu.chunk_len;
    a.chunk_cap = chunk_cap;
    a.hot_deg = tu.hot_deg;
    a.local_max = tu.local_max;
    a.local_work = tu.local_work;
    a.trace = trace_dev;
    a.trace_cap = trace_cap;
    bool direct = is_device_ptr(core_out);
    if (direct) a.deg = core_out;
    else DSG_TRY_CUDA(sc.get(&a.deg, n));
    DSG_TRY_CUDA(sc.get(&a.remA, n));
    DSG_TRY_CUDA(sc.get(&a.remB, n));
    DSG_TRY_CUDA(sc.get(&a.QA, n));
    DSG_TRY_CUDA(sc.get(&a.CA, chunk_cap));
    DSG_TRY_CUDA(sc.get(&a.Q, n));
    DSG_TRY_CUDA(sc.get(&a.C, chunk_cap));
    DSG_TRY_CUDA(sc.get(&a.ctl, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(a.ctl, 0, sizeof(CoreCtl), s));
    DSG_TRY_CUDA(cudaMemsetAsync(&a.ctl->next_min[0], 0xff, 2 * sizeof(uint32_t), s));
    cudaError_t e;
    switch (tu.block) {
        case 256: e = launch_kcore<256>(a, tu.blocks_per_sm, s); break;
        case 1024: e = launch_kcore<1024>(a, tu.blocks_per_sm, s); break;
        default: e = launch_kcore<512>(a, tu.blocks_per_sm, s); break;
    }
    DSG_TRY_CUDA(e);
    CoreCtl c;
    DSG_TRY_CUDA(cudaMemcpyAsync(&c, a.ctl, sizeof(CoreCtl), cudaMemcpyDeviceToHost, s));
    if (!direct) DSG_TRY_CUDA(copy_any(core_out, a.deg, (size_t)n * 4, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    if (c.dbg[0]) {
        set_error("kcore bounds check: site %llu index %llu capacity %llu level %llu", c.dbg[0], c.dbg[1], c.dbg[2],
                  c.dbg[3]);
        return DSG_ECUDA;
    }
    if (stamps) *stamps = c.stamps;
    const uint64_t vals[5] = {c.levels, c.subrounds, c.rem_scanned, c.rem_written, c.atomics};
    for (uint32_t i = 0; stats && i < nstats && i < 5; ++i) stats[i] = vals[i];
    return status_from_err(c.err, "kcore");
}

}  // namespace dsg

using namespace dsg;

extern "C" dsg_status dsg_kcore(const dsg_graph* g, uint32_t* out_core) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    DSG_CHECK_ARG(out_core || g->n == 0, "out_core is NULL");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    return run_kcore(g, out_core, nullptr, 0);
}

extern "C" dsg_status dsg_kcore_stats(const dsg_graph* g, uint32_t* out_core, uint64_t* stats, uint32_t nstats) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    DSG_CHECK_ARG(out_core || g->n == 0, "out_core is NULL");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    return run_kcore(g, out_core, stats, nstats);
}

// Level timestamps of one core decomposition (debug/analysis): pairs
// (%globaltimer, kind << 32 | k) after every grid barrier; kind 0 = start,
// 1 = init, 2 = level scan, 3 = drain sub-round.  *count = pairs taken.
extern "C" dsg_status dsg_debug_kcore_trace(const dsg_graph* g, uint64_t* ts, uint64_t cap, uint64_t* count) {
    clear_error();
    DSG_CHECK_ARG(g && ts && cap >= 2, "graph/ts/cap");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    Scratch sc(g->stream);
    uint64_t* dts;
    uint32_t* core;
    DSG_TRY_CUDA(sc.get(&dts, cap));
    DSG_TRY_CUDA(sc.get(&core, g->n ? g->n : 1));
    uint64_t stamps = 0;
    dsg_status st = run_kcore(g, core, nullptr, 0, dts, cap, &stamps);
    if (st != DSG_OK) return st;
    uint64_t k = 2 * stamps < cap ? 2 * stamps : cap;
    DSG_TRY_CUDA(copy_any(ts, dts, k * 8, g->stream));
    DSG_TRY_CUDA(cudaStreamSynchronize(g->stream));
    if (count) *count = stamps;
    return DSG_OK;
}
