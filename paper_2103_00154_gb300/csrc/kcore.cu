// Core numbers by the level-synchronous peel of Algorithm 2's first phase
// (PKC), as one persistent cooperative kernel.
//
// Level k (Alg. 2 first phase), in sub-rounds separated by grid barriers:
//   sub-round 0 scans the remaining vertices: degree <= k joins the level's
//     frontier (Alg. 2 "if v.deg = k: buff[end++] <- v"), degree > k stays in
//     the (compacted) remaining list; each block then drains the vertices it
//     found itself: for every frontier vertex v and neighbour u with
//     deg[u] > k, a = atomicSub(deg[u], 1); a == k+1 puts u in the frontier
//     (it just reached k); a <= k is undone with atomicAdd (another thread got
//     there first) -- Alg. 2's drain loop;
//   later sub-rounds drain the vertices that reached k and did not fit the
//     finding block's own queue;
//   the level ends when a sub-round adds nothing; "visited" grows by the
//   frontier size (Alg. 2 "atomicAdd(visited, end)").
// Scanning and draining share sub-round 0, so a level with no cascade costs
// one grid barrier.  Because other blocks' drains run while a block scans, a
// vertex is taken into a frontier by claiming its bit in a bitmap (atomicOr):
// whichever of the scan and the drain that brought it to k claims it first
// drains it, exactly once.  A scanned degree below k can only be such a
// vertex caught between a decrement and its undo: every vertex whose degree
// was below k at the level's start was claimed at an earlier level.
// Empty levels are skipped: the next k is the least degree above k seen by the
// scan and by every decrement of the level (the last value each vertex takes
// is among them, so no level with work is skipped).
// When visited == n, deg[v] is the core number of v.
//
// Counters that blocks read after a barrier (frontier sizes, claims, the
// remaining-list cursor, the least degree) live in a ring of three slots
// indexed by the sub-round: sub-round j adds into slot j % 3, every block
// reads it after barrier j, and block 0 clears slot (j + 1) % 3 during
// sub-round j -- after every block has read it (two barriers earlier) and
// before anyone adds into it (after barrier j).
#include <string.h>

#include <cooperative_groups.h>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace cg = cooperative_groups;

namespace dsg {

struct __align__(128) CoreSlot {
    unsigned long long qcnt;    // drain-frontier short rows pushed
    unsigned long long ccnt;    // chunk items pushed
    unsigned long long pushed;  // vertices claimed
    uint32_t nmin;              // least degree above k seen
    uint32_t pad[25];
};

struct __align__(128) CoreCtl {
    uint32_t bar;
    uint32_t pad0[31];
    uint32_t err;
    uint32_t pad1[31];
    uint32_t init_min;
    uint32_t pad2[31];
    CoreSlot slot[3];
    unsigned long long atomics;  // degree atomics (decrements + undos), never read in the kernel
    unsigned long long pad3[15];
    unsigned long long rem_scanned, rem_written;  // statistics, summed by every block
    unsigned long long levels, subrounds;
    unsigned long long dbg[4];   // bounds-check builds: first bad access (site, index, capacity, level)
    unsigned long long stamps;
};

// Bounds checks of the debug build (DSG_DEBUG_BOUNDS): a bad index is
// recorded once in ctl->dbg and the access is skipped.
#ifdef DSG_DEBUG_BOUNDS
#define DSG_BOUND(ctl, site, idx, cap, lvl, skip)                                                      \
    do {                                                                                              \
        if ((uint64_t)(idx) >= (uint64_t)(cap)) {                                                     \
            atomicOr(&(ctl)->err, ERR_RANGE);                                                         \
            if (atomicCAS(&(ctl)->dbg[0], 0ull, (unsigned long long)(site)) == 0) {                   \
                (ctl)->dbg[1] = (idx);                                                                \
                (ctl)->dbg[2] = (cap);                                                                \
                (ctl)->dbg[3] = (lvl);                                                                \
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
    uint32_t* claim;  // one bit per vertex: taken into a frontier
    uint32_t* remA;   // per-block segments: the vertices each block's scan keeps
    uint32_t* remB;
    uint32_t* QA;     // per-block segments: vertices the block's scan claimed ...
    uint64_t* QB;     // ... their row starts
    uint32_t* QL;     // ... and row lengths
    uint64_t seg;     // segment length per block
    uint32_t* Q;      // drain frontier (short rows), all levels ...
    uint64_t* QgB;    // ... their row starts
    uint32_t* QgL;    // ... and row lengths
    uint64_t* C;      // chunk items (long rows), all levels
    CoreCtl* ctl;
    uint64_t limit_ns;
    uint32_t short_max;
    uint32_t chunk_len;
    uint32_t hot_deg;
    uint32_t local_max;   // rows up to this length found while draining stay in the block
    uint32_t local_work;  // ... while the block's local entries this sub-round stay within this
    uint32_t inline_max;  // rows up to this length claimed by a block's scan may be drained by that block
    uint64_t chunk_cap;
    uint64_t* trace;      // nullable: block 0 stamps (%globaltimer, kind) after every barrier
    uint64_t trace_cap;
};

// Block-local frontier: vertices that reach k while this block drains are
// drained by the same block in the same sub-round (PKC's thread-local buff,
// Algorithm 2), so a chain of degree-k vertices costs no grid barrier per
// link.  Overflow goes to the global frontier of the next sub-round.
template <int TB>
constexpr uint32_t local_q_cap() { return TB >= 1024 ? 640 : 1024; }

template <int TB>
struct CoreSmem {
    static constexpr uint32_t kLocalQ = local_q_cap<TB>();
    TileSmem<TB> tile;
    BlockTile<TB> btile;
    AggTable agg;
    uint32_t lq[kLocalQ];   // vertices ...
    uint64_t lqb[kLocalQ];  // ... their row starts
    uint32_t lql[kLocalQ];  // ... and row lengths
    uint32_t lq_tail;
    uint32_t lq_work;  // row entries this block has taken on locally in this sub-round
    uint32_t own;      // vertices this block's scan claimed in this sub-round
    uint32_t kept;     // vertices this block's scan kept
    uint32_t acc_min;  // block reductions at the end of a sub-round
    unsigned long long acc_pushed, acc_atomics;
    uint64_t bases[4];
    uint64_t red[33];
    uint32_t redm[33];
};

// Claim v for a frontier; true for exactly one caller.
__device__ __forceinline__ bool claim_vertex(uint32_t* claim, uint32_t v) {
    const uint32_t bit = 1u << (v & 31u);
    return !(atomicOr(&claim[v >> 5], bit) & bit);
}

// Put v (row start beg, length len) into the drain frontier of the next
// sub-round: short rows by id (with start and length) into Q, long rows as
// chunk items into C, at positions after the items of earlier sub-rounds
// (qbase / cbase) counted in slot S.  Called by any subset of lanes; short
// pushes are aggregated over the lanes that take this path together.
__device__ __forceinline__ void push_frontier(const CoreArgs& a, CoreSlot* S, uint64_t qbase, uint64_t cbase,
                                              uint32_t v, uint64_t beg, uint64_t len, uint32_t short_max) {
    if (len <= short_max) {
        cg::coalesced_group g = cg::coalesced_threads();
        unsigned long long base = 0;
        if (g.thread_rank() == 0) base = atomicAdd(&S->qcnt, (unsigned long long)g.size());
        base = g.shfl(base, 0);
        const uint64_t at = qbase + base + g.thread_rank();
        DSG_BOUND(a.ctl, 1, at, a.n, 0, return);
        a.Q[at] = v;
        a.QgB[at] = beg;
        a.QgL[at] = (uint32_t)len;
    } else {
        uint64_t nch = (len + a.chunk_len - 1) / a.chunk_len;
        unsigned long long c0 = atomicAdd(&S->ccnt, (unsigned long long)nch);
        DSG_BOUND(a.ctl, 2, cbase + c0 + nch - 1, a.chunk_cap, 0, return);
        for (uint64_t c = 0; c < nch; ++c) a.C[cbase + c0 + c] = ((uint64_t)v << 32) | c;
    }
}

template <int TB>
__global__ void __launch_bounds__(TB) kcore_kernel(CoreArgs a) {
    __shared__ CoreSmem<TB> sm;
    CoreCtl* ctl = a.ctl;
    const uint32_t tid = threadIdx.x;
    const uint32_t n = a.n;
    uint64_t nstamp = 0;
    // trace entries: 2 words each, (time, kind << 32 | k); kind 0 start, 1 init, 2 scan sub-round, 3 drain
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
    // ---- init: deg = row length, claims cleared; least degree -> first level
    {
        uint32_t mn = 0xffffffffu;
        for (uint64_t v = (uint64_t)blockIdx.x * TB + tid; v < n; v += (uint64_t)gridDim.x * TB) {
            uint32_t d = (uint32_t)(a.off[v + 1] - a.off[v]);
            a.deg[v] = d;
            mn = min(mn, d);
        }
        const uint64_t words = ((uint64_t)n + 31) >> 5;
        for (uint64_t w = (uint64_t)blockIdx.x * TB + tid; w < words; w += (uint64_t)gridDim.x * TB) a.claim[w] = 0;
        mn = block_min_u32(mn, sm.redm);
        if (tid == 0 && mn != 0xffffffffu) atomicMin(&ctl->init_min, mn);
    }
    if (!grid_barrier(&ctl->bar, &ctl->err, a.limit_ns)) return;
    stamp(1, 0);
    uint32_t k = ld_relaxed_u32(&ctl->init_min);
    // remaining vertices: level 0 scans every vertex (block b the tiles
    // b, b + grid, ...); later levels scan the block's own segment of the
    // previous level's kept vertices
    const uint64_t segoff = (uint64_t)blockIdx.x * a.seg;
    uint64_t my_n = 0;
    const uint32_t* my_rem = nullptr;  // level 0: identity
    uint32_t* my_rem_next = a.remA + segoff;
    uint32_t* const myQA = a.QA + segoff;
    uint64_t* const myQB = a.QB + segoff;
    uint32_t* const myQL = a.QL + segoff;
    uint64_t qpos = 0, cpos = 0, qlo = 0, qhi = 0, clo = 0, chi = 0;
    uint64_t visited = 0, j = 0;
    uint64_t level = 0, subrounds = 0;
    uint32_t* deg = a.deg;
    for (;;) {
        uint32_t level_min = 0xffffffffu;
        uint64_t my_n_next = 0;
        for (bool first = true;; first = false) {
            CoreSlot* S = &ctl->slot[j % 3];
            if (blockIdx.x == 0 && tid == 0) {
                CoreSlot* R = &ctl->slot[(j + 1) % 3];
                R->qcnt = 0;
                R->ccnt = 0;
                R->pushed = 0;
                R->nmin = 0xffffffffu;
            }
            uint32_t dmn = 0xffffffffu;
            uint64_t dpushed = 0, natom = 0;
            // u reached k: drain it in this block if there is room, else globally
            auto reach_k = [&](uint32_t u) {
                // the decrement that brought u to k is unique; only a scan of the
                // same sub-round can also see u at k, so only there is the bit raced for
                if (first) {
                    if (!claim_vertex(a.claim, u)) return;  // the scan took it
                } else {
                    atomicOr(&a.claim[u >> 5], 1u << (u & 31u));
                }
                const uint64_t beg = a.off[u];
                const uint64_t len = a.off[u + 1] - beg;
                ++dpushed;
                // keep it in the block while the block's own share stays small:
                // past local_work entries a grid-wide sub-round is cheaper
                if (len <= a.local_max && atomicAdd(&sm.lq_work, (uint32_t)len) + len <= a.local_work) {
                    uint32_t pos = atomicAdd(&sm.lq_tail, 1u);
                    if (pos < CoreSmem<TB>::kLocalQ) {
                        sm.lq[pos] = u;
                        sm.lqb[pos] = beg;
                        sm.lql[pos] = (uint32_t)len;
                        return;
                    }
                }
                push_frontier(a, S, qpos, cpos, u, beg, len, a.short_max);
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
                for (uint32_t jj = 0; jj < kBatch; ++jj) {
                    if (!(valid >> jj & 1u)) continue;
#ifdef DSG_DEBUG_BOUNDS
                    if (u[jj] >= n) {
                        DSG_BOUND(ctl, 4, u[jj], n, level, (void)0);
                        continue;
                    }
#endif
                    if (u[jj] == v[jj]) continue;
                    d[jj] = deg[u[jj]];
                    need |= 1u << jj;
                }
#pragma unroll
                for (uint32_t jj = 0; jj < kBatch; ++jj) {
                    if (!(need >> jj & 1u)) continue;
                    if (d[jj] <= k || (d[jj] >= hot && agg_add(sm.agg, u[jj]))) {
                        need &= ~(1u << jj);  // already at k, or settled at the flush
                        continue;
                    }
                    old[jj] = atomicSub(&deg[u[jj]], 1u);
                    ++natom;
                }
#pragma unroll
                for (uint32_t jj = 0; jj < kBatch; ++jj)
                    if (need >> jj & 1u) settle(u[jj], old[jj], 1u);
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
                sm.own = 0;
                sm.kept = 0;
                sm.acc_min = 0xffffffffu;
                sm.acc_pushed = 0;
                sm.acc_atomics = 0;
            }
            __syncthreads();
            if (first) {
                // ---- scan: claim degree <= k, keep degree > k, drop the claimed
                uint32_t mn = 0xffffffffu;
                const uint64_t lim = my_rem ? my_n : n;
                const uint64_t stride = my_rem ? TB : (uint64_t)gridDim.x * TB;
                uint64_t scanned = 0;
                for (uint64_t t = my_rem ? 0 : (uint64_t)blockIdx.x * TB; t < lim; t += stride) {
                    const uint64_t i = t + tid;
                    bool keep = false;
                    uint32_t v = 0;
                    if (i < lim) {
                        ++scanned;
                        v = my_rem ? my_rem[i] : (uint32_t)i;
                        const uint32_t dv = deg[v];
                        const uint32_t taken = a.claim[v >> 5] >> (v & 31u) & 1u;
                        if (!taken) {
                            if (dv > k) {
                                keep = true;
                                mn = min(mn, dv);
                            } else if (claim_vertex(a.claim, v)) {
                                ++dpushed;
                                const uint64_t beg = a.off[v];
                                const uint64_t len = a.off[v + 1] - beg;
                                // drained by this block, or, for rows above inline_max,
                                // spread over every warp in the next sub-round
                                if (len <= a.inline_max) {
                                    uint32_t pos = atomicAdd(&sm.own, 1u);
                                    DSG_BOUND(ctl, 5, pos, a.seg, level, pos = 0);
                                    myQA[pos] = v;
                                    myQB[pos] = beg;
                                    myQL[pos] = (uint32_t)len;
                                } else {
                                    push_frontier(a, S, qpos, cpos, v, beg, len, a.short_max);
                                }
                            }
                        }
                    }
                    // keep: warp ballot, one shared-memory atomic per warp
                    const uint32_t bal = __ballot_sync(kFullMask, keep);
                    uint32_t base = 0;
                    if ((tid & 31u) == 0 && bal) base = atomicAdd(&sm.kept, (uint32_t)__popc(bal));
                    base = __shfl_sync(kFullMask, base, 0);
                    if (keep) {
                        uint64_t at = base + __popc(bal & lanemask_lt());
                        DSG_BOUND(ctl, 3, at, a.seg, level, keep = false);
                        if (keep) my_rem_next[at] = v;
                    }
                }
                dmn = min(dmn, mn);
                __syncthreads();
                // ---- drain what this block's scan claimed
                const uint32_t own = (uint32_t)min((uint64_t)sm.own, a.seg);
                my_n_next = sm.kept;
                {
                    const uint64_t bs = block_sum<uint64_t>(scanned, sm.red);
                    if (tid == 0) {
                        atomicAdd(&ctl->rem_scanned, (unsigned long long)bs);
                        atomicAdd(&ctl->rem_written, (unsigned long long)my_n_next);
                    }
                }
                scan_block_rows<TB>(a.adj, myQA, myQB, myQL, own, sm.btile, visit);
            } else {
                scan_frontier<TB>(a.off, a.adj, a.Q, qlo, qhi, a.C, clo, chi, a.chunk_len, visit, n, a.QgB, a.QgL);
            }
            flush();
            // drain what this block found, until it finds nothing more
            for (uint32_t lq_lo = 0;;) {
                uint32_t lq_hi = min(sm.lq_tail, CoreSmem<TB>::kLocalQ);
                __syncthreads();
                if (lq_lo >= lq_hi) break;
                scan_block_rows<TB>(a.adj, sm.lq + lq_lo, sm.lqb + lq_lo, sm.lql + lq_lo, lq_hi - lq_lo, sm.btile,
                                    visit);
                flush();
                lq_lo = lq_hi;
            }
            // block reductions: warp shuffles, one shared atomic per warp, then
            // thread 0 adds the block's totals (the barrier synchronises first)
            dmn = warp_min(dmn);
            dpushed = warp_sum(dpushed);
            natom = warp_sum(natom);
            if ((tid & 31u) == 0) {
                if (dmn != 0xffffffffu) atomicMin(&sm.acc_min, dmn);
                if (dpushed) atomicAdd(&sm.acc_pushed, (unsigned long long)dpushed);
                if (natom) atomicAdd(&sm.acc_atomics, (unsigned long long)natom);
            }
            __syncthreads();
            if (tid == 0) {
                if (sm.acc_min != 0xffffffffu) atomicMin(&S->nmin, sm.acc_min);
                if (sm.acc_pushed) atomicAdd(&S->pushed, sm.acc_pushed);
                if (sm.acc_atomics) atomicAdd(&ctl->atomics, sm.acc_atomics);
            }
            if (!grid_barrier(&ctl->bar, &ctl->err, a.limit_ns)) return;
            stamp(first ? 2 : 3, k);
            ++subrounds;
            const uint64_t qcnt = ld_relaxed_u64(&S->qcnt);
            const uint64_t ccnt = ld_relaxed_u64(&S->ccnt);
            visited += ld_relaxed_u64(&S->pushed);
            level_min = min(level_min, ld_relaxed_u32(&S->nmin));
            qlo = qpos;
            qhi = qpos + qcnt;
            qpos = qhi;
            clo = cpos;
            chi = cpos + ccnt;
            cpos = chi;
            ++j;
            if (qcnt == 0 && ccnt == 0) break;
        }
        ++level;
        if (visited >= n) break;
        if (level_min == 0xffffffffu || level_min <= k) {
            // nothing left above k yet visited < n: cannot happen on valid input
            if (blockIdx.x == 0 && tid == 0) atomicOr(&ctl->err, ERR_CAPACITY);
            break;
        }
        k = level_min;
        my_n = my_n_next;
        my_rem = my_rem_next;
        my_rem_next = (my_rem_next == a.remA + segoff) ? a.remB + segoff : a.remA + segoff;
    }
    if (blockIdx.x == 0 && tid == 0) {
        ctl->stamps = nstamp;
        ctl->levels = level;
        ctl->subrounds = subrounds;
    }
}

template <int TB>
static cudaError_t kcore_grid(const CoreArgs& a, uint32_t blocks_per_sm, uint32_t* grid) {
    return coop_grid(kcore_kernel<TB>, TB, 0, a.n, blocks_per_sm, grid);
}

template <int TB>
static cudaError_t launch_kcore(CoreArgs& a, uint32_t grid, cudaStream_t s) {
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
    a.inline_max = tu.inline_max;
    a.trace = trace_dev;
    a.trace_cap = trace_cap;
    uint32_t grid = 1;
    cudaError_t e;
    switch (tu.block) {
        case 256: e = kcore_grid<256>(a, tu.blocks_per_sm, &grid); break;
        case 1024: e = kcore_grid<1024>(a, tu.blocks_per_sm, &grid); break;
        default: e = kcore_grid<512>(a, tu.blocks_per_sm, &grid); break;
    }
    DSG_TRY_CUDA(e);
    // a block scans at most ceil(n / (grid * block)) tiles of `block` vertices
    const uint64_t span = (uint64_t)grid * tu.block;
    a.seg = ((uint64_t)n + span - 1) / span * tu.block;
    bool direct = is_device_ptr(core_out);
    if (direct) a.deg = core_out;
    else DSG_TRY_CUDA(sc.get(&a.deg, n));
    DSG_TRY_CUDA(sc.get(&a.claim, ((uint64_t)n + 31) / 32));
    DSG_TRY_CUDA(sc.get(&a.remA, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.remB, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.QA, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.QB, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.QL, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.Q, n));
    DSG_TRY_CUDA(sc.get(&a.QgB, n));
    DSG_TRY_CUDA(sc.get(&a.QgL, n));
    DSG_TRY_CUDA(sc.get(&a.C, chunk_cap));
    DSG_TRY_CUDA(sc.get(&a.ctl, 1));
    {
        CoreCtl init;
        memset(&init, 0, sizeof(init));
        init.init_min = 0xffffffffu;
        for (int i = 0; i < 3; ++i) init.slot[i].nmin = 0xffffffffu;
        DSG_TRY_CUDA(cudaMemcpyAsync(a.ctl, &init, sizeof(CoreCtl), cudaMemcpyHostToDevice, s));
    }
    switch (tu.block) {
        case 256: e = launch_kcore<256>(a, grid, s); break;
        case 1024: e = launch_kcore<1024>(a, grid, s); break;
        default: e = launch_kcore<512>(a, grid, s); break;
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
