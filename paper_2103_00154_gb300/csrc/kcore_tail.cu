// The last levels of Algorithm 2's first phase (core numbers) on a small
// remaining graph, by one thread-block cluster.
//
// Once few vertices remain, a level of the grid-wide kernel costs mostly the
// latency of its cascade (a vertex brought to k by a drain is drained in the
// same level, and so on, several links deep), and each link there is a few
// global-memory round trips plus block barriers.  Here the remaining graph is
// first compacted -- its vertices renumbered 0..r-1 and each row cut down to
// the neighbours that remain, which changes no degree: a remaining vertex's
// degree already counts exactly its remaining neighbours, and a drain never
// lowers the degree of a vertex that is gone -- and then one cluster runs the
// remaining levels with every vertex's degree, row bounds and queue slot in
// the distributed shared memory of the cluster: vertex i belongs to block
// i % C.
//
// Level k:
//   scan: each block walks its own vertices not yet taken (a list compacted
//     every level) and takes those of degree <= k into its queue; the scan
//     takes are added to a cluster-wide pending count, and a cluster barrier
//     separates the scan from the drain, so no degree changes while any
//     block scans;
//   every block copies the cluster's taken bits (the union of the blocks'
//     own bitmaps) into its shared memory, so a drain skips a neighbour that
//     is gone with a local look-up;
//   drain: each block drains its queue in batches, all its threads spread
//     over the batch's rows; a neighbour that is not gone loses one degree
//     (a DSMEM atomic at its owner); if that brought it from k + 1 to k the
//     decrementer is the one thread that does so: it reads the vertex's row
//     bounds at the owner, asks L2 for the row, and queues the vertex at its
//     owner (pending count up, a slot at the owner, one store of the owner's
//     local index); if it was at or below k already (taken during this
//     level) the decrement is undone, which leaves the degrees Algorithm 2's
//     read-then-decrement drain leaves.  A block gives a batch's count back
//     to the pending count once the batch and the takes it made are
//     registered, so the count reaches zero only when the level's cascade is
//     over; the owners drain, so a cascade spreads over the cluster;
//   the blocks meet at a cluster barrier and sum the level's takes and least
//   degree above k, so every block takes the same decisions.
// Every wait is bounded (ERR_TIMEOUT).
#include <cooperative_groups.h>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace cg = cooperative_groups;

namespace dsg {

constexpr uint32_t kTailTB = 1024;
constexpr uint32_t kTailC = 16;                       // blocks in the cluster
constexpr uint32_t kTailVPC = kTailMaxVertices / kTailC;  // vertices per block at most
constexpr uint32_t kTailWPB = kTailVPC / 32;          // bitmap words per block
constexpr uint16_t kSlotEmpty = 0xffffu;
constexpr uint32_t kOffMax = 0xffffffffu;             // compacted row offsets must stay below this

struct TailStats {
    unsigned long long levels, rem_scanned, atomics, claims, stamps;
    uint32_t err;
};

struct TailArgs {
    uint32_t r;                 // remaining vertices, numbered 0..r-1
    const uint64_t* off;        // compacted rows, r + 1 (every offset below 2^32 - 1)
    const uint32_t* adj;        // compacted neighbour numbers
    const uint32_t* cdeg;       // degree of each remaining vertex when the tail starts
    const uint32_t* rid;        // original id of each remaining vertex
    uint32_t* core;             // core numbers by original id (written for the remaining vertices)
    TailStats* stats;
    uint64_t limit_ns;          // bound of every wait
    uint64_t* trace;            // nullable: block 0 stamps (%globaltimer, kind << 32 | k) per level phase
    uint64_t trace_cap;         // words of trace
};

struct TailSmem {
    uint32_t deg[kTailVPC];            // this block's vertices' degrees (other blocks decrement them)
    uint32_t rbeg[kTailVPC];           // ... their row starts and lengths in the compacted adjacency
    uint32_t rlen[kTailVPC];
    uint32_t taken[kTailWPB];          // this block's vertices taken into a level (written by this block)
    uint32_t gone[kTailC * kTailWPB];  // copy of every block's taken bits, block b's at [b * kTailWPB]
    uint16_t rem[2][kTailVPC];         // this block's vertices still to scan, by level parity
    uint16_t q[kTailVPC];              // this level's queue of own vertices (local index); kSlotEmpty until
                                       // the taker has written it
    uint32_t start[kTailTB];           // a batch's rows: exclusive prefix of lengths ...
    uint32_t beg[kTailTB];             // ... row starts
    uint32_t red[33];
    uint64_t red64[33];
    uint32_t qtail, nkeep, batch_n, batch_total, stop;
    uint32_t pending;                  // block 0's copy: taken vertices of the level not yet drained
    uint32_t pub_min[2], pub_claims[2], pub_err[2];  // a level's totals of this block, by level parity
    uint32_t tot_min, tot_err;
    unsigned long long tot_claims;
};

// Ask L2 to fetch adj[b, b + l) (rounded out to 16-byte boundaries; the
// adjacency allocation is padded to 256 bytes, so the rounding stays inside it).
__device__ __forceinline__ void prefetch_row(const uint32_t* adj, uint32_t b, uint32_t l) {
    if (l == 0) return;
    const uint64_t lo = (uint64_t)b & ~3ull, hi = ((uint64_t)b + l + 3) & ~3ull;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(adj + lo)),
                 "r"((uint32_t)((hi - lo) * 4))
                 : "memory");
}

__global__ void __launch_bounds__(kTailTB, 1) kcore_tail_kernel(TailArgs a) {
    extern __shared__ __align__(16) unsigned char tail_smem_raw[];
    TailSmem& sm = *reinterpret_cast<TailSmem*>(tail_smem_raw);
    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t C = cluster.num_blocks();
    const uint32_t rank = cluster.block_rank();
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const uint32_t r = a.r;
    const uint32_t V = r > rank ? (r - rank + C - 1) / C : 0;  // this block's vertices: i = li * C + rank
    const uint32_t wmax = ((r + C - 1) / C + 31) / 32;         // taken words in use per block
    // ---- degrees, row bounds, the list of this block's vertices; least degree
    uint32_t mn = 0xffffffffu;
    for (uint32_t li = tid; li < V; li += kTailTB) {
        const uint32_t i = li * C + rank;
        const uint32_t d = a.cdeg[i];
        const uint64_t b0 = a.off[i], b1 = a.off[i + 1];
        sm.deg[li] = d;
        sm.rbeg[li] = (uint32_t)b0;
        sm.rlen[li] = (uint32_t)(b1 - b0);
        sm.rem[0][li] = (uint16_t)li;
        mn = min(mn, d);
    }
    for (uint32_t w = tid; w < kTailWPB; w += kTailTB) sm.taken[w] = 0;
    for (uint32_t i = tid; i < kTailVPC; i += kTailTB) sm.q[i] = kSlotEmpty;
    mn = block_min_u32(mn, sm.red);
    if (tid == 0) {
        sm.pub_min[1] = mn;
        sm.qtail = 0;
        sm.pending = 0;
    }
    cluster.sync();
    uint32_t k = 0xffffffffu;
    for (uint32_t b = 0; b < C; ++b) k = min(k, *cluster.map_shared_rank(&sm.pub_min[1], (int)b));
    uint32_t* const pending0 = cluster.map_shared_rank(&sm.pending, 0);
    uint64_t visited = 0, level = 0, scanned = 0, natom = 0, nstamp = 0;
    uint32_t nrem = V;
    bool bad = false, timeout = false;
    // trace pairs: kind 11 scan done, 12 drain done, 13 level over (block 0), 14 the level's claims;
    // block 0's batches: 15 batch taken (time), 16 its vertices << 32 | its entries, 17 batch drained (time)
    auto stamp = [&](uint32_t kind, uint64_t val) {
        if (a.trace && rank == 0 && tid == 0 && 2 * nstamp + 1 < a.trace_cap) {
            a.trace[2 * nstamp] = val;
            a.trace[2 * nstamp + 1] = ((uint64_t)kind << 32) | k;
        }
        ++nstamp;
    };
    while (visited < r) {
        const uint32_t par = (uint32_t)(level & 1);
        const uint16_t* cur = sm.rem[par];
        uint16_t* nxt = sm.rem[par ^ 1u];
        uint32_t lmin = 0xffffffffu;
        if (tid == 0) sm.nkeep = 0;
        __syncthreads();
        // ---- scan: take degree <= k (queued here), keep degree > k; nothing changes a degree meanwhile
        uint32_t lclaims = 0;
        for (uint32_t j0 = 0; j0 < nrem; j0 += kTailTB) {
            const uint32_t j = j0 + tid;
            bool keep = false;
            uint32_t li = 0;
            if (j < nrem) {
                li = cur[j];
                const uint32_t bit = 1u << (li & 31u);
                if (!(sm.taken[li >> 5] & bit)) {
                    const uint32_t d = sm.deg[li];
                    if (d > k) {
                        keep = true;
                        lmin = min(lmin, d);
                    } else {
                        atomicOr(&sm.taken[li >> 5], bit);
                        prefetch_row(a.adj, sm.rbeg[li], sm.rlen[li]);
                        sm.q[atomicAdd(&sm.qtail, 1u)] = (uint16_t)li;
                        ++lclaims;
                    }
                }
            }
            const uint32_t bal = __ballot_sync(kFullMask, keep);
            uint32_t base = 0;
            if (lane == 0 && bal) base = atomicAdd(&sm.nkeep, (uint32_t)__popc(bal));
            base = __shfl_sync(kFullMask, base, 0);
            if (keep) nxt[base + __popc(bal & lanemask_lt())] = (uint16_t)li;
        }
        if (tid == 0) scanned += nrem;
        {
            const uint32_t c = (uint32_t)block_sum<uint64_t>((uint64_t)lclaims, sm.red64);
            if (tid == 0 && c) atomicAdd(pending0, c);
        }
        cluster.sync();  // every scan take is counted and every taken bit of the scan is set
        // ---- the cluster's taken bits, for the drain's look-ups
        for (uint32_t w = tid; w < C * wmax; w += kTailTB) {
            const uint32_t b = w / wmax, ww = w - b * wmax;
            sm.gone[b * kTailWPB + ww] =
                *reinterpret_cast<volatile uint32_t*>(cluster.map_shared_rank(&sm.taken[ww], (int)b));
        }
        __syncthreads();
        stamp(11, global_ns());
        // ---- drain: a neighbour not gone loses one degree at its owner; the one decrement
        // that takes it from k + 1 to k queues it there; one that finds it at or below k
        // (taken during this level) is undone
        auto visit = [&](const uint32_t* u, uint32_t valid) {
            uint32_t old[kBatch], live = 0;
            uint32_t* dp[kBatch];
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj) {
                dp[jj] = nullptr;
                old[jj] = 0;
                if (!(valid >> jj & 1u)) continue;
                if (u[jj] >= r) {
                    bad = true;
                    continue;
                }
                const uint32_t ru = u[jj] % C, lu = u[jj] / C;
                if (sm.gone[ru * kTailWPB + (lu >> 5)] >> (lu & 31u) & 1u) continue;
                dp[jj] = cluster.map_shared_rank(&sm.deg[lu], (int)ru);
                old[jj] = atomicSub(dp[jj], 1u);
                ++natom;
                live |= 1u << jj;
            }
            uint32_t claim = 0;
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj) {
                if (!(live >> jj & 1u)) continue;
                if (old[jj] <= k) {
                    atomicAdd(dp[jj], 1u);
                    ++natom;
                } else if (old[jj] == k + 1) {
                    claim |= 1u << jj;
                } else {
                    lmin = min(lmin, old[jj] - 1);
                }
            }
            // the warp's takes: one pending increment by a leader, a slot at each owner and the
            // row bounds there, then the row asked into L2 and the slot written (the count never
            // reads zero while a take is unqueued)
            const uint32_t wsum = warp_sum((uint32_t)__popc(claim));
            if (wsum == 0) return;
            uint32_t was = 0;
            if (lane == 0) was = atomicAdd(pending0, wsum);
            uint32_t slot[kBatch], rb[kBatch], rl[kBatch];
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj) {
                if (!(claim >> jj & 1u)) continue;
                const uint32_t ru = u[jj] % C, lu = u[jj] / C;
                slot[jj] = atomicAdd(cluster.map_shared_rank(&sm.qtail, (int)ru), 1u);
                rb[jj] = *cluster.map_shared_rank(&sm.rbeg[lu], (int)ru);
                rl[jj] = *cluster.map_shared_rank(&sm.rlen[lu], (int)ru);
            }
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj)
                if (claim >> jj & 1u) prefetch_row(a.adj, rb[jj], rl[jj]);
            was = __shfl_sync(kFullMask, was, 0);
            if (was == 0xffffffffu) bad = true;
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj) {
                if (!(claim >> jj & 1u)) continue;
                if (slot[jj] >= kTailVPC) {
                    bad = true;
                    continue;
                }
                volatile uint16_t* sp = cluster.map_shared_rank(&sm.q[slot[jj]], (int)(u[jj] % C));
                *sp = (uint16_t)(u[jj] / C);
            }
        };
        // ---- drain this block's queue until the cluster has nothing pending
        uint32_t qhead = 0;
        uint64_t wait_start = global_ns();
        for (;;) {
            if (tid == 0) {
                // wait here, alone, for queued work or the level's end: the queue tail is local and
                // polled tightly, the cluster's pending count every few polls
                uint32_t take = 0, stop = 0;
                for (uint32_t spins = 0;; ++spins) {
                    const uint32_t t = *reinterpret_cast<volatile uint32_t*>(&sm.qtail);
                    if (t != qhead) {
                        take = min(t - qhead, kTailTB);
                        break;
                    }
                    if ((spins & 7u) == 7u) {
                        if (*reinterpret_cast<volatile uint32_t*>(pending0) == 0) {
                            // nothing queued here (re-read: a take may have landed meanwhile)
                            if (*reinterpret_cast<volatile uint32_t*>(&sm.qtail) == qhead) {
                                stop = 1;
                                break;
                            }
                            continue;
                        }
                        if (global_ns() - wait_start > a.limit_ns) {
                            stop = 1;
                            timeout = true;
                            break;
                        }
                    }
                }
                sm.stop = stop;
                sm.batch_n = take;
            }
            __syncthreads();
            const uint32_t nb = sm.batch_n;
            if (sm.stop) break;
            // the batch's vertices: slots qhead .. qhead + nb, each written by its taker right
            // after it reserved the slot: wait for it, bounded
            uint32_t len = 0, bg = 0;
            if (tid < nb) {
                volatile uint16_t* sl = &sm.q[qhead + tid];
                uint16_t x = *sl;
                const uint64_t s0 = global_ns();
                while (x == kSlotEmpty) {
                    if (global_ns() - s0 > a.limit_ns) { timeout = true; break; }
                    x = *sl;
                }
                if (x != kSlotEmpty && x < V) {
                    atomicOr(&sm.taken[x >> 5], 1u << (x & 31u));
                    bg = sm.rbeg[x];
                    len = sm.rlen[x];
                } else if (x != kSlotEmpty) {
                    bad = true;
                }
            }
            uint32_t total;
            if (nb == 1) {
                // one row (the common case in the last levels): no scan
                if (tid == 0) {
                    sm.start[0] = 0;
                    sm.beg[0] = bg;
                    sm.batch_total = len;
                }
                __syncthreads();
                total = sm.batch_total;
            } else {
                const uint32_t st = block_excl_scan<uint32_t>(len, sm.red, &total);
                sm.start[tid] = st;
                sm.beg[tid] = bg;
                __syncthreads();
            }
            if (a.trace) {
                stamp(15, global_ns());
                stamp(16, ((uint64_t)nb << 32) | total);
            }
            for (uint32_t w0 = tid & ~31u; w0 < total; w0 += kBatch * kTailTB) {
                uint32_t bu[kBatch], valid = 0;
#pragma unroll
                for (uint32_t j = 0; j < kBatch; ++j) {
                    const uint32_t e = w0 + lane + j * kTailTB;
                    bu[j] = 0;
                    if (e < total) {
                        uint32_t lo = 0, hi = nb;  // row = last whose start is <= e
                        while (hi - lo > 1) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (sm.start[mid] <= e) lo = mid; else hi = mid;
                        }
                        bu[j] = a.adj[sm.beg[lo] + (e - sm.start[lo])];
                        valid |= 1u << j;
                    }
                }
                visit(bu, valid);
            }
            __syncthreads();  // every drain of the batch is done and its takes are counted
            if (a.trace) stamp(17, global_ns());
            if (tid == 0) atomicSub(pending0, nb);
            qhead += nb;
            wait_start = global_ns();
        }
        stamp(12, global_ns());
        // ---- the level's totals over the cluster; queue slots back to empty for the next level
        for (uint32_t i = tid; i < qhead; i += kTailTB) sm.q[i] = kSlotEmpty;
        lmin = block_min_u32(lmin, sm.red);
        const uint32_t to = __syncthreads_or(timeout || bad);
        if (tid == 0) {
            // (level parity: a block writes these again two levels on, after every block passed the
            // next level's barriers and so has read them)
            sm.pub_min[par] = lmin;
            sm.pub_claims[par] = qhead;  // every vertex this block took at this level went through its queue
            sm.pub_err[par] = to;
            sm.qtail = 0;
        }
        nrem = sm.nkeep;
        cluster.sync();  // every block's drains of this level are done and its totals published
        if (tid < 32) {  // one warp gathers the cluster's totals
            uint32_t m_ = 0xffffffffu, e_ = 0, c_ = 0;
            if (tid < C) {
                m_ = *cluster.map_shared_rank(&sm.pub_min[par], (int)tid);
                c_ = *cluster.map_shared_rank(&sm.pub_claims[par], (int)tid);
                e_ = *cluster.map_shared_rank(&sm.pub_err[par], (int)tid);
            }
            m_ = warp_min(m_);
            const uint64_t cs_ = warp_sum<uint64_t>((uint64_t)c_);
            e_ = __reduce_or_sync(kFullMask, e_);
            if (tid == 0) {
                sm.tot_min = m_;
                sm.tot_claims = cs_;
                sm.tot_err = e_;
            }
        }
        __syncthreads();
        const uint32_t kmin = sm.tot_min, err = sm.tot_err;
        const uint64_t claims = sm.tot_claims;
        visited += claims;
        stamp(13, global_ns());
        stamp(14, claims);
        ++level;
        if (visited >= r) break;
        if (err || kmin == 0xffffffffu || kmin <= k) {  // a wait ran out, or an inconsistent remaining graph
            bad = bad || !timeout;
            break;
        }
        k = kmin;
    }
    // ---- core numbers of this block's vertices; then no block may leave
    // while another could still read its shared memory
    for (uint32_t li = tid; li < V; li += kTailTB) a.core[a.rid[li * C + rank]] = sm.deg[li];
    natom = warp_sum(natom);
    scanned = warp_sum(scanned);
    if (lane == 0) {
        if (natom) atomicAdd(&a.stats->atomics, (unsigned long long)natom);
        if (scanned) atomicAdd(&a.stats->rem_scanned, (unsigned long long)scanned);
    }
    if (bad) atomicOr(&a.stats->err, ERR_RANGE);
    if (timeout) atomicOr(&a.stats->err, ERR_TIMEOUT);
    if (rank == 0 && tid == 0) {
        a.stats->levels = level;
        a.stats->claims = visited;
        a.stats->stamps = nstamp;
    }
    cluster.sync();
}

// ---------------------------------------------------------------- compaction

// The vertices not yet taken (claim bit clear), numbered in the order warps
// reach them: rid[i] = original id, newid[v] = i, cdeg[i] = current degree,
// flen[i] = full row length.  *r = their number.
__global__ void tail_collect_kernel(uint32_t n, const uint32_t* __restrict__ claim, const uint32_t* __restrict__ deg,
                                    const uint64_t* __restrict__ off, uint32_t* __restrict__ rid,
                                    uint32_t* __restrict__ newid, uint32_t* __restrict__ cdeg,
                                    uint32_t* __restrict__ flen, uint32_t* __restrict__ r, uint32_t cap) {
    const uint32_t words = (n + 31) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; w0 < words;
         w0 += (gridDim.x * blockDim.x) & ~31u) {
        const uint32_t w = w0 + lane;
        uint32_t free_bits = 0;
        if (w < words) {
            free_bits = ~claim[w];
            const uint32_t hi = n - w * 32;  // vertices in this word
            if (hi < 32) free_bits &= (1u << hi) - 1u;
        }
        const uint32_t c = __popc(free_bits);
        const uint32_t inc = warp_incl_scan(c);
        uint32_t base = 0;
        if (lane == 31 && inc) base = atomicAdd(r, inc);
        base = __shfl_sync(kFullMask, base, 31) + inc - c;
        while (free_bits) {
            const uint32_t b = __ffs(free_bits) - 1;
            free_bits &= free_bits - 1;
            const uint32_t v = w * 32 + b;
            if (base < cap) {
                rid[base] = v;
                newid[v] = base;
                cdeg[base] = deg[v];
                flen[base] = (uint32_t)(off[v + 1] - off[v]);
            }
            ++base;
        }
    }
}

// Compacted rows: every entry of the remaining vertices' full rows whose
// neighbour remains, renumbered, at the row's next free slot (the order in a
// row does not matter to the core numbers).  Edge-balanced over the full rows.
__global__ void __launch_bounds__(256) tail_fill_kernel(uint32_t r, const uint64_t* __restrict__ roff,
                                                        const uint32_t* __restrict__ rid,
                                                        const uint64_t* __restrict__ off,
                                                        const uint32_t* __restrict__ adj,
                                                        const uint32_t* __restrict__ claim,
                                                        const uint32_t* __restrict__ newid,
                                                        const uint64_t* __restrict__ coff,
                                                        uint32_t* __restrict__ fill, uint32_t* __restrict__ cadj,
                                                        uint32_t* __restrict__ err) {
    auto pre = [&](uint64_t) { return 0u; };
    auto put = [&](const uint32_t* i, const uint64_t* j, const uint32_t*, uint32_t valid) {
        uint32_t u[kWalkU], keep = 0;
#pragma unroll
        for (uint32_t t = 0; t < kWalkU; ++t) {
            u[t] = 0;
            if (valid >> t & 1u) u[t] = ld_stream(adj + off[rid[i[t]]] + (j[t] - roff[i[t]]));
        }
#pragma unroll
        for (uint32_t t = 0; t < kWalkU; ++t)
            if ((valid >> t & 1u) && !(claim[u[t] >> 5] >> (u[t] & 31u) & 1u)) keep |= 1u << t;
#pragma unroll
        for (uint32_t t = 0; t < kWalkU; ++t) {
            const uint32_t key = (keep >> t & 1u) ? i[t] : 0xffffffffu;
            const uint32_t peers = __match_any_sync(kFullMask, key);
            const uint32_t leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (key != 0xffffffffu && (threadIdx.x & 31u) == leader) base = atomicAdd(&fill[key], __popc(peers));
            base = __shfl_sync(kFullMask, base, leader);
            if (key != 0xffffffffu) {
                // a remaining vertex keeps exactly its degree's worth of neighbours; anything
                // past its row end means the state was not a finished level: flag, do not write
                const uint64_t at = coff[key] + base + __popc(peers & lanemask_lt());
                if (at < coff[key + 1]) cadj[at] = newid[u[t]];
                else atomicOr(err, ERR_RANGE);
            }
        }
    };
    walk_all_entries(roff, r, pre, put);
}

// core[rid[i]] = ccore[i]: core numbers of the compacted graph back to original ids.
__global__ void tail_scatter_kernel(uint32_t r, const uint32_t* __restrict__ rid, const uint32_t* __restrict__ ccore,
                                    uint32_t* __restrict__ core) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < r) core[rid[i]] = ccore[i];
}

// Scan of n uint32 values into out[0..n] (exclusive, out[n] = total).
dsg_status scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, Scratch& sc, cudaStream_t s);

dsg_status kcore_tail(uint32_t n, const uint64_t* off, const uint32_t* adj, uint32_t* deg, const uint32_t* claim,
                      uint32_t cap, cudaStream_t s, uint64_t* stats5, uint64_t* trace, uint64_t trace_cap,
                      uint64_t* stamps) {
    Scratch sc(s);
    uint32_t *rid, *newid, *cdeg, *flen, *cnt;
    DSG_TRY_CUDA(sc.get(&rid, cap));
    DSG_TRY_CUDA(sc.get(&newid, n));
    DSG_TRY_CUDA(sc.get(&cdeg, cap + 1));
    DSG_TRY_CUDA(sc.get(&flen, cap + 1));
    DSG_TRY_CUDA(sc.get(&cnt, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t), s));
    {
        const uint32_t words = (n + 31) >> 5;
        const uint32_t g = (uint32_t)std::min<uint64_t>(((uint64_t)words + 255) / 256, (uint64_t)dev_info().sms * 8);
        LaunchScope ls("kcore_tail_collect", s);
        tail_collect_kernel<<<g ? g : 1, 256, 0, s>>>(n, claim, deg, off, rid, newid, cdeg, flen, cnt, cap);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    uint32_t r = 0;
    DSG_TRY_CUDA(cudaMemcpyAsync(&r, cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    if (r == 0) return DSG_OK;
    if (r > cap) {
        set_error("kcore tail: %u vertices remain, more than the %u it was sized for", r, cap);
        return DSG_ECUDA;
    }
    uint64_t *coff, *roff;
    DSG_TRY_CUDA(sc.get(&coff, (size_t)r + 1));
    DSG_TRY_CUDA(sc.get(&roff, (size_t)r + 1));
    dsg_status st = scan_u32(cdeg, r, coff, sc, s);
    if (st != DSG_OK) return st;
    st = scan_u32(flen, r, roff, sc, s);
    if (st != DSG_OK) return st;
    uint64_t ecount = 0;
    DSG_TRY_CUDA(cudaMemcpyAsync(&ecount, coff + r, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    uint32_t *cadj, *fill;
    DSG_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t), s));  // now the fill's error word
    DSG_TRY_CUDA(sc.get(&cadj, ecount ? ecount : 1));
    DSG_TRY_CUDA(sc.get(&fill, r));
    DSG_TRY_CUDA(cudaMemsetAsync(fill, 0, (size_t)r * 4, s));
    {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tail_fill_kernel, 256, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        LaunchScope ls("kcore_tail_fill", s);
        tail_fill_kernel<<<(uint32_t)dev_info().sms * (uint32_t)per_sm, 256, 0, s>>>(r, roff, rid, off, adj, claim,
                                                                                    newid, coff, fill, cadj, cnt);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    if (ecount >= (uint64_t)kOffMax) {
        // row offsets do not fit the cluster's 32-bit row starts: finish with the grid-wide
        // kernel on the compacted graph instead, then put its core numbers in place
        uint32_t* ccore;
        DSG_TRY_CUDA(sc.get(&ccore, r));
        dsg_graph view;
        view.n = r;
        view.m = ecount / 2;
        view.off = coff;
        view.adj = cadj;
        view.owns = false;
        DSG_TRY_CUDA(cudaGetDevice(&view.device));
        view.stream = s;
        view.no_tail = true;
        uint64_t sub[5] = {0, 0, 0, 0, 0};
        dsg_status st2 = run_kcore(&view, ccore, sub, 5);
        if (st2 != DSG_OK) return st2;
        {
            LaunchScope ls("kcore_tail_scatter", s);
            tail_scatter_kernel<<<(r + 255) / 256, 256, 0, s>>>(r, rid, ccore, deg);
        }
        DSG_TRY_CUDA(cudaGetLastError());
        DSG_TRY_CUDA(cudaStreamSynchronize(s));
        if (stats5) {
            stats5[0] += sub[0];
            stats5[2] += sub[2];
            stats5[4] += sub[4];
        }
        if (stamps) *stamps = 0;
        return DSG_OK;
    }
    // ---- the cluster: 16 blocks (each holds at most kTailVPC vertices, so 16 always suffice)
    const uint32_t C = kTailC;
    const size_t smem = sizeof(TailSmem);
    DSG_TRY_CUDA(cudaFuncSetAttribute(kcore_tail_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (cudaFuncSetAttribute(kcore_tail_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        set_error("kcore tail: %u vertices need a cluster of %u blocks, which this device does not allow", r, C);
        return DSG_ECUDA;
    }
    TailArgs ta;
    ta.r = r;
    ta.off = coff;
    ta.adj = cadj;
    ta.cdeg = cdeg;
    ta.rid = rid;
    ta.core = deg;
    ta.limit_ns = wait_limit_ns();
    DSG_TRY_CUDA(sc.get(&ta.stats, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(ta.stats, 0, sizeof(TailStats), s));
    ta.trace = trace;
    ta.trace_cap = trace ? trace_cap : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kTailTB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    DSG_TRY_CUDA(cudaOccupancyMaxActiveClusters(&clusters, kcore_tail_kernel, &cfg));
    if (clusters < 1) {
        set_error("kcore tail: a cluster of %u blocks with %zu bytes of shared memory each does not fit", C, smem);
        return DSG_ECUDA;
    }
    {
        LaunchScope ls("kcore_tail", s);
        DSG_TRY_CUDA(cudaLaunchKernelEx(&cfg, kcore_tail_kernel, ta));
    }
    TailStats h;
    uint32_t fill_err = 0;
    DSG_TRY_CUDA(cudaMemcpyAsync(&h, ta.stats, sizeof(h), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaMemcpyAsync(&fill_err, cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    if (h.err & ERR_TIMEOUT) return status_from_err(h.err, "kcore tail");
    if (h.err || fill_err || h.claims != r) {
        set_error("kcore tail: inconsistent remaining graph (err %u, %llu of %u vertices placed)", h.err, h.claims, r);
        return DSG_ECUDA;
    }
    if (stats5) {
        stats5[0] += h.levels;
        stats5[2] += h.rem_scanned;
        stats5[4] += h.atomics;
    }
    if (stamps) *stamps = h.stamps;
    return DSG_OK;
}

}  // namespace dsg
