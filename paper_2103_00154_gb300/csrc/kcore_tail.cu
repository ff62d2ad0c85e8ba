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
// remaining levels with every vertex's degree, claim bit and queue slot in
// the distributed shared memory of the cluster: vertex i belongs to block
// i % C.  Level k: each block scans its own vertices (a list of the ones not
// yet taken, compacted every level) and claims those of degree <= k; a
// drained vertex's neighbours above k lose one degree each (Algorithm 2's
// drain, reading the degree first); a neighbour brought to k is claimed by
// the decrementer and queued at its owner, so every block drains its own
// vertices and a cascade spreads over the cluster.  A cluster-wide count of
// claimed vertices not yet drained (plus one token per block until its scan
// is done) reaching zero ends the level; the blocks then meet at a cluster
// barrier and sum the level's claims and least degree above k, so every
// block takes the same decisions.  Every wait is bounded (ERR_TIMEOUT).
#include <cooperative_groups.h>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace cg = cooperative_groups;

namespace dsg {

constexpr uint32_t kTailTB = 1024;
constexpr uint32_t kTailVPC = 8192;   // vertices per block at most
constexpr uint32_t kSlotEmpty = 0xffffffffu;

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
    uint32_t deg[kTailVPC];
    uint32_t claim[kTailVPC / 32];
    uint16_t rem[2][kTailVPC];
    uint2 q[kTailVPC];           // this block's vertices to drain at this level: (row start, length);
                                 // x == kSlotEmpty until the claimer has written it
    uint32_t start[kTailTB];     // a batch's rows: exclusive prefix of lengths ...
    uint64_t beg[kTailTB];       // ... row starts
    uint32_t red[33];
    uint64_t red64[33];
    uint32_t qtail, nkeep, batch_n, batch_total, stop;
    uint32_t pending[2];         // block 0 only, by level parity: claimed-not-drained vertices + block tokens
    uint32_t pub_min[2], pub_claims[2], pub_err[2];  // a level's totals, by level parity
    uint32_t tot_min, tot_err;
    unsigned long long tot_claims;
};

__global__ void __launch_bounds__(kTailTB, 1) kcore_tail_kernel(TailArgs a) {
    extern __shared__ __align__(16) unsigned char tail_smem_raw[];
    TailSmem& sm = *reinterpret_cast<TailSmem*>(tail_smem_raw);
    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t C = cluster.num_blocks();
    const uint32_t rank = cluster.block_rank();
    const uint32_t tid = threadIdx.x;
    const uint32_t r = a.r;
    const uint32_t V = r > rank ? (r - rank + C - 1) / C : 0;  // this block's vertices: i = li * C + rank
    // ---- degrees, claim bits, queue slots, the list of this block's vertices; least degree
    uint32_t mn = 0xffffffffu;
    for (uint32_t li = tid; li < V; li += kTailTB) {
        const uint32_t d = a.cdeg[li * C + rank];
        sm.deg[li] = d;
        sm.rem[0][li] = (uint16_t)li;
        mn = min(mn, d);
    }
    for (uint32_t w = tid; w < kTailVPC / 32; w += kTailTB) sm.claim[w] = 0;
    for (uint32_t i = tid; i < kTailVPC; i += kTailTB) sm.q[i] = make_uint2(kSlotEmpty, 0u);
    mn = block_min_u32(mn, sm.red);
    if (tid == 0) {
        sm.pub_min[1] = mn;
        sm.pub_claims[1] = 0;
        sm.pub_err[1] = 0;
        sm.qtail = 0;
        sm.pending[0] = C;  // (block 0's copy is the one used) every block's token for level 0
        sm.pending[1] = 0;
    }
    cluster.sync();
    uint32_t k = 0xffffffffu;
    for (uint32_t q = 0; q < C; ++q) k = min(k, *cluster.map_shared_rank(&sm.pub_min[1], (int)q));
    uint64_t visited = 0, level = 0, scanned = 0, natom = 0, nstamp = 0;
    uint32_t nrem = V;
    bool bad = false, timeout = false;
    // trace pairs: kind 11 scan done, 12 drain done, 13 level over (block 0), 14 the level's claims
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
        uint32_t lmin = 0xffffffffu, lclaims = 0;
        uint32_t* const pending0 = cluster.map_shared_rank(&sm.pending[par], 0);
        if (tid == 0) sm.nkeep = 0;
        __syncthreads();
        // ---- scan: claim degree <= k (queued here), keep degree > k
        for (uint32_t j0 = 0; j0 < nrem; j0 += kTailTB) {
            const uint32_t j = j0 + tid;
            bool keep = false;
            uint32_t li = 0;
            if (j < nrem) {
                li = cur[j];
                const bool taken = (*reinterpret_cast<volatile uint32_t*>(&sm.claim[li >> 5]) >> (li & 31u)) & 1u;
                if (!taken) {
                    const uint32_t d = *reinterpret_cast<volatile uint32_t*>(&sm.deg[li]);
                    if (d > k) {
                        keep = true;
                        lmin = min(lmin, d);
                    } else {
                        const uint32_t bit = 1u << (li & 31u);
                        const uint32_t i = li * C + rank;
                        const uint64_t b0 = a.off[i], b1 = a.off[i + 1];
                        if (!(atomicOr(&sm.claim[li >> 5], bit) & bit)) {
                            ++lclaims;
                            sm.q[atomicAdd(&sm.qtail, 1u)] = make_uint2((uint32_t)b0, (uint32_t)(b1 - b0));
                        }
                    }
                }
            }
            const uint32_t bal = __ballot_sync(kFullMask, keep);
            uint32_t base = 0;
            if ((tid & 31u) == 0 && bal) base = atomicAdd(&sm.nkeep, (uint32_t)__popc(bal));
            base = __shfl_sync(kFullMask, base, 0);
            if (keep) nxt[base + __popc(bal & lanemask_lt())] = (uint16_t)li;
        }
        if (tid == 0) scanned += nrem;
        {
            // the scan's claims count as pending before this block's token is given back
            const uint32_t c = (uint32_t)block_sum<uint64_t>((uint64_t)lclaims, sm.red64);
            if (tid == 0) atomicAdd(pending0, c - 1u);  // + claims - token
        }
        stamp(11, global_ns());
        // ---- drain: a neighbour above k loses one degree (Algorithm 2's
        // drain reads it first; a neighbour at or below k is taken or being
        // taken and is skipped); if a concurrent drain got it to k first, the
        // decrement is undone; one brought to k is claimed and queued at its owner
        auto visit = [&](const uint32_t* u, const uint32_t* v, uint32_t valid) {
            uint32_t d[kBatch], old[kBatch], live = 0;
            uint32_t* dp[kBatch];
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj) {
                dp[jj] = nullptr;
                d[jj] = 0;
                if (!(valid >> jj & 1u)) continue;
                if (u[jj] >= r) {
                    bad = true;
                    continue;
                }
                dp[jj] = cluster.map_shared_rank(&sm.deg[u[jj] / C], (int)(u[jj] % C));
                d[jj] = *reinterpret_cast<volatile uint32_t*>(dp[jj]);
            }
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj) {
                if (dp[jj] && d[jj] > k) {
                    old[jj] = atomicSub(dp[jj], 1u);
                    ++natom;
                    live |= 1u << jj;
                }
            }
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj) {
                if (!(live >> jj & 1u)) continue;
                if (old[jj] <= k) {
                    atomicAdd(dp[jj], 1u);
                    ++natom;
                } else if (old[jj] - 1 == k) {
                    const uint32_t uu = u[jj], lu = uu / C, ow = uu % C;
                    uint32_t* cw = cluster.map_shared_rank(&sm.claim[lu >> 5], (int)ow);
                    const uint32_t bit = 1u << (lu & 31u);
                    const uint64_t b0 = a.off[uu], b1 = a.off[uu + 1];  // loaded alongside the claim
                    if (!(atomicOr(cw, bit) & bit)) {
                        ++lclaims;
                        // pending up and a slot at the owner, both waited for before the slot is
                        // written: the count never reads zero while u is claimed but not yet queued
                        const uint32_t was = atomicAdd(pending0, 1u);
                        const uint32_t slot = atomicAdd(cluster.map_shared_rank(&sm.qtail, (int)ow), 1u);
                        if (was == 0xffffffffu || slot >= kTailVPC) {
                            bad = true;
                        } else {
                            // one 8-byte store: the owner sees the slot empty or complete
                            volatile unsigned long long* sp = reinterpret_cast<volatile unsigned long long*>(
                                cluster.map_shared_rank(&sm.q[slot], (int)ow));
                            *sp = ((unsigned long long)(uint32_t)(b1 - b0) << 32) | (uint32_t)b0;
                        }
                    }
                } else {
                    lmin = min(lmin, old[jj] - 1);
                }
            }
        };
        // ---- drain this block's queue until the cluster has nothing pending
        uint32_t qhead = 0;
        const uint64_t w0 = global_ns();
        uint64_t wait_start = w0;
        for (;;) {
            if (tid == 0) {
                const uint32_t t = *reinterpret_cast<volatile uint32_t*>(&sm.qtail);
                uint32_t take = min(t - qhead, kTailTB);
                sm.stop = 0;
                if (take == 0) {
                    // nothing queued here: the level is over once nothing is pending anywhere
                    if (*reinterpret_cast<volatile uint32_t*>(pending0) == 0) sm.stop = 1;
                    else if (global_ns() - wait_start > a.limit_ns) { sm.stop = 1; timeout = true; }
                    else __nanosleep(64);
                }
                sm.batch_n = take;
            }
            __syncthreads();
            const uint32_t nb = sm.batch_n;
            if (sm.stop) break;
            if (nb == 0) {
                __syncthreads();
                continue;
            }
            // the batch's rows: slots qhead .. qhead + nb, (row start, length) each, written by the
            // claimer right after it reserved the slot (length first, start last): wait for it, bounded
            uint32_t len = 0;
            uint64_t bg = 0;
            if (tid < nb) {
                volatile unsigned long long* sl = reinterpret_cast<volatile unsigned long long*>(&sm.q[qhead + tid]);
                unsigned long long x = *sl;
                const uint64_t s0 = global_ns();
                while ((uint32_t)x == kSlotEmpty) {
                    if (global_ns() - s0 > a.limit_ns) { timeout = true; break; }
                    x = *sl;
                }
                if ((uint32_t)x != kSlotEmpty) {
                    bg = (uint32_t)x;
                    len = (uint32_t)(x >> 32);
                }
            }
            uint32_t total;
            const uint32_t st = block_excl_scan<uint32_t>(len, sm.red, &total);
            sm.start[tid] = st;
            sm.beg[tid] = bg;
            __syncthreads();
            for (uint32_t e0 = tid; e0 < total; e0 += kBatch * kTailTB) {
                uint32_t bu[kBatch], bv[kBatch], valid = 0;
#pragma unroll
                for (uint32_t j = 0; j < kBatch; ++j) {
                    const uint32_t e = e0 + j * kTailTB;
                    bu[j] = 0;
                    bv[j] = 0;
                    if (e < total) {
                        uint32_t lo = 0, hi = nb;  // row = last whose start is <= e
                        while (hi - lo > 1) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (sm.start[mid] <= e) lo = mid; else hi = mid;
                        }
                        bu[j] = ld_stream(a.adj + sm.beg[lo] + (e - sm.start[lo]));
                        valid |= 1u << j;
                    }
                }
                visit(bu, bv, valid);
            }
            __syncthreads();  // every drain of the batch (and the claims it made) is done
            if (tid == 0) atomicSub(pending0, nb);
            qhead += nb;
            wait_start = global_ns();
        }
        stamp(12, global_ns());
        // ---- the level's totals over the cluster; queue slots back to empty for the next level
        for (uint32_t i = tid; i < qhead; i += kTailTB) sm.q[i] = make_uint2(kSlotEmpty, 0u);
        lmin = block_min_u32(lmin, sm.red);
        const uint64_t bc = block_sum<uint64_t>((uint64_t)lclaims, sm.red64);
        const uint32_t to = __syncthreads_or(timeout || bad);
        if (tid == 0) {
            sm.pub_min[par] = lmin;
            sm.pub_claims[par] = (uint32_t)bc;
            sm.pub_err[par] = to;
            sm.qtail = 0;
            // the next level's tokens: that count was last used at the previous level, which every
            // block left before the previous barrier
            if (rank == 0) sm.pending[par ^ 1u] = C;
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
    if ((tid & 31u) == 0) {
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
    if (ecount >= (uint64_t)kSlotEmpty) {
        // row offsets do not fit the cluster's 32-bit queue slots: finish with the grid-wide
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
    const uint32_t C = 16;
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
