// Core numbers by the level-synchronous peel of Algorithm 2's first phase
// (PKC), as one persistent cooperative kernel; the blocks meet once per level,
// on a counter of outstanding work rather than a separate grid barrier.
//
// Level k (Alg. 2 first phase):
//   scan: every block walks its own segment of the remaining vertices; degree
//     <= k joins the level's frontier (Algorithm 2's per-thread buffer),
//     degree > k stays in the (compacted) segment;
//   drain: for every frontier vertex v and every neighbour u,
//     a = atomicSub(deg[u], 1); a == k+1 puts u in the frontier (it just
//     reached k); a <= k is undone with atomicAdd (u was already at or below
//     k) -- Algorithm 2's drain, except that Algorithm 2 first reads deg[u]
//     and skips u at or below k: decrementing at once saves one dependent
//     memory round trip per link of a cascade and leaves the same degrees.
//     A block drains the rows its scan found
//     (up to inline_max entries each) and the vertices that reach k while it
//     drains (rows up to local_max entries, while its local budget lasts:
//     PKC's thread-local buffer); everything else goes to a level-wide queue
//     of row pieces (at most chunk_len entries each) that blocks with no
//     work of their own take from as it comes, so neither hub rows nor
//     cascades that outgrow one block cost an extra grid-wide wait;
//   the level ends when the queue is drained and no block can add to it: a
//     counter holds one token per block (given back when its scan and own
//     draining are done) plus one per queued piece (given back once the piece
//     and everything it led the block to do locally are done), and the level
//     is over when it reaches zero.  Each block adds its least degree above
//     k and its claims to the level's totals before every give-back, so the
//     totals are final once the counter is zero and each block goes on to
//     the next level as soon as it sees that, with no grid barrier;
//   the count of visited vertices grows by the frontier size (as in Algorithm 2).
// Scan and drain overlap, so a vertex is taken into the frontier by claiming
// its bit in a bitmap (atomicOr): whichever of the scan and the decrement that
// brought it to k claims it first drains it, exactly once.  A scanned degree
// below k can only be such a vertex caught between a decrement and its undo:
// every vertex whose degree was below k at the level's start was claimed at an
// earlier level.
// Empty levels are skipped: the next k is the least degree above k seen by the
// scan and by every decrement of the level (the last value each vertex takes
// is among them, so no level with work is skipped).
// When visited == n, deg[v] is the core number of v.
//
// Per-level counters (queue tail, the token count, claims, least
// degree) sit in a ring of three sets, level L using set L % 3.  Block 0
// re-arms set (L+1) % 3 at the start of level L, before it gives back its
// level-L token: no block uses that set before it has seen level L's count at
// zero, and every block read the set's last totals (level L-2's) before it
// gave back its level-(L-1) token, which block 0 waited for.  Queue slots are reused by
// every level; a slot is published by writing the level's tag (level + 1)
// after its contents, so a stale slot is never taken for a new one.
#include <string.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace cg = cooperative_groups;

namespace dsg {

struct __align__(128) CoreLevel {
    unsigned long long pending;  // block tokens + queued pieces not yet drained
    unsigned long long pad0[15];
    unsigned long long tail;     // next queue slot a producer fills
    unsigned long long pad2[15];
    unsigned long long claimed;  // vertices claimed at this level
    uint32_t nmin;               // least degree above k seen
    uint32_t pad3[1];
    unsigned long long t_own, t_queue;  // traced runs: latest %globaltimer at which a block ended each phase
    unsigned long long scan_claims, pieces;  // traced runs: claims by the scan, row pieces queued
    uint32_t pad4[20];
};

struct __align__(128) CoreCtl {
    uint32_t bar;
    uint32_t pad0[31];
    uint32_t err;
    uint32_t pad1[31];
    uint32_t init_min;
    uint32_t pad2[31];
    CoreLevel lvl[3];
    unsigned long long atomics;  // statistics, summed by every block, never read in the kernel
    unsigned long long rem_scanned, rem_written, pieces;
    unsigned long long pad3[12];
    unsigned long long levels;
    unsigned long long dbg[4];   // bounds-check builds: first bad access (site, index, capacity, level)
    unsigned long long stamps;
    unsigned long long tail;     // the level loop stopped with this many vertices left for the cluster tail
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
    uint32_t* IV;     // level queue (cap slots) of row pieces: row owner ...
    uint64_t* IB;     // ... first entry
    uint32_t* IL;     // ... entries (<= chunk_len)
    uint32_t* IR;     // ... publication tag (level + 1)
    uint64_t cap;
    CoreCtl* ctl;
    uint64_t limit_ns;
    uint32_t chunk_len;
    uint32_t local_max;   // rows up to this length found while draining stay in the block
    uint32_t local_work;  // ... while the block's local entries per batch stay within this
    uint32_t inline_max;  // rows up to this length claimed by a block's scan are drained by that block
    uint32_t tail_max;    // leave the level loop once at most this many vertices remain (0: never)
    uint64_t* trace;      // nullable: block 0 stamps (%globaltimer, kind) at each phase end
    uint64_t trace_cap;
};

// Block-local frontier: vertices that reach k while this block drains are
// drained by the same block (PKC's thread-local buff, Algorithm 2), so a
// chain of degree-k vertices costs no queue round trip per link.
template <int TB>
constexpr uint32_t local_q_cap() { return TB >= 1024 ? 640 : 1024; }

#ifndef DSG_TAKE_SLOTS
#define DSG_TAKE_SLOTS 32
#endif
constexpr uint32_t kTakeSlots = DSG_TAKE_SLOTS;  // queue slots a block takes at a time
static_assert(kTakeSlots >= 1 && kTakeSlots <= 32, "a block takes 1..32 queue slots at a time");

template <int TB>
struct CoreSmem {
    static constexpr uint32_t kLocalQ = local_q_cap<TB>();
    TileSmem<TB> tile;
    BlockTile<TB> btile;
    uint32_t lq[kLocalQ];   // vertices ...
    uint64_t lqb[kLocalQ];  // ... their row starts
    uint32_t lql[kLocalQ];  // ... and row lengths
    uint32_t lq_tail;
    uint32_t lq_work;       // row entries this block has taken on locally in this batch
    uint32_t own;           // vertices this block's scan claimed
    uint32_t kept;          // vertices this block's scan kept
    uint32_t tv[kTakeSlots];  // queue pieces taken: row owner ...
    uint64_t tb[kTakeSlots];  // ... first entry
    uint32_t tl[kTakeSlots];  // ... entries
    uint32_t tcount;
    uint32_t flag;
    uint32_t acc_min;       // block reductions: least degree above k, claims (published during the level) ...
    unsigned long long acc_claimed, acc_atomics, acc_pieces;  // ... and statistics (end of the level)
    unsigned long long lvl_claimed;  // the level's totals, read once it is over
    uint32_t lvl_min, lvl_err;
    uint32_t redm[33];
};

// Claim v for a frontier; true for exactly one caller.
__device__ __forceinline__ bool claim_vertex(uint32_t* claim, uint32_t v) {
    const uint32_t bit = 1u << (v & 31u);
    return !(atomicOr(&claim[v >> 5], bit) & bit);
}

// Queue the row of v (start beg, len entries) as pieces of at most chunk_len
// entries for the level counted in P (tag = level + 1).  The token count is
// raised before a piece can be seen.  Called by any subset of lanes; the
// counters are updated once per group of lanes that call together.
__device__ __forceinline__ uint64_t queue_row(const CoreArgs& a, CoreLevel* P, uint32_t tag, uint32_t v,
                                              uint64_t beg, uint64_t len) {
    const uint64_t np = (len + a.chunk_len - 1) / a.chunk_len;
    cg::coalesced_group g = cg::coalesced_threads();
    uint64_t pre = np;  // inclusive prefix of the group's piece counts
    for (uint32_t o = 1; o < g.size(); o <<= 1) {
        const uint64_t t = g.shfl_up(pre, o);
        if (g.thread_rank() >= o) pre += t;
    }
    const uint64_t total = g.shfl(pre, g.size() - 1);
    pre -= np;
    unsigned long long base = 0;
    if (g.thread_rank() == 0 && total) {
        atomicAdd(&P->pending, (unsigned long long)total);
        base = atomicAdd(&P->tail, (unsigned long long)total);
    }
    base = g.shfl(base, 0);
    const uint64_t s0 = base + pre;
    for (uint64_t c = 0; c < np; ++c) {
        const uint64_t at = s0 + c;
        DSG_BOUND(a.ctl, 1, at, a.cap, tag, break);
        a.IV[at] = v;
        a.IB[at] = beg + c * a.chunk_len;
        a.IL[at] = (uint32_t)min((uint64_t)a.chunk_len, len - c * a.chunk_len);
    }
    // each tag is a release store: the lane's piece is visible before its tag
    for (uint64_t c = 0; c < np; ++c) {
        const uint64_t at = s0 + c;
        DSG_BOUND(a.ctl, 6, at, a.cap, tag, break);
        st_release_u32(&a.IR[at], tag);
    }
    return np;
}

template <int TB>
__global__ void __launch_bounds__(TB, TB == 256 ? 3 : 1) kcore_kernel(CoreArgs a) {
    __shared__ CoreSmem<TB> sm;
    CoreCtl* ctl = a.ctl;
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31u;
    const uint32_t n = a.n;
    uint64_t nstamp = 0;
    // trace entries: 2 words each, (time, kind << 32 | k); kind 0 start, 1 init, 2 level end;
    // block 0's own phases: 3 scan done, 4 own rows drained, 5 queue done;
    // after each level: 6 latest own-phase end over all blocks, 7 latest queue-phase end,
    // then (value, kind) pairs 8 claims, 9 claims by the scan, 10 queued pieces
    auto stamp = [&](uint32_t kind, uint32_t kk) {
        if (a.trace && blockIdx.x == 0 && tid == 0 && 2 * nstamp + 1 < a.trace_cap) {
            a.trace[2 * nstamp] = global_ns();
            a.trace[2 * nstamp + 1] = ((uint64_t)kind << 32) | kk;
        }
        ++nstamp;
    };
    stamp(0, 0);
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
    uint64_t visited = 0, level = 0;
    uint32_t* deg = a.deg;
    for (;;) {
        const uint32_t tag = (uint32_t)(level + 1);
        CoreLevel* P = &ctl->lvl[level % 3];
        if (blockIdx.x == 0 && tid == 0) {
            CoreLevel* R = &ctl->lvl[(level + 1) % 3];  // last read at level - 2, next used at level + 1
            R->pending = gridDim.x;
            R->tail = 0;
            R->claimed = 0;
            R->nmin = 0xffffffffu;
            R->t_own = 0;
            R->t_queue = 0;
            R->scan_claims = 0;
            R->pieces = 0;
        }
        uint32_t dmn = 0xffffffffu;
        uint64_t claimed = 0, natom = 0, npieces = 0, nscan_claims = 0;
        // u reached k: drain it in this block if there is room, else queue it
        // (a scan still running elsewhere may have taken it first)
        auto reach_k = [&](uint32_t u) {
            // the row bounds are loaded alongside the claim (one round trip)
            const uint64_t beg = a.off[u];
            const uint64_t end = a.off[u + 1];
            if (!claim_vertex(a.claim, u)) return;
            ++claimed;
            const uint64_t len = end - beg;
            if (len <= a.local_max && atomicAdd(&sm.lq_work, (uint32_t)len) + len <= a.local_work) {
                uint32_t pos = atomicAdd(&sm.lq_tail, 1u);
                if (pos < CoreSmem<TB>::kLocalQ) {
                    sm.lq[pos] = u;
                    sm.lqb[pos] = beg;
                    sm.lql[pos] = (uint32_t)len;
                    return;
                }
            }
            if (len) npieces += queue_row(a, P, tag, u, beg, len);
        };
        // one unit was just taken from u's degree, which was old: a degree
        // already at or below k gets it back (Algorithm 2's undo); reaching k
        // makes u the level's to drain
        auto settle = [&](uint32_t u, uint32_t old) {
            if (old <= k) {
                atomicAdd(&deg[u], 1u);
                ++natom;
                return;
            }
            const uint32_t nv = old - 1;
            if (nv == k) reach_k(u);
            else dmn = min(dmn, nv);
        };
        // every neighbour of a drained vertex that is not taken yet (its claim
        // bit, from a 1-bit-per-vertex map that stays in L2) loses one degree
        // at once (no read of the degree first); a neighbour already at or
        // below k, taken since its bit was read, gets it back in settle
        auto visit = [&](const uint32_t* u, const uint32_t* v, uint32_t valid) {
            uint32_t old[kBatch], cw[kBatch], need = 0;
#ifdef DSG_DEBUG_BOUNDS
            constexpr uint32_t kOutside = 0u;  // an id out of range reaches the bounds check below
#else
            constexpr uint32_t kOutside = 0xffffffffu;
#endif
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj)
                cw[jj] = !(valid >> jj & 1u) || u[jj] == v[jj] ? 0xffffffffu
                         : u[jj] < n                         ? a.claim[u[jj] >> 5]
                                                             : kOutside;
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj) {
                if (!(valid >> jj & 1u) || u[jj] == v[jj]) continue;
                if (cw[jj] >> (u[jj] & 31u) & 1u) continue;  // taken: nothing to take from it
#ifdef DSG_DEBUG_BOUNDS
                if (u[jj] >= n) {
                    DSG_BOUND(ctl, 4, u[jj], n, level, (void)0);
                    continue;
                }
#endif
                old[jj] = atomicSub(&deg[u[jj]], 1u);
                ++natom;
                need |= 1u << jj;
            }
#pragma unroll
            for (uint32_t jj = 0; jj < kBatch; ++jj)
                if (need >> jj & 1u) settle(u[jj], old[jj]);
        };
        // drain what this block found, until it finds nothing more
        auto local_loop = [&]() {
            for (uint32_t lq_lo = 0;;) {
                uint32_t lq_hi = min(sm.lq_tail, CoreSmem<TB>::kLocalQ);
                __syncthreads();
                if (lq_lo >= lq_hi) break;
                scan_block_rows<TB>(a.adj, sm.lq + lq_lo, sm.lqb + lq_lo, sm.lql + lq_lo, lq_hi - lq_lo, sm.btile,
                                    visit);
                lq_lo = lq_hi;
            }
        };
        // Publish the least degree above k and the claims this block has seen
        // since it last did, before the token or pieces that cover them are
        // given back: whoever sees the level's count reach zero then reads
        // final totals, with no grid barrier.
        auto publish = [&]() {
            const uint32_t wm = warp_min(dmn);
            const uint64_t wc = warp_sum(claimed);
            if (lane == 0) {
                if (wm != 0xffffffffu) atomicMin(&sm.acc_min, wm);
                if (wc) atomicAdd(&sm.acc_claimed, (unsigned long long)wc);
            }
            dmn = 0xffffffffu;
            claimed = 0;
            __syncthreads();
            if (tid == 0) {
                if (sm.acc_min != 0xffffffffu) atomicMin(&P->nmin, sm.acc_min);
                if (sm.acc_claimed) atomicAdd(&P->claimed, sm.acc_claimed);
                sm.acc_min = 0xffffffffu;
                sm.acc_claimed = 0;
            }
        };
        if (tid == 0) {
            sm.lq_tail = 0;
            sm.lq_work = 0;
            sm.own = 0;
            sm.kept = 0;
            sm.acc_min = 0xffffffffu;
            sm.acc_claimed = 0;
            sm.acc_atomics = 0;
            sm.acc_pieces = 0;
        }
        __syncthreads();
        // ---- scan: claim degree <= k, keep degree > k, drop the claimed.
        // kScanU tiles per step, their loads issued together.
        {
            constexpr uint32_t kScanU = TB >= 1024 ? 2 : 4;  // 1024-thread blocks have 64 registers
            uint32_t mn = 0xffffffffu;
            const uint64_t lim = my_rem ? my_n : n;
            const uint64_t stride = my_rem ? TB : (uint64_t)gridDim.x * TB;
            uint64_t scanned = 0;
            for (uint64_t t = my_rem ? 0 : (uint64_t)blockIdx.x * TB; t < lim; t += kScanU * stride) {
                uint32_t v[kScanU], dv[kScanU], cw[kScanU];
                bool in[kScanU];
#pragma unroll
                for (uint32_t u = 0; u < kScanU; ++u) {
                    const uint64_t i = t + u * stride + tid;
                    in[u] = i < lim;
                    v[u] = in[u] ? (my_rem ? my_rem[i] : (uint32_t)i) : 0u;
                }
                // the degree first; the claim word only where the degree is at or
                // below k (a vertex taken at an earlier level ended at its core
                // number, below k, so one above k is never taken)
#pragma unroll
                for (uint32_t u = 0; u < kScanU; ++u) dv[u] = in[u] ? deg[v[u]] : 0u;
#pragma unroll
                for (uint32_t u = 0; u < kScanU; ++u) cw[u] = (in[u] && dv[u] <= k) ? a.claim[v[u] >> 5] : 0u;
                bool keep[kScanU], mine[kScanU];
#pragma unroll
                for (uint32_t u = 0; u < kScanU; ++u) {
                    keep[u] = false;
                    mine[u] = false;
                    if (!in[u]) continue;
                    ++scanned;
                    if (cw[u] >> (v[u] & 31u) & 1u) continue;  // taken earlier
                    if (dv[u] > k) {
                        keep[u] = true;
                        mn = min(mn, dv[u]);
                    } else {
                        mine[u] = true;  // a candidate: claimed below
                    }
                }
                // row bounds of the candidates, loaded alongside their claims
                uint64_t beg[kScanU], len[kScanU];
#pragma unroll
                for (uint32_t u = 0; u < kScanU; ++u) {
                    beg[u] = mine[u] ? a.off[v[u]] : 0;
                    len[u] = mine[u] ? a.off[v[u] + 1] : 0;
                }
#pragma unroll
                for (uint32_t u = 0; u < kScanU; ++u)
                    if (mine[u]) mine[u] = claim_vertex(a.claim, v[u]);
#pragma unroll
                for (uint32_t u = 0; u < kScanU; ++u) {
                    if (!mine[u]) continue;
                    ++claimed;
                    ++nscan_claims;
                    const uint64_t ln = len[u] - beg[u];
                    // drained by this block, or, for rows above inline_max,
                    // queued in pieces for every block
                    if (ln <= a.inline_max) {
                        uint32_t pos = atomicAdd(&sm.own, 1u);
                        DSG_BOUND(ctl, 5, pos, a.seg, level, pos = 0);
                        myQA[pos] = v[u];
                        myQB[pos] = beg[u];
                        myQL[pos] = (uint32_t)ln;
                    } else {
                        npieces += queue_row(a, P, tag, v[u], beg[u], ln);
                    }
                }
                // keep: warp ballot, one shared-memory atomic per warp and tile
#pragma unroll
                for (uint32_t u = 0; u < kScanU; ++u) {
                    const uint32_t bal = __ballot_sync(kFullMask, keep[u]);
                    uint32_t base = 0;
                    if (lane == 0 && bal) base = atomicAdd(&sm.kept, (uint32_t)__popc(bal));
                    base = __shfl_sync(kFullMask, base, 0);
                    if (keep[u]) {
                        uint64_t at = base + __popc(bal & lanemask_lt());
                        bool ok = true;
                        DSG_BOUND(ctl, 3, at, a.seg, level, ok = false);
                        if (ok) my_rem_next[at] = v[u];
                    }
                }
            }
            dmn = min(dmn, mn);
            scanned = warp_sum(scanned);
            if (lane == 0 && scanned) atomicAdd(&ctl->rem_scanned, (unsigned long long)scanned);
        }
        __syncthreads();
        stamp(3, k);
        // ---- drain what this block's scan claimed, and what that leads to locally
        {
            const uint32_t own = (uint32_t)min((uint64_t)sm.own, a.seg);
            scan_block_rows<TB>(a.adj, myQA, myQB, myQL, own, sm.btile, visit);
            local_loop();
        }
        // the block adds nothing more except from queue pieces: give back its token
        publish();
        stamp(4, k);
        if (a.trace && tid == 0) atomicMax(&P->t_own, (unsigned long long)global_ns());
        if (tid == 0) {
            __threadfence();  // the block's work and totals before its token
            atomicAdd(&P->pending, ~0ull);  // minus one
        }
        // ---- take queue pieces until the level has none left and no block can add any.
        // Slot s belongs to block s mod grid, so consecutive pieces go to
        // different blocks; a block takes its next kTakeSlots slots at a time.
        // Each poll loads the slots' tags and the level's count together.
        for (uint64_t round = 0;; round += kTakeSlots) {
            const uint64_t slot = (uint64_t)blockIdx.x + (round + tid) * gridDim.x;
            bool todo = tid < kTakeSlots && slot < a.cap;
            if (!__syncthreads_or(todo)) {
                // past the queue's capacity: nothing more can come to this block
                if (tid == 0) {
                    const uint64_t w0 = global_ns();
                    while (ld_volatile_u64((const uint64_t*)&P->pending) != 0) {
                        if (global_ns() - w0 > a.limit_ns || (ld_volatile_u32(&ctl->err) & ERR_TIMEOUT)) {
                            atomicOr(&ctl->err, ERR_TIMEOUT);
                            break;
                        }
                        __nanosleep(256);
                    }
                }
                __syncthreads();
                break;
            }
            uint32_t spins = 0;
            uint64_t wait0 = tid == 0 ? global_ns() : 0;  // start of the current wait (thread 0)
            bool over = false;
            for (;;) {
                const bool rdy = todo && ld_acquire_u32(&a.IR[slot]) == tag;  // the piece was written before its tag
                if (tid == 0) {
                    sm.tcount = 0;
                    sm.lq_tail = 0;
                    sm.lq_work = 0;
                    // zero with this block's slots unready: a ready slot holds a
                    // piece the count still covers
                    sm.flag = ld_volatile_u64((const uint64_t*)&P->pending) == 0 ||
                              (ld_volatile_u32(&ctl->err) & ERR_TIMEOUT);
                }
                __syncthreads();
                if (rdy) {
                    const uint32_t pos = atomicAdd(&sm.tcount, 1u);
                    sm.tv[pos] = a.IV[slot];
                    sm.tb[pos] = a.IB[slot];
                    sm.tl[pos] = a.IL[slot];
                    todo = false;
                }
                __syncthreads();
                const uint32_t got = sm.tcount;
                if (got) {
                    scan_block_rows<TB>(a.adj, sm.tv, sm.tb, sm.tl, got, sm.btile, visit);
                    local_loop();
                    // drained, and whatever they queued is counted: publish, then give them back
                    publish();
                    if (tid == 0) {
                        __threadfence();
                        atomicAdd(&P->pending, 0ull - (unsigned long long)got);
                        wait0 = global_ns();
                    }
                    spins = 0;
                } else if (sm.flag) {
                    over = true;  // the level is over
                }
                if (over || !__syncthreads_or(todo)) break;  // over, or all taken slots done: take the next ones
                if (!got && tid == 0 && (++spins & 63u) == 0 && global_ns() - wait0 > a.limit_ns)
                    atomicOr(&ctl->err, ERR_TIMEOUT);  // seen at the next poll
            }
            if (over) break;
        }
        stamp(5, k);
        if (a.trace) {
            const uint64_t sc = warp_sum(nscan_claims), pc = warp_sum(npieces);
            if (lane == 0 && sc) atomicAdd(&P->scan_claims, (unsigned long long)sc);
            if (lane == 0 && pc) atomicAdd(&P->pieces, (unsigned long long)pc);
            if (tid == 0) atomicMax(&P->t_queue, (unsigned long long)global_ns());
        }
        // ---- the level is over: its totals are final (published before every
        // give-back); statistics are summed for the host
        natom = warp_sum(natom);
        npieces = warp_sum(npieces);
        if (lane == 0) {
            if (natom) atomicAdd(&sm.acc_atomics, (unsigned long long)natom);
            if (npieces) atomicAdd(&sm.acc_pieces, (unsigned long long)npieces);
        }
        if (tid == 0) {
            __threadfence();  // the count was seen at zero: every block's totals are visible
            sm.lvl_claimed = ld_volatile_u64((const uint64_t*)&P->claimed);
            sm.lvl_min = ld_volatile_u32(&P->nmin);
            sm.lvl_err = ld_volatile_u32(&ctl->err) & ERR_TIMEOUT;
        }
        __syncthreads();
        const uint64_t my_n_next = sm.kept;
        const uint64_t lvl_claimed = sm.lvl_claimed;
        const uint32_t level_min = sm.lvl_min;
        if (sm.lvl_err) return;
        if (tid == 0) {
            if (sm.acc_atomics) atomicAdd(&ctl->atomics, sm.acc_atomics);
            if (sm.acc_pieces) atomicAdd(&ctl->pieces, sm.acc_pieces);
            atomicAdd(&ctl->rem_written, (unsigned long long)my_n_next);
        }
        __syncthreads();  // every thread has read the block's totals before they are reset
        stamp(2, k);
        if (a.trace && blockIdx.x == 0 && tid == 0 && 2 * nstamp + 9 < a.trace_cap) {
            // the latest ends of the own-work and queue phases over the blocks
            // (as block 0 sees them: the queue phase of some blocks may still be
            // ending), and the level's claims (all / by the scan) and queued pieces
            a.trace[2 * nstamp] = ld_relaxed_u64(&P->t_own);
            a.trace[2 * nstamp + 1] = (6ull << 32) | k;
            a.trace[2 * nstamp + 2] = ld_relaxed_u64(&P->t_queue);
            a.trace[2 * nstamp + 3] = (7ull << 32) | k;
            a.trace[2 * nstamp + 4] = lvl_claimed;
            a.trace[2 * nstamp + 5] = (8ull << 32) | k;
            a.trace[2 * nstamp + 6] = ld_relaxed_u64(&P->scan_claims);
            a.trace[2 * nstamp + 7] = (9ull << 32) | k;
            a.trace[2 * nstamp + 8] = ld_relaxed_u64(&P->pieces);
            a.trace[2 * nstamp + 9] = (10ull << 32) | k;
        }
        if (a.trace) nstamp += 5;
        visited += lvl_claimed;
        ++level;
        if (visited >= n) break;
        if (a.tail_max && (uint64_t)n - visited <= a.tail_max) {
            // few vertices remain: the cluster finishes them on the compacted graph
            // (every block sees the same totals, so all leave here together)
            if (blockIdx.x == 0 && tid == 0) ctl->tail = (uint64_t)n - visited;
            break;
        }
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
    }
}

template <int TB>
static cudaError_t kcore_grid(const CoreArgs& a, uint32_t blocks_per_sm, uint32_t* grid, uint32_t max_grid) {
    return coop_grid(kcore_kernel<TB>, TB, 0, a.n, blocks_per_sm, grid, max_grid);
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
    Tuning tu = tuning_for(g, 1);
    if (g->force_block) tu.block = g->force_block;
    Scratch sc(s);
    CoreArgs a;
    a.n = n;
    a.off = g->off;
    a.adj = g->adj;
    a.limit_ns = wait_limit_ns();
    a.chunk_len = tu.chunk_len;
    a.local_max = tu.local_max;
    a.local_work = tu.local_work;
    a.inline_max = tu.inline_max;
    a.tail_max = g->no_tail ? 0 : (tu.tail_max < kTailMaxVertices ? tu.tail_max : kTailMaxVertices);
    a.trace = trace_dev;
    a.trace_cap = trace_cap;
    uint32_t grid = 1;
    cudaError_t e;
    switch (tu.block) {
        case 256: e = kcore_grid<256>(a, tu.blocks_per_sm, &grid, g->max_blocks); break;
        case 1024: e = kcore_grid<1024>(a, tu.blocks_per_sm, &grid, g->max_blocks); break;
        default: e = kcore_grid<512>(a, tu.blocks_per_sm, &grid, g->max_blocks); break;
    }
    DSG_TRY_CUDA(e);
    // a block scans at most ceil(n / (grid * block)) tiles of `block` vertices
    const uint64_t span = (uint64_t)grid * tu.block;
    a.seg = ((uint64_t)n + span - 1) / span * tu.block;
    // a level queues at most one piece per chunk_len entries of each row plus
    // one per vertex; blocks may take slots past that and skip them
    a.cap = (uint64_t)n + (2 * g->m) / tu.chunk_len + 1;
    bool direct = is_device_ptr(core_out);
    if (direct) a.deg = core_out;
    else DSG_TRY_CUDA(sc.get(&a.deg, n));
    DSG_TRY_CUDA(sc.get(&a.claim, ((uint64_t)n + 31) / 32));
    DSG_TRY_CUDA(sc.get(&a.remA, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.remB, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.QA, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.QB, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.QL, a.seg * grid));
    DSG_TRY_CUDA(sc.get(&a.IV, a.cap));
    DSG_TRY_CUDA(sc.get(&a.IB, a.cap));
    DSG_TRY_CUDA(sc.get(&a.IL, a.cap));
    DSG_TRY_CUDA(sc.get(&a.IR, a.cap));
    DSG_TRY_CUDA(cudaMemsetAsync(a.IR, 0, a.cap * sizeof(uint32_t), s));
    DSG_TRY_CUDA(sc.get(&a.ctl, 1));
    {
        CoreCtl init;
        memset(&init, 0, sizeof(init));
        init.init_min = 0xffffffffu;
        for (int i = 0; i < 3; ++i) {
            init.lvl[i].pending = grid;
            init.lvl[i].nmin = 0xffffffffu;
        }
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
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    if (c.dbg[0]) {
        set_error("kcore bounds check: site %llu index %llu capacity %llu level %llu", c.dbg[0], c.dbg[1], c.dbg[2],
                  c.dbg[3]);
        return DSG_ECUDA;
    }
    dsg_status st = status_from_err(c.err, "kcore");
    if (st != DSG_OK) return st;
    if (stamps) *stamps = c.stamps;
    // levels, queued pieces, remaining vertices scanned / written, degree atomics
    uint64_t vals[5] = {c.levels, c.pieces, c.rem_scanned, c.rem_written, c.atomics};
    if (c.tail) {
        // a traced run's tail stamps follow the grid kernel's
        const uint64_t used = trace_dev ? std::min<uint64_t>(2 * c.stamps, trace_cap) : 0;
        uint64_t tail_stamps = 0;
        st = kcore_tail(n, g->off, g->adj, a.deg, a.claim, (uint32_t)c.tail, s, vals,
                        trace_dev ? trace_dev + used : nullptr, trace_dev ? trace_cap - used : 0, &tail_stamps);
        if (st != DSG_OK) return st;
        if (stamps) *stamps += tail_stamps;
    }
    if (!direct) DSG_TRY_CUDA(copy_any(core_out, a.deg, (size_t)n * 4, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    for (uint32_t i = 0; stats && i < nstats && i < 5; ++i) stats[i] = vals[i];
    return DSG_OK;
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

// Phase timestamps of one core decomposition (debug/analysis): pairs
// (%globaltimer, kind << 32 | k) as the kernel's trace stamps them (kind 0
// start, 1 degrees initialised, 2 level over, 3/4/5 block 0's phases, then
// per level the five (value, kind) pairs 6..10).  *count = pairs taken.
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
