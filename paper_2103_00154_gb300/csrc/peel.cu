// Algorithm 1 (P-Bahmani): the round-synchronous (2+2eps) densest-subgraph
// peel as one persistent cooperative kernel.
//
// Per round r, with S_r and E_r = |E(S_r)| known to every block:
//   phase 1 (Algorithm 1's first part, over the active vertices): every alive vertex is
//     tested against T_r = floor(2(p+q)E_r / (q|S_r|)), i.e. deg <= 2(1+eps)rho
//     exactly; failures are marked (state word and status map) and queued
//     (short rows with their row bounds, long rows as chunk items), survivors
//     are compacted into the next alive list (warp ballot + block scan + one
//     atomic per block and list); the degrees of the failures are summed (X);
//   grid barrier (Algorithm 1's synchronisation between its two parts);
//   phase 2 (Alg. 1 part 2): every adjacency entry u of every failed v is read
//     once; u's bits in the status map say whether it is still alive (and
//     whether it is a hub); an alive u loses one degree (atomicSub, combined
//     per block for hubs) and the decrement is counted (D);
//   grid barrier; every block derives S_{r+1} and E_{r+1} from the monotone
//     counters and keeps the densest set (strict ">": a later round replaces
//     the best only when strictly denser, as in Algorithm 1); block 0 records
//     the history.
// The edges removed in round r (Algorithm 1's reduction) are (X + D) / 2: the
// failures' degrees count every edge between two failures twice and every
// edge from a failure to a survivor once, and D counts the latter once more.
// So phase 2 never needs to tell a neighbour that failed in this round from
// one that failed earlier, and reads only the status map (2 bits per vertex,
// L2-resident) rather than the state words.
//
// Vertex state is one 32-bit word: an alive vertex holds its degree inside
// S_r (< 2^31); a failed one holds 0x80000000 | (round it failed, 1-based).
// Status map: word u / 16, bit 2 (u % 16) = u has failed, bit 2 (u % 16) + 1
// = u is a hub (first-round degree at or above the hub threshold).
#include <algorithm>
#include <cstdlib>
#include <string>
#include <thread>
#include <vector>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace dsg {

constexpr uint32_t kDead = 0x80000000u;

struct __align__(128) PeelCtl {
    uint32_t bar;
    uint32_t pad0[31];
    uint32_t err;
    uint32_t pad1[31];
    unsigned long long failed;  // sum of |A_t|
    unsigned long long pad2[15];
    unsigned long long nshort;  // cursor of the short-row failed list
    unsigned long long pad3[15];
    unsigned long long nchunk;  // cursor of the chunk-item list
    unsigned long long pad4[15];
    unsigned long long surv;    // cursor of survivor writes (all rounds)
    unsigned long long pad5[15];
    unsigned long long xsum;    // sum over the rounds of the failures' degrees (X)
    unsigned long long pad6[15];
    unsigned long long dec;     // alive-neighbour decrements (D)
    unsigned long long pad7[15];
    unsigned long long cand;    // cursor of candidate-list writes (all rounds)
    unsigned long long pad8[15];
    unsigned long long tested, lazy_rounds;  // statistics kept by block 0: vertex tests, lazy rounds
    unsigned long long rounds, best_round, best_E, best_V;
    unsigned long long stamps;
    unsigned long long cur_S, cur_E;  // |S_r| and |E(S_r)| where the launch stopped
};

struct PeelArgs {
    uint32_t n;
    uint64_t m;
    uint64_t p, q;
    const uint64_t* off;
    const uint32_t* adj;
    uint32_t* st;
    uint32_t* listA;
    uint32_t* listB;
    uint32_t* F;
    uint64_t* FB;         // nullable: row start ...
    uint32_t* FL;         // ... and length of each F entry (else read from off)
    uint64_t* C;
    uint32_t* map;        // status map, (n + 15) / 16 words
    uint32_t* candA;      // nullable (then no lazy rounds): two candidate lists of n entries
    uint32_t* candB;
    uint64_t* hist_S;
    uint64_t* hist_E;
    uint64_t hist_cap;
    PeelCtl* ctl;
    uint64_t limit_ns;
    uint32_t short_max;
    uint32_t chunk_len;
    uint32_t hot_deg;
    uint32_t vec_loads;   // 1: long rows read as aligned 128-bit groups when adj is 16-byte aligned
    uint64_t* trace;      // nullable: block 0 stamps %globaltimer after every barrier
    uint64_t trace_cap;
    // resuming a paused peel (r0 > 0): the state words in st are the pause's,
    // S0/E0/best the pause's values, and the first round scans every vertex,
    // skipping those already failed; max_rounds > 0 pauses after that many rounds
    uint64_t r0, S0, E0, best_round0, best_E0, best_V0;
    uint64_t max_rounds;
};

// floor(2(p+q)E / (qS)) clamped to 32 bits; S > 0.
__device__ __forceinline__ uint32_t peel_threshold(uint64_t p, uint64_t q, uint64_t E, uint64_t S) {
    unsigned __int128 num = (unsigned __int128)2 * (unsigned __int128)(p + q) * (unsigned __int128)E;
    unsigned __int128 den = (unsigned __int128)q * (unsigned __int128)S;
    unsigned __int128 t = num / den;
    return t > (unsigned __int128)0xffffffffu ? 0xffffffffu : (uint32_t)t;
}

template <int TB>
struct PeelSmem {
    TileSmem<TB> tile;
    AggTable agg;
    uint64_t bases[4];
    uint64_t red[33];
    uint32_t surv_at[4][TB / 32];  // a tile's survivors per (slice, warp), then their exclusive prefix in id order
};

// Bits 0..15 of x spread to the even positions 0, 2, ..., 30.
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

template <int TB>
__global__ void __launch_bounds__(TB, 65536 / (TB * 40)) peel_kernel(PeelArgs a) {
    __shared__ PeelSmem<TB> sm;
    PeelCtl* ctl = a.ctl;
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const bool resume = a.r0 > 0;
    uint64_t S = resume ? a.S0 : a.n, E = resume ? a.E0 : a.m;
    uint64_t r = a.r0;
    uint64_t short_lo = 0, chunk_lo = 0, surv_base = 0;
    const uint32_t* alive = nullptr;  // first round: identity (a fresh peel) or every vertex (a resumed one)
    uint32_t* next = a.listA;
    uint64_t alive_len = 0;           // entries of `alive` (after lazy rounds some of them have failed)
    // lazy rounds (thin tail): the candidate list holds every alive vertex whose degree is at or below
    // the bound B; a round whose threshold is within B tests only that list
    const bool lazy_ok = a.candA != nullptr;
    uint32_t* cur_cand = a.candA;
    uint32_t* next_cand = a.candB;
    uint64_t cand_n = 0, cand_base = 0, S_prev = S;
    bool have_cands = false;
    uint32_t B = 0;
    uint64_t best_E = resume ? a.best_E0 : E, best_V = resume ? a.best_V0 : S;
    uint64_t best_round = resume ? a.best_round0 : 0;
    uint64_t nstamp = 0;
    auto stamp = [&]() {
        if (a.trace && blockIdx.x == 0 && tid == 0 && nstamp < a.trace_cap) a.trace[nstamp] = global_ns();
        ++nstamp;
    };
    stamp();
    agg_clear(sm.agg);
    const uint32_t hot = hot_threshold(a.hot_deg);
    // long rows by 128-bit loads when the adjacency is 16-byte aligned (a view into a packed
    // batch may not be); groups are only read whole inside the 2m entries
    const uint64_t vec_end = (a.vec_loads && (reinterpret_cast<uintptr_t>(a.adj) & 15u) == 0) ? 2 * a.m : 0;
    if (blockIdx.x == 0 && tid == 0 && !resume) {
        a.hist_S[0] = S;
        a.hist_E[0] = E;
    }
    while (S > 0) {
        const uint32_t T = peel_threshold(a.p, a.q, E, S);
        const uint32_t mark = kDead | (uint32_t)(r + 1);
        // ------------------------------------------------ phase 1: test + compact
        // the first round of a launch walks vertex ids in order (every vertex, or
        // every vertex a resumed peel has not failed yet) and writes the status map
        // whole, two words per warp; later rounds walk the alive list and set the
        // failures' bits
        const bool fresh = r == 0;                  // identity list, degrees from the rows
        const bool scan_all = !alive && resume;     // a resumed peel's first round: every vertex, failed ones skipped
        const bool by_id = fresh || scan_all;
        // thin: the last round removed less than 1/8 of the vertices; then this round collects the
        // next round's candidates (bound Bn), and it is lazy when the current list covers T
        const bool thin = lazy_ok && !fresh && (S_prev - S) * 8 < S_prev;
        const bool lazy = thin && have_cands && !by_id && T <= B && cand_n * 4 < S;
        const uint32_t Bn = lazy ? B : (thin ? T + T / 128u : 0u);
        const uint64_t span = by_id ? (scan_all ? a.n : S) : (lazy ? cand_n : alive_len);
        const uint32_t* src = lazy ? cur_cand : alive;
        if (blockIdx.x == 0 && tid == 0) {
            ctl->tested += span;
            ctl->lazy_rounds += lazy ? 1u : 0u;
        }
        // a tile is `items` slices of TB: thread tid takes i = t + j TB + tid for
        // j < items (4 in the by-id rounds, whose tiles would otherwise be
        // short; 1 on the alive list); the first pass tests and marks, the
        // second writes the lists at the tile's reserved places
        const uint32_t items = by_id ? 4u : 1u;
        uint64_t X = 0;
        for (uint64_t t = (uint64_t)blockIdx.x * TB * items; t < span; t += (uint64_t)gridDim.x * TB * items) {
            uint32_t fail_m = 0, short_m = 0, surv_m = 0, cand_m = 0, nch_sum = 0;
            uint64_t c_beg = 0, c_len = 0;  // the alive-list rounds' one item: its row, for the second pass
            for (uint32_t j = 0; j < items; ++j) {
                const uint64_t i = t + (uint64_t)j * TB + tid;
                bool valid = i < span;
                bool gone = false;  // failed in an earlier round (resumed first round)
                uint32_t v = 0, d = 0;
                uint64_t len = 0;
                bool fail = false;
                if (valid) {
                    if (by_id) {
                        v = (uint32_t)i;
                        len = a.off[v + 1] - a.off[v];
                        if (fresh) {
                            d = (uint32_t)len;
                        } else {
                            d = a.st[v];
                            gone = (d & kDead) != 0;
                        }
                    } else {
                        v = src[i];
                        d = a.st[v];
                        gone = (d & kDead) != 0;  // an alive list left from before lazy rounds
                    }
                }
                const bool hub = by_id && valid && len >= hot;
                if (valid && !gone) {
                    fail = d <= T;
                    if (fail) {
                        if (!by_id) {
                            c_beg = a.off[v];
                            len = a.off[v + 1] - c_beg;
                            c_len = len;
                        }
                        a.st[v] = mark;
                        X += d;
                        if (len > a.short_max) {
                            nch_sum += (uint32_t)((len + a.chunk_len - 1) / a.chunk_len);
                        } else {
                            short_m |= 1u << j;
                        }
                        fail_m |= 1u << j;
                        if (!by_id) atomicOr(&a.map[v >> 4], 1u << (2u * (v & 15u)));
                    } else {
                        if (!lazy) surv_m |= 1u << j;
                        if (thin && d <= Bn) cand_m |= 1u << j;
                        if (fresh) a.st[v] = d;
                    }
                }
                if (by_id) {
                    // each warp holds 32 consecutive ids starting at a multiple of 32
                    const uint32_t bd = __ballot_sync(kFullMask, fail || gone);
                    const uint32_t bh = __ballot_sync(kFullMask, hub);
                    const uint64_t i0 = t + (uint64_t)j * TB + (tid & ~31u);
                    if (lane == 0 && i0 < a.n) a.map[i0 >> 4] = spread16(bd) | (spread16(bh) << 1);
                    if (lane == 16 && i0 + 16 < a.n)
                        a.map[(i0 >> 4) + 1] = spread16(bd >> 16) | (spread16(bh >> 16) << 1);
                }
            }
            // survivors go to the next list in id order within the tile (slice, then
            // warp, then lane), so the next round reads the states in order
            for (uint32_t j = 0; j < items; ++j) {
                const uint32_t c = __popc(__ballot_sync(kFullMask, surv_m >> j & 1u));
                if (lane == 0) sm.surv_at[j][tid >> 5] = c;
            }
            const uint32_t ns_t = __popc(short_m), nl_t = __popc(fail_m) - ns_t;
            // packed counts: short | long-fail << 32 (at most 4 TB of each per tile)
            uint64_t pk = (uint64_t)ns_t | ((uint64_t)nl_t << 32);
            uint64_t pk_tot;
            uint64_t pk_pre = block_excl_scan<uint64_t>(pk, sm.tile.scan_tmp64, &pk_tot);
            uint32_t ch_tot;
            uint32_t ch_pre = block_excl_scan<uint32_t>(nch_sum, sm.tile.scan_tmp, &ch_tot);
            uint64_t nv = 0;
            if (tid < 32) {
                // exclusive prefix of the (slice, warp) survivor counts, slice-major
                constexpr uint32_t kW = TB / 32;
                const uint32_t per = (items * kW + 31) / 32;  // counts per lane, consecutive
                uint32_t loc[4], sum = 0;
                for (uint32_t q = 0; q < per; ++q) {
                    const uint32_t idx = tid * per + q;
                    loc[q] = idx < items * kW ? sm.surv_at[idx / kW][idx % kW] : 0u;
                    sum += loc[q];
                }
                const uint32_t inc = warp_incl_scan(sum);
                nv = __shfl_sync(kFullMask, inc, 31);
                uint32_t run = inc - sum;
                for (uint32_t q = 0; q < per; ++q) {
                    const uint32_t idx = tid * per + q;
                    if (idx < items * kW) sm.surv_at[idx / kW][idx % kW] = run;
                    run += loc[q];
                }
            }
            if (tid == 0) {
                uint64_t ns = pk_tot & 0xffff, nl = (pk_tot >> 32) & 0xffff;
                sm.bases[0] = ns ? atomicAdd(&ctl->nshort, ns) : 0;
                sm.bases[1] = nv ? atomicAdd(&ctl->surv, nv) : 0;
                sm.bases[2] = ch_tot ? atomicAdd(&ctl->nchunk, (unsigned long long)ch_tot) : 0;
                if (ns + nl) atomicAdd(&ctl->failed, ns + nl);
            }
            __syncthreads();
            uint64_t at_s = sm.bases[0] + (pk_pre & 0xffff);
            const uint64_t v0 = sm.bases[1] - surv_base;
            uint64_t at_c = sm.bases[2] + ch_pre;
            for (uint32_t j = 0; j < items; ++j) {
                const uint64_t i = t + (uint64_t)j * TB + tid;
                uint32_t v = 0, nch = 0;
                if ((fail_m | surv_m | cand_m) >> j & 1u) v = by_id ? (uint32_t)i : src[i];
                if (short_m >> j & 1u) {
                    a.F[at_s] = v;
                    if (a.FB) {
                        const uint64_t b0 = by_id ? a.off[v] : c_beg;
                        a.FB[at_s] = b0;
                        a.FL[at_s] = (uint32_t)(by_id ? a.off[v + 1] - b0 : c_len);
                    }
                    ++at_s;
                } else if (fail_m >> j & 1u) {
                    const uint64_t len = by_id ? a.off[v + 1] - a.off[v] : c_len;
                    nch = (uint32_t)((len + a.chunk_len - 1) / a.chunk_len);
                }
                {
                    const uint32_t sb = __ballot_sync(kFullMask, surv_m >> j & 1u);
                    if (surv_m >> j & 1u) next[v0 + sm.surv_at[j][tid >> 5] + __popc(sb & lanemask_lt())] = v;
                    // candidates for the next round: one atomic per warp
                    const uint32_t cb = __ballot_sync(kFullMask, cand_m >> j & 1u);
                    if (cb) {
                        unsigned long long cbase = 0;
                        if (lane == 0) cbase = atomicAdd(&ctl->cand, (unsigned long long)__popc(cb));
                        cbase = __shfl_sync(kFullMask, cbase, 0);
                        if (cand_m >> j & 1u) next_cand[cbase - cand_base + __popc(cb & lanemask_lt())] = v;
                    }
                }
                // chunk items of the warp's long failures, written by the whole warp
                // (a hub has hundreds of them)
                for (uint32_t pend = __ballot_sync(kFullMask, nch != 0); pend; pend &= pend - 1) {
                    const uint32_t src = __ffs(pend) - 1;
                    const uint32_t cn = __shfl_sync(kFullMask, nch, src);
                    const uint32_t cv = __shfl_sync(kFullMask, v, src);
                    const uint64_t c0 = __shfl_sync(kFullMask, at_c, src);
                    for (uint32_t c = lane; c < cn; c += 32) a.C[c0 + c] = ((uint64_t)cv << 32) | c;
                }
                at_c += nch;
            }
            __syncthreads();
        }
        {
            const uint64_t bx = block_sum<uint64_t>(X, sm.red);
            if (tid == 0 && bx) atomicAdd(&ctl->xsum, (unsigned long long)bx);
        }
        if (!grid_barrier(&ctl->bar, &ctl->err, a.limit_ns)) return;
        stamp();
        const uint64_t failed_hi = ld_relaxed_u64(&ctl->failed);
        const uint64_t short_hi = ld_relaxed_u64(&ctl->nshort);
        const uint64_t chunk_hi = ld_relaxed_u64(&ctl->nchunk);
        // ------------------------------------------------ phase 2: neighbour scan
        uint64_t ndec = 0;
        uint32_t* st = a.st;
        const uint32_t* map = a.map;
        auto visit = [&](const uint32_t* u, const uint32_t*, uint32_t valid) {
            uint32_t w[kBatch];
#pragma unroll
            for (uint32_t j = 0; j < kBatch; ++j) {
#ifdef DSG_DEBUG_BOUNDS
                if ((valid >> j & 1u) && u[j] >= a.n) { atomicOr(&ctl->err, ERR_RANGE); valid &= ~(1u << j); }
#endif
                w[j] = (valid >> j & 1u) ? map[u[j] >> 4] : 1u;
            }
#pragma unroll
            for (uint32_t j = 0; j < kBatch; ++j) {
                if (!(valid >> j & 1u)) continue;
                const uint32_t b = w[j] >> (2u * (u[j] & 15u));
                if (!(b & 1u)) {
                    // alive: one degree less (hubs' decrements combined in the block); in a thin
                    // round the decrement that takes a degree to the bound makes it a candidate
                    if ((b & 2u) && agg_add(sm.agg, u[j])) {
                    } else if (thin) {
                        const uint32_t old = atomicSub(&st[u[j]], 1u);
                        if (old > Bn && old - 1u <= Bn) next_cand[atomicAdd(&ctl->cand, 1ull) - cand_base] = u[j];
                    } else {
                        atomicSub(&st[u[j]], 1u);
                    }
                    ++ndec;
                }
            }
        };
        scan_frontier<TB>(a.off, a.adj, a.F, short_lo, short_hi, a.C, chunk_lo, chunk_hi, a.chunk_len, visit, a.n,
                          a.FB, a.FL, vec_end);
        // flush the combined hub decrements (block_sum below synchronises first)
        __syncthreads();
        for (uint32_t i = tid; i < kAggSlots; i += TB) {
            uint32_t key = sm.agg.key[i];
            if (key != kAggEmpty) {
                const uint32_t c = sm.agg.cnt[i];
                if (thin) {
                    const uint32_t old = atomicSub(&st[key], c);
                    if (old > Bn && old - c <= Bn) next_cand[atomicAdd(&ctl->cand, 1ull) - cand_base] = key;
                } else {
                    atomicSub(&st[key], c);
                }
                sm.agg.key[i] = kAggEmpty;
                sm.agg.cnt[i] = 0;
            }
        }
        const uint64_t bdec = block_sum<uint64_t>(ndec, sm.red);
        if (tid == 0 && bdec) atomicAdd(&ctl->dec, (unsigned long long)bdec);
        if (!grid_barrier(&ctl->bar, &ctl->err, a.limit_ns)) return;
        stamp();
        // edges removed so far: (X + D) / 2 summed over the rounds
        const uint64_t removed = (ld_relaxed_u64(&ctl->xsum) + ld_relaxed_u64(&ctl->dec)) / 2;
        const uint64_t S1 = (uint64_t)a.n - failed_hi;
        const uint64_t E1 = a.m - removed;
        ++r;
        if (blockIdx.x == 0 && tid == 0) {
            if (r < a.hist_cap) {
                a.hist_S[r] = S1;
                a.hist_E[r] = E1;
            } else {
                atomicOr(&ctl->err, ERR_CAPACITY);
            }
        }
        if (S1 > 0 && (unsigned __int128)E1 * best_V > (unsigned __int128)best_E * S1) {
            best_round = r;
            best_E = E1;
            best_V = S1;
        }
        short_lo = short_hi;
        chunk_lo = chunk_hi;
        if (!lazy) {  // a lazy round leaves the alive list as it was (its failures are skipped later)
            surv_base += S1;
            alive_len = S1;
            alive = next;
            next = (next == a.listA) ? a.listB : a.listA;
        }
        {
            const uint64_t cand_hi = ld_relaxed_u64(&ctl->cand);
            if (thin) {
                uint32_t* t_ = cur_cand;
                cur_cand = next_cand;
                next_cand = t_;
                cand_n = cand_hi - cand_base;
                B = Bn;
            }
            have_cands = thin;
            cand_base = cand_hi;
        }
        S_prev = S;
        S = S1;
        E = E1;
        if (r >= a.hist_cap) break;
        if (a.max_rounds && r - a.r0 >= a.max_rounds) break;  // pause: the state stays in st
    }
    if (blockIdx.x == 0 && tid == 0) {
        ctl->stamps = nstamp;
        ctl->rounds = r;
        ctl->best_round = best_round;
        ctl->best_E = best_E;
        ctl->best_V = best_V;
        ctl->cur_S = S;
        ctl->cur_E = E;
    }
}

// peel_round[v] = round v failed; set[v] = peel_round > best_round.
__global__ void peel_finish_kernel(uint32_t n, const uint32_t* __restrict__ st, const PeelCtl* __restrict__ ctl,
                                   uint32_t* __restrict__ peel_round, uint8_t* __restrict__ set) {
    uint64_t br = ctl->best_round;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t pr = st[v] & ~kDead;
        if (peel_round) peel_round[v] = pr;
        if (set) set[v] = pr > br ? 1 : 0;
    }
}

template <int TB>
static cudaError_t launch_peel(PeelArgs& a, uint32_t blocks_per_sm, cudaStream_t s, uint32_t max_grid) {
    uint32_t grid = 1;
    cudaError_t e = coop_grid(peel_kernel<TB>, TB, 0, a.n, blocks_per_sm, &grid, max_grid);
    if (e != cudaSuccess) return e;
    void* params[] = {&a};
    LaunchScope ls("peel_rounds", s);
    return cudaLaunchCooperativeKernel((const void*)peel_kernel<TB>, dim3(grid), dim3(TB), params, 0, s);
}

// Run the peel; results land in the returned control block and, if given,
// in hist / peel_round / set (device pointers).
static dsg_status run_peel(const dsg_graph* g, uint32_t p, uint32_t q, uint64_t* hist_S_out, uint64_t* hist_E_out,
                           uint64_t hist_cap_out, uint32_t* peel_round_out, uint8_t* set_out, PeelCtl* ctl_host,
                           uint64_t* trace_dev = nullptr, uint64_t trace_cap = 0);

dsg_status peel_into(const dsg_graph* g, uint32_t p, uint32_t q, uint8_t* set_dev, uint64_t out4[4],
                     uint64_t* extra2) {
    PeelCtl c;
    dsg_status st;
    if (extra2 && g->n) {
        // the byte model's counters too: sum of |S_r| over the rounds (from the history) and the decrements
        const uint64_t cap = dsg_round_bound(g->n, p, q) + 1;
        std::vector<uint64_t> hs(cap);
        st = run_peel(g, p, q, hs.data(), nullptr, cap, nullptr, set_dev, &c);
        if (st != DSG_OK) return st;
        uint64_t sum = 0;
        for (uint64_t r = 0; r < c.rounds && r < cap; ++r) sum += hs[r];
        extra2[0] = sum;
        extra2[1] = c.dec;
    } else {
        st = run_peel(g, p, q, nullptr, nullptr, 0, nullptr, set_dev, &c);
    }
    if (st != DSG_OK) return st;
    out4[0] = g->n ? c.best_E : 0;
    out4[1] = g->n ? c.best_V : 0;
    out4[2] = c.rounds;
    out4[3] = c.best_round;
    return DSG_OK;
}

static dsg_status run_peel(const dsg_graph* g, uint32_t p, uint32_t q, uint64_t* hist_S_out, uint64_t* hist_E_out,
                           uint64_t hist_cap_out, uint32_t* peel_round_out, uint8_t* set_out, PeelCtl* ctl_host,
                           uint64_t* trace_dev, uint64_t trace_cap) {
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    Tuning tu = tuning_for(g, 0);
    if (g->force_block) tu.block = g->force_block;
    memset(ctl_host, 0, sizeof(PeelCtl));
    if (n == 0) {
        static const uint64_t zero = 0;
        if (hist_S_out && hist_cap_out) DSG_TRY_CUDA(copy_any(hist_S_out, &zero, sizeof(uint64_t), s));
        if (hist_E_out && hist_cap_out) DSG_TRY_CUDA(copy_any(hist_E_out, &zero, sizeof(uint64_t), s));
        DSG_TRY_CUDA(cudaStreamSynchronize(s));
        return DSG_OK;
    }
    uint64_t cap = dsg_round_bound(n, p, q) + 1;
    const uint64_t chunk_cap = (uint64_t)n + (2 * g->m) / tu.chunk_len + 1;
    Scratch sc(s);
    PeelArgs a;
    a.n = n;
    a.m = g->m;
    a.p = p;
    a.q = q;
    a.off = g->off;
    a.adj = g->adj;
    a.hist_cap = cap;
    a.limit_ns = wait_limit_ns();
    a.short_max = tu.short_max;
    a.chunk_len = tu.chunk_len;
    a.hot_deg = tu.hot_deg;
    a.vec_loads = current_tuning().peel_vec;
    a.trace = trace_dev;
    a.trace_cap = trace_cap;
    a.r0 = a.S0 = a.E0 = a.best_round0 = a.best_E0 = a.best_V0 = a.max_rounds = 0;
    DSG_TRY_CUDA(sc.get(&a.st, n));
    DSG_TRY_CUDA(sc.get(&a.listA, n));
    DSG_TRY_CUDA(sc.get(&a.listB, n));
    DSG_TRY_CUDA(sc.get(&a.F, n));
    DSG_TRY_CUDA(sc.get(&a.FB, n));
    DSG_TRY_CUDA(sc.get(&a.FL, n));
    DSG_TRY_CUDA(sc.get(&a.C, chunk_cap));
    DSG_TRY_CUDA(sc.get(&a.map, ((size_t)n + 15) / 16));
    a.candA = a.candB = nullptr;
    if (current_tuning().peel_lazy) {
        DSG_TRY_CUDA(sc.get(&a.candA, n));
        DSG_TRY_CUDA(sc.get(&a.candB, n));
    }
    DSG_TRY_CUDA(sc.get(&a.hist_S, cap));
    DSG_TRY_CUDA(sc.get(&a.hist_E, cap));
    DSG_TRY_CUDA(sc.get(&a.ctl, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(a.ctl, 0, sizeof(PeelCtl), s));
    cudaError_t e;
    switch (tu.block) {
        case 256: e = launch_peel<256>(a, tu.blocks_per_sm, s, g->max_blocks); break;
        case 1024: e = launch_peel<1024>(a, tu.blocks_per_sm, s, g->max_blocks); break;
        default: e = launch_peel<512>(a, tu.blocks_per_sm, s, g->max_blocks); break;
    }
    DSG_TRY_CUDA(e);
    uint32_t* pr_dev = nullptr;
    uint8_t* set_dev = nullptr;
    bool pr_direct = peel_round_out && is_device_ptr(peel_round_out);
    bool set_direct = set_out && is_device_ptr(set_out);
    if (peel_round_out) {
        if (pr_direct) pr_dev = peel_round_out;
        else DSG_TRY_CUDA(sc.get(&pr_dev, n));
    }
    if (set_out) {
        if (set_direct) set_dev = set_out;
        else DSG_TRY_CUDA(sc.get(&set_dev, n));
    }
    if (pr_dev || set_dev) {
        uint64_t want = ((uint64_t)n + 255) / 256, cap_b = (uint64_t)dev_info().sms * 8;
        uint32_t blocks = (uint32_t)(want < cap_b ? want : cap_b);
        {
            LaunchScope ls("peel_finish", s);
            peel_finish_kernel<<<blocks, 256, 0, s>>>(n, a.st, a.ctl, pr_dev, set_dev);
        }
        DSG_TRY_CUDA(cudaGetLastError());
    }
    DSG_TRY_CUDA(cudaMemcpyAsync(ctl_host, a.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    dsg_status st = status_from_err(ctl_host->err, "bahmani peel");
    if (st != DSG_OK) return st;
    uint64_t R = ctl_host->rounds;
    if (hist_S_out || hist_E_out) {
        uint64_t k = R + 1 < hist_cap_out ? R + 1 : hist_cap_out;
        if (hist_S_out) DSG_TRY_CUDA(copy_any(hist_S_out, a.hist_S, k * sizeof(uint64_t), s));
        if (hist_E_out) DSG_TRY_CUDA(copy_any(hist_E_out, a.hist_E, k * sizeof(uint64_t), s));
    }
    if (peel_round_out && !pr_direct) DSG_TRY_CUDA(copy_any(peel_round_out, pr_dev, (size_t)n * 4, s));
    if (set_out && !set_direct) DSG_TRY_CUDA(copy_any(set_out, set_dev, (size_t)n, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    return DSG_OK;
}

}  // namespace dsg

using namespace dsg;

extern "C" {

dsg_status dsg_bahmani(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, uint8_t* out_set, uint64_t* out_E,
                       uint64_t* out_V) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    DSG_CHECK_ARG(eps_den != 0, "eps_den must be positive");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    PeelCtl c;
    dsg_status st = run_peel(g, eps_num, eps_den, nullptr, nullptr, 0, nullptr, out_set, &c);
    if (st != DSG_OK) return st;
    if (out_E) *out_E = g->n ? c.best_E : 0;
    if (out_V) *out_V = g->n ? c.best_V : 0;
    return DSG_OK;
}

// Peels at several eps and the core numbers of one graph.  The two kinds of
// solve are independent, so they may run side by side: the peels on one
// internal stream and the core numbers on another (from a second host thread,
// since each solve waits for its stream), each kernel with 1024-thread blocks
// on at most half the SMs -- one block per SM, so the two grids fit the GPU
// together.  Both streams start after the graph's stream, and the graph's
// stream waits for both before the call returns.
dsg_status dsg_solve(const dsg_graph* g, uint32_t count, const uint32_t* eps_num, const uint32_t* eps_den,
                     uint8_t* const* out_sets, uint64_t* out_E, uint64_t* out_V, uint32_t* out_core) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    DSG_CHECK_ARG(count == 0 || (eps_num && eps_den), "eps arrays are NULL");
    for (uint32_t i = 0; i < count; ++i) DSG_CHECK_ARG(eps_den[i] != 0, "eps_den must be positive");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    auto peels = [&](const dsg_graph* h) -> dsg_status {
        for (uint32_t i = 0; i < count; ++i) {
            PeelCtl c;
            dsg_status st =
                run_peel(h, eps_num[i], eps_den[i], nullptr, nullptr, 0, nullptr, out_sets ? out_sets[i] : nullptr, &c);
            if (st != DSG_OK) return st;
            if (out_E) out_E[i] = g->n ? c.best_E : 0;
            if (out_V) out_V[i] = g->n ? c.best_V : 0;
        }
        return DSG_OK;
    };
    // side by side only pays when the peels are a fair share of the work:
    // each kind then runs on half the GPU; when the autotuned times of this
    // graph's size class say the core numbers dominate, run one after the
    // other with the whole GPU each
    double peel_ms = 0, core_ms = 0;
    const bool tuned = tuned_times(g, &peel_ms, &core_ms);
    const bool mostly_core = tuned && count * peel_ms < 0.25 * core_ms;
    if (count == 0 || !out_core || g->n == 0 || mostly_core) {
        dsg_status st = peels(g);
        if (st != DSG_OK || !out_core) return st;
        return run_kcore(g, out_core, nullptr, 0);
    }
    const uint32_t sms = (uint32_t)dev_info().sms;
    // two streams and three events per calling thread and device, made once
    struct SideBySide {
        int device = -1;
        cudaStream_t sa = nullptr, sb = nullptr;
        cudaEvent_t ev0 = nullptr, eva = nullptr, evb = nullptr;
    };
    static thread_local SideBySide cache[16];
    SideBySide& sbs = cache[g->device & 15];
    if (sbs.device != g->device) {
        DSG_TRY_CUDA(cudaStreamCreateWithFlags(&sbs.sa, cudaStreamNonBlocking));
        DSG_TRY_CUDA(cudaStreamCreateWithFlags(&sbs.sb, cudaStreamNonBlocking));
        DSG_TRY_CUDA(cudaEventCreateWithFlags(&sbs.ev0, cudaEventDisableTiming));
        DSG_TRY_CUDA(cudaEventCreateWithFlags(&sbs.eva, cudaEventDisableTiming));
        DSG_TRY_CUDA(cudaEventCreateWithFlags(&sbs.evb, cudaEventDisableTiming));
        sbs.device = g->device;
    }
    cudaStream_t sa = sbs.sa, sb = sbs.sb;
    cudaEvent_t ev0 = sbs.ev0, eva = sbs.eva, evb = sbs.evb;
    DSG_TRY_CUDA(cudaEventRecord(ev0, g->stream));
    DSG_TRY_CUDA(cudaStreamWaitEvent(sa, ev0, 0));
    DSG_TRY_CUDA(cudaStreamWaitEvent(sb, ev0, 0));
    dsg_graph va = *g, vb = *g;
    va.owns = vb.owns = false;
    va.stream = sa;
    vb.stream = sb;
    va.force_block = vb.force_block = 1024;
    // the peels' share of the SMs: DSG_SOLVE_PEEL_PERMILLE if set, else from
    // the autotuned times (each side's share of the summed time, within
    // [1/4, 3/4]), else half
    double peel_frac = 0.5;
    if (tuned && count * peel_ms + core_ms > 0)
        peel_frac = std::min(0.75, std::max(0.25, count * peel_ms / (count * peel_ms + core_ms)));
    if (const char* e = getenv("DSG_SOLVE_PEEL_PERMILLE")) {
        const long pm = strtol(e, nullptr, 10);
        if (pm > 0 && pm < 1000) peel_frac = pm / 1000.0;
    }
    va.max_blocks = std::max<uint32_t>(1, (uint32_t)(sms * peel_frac + 0.5));
    if (va.max_blocks >= sms) va.max_blocks = sms > 1 ? sms - 1 : 1;
    vb.max_blocks = sms - va.max_blocks > 0 ? sms - va.max_blocks : 1;
    dsg_status st_core = DSG_OK;
    std::string err_core;
    std::thread th([&] {
        cudaSetDevice(g->device);
        st_core = run_kcore(&vb, out_core, nullptr, 0);
        if (st_core != DSG_OK) err_core = dsg_last_error();
    });
    dsg_status st = peels(&va);
    th.join();
    cudaEventRecord(eva, sa);
    cudaEventRecord(evb, sb);
    cudaStreamWaitEvent(g->stream, eva, 0);
    cudaStreamWaitEvent(g->stream, evb, 0);
    if (st != DSG_OK) return st;
    if (st_core != DSG_OK) {
        set_error("%s", err_core.c_str());
        return st_core;
    }
    return DSG_OK;
}

dsg_status dsg_bahmani_trace(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, dsg_trace* t) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    DSG_CHECK_ARG(t, "trace is NULL");
    DSG_CHECK_ARG(eps_den != 0, "eps_den must be positive");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    PeelCtl c;
    dsg_status st = run_peel(g, eps_num, eps_den, t->hist_S, t->hist_E, t->hist_cap, t->peel_round, t->out_set, &c);
    if (st != DSG_OK) return st;
    t->rounds = c.rounds;
    t->best_round = c.best_round;
    t->best_E = g->n ? c.best_E : 0;
    t->best_V = g->n ? c.best_V : 0;
    t->edges_scanned = 2 * g->m;
    t->decrements = g->n ? c.dec : 0;
    t->tested = g->n ? c.tested : 0;
    t->lazy_rounds = g->n ? c.lazy_rounds : 0;
    if (t->hist_cap < c.rounds + 1 && (t->hist_S || t->hist_E)) {
        set_error("bahmani_trace: history needs %llu slots, got %llu", (unsigned long long)(c.rounds + 1),
                  (unsigned long long)t->hist_cap);
        return DSG_EOVERFLOW;
    }
    return DSG_OK;
}

// Phase timestamps of one peel (debug/analysis): ts[i] = %globaltimer after
// the i-th grid barrier (ts[0] = kernel start).  *count = stamps taken.
dsg_status dsg_debug_peel_trace(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, uint64_t* ts, uint64_t cap,
                                uint64_t* count) {
    clear_error();
    DSG_CHECK_ARG(g && ts && cap, "graph/ts/cap");
    DSG_CHECK_ARG(eps_den != 0, "eps_den must be positive");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    Scratch sc(g->stream);
    uint64_t* dts;
    DSG_TRY_CUDA(sc.get(&dts, cap));
    PeelCtl c;
    dsg_status st = run_peel(g, eps_num, eps_den, nullptr, nullptr, 0, nullptr, nullptr, &c, dts, cap);
    if (st != DSG_OK) return st;
    uint64_t k = c.stamps < cap ? c.stamps : cap;
    DSG_TRY_CUDA(copy_any(ts, dts, k * 8, g->stream));
    DSG_TRY_CUDA(cudaStreamSynchronize(g->stream));
    if (count) *count = c.stamps;
    return DSG_OK;
}

}  // extern "C"

// ===================================================== no-allocation variant
//
// Some callers cannot allocate device memory at the moment they want a peel:
// code running under an allocator they do not own (a host application whose
// memory pool is reserved up front, a framework that forbids allocation on
// its hot path), or code that must not risk cudaMalloc's implicit device
// synchronisation.  dsg_bahmani_noalloc serves them: it runs the same
// persistent peel kernel as dsg_bahmani, but every scratch array lives in one
// fixed buffer that belongs to this library file -- a static device array of
// kNoAllocScratchBytes, reserved on each GPU that loads this code and held
// until the process exits.  The caller passes the graph and the outputs.
#include <mutex>

namespace dsg {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch.  Host code may not use the symbol
// itself as an address (on the host it names a shadow variable), so the
// address is looked up with cudaGetSymbolAddress, with the device current,
// the first time a call runs in a CUDA context.  The cache is keyed on the
// context's id, not on the device ordinal: after a context is destroyed and
// made again (cudaDeviceReset, a released primary context) the module is
// loaded again and the array may sit elsewhere, so the new context looks it
// up afresh.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

struct NoAllocSlot {
    unsigned long long ctx_id = 0;  // 0: empty
    unsigned char* addr = nullptr;
};
static std::mutex g_noalloc_mu;
static NoAllocSlot g_noalloc_slots[64];

// Id of the current context (0 when the driver cannot tell: the address is
// then looked up on every call).
static unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

static dsg_status noalloc_scratch(unsigned char** out) {
    int dev = 0;
    DSG_TRY_CUDA(cudaGetDevice(&dev));
    DSG_CHECK_ARG(dev >= 0 && dev < 64, "device ordinal above 63");
    const unsigned long long id = current_ctx_id();
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocSlot& slot = g_noalloc_slots[dev];
    if (id == 0 || slot.ctx_id != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("bahmani_noalloc: cudaGetSymbolAddress of the static scratch failed: %s",
                      cudaGetErrorString(e));
            return DSG_ECUDA;
        }
        slot.addr = static_cast<unsigned char*>(p);
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return DSG_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <int TB>
static cudaError_t launch_peel_noalloc(PeelArgs& a, uint32_t blocks_per_sm, cudaStream_t s) {
    uint32_t grid = 1;
    cudaError_t e = coop_grid(peel_kernel<TB>, TB, 0, a.n, blocks_per_sm, &grid);
    if (e != cudaSuccess) return e;
    void* params[] = {&a};
    LaunchScope ls("peel_rounds", s);
    return cudaLaunchCooperativeKernel((const void*)peel_kernel<TB>, dim3(grid), dim3(TB), params, 0, s);
}

}  // namespace dsg

extern "C" dsg_status dsg_bahmani_noalloc(uint32_t n, const uint64_t* off, const uint32_t* adj, uint32_t eps_num,
                                          uint32_t eps_den, uint8_t* out_set, uint64_t* out_E, uint64_t* out_V,
                                          void* stream) {
    clear_error();
    DSG_CHECK_ARG(eps_den != 0, "eps_den must be positive");
    DSG_CHECK_ARG(n < 0x80000000u, "n must be below 2^31");
    DSG_CHECK_ARG(off && is_device_ptr(off), "off must be a device pointer");
    DSG_CHECK_ARG(!out_set || is_device_ptr(out_set), "out_set must be a device pointer (or NULL)");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t total = 0;
    DSG_TRY_CUDA(cudaMemcpyAsync(&total, off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    DSG_CHECK_ARG(total % 2 == 0, "off[n] must be even for a symmetric CSR");
    DSG_CHECK_ARG(total == 0 || (adj && is_device_ptr(adj)), "adj must be a device pointer");
    if (n == 0) {
        if (out_E) *out_E = 0;
        if (out_V) *out_V = 0;
        return DSG_OK;
    }
    const Tuning tu = current_tuning();
    const uint64_t m = total / 2;
    const uint64_t cap = dsg_round_bound(n, eps_num, eps_den) + 1;
    const uint64_t chunk_cap = (uint64_t)n + (2 * m) / tu.chunk_len + 1;
    const size_t b_list = align256((size_t)n * 4);
    const size_t b_chunk = align256((size_t)chunk_cap * 8);
    const size_t b_hist = align256((size_t)cap * 8);
    const size_t b_ctl = align256(sizeof(PeelCtl));
    const size_t b_map = align256(((size_t)n + 15) / 16 * 4);
    const size_t need = 4 * b_list + b_chunk + b_map + 2 * b_hist + b_ctl;
    if (need > kNoAllocScratchBytes) {
        set_error("bahmani_noalloc: this graph needs %zu bytes of scratch, above the fixed %zu-byte buffer "
                  "(use dsg_bahmani)", need, (size_t)kNoAllocScratchBytes);
        return DSG_EINVAL;
    }
    unsigned char* base = nullptr;
    dsg_status st = noalloc_scratch(&base);
    if (st != DSG_OK) return st;
    PeelArgs a;
    a.n = n;
    a.m = m;
    a.p = eps_num;
    a.q = eps_den;
    a.off = off;
    a.adj = adj;
    size_t o = 0;
    a.st = reinterpret_cast<uint32_t*>(base + o); o += b_list;
    a.listA = reinterpret_cast<uint32_t*>(base + o); o += b_list;
    a.listB = reinterpret_cast<uint32_t*>(base + o); o += b_list;
    a.F = reinterpret_cast<uint32_t*>(base + o); o += b_list;
    a.FB = nullptr;  // short rows' bounds are read from off
    a.FL = nullptr;
    a.C = reinterpret_cast<uint64_t*>(base + o); o += b_chunk;
    a.map = reinterpret_cast<uint32_t*>(base + o); o += b_map;
    a.candA = nullptr;  // no lazy rounds: every round tests the whole alive list
    a.candB = nullptr;
    a.hist_S = reinterpret_cast<uint64_t*>(base + o); o += b_hist;
    a.hist_E = reinterpret_cast<uint64_t*>(base + o); o += b_hist;
    a.ctl = reinterpret_cast<PeelCtl*>(base + o);
    a.hist_cap = cap;
    a.limit_ns = wait_limit_ns();
    a.short_max = tu.short_max;
    a.chunk_len = tu.chunk_len;
    a.hot_deg = tu.hot_deg;
    a.vec_loads = current_tuning().peel_vec;
    a.trace = nullptr;
    a.trace_cap = 0;
    a.r0 = a.S0 = a.E0 = a.best_round0 = a.best_E0 = a.best_V0 = a.max_rounds = 0;
    // The buffer keeps whatever the previous call left; only the control
    // block must start at zero (every other array is written before it is read).
    DSG_TRY_CUDA(cudaMemsetAsync(a.ctl, 0, sizeof(PeelCtl), s));
    cudaError_t e;
    switch (tu.block) {
        case 256: e = launch_peel_noalloc<256>(a, tu.blocks_per_sm, s); break;
        case 1024: e = launch_peel_noalloc<1024>(a, tu.blocks_per_sm, s); break;
        default: e = launch_peel_noalloc<512>(a, tu.blocks_per_sm, s); break;
    }
    DSG_TRY_CUDA(e);
    if (out_set) {
        uint64_t want = ((uint64_t)n + 255) / 256, cap_b = (uint64_t)dev_info().sms * 8;
        uint32_t blocks = (uint32_t)(want < cap_b ? want : cap_b);
        {
            LaunchScope ls("peel_finish", s);
            peel_finish_kernel<<<blocks, 256, 0, s>>>(n, a.st, a.ctl, nullptr, out_set);
        }
        DSG_TRY_CUDA(cudaGetLastError());
    }
    PeelCtl c;
    DSG_TRY_CUDA(cudaMemcpyAsync(&c, a.ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    st = status_from_err(c.err, "bahmani_noalloc");
    if (st != DSG_OK) return st;
    if (out_E) *out_E = c.best_E;
    if (out_V) *out_V = c.best_V;
    return DSG_OK;
}

// ========================================================= snapshot / resume
//
// Algorithm 1's state between two rounds is small: each vertex's state word
// (its degree inside S_r, or the round it failed in), the round r, |S_r|,
// |E(S_r)|, the best round so far with its (E, V), and the history of
// (|S_t|, |E(S_t)|).  A paused peel keeps that state on the device between
// launches; a snapshot writes it to host memory, and resuming rebuilds it on
// a handle of the same graph, so a long peel (eps = 0 on a graph that peels
// slowly) can be checkpointed, moved or continued later with the same result.
struct dsg_peel_state {
    const dsg_graph* g = nullptr;
    uint32_t p = 0, q = 1;
    uint64_t r = 0, S = 0, E = 0, best_round = 0, best_E = 0, best_V = 0, cap = 0, chunk_cap = 0;
    bool done = false;
    dsg::Tuning tu;
    uint32_t *st = nullptr, *listA = nullptr, *listB = nullptr, *F = nullptr, *FL = nullptr, *map = nullptr,
             *candA = nullptr, *candB = nullptr;
    uint64_t *FB = nullptr, *C = nullptr, *hist_S = nullptr, *hist_E = nullptr;
    dsg::PeelCtl* ctl = nullptr;
};

namespace dsg {

static constexpr uint64_t kSnapMagic = 0x314c454550475344ull;  // "DSGPEEL1"
static constexpr uint64_t kSnapHeaderWords = 16;

static void peel_state_release(dsg_peel_state* ps) {
    if (!ps) return;
    cudaStream_t s = ps->g ? ps->g->stream : nullptr;
    void* bufs[] = {ps->st,  ps->listA,  ps->listB,  ps->F,      ps->FB,     ps->FL, ps->C,
                    ps->map, ps->candA,  ps->candB,  ps->hist_S, ps->hist_E, ps->ctl};
    for (void* b : bufs)
        if (b) dev_free(b, s);
    if (s) cudaStreamSynchronize(s);
    delete ps;
}

// A new state on g (device arrays allocated, scalars at round 0).
static dsg_status peel_state_new(const dsg_graph* g, uint32_t p, uint32_t q, dsg_peel_state** out) {
    dsg_peel_state* ps = new dsg_peel_state();
    ps->g = g;
    ps->p = p;
    ps->q = q;
    ps->tu = tuning_for(g, 0);
    if (g->force_block) ps->tu.block = g->force_block;
    const uint32_t n = g->n;
    ps->cap = n ? dsg_round_bound(n, p, q) + 1 : 1;
    ps->chunk_cap = (uint64_t)n + (2 * g->m) / ps->tu.chunk_len + 1;
    ps->S = n;
    ps->E = g->m;
    ps->best_E = g->m;
    ps->best_V = n;
    ps->done = n == 0;
    cudaStream_t s = g->stream;
    const size_t nb = ((size_t)(n ? n : 1) * 4 + 255) & ~size_t(255);
    cudaError_t e = dev_alloc((void**)&ps->st, nb, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->listA, nb, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->listB, nb, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->F, nb, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->FB, 2 * nb, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->FL, nb, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->candA, nb, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->candB, nb, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->C, ps->chunk_cap * 8, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->map, (((size_t)(n ? n : 1) + 15) / 16 * 4 + 255) & ~size_t(255), s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->hist_S, ps->cap * 8, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->hist_E, ps->cap * 8, s);
    if (e == cudaSuccess) e = dev_alloc((void**)&ps->ctl, sizeof(PeelCtl), s);
    if (e != cudaSuccess) {
        set_error("peel state: %s", cudaGetErrorString(e));
        peel_state_release(ps);
        return e == cudaErrorMemoryAllocation ? DSG_ENOMEM : DSG_ECUDA;
    }
    *out = ps;
    return DSG_OK;
}

// Run up to max_rounds rounds (0: to the end) from where ps stands.
static dsg_status peel_state_run(dsg_peel_state* ps, uint64_t max_rounds) {
    if (ps->done) return DSG_OK;
    const dsg_graph* g = ps->g;
    cudaStream_t s = g->stream;
    PeelArgs a;
    a.n = g->n;
    a.m = g->m;
    a.p = ps->p;
    a.q = ps->q;
    a.off = g->off;
    a.adj = g->adj;
    a.st = ps->st;
    a.listA = ps->listA;
    a.listB = ps->listB;
    a.F = ps->F;
    a.FB = ps->FB;
    a.FL = ps->FL;
    a.C = ps->C;
    a.map = ps->map;
    const bool lazy_on = current_tuning().peel_lazy != 0;
    a.candA = lazy_on ? ps->candA : nullptr;
    a.candB = lazy_on ? ps->candB : nullptr;
    a.hist_S = ps->hist_S;
    a.hist_E = ps->hist_E;
    a.hist_cap = ps->cap;
    a.ctl = ps->ctl;
    a.limit_ns = wait_limit_ns();
    a.short_max = ps->tu.short_max;
    a.chunk_len = ps->tu.chunk_len;
    a.hot_deg = ps->tu.hot_deg;
    a.vec_loads = current_tuning().peel_vec;
    a.trace = nullptr;
    a.trace_cap = 0;
    a.r0 = ps->r;
    a.S0 = ps->S;
    a.E0 = ps->E;
    a.best_round0 = ps->best_round;
    a.best_E0 = ps->best_E;
    a.best_V0 = ps->best_V;
    a.max_rounds = max_rounds;
    PeelCtl init;
    memset(&init, 0, sizeof(init));
    init.failed = (uint64_t)g->n - ps->S;  // the counters the kernel derives S and E from
    init.xsum = 2 * (g->m - ps->E);
    DSG_TRY_CUDA(cudaMemcpyAsync(ps->ctl, &init, sizeof(PeelCtl), cudaMemcpyHostToDevice, s));
    cudaError_t e;
    switch (ps->tu.block) {
        case 256: e = launch_peel<256>(a, ps->tu.blocks_per_sm, s, g->max_blocks); break;
        case 1024: e = launch_peel<1024>(a, ps->tu.blocks_per_sm, s, g->max_blocks); break;
        default: e = launch_peel<512>(a, ps->tu.blocks_per_sm, s, g->max_blocks); break;
    }
    DSG_TRY_CUDA(e);
    PeelCtl c;
    DSG_TRY_CUDA(cudaMemcpyAsync(&c, ps->ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    dsg_status st = status_from_err(c.err, "peel");
    if (st != DSG_OK) return st;
    ps->r = c.rounds;
    ps->S = c.cur_S;
    ps->E = c.cur_E;
    ps->best_round = c.best_round;
    ps->best_E = c.best_E;
    ps->best_V = c.best_V;
    ps->done = ps->S == 0;
    return DSG_OK;
}

static uint64_t snapshot_bytes(const dsg_peel_state* ps) {
    return (kSnapHeaderWords + 2 * (ps->r + 1)) * 8 + (uint64_t)ps->g->n * 4;
}

}  // namespace dsg

extern "C" {

dsg_status dsg_peel_begin(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, dsg_peel_state** out) {
    clear_error();
    DSG_CHECK_ARG(g && out, "graph / out is NULL");
    DSG_CHECK_ARG(eps_den != 0, "eps_den must be positive");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    dsg_peel_state* ps = nullptr;
    dsg_status st = peel_state_new(g, eps_num, eps_den, &ps);
    if (st != DSG_OK) return st;
    const uint64_t h[2] = {g->n, g->m};
    cudaError_t e = cudaMemcpyAsync(ps->hist_S, &h[0], 8, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ps->hist_E, &h[1], 8, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        set_error("peel_begin: %s", cudaGetErrorString(e));
        peel_state_release(ps);
        return DSG_ECUDA;
    }
    *out = ps;
    return DSG_OK;
}

dsg_status dsg_peel_advance(dsg_peel_state* ps, uint32_t max_rounds, uint64_t* rounds, uint32_t* done) {
    clear_error();
    DSG_CHECK_ARG(ps, "state is NULL");
    DSG_TRY_CUDA(cudaSetDevice(ps->g->device));
    dsg_status st = peel_state_run(ps, max_rounds);
    if (st != DSG_OK) return st;
    if (rounds) *rounds = ps->r;
    if (done) *done = ps->done ? 1u : 0u;
    return DSG_OK;
}

dsg_status dsg_peel_snapshot_size(const dsg_peel_state* ps, uint64_t* bytes) {
    clear_error();
    DSG_CHECK_ARG(ps && bytes, "state / bytes is NULL");
    *bytes = snapshot_bytes(ps);
    return DSG_OK;
}

dsg_status dsg_peel_snapshot(const dsg_peel_state* ps, void* buf, uint64_t bytes) {
    clear_error();
    DSG_CHECK_ARG(ps && buf, "state / buffer is NULL");
    DSG_CHECK_ARG(bytes >= snapshot_bytes(ps), "buffer smaller than dsg_peel_snapshot_size");
    DSG_TRY_CUDA(cudaSetDevice(ps->g->device));
    uint64_t* w = static_cast<uint64_t*>(buf);
    const uint64_t hl = ps->r + 1;
    const uint64_t h[kSnapHeaderWords] = {kSnapMagic, 1, ps->g->n, ps->g->m, ps->p, ps->q, ps->r, ps->S, ps->E,
                                          ps->best_round, ps->best_E, ps->best_V, hl, 0, 0, 0};
    memcpy(w, h, sizeof(h));
    cudaStream_t s = ps->g->stream;
    DSG_TRY_CUDA(copy_any(w + kSnapHeaderWords, ps->hist_S, hl * 8, s));
    DSG_TRY_CUDA(copy_any(w + kSnapHeaderWords + hl, ps->hist_E, hl * 8, s));
    uint32_t* words = reinterpret_cast<uint32_t*>(w + kSnapHeaderWords + 2 * hl);
    if (ps->r > 0) {
        if (ps->g->n) DSG_TRY_CUDA(copy_any(words, ps->st, (size_t)ps->g->n * 4, s));
    } else {
        memset(words, 0, (size_t)ps->g->n * 4);  // before the first round the state words are not used
    }
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    return DSG_OK;
}

dsg_status dsg_peel_resume(const dsg_graph* g, const void* buf, uint64_t bytes, dsg_peel_state** out) {
    clear_error();
    DSG_CHECK_ARG(g && buf && out, "graph / buffer / out is NULL");
    DSG_CHECK_ARG(bytes >= kSnapHeaderWords * 8, "buffer shorter than a snapshot header");
    const uint64_t* w = static_cast<const uint64_t*>(buf);
    DSG_CHECK_ARG(w[0] == kSnapMagic && w[1] == 1, "not a peel snapshot (magic / version)");
    DSG_CHECK_ARG(w[2] == g->n && w[3] == g->m, "the snapshot was taken on a graph of another size");
    DSG_CHECK_ARG(w[5] != 0 && w[4] <= 0xffffffffull && w[5] <= 0xffffffffull, "bad eps in the snapshot");
    const uint64_t r = w[6], hl = w[12];
    DSG_CHECK_ARG(hl == r + 1, "bad history length in the snapshot");
    DSG_CHECK_ARG(bytes >= (kSnapHeaderWords + 2 * hl) * 8 + (uint64_t)g->n * 4, "snapshot truncated");
    DSG_CHECK_ARG(w[7] <= g->n && w[8] <= g->m && w[9] <= r && w[11] <= g->n, "inconsistent snapshot scalars");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    dsg_peel_state* ps = nullptr;
    dsg_status st = peel_state_new(g, (uint32_t)w[4], (uint32_t)w[5], &ps);
    if (st != DSG_OK) return st;
    if (hl > ps->cap) {
        set_error("peel_resume: the snapshot has %llu rounds, more than the bound %llu for its eps",
                  (unsigned long long)r, (unsigned long long)(ps->cap - 1));
        peel_state_release(ps);
        return DSG_EINVAL;
    }
    ps->r = r;
    ps->S = w[7];
    ps->E = w[8];
    ps->best_round = w[9];
    ps->best_E = w[10];
    ps->best_V = w[11];
    ps->done = ps->S == 0;
    cudaStream_t s = g->stream;
    cudaError_t e = copy_any(ps->hist_S, w + kSnapHeaderWords, hl * 8, s);
    if (e == cudaSuccess) e = copy_any(ps->hist_E, w + kSnapHeaderWords + hl, hl * 8, s);
    if (e == cudaSuccess && r > 0 && g->n)
        e = copy_any(ps->st, reinterpret_cast<const uint32_t*>(w + kSnapHeaderWords + 2 * hl), (size_t)g->n * 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error("peel_resume: %s", cudaGetErrorString(e));
        peel_state_release(ps);
        return DSG_ECUDA;
    }
    *out = ps;
    return DSG_OK;
}

dsg_status dsg_peel_finish(dsg_peel_state* ps, uint8_t* out_set, uint64_t* out_E, uint64_t* out_V,
                           uint64_t* out_rounds, uint64_t* hist_S, uint64_t* hist_E, uint64_t hist_cap) {
    clear_error();
    DSG_CHECK_ARG(ps, "state is NULL");
    DSG_TRY_CUDA(cudaSetDevice(ps->g->device));
    dsg_status st = peel_state_run(ps, 0);
    if (st != DSG_OK) return st;
    const dsg_graph* g = ps->g;
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    if (out_set && n) {
        Scratch sc(s);
        uint8_t* set_dev = out_set;
        const bool direct = is_device_ptr(out_set);
        if (!direct) DSG_TRY_CUDA(sc.get(&set_dev, n));
        PeelCtl c;
        memset(&c, 0, sizeof(c));
        c.best_round = ps->best_round;
        DSG_TRY_CUDA(cudaMemcpyAsync(ps->ctl, &c, sizeof(PeelCtl), cudaMemcpyHostToDevice, s));
        uint64_t want = ((uint64_t)n + 255) / 256, cap_b = (uint64_t)dev_info().sms * 8;
        {
            LaunchScope ls("peel_finish", s);
            peel_finish_kernel<<<(uint32_t)(want < cap_b ? want : cap_b), 256, 0, s>>>(n, ps->st, ps->ctl, nullptr,
                                                                                       set_dev);
        }
        DSG_TRY_CUDA(cudaGetLastError());
        if (!direct) DSG_TRY_CUDA(copy_any(out_set, set_dev, n, s));
        DSG_TRY_CUDA(cudaStreamSynchronize(s));
    }
    const uint64_t R = ps->r;
    if (hist_S || hist_E) {
        const uint64_t k = R + 1 < hist_cap ? R + 1 : hist_cap;
        if (hist_S && k) DSG_TRY_CUDA(copy_any(hist_S, ps->hist_S, k * 8, s));
        if (hist_E && k) DSG_TRY_CUDA(copy_any(hist_E, ps->hist_E, k * 8, s));
        DSG_TRY_CUDA(cudaStreamSynchronize(s));
    }
    if (out_E) *out_E = n ? ps->best_E : 0;
    if (out_V) *out_V = n ? ps->best_V : 0;
    if (out_rounds) *out_rounds = R;
    if ((hist_S || hist_E) && hist_cap < R + 1) {
        set_error("peel_finish: history needs %llu slots, got %llu", (unsigned long long)(R + 1),
                  (unsigned long long)hist_cap);
        return DSG_EOVERFLOW;
    }
    return DSG_OK;
}

void dsg_peel_free(dsg_peel_state* ps) {
    if (ps && ps->g) cudaSetDevice(ps->g->device);
    peel_state_release(ps);
}

}  // extern "C"
