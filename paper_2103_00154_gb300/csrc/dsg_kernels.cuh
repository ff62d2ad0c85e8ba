// Shared pieces of the peel and core kernels: the frontier representation
// (short rows listed by vertex, long rows cut into fixed-size chunk items),
// the row scanner that walks a frontier's adjacency, and entry points shared
// between translation units.
#pragma once

#include "dsg_common.cuh"

namespace dsg {

// Adjacency entries are read once per solve: load them with the streaming
// (evict-first) policy so they do not push the per-vertex state (degrees,
// marks), which every entry looks up at random, out of L2.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) { return __ldcs(p); }

// Tuning knobs of the round kernels (see tune.cu for the defaults and the
// autotuner that picks them).
struct Tuning {
    uint32_t block = 512;       // threads per block of the persistent kernels
    uint32_t blocks_per_sm = 0; // 0: as many as fit
    uint32_t short_max = 32;    // rows up to this length go through the tile path
    uint32_t chunk_len = 256;   // long rows are cut into items of this many entries
    uint32_t hot_deg = 0;       // decrements of vertices at or above this degree are combined in shared memory
                                // (0: four times the number of blocks, i.e. hubs expected to be hit
                                // several times by every block)
    uint32_t local_max = 1024;  // k-core: rows up to this length reached while draining stay in the block
    uint32_t local_work = 16384; // k-core: ... while that block's local share of the sub-round stays within this
    uint32_t inline_max = 256;   // k-core: rows up to this length claimed by a block's level scan are drained by
                                 // that block; longer ones by every warp in the next sub-round
    uint32_t tail_max = 65536;   // k-core: once at most this many vertices remain, one thread-block cluster
                                 // finishes the levels on the compacted remaining graph (0: never)
    uint32_t batch_split = 0;    // batches: a graph whose work (2m + n) exceeds this is solved by the
                                 // grid-wide kernels (0: above twice a block's share and 2^20)
    uint32_t batch_block = 512;  // batches: threads per block of the block-per-graph kernel
    uint32_t peel_lazy = 1;      // peel: thin-tail rounds test only the candidate list (0: every round
                                 // tests the whole alive list); read from the global tuning only
    uint32_t peel_vec = 0;       // peel: long rows read as aligned 128-bit groups (0: one entry per lane);
                                 // read from the global tuning only
};

// Tuning of a batch of G graphs with `work` = sum of (2m + n): the autotuned
// entry of its class if there is one, else current_tuning().
Tuning tuning_for_batch(uint32_t G, uint64_t work);

Tuning current_tuning();

// Tuning for a solve of kernel 0 (peel) or 1 (core numbers) on graph g: the
// autotuned entry of g's size class if there is one, else current_tuning().
Tuning tuning_for(const dsg_graph* g, int kernel);

// Autotuned solve times (ms) of g's size class for the peel (at the tuning
// eps) and the core numbers; false unless both were tuned.
bool tuned_times(const dsg_graph* g, double* peel_ms, double* core_ms);

// Counts one kernel launch and, when profiling is on, brackets it with CUDA
// events on its stream.  Construct right before the launch, destroy right
// after it:  { LaunchScope ls("name", s); kernel<<<...>>>(...); }
class LaunchScope {
  public:
    LaunchScope(const char* name, cudaStream_t s);
    ~LaunchScope();
  private:
    const char* name_;
    cudaStream_t s_;
    void* a_ = nullptr;
    void* b_ = nullptr;
    bool timed_ = false;
};

// Ingest raw pairs held in a CSR (each entry (v, adj[j]) is one pair).
dsg_status ingest_from_csr_entries(uint32_t n, const uint64_t* off, const uint32_t* adj, uint64_t total,
                                   uint32_t flags, cudaStream_t s, dsg_graph** out);

// One peel on a graph (any dsg_graph, including a view into a packed batch):
// set_dev (device, nullable) gets the densest-set mask; out4 = E, V, rounds,
// best_round.
// extra2 (nullable): sum over the rounds of |S_r| and the alive-neighbour decrements.
dsg_status peel_into(const dsg_graph* g, uint32_t p, uint32_t q, uint8_t* set_dev, uint64_t out4[4],
                     uint64_t* extra2 = nullptr);

// Core numbers of a graph into core_out (host or device); stats nullable.
dsg_status run_kcore(const dsg_graph* g, uint32_t* core_out, uint64_t* stats, uint32_t nstats,
                     uint64_t* trace_dev = nullptr, uint64_t trace_cap = 0, uint64_t* stamps = nullptr);

// The last levels of the core numbers on the compacted remaining graph (the
// vertices whose claim bit is clear; deg holds their degrees), by one
// thread-block cluster; writes their core numbers into deg and adds its
// levels, scanned remaining entries and atomics into stats5[0], [2], [4];
// with a trace buffer, block 0 stamps each level's phases there.
constexpr uint32_t kTailMaxVertices = 16 * 8192;
dsg_status kcore_tail(uint32_t n, const uint64_t* off, const uint32_t* adj, uint32_t* deg, const uint32_t* claim,
                      uint32_t cap, cudaStream_t s, uint64_t* stats5, uint64_t* trace = nullptr,
                      uint64_t trace_cap = 0, uint64_t* stamps = nullptr);

// Device check that a graph is canonical (sorted rows, no loops, no repeats,
// symmetric, ids < n).  DSG_EINVAL with a message if not.
dsg_status validate_csr(const dsg_graph* g);

// Grid size for a cooperative launch of `kernel` with `block` threads and
// `smem` dynamic shared memory, capped so small problems use few blocks (and
// at max_grid when that is non-zero).
template <class K>
cudaError_t coop_grid(K kernel, uint32_t block, size_t smem, uint64_t work_items, uint32_t blocks_per_sm,
                      uint32_t* grid, uint32_t max_grid = 0) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, (int)block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (blocks_per_sm && (int)blocks_per_sm < per_sm) per_sm = (int)blocks_per_sm;
    uint64_t g = (uint64_t)per_sm * (uint64_t)dev_info().sms;
    uint64_t need = (work_items + block - 1) / block;
    if (need < 1) need = 1;
    if (g > need) g = need;
    if (max_grid && g > max_grid) g = max_grid;
    *grid = (uint32_t)g;
    return cudaSuccess;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const unsigned long long* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Per-block table that combines degree decrements aimed at the same
// high-degree vertex, so a hub adjacent to thousands of failing vertices
// takes one global atomic per block and phase instead of one per edge.
// Open addressing over kAggSlots (key, count) pairs; a full probe sequence
// falls back to a direct global atomic.
constexpr uint32_t kAggBits = 11;
constexpr uint32_t kAggSlots = 1u << kAggBits;
constexpr uint32_t kAggEmpty = 0xffffffffu;

// The degree at which combining pays: a vertex takes about deg / gridDim.x
// decrements per block, so combining helps once that is well above one.
__device__ __forceinline__ uint32_t hot_threshold(uint32_t hot_deg) {
    return hot_deg ? hot_deg : 4u * gridDim.x;
}

struct AggTable {
    uint32_t key[kAggSlots];
    uint32_t cnt[kAggSlots];
};

__device__ __forceinline__ void agg_clear(AggTable& t) {
    for (uint32_t i = threadIdx.x; i < kAggSlots; i += blockDim.x) {
        t.key[i] = kAggEmpty;
        t.cnt[i] = 0;
    }
}

// Adds one to u's slot; false if no slot could be claimed.
__device__ __forceinline__ bool agg_add(AggTable& t, uint32_t u) {
    uint32_t h = (u * 0x9E3779B1u) >> (32 - kAggBits);
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
        uint32_t s = (h + i) & (kAggSlots - 1);
        uint32_t prev = atomicCAS(&t.key[s], kAggEmpty, u);
        if (prev == kAggEmpty || prev == u) {
            atomicAdd(&t.cnt[s], 1u);
            return true;
        }
    }
    return false;
}

// Shared scratch of the block-wide scans and reductions of the round kernels.
template <int TB>
struct TileSmem {
    uint32_t scan_tmp[33];
    uint64_t scan_tmp64[33];
};

constexpr uint32_t kBatch = 4;  // entries handed to a visitor per thread and call

// Shared memory of the block-wide walker below.
template <int TB>
struct BlockTile {
    uint32_t start[TB];  // exclusive prefix of row lengths
    uint64_t beg[TB];    // row start in adj
    uint32_t v[TB];      // row owner
    uint32_t scan_tmp[33];
};

// Walk the rows of a block-private list F[lo, hi) with the whole block:
// TB rows at a time, their lengths prefix-summed, the concatenated entries
// spread evenly over all threads (a few long rows are shared by every warp).
// Same visitor contract as scan_frontier; every thread of the block calls it.
template <int TB, class Fn>
__device__ __forceinline__ void scan_block_list(const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj,
                                                const uint32_t* F, uint64_t lo, uint64_t hi, BlockTile<TB>& sm,
                                                Fn& fn) {
    const uint32_t tid = threadIdx.x;
    for (uint64_t t = lo; t < hi; t += TB) {
        uint32_t cnt = (uint32_t)min((uint64_t)TB, hi - t);
        uint32_t v = 0, len = 0;
        uint64_t b = 0;
        if (tid < cnt) {
            v = F[t + tid];
            b = off[v];
            len = (uint32_t)(off[v + 1] - b);
        }
        uint32_t total;
        uint32_t st = block_excl_scan<uint32_t>(len, sm.scan_tmp, &total);
        sm.start[tid] = st;
        sm.beg[tid] = b;
        sm.v[tid] = v;
        __syncthreads();
        for (uint32_t e0 = tid; e0 < total; e0 += kBatch * TB) {
            uint32_t bu[kBatch], bv[kBatch], valid = 0;
#pragma unroll
            for (uint32_t j = 0; j < kBatch; ++j) {
                uint32_t e = e0 + j * TB;
                bu[j] = 0;
                bv[j] = 0;
                if (e < total) {
                    uint32_t a = 0, z = cnt;  // owner = last row whose start is <= e
                    while (z - a > 1) {
                        uint32_t mid = (a + z) >> 1;
                        if (sm.start[mid] <= e) a = mid; else z = mid;
                    }
                    bu[j] = ld_stream(adj + sm.beg[a] + (e - sm.start[a]));
                    bv[j] = sm.v[a];
                    valid |= 1u << j;
                }
            }
            fn(bu, bv, valid);
        }
        __syncthreads();
    }
}

// scan_block_list over rows whose starts and lengths are already known:
// rows F[0, cnt) with row starts B[] and lengths L[].
template <int TB, class Fn>
__device__ __forceinline__ void scan_block_rows(const uint32_t* __restrict__ adj, const uint32_t* F,
                                                const uint64_t* B, const uint32_t* L, uint32_t cnt_all,
                                                BlockTile<TB>& sm, Fn& fn) {
    const uint32_t tid = threadIdx.x;
    for (uint32_t t = 0; t < cnt_all; t += TB) {
        const uint32_t cnt = min((uint32_t)TB, cnt_all - t);
        uint32_t v = 0, len = 0;
        uint64_t b = 0;
        if (tid < cnt) {
            v = F[t + tid];
            b = B[t + tid];
            len = L[t + tid];
        }
        uint32_t total;
        const uint32_t st = block_excl_scan<uint32_t>(len, sm.scan_tmp, &total);
        sm.start[tid] = st;
        sm.beg[tid] = b;
        sm.v[tid] = v;
        __syncthreads();
        for (uint32_t e0 = tid; e0 < total; e0 += kBatch * TB) {
            uint32_t bu[kBatch], bv[kBatch], valid = 0;
#pragma unroll
            for (uint32_t j = 0; j < kBatch; ++j) {
                const uint32_t e = e0 + j * TB;
                bu[j] = 0;
                bv[j] = 0;
                if (e < total) {
                    uint32_t a = 0, z = cnt;  // owner = last row whose start is <= e
                    while (z - a > 1) {
                        const uint32_t mid = (a + z) >> 1;
                        if (sm.start[mid] <= e) a = mid; else z = mid;
                    }
                    bu[j] = ld_stream(adj + sm.beg[a] + (e - sm.start[a]));
                    bv[j] = sm.v[a];
                    valid |= 1u << j;
                }
            }
            fn(bu, bv, valid);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- edge walker
// Visit every adjacency position j in [0, off[n]) with its row owner.
// Each warp takes one contiguous span of positions, finds the row of its first
// position by binary search over off, and then moves through the span
// kWalkU * 32 consecutive positions at a time (lane l takes l, l + 32, ...):
// pre(j) is issued for every position of a step before the owners are
// searched (so its loads overlap the search), and a lane finds each
// position's row among the next 32 row starts (one coalesced read by the
// warp) with a 5-step shuffle search; positions past those 32 rows (runs of
// short or empty rows) find their 32-row block from a coarse sample of the
// row starts (one coalesced read over 1,024 rows) and their row by a 5-step
// binary search inside it.
// fn(owner[], j[], pre[], valid) is called by all lanes together, bit t of
// valid set when slot t holds a position.
constexpr uint32_t kWalkU = 4;

template <class Pre, class Fn>
__device__ __forceinline__ void walk_all_entries(const uint64_t* __restrict__ off, uint32_t n, Pre& pre, Fn& fn) {
    const uint64_t total = off[n];
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    constexpr uint32_t kStep = 32 * kWalkU;
    uint64_t span = (total + nw - 1) / nw;
    span = span < 2 * kStep ? 2 * kStep : ((span + kStep - 1) / kStep * kStep);
    const uint64_t j0 = gw * span;
    if (j0 >= total) return;
    const uint64_t j1 = min(total, j0 + span);
    // row r with off[r] <= j0 < off[r + 1]
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (off[mid] <= j0) lo = mid; else hi = mid;
    }
    uint32_t r = lo;
    for (uint64_t jb = j0; jb < j1; jb += kStep) {
        uint64_t j[kWalkU];
        uint32_t pv[kWalkU], owner[kWalkU], valid = 0, done = 0;
#pragma unroll
        for (uint32_t t = 0; t < kWalkU; ++t) {
            j[t] = jb + lane + 32 * t;
            owner[t] = r;
            pv[t] = 0;
            if (j[t] < j1) {
                valid |= 1u << t;
                pv[t] = pre(j[t]);
            }
        }
        done = ~valid & ((1u << kWalkU) - 1);
        {
            const uint32_t base = r;
            const uint32_t idx = base + 1 + lane;
            const uint64_t w = off[idx < n ? idx : n];
            const uint64_t w31 = __shfl_sync(kFullMask, w, 31);
#pragma unroll
            for (uint32_t t = 0; t < kWalkU; ++t) {
                uint32_t c = 0;
#pragma unroll
                for (uint32_t step = 16; step > 0; step >>= 1) {
                    const uint64_t wv = __shfl_sync(kFullMask, w, c + step - 1);
                    if (wv <= j[t]) c += step;
                }
                if (c == 31 && w31 <= j[t]) c = 32;
                if (!(done >> t & 1u) && c < 32) {
                    owner[t] = base + c;
                    done |= 1u << t;
                }
            }
            // positions past the window (runs of short or empty rows): every
            // pending position lies at or above off[b].  Lane l reads
            // off[b + S l] (one coalesced read; S rows apart), a position's
            // count of those <= it names the S-row block holding its row, and
            // a binary search over that block's row starts (log2 S steps, all
            // lanes and slots at once) places it.  Positions beyond the 32
            // blocks move b up by 31 S; a pass that places nothing widens S;
            // after 64 passes a plain binary search places what is left.
            uint64_t b = (uint64_t)base + 32, S = 32;
            for (uint32_t pass = 0; __any_sync(kFullMask, done != (1u << kWalkU) - 1); ++pass) {
                if (pass == 64) {
                    // rows spread very far apart: a binary search over [b, n) places the rest
#pragma unroll
                    for (uint32_t t = 0; t < kWalkU; ++t) {
                        if (done >> t & 1u) continue;
                        uint64_t lo = b, hi = n;  // off[b] <= j < off[n]
                        while (hi - lo > 1) {
                            const uint64_t mid = lo + ((hi - lo) >> 1);
                            if (off[mid] <= j[t]) lo = mid; else hi = mid;
                        }
                        owner[t] = (uint32_t)lo;
                        done |= 1u << t;
                    }
                    break;
                }
                const uint64_t cidx = b + S * lane;
                const uint64_t cw = off[cidx < n ? cidx : n];  // off[n] = total: above every position
                const uint64_t cw31 = __shfl_sync(kFullMask, cw, 31);
                uint32_t placed = 0;
#pragma unroll
                for (uint32_t t = 0; t < kWalkU; ++t) {
                    uint32_t c = 0;
#pragma unroll
                    for (uint32_t step = 16; step > 0; step >>= 1) {
                        const uint64_t wv = __shfl_sync(kFullMask, cw, c + step - 1);
                        if (wv <= j[t]) c += step;
                    }
                    if (c == 31 && cw31 <= j[t]) c = 32;
                    if (!(done >> t & 1u) && c < 32) {
                        // off[b + S (c-1)] <= j < off[min(b + S c, n)]; c >= 1 since off[b] <= j
                        uint64_t lo = b + S * (c - 1), hi = b + S * c;
                        if (hi > n) hi = n;
                        while (hi - lo > 1) {
                            const uint64_t mid = lo + ((hi - lo) >> 1);
                            if (off[mid] <= j[t]) lo = mid; else hi = mid;
                        }
                        owner[t] = (uint32_t)lo;
                        done |= 1u << t;
                        ++placed;
                    }
                }
                // what is still pending lies at or above off[b + 31 S]
                b += 31 * S;
                if (!__any_sync(kFullMask, placed != 0)) S *= 32;
            }
        }
        fn(owner, j, pv, valid);
        // next step starts at or after the row of this step's last position
        const uint32_t last = valid >> (kWalkU - 1) & 1u ? owner[kWalkU - 1] : r;
        r = __shfl_sync(kFullMask, last, 31);
        if (!__shfl_sync(kFullMask, valid >> (kWalkU - 1) & 1u, 31)) break;  // span's final step
    }
}

// Walk every adjacency entry of a frontier, handing entries to the visitor
// four at a time per thread so the visitor can issue four independent loads
// (then four independent atomics) before it waits on any of them.  No block
// barrier is used: every warp works on its own share.
//   short rows: F[lo, hi), one vertex per entry; a warp takes 32 of them,
//     prefix-sums their lengths with shuffles and spreads the concatenated
//     entries over its lanes (consecutive lanes read consecutive entries); a
//     lane finds the row owning an entry by a 5-step shuffle binary search.
//   long rows: C[clo, chi), items (v << 32 | c) standing for entries
//     [off[v] + c*chunk_len, min(off[v+1], off[v] + (c+1)*chunk_len)); one warp
//     per item, 32 consecutive entries per step, four steps in flight.
// fn(u[4], v[4], valid) is called with bit j of `valid` set for each filled
// slot j (u = neighbour, v = row owner).  All lanes of a warp call fn
// together (valid may be 0).
// LOCAL = true: F is this block's own list (e.g. in shared memory) and only
// this block's warps walk it; C is ignored.
// FB / FL (nullable): row starts and lengths stored beside F, saving the
// offset loads of the short rows.
// vec_end (0: off): adj is 16-byte aligned and holds at least vec_end
// entries; long rows are then read with 128-bit loads.
template <int TB, bool LOCAL = false, class Fn>
__device__ __forceinline__ void scan_frontier(const uint64_t* __restrict__ off, const uint32_t* __restrict__ adj,
                                              const uint32_t* F, uint64_t lo, uint64_t hi,
                                              const uint64_t* __restrict__ C, uint64_t clo, uint64_t chi,
                                              uint32_t chunk_len, Fn& fn, uint32_t dbg_n = 0,
                                              const uint64_t* FB = nullptr, const uint32_t* FL = nullptr,
                                              uint64_t vec_end = 0) {
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31u;
    const uint64_t gw = LOCAL ? (uint64_t)(tid >> 5) : ((uint64_t)blockIdx.x * TB + tid) >> 5;
    const uint64_t nw = LOCAL ? (uint64_t)(TB >> 5) : ((uint64_t)gridDim.x * TB) >> 5;
    // ---- short rows, 32 per warp, edge-balanced over the warp's lanes
    auto short_group = [&](uint64_t g0) {
        uint64_t i = g0 + lane;
        uint32_t v = 0, len = 0;
        uint64_t b = 0;
        if (i < hi) {
            v = F[i];
#ifdef DSG_DEBUG_BOUNDS
            if (v >= dbg_n) {
                uint32_t bu[kBatch] = {0xfffffffeu}, bv[kBatch] = {v};
                fn(bu, bv, 1u);
                v = 0;
            }
#endif
            if (FB) {
                b = FB[i];
                len = FL[i];
            } else {
                b = off[v];
                len = (uint32_t)(off[v + 1] - b);
            }
        }
        const uint32_t inc = warp_incl_scan(len);
        const uint32_t total = __shfl_sync(kFullMask, inc, 31);
        const uint32_t st = inc - len;
        for (uint32_t e0 = lane; e0 < ((total + 31u) & ~31u); e0 += 32 * kBatch) {
            uint32_t bu[kBatch], bv[kBatch], valid = 0;
#pragma unroll
            for (uint32_t j = 0; j < kBatch; ++j) {
                const uint32_t e = e0 + 32 * j;
                // owner = last lane whose start is <= e (all lanes take part in the shuffles)
                uint32_t a = 0;
#pragma unroll
                for (uint32_t step = 16; step > 0; step >>= 1) {
                    uint32_t s_mid = __shfl_sync(kFullMask, st, a + step);
                    if (a + step < 32 && s_mid <= e) a += step;
                }
                const uint32_t ost = __shfl_sync(kFullMask, st, a);
                const uint64_t ob = __shfl_sync(kFullMask, b, a);
                const uint32_t ov = __shfl_sync(kFullMask, v, a);
                bu[j] = 0;
                bv[j] = ov;
                if (e < total) {
                    uint64_t pos = ob + (e - ost);
#ifdef DSG_DEBUG_BOUNDS
                    if (pos >= off[dbg_n]) { bu[j] = 0xffffffffu; bv[j] = 0xffffffffu; valid |= 1u << j; continue; }
#endif
                    bu[j] = ld_stream(adj + pos);
                    valid |= 1u << j;
                }
            }
            fn(bu, bv, valid);
        }
    };
    // ---- long rows, one warp per chunk item
    auto chunk_item = [&](uint64_t it) {
        uint64_t item = C[it];
        uint32_t v = (uint32_t)(item >> 32);
#ifdef DSG_DEBUG_BOUNDS
        if (v >= dbg_n) {
            uint32_t bu[kBatch] = {0xfffffffdu}, bv[kBatch] = {v};
            fn(bu, bv, 1u);
            return;
        }
#endif
        uint64_t c = item & 0xffffffffull;
        uint64_t b = off[v], e_end = off[v + 1];
        uint64_t beg = b + c * chunk_len;
        uint64_t end = min(e_end, beg + chunk_len);
        if (vec_end) {
            // 128-bit loads: lane l takes the aligned group of four entries 4g..4g+3, g = g0 + l
            // (+ 32 per step); entries of a group outside [beg, end) are masked off, and a
            // group that reaches past vec_end is read entry by entry
            static_assert(kBatch == 4, "one 16-byte group per visitor call");
            const uint64_t g0 = beg >> 2, g1 = (end + 3) >> 2;
            for (uint64_t gb = g0; gb < g1; gb += 32) {
                const uint64_t g = gb + lane;
                uint32_t bu[kBatch] = {0u, 0u, 0u, 0u}, bv[kBatch] = {v, v, v, v}, valid = 0;
                if (g < g1) {
                    const uint64_t e0 = g * 4;
                    if (e0 + 4 <= vec_end) {
                        const uint4 q = __ldcs(reinterpret_cast<const uint4*>(adj) + g);
                        bu[0] = q.x;
                        bu[1] = q.y;
                        bu[2] = q.z;
                        bu[3] = q.w;
                    } else {
#pragma unroll
                        for (uint32_t j = 0; j < kBatch; ++j)
                            if (e0 + j >= beg && e0 + j < end) bu[j] = ld_stream(adj + e0 + j);
                    }
#pragma unroll
                    for (uint32_t j = 0; j < kBatch; ++j)
                        if (e0 + j >= beg && e0 + j < end) valid |= 1u << j;
                }
                fn(bu, bv, valid);
            }
            return;
        }
        for (uint64_t j0 = beg + lane; j0 < end; j0 += 32 * kBatch) {
            uint32_t bu[kBatch], bv[kBatch], valid = 0;
#pragma unroll
            for (uint32_t j = 0; j < kBatch; ++j) {
                uint64_t jj = j0 + 32 * j;
                bu[j] = 0;
                bv[j] = v;
                if (jj < end) {
                    bu[j] = ld_stream(adj + jj);
                    valid |= 1u << j;
                }
            }
            fn(bu, bv, valid);
        }
    };
    for (uint64_t g0 = lo + gw * 32; g0 < hi; g0 += nw * 32) short_group(g0);
    for (uint64_t it = LOCAL ? chi : clo + gw; it < chi; it += nw) chunk_item(it);
}

}  // namespace dsg
