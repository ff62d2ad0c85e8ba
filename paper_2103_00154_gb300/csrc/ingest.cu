// CSR ingest: raw undirected pairs -> canonical CSR (Def. 1: a simple graph,
// E a set of edges between distinct vertices).
//
//   1. histogram  the non-loop entries (each pair gives owner -> neighbour in
//                 both directions) counted over <= 2^16 ranges of vertex ids
//   2. plan       ranges cut into buckets of consecutive owners holding
//                 similar numbers of entries
//   3. scatter    every entry appended to its owner's bucket
//   4. rows       one block per bucket: its owners' counts, row starts and
//                 entries placed in their rows, in shared memory
//   5. sort       each row sorted and de-duplicated in place; rows are binned
//                 by length: <= 32 entries one warp, one value per lane;
//                 <= 1024 one warp holding up to 32 values per lane (register
//                 bitonic network, no shared memory); <= 8192 one block (each
//                 warp sorts 1024 values in registers, cross-warp merge steps
//                 go through shared memory); longer ("giant") rows one block
//                 each, by a stable LSD radix sort on 8-bit digits
//   6. scan       final row lengths -> off
//   7. copy       unique entries into adj
// The result is byte-identical to sorting the (min, max) keys and removing
// repeats, because a canonical CSR of a given edge set is unique.
#include <cooperative_groups.h>

#include <algorithm>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

namespace cg = cooperative_groups;

namespace dsg {

constexpr uint32_t kPad = 0xffffffffu;
constexpr uint32_t kScanTile = 2048;
constexpr uint32_t kBlockRowMax = 8192;  // longest row sorted by one block (8 warps x 1024)
constexpr int kClasses = 9;              // 0..4: warp rows E = 2..32, 5..7: block rows of 2/4/8 warps, 8: giant
constexpr int kGiant = 8;

__global__ void validate_off_kernel(uint32_t n, const uint64_t* __restrict__ off, uint32_t* bad);

struct IngestCtl {
    uint32_t err;
    uint32_t cls_count[kClasses];   // rows per sort class
    uint32_t cls_fill[kClasses];    // list cursors
    uint32_t pad;
    unsigned long long giant_entries;
};

// sort class of a row of raw length len (-1: at most 32 entries)
__device__ __forceinline__ int row_class(uint32_t len) {
    if (len <= 32) return -1;
    if (len <= 64) return 0;
    if (len <= 128) return 1;
    if (len <= 256) return 2;
    if (len <= 512) return 3;
    if (len <= 1024) return 4;
    if (len <= 2048) return 5;
    if (len <= 4096) return 6;
    if (len <= kBlockRowMax) return 7;
    return kGiant;
}

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

// Exclusive scan of n uint32 values into out[0..n], out[n] = total (device
// buffers, stream-ordered; the tile sums live in sc).
dsg_status scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, Scratch& sc, cudaStream_t s) {
    uint64_t* sums;
    DSG_TRY_CUDA(sc.get(&sums, n / kScanTile + 2));
    DSG_TRY_CUDA(device_scan(in, n, out, sums, s));
    return DSG_OK;
}

// ----------------------------------------------------------- count / scatter

// ------------------------------------------ bucketed count and scatter
// Rows are built without a global atomic per entry.  The directed entries
// (owner -> neighbour; each non-loop pair gives two) are first appended to
// buckets of consecutive owners -- one global atomic per block tile and
// bucket, and each bucket's tail is written sequentially, so the writes merge
// into whole sectors in L2 -- and then one block per bucket counts the
// bucket's owners and places their entries with shared-memory counters and
// cursors, writing only inside the bucket's own (small) region of the rows.
// Bucket boundaries come from an exact histogram of the entries over at most
// 2^15 equal ranges of vertex ids: a range starts a new bucket where the
// entries before it cross a multiple of the target bucket size, or every
// span_cut ranges (so a bucket's vertices fit the row builder's counters),
// so buckets hold similar numbers of entries whatever the degree
// distribution.  Which buckets are formed changes speed, never the result.
constexpr uint32_t kRangesMax = 32768;
constexpr uint32_t kBucketTarget = 8192;     // buckets aimed for by entry count
constexpr uint64_t kBucketMinEntries = 4096; // ... but none smaller than this by entry count
constexpr uint32_t kSpanMax = 16384;         // owners the row builder counts at once (64 KB of counters)
constexpr uint32_t kSpanCutBuckets = 4096;   // span cuts at most
constexpr uint32_t kBucketsMax = kBucketTarget + 1 + kSpanCutBuckets + 1;

struct BucketPlan {
    uint32_t rshift;    // range of a vertex v: v >> rshift
    uint32_t nranges;   // ceil(n / 2^rshift) <= kRangesMax
    uint32_t span_cut;  // a bucket also starts at every multiple of span_cut ranges
};

static BucketPlan bucket_plan_for(uint32_t n) {
    BucketPlan pl;
    pl.rshift = 0;
    while (((uint64_t)n + (1ull << pl.rshift) - 1) >> pl.rshift > kRangesMax) ++pl.rshift;
    pl.nranges = (uint32_t)(((uint64_t)n + (1ull << pl.rshift) - 1) >> pl.rshift);
    const uint32_t width = 1u << pl.rshift;
    uint32_t cut = width <= kSpanMax ? kSpanMax / width : 1;
    const uint32_t need = (pl.nranges + kSpanCutBuckets - 1) / kSpanCutBuckets;  // at most kSpanCutBuckets cuts
    pl.span_cut = cut > need ? cut : need;
    return pl;
}

// Exact histogram of the entries over the vertex ranges: each block counts
// its share of the pairs in shared memory (32-bit counts) and adds its counts
// to the global ones once.  Ids out of range set ERR_RANGE.
__global__ void __launch_bounds__(1024) range_hist_kernel(uint32_t n, uint64_t m_raw, const uint32_t* __restrict__ src,
                                                          const uint32_t* __restrict__ dst, BucketPlan pl,
                                                          uint32_t* __restrict__ range_cnt, IngestCtl* ctl) {
    extern __shared__ uint32_t hc[];
    for (uint32_t r = threadIdx.x; r < pl.nranges; r += blockDim.x) hc[r] = 0;
    __syncthreads();
    bool bad = false;
    // four pairs per thread and step, their loads in flight together
    constexpr uint32_t kU = 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < m_raw; i0 += kU * stride) {
        uint32_t u[kU], v[kU];
#pragma unroll
        for (uint32_t j = 0; j < kU; ++j) {
            const uint64_t i = i0 + j * stride;
            u[j] = i < m_raw ? src[i] : 0u;
            v[j] = i < m_raw ? dst[i] : 0u;
        }
#pragma unroll
        for (uint32_t j = 0; j < kU; ++j) {
            if (i0 + j * stride >= m_raw) continue;
            if (u[j] >= n || v[j] >= n) {
                bad = true;
                continue;
            }
            if (u[j] == v[j]) continue;
            atomicAdd(&hc[u[j] >> pl.rshift], 1u);
            atomicAdd(&hc[v[j] >> pl.rshift], 1u);
        }
    }
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < pl.nranges; r += blockDim.x)
        if (hc[r]) atomicAdd(&range_cnt[r], hc[r]);
    if (bad) atomicOr(&ctl->err, ERR_RANGE);
}

// One block: buckets from the range histogram.  Range r starts a bucket when
// r == 0, when the entries before it and those before range r-1 lie in
// different multiples of the target, or when r is a multiple of span_cut.
// Writes range_bucket[r], the first vertex and the entry base of every
// bucket (bucket_v0[F] = n, bucket_base[F] = total entries), start[n] =
// total, *nb = F and *maxb = the largest bucket's entries.
constexpr uint32_t kPlanPer = kRangesMax / 1024;  // ranges per thread

__global__ void __launch_bounds__(1024) bucket_plan_kernel(uint32_t n, const uint32_t* __restrict__ range_cnt,
                                                           BucketPlan pl, uint16_t* __restrict__ range_bucket,
                                                           uint32_t* __restrict__ bucket_v0,
                                                           uint64_t* __restrict__ bucket_base,
                                                           uint64_t* __restrict__ start, uint32_t* __restrict__ nb,
                                                           unsigned long long* __restrict__ maxb) {
    __shared__ uint64_t tmp64[33];
    __shared__ uint32_t tmp32[33];
    const uint32_t r0 = threadIdx.x * kPlanPer;
    auto c = [&](uint32_t j) -> uint64_t { return r0 + j < pl.nranges ? range_cnt[r0 + j] : 0; };
    uint64_t mine = 0;
    for (uint32_t j = 0; j < kPlanPer; ++j) mine += c(j);
    uint64_t total;
    uint64_t pre = block_excl_scan<uint64_t>(mine, tmp64, &total);
    uint64_t target = (total + kBucketTarget - 1) / kBucketTarget;
    if (target < kBucketMinEntries) target = kBucketMinEntries;
    // flags, then bucket ids by a scan of the flags
    uint64_t flags = 0;
    uint32_t nf = 0;
    uint64_t p = pre;  // entries before range r0 + j
    for (uint32_t j = 0; j < kPlanPer; ++j) {
        const uint32_t r = r0 + j;
        const uint64_t cj = c(j);
        if (r < pl.nranges) {
            const uint64_t prev = r == 0 ? 0 : p - range_cnt[r - 1];
            const bool f = r == 0 || p / target != prev / target || r % pl.span_cut == 0;
            if (f) {
                flags |= 1ull << j;
                ++nf;
            }
        }
        p += cj;
    }
    uint32_t nf_total;
    const uint32_t id0 = block_excl_scan<uint32_t>(nf, tmp32, &nf_total);
    uint32_t id = id0;
    p = pre;
    for (uint32_t j = 0; j < kPlanPer; ++j) {
        const uint32_t r = r0 + j;
        if (r < pl.nranges) {
            if (flags >> j & 1ull) {
                bucket_v0[id] = r << pl.rshift;
                bucket_base[id] = p;
                ++id;
            }
            range_bucket[r] = (uint16_t)(id - 1);
        }
        p += c(j);
    }
    if (threadIdx.x == 0) {
        bucket_v0[nf_total] = n;
        bucket_base[nf_total] = total;
        start[n] = total;
        *nb = nf_total;
    }
    __syncthreads();  // every bucket base is written (and visible to the block)
    uint64_t big = 0;
    for (uint32_t b = id0; b < id; ++b) big = max(big, bucket_base[b + 1] - bucket_base[b]);
    if (big) atomicMax(maxb, (unsigned long long)big);
}

// The buckets are reached in two partition passes of small fan-out, so that a
// block's tile holds many entries for each destination and writes them as
// contiguous runs: pass A sends every entry of the raw pairs to its group of
// kGroupFine consecutive buckets, pass B splits each group into its buckets.
// A pass ranks a tile's entries per destination in shared memory, reserves
// each destination's share with one global atomic, reorders the tile in
// shared memory by destination and writes it out, consecutive threads to
// consecutive addresses.  Entries are owner << 32 | neighbour.
constexpr uint32_t kGroupFine = 64;                                       // buckets per group
constexpr uint32_t kPartTB = 512;
constexpr uint32_t kPartPer = 8;                                          // entries per thread and tile
constexpr uint32_t kPartTile = kPartTB * kPartPer;                        // entries per tile
constexpr uint32_t kBigChunk = 32768;  // entries per work item of a big bucket in the row builder
constexpr uint32_t kRowsTB = 512;      // threads of the row builder's blocks

// Per-bucket and per-group work: the groups' entry bases, pass B's chunks of
// each group, the row builder's items (one per bucket, or one per kBigChunk
// entries of a bucket above twice the target: a "big" bucket), as prefix
// arrays the consumers search.  One block.
struct PartPlan {
    uint32_t groups;       // G
    uint32_t b_items;      // pass B chunks in all
    uint32_t r_items;      // row-builder items in all
    uint32_t big;          // big buckets
    uint64_t target;       // bucket target (entries)
};

__global__ void __launch_bounds__(1024) part_plan_kernel(const uint32_t* __restrict__ nbp,
                                                         const uint64_t* __restrict__ bucket_base,
                                                         uint64_t* __restrict__ group_base,
                                                         uint32_t* __restrict__ b_pre, uint32_t* __restrict__ r_pre,
                                                         uint32_t* __restrict__ big_list, PartPlan* __restrict__ pp) {
    __shared__ uint32_t tmp[33];
    const uint32_t F = *nbp;
    const uint64_t total = bucket_base[F];
    uint64_t target = (total + kBucketTarget - 1) / kBucketTarget;
    if (target < kBucketMinEntries) target = kBucketMinEntries;
    const uint32_t G = (F + kGroupFine - 1) / kGroupFine;
    // groups: base and pass-B chunk counts (G <= kGroupsMax <= 1024: one per thread)
    {
        const uint32_t g = threadIdx.x;
        uint32_t chunks = 0;
        if (g <= G) group_base[g] = bucket_base[min(g * kGroupFine, F)];
        if (g < G) {
            const uint64_t m = bucket_base[min((g + 1) * kGroupFine, F)] - bucket_base[g * kGroupFine];
            chunks = (uint32_t)((m + kPartTile - 1) / kPartTile);
        }
        uint32_t tot;
        const uint32_t pre = block_excl_scan<uint32_t>(chunks, tmp, &tot);
        if (g < G) b_pre[g] = pre;
        if (threadIdx.x == 0) {
            b_pre[G] = tot;
            pp->b_items = tot;
            pp->groups = G;
            pp->target = target;
        }
    }
    // buckets: row-builder items, in chunks of 1024 buckets
    uint32_t carry = 0, nbig = 0;
    for (uint32_t b0 = 0; b0 < F; b0 += 1024) {
        const uint32_t b = b0 + threadIdx.x;
        uint32_t items = 0;
        bool big = false;
        if (b < F) {
            const uint64_t m = bucket_base[b + 1] - bucket_base[b];
            big = m > 2 * target;
            items = big ? (uint32_t)((m + kBigChunk - 1) / kBigChunk) : 1u;
        }
        uint32_t tot;
        const uint32_t pre = block_excl_scan<uint32_t>(items, tmp, &tot);
        if (b < F) r_pre[b] = carry + pre;
        carry += tot;
        const uint32_t nb = __syncthreads_count(big);
        const uint32_t bpre = block_excl_scan<uint32_t>(big ? 1u : 0u, tmp, &tot);
        if (big) big_list[nbig + bpre] = b;
        nbig += nb;
    }
    if (threadIdx.x == 0) {
        r_pre[F] = carry;
        pp->r_items = carry;
        pp->big = nbig;
    }
}

// Last index i in [0, cnt) with pre[i] <= x (pre ascending, pre[0] = 0).
__device__ __forceinline__ uint32_t find_item(const uint32_t* __restrict__ pre, uint32_t cnt, uint32_t x) {
    uint32_t lo = 0, hi = cnt;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Shared memory of a partition pass: the range -> bucket table, the tile
// reordered by destination, each slot's destination, and per destination its
// count, first slot in the tile and reserved global offset.
struct PartSmem {
    uint64_t stage[kPartTile];
    uint16_t dest[kPartTile];
    uint32_t cnt[256], first[256];
    unsigned long long base[256];
    uint32_t scan_tmp[33];
    uint32_t item;
};

// Reorder the tile's entries (x[j] to destination d[j], local rank r[j]) by
// destination and write each destination's run at dst_base[d] + the
// reservation; every thread of the block calls it.
__device__ __forceinline__ void part_write(PartSmem& sm, uint32_t ndest, const uint64_t (&x)[kPartPer],
                                           const uint32_t (&d)[kPartPer], const uint32_t (&rk)[kPartPer],
                                           const uint64_t* __restrict__ dst_base,
                                           unsigned long long* __restrict__ dst_fill, uint32_t d_first,
                                           uint64_t* __restrict__ out) {
    __syncthreads();  // counts complete
    uint32_t c = threadIdx.x < ndest ? sm.cnt[threadIdx.x] : 0u;
    uint32_t tot;
    const uint32_t f = block_excl_scan<uint32_t>(c, sm.scan_tmp, &tot);
    if (threadIdx.x < ndest) {
        sm.first[threadIdx.x] = f;
        sm.base[threadIdx.x] = c ? dst_base[d_first + threadIdx.x] +
                                       atomicAdd(&dst_fill[d_first + threadIdx.x], (unsigned long long)c)
                                 : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (uint32_t j = 0; j < kPartPer; ++j) {
        if (d[j] == kPad) continue;
        const uint32_t pos = sm.first[d[j]] + rk[j];
        sm.stage[pos] = x[j];
        sm.dest[pos] = (uint16_t)d[j];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tot; i += kPartTB) {
        const uint32_t dd = sm.dest[i];
        out[sm.base[dd] + (i - sm.first[dd])] = sm.stage[i];
    }
    __syncthreads();
    if (threadIdx.x < 256) sm.cnt[threadIdx.x] = 0;
    __syncthreads();  // counts cleared before the next tile ranks into them
}

// Pass A: raw pairs -> groups.  Tiles of kPartTile / 2 pairs.
__global__ void __launch_bounds__(kPartTB, 2) part_pairs_kernel(uint32_t n, uint64_t m_raw,
                                                                const uint32_t* __restrict__ src,
                                                                const uint32_t* __restrict__ dst, BucketPlan pl,
                                                                const uint16_t* __restrict__ range_bucket,
                                                                const PartPlan* __restrict__ pp,
                                                                const uint64_t* __restrict__ group_base,
                                                                unsigned long long* __restrict__ group_fill,
                                                                uint64_t* __restrict__ E1) {
    extern __shared__ __align__(16) unsigned char part_smem_raw[];
    PartSmem& sm = *reinterpret_cast<PartSmem*>(part_smem_raw);
    uint16_t* tab = reinterpret_cast<uint16_t*>(part_smem_raw + sizeof(PartSmem));
    for (uint32_t r = threadIdx.x; r < pl.nranges; r += kPartTB) tab[r] = range_bucket[r];
    if (threadIdx.x < 256) sm.cnt[threadIdx.x] = 0;
    const uint32_t G = pp->groups;
    constexpr uint32_t kPairs = kPartTile / 2;
    const uint64_t ntiles = (m_raw + kPairs - 1) / kPairs;
    __syncthreads();
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint64_t x[kPartPer];
        uint32_t d[kPartPer], rk[kPartPer];
        // the tile's loads first, all in flight together, then the ranking
        uint32_t su[kPartPer / 2], sv[kPartPer / 2];
#pragma unroll
        for (uint32_t j = 0; j < kPartPer / 2; ++j) {
            const uint64_t i = t * kPairs + (uint64_t)j * kPartTB + threadIdx.x;
            su[j] = i < m_raw ? src[i] : 0u;
            sv[j] = i < m_raw ? dst[i] : 0u;
        }
#pragma unroll
        for (uint32_t j = 0; j < kPartPer / 2; ++j) {
            const uint64_t i = t * kPairs + (uint64_t)j * kPartTB + threadIdx.x;
            d[2 * j] = d[2 * j + 1] = kPad;
            x[2 * j] = x[2 * j + 1] = 0;
            if (i < m_raw) {
                const uint32_t u = su[j], v = sv[j];
                // ids out of range were flagged by the histogram; the call fails after this pass
                if (u != v && u < n && v < n) {
                    x[2 * j] = ((uint64_t)u << 32) | v;
                    x[2 * j + 1] = ((uint64_t)v << 32) | u;
                    d[2 * j] = tab[u >> pl.rshift] / kGroupFine;
                    d[2 * j + 1] = tab[v >> pl.rshift] / kGroupFine;
                    rk[2 * j] = atomicAdd(&sm.cnt[d[2 * j]], 1u);
                    rk[2 * j + 1] = atomicAdd(&sm.cnt[d[2 * j + 1]], 1u);
                }
            }
        }
        part_write(sm, G, x, d, rk, group_base, group_fill, 0, E1);
    }
}

// Pass B: each group's entries -> its buckets.  Items: kPartTile-entry chunks of a group.
__global__ void __launch_bounds__(kPartTB, 2) part_groups_kernel(BucketPlan pl, const uint16_t* __restrict__ range_bucket,
                                                                 const uint32_t* __restrict__ nbp,
                                                                 const PartPlan* __restrict__ pp,
                                                                 const uint64_t* __restrict__ group_base,
                                                                 const uint32_t* __restrict__ b_pre,
                                                                 const uint64_t* __restrict__ bucket_base,
                                                                 unsigned long long* __restrict__ bucket_fill,
                                                                 const uint64_t* __restrict__ E1,
                                                                 uint64_t* __restrict__ E2) {
    extern __shared__ __align__(16) unsigned char part_smem_raw[];
    PartSmem& sm = *reinterpret_cast<PartSmem*>(part_smem_raw);
    uint16_t* tab = reinterpret_cast<uint16_t*>(part_smem_raw + sizeof(PartSmem));
    for (uint32_t r = threadIdx.x; r < pl.nranges; r += kPartTB) tab[r] = range_bucket[r];
    if (threadIdx.x < 256) sm.cnt[threadIdx.x] = 0;
    const uint32_t F = *nbp, G = pp->groups, items = pp->b_items;
    __syncthreads();
    for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
        const uint32_t g = find_item(b_pre, G, it);
        const uint64_t lo = group_base[g] + (uint64_t)(it - b_pre[g]) * kPartTile;
        const uint64_t hi = min(group_base[g + 1], lo + kPartTile);
        const uint32_t f0 = g * kGroupFine;
        const uint32_t nd = min(kGroupFine, F - f0);
        uint64_t x[kPartPer];
        uint32_t d[kPartPer], rk[kPartPer];
        // the tile's loads first, all in flight together, then the ranking
#pragma unroll
        for (uint32_t j = 0; j < kPartPer; ++j) {
            const uint64_t e = lo + (uint64_t)j * kPartTB + threadIdx.x;
            x[j] = e < hi ? E1[e] : 0ull;
        }
#pragma unroll
        for (uint32_t j = 0; j < kPartPer; ++j) {
            const uint64_t e = lo + (uint64_t)j * kPartTB + threadIdx.x;
            d[j] = kPad;
            if (e < hi) {
                d[j] = tab[(uint32_t)(x[j] >> 32) >> pl.rshift] - f0;
                rk[j] = atomicAdd(&sm.cnt[d[j]], 1u);
            }
        }
        part_write(sm, nd, x, d, rk, bucket_base, bucket_fill, f0, E2);
    }
}

// Count, in cs[0, len), the entries of E2[lo, hi) whose owner (high word)
// lies in [a, a + len); four entries per thread and step, loads first.
__device__ __forceinline__ void count_owners(const uint64_t* __restrict__ E2, uint64_t lo, uint64_t hi, uint32_t a,
                                             uint32_t len, uint32_t* cs) {
    constexpr uint32_t kU = 4;
    for (uint64_t e0 = lo + threadIdx.x; e0 < hi; e0 += kU * kRowsTB) {
        uint32_t o[kU];
#pragma unroll
        for (uint32_t j = 0; j < kU; ++j) {
            const uint64_t e = e0 + (uint64_t)j * kRowsTB;
            o[j] = e < hi ? (uint32_t)(E2[e] >> 32) - a : 0xffffffffu;
        }
#pragma unroll
        for (uint32_t j = 0; j < kU; ++j)
            if (o[j] < len) atomicAdd(&cs[o[j]], 1u);
    }
}

// Big buckets, step 1: every kBigChunk-entry chunk counts its owners in
// shared memory and adds the counts into cnt[] (zero beforehand).  The
// blocks share out the row builder's items, doing those of big buckets.
__global__ void __launch_bounds__(kRowsTB) big_count_kernel(const uint32_t* __restrict__ nbp,
                                                            const PartPlan* __restrict__ pp,
                                                            const uint32_t* __restrict__ r_pre,
                                                            const uint32_t* __restrict__ bucket_v0,
                                                            const uint64_t* __restrict__ bucket_base,
                                                            const uint64_t* __restrict__ E2, uint32_t* __restrict__ cnt) {
    extern __shared__ uint32_t cs[];
    const uint32_t F = *nbp, items = pp->r_items;
    const uint64_t target = pp->target;
    for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
        const uint32_t b = find_item(r_pre, F, it);
        const uint64_t e0 = bucket_base[b], e1 = bucket_base[b + 1];
        if (e1 - e0 <= 2 * target) continue;  // a small bucket: counted by the row builder
        const uint32_t v0 = bucket_v0[b], v1 = bucket_v0[b + 1];
        const uint64_t lo = e0 + (uint64_t)(it - r_pre[b]) * kBigChunk;
        const uint64_t hi = min(e1, lo + kBigChunk);
        for (uint32_t a = v0; a < v1; a += min(kSpanMax, v1 - a)) {
            const uint32_t len = min(kSpanMax, v1 - a);
            for (uint32_t i = threadIdx.x; i < len; i += kRowsTB) cs[i] = 0;
            __syncthreads();
            count_owners(E2, lo, hi, a, len, cs);
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < len; i += kRowsTB)
                if (cs[i]) atomicAdd(&cnt[a + i], cs[i]);
            __syncthreads();
        }
    }
}

// Big buckets, step 2: one block per big bucket turns its counts into row
// starts (start[v]), clears the cursors and classifies the rows.
__global__ void __launch_bounds__(kRowsTB) big_starts_kernel(const PartPlan* __restrict__ pp,
                                                             const uint32_t* __restrict__ big_list,
                                                             const uint32_t* __restrict__ bucket_v0,
                                                             const uint64_t* __restrict__ bucket_base,
                                                             const uint32_t* __restrict__ cnt,
                                                             uint64_t* __restrict__ start, uint32_t* __restrict__ fill,
                                                             IngestCtl* ctl) {
    __shared__ uint64_t scan64[33];
    __shared__ uint32_t cls[kClasses];
    __shared__ unsigned long long giant;
    if (threadIdx.x < kClasses) cls[threadIdx.x] = 0;
    if (threadIdx.x == 0) giant = 0;
    __syncthreads();
    const uint32_t nbig = pp->big;
    for (uint32_t bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
        const uint32_t b = big_list[bi];
        const uint32_t v0 = bucket_v0[b], v1 = bucket_v0[b + 1];
        uint64_t run0 = bucket_base[b];
        for (uint32_t c0 = v0; c0 < v1; c0 += kRowsTB) {
            const uint32_t v = c0 + threadIdx.x;
            const uint32_t c = v < v1 ? cnt[v] : 0u;
            uint64_t tot;
            const uint64_t pre = block_excl_scan<uint64_t>((uint64_t)c, scan64, &tot);
            if (v < v1) {
                start[v] = run0 + pre;
                fill[v] = 0;
                const int k = row_class(c);
                if (k >= 0) atomicAdd(&cls[k], 1u);
                if (k == kGiant) atomicAdd(&giant, (unsigned long long)c);
            }
            run0 += tot;
        }
    }
    __syncthreads();
    if (threadIdx.x < kClasses && cls[threadIdx.x]) atomicAdd(&ctl->cls_count[threadIdx.x], cls[threadIdx.x]);
    if (threadIdx.x == 0 && giant) atomicAdd(&ctl->giant_entries, giant);
}

// Row builder.  Items (from a device counter): a small bucket is one item --
// its owners are counted, their row starts written (start[v], cnt[v]) and
// their neighbours placed in tmp, kSpanMax owners at a time, with counts and
// cursors in shared memory, writes staying inside the bucket's region; a
// big bucket is one item per kBigChunk entries -- the chunk counts its
// owners, reserves its share of each owner's row (fill[v]) and places its
// entries there.
__global__ void __launch_bounds__(kRowsTB, 2) bucket_rows_kernel(const uint32_t* __restrict__ nbp,
                                                              const PartPlan* __restrict__ pp,
                                                              const uint32_t* __restrict__ r_pre,
                                                              const uint32_t* __restrict__ bucket_v0,
                                                              const uint64_t* __restrict__ bucket_base,
                                                              const uint64_t* __restrict__ E2,
                                                              uint32_t* __restrict__ cnt, uint64_t* __restrict__ start,
                                                              uint32_t* __restrict__ fill, uint32_t* __restrict__ tmp,
                                                              uint32_t* __restrict__ ticket, IngestCtl* ctl) {
    extern __shared__ uint32_t cs[];  // kSpanMax counters / cursors
    __shared__ uint64_t scan64[33];
    __shared__ uint32_t s_it;
    __shared__ uint32_t cls[kClasses];
    __shared__ unsigned long long giant;
    constexpr uint32_t kPer = kSpanMax / kRowsTB;
    const uint32_t F = *nbp, items = pp->r_items;
    const uint64_t target = pp->target;
    if (threadIdx.x < kClasses) cls[threadIdx.x] = 0;
    if (threadIdx.x == 0) giant = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_it = atomicAdd(ticket, 1u);
        __syncthreads();
        const uint32_t it = s_it;
        if (it >= items) break;
        const uint32_t b = find_item(r_pre, F, it);
        const uint32_t v0 = bucket_v0[b], v1 = bucket_v0[b + 1];
        const uint64_t e0 = bucket_base[b], e1 = bucket_base[b + 1];
        if (e1 - e0 > 2 * target) {
            // ---- a chunk of a big bucket
            const uint64_t lo = e0 + (uint64_t)(it - r_pre[b]) * kBigChunk;
            const uint64_t hi = min(e1, lo + kBigChunk);
            for (uint32_t a = v0; a < v1; a += min(kSpanMax, v1 - a)) {
                const uint32_t len = min(kSpanMax, v1 - a);
                for (uint32_t i = threadIdx.x; i < len; i += kRowsTB) cs[i] = 0;
                __syncthreads();
                count_owners(E2, lo, hi, a, len, cs);
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < len; i += kRowsTB) {
                    const uint32_t c = cs[i];
                    if (c) cs[i] = atomicAdd(&fill[a + i], c);  // this chunk's first slot in the row
                }
                __syncthreads();
                for (uint64_t e = lo + threadIdx.x; e < hi; e += kRowsTB) {
                    const uint64_t x = E2[e];
                    const uint32_t o = (uint32_t)(x >> 32) - a;
                    if (o < len) tmp[start[a + o] + atomicAdd(&cs[o], 1u)] = (uint32_t)x;
                }
                __syncthreads();
            }
            continue;
        }
        // ---- a small bucket, whole
        uint64_t sub_base = e0;
        for (uint32_t a = v0; a < v1; a += min(kSpanMax, v1 - a)) {
            const uint32_t len = min(kSpanMax, v1 - a);
            for (uint32_t i = threadIdx.x; i < len; i += kRowsTB) cs[i] = 0;
            __syncthreads();
            count_owners(E2, e0, e1, a, len, cs);
            __syncthreads();
            // exclusive scan of the counts: each thread kPer consecutive owners
            uint64_t mine = 0;
            for (uint32_t j = 0; j < kPer; ++j) {
                const uint32_t i = threadIdx.x * kPer + j;
                if (i < len) mine += cs[i];
            }
            uint64_t sub_total;
            uint64_t run = block_excl_scan<uint64_t>(mine, scan64, &sub_total);
            for (uint32_t j = 0; j < kPer; ++j) {
                const uint32_t i = threadIdx.x * kPer + j;
                if (i >= len) break;
                const uint32_t c = cs[i];
                cnt[a + i] = c;
                start[a + i] = sub_base + run;
                cs[i] = (uint32_t)run;  // cursor, relative to sub_base
                // the row's sort class (rows of at most 32 entries are sorted by class -1)
                const int k = row_class(c);
                if (k >= 0) atomicAdd(&cls[k], 1u);
                if (k == kGiant) atomicAdd(&giant, (unsigned long long)c);
                run += c;
            }
            __syncthreads();
            for (uint64_t e = e0 + threadIdx.x; e < e1; e += kRowsTB) {
                const uint64_t x = E2[e];
                const uint32_t o = (uint32_t)(x >> 32) - a;
                if (o < len) tmp[sub_base + atomicAdd(&cs[o], 1u)] = (uint32_t)x;
            }
            sub_base += sub_total;
            __syncthreads();
        }
    }
    __syncthreads();
    if (threadIdx.x < kClasses && cls[threadIdx.x]) atomicAdd(&ctl->cls_count[threadIdx.x], cls[threadIdx.x]);
    if (threadIdx.x == 0 && giant) atomicAdd(&ctl->giant_entries, giant);
}

// ----------------------------------------------------------- row sort

struct ClassLists {
    uint32_t* rows;             // all class lists, back to back
    uint32_t base[kClasses];    // start of each class in rows
};

// Rows of <= 32 entries, 32 / W rows at a time per warp: row s of a batch in
// lanes [sW, sW + W), one value per lane, a bitonic network over shuffles
// within the segment (ascending in every segment), dedup by comparing with
// the previous lane of the segment.  W = 8, 16 or 32 by the rows' lengths.
// `mask`: the group's rows (lane = row v0 + lane) still to do in this width.
template <uint32_t W>
__device__ __forceinline__ void sort_small_batches(uint32_t mask, uint64_t v0, uint32_t mylen, uint64_t mystart,
                                                   uint32_t* __restrict__ tmp, uint32_t* __restrict__ newlen,
                                                   uint32_t lane) {
    constexpr uint32_t R = 32 / W;
    const uint32_t seg = lane / W, p = lane % W;
    const uint32_t segmask = (W == 32 ? 0xffffffffu : ((1u << W) - 1u)) << (seg * W);
    while (mask) {
        uint32_t src = 32;  // this segment's row (lane of the group), 32: none
#pragma unroll
        for (uint32_t r = 0; r < R; ++r) {
            if (mask) {
                const uint32_t l = __ffs(mask) - 1;
                mask &= mask - 1;
                if (seg == r) src = l;
            }
        }
        const uint32_t len = __shfl_sync(kFullMask, mylen, src & 31u);
        const uint64_t b = __shfl_sync(kFullMask, mystart, src & 31u);
        uint32_t x = (src < 32 && p < len) ? tmp[b + p] : kPad;
#pragma unroll
        for (uint32_t k = 2; k <= W; k <<= 1) {
#pragma unroll
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                const uint32_t y = __shfl_xor_sync(kFullMask, x, j);
                const bool up = k == W || (lane & k) == 0;
                const bool lower = (lane & j) == 0;
                // lower lane keeps min when ascending, max when descending
                x = (lower == up) ? min(x, y) : max(x, y);
            }
        }
        const uint32_t prev = __shfl_up_sync(kFullMask, x, 1);
        const bool keep = x != kPad && (p == 0 || x != prev);
        const uint32_t bal = __ballot_sync(kFullMask, keep) & segmask;
        if (keep) tmp[b + __popc(bal & lanemask_lt())] = x;
        if (p == 0 && src < 32) newlen[v0 + src] = __popc(bal);
    }
}

// Rows of <= 32 entries are sorted and deduplicated in place by
// sort_small_batches (a warp takes 32 consecutive rows at a time); longer
// rows are appended to their class list (warp-aggregated per class).
__global__ void sort_small_rows(uint32_t n, const uint64_t* __restrict__ start, const uint32_t* __restrict__ cnt,
                                uint32_t* __restrict__ tmp, uint32_t* __restrict__ newlen, ClassLists lists,
                                IngestCtl* ctl) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v0 = gw * 32; v0 < n; v0 += nw * 32) {
        uint64_t vl = v0 + lane;
        uint32_t mylen = vl < n ? cnt[vl] : 0;
        int cls = vl < n ? row_class(mylen) : -1;
        uint32_t same = __match_any_sync(kFullMask, cls);
        if (cls >= 0) {
            uint32_t leader = __ffs(same) - 1;
            uint32_t b = 0;
            if (lane == leader) b = atomicAdd(&ctl->cls_fill[cls], (uint32_t)__popc(same));
            b = __shfl_sync(same, b, leader);
            lists.rows[lists.base[cls] + b + __popc(same & lanemask_lt())] = (uint32_t)vl;
        }
        const bool small = vl < n && cls < 0;
        if (small && mylen == 0) newlen[vl] = 0;
        const uint64_t mystart = (small && mylen) ? start[vl] : 0;
        sort_small_batches<8>(__ballot_sync(kFullMask, small && mylen && mylen <= 8), v0, mylen, mystart, tmp,
                              newlen, lane);
        sort_small_batches<16>(__ballot_sync(kFullMask, small && mylen > 8 && mylen <= 16), v0, mylen, mystart,
                               tmp, newlen, lane);
        sort_small_batches<32>(__ballot_sync(kFullMask, small && mylen > 16), v0, mylen, mystart, tmp, newlen,
                               lane);
    }
}

// ---- bitonic network over values held in registers by one warp.
// Value e of lane l has index base + 32e + l.  A compare-exchange at distance
// J >= 32 pairs two registers of the same lane; J < 32 pairs two lanes.  The
// direction of a pair is ascending when (index & k) == 0 (k = block size of
// the current merge), as in the textbook network.
template <int E, uint32_t J>
__device__ __forceinline__ void bitonic_step(uint32_t (&x)[E], uint32_t base, uint32_t k, uint32_t lane) {
    if constexpr (J >= 32) {
        constexpr uint32_t je = J / 32;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if ((e & je) == 0) {
                bool asc = ((base + (uint32_t)e * 32 + lane) & k) == 0;
                uint32_t a = x[e], b = x[e | je];
                x[e] = asc ? min(a, b) : max(a, b);
                x[e | je] = asc ? max(a, b) : min(a, b);
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            uint32_t y = __shfl_xor_sync(kFullMask, x[e], J);
            bool asc = ((base + (uint32_t)e * 32 + lane) & k) == 0;
            bool lower = (lane & J) == 0;
            x[e] = (lower == asc) ? min(x[e], y) : max(x[e], y);
        }
    }
}

// steps J, J/2, ..., 1 of a merge with block size k
template <int E, uint32_t J>
__device__ __forceinline__ void bitonic_merge(uint32_t (&x)[E], uint32_t base, uint32_t k, uint32_t lane) {
    bitonic_step<E, J>(x, base, k, lane);
    if constexpr (J > 1) bitonic_merge<E, J / 2>(x, base, k, lane);
}

// all merges k = 2, 4, ..., K: afterwards the warp's values are sorted, in
// the direction the next merge (block size 2K) expects
template <int E, uint32_t K>
__device__ __forceinline__ void bitonic_sort(uint32_t (&x)[E], uint32_t base, uint32_t lane) {
    if constexpr (K > 2) bitonic_sort<E, K / 2>(x, base, lane);
    bitonic_merge<E, K / 2>(x, base, K, lane);
}

// Write the first of each run of equal sorted values (ascending, kPad last)
// of the warp's registers to out[pos0 ...]; prev_in is the value before
// index 0 (kPad if none).  Returns the number written.
template <int E>
__device__ __forceinline__ uint32_t warp_unique_write(const uint32_t (&x)[E], uint32_t prev_in, uint32_t lane,
                                                      uint32_t* out) {
    uint32_t pos = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        uint32_t up = __shfl_up_sync(kFullMask, x[e], 1);
        uint32_t last_prev = e == 0 ? prev_in : __shfl_sync(kFullMask, x[e > 0 ? e - 1 : 0], 31);
        uint32_t prev = lane == 0 ? last_prev : up;
        bool keep = x[e] != kPad && x[e] != prev;
        uint32_t bal = __ballot_sync(kFullMask, keep);
        if (keep) out[pos + __popc(bal & lanemask_lt())] = x[e];
        pos += __popc(bal);
    }
    return pos;
}

// Rows of 33..1024 entries: one warp per row, E values per lane.
template <int E>
__global__ void __launch_bounds__(256) sort_warp_rows(const uint32_t* __restrict__ list, uint32_t count,
                                                      const uint64_t* __restrict__ start,
                                                      const uint32_t* __restrict__ cnt, uint32_t* __restrict__ tmp,
                                                      uint32_t* __restrict__ newlen) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t r = gw; r < count; r += nw) {
        uint32_t v = list[r];
        uint32_t len = cnt[v];
        uint64_t b = start[v];
        uint32_t x[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            uint32_t i = (uint32_t)e * 32 + lane;
            x[e] = i < len ? tmp[b + i] : kPad;
        }
        bitonic_sort<E, 32 * E>(x, 0, lane);
        uint32_t kept = warp_unique_write<E>(x, kPad, lane, tmp + b);
        if (lane == 0) newlen[v] = kept;
    }
}

// Sorting by one block of kBlockWarps warps (each warp sorts 1024 values in
// registers; merges with block size 2048..p2 run their cross-warp steps,
// distance >= 1024, through shared memory and the rest in registers), then
// keeping the first of each run of equal values.
template <uint32_t kBlockWarps>
struct BlockSortSmem {
    uint32_t s[kBlockWarps * 1024];
    uint32_t wlast[kBlockWarps];
    uint32_t wcount[kBlockWarps];
};

// in[0, len), 1 <= len <= kBlockWarps * 1024, sorted and de-duplicated into
// out[0, kept) (out may be in: every value is in registers before any is
// written); returns kept.  Every thread of the block calls it.
template <uint32_t kBlockWarps>
__device__ __forceinline__ uint32_t block_sort_unique(const uint32_t* in, uint32_t len, uint32_t* out,
                                                      BlockSortSmem<kBlockWarps>& sm) {
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t base = w * 1024;
    uint32_t p2 = 2048;
    while (p2 < len) p2 <<= 1;
    const bool active = base < p2;
    uint32_t x[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        uint32_t i = base + (uint32_t)e * 32 + lane;
        x[e] = (active && i < len) ? in[i] : kPad;
    }
    if (active) bitonic_sort<32, 1024>(x, base, lane);
    for (uint32_t k = 2048; k <= p2; k <<= 1) {
        for (uint32_t j = k >> 1; j >= 1024; j >>= 1) {
            if (active) {
#pragma unroll
                for (int e = 0; e < 32; ++e) sm.s[base + (uint32_t)e * 32 + lane] = x[e];
            }
            __syncthreads();
            if (active) {
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    uint32_t i = base + (uint32_t)e * 32 + lane;
                    uint32_t y = sm.s[i ^ j];
                    bool asc = (i & k) == 0;
                    bool lower = (i & j) == 0;
                    x[e] = (lower == asc) ? min(x[e], y) : max(x[e], y);
                }
            }
            __syncthreads();
        }
        if (active) bitonic_merge<32, 512>(x, base, k, lane);
    }
    // de-duplicate across the block: each warp needs the previous warp's last value
    if (lane == 31) sm.wlast[w] = x[31];
    __syncthreads();
    uint32_t prev_in = (w == 0 || !active) ? kPad : sm.wlast[w - 1];
    // count first, then write at the prefix of the warps' counts
    uint32_t mine = 0;
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        uint32_t up = __shfl_up_sync(kFullMask, x[e], 1);
        uint32_t last_prev = e == 0 ? prev_in : __shfl_sync(kFullMask, x[e > 0 ? e - 1 : 0], 31);
        uint32_t prev = lane == 0 ? last_prev : up;
        mine += __popc(__ballot_sync(kFullMask, x[e] != kPad && x[e] != prev));
    }
    if (lane == 0) sm.wcount[w] = active ? mine : 0;
    __syncthreads();
    uint32_t off = 0, total = 0;
    for (uint32_t q = 0; q < kBlockWarps; ++q) {
        if (q < w) off += sm.wcount[q];
        total += sm.wcount[q];
    }
    if (active) warp_unique_write<32>(x, prev_in, lane, out + off);
    __syncthreads();
    return total;
}

// Rows of 1025..8192 entries: one block of kBlockWarps warps per row.
template <uint32_t kBlockWarps>
__global__ void __launch_bounds__(kBlockWarps * 32) sort_block_rows(const uint32_t* __restrict__ list,
                                                                    uint32_t count,
                                                                    const uint64_t* __restrict__ start,
                                                                    const uint32_t* __restrict__ cnt,
                                                                    uint32_t* __restrict__ tmp,
                                                                    uint32_t* __restrict__ newlen) {
    __shared__ BlockSortSmem<kBlockWarps> sm;
    for (uint32_t r = blockIdx.x; r < count; r += gridDim.x) {
        const uint32_t v = list[r];
        uint32_t* row = tmp + start[v];
        const uint32_t kept = block_sort_unique<kBlockWarps>(row, cnt[v], row, sm);
        if (threadIdx.x == 0) newlen[v] = kept;
    }
}

// ---- giant rows (> kBlockRowMax entries), one block of 8 warps per row:
// splitters taken from a sorted sample of the row (1,024 values spread over
// it) cut its values into ranges of about kSplitTarget entries; the row is
// counted and scattered by range into the spare buffer (equal values share a
// range, so no run of equal ids crosses two ranges), each range is sorted and
// de-duplicated by the block like a block row, and the ranges' unique values
// are copied back, in range order, to the row's place in tmp.  A row with a
// range above kBlockRowMax entries (a very skewed row) goes to a list that
// the radix kernel below sorts instead.
constexpr uint32_t kSplitTarget = 5000;
constexpr uint32_t kSplitMaxRanges = 64;

struct SplitSmem {
    BlockSortSmem<8> bs;
    uint32_t spl[kSplitMaxRanges];         // splitters: range of x = number of splitters <= x
    uint32_t rcnt[kSplitMaxRanges];        // entries per range ...
    uint32_t rcur[kSplitMaxRanges];        // ... scatter cursors ...
    uint32_t rstart[kSplitMaxRanges + 1];  // ... first slot of each range
    uint32_t kept[kSplitMaxRanges + 1];    // unique values per range, then their exclusive prefix
    uint32_t row, nsp, too_big;
};

__device__ __forceinline__ uint32_t split_range(const uint32_t* spl, uint32_t nsp, uint32_t x) {
    uint32_t lo = 0, hi = nsp;  // first splitter > x
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (spl[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) giant_split_kernel(const uint32_t* __restrict__ list, uint32_t count,
                                                          const uint64_t* __restrict__ start,
                                                          const uint32_t* __restrict__ cnt, uint32_t* __restrict__ tmp,
                                                          uint32_t* __restrict__ spare, uint32_t* __restrict__ newlen,
                                                          uint32_t* __restrict__ ticket,
                                                          uint32_t* __restrict__ skewed, uint32_t* __restrict__ nskewed) {
    __shared__ SplitSmem sm;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    for (;;) {
        __syncthreads();
        if (tid == 0) sm.row = atomicAdd(ticket, 1u);
        __syncthreads();
        const uint32_t r = sm.row;
        if (r >= count) break;
        const uint32_t v = list[r];
        const uint32_t L = cnt[v];
        uint32_t* A = tmp + start[v];
        uint32_t* B = spare + start[v];
        const uint32_t nr = min(kSplitMaxRanges, (L + kSplitTarget - 1) / kSplitTarget);
        // ---- the sample, sorted by warp 0; splitters at its nr-quantiles
        if (w == 0) {
            uint32_t x[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) x[e] = A[((uint64_t)((uint32_t)e * 32 + lane) * L) >> 10];
            bitonic_sort<32, 1024>(x, 0, lane);
#pragma unroll
            for (int e = 0; e < 32; ++e) sm.bs.s[(uint32_t)e * 32 + lane] = x[e];
        }
        if (tid < kSplitMaxRanges) {
            sm.rcnt[tid] = 0;
            sm.rcur[tid] = 0;
        }
        __syncthreads();
        if (tid + 1 < nr) sm.spl[tid] = sm.bs.s[((tid + 1) * 1024) / nr];
        if (tid == 0) sm.nsp = nr - 1;
        __syncthreads();
        const uint32_t nsp = sm.nsp;
        // ---- entries per range
        for (uint32_t i0 = 0; i0 < L; i0 += 4 * 256) {
            uint32_t x[4];
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) x[j] = i0 + j * 256 + tid < L ? A[i0 + j * 256 + tid] : 0u;
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) {
                const uint32_t rg = i0 + j * 256 + tid < L ? split_range(sm.spl, nsp, x[j]) : kSplitMaxRanges;
                const uint32_t peers = __match_any_sync(kFullMask, rg);
                if (rg < kSplitMaxRanges && lane == (uint32_t)(__ffs(peers) - 1))
                    atomicAdd(&sm.rcnt[rg], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();
        if (w == 0) {
            const uint32_t c0 = lane < nr ? sm.rcnt[lane] : 0u, c1 = lane + 32 < nr ? sm.rcnt[lane + 32] : 0u;
            const uint32_t i0 = warp_incl_scan(c0), i1 = warp_incl_scan(c1);
            const uint32_t t0 = __shfl_sync(kFullMask, i0, 31);
            const uint32_t tot = t0 + __shfl_sync(kFullMask, i1, 31);
            sm.rstart[lane] = i0 - c0;
            sm.rstart[lane + 32] = t0 + i1 - c1;
            if (lane == 0) sm.rstart[kSplitMaxRanges] = tot;
            const uint32_t big = __ballot_sync(kFullMask, c0 > kBlockRowMax || c1 > kBlockRowMax);
            if (lane == 0) sm.too_big = big != 0;
        }
        __syncthreads();
        if (sm.too_big) {
            if (tid == 0) skewed[atomicAdd(nskewed, 1u)] = v;
            continue;
        }
        // ---- scatter by range (order inside a range does not matter: it is sorted next)
        for (uint32_t i0 = 0; i0 < L; i0 += 4 * 256) {
            uint32_t x[4];
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) x[j] = i0 + j * 256 + tid < L ? A[i0 + j * 256 + tid] : 0u;
#pragma unroll
            for (uint32_t j = 0; j < 4; ++j) {
                const uint32_t rg = i0 + j * 256 + tid < L ? split_range(sm.spl, nsp, x[j]) : kSplitMaxRanges;
                const uint32_t peers = __match_any_sync(kFullMask, rg);
                const uint32_t leader = __ffs(peers) - 1;
                uint32_t base = 0;
                if (rg < kSplitMaxRanges && lane == leader) base = atomicAdd(&sm.rcur[rg], (uint32_t)__popc(peers));
                base = __shfl_sync(kFullMask, base, leader);
                if (rg < kSplitMaxRanges) B[sm.rstart[rg] + base + __popc(peers & lanemask_lt())] = x[j];
            }
        }
        __syncthreads();
        // ---- each range sorted and de-duplicated in place
        for (uint32_t g = 0; g < nr; ++g) {
            const uint32_t c = sm.rcnt[g];
            uint32_t k = 0;
            if (c) k = block_sort_unique<8>(B + sm.rstart[g], c, B + sm.rstart[g], sm.bs);
            if (tid == 0) sm.kept[g] = k;
        }
        __syncthreads();
        if (w == 0) {
            const uint32_t c0 = lane < nr ? sm.kept[lane] : 0u, c1 = lane + 32 < nr ? sm.kept[lane + 32] : 0u;
            const uint32_t i0 = warp_incl_scan(c0), i1 = warp_incl_scan(c1);
            const uint32_t t0 = __shfl_sync(kFullMask, i0, 31);
            const uint32_t tot = t0 + __shfl_sync(kFullMask, i1, 31);
            __syncwarp();
            sm.kept[lane] = i0 - c0;
            sm.kept[lane + 32] = t0 + i1 - c1;
            if (lane == 0) {
                sm.kept[kSplitMaxRanges] = tot;
                newlen[v] = tot;
            }
        }
        __syncthreads();
        // ---- the ranges' unique values back to the row, in order
        for (uint32_t g = 0; g < nr; ++g) {
            const uint32_t k = (g + 1 < nr ? sm.kept[g + 1] : sm.kept[kSplitMaxRanges]) - sm.kept[g];
            const uint32_t* src = B + sm.rstart[g];
            uint32_t* dst = A + sm.kept[g];
            for (uint32_t j = tid; j < k; j += 256) dst[j] = src[j];
        }
    }
}

// ---- skewed giant rows (a splitter range above kBlockRowMax entries): one
// block per row sorts it by an LSD radix sort on 8-bit digits of the
// neighbour ids (as many passes as n's ids need), ping-ponging between the
// row's place in tmp and in spare; the rows come from a list whose length is
// in device memory.  Each
// pass is stable: a digit histogram of the row gives every digit's first
// slot, then the row is walked in order one block-sized tile at a time, and
// a key's slot is its digit's next free slot plus the number of earlier keys
// of the tile with the same digit (warp match within a warp, per-warp digit
// counts across warps).  The sorted row is then de-duplicated into tmp.
constexpr uint32_t kRadixTB = 1024;
constexpr uint32_t kRadixWarps = kRadixTB / 32;

struct RadixSmem {
    uint32_t base[256];                // next free slot of each digit
    uint32_t wcnt[kRadixWarps][256];   // per-warp digit counts of a tile, then their exclusive prefixes
    uint32_t scan_tmp[33];
    uint32_t row, kept;
};

__global__ void __launch_bounds__(kRadixTB) giant_radix_kernel(const uint32_t* __restrict__ list,
                                                               const uint32_t* __restrict__ count_dev,
                                                               const uint64_t* __restrict__ start,
                                                               const uint32_t* __restrict__ cnt,
                                                               uint32_t* __restrict__ tmp,
                                                               uint32_t* __restrict__ spare, uint32_t passes,
                                                               uint32_t* __restrict__ newlen,
                                                               uint32_t* __restrict__ ticket) {
    __shared__ RadixSmem sm;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    for (uint32_t i = tid; i < kRadixWarps * 256; i += kRadixTB) (&sm.wcnt[0][0])[i] = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) sm.row = atomicAdd(ticket, 1u);
        __syncthreads();
        const uint32_t r = sm.row;
        if (r >= *count_dev) break;
        const uint32_t v = list[r];
        const uint32_t len = cnt[v];
        uint32_t* A = tmp + start[v];
        uint32_t* B = spare + start[v];
        for (uint32_t pass = 0; pass < passes; ++pass) {
            const uint32_t shift = 8 * pass;
            if (tid < 256) sm.base[tid] = 0;
            __syncthreads();
            for (uint32_t i0 = 0; i0 < len; i0 += kRadixTB) {
                const uint32_t i = i0 + tid;
                const uint32_t d = i < len ? (A[i] >> shift) & 255u : 256u;
                const uint32_t peers = __match_any_sync(kFullMask, d);
                if (d < 256u && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&sm.base[d], (uint32_t)__popc(peers));
            }
            __syncthreads();
            // exclusive scan of the 256 digit counts: warps 0..7 scan their 32
            // digits, then add the totals of the warps before them
            uint32_t cnt_d = 0, inc_d = 0;
            if (tid < 256) {
                cnt_d = sm.base[tid];
                inc_d = warp_incl_scan(cnt_d);
                if (lane == 31) sm.scan_tmp[w] = inc_d;
            }
            __syncthreads();
            if (tid < 256) {
                uint32_t add = 0;
                for (uint32_t q = 0; q < w; ++q) add += sm.scan_tmp[q];
                sm.base[tid] = add + inc_d - cnt_d;
            }
            __syncthreads();
            for (uint32_t i0 = 0; i0 < len; i0 += kRadixTB) {
                const uint32_t i = i0 + tid;
                const bool valid = i < len;
                const uint32_t key = valid ? A[i] : 0u;
                const uint32_t d = valid ? (key >> shift) & 255u : 256u;
                const uint32_t peers = __match_any_sync(kFullMask, d);
                const uint32_t rank = __popc(peers & lanemask_lt());
                if (valid && lane == (uint32_t)(__ffs(peers) - 1)) sm.wcnt[w][d] = __popc(peers);
                __syncthreads();
                uint32_t col = 0;
                if (tid < 256) {  // per digit: exclusive prefix over the warps, in place
                    for (uint32_t q = 0; q < kRadixWarps; ++q) {
                        const uint32_t c = sm.wcnt[q][tid];
                        sm.wcnt[q][tid] = col;
                        col += c;
                    }
                }
                __syncthreads();
                if (valid) B[sm.base[d] + sm.wcnt[w][d] + rank] = key;
                __syncthreads();
                if (tid < 256) {
                    sm.base[tid] += col;
                    for (uint32_t q = 0; q < kRadixWarps; ++q) sm.wcnt[q][tid] = 0;
                }
                __syncthreads();
            }
            uint32_t* t = A;
            A = B;
            B = t;
        }
        // A holds the sorted row: keep the first of each run of equal ids, in
        // tmp (in place when A is tmp: a tile is read whole before any of its
        // writes, which land at or below the tile's own positions)
        uint32_t* out = tmp + start[v];
        uint32_t kept = 0, prev_last = kPad;
        for (uint32_t i0 = 0; i0 < len; i0 += kRadixTB) {
            const uint32_t i = i0 + tid;
            const uint32_t key = i < len ? A[i] : kPad;
            const uint32_t before = i == i0 ? prev_last : (i - 1 < len ? A[i - 1] : kPad);
            const uint32_t last = A[min(len, i0 + kRadixTB) - 1];
            const bool keep = i < len && key != before;
            uint32_t tot;
            const uint32_t pos = block_excl_scan<uint32_t>(keep ? 1u : 0u, sm.scan_tmp, &tot);
            if (keep) out[kept + pos] = key;
            kept += tot;
            prev_last = last;
            __syncthreads();
        }
        if (tid == 0) newlen[v] = kept;
    }
}

// adj[j] = tmp[start[v] + (j - off[v])] for every position j of row v: the
// output positions are split evenly over the warps (rows of any length).
__global__ void __launch_bounds__(256) copy_rows(uint32_t n, const uint64_t* __restrict__ start,
                                                 const uint32_t* __restrict__ tmp, const uint64_t* __restrict__ off,
                                                 uint32_t* __restrict__ adj) {
    auto pre = [&](uint64_t) { return 0u; };
    auto put = [&](const uint32_t* v, const uint64_t* j, const uint32_t*, uint32_t valid) {
        uint32_t val[kWalkU];
#pragma unroll
        for (uint32_t t = 0; t < kWalkU; ++t)
            if (valid >> t & 1u) val[t] = tmp[start[v[t]] + (j[t] - off[v[t]])];
#pragma unroll
        for (uint32_t t = 0; t < kWalkU; ++t)
            if (valid >> t & 1u) adj[j[t]] = val[t];
    };
    walk_all_entries(off, n, pre, put);
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
    uint32_t *cnt, *tmp, *newlen;
    uint64_t *start, *sums;
    IngestCtl* ctl;
    const uint64_t nt = (uint64_t)n / kScanTile + 2;
    DSG_TRY_CUDA(sc.get(&cnt, (size_t)n + 1));
    DSG_TRY_CUDA(sc.get(&start, (size_t)n + 1));
    DSG_TRY_CUDA(sc.get(&sums, nt));
    DSG_TRY_CUDA(sc.get(&newlen, (size_t)n + 1));
    DSG_TRY_CUDA(sc.get(&ctl, 1));
    DSG_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(IngestCtl), s));
    DSG_TRY_CUDA(cudaMemsetAsync(newlen, 0, ((size_t)n + 1) * 4, s));
    const uint32_t sms = (uint32_t)dev_info().sms;
    // ---- buckets of consecutive owners, from an exact histogram over vertex ranges
    const BucketPlan pl = bucket_plan_for(n);
    const uint64_t cap = 2 * m_raw;  // directed entries at most
    uint32_t *range_cnt, *bucket_v0, *nb, *ticket, *b_pre, *r_pre, *big_list, *fill;
    uint16_t* range_bucket;
    uint64_t *bucket_base, *group_base, *E1, *E2;
    unsigned long long *bucket_fill, *group_fill, *maxb;
    PartPlan* pp;
    DSG_TRY_CUDA(sc.get(&range_cnt, pl.nranges ? pl.nranges : 1));
    DSG_TRY_CUDA(sc.get(&range_bucket, pl.nranges ? pl.nranges : 1));
    // buckets never outnumber the ranges (each starts at a range)
    const size_t fcap = std::min<size_t>(kBucketsMax, (size_t)pl.nranges + 1);
    const size_t gcap = (fcap + kGroupFine - 1) / kGroupFine;
    DSG_TRY_CUDA(sc.get(&bucket_v0, fcap + 1));
    DSG_TRY_CUDA(sc.get(&bucket_base, fcap + 1));
    DSG_TRY_CUDA(sc.get(&bucket_fill, fcap));
    DSG_TRY_CUDA(sc.get(&group_base, gcap + 1));
    DSG_TRY_CUDA(sc.get(&group_fill, gcap));
    DSG_TRY_CUDA(sc.get(&b_pre, gcap + 1));
    DSG_TRY_CUDA(sc.get(&r_pre, fcap + 1));
    DSG_TRY_CUDA(sc.get(&big_list, fcap));
    DSG_TRY_CUDA(sc.get(&pp, 1));
    DSG_TRY_CUDA(sc.get(&nb, 2));
    DSG_TRY_CUDA(sc.get(&maxb, 1));
    ticket = nb + 1;
    DSG_TRY_CUDA(sc.get(&E1, cap ? cap : 1));
    DSG_TRY_CUDA(sc.get(&E2, cap ? cap : 1));
    DSG_TRY_CUDA(sc.get(&tmp, cap ? cap : 1));
    DSG_TRY_CUDA(sc.get(&fill, (size_t)n + 1));
    DSG_TRY_CUDA(cudaMemsetAsync(range_cnt, 0, (size_t)(pl.nranges ? pl.nranges : 1) * 4, s));
    DSG_TRY_CUDA(cudaMemsetAsync(bucket_fill, 0, fcap * 8, s));
    DSG_TRY_CUDA(cudaMemsetAsync(group_fill, 0, gcap * 8, s));
    DSG_TRY_CUDA(cudaMemsetAsync(nb, 0, 2 * sizeof(uint32_t), s));
    DSG_TRY_CUDA(cudaMemsetAsync(maxb, 0, sizeof(unsigned long long), s));
    DSG_TRY_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)n + 1) * 4, s));  // big buckets add their counts into it
    const size_t hist_smem = (size_t)pl.nranges * 4;
    const size_t part_smem = sizeof(PartSmem) + (((size_t)pl.nranges * 2 + 15) & ~size_t(15));
    const size_t rows_smem = (size_t)kSpanMax * 4;
    {
        static bool smem_set[64] = {};  // the attributes are per function and device, set once (idempotent)
        if (!smem_set[dev & 63]) {
            const int part_max = (int)(sizeof(PartSmem) + (size_t)kRangesMax * 2);
            DSG_TRY_CUDA(cudaFuncSetAttribute(range_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(kRangesMax * 4)));
            DSG_TRY_CUDA(cudaFuncSetAttribute(part_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, part_max));
            DSG_TRY_CUDA(cudaFuncSetAttribute(part_groups_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              part_max));
            DSG_TRY_CUDA(cudaFuncSetAttribute(big_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)rows_smem));
            DSG_TRY_CUDA(cudaFuncSetAttribute(bucket_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)rows_smem));
            smem_set[dev & 63] = true;
        }
    }
    if (m_raw) {
        const uint32_t g = (uint32_t)std::min<uint64_t>((m_raw + 65535) / 65536, sms);
        LaunchScope ls_("ingest_range_hist", s);
        range_hist_kernel<<<g, 1024, hist_smem, s>>>(n, m_raw, src, dst, pl, range_cnt, ctl);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    {
        LaunchScope ls_("ingest_bucket_plan", s);
        bucket_plan_kernel<<<1, 1024, 0, s>>>(n, range_cnt, pl, range_bucket, bucket_v0, bucket_base, start, nb,
                                              maxb);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    {
        LaunchScope ls_("ingest_part_plan", s);
        part_plan_kernel<<<1, 1024, 0, s>>>(nb, bucket_base, group_base, b_pre, r_pre, big_list, pp);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    int per_sm_rows = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_rows, bucket_rows_kernel, kRowsTB, rows_smem) !=
            cudaSuccess || per_sm_rows < 1)
        per_sm_rows = 1;
    if (m_raw) {
        {
            LaunchScope ls_("ingest_part_pairs", s);
            part_pairs_kernel<<<2 * sms, kPartTB, part_smem, s>>>(n, m_raw, src, dst, pl, range_bucket, pp, group_base,
                                                              group_fill, E1);
        }
        DSG_TRY_CUDA(cudaGetLastError());
        {
            LaunchScope ls_("ingest_part_groups", s);
            part_groups_kernel<<<2 * sms, kPartTB, part_smem, s>>>(pl, range_bucket, nb, pp, group_base, b_pre,
                                                               bucket_base, bucket_fill, E1, E2);
        }
        DSG_TRY_CUDA(cudaGetLastError());
        {
            LaunchScope ls_("ingest_big_count", s);
            big_count_kernel<<<sms * (uint32_t)per_sm_rows, kRowsTB, rows_smem, s>>>(nb, pp, r_pre, bucket_v0,
                                                                                    bucket_base, E2, cnt);
        }
        DSG_TRY_CUDA(cudaGetLastError());
        {
            LaunchScope ls_("ingest_big_starts", s);
            big_starts_kernel<<<sms, kRowsTB, 0, s>>>(pp, big_list, bucket_v0, bucket_base, cnt, start, fill, ctl);
        }
        DSG_TRY_CUDA(cudaGetLastError());
    }
    {
        LaunchScope ls_("ingest_bucket_rows", s);
        bucket_rows_kernel<<<sms * (uint32_t)per_sm_rows, kRowsTB, rows_smem, s>>>(
            nb, pp, r_pre, bucket_v0, bucket_base, E2, cnt, start, fill, tmp, ticket, ctl);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    IngestCtl hc;
    uint64_t total = 0;
    DSG_TRY_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaMemcpyAsync(&total, start + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    DSG_TRY_CUDA(cudaStreamSynchronize(s));
    if (hc.err & ERR_RANGE) {
        set_error("graph_from_edges: a vertex id is >= n");
        return DSG_EINVAL;
    }
    ClassLists lists;
    uint32_t nlist = 0;
    for (int c = 0; c < kClasses; ++c) {
        lists.base[c] = nlist;
        nlist += hc.cls_count[c];
    }
    DSG_TRY_CUDA(sc.get(&lists.rows, nlist ? nlist : 1));
    {
        LaunchScope ls_("ingest_sort_small_rows", s);
        sort_small_rows<<<grid_for((uint64_t)n, 256), 256, 0, s>>>(n, start, cnt, tmp, newlen, lists, ctl);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    auto warp_grid = [&](uint32_t rows) { return (uint32_t)std::min<uint64_t>((rows + 7) / 8, (uint64_t)sms * 16); };
    if (hc.cls_count[0]) { LaunchScope ls_("ingest_sort_warp_rows", s); sort_warp_rows<2><<<warp_grid(hc.cls_count[0]), 256, 0, s>>>(lists.rows + lists.base[0], hc.cls_count[0], start, cnt, tmp, newlen); }
    if (hc.cls_count[1]) { LaunchScope ls_("ingest_sort_warp_rows", s); sort_warp_rows<4><<<warp_grid(hc.cls_count[1]), 256, 0, s>>>(lists.rows + lists.base[1], hc.cls_count[1], start, cnt, tmp, newlen); }
    if (hc.cls_count[2]) { LaunchScope ls_("ingest_sort_warp_rows", s); sort_warp_rows<8><<<warp_grid(hc.cls_count[2]), 256, 0, s>>>(lists.rows + lists.base[2], hc.cls_count[2], start, cnt, tmp, newlen); }
    if (hc.cls_count[3]) { LaunchScope ls_("ingest_sort_warp_rows", s); sort_warp_rows<16><<<warp_grid(hc.cls_count[3]), 256, 0, s>>>(lists.rows + lists.base[3], hc.cls_count[3], start, cnt, tmp, newlen); }
    if (hc.cls_count[4]) { LaunchScope ls_("ingest_sort_warp_rows", s); sort_warp_rows<32><<<warp_grid(hc.cls_count[4]), 256, 0, s>>>(lists.rows + lists.base[4], hc.cls_count[4], start, cnt, tmp, newlen); }
    DSG_TRY_CUDA(cudaGetLastError());
    // block rows: 2, 4 or 8 warps (each sorting 1024 values in registers) per row
    if (hc.cls_count[5]) {
        LaunchScope ls_("ingest_sort_block_rows", s);
        uint32_t g = (uint32_t)std::min<uint64_t>(hc.cls_count[5], (uint64_t)sms * 16);
        sort_block_rows<2><<<g, 64, 0, s>>>(lists.rows + lists.base[5], hc.cls_count[5], start, cnt, tmp, newlen);
    }
    if (hc.cls_count[6]) {
        LaunchScope ls_("ingest_sort_block_rows", s);
        uint32_t g = (uint32_t)std::min<uint64_t>(hc.cls_count[6], (uint64_t)sms * 8);
        sort_block_rows<4><<<g, 128, 0, s>>>(lists.rows + lists.base[6], hc.cls_count[6], start, cnt, tmp, newlen);
    }
    if (hc.cls_count[7]) {
        LaunchScope ls_("ingest_sort_block_rows", s);
        uint32_t g = (uint32_t)std::min<uint64_t>(hc.cls_count[7], (uint64_t)sms * 4);
        sort_block_rows<8><<<g, 256, 0, s>>>(lists.rows + lists.base[7], hc.cls_count[7], start, cnt, tmp, newlen);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    if (hc.cls_count[kGiant]) {
        const uint32_t ng = hc.cls_count[kGiant];
        const uint32_t* glist = lists.rows + lists.base[kGiant];
        uint32_t nbits = 1;
        while (nbits < 32 && ((uint64_t)n - 1) >> nbits) ++nbits;
        const uint32_t passes = (nbits + 7) / 8;
        // the bucket entries are no longer needed: their space is the spare buffer of both sorts
        uint32_t* spare = reinterpret_cast<uint32_t*>(E1);
        uint32_t *gticket, *skewed;  // gticket[0]: split rows taken, [1]: skewed rows listed, [2]: radix rows taken
        DSG_TRY_CUDA(sc.get(&gticket, 3));
        DSG_TRY_CUDA(sc.get(&skewed, ng));
        DSG_TRY_CUDA(cudaMemsetAsync(gticket, 0, 3 * sizeof(uint32_t), s));
        {
            LaunchScope ls_("ingest_giant_rows", s);
            giant_split_kernel<<<std::min<uint32_t>(ng, 2 * sms), 256, 0, s>>>(glist, ng, start, cnt, tmp, spare,
                                                                             newlen, gticket, skewed, gticket + 1);
        }
        DSG_TRY_CUDA(cudaGetLastError());
        {
            LaunchScope ls_("ingest_giant_skewed", s);
            giant_radix_kernel<<<std::min<uint32_t>(ng, sms), kRadixTB, 0, s>>>(skewed, gticket + 1, start, cnt, tmp,
                                                                              spare, passes, newlen, gticket + 2);
        }
    }
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
        if (total2) {
            // one resident wave: every warp walks an equal share of the positions
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, copy_rows, 256, 0) != cudaSuccess || per_sm < 1)
                per_sm = 1;
            LaunchScope ls_("ingest_copy_rows", s);
            copy_rows<<<(uint32_t)dev_info().sms * (uint32_t)per_sm, 256, 0, s>>>(n, start, tmp, g->off, g->adj);
        }
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
