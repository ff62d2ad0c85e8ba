// CSR ingest: raw undirected pairs -> canonical CSR (Def. 1: a simple graph,
// E a set of edges between distinct vertices).
//
//   1. count   every non-loop pair adds one to the row of each endpoint
//              (frequent endpoints, found from a sample of the pairs, are
//              counted per block in shared memory)
//   2. scan    row starts of the (still repeated) entries
//   3. scatter each pair is written into both rows (a frequent endpoint's
//              entries from one block go to a range reserved for that block)
//   4. sort    each row sorted and de-duplicated in place; rows are binned by
//              length: <= 32 entries one warp, one value per lane; <= 1024
//              one warp holding up to 32 values per lane (register bitonic
//              network, no shared memory); <= 8192 one block (each warp sorts
//              1024 values in registers, cross-warp merge steps go through
//              shared memory); longer ("giant") rows are split by value
//              window and each window is de-duplicated and ordered through a
//              shared-memory bitmap
//   5. scan    final row lengths -> off
//   6. copy    unique entries into adj
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
constexpr uint32_t kWinBits = 13;        // giant rows: value windows of 8192 ids
constexpr uint32_t kWin = 1u << kWinBits;
constexpr uint32_t kWinWords = kWin / 32;
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

// ----------------------------------------------------------- count / scatter

// ------------------------------------------------ hot vertices (count, scatter)
// A vertex that is an endpoint of a large share of the raw pairs (a hub)
// would take one global atomic per pair in count and scatter, all on one
// address.  A sample of the pairs names such vertices; count and scatter
// then combine their increments per block in shared memory, and each block
// writes a hub's entries into a range of the hub's row reserved for it (the
// blocks' counts are prefix-summed per hub between the two passes).  Which
// vertices are hot only changes speed, never the result.
constexpr uint32_t kHotMax = 1024;          // hot vertices at most
constexpr uint32_t kHotSlots = 2048;        // shared-memory hash of the hot ids
constexpr uint32_t kSamplePairs = 32768;    // pairs sampled to find them
constexpr uint32_t kSampleSlots = 8192;     // shared-memory hash of the sampled endpoints
constexpr uint32_t kHotMinHits = 4;         // sample hits that make a vertex hot
constexpr uint32_t kHotEmpty = 0xffffffffu;
constexpr uint64_t kHotPassMinPairs = 1ull << 22;  // inputs with fewer pairs skip the pass

__device__ __forceinline__ uint32_t hot_hash(uint32_t x) { return (x * 0x9E3779B1u) >> 21; }  // 11 bits

__host__ __device__ __forceinline__ uint64_t sample_stride(uint64_t m_raw) {
    return m_raw > kSamplePairs ? m_raw / kSamplePairs : 1;
}
__host__ __device__ __forceinline__ uint64_t sample_take(uint64_t m_raw) {
    return m_raw < kSamplePairs ? m_raw : kSamplePairs;
}

// Gather every stride-th pair into one contiguous buffer, a pair per thread
// over many SMs (one block fetching 32 K scattered pairs is bound by its own
// outstanding loads).
__global__ void __launch_bounds__(256) hot_gather(uint64_t m_raw, const uint32_t* __restrict__ src,
                                                  const uint32_t* __restrict__ dst, uint2* __restrict__ sample) {
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < sample_take(m_raw)) {
        const uint64_t at = k * sample_stride(m_raw);
        sample[k] = make_uint2(src[at], dst[at]);
    }
}

// Endpoint frequencies over the gathered sample, split over kHotParts blocks
// by a hash of the id (every block reads the whole sample and counts only its
// own part, so no id is counted twice and the hashing work is shared).  Each
// block lists its ids with at least kHotMinHits hits as (id, hits capped at
// 255) and adds them to a histogram of the hit counts.
constexpr uint32_t kHotParts = 8;

__device__ __forceinline__ uint32_t hot_part(uint32_t x) { return (x * 0x9E3779B1u) >> 29; }  // 3 bits
__device__ __forceinline__ uint32_t sample_slot(uint32_t x) { return (x * 0x85EBCA6Bu) >> 19; }  // 13 bits

__global__ void __launch_bounds__(1024) hot_sample(uint32_t n, uint64_t m_raw, const uint2* __restrict__ sample,
                                                   uint2* __restrict__ cand, uint32_t* __restrict__ cand_n,
                                                   uint32_t* __restrict__ hist) {
    extern __shared__ uint32_t sample_smem[];  // kSampleSlots keys, then kSampleSlots counts
    uint32_t* key = sample_smem;
    uint32_t* cnt = sample_smem + kSampleSlots;
    __shared__ uint32_t lhist[256];
    __shared__ uint32_t nq, base, fill;
    for (uint32_t i = threadIdx.x; i < kSampleSlots; i += blockDim.x) {
        key[i] = kHotEmpty;
        cnt[i] = 0;
    }
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) lhist[i] = 0;
    if (threadIdx.x == 0) nq = fill = 0;
    __syncthreads();
    const uint64_t take = sample_take(m_raw);
    constexpr uint32_t kU = 8;  // pairs loaded per thread before any is counted
    for (uint64_t k0 = threadIdx.x; k0 < take; k0 += (uint64_t)blockDim.x * kU) {
        uint32_t e[2 * kU];
#pragma unroll
        for (uint32_t t = 0; t < kU; ++t) {
            const uint64_t k = k0 + (uint64_t)t * blockDim.x;
            e[2 * t] = e[2 * t + 1] = kHotEmpty;
            if (k < take) {
                const uint2 p = sample[k];
                e[2 * t] = p.x;
                e[2 * t + 1] = p.y;
            }
        }
#pragma unroll
        for (uint32_t t = 0; t < 2 * kU; ++t) {
            const uint32_t x = e[t];
            if (x >= n || e[t ^ 1u] == x || hot_part(x) != blockIdx.x) continue;  // padding, a loop, another part
            uint32_t h = sample_slot(x);
            for (uint32_t probe = 0; probe < 8; ++probe, h = (h + 1) & (kSampleSlots - 1)) {
                const uint32_t cur = key[h];
                const uint32_t prev = cur == x ? x : (cur == kHotEmpty ? atomicCAS(&key[h], kHotEmpty, x) : cur);
                if (prev == kHotEmpty || prev == x) {
                    atomicAdd(&cnt[h], 1u);
                    break;
                }
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kSampleSlots; i += blockDim.x)
        if (key[i] != kHotEmpty && cnt[i] >= kHotMinHits) {
            atomicAdd(&lhist[min(cnt[i], 255u)], 1u);
            atomicAdd(&nq, 1u);
        }
    __syncthreads();
    if (threadIdx.x == 0) base = nq ? atomicAdd(cand_n, nq) : 0u;
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x)
        if (lhist[i]) atomicAdd(&hist[i], lhist[i]);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kSampleSlots; i += blockDim.x)
        if (key[i] != kHotEmpty && cnt[i] >= kHotMinHits) cand[base + atomicAdd(&fill, 1u)] = make_uint2(key[i], min(cnt[i], 255u));
}

// Keep the most frequent candidates: the histogram of their hit counts gives
// the count above which all fit in kHotMax, and the boundary count fills the rest.
__global__ void __launch_bounds__(1024) hot_select(const uint2* __restrict__ cand, const uint32_t* __restrict__ cand_n,
                                                   const uint32_t* __restrict__ hist, uint32_t* __restrict__ hot_ids,
                                                   uint32_t* __restrict__ hot_n) {
    __shared__ uint32_t cut, room, extra, nsel;
    if (threadIdx.x == 0) {
        uint32_t acc = 0, b = 255;
        while (b >= kHotMinHits && acc + hist[b] <= kHotMax) acc += hist[b--];
        cut = b;                // buckets above cut are taken whole
        room = kHotMax - acc;  // slots left for bucket cut
        extra = 0;
        nsel = 0;
    }
    __syncthreads();
    const uint32_t nc = *cand_n;
    for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
        const uint2 c = cand[i];
        bool take = c.y > cut;
        if (!take && c.y == cut) take = atomicAdd(&extra, 1u) < room;
        if (take) {
            const uint32_t at = atomicAdd(&nsel, 1u);
            if (at < kHotMax) hot_ids[at] = c.x;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *hot_n = min(nsel, kHotMax);
}

// Shared-memory table of the hot ids: slot -> (id, index in the hot list).
struct HotTable {
    uint32_t key[kHotSlots];
    uint16_t idx[kHotSlots];
    uint32_t local[kHotMax];  // this block's count or cursor per hot vertex
};

__device__ __forceinline__ void hot_build(HotTable& t, const uint32_t* hot_ids, uint32_t hot_n) {
    for (uint32_t i = threadIdx.x; i < kHotSlots; i += blockDim.x) t.key[i] = kHotEmpty;
    for (uint32_t i = threadIdx.x; i < kHotMax; i += blockDim.x) t.local[i] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < hot_n; i += blockDim.x) {
        const uint32_t x = hot_ids[i];
        uint32_t h = hot_hash(x);
        while (true) {
            if (atomicCAS(&t.key[h], kHotEmpty, x) == kHotEmpty) {
                t.idx[h] = (uint16_t)i;
                break;
            }
            h = (h + 1) & (kHotSlots - 1);
        }
    }
    __syncthreads();
}

// index of x in the hot list, or -1
__device__ __forceinline__ int hot_find(const HotTable& t, uint32_t x) {
    uint32_t h = hot_hash(x);
    while (true) {
        const uint32_t k = t.key[h];
        if (k == x) return t.idx[h];
        if (k == kHotEmpty) return -1;
        h = (h + 1) & (kHotSlots - 1);
    }
}

// count: one per endpoint of every non-loop pair; hot endpoints are counted
// in shared memory and also recorded per block (blk[block * kHotMax + h]).
__global__ void __launch_bounds__(256) count_kernel(uint32_t n, uint64_t m_raw, const uint32_t* __restrict__ src,
                                                    const uint32_t* __restrict__ dst, uint32_t* __restrict__ cnt,
                                                    const uint32_t* __restrict__ hot_ids,
                                                    const uint32_t* __restrict__ hot_n_p, uint32_t* __restrict__ blk,
                                                    IngestCtl* ctl) {
    __shared__ HotTable t;
    const uint32_t hot_n = *hot_n_p;
    hot_build(t, hot_ids, hot_n);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_raw;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = src[i], v = dst[i];
        if (u >= n || v >= n) {
            atomicOr(&ctl->err, ERR_RANGE);
            continue;
        }
        if (u == v) continue;
        int hu = hot_find(t, u), hv = hot_find(t, v);
        if (hu >= 0) atomicAdd(&t.local[hu], 1u); else atomicAdd(&cnt[u], 1u);
        if (hv >= 0) atomicAdd(&t.local[hv], 1u); else atomicAdd(&cnt[v], 1u);
    }
    __syncthreads();
    for (uint32_t h = threadIdx.x; h < hot_n; h += blockDim.x) {
        const uint32_t c = t.local[h];
        blk[(uint64_t)blockIdx.x * kHotMax + h] = c;
        if (c) atomicAdd(&cnt[hot_ids[h]], c);
    }
}

// per hot vertex h: exclusive prefix of the blocks' counts -> each block's
// first slot in the hub's row
__global__ void __launch_bounds__(256) hot_block_bases(const uint32_t* __restrict__ hot_n_p, uint32_t nblk,
                                                       uint32_t* __restrict__ blk) {
    __shared__ uint32_t tmp[33];
    const uint32_t h = blockIdx.x;
    if (h >= *hot_n_p) return;
    uint32_t carry = 0;
    for (uint32_t b0 = 0; b0 < nblk; b0 += blockDim.x) {
        const uint32_t b = b0 + threadIdx.x;
        const uint32_t c = b < nblk ? blk[(uint64_t)b * kHotMax + h] : 0u;
        uint32_t tot;
        const uint32_t pre = block_excl_scan<uint32_t>(c, tmp, &tot);
        if (b < nblk) blk[(uint64_t)b * kHotMax + h] = carry + pre;
        carry += tot;
    }
}

// scatter: each pair into both rows; hot rows at the block's reserved range
// (same grid and pair-to-block assignment as count_kernel).
__global__ void __launch_bounds__(256) scatter_kernel(uint32_t n, uint64_t m_raw, const uint32_t* __restrict__ src,
                                                      const uint32_t* __restrict__ dst,
                                                      const uint64_t* __restrict__ start, uint32_t* __restrict__ fill,
                                                      const uint32_t* __restrict__ hot_ids,
                                                      const uint32_t* __restrict__ hot_n_p,
                                                      const uint32_t* __restrict__ blk, uint32_t* __restrict__ tmp) {
    __shared__ HotTable t;
    const uint32_t hot_n = *hot_n_p;
    hot_build(t, hot_ids, hot_n);
    const uint32_t* myblk = blk + (uint64_t)blockIdx.x * kHotMax;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_raw;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = src[i], v = dst[i];
        if (u >= n || v >= n || u == v) continue;
        const int hu = hot_find(t, u), hv = hot_find(t, v);
        const uint64_t pu = hu >= 0 ? start[u] + myblk[hu] + atomicAdd(&t.local[hu], 1u)
                                    : start[u] + atomicAdd(&fill[u], 1u);
        const uint64_t pv = hv >= 0 ? start[v] + myblk[hv] + atomicAdd(&t.local[hv], 1u)
                                    : start[v] + atomicAdd(&fill[v], 1u);
        tmp[pu] = v;
        tmp[pv] = u;
    }
}

// ----------------------------------------------------------- row sort

__global__ void classify_count(uint32_t n, const uint32_t* __restrict__ cnt, IngestCtl* ctl) {
    __shared__ uint32_t c[kClasses];
    __shared__ unsigned long long giant;
    if (threadIdx.x < kClasses) c[threadIdx.x] = 0;
    if (threadIdx.x == 0) giant = 0;
    __syncthreads();
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t len = cnt[v];
        int k = row_class(len);
        if (k >= 0) atomicAdd(&c[k], 1u);
        if (k == kGiant) atomicAdd(&giant, (unsigned long long)len);
    }
    __syncthreads();
    if (threadIdx.x < kClasses && c[threadIdx.x]) atomicAdd(&ctl->cls_count[threadIdx.x], c[threadIdx.x]);
    if (threadIdx.x == 0 && giant) atomicAdd(&ctl->giant_entries, giant);
}

struct ClassLists {
    uint32_t* rows;             // all class lists, back to back
    uint32_t base[kClasses];    // start of each class in rows
};

// Rows of <= 32 entries: one warp per row, one value per lane, bitonic
// network over shuffles, dedup by comparing with the previous lane.  Longer
// rows are appended to their class list (warp-aggregated per class).
__global__ void sort_small_rows(uint32_t n, const uint64_t* __restrict__ start, const uint32_t* __restrict__ cnt,
                                uint32_t* __restrict__ tmp, uint32_t* __restrict__ newlen, ClassLists lists,
                                IngestCtl* ctl) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // one warp walks 32 rows at a time for the class append, then sorts its small rows
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
        uint32_t small = __ballot_sync(kFullMask, vl < n && cls < 0);
        while (small) {
            uint32_t src_lane = __ffs(small) - 1;
            small &= small - 1;
            uint64_t v = v0 + src_lane;
            uint32_t len = __shfl_sync(kFullMask, mylen, src_lane);
            if (len == 0) {
                if (lane == 0) newlen[v] = 0;
                continue;
            }
            uint64_t b = start[v];
            uint32_t x = lane < len ? tmp[b + lane] : kPad;
#pragma unroll
            for (uint32_t k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    uint32_t y = __shfl_xor_sync(kFullMask, x, j);
                    bool up = (lane & k) == 0;
                    bool lower = (lane & j) == 0;
                    // lower lane keeps min when ascending, max when descending
                    x = (lower == up) ? min(x, y) : max(x, y);
                }
            }
            uint32_t prev = __shfl_up_sync(kFullMask, x, 1);
            bool keep = x != kPad && (lane == 0 || x != prev);
            uint32_t bal = __ballot_sync(kFullMask, keep);
            if (keep) tmp[b + __popc(bal & lanemask_lt())] = x;
            if (lane == 0) newlen[v] = __popc(bal);
        }
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

// Rows of 1025..8192 entries: one block of 8 warps per row.  Each active warp
// sorts 1024 values in registers; merges with block size 2048..p2 run their
// cross-warp steps (distance >= 1024) through shared memory and the rest in
// registers.
template <uint32_t kBlockWarps>
__global__ void __launch_bounds__(kBlockWarps * 32) sort_block_rows(const uint32_t* __restrict__ list,
                                                                    uint32_t count,
                                                                    const uint64_t* __restrict__ start,
                                                                    const uint32_t* __restrict__ cnt,
                                                                    uint32_t* __restrict__ tmp,
                                                                    uint32_t* __restrict__ newlen) {
    __shared__ uint32_t s[kBlockWarps * 1024];
    __shared__ uint32_t wlast[kBlockWarps];
    __shared__ uint32_t wcount[kBlockWarps];
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t base = w * 1024;
    for (uint32_t r = blockIdx.x; r < count; r += gridDim.x) {
        uint32_t v = list[r];
        uint32_t len = cnt[v];
        uint64_t b = start[v];
        uint32_t p2 = 2048;
        while (p2 < len) p2 <<= 1;
        const bool active = base < p2;
        uint32_t x[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            uint32_t i = base + (uint32_t)e * 32 + lane;
            x[e] = (active && i < len) ? tmp[b + i] : kPad;
        }
        if (active) bitonic_sort<32, 1024>(x, base, lane);
        for (uint32_t k = 2048; k <= p2; k <<= 1) {
            for (uint32_t j = k >> 1; j >= 1024; j >>= 1) {
                if (active) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) s[base + (uint32_t)e * 32 + lane] = x[e];
                }
                __syncthreads();
                if (active) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        uint32_t i = base + (uint32_t)e * 32 + lane;
                        uint32_t y = s[i ^ j];
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
        if (lane == 31) wlast[w] = x[31];
        __syncthreads();
        uint32_t prev_in = (w == 0 || !active) ? kPad : wlast[w - 1];
        // count first, then write at the prefix of the warps' counts
        uint32_t mine = 0;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            uint32_t up = __shfl_up_sync(kFullMask, x[e], 1);
            uint32_t last_prev = e == 0 ? prev_in : __shfl_sync(kFullMask, x[e > 0 ? e - 1 : 0], 31);
            uint32_t prev = lane == 0 ? last_prev : up;
            mine += __popc(__ballot_sync(kFullMask, x[e] != kPad && x[e] != prev));
        }
        if (lane == 0) wcount[w] = active ? mine : 0;
        __syncthreads();
        uint32_t off = 0, total = 0;
        for (uint32_t q = 0; q < kBlockWarps; ++q) {
            if (q < w) off += wcount[q];
            total += wcount[q];
        }
        if (active) warp_unique_write<32>(x, prev_in, lane, tmp + b + off);
        if (threadIdx.x == 0) newlen[v] = total;
        __syncthreads();
    }
}

// ---- giant rows (> 8192 entries): partition each row by value window of
// kWin ids (a counting sort on value >> kWinBits), then de-duplicate and order
// each window with a kWin-bit bitmap in shared memory.

// window histogram; grid.y walks giant rows, grid.x chunks of a row
__global__ void giant_hist(const uint32_t* __restrict__ list, uint32_t count, const uint64_t* __restrict__ start,
                           const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ tmp, uint32_t nwin,
                           uint32_t* __restrict__ hist) {
    extern __shared__ uint32_t sh[];
    const bool use_smem = nwin <= 4096;
    for (uint32_t r = blockIdx.y; r < count; r += gridDim.y) {
        uint32_t v = list[r];
        uint32_t len = cnt[v];
        uint64_t b = start[v];
        uint32_t* h = hist + (uint64_t)r * nwin;
        if (use_smem) {
            for (uint32_t i = threadIdx.x; i < nwin; i += blockDim.x) sh[i] = 0;
            __syncthreads();
        }
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
            uint32_t wv = tmp[b + i] >> kWinBits;
            if (use_smem) atomicAdd(&sh[wv], 1u);
            else atomicAdd(&h[wv], 1u);
        }
        if (use_smem) {
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < nwin; i += blockDim.x)
                if (sh[i]) atomicAdd(&h[i], sh[i]);
            __syncthreads();
        }
    }
}

__global__ void giant_scatter(const uint32_t* __restrict__ list, uint32_t count, const uint64_t* __restrict__ start,
                              const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ tmp, uint32_t nwin,
                              const uint64_t* __restrict__ hoff, uint32_t* __restrict__ cursor,
                              uint32_t* __restrict__ spare) {
    for (uint32_t r = blockIdx.y; r < count; r += gridDim.y) {
        uint32_t v = list[r];
        uint32_t len = cnt[v];
        uint64_t b = start[v];
        const uint64_t* ho = hoff + (uint64_t)r * nwin;
        uint32_t* cur = cursor + (uint64_t)r * nwin;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
            uint32_t x = tmp[b + i];
            uint32_t wv = x >> kWinBits;
            spare[b + (ho[wv] - ho[0]) + atomicAdd(&cur[wv], 1u)] = x;
        }
    }
}

// one warp per (row, window); EMIT = false counts the window's distinct
// values into ucnt, EMIT = true writes them in order at their row position
template <bool EMIT>
__global__ void __launch_bounds__(256) giant_windows(const uint32_t* __restrict__ list, uint32_t count,
                                                     const uint64_t* __restrict__ start, uint32_t nwin,
                                                     const uint32_t* __restrict__ hist,
                                                     const uint64_t* __restrict__ hoff,
                                                     const uint32_t* __restrict__ spare, uint32_t* __restrict__ ucnt,
                                                     const uint64_t* __restrict__ uoff, uint32_t* __restrict__ tmp,
                                                     uint32_t* __restrict__ newlen) {
    __shared__ uint32_t bm[8][kWinWords];
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint64_t total = (uint64_t)count * nwin;
    for (uint64_t it = (uint64_t)blockIdx.x * 8 + w; it < total; it += (uint64_t)gridDim.x * 8) {
        uint32_t r = (uint32_t)(it / nwin), wi = (uint32_t)(it % nwin);
        uint32_t v = list[r];
        uint64_t b = start[v];
        const uint64_t* ho = hoff + (uint64_t)r * nwin;
        if (EMIT && wi == 0 && lane == 0) newlen[v] = (uint32_t)(uoff[(uint64_t)r * nwin + nwin] - uoff[(uint64_t)r * nwin]);
        uint32_t h = hist[it];
        if (h == 0) {
            if (!EMIT && lane == 0) ucnt[it] = 0;  // every window's count feeds the scan
            continue;
        }
#pragma unroll
        for (uint32_t q = 0; q < kWinWords / 32; ++q) bm[w][q * 32 + lane] = 0;
        __syncwarp();
        uint64_t seg = b + (ho[wi] - ho[0]);
        for (uint32_t i = lane; i < h; i += 32) {
            uint32_t x = spare[seg + i] & (kWin - 1);
            atomicOr(&bm[w][x >> 5], 1u << (x & 31));
        }
        __syncwarp();
        // lane owns words [lane * 8, lane * 8 + 8)
        uint32_t words[kWinWords / 32], c = 0;
#pragma unroll
        for (uint32_t q = 0; q < kWinWords / 32; ++q) {
            words[q] = bm[w][lane * (kWinWords / 32) + q];
            c += __popc(words[q]);
        }
        if (!EMIT) {
            uint32_t tot = warp_sum(c);
            if (lane == 0) ucnt[it] = tot;
        } else {
            uint32_t inc = warp_incl_scan(c);
            uint64_t pos = b + (uoff[it] - uoff[(uint64_t)r * nwin]) + (inc - c);
            uint32_t vbase = wi * kWin + lane * (kWinWords / 32) * 32;
#pragma unroll
            for (uint32_t q = 0; q < kWinWords / 32; ++q) {
                uint32_t m = words[q];
                while (m) {
                    uint32_t bit = __ffs(m) - 1;
                    m &= m - 1;
                    tmp[pos++] = vbase + q * 32 + bit;
                }
            }
        }
        __syncwarp();
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
    DSG_TRY_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)n + 1) * 4, s));
    DSG_TRY_CUDA(cudaMemsetAsync(ctl, 0, sizeof(IngestCtl), s));
    // count and scatter run on the same grid, so each block meets the same pairs
    const uint32_t pair_grid = (uint32_t)std::min<uint64_t>((m_raw + 255) / 256 + 1, (uint64_t)dev_info().sms * 8);
    // small inputs skip the hot-endpoint pass: no address is hit often enough
    // to matter, and its fixed cost would dominate
    const bool hot_pass = m_raw >= kHotPassMinPairs;
    uint32_t *hot_ids, *hot_n, *blk;
    DSG_TRY_CUDA(sc.get(&hot_ids, kHotMax));
    DSG_TRY_CUDA(sc.get(&hot_n, 1));
    DSG_TRY_CUDA(sc.get(&blk, hot_pass ? (size_t)pair_grid * kHotMax : 1));
    if (hot_pass) {
        const size_t smem = 2 * kSampleSlots * sizeof(uint32_t);
        static bool smem_set[64] = {};  // the attribute is per function and device, set once (idempotent)
        if (!smem_set[dev & 63]) {
            DSG_TRY_CUDA(cudaFuncSetAttribute(hot_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            smem_set[dev & 63] = true;
        }
        uint2* sample;
        DSG_TRY_CUDA(sc.get(&sample, (size_t)sample_take(m_raw)));
        {
            LaunchScope ls_("ingest_hot_gather", s);
            hot_gather<<<(uint32_t)((sample_take(m_raw) + 255) / 256), 256, 0, s>>>(m_raw, src, dst, sample);
        }
        uint2* cand;         // (id, hits) of the frequent sampled endpoints, every part's
        uint32_t* cand_cnt;  // [0, 256) histogram of their hits, [256] their number
        DSG_TRY_CUDA(sc.get(&cand, (size_t)kHotParts * kSampleSlots));
        DSG_TRY_CUDA(sc.get(&cand_cnt, 257));
        DSG_TRY_CUDA(cudaMemsetAsync(cand_cnt, 0, 257 * sizeof(uint32_t), s));
        {
            LaunchScope ls_("ingest_hot_sample", s);
            hot_sample<<<kHotParts, 1024, smem, s>>>(n, m_raw, sample, cand, cand_cnt + 256, cand_cnt);
        }
        {
            LaunchScope ls_("ingest_hot_select", s);
            hot_select<<<1, 1024, 0, s>>>(cand, cand_cnt + 256, cand_cnt, hot_ids, hot_n);
        }
    } else {
        DSG_TRY_CUDA(cudaMemsetAsync(hot_n, 0, 4, s));
    }
    { LaunchScope ls_("ingest_count_kernel", s); count_kernel<<<pair_grid, 256, 0, s>>>(n, m_raw, src, dst, cnt, hot_ids, hot_n, blk, ctl); }
    DSG_TRY_CUDA(cudaGetLastError());
    if (hot_pass) {
        LaunchScope ls_("ingest_hot_bases", s);
        hot_block_bases<<<kHotMax, 256, 0, s>>>(hot_n, pair_grid, blk);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    DSG_TRY_CUDA(device_scan(cnt, n, start, sums, s));
    { LaunchScope ls_("ingest_classify_count", s); classify_count<<<grid_for(n, 256), 256, 0, s>>>(n, cnt, ctl); }
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
    DSG_TRY_CUDA(sc.get(&tmp, total ? total : 1));
    DSG_TRY_CUDA(sc.get(&lists.rows, nlist ? nlist : 1));
    DSG_TRY_CUDA(cudaMemsetAsync(newlen, 0, ((size_t)n + 1) * 4, s));  // reused as the fill counter
    { LaunchScope ls_("ingest_scatter_kernel", s); scatter_kernel<<<pair_grid, 256, 0, s>>>(n, m_raw, src, dst, start, newlen, hot_ids, hot_n, blk, tmp); }
    DSG_TRY_CUDA(cudaGetLastError());
    {
        LaunchScope ls_("ingest_sort_small_rows", s);
        sort_small_rows<<<grid_for((uint64_t)n, 256), 256, 0, s>>>(n, start, cnt, tmp, newlen, lists, ctl);
    }
    DSG_TRY_CUDA(cudaGetLastError());
    const uint32_t sms = (uint32_t)dev_info().sms;
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
        const uint32_t nwin = (uint32_t)(((uint64_t)n + kWin - 1) >> kWinBits);
        const uint64_t pairs = (uint64_t)ng * nwin;
        uint32_t *hist, *cursor, *ucnt, *spare;
        uint64_t *hoff, *uoff, *gsums;
        DSG_TRY_CUDA(sc.get(&spare, total ? total : 1));
        DSG_TRY_CUDA(sc.get(&hist, pairs));
        DSG_TRY_CUDA(sc.get(&cursor, pairs));
        DSG_TRY_CUDA(sc.get(&ucnt, pairs));
        DSG_TRY_CUDA(sc.get(&hoff, pairs + 1));
        DSG_TRY_CUDA(sc.get(&uoff, pairs + 1));
        DSG_TRY_CUDA(sc.get(&gsums, pairs / kScanTile + 2));
        DSG_TRY_CUDA(cudaMemsetAsync(hist, 0, pairs * 4, s));
        DSG_TRY_CUDA(cudaMemsetAsync(cursor, 0, pairs * 4, s));
        dim3 grid(32, std::min<uint32_t>(ng, 65535u));
        size_t smem = nwin <= 4096 ? (size_t)nwin * 4 : 0;
        { LaunchScope ls_("ingest_giant_rows", s); giant_hist<<<grid, 256, smem, s>>>(glist, ng, start, cnt, tmp, nwin, hist); }
        DSG_TRY_CUDA(cudaGetLastError());
        DSG_TRY_CUDA(device_scan(hist, pairs, hoff, gsums, s));
        { LaunchScope ls_("ingest_giant_rows", s); giant_scatter<<<grid, 256, 0, s>>>(glist, ng, start, cnt, tmp, nwin, hoff, cursor, spare); }
        DSG_TRY_CUDA(cudaGetLastError());
        uint32_t wg = (uint32_t)std::min<uint64_t>((pairs + 7) / 8, (uint64_t)sms * 32);
        { LaunchScope ls_("ingest_giant_rows", s); giant_windows<false><<<wg, 256, 0, s>>>(glist, ng, start, nwin, hist, hoff, spare, ucnt, nullptr, tmp, newlen); }
        DSG_TRY_CUDA(cudaGetLastError());
        DSG_TRY_CUDA(device_scan(ucnt, pairs, uoff, gsums, s));
        { LaunchScope ls_("ingest_giant_rows", s); giant_windows<true><<<wg, 256, 0, s>>>(glist, ng, start, nwin, hist, hoff, spare, ucnt, uoff, tmp, newlen); }
        DSG_TRY_CUDA(cudaGetLastError());
    }
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
