/*
 * dsg.h -- C ABI of libdsg, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of "Parallel Algorithms for Densest Subgraph
 * Discovery Using Shared Memory Model" (De Zoysa et al., arXiv 2103.00154):
 *
 *   - the round-synchronous (2+2eps) densest-subgraph peel of Algorithm 1
 *     (P-Bahmani), with the threshold test done exactly in integers, and
 *   - core numbers by the level-synchronous peel of Algorithm 2's first
 *     phase (PKC).
 *
 * Conventions (all entry points):
 *   - Every call returns a dsg_status.  On error the outputs are left
 *     untouched and dsg_last_error() gives a message (thread-local).
 *   - Graphs are simple and undirected with vertices 0..n-1 (Def. 1).
 *     n must be below 2^31.  Adjacency is CSR: off[n+1] (uint64), adj[off[n]]
 *     (uint32); each edge appears in both rows; rows sorted ascending, no
 *     self-loops, no repeats ("canonical").
 *   - Pointer arguments are host or device pointers; the library tells them
 *     apart with cudaPointerGetAttributes.  Input arrays are copied unless
 *     DSG_PTRS_DEVICE is given, in which case the caller keeps ownership and
 *     the arrays must outlive the graph handle.  Output arrays are
 *     caller-allocated (host or device memory).
 *   - Each graph handle carries a CUDA stream (given at creation, the
 *     legacy default stream if NULL); all work of calls on that handle is
 *     ordered on it.  The calls below return once their results are
 *     written (they synchronise that stream).
 *   - Density values are exact rationals E/V (uint64 pairs).
 */
#ifndef DSG_H
#define DSG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DSG_OK = 0,
    DSG_EINVAL = 1,     /* bad argument: null pointer, q == 0, n >= 2^31, malformed CSR under VALIDATE */
    DSG_ENOMEM = 2,     /* device or host allocation failed */
    DSG_ECUDA = 3,      /* a CUDA runtime call failed */
    DSG_ETIMEOUT = 4,   /* a bounded device-side wait ran out (the kernel returned; the context stays usable) */
    DSG_EBUSY = 5,      /* serving: no slot / memory free right now (back-pressure) */
    DSG_EAGAIN = 6,     /* serving: result not ready yet */
    DSG_ENOTFOUND = 7,  /* serving: unknown ticket */
    DSG_EOVERFLOW = 8   /* an output capacity given by the caller is too small */
} dsg_status;

/* flags for dsg_graph_from_csr / dsg_graph_from_edges */
#define DSG_CSR_CANONICALIZE 0x1u /* input may hold loops, repeats, one-sided edges, unsorted rows */
#define DSG_CSR_VALIDATE 0x2u     /* check the CSR is canonical on the device; DSG_EINVAL if not */
#define DSG_PTRS_DEVICE 0x4u      /* inputs are device pointers owned by the caller (no copy) */

typedef struct dsg_graph dsg_graph; /* opaque: device CSR plus the stream of its calls */

/* ---------------------------------------------------------------- graphs */

/*
 * Build a device graph from a CSR (Def. 1 graph; the paper's "super map" of
 * Sec. 3.1 "Data structures" is replaced by CSR over ids 0..n-1).
 *   n      vertex count (< 2^31)
 *   off    n+1 uint64 row offsets, off[0] = 0
 *   adj    off[n] uint32 neighbour ids
 *   flags  DSG_CSR_CANONICALIZE | DSG_CSR_VALIDATE | DSG_PTRS_DEVICE
 *          (CANONICALIZE runs the edge-list ingest on the CSR entries and
 *          always copies; it cannot be combined with PTRS_DEVICE ownership)
 *   stream cudaStream_t for this graph's work (NULL: default stream)
 *   out    receives the handle (free with dsg_graph_free)
 */
dsg_status dsg_graph_from_csr(uint32_t n, const uint64_t* off, const uint32_t* adj, uint32_t flags, void* stream,
                              dsg_graph** out);

/*
 * Ingest raw undirected pairs (src[i], dst[i]), i < m_raw, over ids 0..n-1:
 * drop self-loops, merge repeats and both orientations, emit both
 * directions, sort each row (Def. 1: E is a set of edges between distinct
 * vertices).  Runs on the device.  With DSG_PTRS_DEVICE, src/dst are device
 * arrays read in place.  DSG_EINVAL if an id is >= n.
 */
dsg_status dsg_graph_from_edges(uint32_t n, uint64_t m_raw, const uint32_t* src, const uint32_t* dst, uint32_t flags,
                                void* stream, dsg_graph** out);

/* n and the undirected edge count m (= off[n]/2) of a graph. */
dsg_status dsg_graph_info(const dsg_graph* g, uint32_t* n, uint64_t* m);

/* Copy the canonical CSR out: off[n+1], adj[2m] (host or device buffers). */
dsg_status dsg_graph_csr(const dsg_graph* g, uint64_t* off, uint32_t* adj);

/* Re-target the graph's calls to another stream. */
dsg_status dsg_graph_set_stream(dsg_graph* g, void* stream);

/* A second handle over g's device CSR, bound to `stream` (no copy; the view
 * must be freed before g).  With views on different streams, independent
 * solves of one graph (peels at several eps, core numbers) can be issued
 * side by side.  No counterpart in the paper. */
dsg_status dsg_graph_view(const dsg_graph* g, void* stream, dsg_graph** out);

/* Cap the grid of the persistent kernels (peel, core numbers) launched for
 * this handle at max_blocks blocks (0: as many as the GPU holds), so that
 * solves on two handles, capped to fit the GPU together, run side by side;
 * a solve's result never depends on the cap.  No counterpart in the paper. */
dsg_status dsg_graph_set_max_blocks(dsg_graph* g, uint32_t max_blocks);

/* Release a graph and its device memory.  NULL is ignored. */
void dsg_graph_free(dsg_graph* g);

/* ----------------------------------------------------- Algorithm 1 (peel) */

/*
 * Bahmani (2+2eps) peel, Algorithm 1 (P-Bahmani), eps = eps_num/eps_den:
 *   S_0 = V; in round r every v in S_r with deg_{S_r}(v) <= 2(1+eps)|E(S_r)|/|S_r|
 *   fails (tested exactly: deg * q * |S| <= 2 (p+q) |E|, against the degrees
 *   at the start of the round); failed vertices and their edges leave;
 *   |S| and |E(S)| are reduced; the densest S seen is kept, strict ">" so the
 *   earliest round wins a tie; the loop stops when S is empty.  eps = 0 is
 *   allowed.
 *   out_set  n bytes, nullable: 1 for vertices of the densest set found
 *   out_E/V  nullable: |E(S~)| and |S~| (zero for n = 0)
 * DSG_EINVAL if eps_den == 0.
 */
dsg_status dsg_bahmani(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, uint8_t* out_set, uint64_t* out_E,
                       uint64_t* out_V);

/* Full record of one peel (Algorithm 1), for checking and analysis. */
typedef struct {
    uint64_t rounds;      /* out: R, the number of rounds run */
    uint64_t best_round;  /* out: round whose set S_r is the answer */
    uint64_t best_E;      /* out: |E(S~)| */
    uint64_t best_V;      /* out: |S~| */
    uint64_t hist_cap;    /* in: capacity of hist_S / hist_E (needs R+1) */
    uint64_t* hist_S;     /* out, nullable: |S_r| for r = 0..R */
    uint64_t* hist_E;     /* out, nullable: |E(S_r)| for r = 0..R */
    uint32_t* peel_round; /* out, nullable, n entries: round (1-based) in which v failed */
    uint8_t* out_set;     /* out, nullable, n entries: membership in S~ */
    uint64_t edges_scanned; /* out: adjacency entries read by the neighbour scans (= 2m) */
    uint64_t decrements;    /* out: degree decrements of surviving neighbours (edges whose
                               ends failed in different rounds) */
    uint64_t tested;        /* out: vertex tests of the threshold passes, summed over the rounds */
    uint64_t lazy_rounds;   /* out: rounds that tested only the candidate list (see dsg_set_peel_lazy) */
} dsg_trace;

/* As dsg_bahmani, recording the per-round history.  DSG_EOVERFLOW if
 * hist_cap < R+1 (the scalar outputs are still written). */
dsg_status dsg_bahmani_trace(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, dsg_trace* t);

/* Upper bound on R+1 for a graph of n vertices: ceil(log_{(p+q)/q} n) + 2
 * when p > 0 (each round with edges leaves fewer than q/(p+q) of the
 * vertices), n + 1 when p == 0. */
uint64_t dsg_round_bound(uint32_t n, uint32_t eps_num, uint32_t eps_den);

/*
 * dsg_bahmani without any device allocation.  The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory when they
 * run the peel (their memory is reserved by an allocator they do not own, or
 * their hot path must not call cudaMalloc, which can synchronise the device).
 * It runs the same kernel as dsg_bahmani with every scratch array carved from
 * one fixed 64 MiB buffer that this library keeps in device memory: the
 * buffer is reserved on every GPU that loads the library and held until the
 * process exits.
 *   n, off, adj  canonical CSR in DEVICE memory (as dsg_graph_from_csr)
 *   out_set      nullable, n bytes of DEVICE memory
 *   out_E/out_V  nullable host pointers
 *   stream       cudaStream_t to run on (NULL: default stream).  Every call
 *                waits for this stream twice: it reads off[n] back before
 *                the launch and the results after it.
 * Limits: the scratch is nine arrays, each rounded up to a multiple of 256
 * bytes: four of 4n bytes (vertex state, two alive lists, failed list), the
 * chunk items 8(n + 2m/chunk_len + 1) bytes, the status map 4 ceil(n/16)
 * bytes, two round histories of 8(dsg_round_bound(n, p, q) + 1) bytes, and a
 * control block of about 1 KB; chunk_len is the current tuning's
 * (dsg_set_tuning; 256 by default).  A graph whose scratch exceeds 64 MiB is
 * rejected with DSG_EINVAL before any GPU work (with eps > 0 and the default
 * chunk_len that admits n up to about 2.7 million at m = 8n).
 * The first call in each CUDA context (the first on a device, and the first
 * after that device's context was destroyed and made again) looks the
 * buffer's device address up, with the device current.  Because every call
 * synchronises its stream (above), no call can be made on a stream that is
 * being captured into a CUDA graph.  All calls share the one buffer and it
 * keeps the last call's contents: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 */
dsg_status dsg_bahmani_noalloc(uint32_t n, const uint64_t* off, const uint32_t* adj, uint32_t eps_num,
                               uint32_t eps_den, uint8_t* out_set, uint64_t* out_E, uint64_t* out_V, void* stream);

/*
 * Snapshot / resume of Algorithm 1 (Sec. 3.1).  The algorithm's state
 * between two rounds -- each vertex's degree inside S_r or the round it
 * failed in, the round r, |S_r|, |E(S_r)|, the densest round so far with its
 * (|E|, |V|), and the per-round history -- is all it needs to go on, so a
 * peel can be paused, written to host memory and continued later (on the
 * same or another handle of the same graph, on any device) with exactly the
 * result of an uninterrupted dsg_bahmani.
 *   dsg_peel_begin         a paused peel of g at eps_num / eps_den, at round 0.
 *                          g must outlive the state.
 *   dsg_peel_advance       run at most max_rounds more rounds (0: to the end);
 *                          *rounds (nullable) = rounds done so far, *done
 *                          (nullable) = 1 once S is empty.
 *   dsg_peel_snapshot_size bytes of its snapshot now: 8 (16 + 2 (r + 1)) +
 *                          4 n.
 *   dsg_peel_snapshot      write the snapshot into a caller-owned host buffer
 *                          of at least that many bytes (DSG_EINVAL if smaller):
 *                          16 u64 header words (magic "DSGPEEL1", version 1, n,
 *                          m, p, q, r, |S_r|, |E(S_r)|, best round, best E,
 *                          best V, history length r + 1, 3 reserved), the
 *                          histories of |S_t| and |E(S_t)| (u64 each), then n
 *                          u32 state words (degree, or 0x80000000 | failure
 *                          round).
 *   dsg_peel_resume        a paused peel rebuilt from a snapshot on g; DSG_EINVAL
 *                          if the buffer is not a snapshot, is truncated, or was
 *                          taken on a graph with another n or m.
 *   dsg_peel_finish        run to the end; out_set (n bytes, host or device,
 *                          nullable), out_E / out_V / out_rounds (nullable), and
 *                          the histories into hist_S / hist_E (nullable, hist_cap
 *                          slots; DSG_EOVERFLOW if fewer than R + 1, the scalars
 *                          still written).  The state stays valid.
 *   dsg_peel_free          release the state's device memory.
 */
typedef struct dsg_peel_state dsg_peel_state;
dsg_status dsg_peel_begin(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, dsg_peel_state** out);
dsg_status dsg_peel_advance(dsg_peel_state* st, uint32_t max_rounds, uint64_t* rounds, uint32_t* done);
dsg_status dsg_peel_snapshot_size(const dsg_peel_state* st, uint64_t* bytes);
dsg_status dsg_peel_snapshot(const dsg_peel_state* st, void* buf, uint64_t bytes);
dsg_status dsg_peel_resume(const dsg_graph* g, const void* buf, uint64_t bytes, dsg_peel_state** out);
dsg_status dsg_peel_finish(dsg_peel_state* st, uint8_t* out_set, uint64_t* out_E, uint64_t* out_V,
                           uint64_t* out_rounds, uint64_t* hist_S, uint64_t* hist_E, uint64_t hist_cap);
void dsg_peel_free(dsg_peel_state* st);

/* --------------------------------------------- Algorithm 2, first phase */

/*
 * Core numbers (Def. 2) by the level-synchronous peel of Algorithm 2's first
 * phase (PKC): level k collects the remaining vertices of degree k, then
 * drains them, taking one from each neighbour above k and collecting a
 * neighbour when it reaches k; levels with no vertex are skipped.
 *   out_core  n uint32 (host or device)
 */
dsg_status dsg_kcore(const dsg_graph* g, uint32_t* out_core);

/* As dsg_kcore, also writing up to nstats counters of the run into stats:
 *   [0] levels run (the blocks meet once per level, on its work counter)
 *   [1] row pieces queued to the level-wide work queue
 *   [2] remaining-list entries scanned (sum over levels)
 *   [3] remaining-list entries written (sum over levels)
 *   [4] degree atomics issued (decrements plus undos) */
dsg_status dsg_kcore_stats(const dsg_graph* g, uint32_t* out_core, uint64_t* stats, uint32_t nstats);

/* ------------------------------------------------------------- batches */

/*
 * Many independent graphs solved in one launch (the peel of Algorithm 1 for
 * every graph, core numbers of Algorithm 2's first phase for those asking).
 * Concatenated CSR: graph g owns vertex slots [vtx_base[g], vtx_base[g+1]);
 * the row of its local vertex v is adj[off[vtx_base[g]+v] .. off[vtx_base[g]+v+1])
 * and holds LOCAL neighbour ids (0..n_g-1); each graph's rows are canonical.
 * Arrays may be host or device memory (host arrays are copied).
 */
typedef struct {
    uint32_t num_graphs;        /* G */
    const uint64_t* vtx_base;   /* G+1, vtx_base[0] = 0 */
    const uint64_t* off;        /* vtx_base[G]+1 row offsets into adj */
    const uint32_t* adj;        /* off[vtx_base[G]] local neighbour ids */
    const uint32_t* eps_num;    /* G: eps_g = eps_num[g] / eps_den[g] */
    const uint32_t* eps_den;    /* G, positive */
    const uint8_t* want_core;   /* G, nullable (NULL: every graph, if result.core is set) */
} dsg_batch;

typedef struct {
    uint64_t* E;            /* G, nullable: |E(S~)| per graph (host) */
    uint64_t* V;            /* G, nullable: |S~| */
    uint64_t* rounds;       /* G, nullable: R */
    uint64_t* best_round;   /* G, nullable */
    uint8_t* out_set;       /* vtx_base[G], nullable: densest-set membership (host or device) */
    uint32_t* core;         /* vtx_base[G], nullable: core numbers (host or device; untouched
                               for graphs with want_core[g] == 0) */
    uint64_t* stats;        /* 4, nullable (host): over the batch, the sum over graphs and rounds of
                               |S_r|, the peels' alive-neighbour decrements, the adjacency entries
                               (2m summed), and how many graphs the grid-wide kernels solved */
} dsg_batch_result;

/*
 * Solve a batch in one persistent launch: blocks pull graphs largest first
 * and each block solves its graph alone (block barriers instead of grid
 * barriers).  Results equal those of dsg_bahmani / dsg_kcore on each graph
 * alone.  DSG_EINVAL on malformed offsets or eps_den == 0.
 */
dsg_status dsg_batch_solve(const dsg_batch* b, dsg_batch_result* r, void* stream);
/* Which graphs of a batch the grid-wide kernels solve (before the
 * block-per-graph launch): those whose work 2m + n exceeds min_work; 0 (the
 * default) means those above twice one block's share of the batch's work and
 * above 2^20; 0xffffffff keeps every graph in the block-per-graph launch.
 * DSG_BATCH_SPLIT.  Results never depend on it. */
dsg_status dsg_set_batch_split(uint32_t min_work);
/* Autotune dsg_batch_solve for this batch's class (device, floor(log2 G),
 * floor(log2 of the summed 2m + n)): coordinate descent over the
 * block-per-graph kernel's block size (256 / 512 / 1024), the hub threshold
 * and the grid-wide split, timing whole solves of b (their results are
 * discarded); later batches of the class use the winner.  Results never
 * depend on it.  *trials (nullable) = solves timed. */
dsg_status dsg_batch_autotune(const dsg_batch* b, uint32_t* trials);

/* ------------------------------------------------------------- serving */

/*
 * A serving loop on one GPU: requests (raw pairs + eps) are admitted while
 * their device-memory charge fits a budget, ingested into resident graphs,
 * and solved by continuous batching -- whatever was ingested while the
 * previous batch ran forms the next block-per-graph launch (see
 * dsg_batch_solve), so arrivals overlap with work already on the device.  A
 * request's results do not depend on what it is batched with.  All calls
 * are thread-safe.
 */
typedef struct dsg_server dsg_server;

typedef struct {
    uint32_t max_batch;    /* most graphs per launch (0: 1024) */
    uint32_t max_pending;  /* queued, not yet admitted requests before DSG_EBUSY (0: 65536) */
    uint64_t hbm_budget;   /* device bytes admitted requests may hold (0: half the free memory) */
    uint32_t max_inflight; /* batches on the device at once, each on its own stream (0: 4) */
    uint32_t ingest_threads; /* host threads ingesting admitted requests, each on its own stream (0: 4) */
    uint64_t big_work;     /* a request whose 2 m_raw + n exceeds this is solved on its own by the
                              grid-wide kernels on big_sms SMs, not in a block-per-graph batch
                              (0: 2^23; UINT64_MAX: never) */
    uint32_t big_sms;      /* SMs each grid-wide solve of a big request uses (0: a quarter of them
                              divided by big_threads); the block-per-graph batches use the rest */
    uint64_t max_batch_work; /* a launch closes before the next ready request would take its summed
                                work (2m + n of its graphs) past this, so one launch's run time, and
                                the wait of the requests behind it, stays bounded (0: no limit) */
    uint32_t big_threads;  /* host threads solving big requests, each on its own stream with big_sms
                              SMs (0: 2) */
} dsg_serve_config;

#define DSG_REQ_BORROW 0x1u   /* src/dst stay valid and unchanged until the request completes: no copy */

typedef struct {
    uint32_t n;              /* vertices 0..n-1 */
    uint64_t m_raw;          /* raw pairs */
    const uint32_t* src;     /* host memory, copied by dsg_serve_submit unless DSG_REQ_BORROW */
    const uint32_t* dst;
    uint32_t eps_num, eps_den;
    uint32_t want_core;      /* nonzero: also compute core numbers */
    uint32_t flags;          /* DSG_REQ_BORROW */
    uint8_t* out_set;        /* nullable host buffer (n bytes), filled before completion */
    uint32_t* core;          /* nullable host buffer (n entries), filled when want_core */
} dsg_request;

typedef struct {
    dsg_status status;
    uint32_t n;
    uint64_t m;              /* undirected edges after ingest */
    uint64_t E, V, rounds, best_round;
    double latency_us;       /* submit to completion */
} dsg_response;

typedef struct {
    uint64_t submitted, admitted, completed, rejected, pending, in_flight, batches;
    uint64_t hbm_in_use, hbm_budget;
    double p50_us, p99_us;   /* latency of completed requests */
    double graphs_per_s;     /* completed / uptime */
    double uptime_s;
    /* where the time went: requests solved alone by the grid-wide kernels,
     * host seconds the ingest threads spent ingesting (summed over threads)
     * and the big-request thread spent solving, and device seconds of the
     * block-per-graph launches (summed over launches, which may overlap) */
    uint64_t big_done;
    double ingest_busy_s, big_busy_s, batch_device_s;
} dsg_serve_info;

dsg_status dsg_serve_create(const dsg_serve_config* cfg, dsg_server** out);
/* DSG_EBUSY when the queue is full (back-pressure: retry later); DSG_EINVAL
 * when the request can never fit the budget. */
dsg_status dsg_serve_submit(dsg_server* s, const dsg_request* r, uint64_t* ticket);
/* Waits up to timeout_us for the ticket; DSG_EAGAIN if still running,
 * DSG_ENOTFOUND for an unknown (or already collected) ticket.  A collected
 * ticket is released. */
dsg_status dsg_serve_poll(dsg_server* s, uint64_t ticket, dsg_response* resp, uint32_t timeout_us);
dsg_status dsg_serve_stats(dsg_server* s, dsg_serve_info* out);
/* Cancels requests not yet admitted, finishes the admitted ones, frees all. */
void dsg_serve_destroy(dsg_server* s);

/* ------------------------------------------------------------- tuning */

/*
 * Launch parameters of the round kernels (not part of the method):
 *   block          threads per block of the persistent kernels: 256, 512, 1024
 *   blocks_per_sm  resident blocks per SM (0 = as many as fit)
 *   short_max      rows up to this length are scanned edge-balanced inside a
 *                  block; longer rows are cut into chunk items
 *   chunk_len      entries per chunk item (one warp each), >= 32
 * Process-wide; also read from DSG_BLOCK, DSG_BLOCKS_PER_SM, DSG_SHORT_MAX and
 * DSG_CHUNK_LEN at first use.  Results never depend on these.
 */
dsg_status dsg_set_tuning(uint32_t block, uint32_t blocks_per_sm, uint32_t short_max, uint32_t chunk_len);
dsg_status dsg_get_tuning(uint32_t* block, uint32_t* blocks_per_sm, uint32_t* short_max, uint32_t* chunk_len);
/* Bahmani peel: degree at or above which decrements of a vertex are first
 * combined in a per-block shared-memory table (one global atomic per block and
 * phase for a hub instead of one per edge).  0 (the default) means four times
 * the number of blocks of the launch; DSG_HOT_DEG.  Results never depend on
 * it.  The core numbers decrement every neighbour at once and ignore it. */
dsg_status dsg_set_hot_degree(uint32_t hot_deg);
/* Core numbers: a vertex whose row has at most local_max entries and that
 * reaches the current level while a block drains is drained by that block
 * from a shared-memory queue (PKC's thread-local buffer), as long as the
 * entries the block takes on this way stay within local_work (for its own
 * rows of the level, and again for each batch of queue pieces it takes);
 * other rows go to the level-wide queue of row pieces that every block
 * drains.  Defaults 1024 / 16384; DSG_LOCAL_MAX, DSG_LOCAL_WORK.  Results
 * never depend on them. */
dsg_status dsg_set_local_max(uint32_t local_max, uint32_t local_work);
/* Core numbers: a vertex whose row has at most inline_max entries and that a
 * block's level scan claims is drained by that block; longer rows go to the
 * level-wide queue in pieces of at most chunk_len entries, which every block
 * takes from.  Default 256; DSG_INLINE_MAX.  Results never depend on it. */
dsg_status dsg_set_inline_max(uint32_t inline_max);
/* Core numbers: once at most max_vertices vertices remain after a level, the
 * remaining graph is compacted (rows cut to the remaining neighbours, which
 * leaves every remaining degree as it is) and one thread-block cluster runs
 * the remaining levels with the degrees in its distributed shared memory.
 * 0 turns it off; at most 131072 (16 blocks of 8192 vertices).  Default
 * 65536; DSG_KCORE_TAIL.  Results never depend on it. */
dsg_status dsg_set_kcore_tail(uint32_t max_vertices);
/* Peel (Algorithm 1) in a thin tail: once a round removes less than 1/8 of
 * the vertices left, the next round also collects candidates -- every alive
 * vertex whose degree is at or below a bound B = T + floor(T/128) (T the
 * round's threshold), from the surviving vertices it tests and from the
 * decrements that bring a degree down to B -- and a following round whose
 * threshold is at most B and whose candidates number less than a quarter of
 * the vertices left tests only those candidates instead of every alive
 * vertex.  A vertex failing in that round has degree <= T <= B and so is
 * among them: the rounds are the same, with fewer vertex tests
 * (dsg_trace.tested).  1 (default) on, 0 off; DSG_PEEL_LAZY.  Results never
 * depend on it. */
dsg_status dsg_set_peel_lazy(uint32_t on);
/* Peel (Algorithm 1): 1 reads the long rows' chunks as aligned 16-byte
 * groups, four consecutive entries per lane (one 128-bit load each, entries
 * outside the chunk masked off); 0 (default) reads one entry per lane, 32
 * consecutive entries per warp load, four loads in flight.  Used only when
 * the adjacency array is 16-byte aligned.  DSG_PEEL_VEC.  Results never
 * depend on it. */
dsg_status dsg_set_peel_vec(uint32_t on);

/*
 * Densest k-core and CBDS-P (Algorithm 2).
 *
 * dsg_densest_core: the k-core {v : core(v) >= k} of highest density
 * |E_k| / |V_k| over all k (Sec. 3.2, the approach of Algorithm 2's first
 * phase; a 2-approximation of the densest subgraph).  On equal density the
 * smallest k (the largest core) wins.  res gets k_star, E_core = |E_k*|,
 * V_core = |V_k*|, and E = E_core, V = V_core, n_legit = 0.
 *
 * dsg_cbds: the same, followed by Algorithm 2's second phase, which adds to
 * the densest core every vertex v outside it whose core number lies strictly
 * between the core's density and k* and which has more neighbours inside the
 * core than that density ("legit"); each adds those edges, and the edges
 * among legit vertices are added once.  res->E = m_e, res->V = m_v (the
 * augmented subgraph's edges and vertices), res->n_legit = #legit.
 *
 *   core     nullable, n core numbers (host or device) to use instead of
 *            computing them (phase 1); every value must be below n (EINVAL
 *            otherwise).  The results are defined for whatever values are
 *            given; only true core numbers give the paper's method.
 *   out_core nullable, n entries (host or device): the core numbers used.
 *   out_set  nullable, n bytes (host or device): 1 for the vertices of the
 *            result (densest core, plus the legit vertices for dsg_cbds).
 * Densities are compared exactly (128-bit cross-multiplication).  n = 0:
 * all zeros.  Outputs are untouched on error.
 */
typedef struct dsg_cbds_result {
    uint64_t k_star;  /* densest core's k */
    uint64_t E_core;  /* |E| of the densest core */
    uint64_t V_core;  /* |V| of the densest core */
    uint64_t E;       /* |E| of the result */
    uint64_t V;       /* |V| of the result */
    uint64_t n_legit; /* vertices added by the second phase */
} dsg_cbds_result;

dsg_status dsg_densest_core(const dsg_graph* g, const uint32_t* core, uint32_t* out_core, uint8_t* out_set,
                            dsg_cbds_result* res);
dsg_status dsg_cbds(const dsg_graph* g, const uint32_t* core, uint32_t* out_core, uint8_t* out_set,
                    dsg_cbds_result* res);

/*
 * Autotuner.  dsg_autotune times candidate launch parameters for the peel
 * (what bit 0, at eps_num/eps_den) and/or the core numbers (bit 1) on graph g
 * by coordinate descent over block size, hub threshold, chunk length and
 * short-row limit (peel) or block size, hub threshold, the local-drain
 * limits and the inline-drain limit (core numbers), keeping a change only
 * when it is at least 2%
 * faster.  The winner is recorded for g's size class (floor log2 n,
 * floor log2 2m) on this device and used by every later solve of a graph of
 * that class; *trials gets the number of timed solves.  The table is saved
 * to DSG_TUNE_FILE (if set) after tuning and loaded from it at first use.
 * Results never depend on tuning.
 */
dsg_status dsg_autotune(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, uint32_t what, uint32_t* trials);
dsg_status dsg_tune_save(const char* path);
dsg_status dsg_tune_load(const char* path, uint32_t* entries);
void dsg_tune_clear(void);
uint32_t dsg_tune_entries(void);
/* The launch parameters a solve of kernel 0 (peel) or 1 (core numbers) on g
 * would use now: out = {block, blocks_per_sm, short_max, chunk_len, hot_deg,
 * local_max, local_work, inline_max, kcore_tail}. */
dsg_status dsg_tune_lookup(const dsg_graph* g, uint32_t kernel, uint32_t out[9]);

/*
 * Device-memory allocator hook (no counterpart in the paper; lets a host
 * framework's caching allocator own every device buffer the library makes:
 * graph CSR arrays and per-call scratch).  alloc(bytes, ctx, stream) returns
 * device memory of the current device usable in stream order on `stream`
 * (NULL = out of memory, reported as DSG_ENOMEM); free(ptr, ctx, stream)
 * takes it back in stream order.  Each pointer returns to the allocator that
 * made it, so the hook may be changed between calls; passing NULL for either
 * function restores the built-in stream-ordered pool.  Process-wide; do not
 * change it while a call is running on another thread.
 */
typedef void* (*dsg_alloc_fn)(size_t bytes, void* ctx, void* stream);
typedef void (*dsg_free_fn)(void* ptr, void* ctx, void* stream);
void dsg_set_allocator(dsg_alloc_fn alloc, dsg_free_fn free_fn, void* ctx);

/*
 * Several Bahmani peels (eps_num[i] / eps_den[i], i < count) and the core
 * numbers of one graph in one call: the same results as count dsg_bahmani
 * calls plus one dsg_kcore call (out_sets[i], out_E[i], out_V[i]; out_core),
 * with the peels and the core decomposition running side by side on two
 * internal streams, the peels on the share of the SMs that their autotuned
 * time has in the summed time (within 1/4 and 3/4; half when the graph's size
 * class is not tuned; the environment variable DSG_SOLVE_PEEL_PERMILLE, 1..999,
 * overrides it) -- unless the autotuned times show the core numbers taking
 * over four times as long as the peels, in which case they run one after the
 * other on the whole GPU.  Results never depend on the choice.  out_sets (and its entries),
 * out_E, out_V nullable; out_core NULL runs the peels only.  Work starts
 * after what is queued on the graph's stream, which waits for all of it
 * before the call returns.  No counterpart in the paper (its two algorithms
 * are separate programs).
 */
dsg_status dsg_solve(const dsg_graph* g, uint32_t count, const uint32_t* eps_num, const uint32_t* eps_den,
                     uint8_t* const* out_sets, uint64_t* out_E, uint64_t* out_V, uint32_t* out_core);

/* Upper bound (ns) on every device-side wait (grid barriers, queue polls).
 * A wait that runs out makes its kernel return and the call report
 * DSG_ETIMEOUT.  0 restores the default (10 s, or DSG_WAIT_LIMIT_NS). */
void dsg_set_wait_limit_ns(uint64_t ns);

/*
 * Fault-detection probe.  Launches a kernel whose bounded wait can never be
 * satisfied -- which = 0: one thread polls a device flag that nothing sets;
 * which = 1: a two-block cooperative grid where one block skips the grid
 * barrier the other waits in -- and returns the status the library's own
 * time-out path produces (DSG_ETIMEOUT after limit_ns, 0 < limit_ns <= 10 s).
 * No fault, trap or unbounded spin is involved.
 */
dsg_status dsg_debug_wait_timeout(uint32_t which, uint64_t limit_ns);

/*
 * Analysis probes (no counterpart in the paper; used to measure the round
 * machinery, not part of the method).
 *   dsg_debug_peel_trace   one Algorithm 1 run recording %globaltimer (ns)
 *                          at kernel start and after every grid barrier
 *                          (2 per round) into ts[cap]; *count = stamps taken
 *   dsg_debug_kcore_trace  one core decomposition recording pairs
 *                          (ns, kind << 32 | k): kind 0 start, 1 degrees
 *                          initialised, 2 level over (block 0), 3/4/5 block
 *                          0's scan / own rows / queue phase done; after
 *                          each level five (value, kind << 32 | k) pairs:
 *                          6/7 latest own / queue phase end over the blocks
 *                          (ns, as block 0 sees them), 8 claims, 9 claims by
 *                          the scan, 10 queued row pieces; *count = pairs
 */
dsg_status dsg_debug_peel_trace(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, uint64_t* ts, uint64_t cap,
                                uint64_t* count);
dsg_status dsg_debug_kcore_trace(const dsg_graph* g, uint64_t* ts, uint64_t cap, uint64_t* count);

/* ------------------------------------------------------- launch accounting */

/* Number of kernels this library has launched in the process. */
unsigned long long dsg_launch_count(void);
/* With profiling on, every launch is bracketed by CUDA events on the stream
 * it runs on; dsg_profile_report writes one line "kernel launches total_ms"
 * per kernel into buf (at most cap bytes) and returns the kernel count. */
void dsg_profile_enable(int on);
void dsg_profile_reset(void);
int dsg_profile_report(char* buf, size_t cap);

/* ------------------------------------------------------------- errors */

const char* dsg_status_string(dsg_status s);
/* Message of the last failing call on this thread ("" if none). */
const char* dsg_last_error(void);

/* Library version string. */
const char* dsg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DSG_H */
