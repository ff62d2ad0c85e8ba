/*
 * ORACLE -- test infrastructure, not product code.
 *
 * A plain, serial, deliberately slow CPU statement of what the densest-
 * subgraph hot path computes, written from the paper ("Parallel Algorithms
 * for Densest Subgraph Discovery Using Shared Memory Model", De Zoysa et al.,
 * arXiv 2103.00154).  Only the test suite, the smoke check and the bench's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library; the two meet only in the seeded input generators.
 *
 * Contents (each function cites the passage it follows):
 *   orc_canonical_csr     simple undirected graph from raw pairs (Def. 1; graph
 *                         store of Sec. 3.1 "Data structures")
 *   orc_bahmani           round-synchronous (2+2eps) peel, Algorithm 1, incremental
 *   orc_bahmani_recompute the same peel recomputing deg and |E(S)| from scratch
 *                         every round (second, independent statement)
 *   orc_kcore_bz          core numbers by Batagelj-Zaversnik bucket peeling (Def. 2)
 *   orc_kcore_naive       core numbers by per-k iterative deletion (Def. 2)
 *   orc_kcore_pkc         core numbers by the level-synchronous scheme of
 *                         Algorithm 2, first phase, run serially
 *   orc_densest_core      densest k-core (V_k, E_k) scan (Sec. 3.2 approach)
 *   orc_cbds_phase2       vertex augmentation of the densest core, Algorithm 2
 *                         second phase
 *   orc_brute_densest     exact densest subgraph by subset enumeration (n <= 24)
 *   orc_goldberg_densest  exact densest subgraph by Goldberg's min-cut
 *                         construction with Dinkelbach iteration (Sec. 2, ref. [32])
 *
 * All arithmetic is integer; densities are exact rationals compared by
 * 128-bit cross-multiplication.
 *
 * Parity status: every function is pinned by tests against closed forms,
 * brute force, a max-flow optimum, a library routine (networkx core_number)
 * or a second independent statement in this file; see tests/test_oracle_*.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* ------------------------------------------------------------------ ingest */

/*
 * Simple undirected graph from raw pairs.  Def. 1 takes E as a set of edges
 * between distinct vertices; the paper's graph store (Sec. 3.1, "Data
 * structures") keys each vertex's neighbours in a hash map, which removes
 * repeated pairs.  Self-loops are dropped (the reading taken for both sides).
 *
 * Steps: drop u == v; write each pair as (min, max); sort; unique; emit both
 * directions; count row lengths; prefix-sum into off; fill rows; sort each row.
 * off has n+1 entries; adj must hold 2 * m_raw entries.  Returns off[n] (= 2m),
 * or -1 on bad input / allocation failure.
 */
int64_t orc_canonical_csr(uint32_t n, uint64_t m_raw, const uint32_t* src, const uint32_t* dst, uint64_t* off,
                          uint32_t* adj) {
    uint64_t* keys = (uint64_t*)malloc((m_raw ? m_raw : 1) * sizeof(uint64_t));
    if (!keys) return -1;
    uint64_t k = 0;
    for (uint64_t i = 0; i < m_raw; ++i) {
        uint32_t u = src[i], v = dst[i];
        if (u >= n || v >= n) { free(keys); return -1; }
        if (u == v) continue;
        uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
        keys[k++] = (lo << 32) | hi;
    }
    qsort(keys, k, sizeof(uint64_t), cmp_u64);
    uint64_t m = 0;
    for (uint64_t i = 0; i < k; ++i)
        if (i == 0 || keys[i] != keys[i - 1]) keys[m++] = keys[i];
    uint64_t* cnt = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!cnt) { free(keys); return -1; }
    for (uint64_t i = 0; i < m; ++i) {
        cnt[keys[i] >> 32]++;
        cnt[keys[i] & 0xffffffffu]++;
    }
    off[0] = 0;
    for (uint32_t v = 0; v < n; ++v) off[v + 1] = off[v] + cnt[v];
    for (uint32_t v = 0; v < n; ++v) cnt[v] = off[v];
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t u = (uint32_t)(keys[i] >> 32), v = (uint32_t)(keys[i] & 0xffffffffu);
        adj[cnt[u]++] = v;
        adj[cnt[v]++] = u;
    }
    for (uint32_t v = 0; v < n; ++v) qsort(adj + off[v], off[v + 1] - off[v], sizeof(uint32_t), cmp_u32);
    free(cnt);
    free(keys);
    return (int64_t)off[n];
}

/* ------------------------------------------------------------ Bahmani peel */

/*
 * out[0] = R (rounds run), out[1] = best_round, out[2] = E_best, out[3] = V_best.
 * hist_S / hist_E receive |S_r| and |E(S_r)| for r = 0..R (need R+1 slots;
 * returns -2 if hist_cap is too small).  peel_round[v] = the round number
 * (1-based) in which v failed the threshold test.
 */
#define BEST_OUT(o, R, br, be, bv) do { o[0] = (R); o[1] = (br); o[2] = (be); o[3] = (bv); } while (0)

/*
 * Algorithm 1 (P-Bahmani), serial.  eps = p/q.
 *
 *   S <- V, E <- |E(V)|, best <- (round 0, E, |V|)                (init, rho_0 = rho(V))
 *   while |S| > 0:
 *     part 1: every v in S with deg_S(v) <= 2(1+eps) rho(S) fails   (threshold test)
 *             -- tested as deg * q * |S| <= 2 (p+q) * |E|, exactly in 128 bits;
 *             all tests see the degrees at the start of the round (barrier)
 *     part 2: remove the failed vertices and every edge they touch;
 *             each surviving neighbour loses one degree per removed edge,
 *             and |E| drops by the number of distinct removed edges
 *     reduce: |S| and |E| of the new set
 *     keep best: if rho(S) > rho(best) (strict), best <- S
 *
 * Returns 0, or -1 (allocation), -2 (history capacity), -3 (q == 0), -4 (a round
 * removed no vertex, which the minimum-degree vertex rules out).
 */
int orc_bahmani(uint32_t n, const uint64_t* off, const uint32_t* adj, uint64_t p, uint64_t q, uint32_t* peel_round,
                uint64_t* hist_S, uint64_t* hist_E, uint64_t hist_cap, uint64_t* out) {
    if (q == 0) return -3;
    if (hist_cap < 1) return -2;
    uint64_t* deg = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint8_t* alive = (uint8_t*)malloc((size_t)n + 1);
    uint32_t* failed = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!deg || !alive || !failed) { free(deg); free(alive); free(failed); return -1; }
    for (uint32_t v = 0; v < n; ++v) {
        deg[v] = off[v + 1] - off[v];
        alive[v] = 1;
        peel_round[v] = 0;
    }
    uint64_t S = n, E = off[n] / 2;
    uint64_t best_round = 0, bestE = E, bestV = S;
    uint64_t r = 0;
    hist_S[0] = S;
    hist_E[0] = E;
    while (S > 0) {
        /* part 1: threshold test against the round-start degrees */
        uint64_t nf = 0;
        u128 rhs = (u128)2 * ((u128)p + q) * E; /* 2 (p + q) |E| */
        for (uint32_t v = 0; v < n; ++v)
            if (alive[v] && (u128)deg[v] * q * S <= rhs) failed[nf++] = v;
        if (nf == 0) { free(deg); free(alive); free(failed); return -4; } /* a round must remove a vertex */
        /* barrier: only now do the failed vertices leave S */
        for (uint64_t i = 0; i < nf; ++i) {
            alive[failed[i]] = 0;
            peel_round[failed[i]] = (uint32_t)(r + 1);
        }
        /* part 2: drop every edge with an endpoint in the failed set */
        uint64_t removed = 0;
        for (uint64_t i = 0; i < nf; ++i) {
            uint32_t v = failed[i];
            for (uint64_t j = off[v]; j < off[v + 1]; ++j) {
                uint32_t u = adj[j];
                if (alive[u]) { /* survivor: edge (v,u) goes, u loses one degree */
                    deg[u] -= 1;
                    removed += 1;
                } else if (peel_round[u] == r + 1 && u > v) { /* both failed now: count once */
                    removed += 1;
                }
            }
        }
        /* reduce */
        S -= nf;
        E -= removed;
        r += 1;
        if (r >= hist_cap) { free(deg); free(alive); free(failed); return -2; }
        hist_S[r] = S;
        hist_E[r] = E;
        /* keep the densest set seen, strict improvement only */
        if (S > 0 && (u128)E * bestV > (u128)bestE * S) {
            best_round = r;
            bestE = E;
            bestV = S;
        }
    }
    BEST_OUT(out, r, best_round, bestE, bestV);
    free(deg);
    free(alive);
    free(failed);
    return 0;
}

/*
 * The same peel with no incremental state: every round rebuilds the alive
 * set's induced degrees and edge count straight from the adjacency lists.
 * Same outputs and return codes as orc_bahmani.
 */
int orc_bahmani_recompute(uint32_t n, const uint64_t* off, const uint32_t* adj, uint64_t p, uint64_t q,
                          uint32_t* peel_round, uint64_t* hist_S, uint64_t* hist_E, uint64_t hist_cap,
                          uint64_t* out) {
    if (q == 0) return -3;
    if (hist_cap < 1) return -2;
    uint64_t* dS = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint8_t* inS = (uint8_t*)malloc((size_t)n + 1);
    uint8_t* fail = (uint8_t*)malloc((size_t)n + 1);
    if (!dS || !inS || !fail) { free(dS); free(inS); free(fail); return -1; }
    for (uint32_t v = 0; v < n; ++v) { inS[v] = 1; peel_round[v] = 0; }
    uint64_t r = 0, best_round = 0, bestE = 0, bestV = 0;
    for (;;) {
        uint64_t S = 0, twoE = 0;
        for (uint32_t v = 0; v < n; ++v) {
            dS[v] = 0;
            if (!inS[v]) continue;
            ++S;
            for (uint64_t j = off[v]; j < off[v + 1]; ++j) dS[v] += inS[adj[j]];
            twoE += dS[v];
        }
        uint64_t E = twoE / 2;
        if (r >= hist_cap) { free(dS); free(inS); free(fail); return -2; }
        hist_S[r] = S;
        hist_E[r] = E;
        if (r == 0) { bestE = E; bestV = S; }
        else if (S > 0 && (u128)E * bestV > (u128)bestE * S) { best_round = r; bestE = E; bestV = S; }
        if (S == 0) break;
        for (uint32_t v = 0; v < n; ++v)
            fail[v] = inS[v] && ((u128)dS[v] * q * S <= (u128)2 * ((u128)p + q) * E);
        uint64_t nf = 0;
        for (uint32_t v = 0; v < n; ++v)
            if (fail[v]) { inS[v] = 0; peel_round[v] = (uint32_t)(r + 1); ++nf; }
        if (nf == 0) { free(dS); free(inS); free(fail); return -4; } /* a round must remove a vertex */
        ++r;
    }
    BEST_OUT(out, r, best_round, bestE, bestV);
    free(dS);
    free(inS);
    free(fail);
    return 0;
}

/* -------------------------------------------------------------- core numbers */

/*
 * Def. 2: the k-core is the largest subgraph with minimum degree >= k; the
 * core number of v is the largest k whose k-core contains v.
 *
 * Batagelj & Zaversnik, "An O(m) Algorithm for Cores Decomposition of
 * Networks" (2003): vertices kept in an array ordered by current degree,
 * with bucket starts; repeatedly take the vertex of least current degree,
 * fix its core number, and move each neighbour of larger current degree one
 * bucket down.
 */
int orc_kcore_bz(uint32_t n, const uint64_t* off, const uint32_t* adj, uint32_t* core) {
    if (n == 0) return 0;
    uint64_t md = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (off[v + 1] - off[v] > md) md = off[v + 1] - off[v];
    uint64_t* d = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    uint64_t* bin = (uint64_t*)calloc(md + 2, sizeof(uint64_t));
    uint64_t* pos = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
    uint32_t* vert = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!d || !bin || !pos || !vert) { free(d); free(bin); free(pos); free(vert); return -1; }
    for (uint32_t v = 0; v < n; ++v) { d[v] = off[v + 1] - off[v]; bin[d[v]]++; }
    uint64_t start = 0;
    for (uint64_t k = 0; k <= md; ++k) { uint64_t c = bin[k]; bin[k] = start; start += c; }
    for (uint32_t v = 0; v < n; ++v) { pos[v] = bin[d[v]]; vert[pos[v]] = v; bin[d[v]]++; }
    for (uint64_t k = md; k > 0; --k) bin[k] = bin[k - 1];
    bin[0] = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t v = vert[i];
        for (uint64_t j = off[v]; j < off[v + 1]; ++j) {
            uint32_t u = adj[j];
            if (d[u] > d[v]) {
                uint64_t du = d[u], pu = pos[u], pw = bin[du];
                uint32_t w = vert[pw];
                if (u != w) { pos[u] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = u; }
                bin[du]++;
                d[u]--;
            }
        }
    }
    for (uint32_t v = 0; v < n; ++v) core[v] = (uint32_t)d[v];
    free(d); free(bin); free(pos); free(vert);
    return 0;
}

/*
 * Def. 2 by brute repetition: for k = 1, 2, ... delete from the (k-1)-core
 * every vertex whose degree inside the remaining set is below k, repeatedly,
 * until none is left; a vertex deleted while building the k-core has core
 * number k-1.
 */
int orc_kcore_naive(uint32_t n, const uint64_t* off, const uint32_t* adj, uint32_t* core) {
    uint8_t* in = (uint8_t*)malloc((size_t)n + 1);
    uint64_t* d = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!in || !d) { free(in); free(d); return -1; }
    uint64_t left = n;
    for (uint32_t v = 0; v < n; ++v) { in[v] = 1; core[v] = 0; }
    for (uint64_t k = 1; left > 0; ++k) {
        int changed = 1;
        while (changed) {
            changed = 0;
            for (uint32_t v = 0; v < n; ++v) {
                if (!in[v]) continue;
                d[v] = 0;
                for (uint64_t j = off[v]; j < off[v + 1]; ++j) d[v] += in[adj[j]];
            }
            for (uint32_t v = 0; v < n; ++v)
                if (in[v] && d[v] < k) { in[v] = 0; core[v] = (uint32_t)(k - 1); --left; changed = 1; }
        }
    }
    free(in);
    free(d);
    return 0;
}

/*
 * Algorithm 2, first phase (the PKC scheme of Kabir & Madduri), run by one
 * thread.  Level k: buffer every vertex whose current degree equals k; drain
 * the buffer, and for each buffered v and each neighbour u != v with
 * degree above k, take one from u's degree and append u to the buffer when
 * it has just reached k.  (Alone, the undo branch for a degree that already
 * fell to k never fires.)  The level ends when the buffer is drained; the
 * visited count grows by the buffer length; k advances.  At the end each
 * vertex's degree is its core number.
 */
int orc_kcore_pkc(uint32_t n, const uint64_t* off, const uint32_t* adj, uint32_t* core) {
    uint64_t* deg = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t* buff = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!deg || !buff) { free(deg); free(buff); return -1; }
    for (uint32_t v = 0; v < n; ++v) deg[v] = off[v + 1] - off[v];
    uint64_t visited = 0;
    for (uint64_t k = 0; visited < n; ++k) {
        uint64_t start = 0, end = 0;
        for (uint32_t v = 0; v < n; ++v)
            if (deg[v] == k) buff[end++] = v;
        while (start < end) {
            uint32_t v = buff[start++];
            for (uint64_t j = off[v]; j < off[v + 1]; ++j) {
                uint32_t u = adj[j];
                if (u == v || deg[u] <= k) continue;
                uint64_t a = deg[u];
                deg[u] = a - 1;
                if (a == k + 1) buff[end++] = u;
                if (a <= k) deg[u] += 1;
            }
        }
        visited += end;
    }
    for (uint32_t v = 0; v < n; ++v) core[v] = (uint32_t)deg[v];
    free(deg);
    free(buff);
    return 0;
}

/*
 * Densest core (Sec. 3.2 approach: the densest k-core is a 2-approximation,
 * Tatti et al.).  For every k with a non-empty k-core: V_k = #{v : core >= k},
 * E_k = #{edges whose endpoints both have core >= k}; the best k is the one
 * of largest E_k / V_k, the smallest such k on ties (levels are visited in
 * increasing k with a strict comparison).  Algorithm 2 takes a level's
 * density after that level's vertices joined `visited` yet labels it with k;
 * the label is paired here with the k-core {core >= k} itself, the set its
 * second phase compares neighbours against (deg >= max_density_core).
 * out[0] = k*, out[1] = E_k*, out[2] = V_k*.  n == 0 gives zeros.
 */
int orc_densest_core(uint32_t n, const uint64_t* off, const uint32_t* adj, const uint32_t* core, uint64_t* out) {
    out[0] = out[1] = out[2] = 0;
    uint32_t kmax = 0;
    for (uint32_t v = 0; v < n; ++v) if (core[v] > kmax) kmax = core[v];
    int have = 0;
    for (uint64_t k = 0; n > 0 && k <= kmax; ++k) {
        uint64_t V = 0, twoE = 0;
        for (uint32_t v = 0; v < n; ++v) {
            if (core[v] < k) continue;
            ++V;
            for (uint64_t j = off[v]; j < off[v + 1]; ++j) twoE += core[adj[j]] >= k;
        }
        uint64_t E = twoE / 2;
        if (V == 0) continue;
        if (!have || (u128)E * out[2] > (u128)out[1] * V) { out[0] = k; out[1] = E; out[2] = V; have = 1; }
    }
    return 0;
}

/* --------------------------------------------------------- exact densest */

/*
 * Exact densest subgraph by enumeration of all 2^n vertex subsets (n <= 24).
 * out[0] = E*, out[1] = V* of a densest non-empty subset; mask_out (nullable)
 * gets that subset as a bit mask.  The first subset in counting order wins
 * ties.  Graph with no vertex: zeros.
 */
int orc_brute_densest(uint32_t n, const uint64_t* off, const uint32_t* adj, uint64_t* out, uint64_t* mask_out) {
    out[0] = out[1] = 0;
    if (mask_out) *mask_out = 0;
    if (n == 0) return 0;
    if (n > 24) return -1;
    uint32_t nb[24] = {0};
    for (uint32_t v = 0; v < n; ++v)
        for (uint64_t j = off[v]; j < off[v + 1]; ++j) nb[v] |= 1u << adj[j];
    uint64_t bestE = 0, bestV = 0, bestM = 0;
    for (uint32_t s = 1; s < (1u << n); ++s) {
        uint64_t V = (uint64_t)__builtin_popcount(s), twoE = 0;
        for (uint32_t v = 0; v < n; ++v)
            if (s >> v & 1) twoE += (uint64_t)__builtin_popcount(nb[v] & s);
        uint64_t E = twoE / 2;
        if (bestV == 0 || (u128)E * bestV > (u128)bestE * V) { bestE = E; bestV = V; bestM = s; }
    }
    out[0] = bestE;
    out[1] = bestV;
    if (mask_out) *mask_out = bestM;
    return 0;
}

/* Dinic max-flow on a small int64 network (used only by the Goldberg check). */
typedef struct { uint32_t to; int64_t cap; } arc_t;
typedef struct {
    uint32_t nv, na, cap_arcs;
    arc_t* arcs;
    uint32_t* next;   /* next arc out of the same node */
    uint32_t* head;   /* first arc out of each node */
    int32_t* level;
    uint32_t* it;
    uint32_t* queue;
} net_t;

static int net_init(net_t* g, uint32_t nv, uint32_t max_arcs) {
    memset(g, 0, sizeof(*g));
    g->nv = nv;
    g->cap_arcs = max_arcs;
    g->arcs = (arc_t*)malloc((size_t)max_arcs * sizeof(arc_t));
    g->next = (uint32_t*)malloc((size_t)max_arcs * sizeof(uint32_t));
    g->head = (uint32_t*)malloc((size_t)nv * sizeof(uint32_t));
    g->level = (int32_t*)malloc((size_t)nv * sizeof(int32_t));
    g->it = (uint32_t*)malloc((size_t)nv * sizeof(uint32_t));
    g->queue = (uint32_t*)malloc((size_t)nv * sizeof(uint32_t));
    if (!g->arcs || !g->next || !g->head || !g->level || !g->it || !g->queue) return -1;
    for (uint32_t i = 0; i < nv; ++i) g->head[i] = UINT32_MAX;
    return 0;
}

static void net_free(net_t* g) {
    free(g->arcs); free(g->next); free(g->head); free(g->level); free(g->it); free(g->queue);
}

/* arc a -> b with capacity c, and its residual twin b -> a with capacity rc */
static void net_add(net_t* g, uint32_t a, uint32_t b, int64_t c, int64_t rc) {
    uint32_t i = g->na++;
    g->arcs[i].to = b; g->arcs[i].cap = c; g->next[i] = g->head[a]; g->head[a] = i;
    i = g->na++;
    g->arcs[i].to = a; g->arcs[i].cap = rc; g->next[i] = g->head[b]; g->head[b] = i;
}

static int net_bfs(net_t* g, uint32_t s, uint32_t t) {
    for (uint32_t i = 0; i < g->nv; ++i) g->level[i] = -1;
    uint32_t qh = 0, qt = 0;
    g->level[s] = 0;
    g->queue[qt++] = s;
    while (qh < qt) {
        uint32_t x = g->queue[qh++];
        for (uint32_t a = g->head[x]; a != UINT32_MAX; a = g->next[a])
            if (g->arcs[a].cap > 0 && g->level[g->arcs[a].to] < 0) {
                g->level[g->arcs[a].to] = g->level[x] + 1;
                g->queue[qt++] = g->arcs[a].to;
            }
    }
    return g->level[t] >= 0;
}

/* iterative blocking-flow DFS from s; returns the flow pushed along one path */
static int64_t net_dfs(net_t* g, uint32_t s, uint32_t t, uint32_t* stack_node, uint32_t* stack_arc) {
    uint32_t depth = 0;
    stack_node[0] = s;
    for (;;) {
        uint32_t x = stack_node[depth];
        if (x == t) {
            int64_t f = INT64_MAX;
            for (uint32_t i = 0; i < depth; ++i)
                if (g->arcs[stack_arc[i]].cap < f) f = g->arcs[stack_arc[i]].cap;
            for (uint32_t i = 0; i < depth; ++i) {
                g->arcs[stack_arc[i]].cap -= f;
                g->arcs[stack_arc[i] ^ 1u].cap += f;
            }
            return f;
        }
        uint32_t a = g->it[x];
        while (a != UINT32_MAX &&
               !(g->arcs[a].cap > 0 && g->level[g->arcs[a].to] == g->level[x] + 1))
            a = g->next[a];
        g->it[x] = a;
        if (a == UINT32_MAX) {
            if (depth == 0) return 0;
            g->level[x] = -1; /* dead end */
            --depth;
            g->it[stack_node[depth]] = g->next[g->it[stack_node[depth]]];
            continue;
        }
        stack_arc[depth] = a;
        stack_node[++depth] = g->arcs[a].to;
    }
}

static int64_t net_maxflow(net_t* g, uint32_t s, uint32_t t) {
    int64_t flow = 0;
    uint32_t* sn = (uint32_t*)malloc(((size_t)g->nv + 1) * sizeof(uint32_t));
    uint32_t* sa = (uint32_t*)malloc(((size_t)g->nv + 1) * sizeof(uint32_t));
    if (!sn || !sa) { free(sn); free(sa); return -1; }
    while (net_bfs(g, s, t)) {
        for (uint32_t i = 0; i < g->nv; ++i) g->it[i] = g->head[i];
        int64_t f;
        while ((f = net_dfs(g, s, t, sn, sa)) > 0) flow += f;
    }
    free(sn);
    free(sa);
    return flow;
}

/*
 * Exact densest subgraph (Goldberg, "Finding a maximum density subgraph",
 * 1984 -- the paper's ref. [32]).  For a guess g = a/b the network
 *     s -> v : m b,   v -> t : m b + 2a - deg(v) b,   u <-> v : b per edge
 * has minimum cut b m n - 2 max_S (b |E(S)| - a |S|), and the source side of
 * a minimum cut attains the max.  Dinkelbach iteration: start from g = rho(V);
 * while the max is positive, replace g by rho of the maximiser (which is
 * strictly larger); stop at zero.  The final g is rho* exactly.
 * out[0] = E*, out[1] = V*.  mask_out (nullable, n bytes) marks the set.
 * Returns 0, or -1 on allocation failure / capacity overflow.
 */
int orc_goldberg_densest(uint32_t n, const uint64_t* off, const uint32_t* adj, uint64_t* out, uint8_t* mask_out) {
    out[0] = out[1] = 0;
    if (n == 0) return 0;
    uint64_t m = off[n] / 2;
    uint64_t a = m, b = n; /* g = m / n */
    uint8_t* side = (uint8_t*)calloc(n, 1);
    if (!side) return -1;
    if (mask_out) memset(mask_out, 1, n);
    out[0] = m;
    out[1] = n;
    if (m == 0) { free(side); return 0; }
    for (int iter = 0; iter < 10000; ++iter) {
        /* capacities up to m*b + 2a: keep within int64 */
        if ((u128)m * b + 2 * (u128)a >= ((u128)1 << 62)) { free(side); return -1; }
        net_t g;
        uint32_t s = n, t = n + 1;
        if (net_init(&g, n + 2, (uint32_t)(4 * (uint64_t)n + 2 * off[n] + 4)) != 0) {
            net_free(&g); free(side); return -1;
        }
        for (uint32_t v = 0; v < n; ++v) {
            int64_t dv = (int64_t)(off[v + 1] - off[v]);
            net_add(&g, s, v, (int64_t)(m * b), 0);
            net_add(&g, v, t, (int64_t)(m * b + 2 * a) - dv * (int64_t)b, 0);
        }
        for (uint32_t v = 0; v < n; ++v)
            for (uint64_t j = off[v]; j < off[v + 1]; ++j)
                if (adj[j] > v) net_add(&g, v, adj[j], (int64_t)b, (int64_t)b);
        int64_t cut = net_maxflow(&g, s, t);
        if (cut < 0) { net_free(&g); free(side); return -1; }
        /* source side of the min cut: reachable from s in the residual graph */
        net_bfs(&g, s, t);
        uint64_t V = 0, twoE = 0;
        for (uint32_t v = 0; v < n; ++v) side[v] = g.level[v] >= 0;
        for (uint32_t v = 0; v < n; ++v) {
            if (!side[v]) continue;
            ++V;
            for (uint64_t j = off[v]; j < off[v + 1]; ++j) twoE += side[adj[j]];
        }
        net_free(&g);
        uint64_t E = twoE / 2;
        /* value of the maximiser: b E - a V (zero for the empty set) */
        if (V == 0 || (u128)E * b <= (u128)a * V) break;
        a = E;
        b = V;
        out[0] = E;
        out[1] = V;
        if (mask_out) memcpy(mask_out, side, n);
    }
    free(side);
    return 0;
}

/* ------------------------------------------------------- CBDS-P phase two */

/*
 * Algorithm 2, second phase, serial, on the core numbers of the first phase
 * and the densest core (k*, E_k*, V_k*) found by orc_densest_core.
 *
 *   eligible: vertices whose degree value (their core number after phase 1)
 *             lies strictly between the densest core's density and k*
 *   legit count of an eligible v: its neighbours whose core >= k*
 *             (a self-loop would count one half; canonical graphs have none)
 *   legit:    count > density of the densest core; each adds its count to
 *             the running edge total
 *   pairs:    every edge between two legit vertices is added once
 *   result:   m_e = E_k* + counts + legit pairs, m_v = V_k* + #legit
 *
 * Density comparisons are exact: a value x (an integer) exceeds E/V iff
 * x * V > E.  out[0] = m_e, out[1] = m_v, out[2] = #legit.  legit_mask
 * (nullable, n bytes) marks the legit vertices.
 */
int orc_cbds_phase2(uint32_t n, const uint64_t* off, const uint32_t* adj, const uint32_t* core, uint64_t kstar,
                    uint64_t Ek, uint64_t Vk, uint64_t* out, uint8_t* legit_mask) {
    out[0] = Ek; out[1] = Vk; out[2] = 0;
    if (n == 0 || Vk == 0) return 0;
    uint8_t* legit = (uint8_t*)calloc(n, 1);
    if (!legit) return -1;
    uint64_t inter = 0, nleg = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint64_t dv = core[v];
        /* dv > Ek/Vk  and  dv < k* */
        if (!((u128)dv * Vk > Ek && dv < kstar)) continue;
        uint64_t cnt = 0;
        for (uint64_t j = off[v]; j < off[v + 1]; ++j) cnt += core[adj[j]] >= kstar;
        if ((u128)cnt * Vk > Ek) { legit[v] = 1; inter += cnt; ++nleg; }
    }
    for (uint32_t v = 0; v < n; ++v) {
        if (!legit[v]) continue;
        for (uint64_t j = off[v]; j < off[v + 1]; ++j)
            if (adj[j] > v && legit[adj[j]]) ++inter;
    }
    out[0] = Ek + inter;
    out[1] = Vk + nleg;
    out[2] = nleg;
    if (legit_mask) memcpy(legit_mask, legit, n);
    free(legit);
    return 0;
}
