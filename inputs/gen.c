/*
 * Seeded synthetic graph generators (raw undirected edge pairs).
 *
 * These produce INPUTS only: raw (src, dst) pairs that may contain
 * self-loops, duplicates and both orientations of an edge.  They hold none
 * of the densest-subgraph method's arithmetic; canonicalisation (dropping
 * loops, dedup, symmetrisation) is the job of the ingest step on each side.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator.  Draw i of stream k is mix(key(seed, k) + (i + 1) * GAMMA), so
 * every value depends only on (seed, stream, index) and the threaded
 * generators give the same bytes for any thread count and on any machine.
 *
 * Build with -ffp-contract=off so the few floating-point steps (quadrant
 * choice, alias tables) round the same way on x86-64 and AArch64.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of stream `k` under `seed`: two rounds of the finaliser so that
 * neighbouring seeds and streams land far apart. */
static inline uint64_t stream_key(uint64_t seed, uint64_t k) {
    return mix64(mix64(seed ^ 0x6A09E667F3BCC909ULL) + k * 0xD1B54A32D192ED03ULL);
}

static inline uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GAMMA); }

/* uniform double in [0, 1) from the top 53 bits */
static inline double unit(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

/* uniform integer in [0, n) by multiply-high (Lemire) */
static inline uint32_t below(uint64_t x, uint32_t n) {
    return (uint32_t)(((unsigned __int128)x * n) >> 64);
}

uint64_t gen_draw(uint64_t seed, uint64_t stream, uint64_t i) { return draw(stream_key(seed, stream), i); }

/* ---------------------------------------------------------------- threads */

typedef struct {
    void (*fn)(void*, uint64_t, uint64_t);
    void* ctx;
    uint64_t lo, hi;
} span_t;

static void* span_main(void* a) {
    span_t* s = (span_t*)a;
    s->fn(s->ctx, s->lo, s->hi);
    return NULL;
}

/* Run fn(ctx, lo, hi) over [0, total) split into `threads` contiguous spans. */
static void parallel_for(uint64_t total, int threads, void (*fn)(void*, uint64_t, uint64_t), void* ctx) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if ((uint64_t)threads > total / 65536 + 1) threads = (int)(total / 65536 + 1);
    pthread_t tid[256];
    span_t sp[256];
    for (int t = 0; t < threads; ++t) {
        sp[t].fn = fn;
        sp[t].ctx = ctx;
        sp[t].lo = total * (uint64_t)t / (uint64_t)threads;
        sp[t].hi = total * (uint64_t)(t + 1) / (uint64_t)threads;
    }
    int joined[256] = {0};
    for (int t = 1; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, span_main, &sp[t]) == 0) joined[t] = 1;
        else span_main(&sp[t]); /* no thread available: run the span inline */
    }
    span_main(&sp[0]);
    for (int t = 1; t < threads; ++t)
        if (joined[t]) pthread_join(tid[t], NULL);
}

/* ------------------------------------------------ Erdos-Renyi G(n, m) */

/* m distinct non-loop unordered pairs drawn uniformly without replacement:
 * pairs are drawn in counter order and a pair already taken (in either
 * orientation) or a loop is skipped.  Serial by construction.
 * Returns the number of pairs written (m, or fewer if m exceeds n(n-1)/2). */
uint64_t gen_er(uint32_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst) {
    if (n < 2) return 0;
    uint64_t maxm = (uint64_t)n * (n - 1) / 2;
    if (m > maxm) m = maxm;
    uint64_t cap = 1;
    while (cap < 2 * m + 16) cap <<= 1;
    uint64_t* table = (uint64_t*)malloc(cap * sizeof(uint64_t));
    if (!table) return 0;
    memset(table, 0xff, cap * sizeof(uint64_t));
    uint64_t key = stream_key(seed, 1);
    uint64_t got = 0;
    for (uint64_t i = 0; got < m; ++i) {
        uint32_t u = below(draw(key, 2 * i), n);
        uint32_t v = below(draw(key, 2 * i + 1), n);
        if (u == v) continue;
        uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
        uint64_t k = (lo << 32) | hi;
        uint64_t h = mix64(k) & (cap - 1);
        int dup = 0;
        while (table[h] != ~0ULL) {
            if (table[h] == k) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        table[h] = k;
        src[got] = u;
        dst[got] = v;
        ++got;
    }
    free(table);
    return got;
}

/* m pairs drawn uniformly WITH replacement (loops and repeats possible;
 * ingest drops them).  Threaded. */
typedef struct {
    uint32_t n;
    uint64_t key;
    uint32_t *src, *dst;
} erf_ctx;

static void erf_span(void* c, uint64_t lo, uint64_t hi) {
    erf_ctx* x = (erf_ctx*)c;
    for (uint64_t i = lo; i < hi; ++i) {
        x->src[i] = below(draw(x->key, 2 * i), x->n);
        x->dst[i] = below(draw(x->key, 2 * i + 1), x->n);
    }
}

void gen_er_pairs(uint32_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst, int threads) {
    erf_ctx x = {n ? n : 1, stream_key(seed, 6), src, dst};
    parallel_for(m, threads, erf_span, &x);
}

/* ------------------------------------------------------- planted block */

/* Block = the first k vertices of a seeded Fisher-Yates permutation of
 * [0, n); every pair inside the block is kept independently with
 * probability p.  Writes at most `cap` pairs; returns the count (or the
 * count it would have written, if larger than cap). */
uint64_t gen_block(uint32_t n, uint32_t k, double p, uint64_t seed, uint32_t* src, uint32_t* dst, uint64_t cap) {
    if (k > n) k = n;
    uint32_t* perm = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    if (!perm) return 0;
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    uint64_t key = stream_key(seed, 2);
    for (uint32_t i = 0; i < k; ++i) { /* partial shuffle: positions 0..k-1 */
        uint32_t j = i + below(draw(key, i), n - i);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    uint64_t key2 = stream_key(seed, 3);
    uint64_t got = 0, idx = 0;
    for (uint32_t i = 0; i < k; ++i)
        for (uint32_t j = i + 1; j < k; ++j, ++idx)
            if (unit(draw(key2, idx)) < p) {
                if (got < cap) { src[got] = perm[i]; dst[got] = perm[j]; }
                ++got;
            }
    free(perm);
    return got;
}

/* ---------------------------------------------------------------- R-MAT */

typedef struct {
    uint32_t scale;
    double a, ab, abc;
    uint64_t key;
    uint32_t *src, *dst;
} rmat_ctx;

static void rmat_span(void* c, uint64_t lo, uint64_t hi) {
    rmat_ctx* x = (rmat_ctx*)c;
    for (uint64_t e = lo; e < hi; ++e) {
        uint32_t s = 0, d = 0;
        for (uint32_t l = 0; l < x->scale; ++l) {
            double u = unit(draw(x->key, e * x->scale + l));
            uint32_t bs = 0, bd = 0;
            if (u < x->a) { bs = 0; bd = 0; }
            else if (u < x->ab) { bs = 0; bd = 1; }
            else if (u < x->abc) { bs = 1; bd = 0; }
            else { bs = 1; bd = 1; }
            s = (s << 1) | bs;
            d = (d << 1) | bd;
        }
        x->src[e] = s;
        x->dst[e] = d;
    }
}

/* m R-MAT draws over 2^scale vertices, quadrant probabilities (a, b, c, 1-a-b-c),
 * one uniform per recursion level.  No vertex relabelling. */
void gen_rmat(uint32_t scale, uint64_t m, double a, double b, double c, uint64_t seed, uint32_t* src, uint32_t* dst,
              int threads) {
    rmat_ctx x = {scale, a, a + b, a + b + c, stream_key(seed, 4), src, dst};
    parallel_for(m, threads, rmat_span, &x);
}

/* ----------------------------------------------------------- Chung-Lu */

/* Weights w_i = C (i + i0)^(-1/(gamma-1)), i = 0..n-1, with i0 chosen by
 * bisection so that w_0 / mean(w) = wmax / mean and C so that mean(w) = mean.
 * If wmax <= 0 the structural cut-off sqrt(n * mean) is used for wmax. */
int gen_chung_lu_weights(uint32_t n, double gamma, double mean, double wmax, double* w) {
    if (n == 0) return 0;
    double beta = 1.0 / (gamma - 1.0);
    if (wmax <= 0) wmax = sqrt((double)n * mean);
    double target = wmax / mean;
    double lo = 1e-6, hi = 1e12;
    for (int it = 0; it < 200; ++it) {
        double mid = sqrt(lo * hi);
        double s = 0;
        for (uint32_t i = 0; i < n; ++i) s += pow((double)i + mid, -beta);
        double r = pow(mid, -beta) / (s / (double)n);
        if (r > target) lo = mid; else hi = mid;
    }
    double i0 = lo, s = 0;
    for (uint32_t i = 0; i < n; ++i) { w[i] = pow((double)i + i0, -beta); s += w[i]; }
    double scalef = mean * (double)n / s;
    for (uint32_t i = 0; i < n; ++i) {
        w[i] *= scalef;
        if (w[i] > wmax) w[i] = wmax;
    }
    return 0;
}

typedef struct {
    uint32_t n;
    const double* prob;
    const uint32_t* alias;
    uint64_t key;
    uint32_t *src, *dst;
} cl_ctx;

static inline uint32_t alias_pick(const cl_ctx* x, uint64_t i) {
    uint32_t j = below(draw(x->key, 2 * i), x->n);
    double u = unit(draw(x->key, 2 * i + 1));
    return u < x->prob[j] ? j : x->alias[j];
}

static void cl_span(void* c, uint64_t lo, uint64_t hi) {
    cl_ctx* x = (cl_ctx*)c;
    for (uint64_t e = lo; e < hi; ++e) {
        x->src[e] = alias_pick(x, 2 * e);
        x->dst[e] = alias_pick(x, 2 * e + 1);
    }
}

/* m_draws pairs whose endpoints are drawn independently with probability
 * proportional to the Chung-Lu weights (Walker/Vose alias method). */
int gen_chung_lu(uint32_t n, uint64_t m_draws, double gamma, double mean, double wmax, uint64_t seed, uint32_t* src,
                 uint32_t* dst, int threads) {
    if (n == 0) return 0;
    double* w = (double*)malloc((size_t)n * sizeof(double));
    double* prob = (double*)malloc((size_t)n * sizeof(double));
    uint32_t* alias = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t* small = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t* large = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!w || !prob || !alias || !small || !large) {
        free(w); free(prob); free(alias); free(small); free(large);
        return -1;
    }
    gen_chung_lu_weights(n, gamma, mean, wmax, w);
    double s = 0;
    for (uint32_t i = 0; i < n; ++i) s += w[i];
    uint32_t ns = 0, nl = 0;
    for (uint32_t i = 0; i < n; ++i) {
        prob[i] = w[i] * (double)n / s;
        alias[i] = i;
        if (prob[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns && nl) {
        uint32_t l = small[--ns], g = large[nl - 1];
        alias[l] = g;
        prob[g] = (prob[g] + prob[l]) - 1.0;
        if (prob[g] < 1.0) { --nl; small[ns++] = g; }
    }
    while (nl) prob[large[--nl]] = 1.0;
    while (ns) prob[small[--ns]] = 1.0;
    cl_ctx x = {n, prob, alias, stream_key(seed, 5), src, dst};
    parallel_for(m_draws, threads, cl_span, &x);
    free(w); free(prob); free(alias); free(small); free(large);
    return 0;
}
