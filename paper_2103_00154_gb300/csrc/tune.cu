// Tuning knobs of the round kernels: defaults, environment overrides and the
// setter used by the autotuner.
#include <stdlib.h>

#include <mutex>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

extern "C" dsg_status dsg_tune_save(const char* path);

namespace dsg {

static std::mutex g_tune_mu;
static Tuning g_tune;
static bool g_tune_set = false;

static uint32_t env_u32(const char* name, uint32_t dflt) {
    const char* e = getenv(name);
    if (!e || !*e) return dflt;
    return (uint32_t)strtoul(e, nullptr, 10);
}

Tuning current_tuning() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune_set) {
        Tuning t;
        t.block = env_u32("DSG_BLOCK", t.block);
        t.blocks_per_sm = env_u32("DSG_BLOCKS_PER_SM", t.blocks_per_sm);
        t.short_max = env_u32("DSG_SHORT_MAX", t.short_max);
        t.chunk_len = env_u32("DSG_CHUNK_LEN", t.chunk_len);
        t.hot_deg = env_u32("DSG_HOT_DEG", t.hot_deg);
        t.local_max = env_u32("DSG_LOCAL_MAX", t.local_max);
        t.local_work = env_u32("DSG_LOCAL_WORK", t.local_work);
        t.inline_max = env_u32("DSG_INLINE_MAX", t.inline_max);
        t.tail_max = env_u32("DSG_KCORE_TAIL", t.tail_max);
        t.batch_split = env_u32("DSG_BATCH_SPLIT", t.batch_split);
        t.peel_lazy = env_u32("DSG_PEEL_LAZY", t.peel_lazy) ? 1u : 0u;
        t.peel_vec = env_u32("DSG_PEEL_VEC", t.peel_vec) ? 1u : 0u;
        if (t.tail_max > kTailMaxVertices) t.tail_max = kTailMaxVertices;
        if (t.block != 256 && t.block != 512 && t.block != 1024) t.block = 512;
        if (t.chunk_len < 32) t.chunk_len = 32;
        if (t.short_max < 1) t.short_max = 1;
        g_tune = t;
        g_tune_set = true;
    }
    return g_tune;
}

}  // namespace dsg

using namespace dsg;

extern "C" dsg_status dsg_set_tuning(uint32_t block, uint32_t blocks_per_sm, uint32_t short_max, uint32_t chunk_len) {
    clear_error();
    DSG_CHECK_ARG(block == 256 || block == 512 || block == 1024, "block must be 256, 512 or 1024");
    DSG_CHECK_ARG(chunk_len >= 32 && chunk_len <= (1u << 20), "chunk_len must be in [32, 2^20]");
    DSG_CHECK_ARG(short_max >= 1 && short_max <= 4096, "short_max must be in [1, 4096]");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.block = block;
    g_tune.blocks_per_sm = blocks_per_sm;
    g_tune.short_max = short_max;
    g_tune.chunk_len = chunk_len;
    g_tune_set = true;
    return DSG_OK;
}

extern "C" dsg_status dsg_set_hot_degree(uint32_t hot_deg) {
    clear_error();
    current_tuning();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.hot_deg = hot_deg;
    return DSG_OK;
}

extern "C" dsg_status dsg_set_local_max(uint32_t local_max, uint32_t local_work) {
    clear_error();
    current_tuning();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.local_max = local_max;
    g_tune.local_work = local_work;
    return DSG_OK;
}

extern "C" dsg_status dsg_set_inline_max(uint32_t inline_max) {
    clear_error();
    current_tuning();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.inline_max = inline_max;
    return DSG_OK;
}

extern "C" dsg_status dsg_set_kcore_tail(uint32_t max_vertices) {
    clear_error();
    DSG_CHECK_ARG(max_vertices <= kTailMaxVertices, "max_vertices must be at most 131072");
    current_tuning();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.tail_max = max_vertices;
    return DSG_OK;
}

extern "C" dsg_status dsg_set_peel_lazy(uint32_t on) {
    clear_error();
    current_tuning();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.peel_lazy = on ? 1u : 0u;
    return DSG_OK;
}

extern "C" dsg_status dsg_set_peel_vec(uint32_t on) {
    clear_error();
    current_tuning();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.peel_vec = on ? 1u : 0u;
    return DSG_OK;
}

extern "C" dsg_status dsg_set_batch_split(uint32_t min_work) {
    clear_error();
    current_tuning();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.batch_split = min_work;
    return DSG_OK;
}

extern "C" dsg_status dsg_get_tuning(uint32_t* block, uint32_t* blocks_per_sm, uint32_t* short_max,
                                     uint32_t* chunk_len) {
    Tuning t = current_tuning();
    if (block) *block = t.block;
    if (blocks_per_sm) *blocks_per_sm = t.blocks_per_sm;
    if (short_max) *short_max = t.short_max;
    if (chunk_len) *chunk_len = t.chunk_len;
    return DSG_OK;
}

// ===================================================================== autotuner
//
// Launch parameters are picked per (device, kernel, graph-size class): the
// class of a graph is (floor(log2 n), floor(log2 2m)).  dsg_autotune times
// candidate settings on a given graph by coordinate descent (one knob at a
// time, keeping a change only when it is at least 2% faster) and records the
// winner for the graph's class; solves on graphs of a tuned class use it.
// The table can be saved to / loaded from a small JSON file, and is loaded
// from DSG_TUNE_FILE at first use.
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <vector>

namespace dsg {

static std::map<std::string, Tuning> g_table;
static std::map<std::string, double> g_table_ms;
static bool g_table_loaded = false;
static thread_local const Tuning* g_forced = nullptr;

static int ilog2(uint64_t x) {
    int l = 0;
    while (x > 1) { x >>= 1; ++l; }
    return l;
}

static std::string device_key() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
    char buf[320];
    snprintf(buf, sizeof(buf), "%s/%d", pr.name, pr.multiProcessorCount);
    return buf;
}

static std::string class_key(const dsg_graph* g, int kernel) {
    char buf[400];
    snprintf(buf, sizeof(buf), "%s|%s|%d:%d", device_key().c_str(), kernel == 0 ? "peel" : "kcore", ilog2(g->n),
             ilog2(2 * g->m));
    return buf;
}

static bool parse_u32(const char* obj, const char* name, uint32_t* out) {
    char pat[64];
    snprintf(pat, sizeof(pat), "\"%s\":", name);
    const char* p = strstr(obj, pat);
    if (!p) return false;
    *out = (uint32_t)strtoul(p + strlen(pat), nullptr, 10);
    return true;
}

static int load_table_locked(const char* path) {
    FILE* f = fopen(path, "rb");
    if (!f) return -1;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, k);
    fclose(f);
    int loaded = 0;
    size_t pos = 0;
    while ((pos = text.find("{\"key\": \"", pos)) != std::string::npos) {
        size_t ks = pos + 9, ke = text.find('"', ks);
        size_t oe = text.find('}', ke);
        if (ke == std::string::npos || oe == std::string::npos) break;
        std::string key = text.substr(ks, ke - ks);
        std::string obj = text.substr(ke, oe - ke);
        Tuning t;
        parse_u32(obj.c_str(), "block", &t.block);
        parse_u32(obj.c_str(), "blocks_per_sm", &t.blocks_per_sm);
        parse_u32(obj.c_str(), "short_max", &t.short_max);
        parse_u32(obj.c_str(), "chunk_len", &t.chunk_len);
        parse_u32(obj.c_str(), "hot_deg", &t.hot_deg);
        parse_u32(obj.c_str(), "local_max", &t.local_max);
        parse_u32(obj.c_str(), "local_work", &t.local_work);
        parse_u32(obj.c_str(), "inline_max", &t.inline_max);
        parse_u32(obj.c_str(), "kcore_tail", &t.tail_max);
        parse_u32(obj.c_str(), "batch_split", &t.batch_split);
        parse_u32(obj.c_str(), "batch_block", &t.batch_block);
        if (t.batch_block != 256 && t.batch_block != 512 && t.batch_block != 1024) t.batch_block = 512;
        if (t.tail_max > kTailMaxVertices) t.tail_max = kTailMaxVertices;
        if ((t.block == 256 || t.block == 512 || t.block == 1024) && t.chunk_len >= 32 && t.short_max >= 1) {
            g_table[key] = t;
            ++loaded;
        }
        pos = oe;
    }
    return loaded;
}

static void ensure_table_loaded_locked() {
    if (g_table_loaded) return;
    g_table_loaded = true;
    const char* e = getenv("DSG_TUNE_FILE");
    if (e && *e) load_table_locked(e);
}

Tuning tuning_for(const dsg_graph* g, int kernel) {
    if (g_forced) return *g_forced;
    Tuning base = current_tuning();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    ensure_table_loaded_locked();
    if (g_table.empty()) return base;
    auto it = g_table.find(class_key(g, kernel));
    return it == g_table.end() ? base : it->second;
}

// Autotuned solve times (ms) of g's size class, when both kernels were tuned.
bool tuned_times(const dsg_graph* g, double* peel_ms, double* core_ms) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto a = g_table_ms.find(class_key(g, 0));
    auto b = g_table_ms.find(class_key(g, 1));
    if (a == g_table_ms.end() || b == g_table_ms.end()) return false;
    *peel_ms = a->second;
    *core_ms = b->second;
    return true;
}


static std::string batch_key(uint32_t G, uint64_t work) {
    char buf[400];
    snprintf(buf, sizeof(buf), "%s|batch|%d:%d", device_key().c_str(), ilog2(G), ilog2(work));
    return buf;
}

Tuning tuning_for_batch(uint32_t G, uint64_t work) {
    if (g_forced) return *g_forced;
    Tuning base = current_tuning();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    ensure_table_loaded_locked();
    auto it = g_table.find(batch_key(G, work));
    return it == g_table.end() ? base : it->second;
}

// Device time of one solve with tuning t forced (best of `reps`), or a negative
// value if the solve failed.  flush (nullable): flush_bytes written before
// each solve, so every timed solve starts with a cold L2 like a first solve.
static double time_solve(const dsg_graph* g, int kernel, uint32_t p, uint32_t q, const Tuning& t, uint32_t* core,
                         int reps, void* flush, size_t flush_bytes) {
    g_forced = &t;
    double best = -1;
    for (int r = 0; r < reps; ++r) {
        if (flush) cudaMemsetAsync(flush, r & 0xff, flush_bytes, g->stream);
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, g->stream);
        dsg_status st;
        if (kernel == 0) {
            uint64_t out4[4];
            st = peel_into(g, p, q, nullptr, out4);
        } else {
            st = run_kcore(g, core, nullptr, 0, nullptr, 0, nullptr);
        }
        cudaEventRecord(b, g->stream);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (st != DSG_OK) {
            best = -1;
            break;
        }
        if (best < 0 || ms < best) best = ms;
    }
    g_forced = nullptr;
    return best;
}

}  // namespace dsg

extern "C" dsg_status dsg_autotune(const dsg_graph* g, uint32_t eps_num, uint32_t eps_den, uint32_t what,
                                   uint32_t* trials_out) {
    clear_error();
    DSG_CHECK_ARG(g, "graph is NULL");
    DSG_CHECK_ARG(eps_den != 0, "eps_den must be positive");
    DSG_TRY_CUDA(cudaSetDevice(g->device));
    uint32_t trials = 0;
    uint32_t* core = nullptr;
    if (what & 2) DSG_TRY_CUDA(dev_alloc((void**)&core, ((size_t)g->n + 1) * 4, g->stream));
    // a buffer of twice the L2 to write before each timed solve (none if it cannot be had:
    // then the solves are timed warm)
    void* flush = nullptr;
    const size_t flush_bytes = 2 * (size_t)dev_info().l2_bytes;
    if (flush_bytes && dev_alloc(&flush, flush_bytes, g->stream) != cudaSuccess) {
        flush = nullptr;
        cudaGetLastError();
    }
    auto release = [&]() {
        if (core) dev_free(core, g->stream);
        if (flush) dev_free(flush, g->stream);
    };
    for (int kernel = 0; kernel < 2; ++kernel) {
        if (!(what & (1u << kernel))) continue;
        Tuning best = tuning_for(g, kernel);
        double t_best = time_solve(g, kernel, eps_num, eps_den, best, core, 3, flush, flush_bytes);
        ++trials;
        if (t_best < 0) {
            release();
            return DSG_ECUDA;
        }
        struct Knob {
            uint32_t Tuning::*field;
            uint32_t values[4];
            int count;
        };
        const Knob peel_knobs[] = {{&Tuning::block, {256, 512, 1024}, 3},
                                   {&Tuning::hot_deg, {0, 1024, 4096, 16384}, 4},
                                   {&Tuning::chunk_len, {128, 256, 1024}, 3},
                                   {&Tuning::short_max, {16, 32, 64}, 3}};
        const Knob core_knobs[] = {{&Tuning::block, {256, 512, 1024}, 3},
                                   {&Tuning::local_max, {256, 1024, 4096}, 3},
                                   {&Tuning::local_work, {4096, 16384, 65536}, 3},
                                   {&Tuning::inline_max, {256, 1024, 4096, 16384}, 4},
                                   {&Tuning::chunk_len, {256, 1024, 2048}, 3},
                                   {&Tuning::tail_max, {0, 16384, 32768, 131072}, 4}};
        const Knob* knobs = kernel == 0 ? peel_knobs : core_knobs;
        const int nknobs = kernel == 0 ? 4 : 6;
        for (int kk = 0; kk < nknobs; ++kk) {
            for (int vi = 0; vi < knobs[kk].count; ++vi) {
                Tuning cand = best;
                cand.*(knobs[kk].field) = knobs[kk].values[vi];
                if (cand.*(knobs[kk].field) == best.*(knobs[kk].field)) continue;
                double t = time_solve(g, kernel, eps_num, eps_den, cand, core, 3, flush, flush_bytes);
                ++trials;
                if (t >= 0 && t < 0.98 * t_best) {
                    best = cand;
                    t_best = t;
                }
            }
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        ensure_table_loaded_locked();
        std::string key = class_key(g, kernel);
        g_table[key] = best;
        g_table_ms[key] = t_best;
    }
    release();
    cudaStreamSynchronize(g->stream);
    if (trials_out) *trials_out = trials;
    const char* e = getenv("DSG_TUNE_FILE");
    if (e && *e) dsg_tune_save(e);
    return DSG_OK;
}

extern "C" dsg_status dsg_tune_save(const char* path) {
    clear_error();
    DSG_CHECK_ARG(path, "path is NULL");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    ensure_table_loaded_locked();
    std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) {
        set_error("tune_save: cannot write %s", path);
        return DSG_EINVAL;
    }
    fprintf(f, "{\"dsg_tuning\": 1, \"entries\": [\n");
    size_t i = 0;
    for (auto& kv : g_table) {
        const Tuning& t = kv.second;
        auto ms = g_table_ms.find(kv.first);
        fprintf(f,
                "  {\"key\": \"%s\", \"block\": %u, \"blocks_per_sm\": %u, \"short_max\": %u, \"chunk_len\": %u, "
                "\"hot_deg\": %u, \"local_max\": %u, \"local_work\": %u, \"inline_max\": %u, \"kcore_tail\": %u, "
                "\"batch_split\": %u, \"batch_block\": %u, \"ms\": %.4f}%s\n",
                kv.first.c_str(), t.block, t.blocks_per_sm, t.short_max, t.chunk_len, t.hot_deg, t.local_max,
                t.local_work, t.inline_max, t.tail_max, t.batch_split, t.batch_block,
                ms == g_table_ms.end() ? -1.0 : ms->second,
                ++i < g_table.size() ? "," : "");
    }
    fprintf(f, "]}\n");
    fclose(f);
    if (rename(tmp.c_str(), path) != 0) {
        set_error("tune_save: cannot move %s into place", tmp.c_str());
        return DSG_EINVAL;
    }
    return DSG_OK;
}

extern "C" dsg_status dsg_tune_load(const char* path, uint32_t* entries) {
    clear_error();
    DSG_CHECK_ARG(path, "path is NULL");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table_loaded = true;
    int k = load_table_locked(path);
    if (k < 0) {
        set_error("tune_load: cannot read %s", path);
        return DSG_EINVAL;
    }
    if (entries) *entries = (uint32_t)k;
    return DSG_OK;
}

extern "C" void dsg_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table.clear();
    g_table_ms.clear();
    g_table_loaded = true;
}

extern "C" uint32_t dsg_tune_entries(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (uint32_t)g_table.size();
}

extern "C" dsg_status dsg_tune_lookup(const dsg_graph* g, uint32_t kernel, uint32_t out[9]) {
    clear_error();
    DSG_CHECK_ARG(g && out, "graph or out is NULL");
    DSG_CHECK_ARG(kernel <= 1, "kernel must be 0 (peel) or 1 (core numbers)");
    const Tuning t = tuning_for(g, (int)kernel);
    const uint32_t v[9] = {t.block,   t.blocks_per_sm, t.short_max,  t.chunk_len, t.hot_deg,
                           t.local_max, t.local_work,  t.inline_max, t.tail_max};
    memcpy(out, v, sizeof(v));
    return DSG_OK;
}

// Batches: coordinate descent over the block-per-graph kernel's block size,
// the hub threshold and the split between the grid-wide kernels and the
// block-per-graph launch, timing whole dsg_batch_solve calls on the caller's
// batch (results discarded); the winner is kept for the batch's class
// (device, floor(log2 G), floor(log2 sum of 2m + n)).
extern "C" dsg_status dsg_batch_autotune(const dsg_batch* b, uint32_t* trials_out) {
    clear_error();
    DSG_CHECK_ARG(b && b->vtx_base && b->off, "batch is NULL");
    const uint32_t G = b->num_graphs;
    if (G == 0) return DSG_OK;
    std::vector<uint64_t> vb(G + 1);
    DSG_TRY_CUDA(copy_any(vb.data(), b->vtx_base, (G + 1) * sizeof(uint64_t), nullptr));
    uint64_t total = 0;
    DSG_TRY_CUDA(copy_any(&total, b->off + vb[G], sizeof(uint64_t), nullptr));
    DSG_TRY_CUDA(cudaDeviceSynchronize());
    const uint64_t work = total + vb[G];
    std::vector<uint64_t> E(G), V(G);
    dsg_batch_result r;
    memset(&r, 0, sizeof(r));
    r.E = E.data();
    r.V = V.data();
    uint32_t trials = 0;
    auto time_one = [&](const Tuning& t) -> double {
        g_forced = &t;
        double best = -1;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, nullptr);
            dsg_status st = dsg_batch_solve(b, &r, nullptr);
            cudaEventRecord(e1, nullptr);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (st != DSG_OK) {
                best = -1;
                break;
            }
            if (best < 0 || ms < best) best = ms;
        }
        g_forced = nullptr;
        ++trials;
        return best;
    };
    Tuning best = tuning_for_batch(G, work);
    double t_best = time_one(best);
    if (t_best < 0) return DSG_ECUDA;
    struct Knob {
        uint32_t Tuning::*field;
        uint32_t values[4];
        int count;
    };
    const Knob knobs[] = {{&Tuning::batch_block, {256, 512, 1024}, 3},
                          {&Tuning::hot_deg, {0, 1024, 16384}, 3},
                          {&Tuning::batch_split, {0, 1u << 22, 0xffffffffu}, 3}};
    for (const Knob& k : knobs) {
        for (int vi = 0; vi < k.count; ++vi) {
            Tuning cand = best;
            cand.*(k.field) = k.values[vi];
            if (cand.*(k.field) == best.*(k.field)) continue;
            const double t = time_one(cand);
            if (t >= 0 && t < 0.98 * t_best) {
                best = cand;
                t_best = t;
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        ensure_table_loaded_locked();
        const std::string key = batch_key(G, work);
        g_table[key] = best;
        g_table_ms[key] = t_best;
    }
    if (trials_out) *trials_out = trials;
    const char* e = getenv("DSG_TUNE_FILE");
    if (e && *e) dsg_tune_save(e);
    return DSG_OK;
}
