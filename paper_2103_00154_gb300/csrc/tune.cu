// Tuning knobs of the round kernels: defaults, environment overrides and the
// setter used by the autotuner.
#include <stdlib.h>

#include <mutex>

#include "dsg_common.cuh"
#include "dsg_kernels.cuh"

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

extern "C" dsg_status dsg_get_tuning(uint32_t* block, uint32_t* blocks_per_sm, uint32_t* short_max,
                                     uint32_t* chunk_len) {
    Tuning t = current_tuning();
    if (block) *block = t.block;
    if (blocks_per_sm) *blocks_per_sm = t.blocks_per_sm;
    if (short_max) *short_max = t.short_max;
    if (chunk_len) *chunk_len = t.chunk_len;
    return DSG_OK;
}
