// Batched solve internals shared by dsg_batch_solve and the server: the
// per-graph tables of one block-per-graph launch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dsg {

struct BatchArgs {
    uint32_t G;
    const uint64_t* const* goff;  // per graph: its n+1 row offsets (positions in its gadj)
    const uint32_t* const* gadj;  // per graph: adjacency base
    const uint64_t* slot;         // per graph: first scratch / output slot
    const uint32_t* gn;           // per graph: vertex count
    const uint32_t* p;
    const uint32_t* q;
    const uint8_t* want_core;
    const uint32_t* order;  // graph ids, largest first
    uint32_t* st;           // peel state per vertex slot
    uint32_t* la;           // scratch lists per vertex slot (x3)
    uint32_t* lb;
    uint32_t* lf;
    uint32_t* core;         // core numbers per vertex slot (nullable)
    uint8_t* out_set;       // membership in the densest set found (nullable)
    uint64_t* res;          // 4 per graph: E, V, rounds, best_round
    unsigned long long* next;
    uint32_t hot_deg;
    unsigned long long* stats;  // nullable, 3 counters summed over the batch: sum over graphs and rounds of
                                // |S_r|, alive-neighbour decrements of the peels, adjacency entries scanned
};


// Launch the block-per-graph kernel over a.order[0, a.G) on stream s
// (asynchronous) with `block` threads per block (256, 512 or 1024; 0: 512),
// at most max_grid blocks (0: as many as fit).  a.next must be zeroed and
// every table filled.
cudaError_t batch_launch(const BatchArgs& a, cudaStream_t s, uint32_t block = 0, uint32_t max_grid = 0);

// Blocks of `block` threads the block-per-graph kernel can keep resident on the GPU.
uint32_t batch_slots_for(uint32_t block);

}  // namespace dsg
