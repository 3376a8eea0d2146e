// st_kernels.cuh -- launch interface between the host runtime and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "st_device.cuh"

namespace st {

// counters (same order as st_counters)
enum {
    C_PAIRS = 0, C_TRIPLETS, C_EXT_OK, C_CANDS, C_KEPT, C_UV_INIT, C_UV_CANDS, C_SEEDS,
    C_MATCH_PAIRS, C_MATCH_PRESEL, C_MATCHED, C_HITS, C_EVENTS, C_MATCH_EVAL, C_N
};

struct BuildArgs {
    int64_t n_events;
    const int64_t* ev_off;
    const float* x;
    const int32_t* zone;
    const float* z;       // may be null
    const float* dxdy;    // may be null
    int32_t max_hits;
    int32_t bins;         // buckets per container slot (power of two)
    int32_t smem_hits;    // per-hit arrays in shared memory up to this many hits
    int64_t cont_cap;     // entries of cx / corig
    float* cx;            // container x
    int32_t* corig;       // container: event-local hit index
    int32_t* zoff;        // [n_events * 25]
    int32_t* status;      // [n_events]
    uint8_t* big;         // per-CTA per-hit arrays for larger events
    int64_t big_stride;   // bytes per CTA
    int32_t* item_class;  // [2 n_events] cost class of each (event, half) seeding item
    int32_t* class_count; // [128] items per class, zero before the launch
    int32_t* class_fill;  // [128] places taken per class, zero before the launch
    int32_t* order;       // [2 n_events] the seeding items, costliest class first
    int32_t* zero2 = nullptr;  // [2 n_events] cleared by k_order (fused matching's counters), may be null
    int32_t* queue;
    unsigned long long* counters;
};

struct SeedArgs {
    int64_t n_events;
    const int64_t* ev_off;
    const float* cx;
    const int32_t* corig;
    const int32_t* zoff;
    int32_t* status;
    int32_t smem_hits;    // hits of a half staged in shared memory up to this
    int32_t cand_cap;     // candidates per work item
    int32_t tbl_smem;     // clone table entries in shared memory
    int32_t key_smem;     // UV keys in shared memory
    uint8_t* slot;        // per-CTA scratch
    int64_t slot_stride;  // bytes per CTA
    int32_t max_xhits;    // size of the per-CTA clone table in scratch
    // staging pool of seed records
    int32_t* pool_hits;
    float* pool_params;
    float* pool_state;
    int8_t* pool_n;
    int64_t pool_cap;
    unsigned long long* pool_ctr;
    int32_t* item_start;
    int32_t* item_count;
    const int32_t* order;  // the order k_build gave the items
    int32_t* queue;
    unsigned long long* counters;
    // matching fused into the seeding kernel (velo null: seeding only): the
    // CTA that finishes an event's second half matches the event, or near
    // the end announces it for CTAs without seeding work
    const int64_t* velo_off = nullptr;
    const float* velo = nullptr;
    int32_t velo_smem = 0;
    int32_t defer_match = 0;       // near the end, leave matching to CTAs without seeding work
    int32_t* ev_done = nullptr;    // [n_events] halves finished; zero before the launch
    int32_t* ready = nullptr;      // [n_events] announced events (event + 1); zero before
    int32_t* ready_ctr = nullptr;  // events announced; zero before
    int32_t* m_claim = nullptr;    // announcements claimed; zero before
    int32_t* done_ctr = nullptr;   // events with both halves finished; zero before
    int32_t* fault = nullptr;      // set if a wait gave up; zero before
    unsigned long long wait_ns = 0;  // longest wait for an announced event (globaltimer ns); 0: give up at once
    int32_t* pool_velo = nullptr;  // [pool_cap] matched VELO segment per seed record
    float* pool_chi2 = nullptr;    // [pool_cap]
    int32_t* n_long = nullptr;     // [n_events], may be null
};

struct GatherArgs {
    int64_t n_events;
    const int32_t* item_start;
    const int32_t* item_count;
    const int32_t* pool_hits;
    const float* pool_params;
    const float* pool_state;
    const int8_t* pool_n;
    int64_t cap;
    int32_t* ev_off;
    int32_t* hits;
    float* params;
    float* state;
    int8_t* n_hits;
    int32_t* status;
    // fused matching: its per-record results go to the Long-track arrays too
    const int32_t* pool_velo = nullptr;  // null: nothing to copy
    const float* pool_chi2 = nullptr;
    int32_t* velo_idx = nullptr;
    float* chi2 = nullptr;
    const int32_t* fault = nullptr;      // non-zero: every event of the launch gets ST_TIMEOUT
};

struct MatchArgs {
    int64_t n_events;
    const int8_t* seed_n;  // (nx, nuv) per seed
    float* ghost_prob;     // per seed (final selection)
    const int64_t* velo_off;
    const float* velo;
    const int32_t* seed_off;
    const float* seed_state;
    int32_t* velo_idx;
    float* chi2;
    int32_t* n_long;
    int32_t velo_smem;    // VELO segments per shared-memory chunk
    int32_t* queue;
    unsigned long long* counters;
};

size_t build_smem_bytes(int bins, int smem_hits);
size_t seed_smem_bytes(int threads, int smem_hits, int tbl_smem, int key_smem);
size_t seed_slot_bytes(int cand_cap, int max_xhits);
size_t match_smem_bytes(int velo_smem);

// chained: k_order, k_seed and k_scan are launched as programmatic dependents
// of the stream's previous kernel (the caller puts no other stream work
// between them; k_gather always follows k_scan that way).  Their CTAs may
// then wait on the SMs for that kernel, which only pays where no other
// stream's kernels want those SMs.
cudaError_t launch_build(const DevParams& P, const BuildArgs& a, int grid, int threads, cudaStream_t s,
                         bool chained = true);
cudaError_t launch_seed(const DevParams& P, const SeedArgs& a, int grid, int threads, cudaStream_t s,
                        bool chained = true);
cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s, bool chained = true);
cudaError_t launch_match(const DevParams& P, const MatchArgs& a, int grid, int threads, cudaStream_t s);

// occupancy helpers
int build_blocks_per_sm(int threads, size_t smem);
int seed_blocks_per_sm(int threads, size_t smem);
int match_blocks_per_sm(int threads, size_t smem);
cudaError_t set_smem_limits(size_t optin);
cudaError_t smem_limits_hold(size_t optin, bool& hold);

}  // namespace st
