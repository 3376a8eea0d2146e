// st_ut.cuh -- UT-hit search of the Long tracks (Section 4.3): parameters and
// launch interface.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace st {

// Constants of the UT search, derived on the host from st_config.
struct UtParams {
    float z_velo;
    float dz[4], dz2[4];  // z_UT - z_velo and its square, per UT layer
    float t[4];           // stereo slopes of the UT layers
    float gA, gB;         // Eq. (gamma_parametrisation): gamma = gA + gB * q/p (per MeV)
    float inv_kick;       // q/p = (tx_SciFi - tx_VELO) * inv_kick
    float loose[16];      // per layer A, B (mm GeV/c), min, max; max = 0: no loose search
    float tight[16];      // per layer A, B, min, max; max = 0: no tight search
    int min_hits;         // Long tracks keep their VELO segment with at least this many hits
};

struct UtArgs {
    int64_t n_events;
    const int64_t* ut_off;   // [n_events + 1] into ut_x / ut_layer
    const float* ut_x;
    const int32_t* ut_layer;
    const int64_t* velo_off;
    const float* velo;       // x, y, tx, ty at z_velo
    const int32_t* seed_off; // per-event seed ranges (st_seeds.ev_off)
    const float* seed_state; // x, y, tx, ty at z_state
    int32_t* velo_idx;       // in: matched VELO segment per seed; out: -1 if dropped
    float* chi2;             // zeroed for dropped pairs
    int32_t* n_long;         // may be null
    int32_t* status;         // per event; ST_EINVAL for an invalid UT hit
    int32_t* ut_hits;        // [seeds * 4]
    int8_t* ut_n;            // [seeds]
    float* gamma;            // [seeds]
};

cudaError_t launch_ut(const UtParams& U, const UtArgs& a, int grid, cudaStream_t s);

}  // namespace st
