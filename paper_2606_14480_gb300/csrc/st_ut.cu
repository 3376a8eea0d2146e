// st_ut.cu -- UT hits of the Long tracks (Section 4.3), sm_103a.
//
// One CTA per event.  The event's UT hits are staged in shared memory grouped
// by (layer, 32 mm bucket of x) with a counting sort, so a search window of a
// few mm reads one or two buckets (the order within a bucket does not matter:
// every choice below breaks ties explicitly by x, then by the hit's index).  One thread per seed with a matched VELO segment: the
// segment is extrapolated with Eq. (velo_ut_extrapolation), gamma_x from Eq.
// (gamma_parametrisation) at the pair's q/p, through the four UT layers in
// order; until a hit is found each layer is searched in its loose window and
// the closest hit refits gamma_x through itself, later layers in their tight
// windows (closest hit attached).  A Long track with fewer than min_hits UT
// hits loses its VELO segment.
#include <cfloat>

#include "st_device.cuh"
#include "st_ut.cuh"

namespace st {

constexpr int kUtThreads = 256;
constexpr int kUtSmem = 4096;  // UT hits of one event staged in shared memory
constexpr int kUtBins = 64;    // x buckets per layer over [-1024, 1024) mm (edge buckets extend)
constexpr float kUtRange = 1024.f;

__device__ __forceinline__ int ut_bin(float x) {
    const int b = __float2int_rd((x + kUtRange) * (kUtBins / (2.f * kUtRange)));
    return min(max(b, 0), kUtBins - 1);
}

__global__ void __launch_bounds__(kUtThreads) k_ut(const __grid_constant__ UtParams U, const __grid_constant__ UtArgs A) {
    __shared__ float sx[kUtSmem];
    __shared__ int si[kUtSmem];
    __shared__ int s_off[4 * kUtBins + 1], s_cur[4 * kUtBins], s_nl;
    const int tid = threadIdx.x, T = blockDim.x;
    for (int64_t e = blockIdx.x; e < A.n_events; e += gridDim.x) {
        const int64_t u0 = A.ut_off[e];
        const int nu = static_cast<int>(A.ut_off[e + 1] - u0);
        const bool staged = nu <= kUtSmem;
        for (int k = tid; k < 4 * kUtBins; k += T) s_cur[k] = 0;
        if (tid == 0) s_nl = 0;
        __syncthreads();
        bool bad = false;
        for (int i = tid; i < nu; i += T) {
            const int l = A.ut_layer[u0 + i];
            const float x = A.ut_x[u0 + i];
            if (l < 0 || l > 3 || !isfinite(x)) bad = true;
            else if (staged) atomicAdd(&s_cur[l * kUtBins + ut_bin(x)], 1);
        }
        // an event with an invalid UT hit gets ST_EINVAL and no UT hits
        const bool skip = __syncthreads_or(bad) != 0;
        if (skip && tid == 0) A.status[e] = -1;  // ST_EINVAL
        if (staged && !skip) {
            if (tid < 32) {  // exclusive scan of the 256 bucket counts by one warp
                int c[8], t = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    c[q] = s_cur[8 * tid + q];
                    t += c[q];
                }
                int x = t;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (tid >= o) x += y;
                }
                int run = x - t;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    s_off[8 * tid + q] = run;
                    s_cur[8 * tid + q] = run;
                    run += c[q];
                }
                if (tid == 31) s_off[4 * kUtBins] = run;
            }
            __syncthreads();
            for (int i = tid; i < nu; i += T) {
                const int l = A.ut_layer[u0 + i];
                const float x = A.ut_x[u0 + i];
                const int k = atomicAdd(&s_cur[l * kUtBins + ut_bin(x)], 1);
                sx[k] = x;
                si[k] = i;
            }
            __syncthreads();
        }
        const int64_t s0 = A.seed_off[e];
        const int ns = A.seed_off[e + 1] - static_cast<int>(s0);
        const int64_t v0 = A.velo_off[e];
        int kept = 0;
        for (int s = tid; s < ns; s += T) {
            const int64_t r = s0 + s;
            int hits[4] = {-1, -1, -1, -1};
            int n = 0;
            float g = 0.f;
            const int v = A.velo_idx[r];
            if (v >= 0 && !skip) {
                const float* vs = A.velo + (v0 + v) * 4;
                const float xV = vs[0], yV = vs[1], txV = vs[2], tyV = vs[3];
                const float qop = (A.seed_state[r * 4 + 2] - txV) * U.inv_kick;
                const float inv_p = 1000.f * fabsf(qop);  // 1/p in (GeV/c)^-1
                g = fmaf(U.gB, qop, U.gA);
                bool found = false;
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const float* w = found ? &U.tight[4 * l] : &U.loose[4 * l];
                    if (!(w[3] > 0.f)) continue;
                    const float win = fminf(fmaxf(fmaf(w[1], inv_p, w[0]), w[2]), w[3]);
                    // straight part of the extrapolation as a float-float, so
                    // that the refit of gamma below keeps its precision
                    float p, pe, lh, ll;
                    two_prod(txV, U.dz[l], p, pe);
                    two_sum(xV, p, lh, ll);
                    ll += pe;
                    const float yt = fmaf(tyV, U.dz[l], yV);
                    const float ys = yt * U.t[l];
                    const float xm = lh + (ll + fmaf(g, U.dz2[l], -ys));
                    int best = -1;
                    float bd = 0.f, bx = 0.f;
                    auto consider = [&](float xh, int idx) {
                        const float d = fabsf(xh - xm);
                        if (!(d <= win)) return;
                        if (best < 0 || d < bd || (d == bd && (xh < bx || (xh == bx && idx < best)))) {
                            best = idx;
                            bd = d;
                            bx = xh;
                        }
                    };
                    if (staged) {
                        const int k0 = s_off[l * kUtBins + ut_bin(xm - win)];
                        const int k1 = s_off[l * kUtBins + ut_bin(xm + win) + 1];
                        for (int k = k0; k < k1; ++k) consider(sx[k], si[k]);
                    } else {
                        for (int i = 0; i < nu; ++i)
                            if (A.ut_layer[u0 + i] == l) consider(A.ut_x[u0 + i], i);
                    }
                    if (best < 0) continue;
                    hits[l] = best;
                    ++n;
                    if (!found) {
                        // gamma_x through this hit: (x_hit + y t - x_V - tx_V dz) / dz^2
                        g = (((bx - lh) - ll) + ys) / U.dz2[l];
                        found = true;
                    }
                }
            }
#pragma unroll
            for (int l = 0; l < 4; ++l) A.ut_hits[r * 4 + l] = hits[l];
            A.ut_n[r] = static_cast<int8_t>(n);
            A.gamma[r] = g;
            if (v >= 0 && n < U.min_hits) {
                A.velo_idx[r] = -1;
                A.chi2[r] = 0.f;
            }
            kept += v >= 0 && n >= U.min_hits;
        }
        kept = warp_sum(kept);
        if ((tid & 31) == 0 && kept) atomicAdd(&s_nl, kept);
        __syncthreads();
        if (tid == 0 && A.n_long) A.n_long[e] = s_nl;
        __syncthreads();
    }
}

cudaError_t launch_ut(const UtParams& U, const UtArgs& a, int grid, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    k_ut<<<grid, kUtThreads, 0, s>>>(U, a);
    return cudaGetLastError();
}

}  // namespace st
