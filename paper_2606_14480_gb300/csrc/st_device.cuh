// st_device.cuh -- device-side constants and helpers of libst (sm_103a).
//
// DevParams holds every constant the kernels need, derived once on the host
// in double precision from st_config and rounded to float (float-float pairs
// where a value enters a compensated computation).  It is passed by value as a
// __grid_constant__ kernel parameter.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace st {

constexpr int kLayers = 12;
constexpr int kZones = 24;
constexpr int kSlotsPerHalf = 12;  // 6 x-layer zones, then 6 stereo zones
constexpr int kZoffStride = 25;    // per event: 24 slot starts + end
constexpr int kMasks = 7;          // x-layer hit patterns with >= 5 hits
constexpr int kMaxThreads = 512;

// Container order of an event: half-major; within a half the x-layers
// (0,3,4,7,8,11) then the stereo layers (1,2,5,6,9,10), each sorted by x.
// slot(zone) = 12*half + (x-slot or 6 + stereo slot).

struct IterP {
    int s1, s2, s3;        // x-slots of the initial layers T1, T2, T3
    int ext[3];            // x-slots of the other three x-layers, ascending
    float scale3;          // (z3 + alpha_corr) / z1
    float dx3;             // Delta x3^max
    float inv_dz31;        // 1 / (z3 - z1)
    float dz21;            // z2 - z1
    float z1;
    float k3, inv_k3;      // chord deviation per unit c_x at z2
    float c0;              // band widening in c_x units
    float mlo_k, mhi_k;    // m_lo * kappa_c, m_hi * kappa_c
    float q31;             // (f3 - f1) / (z3 - z1)
    float zb1, f1;         // zb and f of T1
};

struct DevParams {
    // x-slot geometry: zb = z - z_ref (exact), f = zb^2 (1 + d zb) as hi + lo
    float xzb[6], xf_hi[6], xf_lo[6];
    // stereo-slot geometry (slots ordered by z)
    float uz[6], uzb[6], uf_hi[6], uf_lo[6], ut[6], uzt[6];
    float uinv_t[6], uinv_z[6];  // 1/dxdy and 1/z of the stereo slots
    float zc_uv;           // centring z of the y-z line fit (uzt = uz - zc_uv)
    IterP it[3];
    int n_iter;
    int iter_mode;  // 1: iterations in sequence with hit cleanup
    float invp_a, invp_b;
    float ext_tol, chi2x_max, inv_sx2, w_chi2, w5;
    float G[kMasks][3][6]; // least-squares gain per x-hit pattern
    int mask_index[64];    // 6-bit x-hit pattern -> G index, -1 if < 5 hits
    int uv_init[2];        // stereo slot of the initial layer of each pass
    int uv_rem[2][5];      // the other stereo slots of each pass, ascending z
    int n_uv_min;
    float uv_tol;
    float uv_ylo[2], uv_yhi[2];  // first-layer y window per half
    float inv_sy2;
    // Hough-cluster UV variant
    int uv_mode;
    int h_bins, h_fine, h_clusters;
    float h_lo[2];         // lower edge of the coarse t_y range per half
    float h_w, h_inv_w;    // coarse bin width and its inverse
    float h_step;          // sub-bin width in coarse-bin units (2 / h_fine)
    // seed state
    float zS, zbS, fS, dfS;
    // matching
    float zV, zMY;
    float A_hi, A_lo, Bx, Cx, Dx, Ex;
    float dAV_hi, dAV_lo;  // A - z_velo
    float dAS_hi, dAS_lo;  // A - z_state
    float dMV_hi, dMV_lo;  // z_match_y - z_velo
    float dMS_hi, dMS_lo;  // z_match_y - z_state
    float cut_x, cut_y, cut_tx, cut_ty;
    float tolx_a, tolx_b, toly_a, toly_b, inv_toltx, inv_tolty, chi2m_max;
    int velo_unique;
    // final selection (Section 4.4): ghost network weights, cut, clone margin
    int final_sel;
    float ghost_max, clone_margin;
    float nn[337];  // mean[8], inv_scale[8], W1[32][8], b1[32], w2[32], b2
    // per layer, for the optional z / dxdy input check
    float zl[12], tl[12];
    int slot_of_zone[24];
};

// ---------------------------------------------------------------------------
// error-free transformations (Knuth's TwoSum, FMA-based TwoProduct)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// ---------------------------------------------------------------------------
// searches over an ascending float array
// ---------------------------------------------------------------------------

// first index i in [0, n) with a[i] >= v (n if none)
__device__ __forceinline__ int lower_bound_f(const float* a, int n, float v) {
    int lo = 0, len = n;
    while (len > 0) {
        int h = len >> 1;
        if (a[lo + h] < v) {
            lo += h + 1;
            len -= h + 1;
        } else {
            len = h;
        }
    }
    return lo;
}

// first index i in [0, n) with a[i] > v (n if none)
__device__ __forceinline__ int upper_bound_f(const float* a, int n, float v) {
    int lo = 0, len = n;
    while (len > 0) {
        int h = len >> 1;
        if (!(v < a[lo + h])) {
            lo += h + 1;
            len -= h + 1;
        } else {
            len = h;
        }
    }
    return lo;
}

// largest t in [0, n) with s[t] <= p, for a non-decreasing int array s with
// s[0] = 0 <= p (the owner of item p in a load-balanced expansion)
__device__ __forceinline__ int owner_of(const int* s, int n, int p) {
    int lo = 0, len = n;
    while (len > 0) {
        int h = len >> 1;
        if (s[lo + h] <= p) {
            lo += h + 1;
            len -= h + 1;
        } else {
            len = h;
        }
    }
    return lo - 1;
}

// ---------------------------------------------------------------------------
// block-wide exclusive scan of one int per thread; returns the exclusive
// prefix, writes the block total.  `tmp` holds >= 33 ints of shared memory.
// Contains __syncthreads(); every thread of the block must call it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_exscan(int v, int* tmp, int& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? tmp[lane] : 0;
        int ww = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, ww, o);
            if (lane >= o) ww += y;
        }
        if (lane < nw) tmp[lane] = ww - w;
        if (lane == 31) tmp[32] = ww;
    }
    __syncthreads();
    int res = x - v + tmp[wid];
    total = tmp[32];
    __syncthreads();
    return res;
}

// The same scan with one barrier: every warp adds up the partial sums of the
// warps before it itself.  Consecutive calls alternate between the two halves
// of `buf` (>= 34 ints) under the block-uniform toggle `par`, so a call never
// overwrites partial sums that a slower thread may still read from the
// previous call (the barrier of the call in between orders them).
__device__ __forceinline__ int block_exscan1(int v, int* buf, int& par, int& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    int* t = buf + (par ? 17 : 0);
    par ^= 1;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) t[wid] = x;
    __syncthreads();
    int w = lane < nw ? t[lane] : 0;
    int before = lane < wid ? w : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        w += __shfl_xor_sync(0xffffffffu, w, o);
        before += __shfl_xor_sync(0xffffffffu, before, o);
    }
    total = w;
    return x - v + before;
}

// block_exscan1 that also returns whether any thread's flag was set (the
// flag rides in bit 30 of the warp partials; the values must stay below 2^30).
__device__ __forceinline__ int block_exscan1_any(int v, bool flag, int* buf, int& par, int& total, bool& any) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    int* t = buf + (par ? 17 : 0);
    par ^= 1;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const int f = __any_sync(0xffffffffu, flag) ? (1 << 30) : 0;
    if (lane == 31) t[wid] = x | f;
    __syncthreads();
    const int tw = lane < nw ? t[lane] : 0;
    int w = tw & ((1 << 30) - 1);
    int before = lane < wid ? w : 0;
    const bool fa = __any_sync(0xffffffffu, (tw >> 30) & 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        w += __shfl_xor_sync(0xffffffffu, w, o);
        before += __shfl_xor_sync(0xffffffffu, before, o);
    }
    total = w;
    any = fa;
    return x - v + before;
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace st
