// st_kernels.cu -- sm_103a kernels of the SciFi Seeding + VELO-SciFi Matching
// hot path.  All kernels are persistent: a grid of (SMs x resident CTAs) pulls
// work items (events, or detector halves of events) from a device counter.
//
//   k_build   one event per item: validate hits, sort them by (container
//             slot, x, index) with a bucketed rank sort in shared memory, write
//             the per-event container (x, original index) and slot offsets.
//   k_order   one CTA: the seeding items sorted by cost class, costliest
//             first, the order in which k_seed's queue hands them out.
//   k_seed    one detector half of one event per item (the paper keeps the
//             halves apart, Section 5.2): XZ seeding of the iterations with
//             load-balanced expansion of pairs and triplets, extension and
//             compensated least-squares fit, O(n) clone killing with a 64-bit
//             atomicMin table, UV seeding (iterative or Hough clusters) with a
//             64-bit atomicMin per seed, and the seed records; HLT2-style
//             iterations run as passes with a taken-hit bitmask.  In the
//             batch path the CTA that finishes an event's second half also
//             matches the event.
//   k_scan / k_gather   per-event CSR of the seed records.
//   k_match   one event per item: VELO segments bucketed by ty in shared
//             memory, one thread per seed for its lowest chi2_match, then
//             optionally the final selection (ghost network, clones).
//
// k_order, k_seed, k_scan and k_gather are launched as programmatic
// dependents of the kernel before them in the stream: their CTAs may be
// scheduled while it finishes, and wait (griddepcontrol.wait) for its
// completion and its memory before they read or write anything it touches.
// Launched without that attribute, the wait returns at once.
#include <algorithm>
#include <cfloat>
#include <utility>

#include "st_kernels.cuh"

namespace st {

typedef unsigned long long ull;


static __host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Programmatic dependent launch (PTX griddepcontrol): let the next kernel of
// the stream be scheduled once every CTA of this grid has signalled or ended,
// and wait for the completion and memory of the grids this one depends on.
__device__ __forceinline__ void pdl_signal() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Bulk copies (the TMA's untiled form, cp.async.bulk) into shared memory,
// completing on an mbarrier: one thread initialises the barrier, one thread
// issues each copy with the byte count it expects, every thread waits for the
// phase.  Both addresses 16-byte aligned, the size a multiple of 16 bytes.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(ull* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, unsigned bytes, ull* b) {
    // the CTA's earlier reads of dst (ordered by a barrier) before the copy's writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(b))
                 : "memory");
}
// Polls the barrier's phase `parity`; false after max_polls unsuccessful polls.
__device__ __forceinline__ bool mbar_wait(ull* b, unsigned parity, int max_polls) {
    const uint32_t a = smem_addr(b);
    for (int i = 0; i < max_polls; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
// A staging copy that has not landed after this many polls (each of which
// may suspend the thread for a while) is given up: the launch is marked
// faulty and the item reads its hits from global memory.
constexpr int kStagePolls = 1 << 22;

// First container index of event e: events are laid out back to back with
// three spare entries each, rounded up to a multiple of four floats so that
// every event starts 16-byte aligned.
__device__ __forceinline__ int64_t cont_base(const int64_t* ev_off, int64_t e) {
    int64_t b = (ev_off[e] - ev_off[0]) + 3 * e;
    return (b + 3) & ~int64_t(3);
}

// Sum per-thread counters over the CTA (warp shuffles, then shared memory)
// and add them to the global counters with one atomic per counter per CTA.
// Every thread of the CTA must call it.
__device__ __forceinline__ void flush_counters(unsigned long long* dst, const ull* c, int n) {
    __shared__ ull s_acc[16];
    if (threadIdx.x < 16) s_acc[threadIdx.x] = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        ull v = c[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_acc[k], v);
    }
    __syncthreads();
    if (threadIdx.x < n && s_acc[threadIdx.x]) atomicAdd(dst + threadIdx.x, s_acc[threadIdx.x]);
}

// ===========================================================================
// container build
// ===========================================================================

constexpr float kBinRange = 3500.f;

// Seeding items are handed out costliest first (largest-processing-time
// order), so that no large item starts when the rest of the batch is nearly
// done.  The cost of a (event, half) item is the size of its two-hit search
// domain, sum over iterations of n(T1) n(T3), plus its hit count; its class
// is that cost on a quarter-octave scale.
constexpr int kCostClasses = 128;
static_assert(kCostClasses % 32 == 0, "one warp scans the classes");

__device__ __forceinline__ int cost_class(ull cost) {
    if (cost < 4u) return static_cast<int>(cost);
    const int oct = 63 - __clzll(static_cast<long long>(cost));
    return min(4 * oct + static_cast<int>((cost >> (oct - 2)) & 3u), kCostClasses - 1);
}

__device__ __forceinline__ void set_item_class(const BuildArgs& A, int64_t item, int c) {
    A.item_class[item] = c;
    atomicAdd(A.class_count + c, 1);
}

// shared memory of k_build: bucket counts / fill cursors and bucket starts,
// the block scan's scratch, then 10 bytes per hit (x, bucket, the hits
// grouped by bucket, the sorted order)
size_t build_smem_bytes(int bins, int smem_hits) {
    const int NB = kZones * bins;
    return align16(sizeof(int) * (2 * NB + 1 + 36)) + align16(size_t(10) * smem_hits);
}

// Per event (one CTA): validate and bucket the hits by (container slot, x),
// place them bucket by bucket, rank each hit inside its bucket by (x, index)
// and write the sorted event out in order.  Per-hit arrays: x (hx), bucket
// (bk), the hits grouped by bucket (pm) and the sorted order (so), which the
// ranking fills directly.  Between two events of a CTA the bucket
// counts are cleared during the ranking and the next event's ticket and
// offsets are fetched during the placement, so the next event starts with
// its loads.  At most 32 registers: up to eight 256-thread CTAs per SM.
__global__ void __launch_bounds__(kMaxThreads, 4)
k_build(const __grid_constant__ DevParams P, const __grid_constant__ BuildArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = A.bins, NB = kZones * B, T = blockDim.x, tid = threadIdx.x;
    int* cnt = reinterpret_cast<int*>(smem);  // counts, then fill cursors, then cleared
    int* off = cnt + NB;
    int* tmp = off + NB + 1;
    unsigned char* harea = smem + align16(sizeof(int) * (2 * NB + 1 + 36));
    // the CTA's next event and its hit range, published by thread 0
    __shared__ int s_item, s_bad;
    __shared__ long long s_h0, s_h1;
    // per-zone / per-layer constants indexed by each hit's zone: in shared
    // memory (reads of kernel parameters at lane-dependent indices serialise)
    __shared__ int s_slot[kZones];
    __shared__ float s_zl[kLayers], s_tl[kLayers];
    if (tid < kZones) s_slot[tid] = P.slot_of_zone[tid];
    if (tid < kLayers) {
        s_zl[tid] = P.zl[tid];
        s_tl[tid] = P.tl[tid];
    }
    ull ctr[2] = {0, 0};
    int spar = 0;  // which half of tmp the next block scan uses
    pdl_signal();  // k_order may be scheduled; it waits for this grid
    for (int k = tid; k < NB; k += T) cnt[k] = 0;
    if (tid == 0) {
        s_bad = 0;
        s_item = atomicAdd(A.queue, 1);
        if (s_item < A.n_events) {
            s_h0 = A.ev_off[s_item];
            s_h1 = A.ev_off[s_item + 1];
        }
    }
    // thread 0: the next ticket and the offsets of its event
    auto next_item = [&]() {
        const int q = atomicAdd(A.queue, 1);
        if (q < A.n_events) {
            s_h0 = A.ev_off[q];
            s_h1 = A.ev_off[q + 1];
        }
        s_item = q;
    };

    for (;;) {
        __syncthreads();
        const int64_t e = s_item;
        if (e >= A.n_events) break;
        const int64_t h0 = s_h0;
        const int64_t n64 = s_h1 - h0;
        int32_t* zo = A.zoff + e * kZoffStride;
        const int64_t cb = cont_base(A.ev_off, e);
        if (n64 < 0 || n64 > A.max_hits || cb + n64 > A.cont_cap) {
            // too large for max_hits, or an earlier oversized event pushed this
            // one past the container
            for (int k = tid; k < kZoffStride; k += T) zo[k] = 0;
            if (tid < 2) set_item_class(A, 2 * e + tid, 0);
            __syncthreads();  // every thread has read s_item
            if (tid == 0) {
                A.status[e] = -3;  // ST_OVERFLOW
                next_item();
            }
            continue;
        }
        const int n = static_cast<int>(n64);
        const bool in_smem = n <= A.smem_hits;
        unsigned char* base = in_smem ? harea : A.big + int64_t(blockIdx.x) * A.big_stride;
        const int cap = in_smem ? A.smem_hits : A.max_hits;
        float* hx = reinterpret_cast<float*>(base);
        uint16_t* bk = reinterpret_cast<uint16_t*>(hx + cap);
        uint16_t* pm = bk + cap;
        uint16_t* so = pm + cap;
        const float binscale = B / (2.f * kBinRange);
        // count: four hits per thread per round, their loads issued together
        for (int i0 = tid; i0 < n; i0 += 4 * T) {
            float xs[4];
            int zs[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * T;
                xs[q] = i < n ? A.x[h0 + i] : 0.f;
                zs[q] = i < n ? A.zone[h0 + i] : 0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q * T;
                if (i >= n) break;
                const float x = xs[q];
                const int zn = zs[q];
                bool bad = !(zn >= 0 && zn < kZones) || !isfinite(x);
                if (!bad) {
                    const int L = zn >> 1;
                    if (A.z && !(fabsf(A.z[h0 + i] - s_zl[L]) <= 1e-3f)) bad = true;
                    if (A.dxdy && !(fabsf(A.dxdy[h0 + i] - s_tl[L]) <= 1e-6f)) bad = true;
                }
                if (bad) {
                    s_bad = 1;
                    continue;
                }
                int bin = __float2int_rd((x + kBinRange) * binscale);
                bin = min(max(bin, 0), B - 1);
                const int b = s_slot[zn] * B + bin;
                hx[i] = x;
                bk[i] = static_cast<uint16_t>(b);
                atomicAdd(&cnt[b], 1);
            }
        }
        __syncthreads();
        if (s_bad) {
            for (int k = tid; k < kZoffStride; k += T) zo[k] = 0;
            for (int k = tid; k < NB; k += T) cnt[k] = 0;
            if (tid < 2) set_item_class(A, 2 * e + tid, 0);
            __syncthreads();  // s_bad read by every thread
            if (tid == 0) {
                A.status[e] = -1;  // ST_EINVAL
                s_bad = 0;
                next_item();
            }
            continue;
        }
        {   // exclusive scan of the bucket counts; the counts become fill cursors
            const int per = (NB + T - 1) / T;
            const int k0 = min(tid * per, NB), k1 = min(k0 + per, NB);
            int sum = 0;
            for (int k = k0; k < k1; ++k) sum += cnt[k];
            int tot;
            int ex = block_exscan1(sum, tmp, spar, tot);
            for (int k = k0; k < k1; ++k) {
                const int c = cnt[k];
                off[k] = ex;
                cnt[k] = ex;
                ex += c;
            }
            if (tid == 0) off[NB] = tot;
        }
        __syncthreads();
        if (tid == 0) next_item();  // read by the other threads after the next loop-top barrier
        for (int i = tid; i < n; i += T) pm[atomicAdd(&cnt[bk[i]], 1)] = static_cast<uint16_t>(i);
        __syncthreads();
        // rank of each hit in its bucket -> its place in the sorted event;
        // the cursors are cleared for the next event.  Threads take the hits
        // in bucket order, so the lanes of a warp mostly share a bucket: equal
        // loop lengths, and the bucket's reads are broadcasts.
        for (int k = tid; k < NB; k += T) cnt[k] = 0;
        for (int d = tid; d < n; d += T) {
            const int i = pm[d];
            const int b = bk[i], s = off[b], c = off[b + 1] - s;
            const float x = hx[i];
            int r = 0;
            for (int k = s; k < s + c; ++k) {
                const int j = pm[k];
                const float xj = hx[j];
                r += (xj < x) || (xj == x && j < i);
            }
            so[s + r] = static_cast<uint16_t>(i);
        }
        __syncthreads();
        // the sorted event goes out in order (coalesced stores)
        for (int d = tid; d < n; d += T) {
            const int i = so[d];
            A.cx[cb + d] = hx[i];
            A.corig[cb + d] = i;
        }
        for (int k = tid; k < kZoffStride; k += T) zo[k] = off[k * B];
        if (tid < 2) {
            auto nz = [&](int sl) { return ull(off[(sl + 1) * B] - off[sl * B]); };
            ull cost = ull(off[(12 * tid + 12) * B] - off[12 * tid * B]);
            for (int it = 0; it < P.n_iter; ++it) cost += nz(12 * tid + P.it[it].s1) * nz(12 * tid + P.it[it].s3);
            set_item_class(A, 2 * e + tid, cost_class(cost));
        }
        if (tid == 0) {
            A.status[e] = 0;
            ctr[0] += n;
            ctr[1] += 1;
        }
    }
    flush_counters(A.counters + C_HITS, ctr, 2);
}

// The seeding items in cost order (a counting sort by class, costliest class
// first), after k_build has counted the classes.  One thread per item; a
// CTA's items of one class take consecutive places from one global atomic.
// The order inside a class does not matter: items are independent and their
// results are gathered per event.
constexpr int kOrderThreads = 1024;

__global__ void __launch_bounds__(kOrderThreads) k_order(const __grid_constant__ BuildArgs A) {
    __shared__ int pos[kCostClasses], s_cnt[kCostClasses];
    const int tid = threadIdx.x;
    pdl_signal();
    pdl_wait();  // k_build's class counts
    const unsigned lane = tid & 31;
    if (tid < 32) {  // first place of each class: exclusive scan from the top class down
        constexpr int kPer = kCostClasses / 32;
        int c[kPer], t = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            c[q] = A.class_count[kCostClasses - 1 - (kPer * tid + q)];
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
        for (int q = 0; q < kPer; ++q) {
            pos[kCostClasses - 1 - (kPer * tid + q)] = run;
            run += c[q];
        }
    }
    for (int k = tid; k < kCostClasses; k += kOrderThreads) s_cnt[k] = 0;
    __syncthreads();
    const int64_t items = 2 * A.n_events;
    const int64_t i = int64_t(blockIdx.x) * kOrderThreads + tid;
    if (A.zero2 && i < items) A.zero2[i] = 0;
    const int c = i < items ? A.item_class[i] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const int leader = __ffs(same) - 1;
    int r = 0;
    if (c >= 0 && static_cast<int>(lane) == leader) r = atomicAdd(&s_cnt[c], __popc(same));
    r = __shfl_sync(0xffffffffu, r, leader) + __popc(same & ((1u << lane) - 1u));
    __syncthreads();
    for (int k = tid; k < kCostClasses; k += kOrderThreads)
        if (s_cnt[k]) pos[k] += atomicAdd(A.class_fill + k, s_cnt[k]);
    __syncthreads();
    if (c >= 0) A.order[pos[c] + r] = static_cast<int32_t>(i);
}

// ===========================================================================
// seeding
// ===========================================================================

// ---------------------------------------------------------------------------
// per-zone bucket tables: lut[b] = first hit of the zone with bin(x) >= b, so
// that a window edge is found with one table read and a short forward scan
// (the same result as a binary search over the sorted zone)
// ---------------------------------------------------------------------------

// The range covers the SciFi's x acceptance (|x| < 3200 mm) and the stereo
// layers' measured coordinate, offset from it by y tan(5 deg) for |y| < 2500 mm
// (hits outside it fall into the end buckets, which stays correct but scans
// longer).  Finer buckets shorten the scans: against 32 mm buckets over
// [-4096, 4096), 27 mm took k_seed from 0.2088 to 0.206 ms for 1000
// Run-3-like events; 18 mm keeps that step time and takes 12% off the
// 10 000-event uneven batch, whose large events hold more hits per bucket
// (9 KB of tables per CTA).
constexpr float kLutRange = 3456.f;
constexpr int kLutBins = 384;  // 18 mm buckets over [-3456, 3456) mm

__device__ __forceinline__ int lut_bin(float v) {
    const int b = __float2int_rd((v + kLutRange) * (kLutBins / (2.f * kLutRange)));
    return min(max(b, 0), kLutBins - 1);
}

// first index i in [0, n) with x[i] >= v (n if none)
__device__ __forceinline__ int zlo(const float* x, const uint16_t* lut, int n, float v) {
    int i = lut[lut_bin(v)];
    while (i < n && x[i] < v) ++i;
    return i;
}

// first index i in [0, n) with x[i] > v (n if none)
__device__ __forceinline__ int zhi(const float* x, const uint16_t* lut, int n, float v) {
    int i = lut[lut_bin(v)];
    while (i < n && !(v < x[i])) ++i;
    return i;
}

// hits taken by earlier iterations (HLT2-style mode), one bit per half-local
// hit position; null when every hit is free
__device__ __forceinline__ bool is_used(const uint32_t* used, int p) {
    return used && ((used[p >> 5] >> (p & 31)) & 1u);
}

// The closest hit to xp within tol in a sorted zone (xs, its bucket table
// lz, n hits starting at half-local position st), ties to the smaller x (the
// first met), skipping hits taken by earlier iterations; its half-local
// position, or -1.  One scan from the table entry of xp - tol: hits below
// xp - tol are passed over (the window start a zlo search would give), the
// scan ends at the first hit above xp + tol.
__device__ __forceinline__ int closest_hit(const float* xs, const uint16_t* lz, int n, int st, float xp, float tol,
                                           const uint32_t* used) {
    const float lo = xp - tol, hi = xp + tol;
    int best = -1;
    float bd = 0.f;
    for (int k = lz[lut_bin(lo)]; k < n; ++k) {
        const float xh = xs[k];
        if (xh > hi) break;
        if (xh < lo || is_used(used, st + k)) continue;
        const float d = fabsf(xh - xp);
        if (d <= tol && (best < 0 || d < bd)) {
            best = st + k;
            bd = d;
        }
    }
    return best;
}

struct Trip {
    int pos[6];
    float th[3], dth[3];
    float chi2, score;
    int nx;
};

// Triplet -> exact 3-hit model, extension to the other x-layers (closest hit
// within ext_tol, ties to the smaller x), least-squares fit and chi2 cut.
// The fit is done on residuals y_j of the hits from the 3-hit model, formed
// with error-free transformations so that they keep ~1e-7 mm accuracy; the
// correction dth = G y and the chi2 are then computed from small numbers.
// Returns 0 (fewer than 5 hits), 1 (chi2 cut) or 2 (candidate).
__device__ int do_triplet(const DevParams& P, const IterP& I, const float* X, const int* szl,
                          const uint16_t* lut, const float* sG, const int* sMask, const uint32_t* used, int k1,
                          int k2, int k3, Trip& o) {
    const int p1 = szl[I.s1] + k1, p2 = szl[I.s2] + k2, p3 = szl[I.s3] + k3;
    const float x1 = X[p1], x2 = X[p2], x3 = X[p3];
    const float t13 = (x3 - x1) * I.inv_dz31;
    const float base = fmaf(I.dz21, t13, x1);
    const float c3 = (x2 - base) * I.inv_k3;
    const float b3 = fmaf(-c3, I.q31, t13);
    const float a3 = x1 - fmaf(c3, I.f1, b3 * I.zb1);
    int nx = 3, m = 0;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        int p;
        if (s == I.s1) {
            p = p1;
        } else if (s == I.s2) {
            p = p2;
        } else if (s == I.s3) {
            p = p3;
        } else {
            const float xp = fmaf(c3, P.xf_hi[s], fmaf(b3, P.xzb[s], a3));
            const int st = szl[s];
            p = closest_hit(X + st, lut + s * kLutBins, szl[s + 1] - st, st, xp, P.ext_tol, used);
            nx += p >= 0;
        }
        o.pos[s] = p;
        m |= (p >= 0) << s;
    }
    if (nx < 5) return 0;
    const float* G = sG + 18 * sMask[m];  // [3][6] gain of this hit pattern
    float y[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        y[s] = 0.f;
        if (o.pos[s] >= 0) {
            float d, e;
            two_sum(X[o.pos[s]], -a3, d, e);
            float v = fmaf(-b3, P.xzb[s], d);
            v = fmaf(-c3, P.xf_hi[s], v);
            y[s] = v + fmaf(-c3, P.xf_lo[s], e);
        }
    }
    float da = 0.f, db = 0.f, dc = 0.f;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        da = fmaf(G[s], y[s], da);
        db = fmaf(G[6 + s], y[s], db);
        dc = fmaf(G[12 + s], y[s], dc);
    }
    float chi2 = 0.f;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        if (o.pos[s] >= 0) {
            const float r = y[s] - fmaf(dc, P.xf_hi[s], fmaf(db, P.xzb[s], da));
            chi2 = fmaf(r, r, chi2);
        }
    }
    chi2 *= P.inv_sx2;
    if (chi2 > P.chi2x_max * static_cast<float>(nx - 3)) return 1;
    o.th[0] = a3; o.th[1] = b3; o.th[2] = c3;
    o.dth[0] = da; o.dth[1] = db; o.dth[2] = dc;
    o.chi2 = chi2;
    o.nx = nx;
    const float sc = fmaf(P.w_chi2, chi2, fabsf(c3 + dc));
    o.score = nx == 6 ? sc : P.w5 * sc;
    return 2;
}
__device__ __noinline__ int do_triplet_out(const DevParams& P, const IterP& I, const float* X, const int* szl,
                                          const uint16_t* lut, const float* sG, const int* sMask,
                                          const uint32_t* used, int k1, int k2, int k3, Trip& o) {
    return do_triplet(P, I, X, szl, lut, sG, sMask, used, k1, k2, k3, o);
}

// x(z) of a seed at stereo slot u (3-hit model plus fit correction)
__device__ __forceinline__ float x_at_uv(const DevParams& P, const float* th, const float* dth, int u) {
    return fmaf(th[2], P.uf_hi[u], fmaf(th[1], P.uzb[u], th[0])) +
           fmaf(dth[2], P.uf_hi[u], fmaf(dth[1], P.uzb[u], dth[0]));
}

struct UV {
    int pos[6];
    int n;
    float chi2, tyr, beta, wm, zm;
};

// The search chain of one UV combination (Section 3.4): start from the
// kinit-th hit of the initial stereo layer of `pass`, ty from the origin,
// closest hit within uv_tol in each remaining stereo layer in increasing z
// with ty averaging.  Xs[u] is the seed's x at stereo slot u.  A chain that
// can no longer reach n_uv_min stops early (it cannot be selected).
__device__ void uv_chain(const DevParams& P, const float* X, const int* szl, const uint16_t* lut,
                         const uint32_t* used, const float* Xs, int pass, int kinit, UV& o) {
    const int ui = P.uv_init[pass];
    const int pi = szl[6 + ui] + kinit;
    const float yi = (Xs[ui] - X[pi]) * P.uinv_t[ui];
    float ty = yi * P.uinv_z[ui];
    int n = 1;
    o.n = 0;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        o.pos[u] = -1;
        if (u == ui) {
            o.pos[u] = pi;
            continue;
        }
        const float Xl = Xs[u];
        const float xp = Xl - P.ut[u] * ty * P.uz[u];
        const int st = szl[6 + u];
        const int best = closest_hit(X + st, lut + (6 + u) * kLutBins, szl[7 + u] - st, st, xp, P.uv_tol, used);
        if (best >= 0) {
            const float yl = (Xl - X[best]) * P.uinv_t[u];
            ty = 0.5f * fmaf(yl, P.uinv_z[u], ty);
            o.pos[u] = best;
            ++n;
        }
        const int rem = (5 - u) - (ui > u ? 1 : 0);  // stereo layers still to search
        if (n + rem < P.n_uv_min) {
            o.n = n;
            return;
        }
    }
    o.n = n;
    o.tyr = ty;
}

// Hough-cluster variant (Section 3.4, second approach), step 1 for one seed:
// every stereo hit of the half whose y lies in the first-layer window goes to
// coarse bin floor((y/z - lo) / w) of its layer's 64-bit occupancy mask; a
// cluster b is bins (b, b+1), its population the number of layers with a hit
// in it, counted for all clusters at once with three bit planes.  The kept
// clusters (most populated first, at least n_uv_min, ties to the smaller b)
// go to out[]; returns how many.
__device__ __forceinline__ int hough_select_in(const DevParams& P, const float* X, const int* szl, const uint16_t* lut,
                            const uint32_t* used, const float* Xs, int h, uint8_t* out) {
    ull s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        const float Xl = Xs[u], t = P.ut[u];
        const float xa = fmaf(-P.uv_yhi[h], t, Xl), xb = fmaf(-P.uv_ylo[h], t, Xl);
        const int st = szl[6 + u], n = szl[7 + u] - st;
        const uint16_t* lz = lut + (6 + u) * kLutBins;
        const int lo = zlo(X + st, lz, n, fminf(xa, xb)), hi = zhi(X + st, lz, n, fmaxf(xa, xb));
        ull m = 0;
        for (int k = lo; k < hi; ++k) {
            if (is_used(used, st + k)) continue;
            const float ty = (Xl - X[st + k]) * P.uinv_t[u] * P.uinv_z[u];
            const int b = min(max(__float2int_rd((ty - P.h_lo[h]) * P.h_inv_w), 0), P.h_bins - 1);
            m |= 1ull << b;
        }
        const ull c = m | (m >> 1);  // bit b: a hit in bin b or b + 1
        const ull c0 = s0 & c;
        s0 ^= c;
        const ull c1 = s1 & c0;
        s1 ^= c0;
        s2 |= c1;
    }
    const ull valid = ~0ull >> (65 - P.h_bins);  // clusters 0 .. bins-2
    int ns = 0;
    for (int p = 6; p >= P.n_uv_min && ns < P.h_clusters; --p) {
        ull e = valid & ((p & 1) ? s0 : ~s0) & ((p & 2) ? s1 : ~s1) & ((p & 4) ? s2 : ~s2);
        while (e && ns < P.h_clusters) {
            out[ns++] = static_cast<uint8_t>(__ffsll(static_cast<long long>(e)) - 1);
            e &= e - 1;
        }
    }
    return ns;
}

// The Hough functions, do_triplet and the cold paths of the UV step each
// come as an inlined body (_in) and a call that is not inlined (_out).  The
// seeding kernel calls the _out forms except in its HLT2-style
// instantiation: their code and registers then stay out of the hot phases
// of the iterative HLT1 path, which never runs the Hough code and rarely
// the cold paths (measured 4.6% faster on the Run-3-like batch, while the
// HLT2-style instantiation is faster with everything inlined).
__device__ __noinline__ int hough_select_out(const DevParams& P, const float* X, const int* szl, const uint16_t* lut,
                                             const uint32_t* used, const float* Xs, int h, uint8_t* out) {
    return hough_select_in(P, X, szl, lut, used, Xs, h, out);
}

// step 2 for one t_y hypothesis: the closest hit within uv_tol in every
// stereo layer (ties to the smaller x); stops once n_uv_min is out of reach.
__device__ __forceinline__ void uv_hough_in(const DevParams& P, const float* X, const int* szl, const uint16_t* lut,
                                           const uint32_t* used, const float* Xs, float ty, UV& o) {
    int n = 0;
    o.n = 0;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        const float xp = Xs[u] - P.ut[u] * ty * P.uz[u];
        const int st = szl[6 + u];
        const int best = closest_hit(X + st, lut + (6 + u) * kLutBins, szl[7 + u] - st, st, xp, P.uv_tol, used);
        o.pos[u] = best;
        n += best >= 0;
        if (n + (5 - u) < P.n_uv_min) {
            o.n = n;
            return;
        }
    }
    o.n = n;
    o.tyr = ty;
}
__device__ __noinline__ void uv_hough_out(const DevParams& P, const float* X, const int* szl, const uint16_t* lut,
                                          const uint32_t* used, const float* Xs, float ty, UV& o) {
    uv_hough_in(P, X, szl, lut, used, Xs, ty, o);
}

__device__ __forceinline__ float hough_ty(const DevParams& P, int h, int b, int f) {
    return fmaf(P.h_w, static_cast<float>(b) + (static_cast<float>(f) + 0.5f) * P.h_step, P.h_lo[h]);
}

// Straight-line fit y = y0 + ty z of a complete chain (o.pos, o.n, o.tyr).
// The y of each hit is formed as a float-float from error-free
// transformations and fitted relative to the line y = tyr z, so chi2_y keeps
// ~1e-6 relative accuracy.
__device__ void uv_fit(const DevParams& P, const float* X, const float* th, const float* dth, UV& o) {
    float w[6];
    float sw = 0.f, sz = 0.f;
    const float ty = o.tyr;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        w[u] = 0.f;
        if (o.pos[u] < 0) continue;
        const float xh = X[o.pos[u]];
        // D = x(z_u) - x_hit as hi + lo
        float s, e, p, pe, s2, e2, p2, pe2, s3, e3;
        two_sum(th[0], -xh, s, e);
        two_prod(th[1], P.uzb[u], p, pe);
        two_sum(s, p, s2, e2);
        two_prod(th[2], P.uf_hi[u], p2, pe2);
        two_sum(s2, p2, s3, e3);
        const float lo = ((e + pe) + (e2 + pe2)) + (e3 + fmaf(th[2], P.uf_lo[u],
                          fmaf(dth[2], P.uf_hi[u], fmaf(dth[1], P.uzb[u], dth[0]))));
        // y = D / t as hi + lo: the remainder of the rounded quotient is exact,
        // so a reciprocal multiply loses nothing
        const float t = P.ut[u], it = P.uinv_t[u];
        const float yh = s3 * it;
        const float rm = fmaf(-yh, t, s3);
        const float yl = (rm + lo) * it;
        w[u] = fmaf(-ty, P.uz[u], yh) + yl;
        sw += w[u];
        sz += P.uzt[u];
    }
    const float inv_n = 1.f / static_cast<float>(o.n);
    const float wm = sw * inv_n, zm = sz * inv_n;
    float szz = 0.f, szw = 0.f;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        if (o.pos[u] < 0) continue;
        const float dz = P.uzt[u] - zm;
        szz = fmaf(dz, dz, szz);
        szw = fmaf(dz, w[u] - wm, szw);
    }
    const float beta = szw / szz;
    float chi2 = 0.f;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        if (o.pos[u] < 0) continue;
        const float r = (w[u] - wm) - beta * (P.uzt[u] - zm);
        chi2 = fmaf(r, r, chi2);
    }
    o.chi2 = chi2 * P.inv_sy2;
    o.beta = beta;
    o.wm = wm;
    o.zm = zm;
}

// A selection key per UV combination: fewer missing hits, then smaller chi2_y,
// then pass A, then the earlier initial hit (the order of Section 3.4's
// choice); the lowest 13 bits carry where the combination's hits were stored
// (kUvNotStored if they were not) and never decide.
constexpr int kUvStore = 8191;
constexpr int kUvNotStored = 8191;

__device__ __forceinline__ ull uv_key(int n, float chi2, int pass, int kinit, int stored) {
    return (ull(6 - n) << 61) | (ull(__float_as_uint(chi2) & 0x7fffffffu) << 30) | (ull(pass) << 29) |
           (ull(kinit) << 13) | ull(stored);
}

// x-z model of kept candidate k: th (3-hit model) and dth (fit correction),
// stored as rows th0..2, dth0..2 of c_f
struct XzModel {
    float th[3], dth[3];
};
__device__ __forceinline__ XzModel xz_model(const float* c_f, int CC, int k) {
    XzModel m;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        m.th[q] = c_f[q * CC + k];
        m.dth[q] = c_f[(3 + q) * CC + k];
    }
    return m;
}

// Cold path of the UV step: a valid combination that found the chain store
// full is fitted where it was found and takes part in the seed's choice by
// its key alone (its hits are searched again if it wins).
__device__ __forceinline__ void uv_fit_unstored_in(const DevParams& P, const float* X, const float* c_f, int CC,
                                                   int k, UV u, ull* ukey, int pass, int kinit) {
    const XzModel m = xz_model(c_f, CC, k);
    uv_fit(P, X, m.th, m.dth, u);
    atomicMin(ukey, uv_key(u.n, u.chi2, pass, kinit, kUvNotStored));
}
__device__ __noinline__ void uv_fit_unstored_out(const DevParams& P, const float* X, const float* c_f, int CC,
                                                 int k, UV u, ull* ukey, int pass, int kinit) {
    uv_fit_unstored_in(P, X, c_f, CC, k, u, ukey, pass, kinit);
}

// Cold path of the output step: the winning combination of a seed whose
// hits were not stored, searched again (same chain, same result) and fitted.
__device__ __forceinline__ UV uv_redo_in(const DevParams& P, const float* X, const int* szl, const uint16_t* lut,
                                         const uint32_t* used, const float* Xs, const float* c_f, int CC, int k,
                                         int h, const uint8_t* hc, ull key) {
    const int kinit = static_cast<int>((key >> 13) & 0xFFFFu);
    UV u;
    if (P.uv_mode == 1) {
        const int r = kinit / P.h_fine;
        uv_hough_in(P, X, szl, lut, used, Xs, hough_ty(P, h, hc[r], kinit - r * P.h_fine), u);
    } else {
        uv_chain(P, X, szl, lut, used, Xs, static_cast<int>((key >> 29) & 1), kinit, u);
    }
    const XzModel m = xz_model(c_f, CC, k);
    uv_fit(P, X, m.th, m.dth, u);
    return u;
}
__device__ __noinline__ UV uv_redo_out(const DevParams& P, const float* X, const int* szl, const uint16_t* lut,
                                       const uint32_t* used, const float* Xs, const float* c_f, int CC, int k, int h,
                                       const uint8_t* hc, ull key) {
    return uv_redo_in(P, X, szl, lut, used, Xs, c_f, CC, k, h, hc, key);
}

__device__ __forceinline__ ull pack_trip(int it, int k1, int k3, int k2) {
    return (ull(it) << 60) | (ull(k1) << 40) | (ull(k3) << 20) | ull(k2);
}

// The two-hit / third-hit windows of one pair: first T2 index and count
// (x2, l2, n2: the T2 slot's hits, bucket table and size).
__device__ __forceinline__ int pair_window(const DevParams& P, const IterP& I, const float* x2,
                                           const uint16_t* l2, int n2, float x1, float x3, int& lo2) {
    const float t13 = (x3 - x1) * I.inv_dz31;
    const float x0 = fmaf(-I.z1, t13, x1);
    const float ip = fmaf(P.invp_b * x0, x0, P.invp_a * fabsf(x0));
    lo2 = 0;
    if (!(ip > 0.f)) return 0;
    const float sg = x0 > 0.f ? 1.f : -1.f;
    const float ulo = fmaf(I.mlo_k, ip, -I.c0), uhi = fmaf(I.mhi_k, ip, I.c0);
    const float bs = fmaf(I.dz21, t13, x1);
    const float xa = fmaf(I.k3, -sg * ulo, bs), xb = fmaf(I.k3, -sg * uhi, bs);
    // the window is narrow (most hold no hit): one forward scan from the
    // bucket-table entry of its start passes the hits below it and counts
    // those in it (lo2 matters only when some are)
    const float lo = fminf(xa, xb), hi = fmaxf(xa, xb);
    int c = 0;
    for (int k = l2[lut_bin(lo)]; k < n2; ++k) {
        const float x = x2[k];
        if (hi < x) break;
        if (x < lo) continue;
        if (c == 0) lo2 = k;
        ++c;
    }
    return c;
}

constexpr int kTripPerCand = 2;  // triplet buffer entries per candidate slot
constexpr int kTripLocal = 12;   // triplets a thread buffers while walking its pairs

size_t seed_smem_bytes(int threads, int smem_hits, int tbl_smem, int key_smem) {
    return align16(sizeof(float) * smem_hits) + align16(sizeof(uint16_t) * 12 * kLutBins) +
           sizeof(ull) * (tbl_smem + key_smem) + sizeof(float) * 6 * key_smem + sizeof(int) * 3 * threads +
           sizeof(int) * (36 + 16);
}

size_t seed_slot_bytes(int cand_cap, int max_xhits) {
    return align16(sizeof(int) * 16 * size_t(cand_cap)) +
           sizeof(ull) * (size_t(max_xhits) + cand_cap + size_t(kTripPerCand) * cand_cap) +
           16 + (2 * sizeof(uint4) + sizeof(uint2)) * kUvStore + sizeof(float) * 6 * size_t(cand_cap) + 8 +
           sizeof(ull) * kTripLocal * kMaxThreads + 9 * size_t(cand_cap) + 4 +
           sizeof(uint32_t) * ((size_t(max_xhits) + 31) / 32);
}

// Two instantiations: CTAs of up to 256 threads with five per SM (48
// registers per thread: more resident warps hide the shared-memory and
// barrier latency better than fewer spills would), and up to 512 threads with
// two per SM (64 registers).
constexpr int kSeedBlocks256 = 5;

// Matching of one event, shared by k_match and the fused seeding kernel
// (defined with the matching kernel below).
struct MatchIO {
    const float* velo;         // x, y, tx, ty at z_velo
    const float* seed_state;   // x, y, tx, ty at z_state, per row
    const int8_t* seed_n;      // (nx, nuv) per row
    int32_t* velo_idx;         // per row
    float* chi2;               // per row
    float* ghost_prob;         // per row (final selection)
};
template <bool kFinal, class Row>
__device__ int match_event(const DevParams& P, const MatchIO& M, int VS, unsigned char* msm, int64_t v0, int nv,
                           int ns, Row row, int* s_cnt, ull& n_grid, ull& n_presel, ull& n_eval);

constexpr int kDeferRounds = 2;       // matching left to idle CTAs once fewer seeding items than this per CTA remain
// A wait for an announced event ends after SeedArgs::wait_ns of the global
// timer; the poll count is a second bound in case the timer stalls.
constexpr int kReadySpinsMax = 1 << 24;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// kSeq: compiled with the HLT2-style pass loop and taken-hit checks; the HLT1
// instantiation has neither (they fold away).
// kFuse: the kernel also matches each event, where the pool holds its
// records (HLT1 instantiation only).  The CTA that finishes the second of an
// event's two halves (a per-event counter) matches the event before its next
// item.  With defer_match, once fewer than kDeferRounds seeding items per CTA
// are left it announces the event in a ready list instead, and CTAs that find
// no seeding item left take the announced events (short items at the end
// balance the CTAs' finishing times); such a CTA waits (bounded) only while
// some event is still being seeded by a running CTA.  Kernels that share the
// GPU with others (the serving pipeline) do not defer: a waiting CTA would
// hold resources the other kernels could use.
template <int kT, int kB, bool kSeq, bool kFuse>
__global__ void __launch_bounds__(kT, kB)
k_seed(const __grid_constant__ DevParams P, const __grid_constant__ SeedArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x, tid = threadIdx.x;
    unsigned char* sp = smem;
    float* sx = reinterpret_cast<float*>(sp);
    sp += align16(sizeof(float) * A.smem_hits);
    uint16_t* lut = reinterpret_cast<uint16_t*>(sp);
    sp += align16(sizeof(uint16_t) * 12 * kLutBins);
    ull* stab = reinterpret_cast<ull*>(sp);
    sp += sizeof(ull) * A.tbl_smem;
    ull* skey = reinterpret_cast<ull*>(sp);
    sp += sizeof(ull) * A.key_smem;
    float* sXs = reinterpret_cast<float*>(sp);  // x at the 6 stereo layers per kept seed
    sp += sizeof(float) * 6 * A.key_smem;
    int* sPS = reinterpret_cast<int*>(sp);
    int* sA = sPS + T;
    int* sB = sA + T;
    int* tmp = sB + T;
    int* szl = tmp + 36;
    __shared__ int s_item;
    __shared__ ull s_start;
    // the x-z fit gains, indexed per thread by hit pattern: kept in shared
    // memory (divergent reads of kernel parameters serialise)
    __shared__ float sG[kMasks * 18];
    __shared__ int sMask[64];
    for (int i = tid; i < kMasks * 18; i += T) sG[i] = (&P.G[0][0][0])[i];
    for (int i = tid; i < 64; i += T) sMask[i] = P.mask_index[i];

    const int CC = A.cand_cap;
    const int TC = kTripPerCand * CC;
    uint8_t* slot = A.slot + int64_t(blockIdx.x) * A.slot_stride;
    int* c_pos = reinterpret_cast<int*>(slot);               // [6][CC]
    float* c_f = reinterpret_cast<float*>(c_pos + 6 * CC);  // [8][CC]: th0..2, dth0..2, chi2, score
    int* c_nx = reinterpret_cast<int*>(c_f + 8 * CC);
    int* kept = c_nx + CC;
    ull* g_tbl = reinterpret_cast<ull*>(slot + align16(sizeof(int) * 16 * size_t(CC)));
    ull* g_key = g_tbl + A.max_xhits;
    ull* trip = g_key + CC;
    // hits + ty of stored UV chains (16-byte aligned: the clone table before it
    // has max_xhits 8-byte entries, which may be odd)
    uint4* vstore = reinterpret_cast<uint4*>((reinterpret_cast<uintptr_t>(trip + TC) + 15) & ~uintptr_t(15));
    float4* vfit = reinterpret_cast<float4*>(vstore + kUvStore);   // (chi2_y, beta, wm, zm) of the fit
    uint2* vmeta = reinterpret_cast<uint2*>(vfit + kUvStore);      // (seed, pass | initial hit << 1)
    float* g_xs = reinterpret_cast<float*>(vmeta + kUvStore);
    // this thread's triplet buffer: entry q at tloc[q * T] (the block's first
    // entries are contiguous, so a round touches few cache lines)
    ull* tloc = reinterpret_cast<ull*>(g_xs + 6 * CC) + tid;
    uint8_t* hcl = reinterpret_cast<uint8_t*>(reinterpret_cast<ull*>(g_xs + 6 * CC) + kTripLocal * kMaxThreads);
    uint8_t* hn = hcl + 8 * CC;  // Hough variant: kept clusters per seed and their count
    // HLT2-style mode: bits of the half's hits taken by earlier iterations
    uint32_t* g_used = reinterpret_cast<uint32_t*>((reinterpret_cast<uintptr_t>(hn + CC) + 3) & ~uintptr_t(3));
    constexpr bool seq = kSeq;
    constexpr bool kOut = !kSeq;  // the out-of-line forms of the rarely run functions
    const uint32_t* used = kSeq ? g_used : nullptr;
    __shared__ int s_nvalid, s_cnt, s_match;
    __shared__ ull s_mctr[4];  // grid pairs, preselected pairs, Long tracks, evaluated pairs
    if (kFuse && tid < 4) s_mctr[tid] = 0;
    int spar = 0;  // which half of tmp the next block scan uses

    // work counters (pairs, triplets, extended, candidates, kept, UV initial
    // hits, valid UV chains, seeds): block totals, added up by thread 0
    __shared__ ull s_ctr[8];
    if (tid < 8) s_ctr[tid] = 0;
    // the staging copies' barrier (one phase per staged item)
    __shared__ ull s_mbar;
    if (tid == 0) mbar_init(&s_mbar, 1);
    unsigned mphase = 0;
    bool stage_ok = true;
    pdl_signal();
    pdl_wait();  // the containers and the item order

    int64_t fin = -1;  // fused: event of the half this CTA finished last
    for (;;) {
        if (kFuse && fin >= 0) __threadfence();  // the half's records, before its count
        __syncthreads();
        if (tid == 0) {
            s_match = -1;
            const int n2 = static_cast<int>(2 * A.n_events);
            if (kFuse && fin >= 0 && atomicAdd(A.ev_done + fin, 1) == 1) {
                // this CTA finished the event's second half (the other half's
                // records were released before its count; the fence orders
                // them before the reads of the matching)
                __threadfence();
                const int left = n2 - min(*reinterpret_cast<volatile int*>(A.queue), n2);
                if (!A.defer_match || left >= kDeferRounds * static_cast<int>(gridDim.x)) {
                    s_match = static_cast<int>(fin);  // matched by this CTA, now
                } else {
                    // near the end: left for whichever CTA runs out of seeding items first
                    atomicExch(A.ready + atomicAdd(A.ready_ctr, 1), static_cast<int>(fin) + 1);
                    __threadfence();
                }
                atomicAdd(A.done_ctr, 1);
            }
            if (s_match < 0) {
                const int q = atomicAdd(A.queue, 1);
                if (q < n2) {
                    s_item = A.order[q];
                } else if (kFuse && A.defer_match) {
                    // no seeding item left, and each is held by a running CTA:
                    // take the next announced event, or stop once every event
                    // is done and none is left for this slot
                    const int n = static_cast<int>(A.n_events);
                    const int m = atomicAdd(A.m_claim, 1);
                    const volatile int* vr = A.ready;
                    int v = 0;
                    bool gave_up = true;
                    const unsigned long long t_wait = global_ns();
                    for (int it = 0; it < kReadySpinsMax; ++it) {
                        // the time limit is checked first: with wait_ns = 0
                        // every wait gives up (the timeout path, for tests)
                        if (global_ns() - t_wait >= A.wait_ns) break;
                        if (m < n) v = vr[m];
                        if (v) {
                            gave_up = false;
                            break;
                        }
                        if (*reinterpret_cast<volatile int*>(A.done_ctr) >= n) {
                            __threadfence();
                            if (m < n) v = vr[m];
                            gave_up = false;
                            break;
                        }
                        __nanosleep(100);
                    }
                    if (gave_up) atomicExch(A.fault, 1);
                    __threadfence();
                    s_match = v - 1;
                    s_item = -1;
                } else {
                    s_item = -1;
                }
            }
        }
        __syncthreads();
        fin = -1;
        if (kFuse && s_match >= 0) {
            const int64_t em = s_match;
            const int c0 = __ldcg(A.item_count + 2 * em), c1 = __ldcg(A.item_count + 2 * em + 1);
            const int64_t r0 = c0 ? __ldcg(A.item_start + 2 * em) : 0;
            const int64_t r1 = c1 ? __ldcg(A.item_start + 2 * em + 1) : 0;
            const int64_t v0 = A.velo_off[em];
            const MatchIO M{A.velo, A.pool_state, A.pool_n, A.pool_velo, A.pool_chi2, nullptr};
            ull ng = 0, np = 0, nev = 0;
            const int nl = match_event<false>(P, M, A.velo_smem, smem, v0,
                                                    static_cast<int>(A.velo_off[em + 1] - v0), c0 + c1,
                                                    [&](int s) { return s < c0 ? r0 + s : r1 + (s - c0); },
                                                    &s_cnt, ng, np, nev);
            ng = warp_sum(ng);
            np = warp_sum(np);
            nev = warp_sum(nev);
            if ((tid & 31) == 0) {
                atomicAdd(&s_mctr[0], ng);
                atomicAdd(&s_mctr[1], np);
                atomicAdd(&s_mctr[3], nev);
            }
            if (tid == 0) {
                atomicAdd(&s_mctr[2], ull(nl));
                if (A.n_long) A.n_long[em] = nl;
            }
            continue;
        }
        const int64_t item = s_item;
        if (item < 0) break;
        const int64_t e = item >> 1;
        const int h = static_cast<int>(item & 1);
        if (kFuse) fin = e;
        if (A.status[e] != 0) {
            if (tid == 0) A.item_count[item] = 0;
            continue;
        }
        const int32_t* zo = A.zoff + e * kZoffStride + 12 * h;
        const int64_t cbh = cont_base(A.ev_off, e) + zo[0];
        const int nh = zo[12] - zo[0];
        if (tid <= 12) szl[tid] = zo[tid] - zo[0];
        const float* X = A.cx + cbh;
        // the half's hits are one contiguous slice: staged in shared memory by
        // one bulk copy of the 16-byte words that hold it (the container's
        // events start 16-byte aligned and are padded to a multiple of 16 bytes)
        const int64_t w0 = cbh & ~int64_t(3);
        const int lead = static_cast<int>(cbh - w0);
        const int nw = (lead + nh + 3) & ~3;
        if (stage_ok && nh > 0 && nw <= A.smem_hits) {
            if (tid == 0) bulk_to_smem(sx, A.cx + w0, 4u * unsigned(nw), &s_mbar);
            const bool got = mbar_wait(&s_mbar, mphase, kStagePolls);
            mphase ^= 1u;
            if (__syncthreads_or(!got)) {
                // the copy did not land: global reads from here on, the launch
                // marked faulty (every event then gets ST_TIMEOUT)
                stage_ok = false;
                if (tid == 0 && A.fault) atomicExch(A.fault, 1);
            } else {
                X = sx + lead;
            }
        }
        __syncthreads();

        // ------------------------------------------------------------ bucket tables
        for (int g = tid; g < nh; g += T) {
            int z = 0;
#pragma unroll
            for (int q = 1; q < 12; ++q) z += g >= szl[q];
            const int st = szl[z], n = szl[z + 1] - st, i = g - st;
            uint16_t* lz = lut + z * kLutBins;
            const int b = lut_bin(X[g]);
            const int bp = i == 0 ? -1 : lut_bin(X[g - 1]);
            for (int q = bp + 1; q <= b; ++q) lz[q] = static_cast<uint16_t>(i);
            if (i == n - 1)
                for (int q = b + 1; q < kLutBins; ++q) lz[q] = static_cast<uint16_t>(n);
        }
        for (int k = tid; k < 12 * kLutBins; k += T) {
            const int z = k / kLutBins;
            if (szl[z + 1] == szl[z]) lut[k] = 0;
        }
        __syncthreads();

        // HLT1: one pass over all iterations, then one clone kill and one UV
        // step.  HLT2-style (seq): one pass per iteration, each with its own
        // clone kill and UV step; the hits of a pass's seeds are marked in
        // g_used before the next pass.  Candidates and kept seeds of all
        // passes are appended to the same lists; the output step takes them
        // all.
        if (seq) {
            for (int i = tid; i < (nh + 31) / 32; i += T) g_used[i] = 0u;
        }
        if (tid == 0) s_nvalid = 0;
        __syncthreads();
        int ncand = 0, nk = 0;
        bool overflow = false;
        const bool hough = P.uv_mode == 1;
        const int n_pass = seq ? P.n_iter : 1;
        for (int ipass = 0; ipass < n_pass; ++ipass) {
        const int it_lo = seq ? ipass : 0, it_hi = seq ? ipass + 1 : P.n_iter;
        int n_items = 0;
        for (int it = it_lo; it < it_hi; ++it) n_items += szl[P.it[it].s1 + 1] - szl[P.it[it].s1];
        const int cb0 = ncand;
        // ------------------------------------------------------------ XZ
        // Each round takes up to T first hits (the pass's iterations' T1
        // layers in order), expands their T3 windows into pairs, and each
        // thread walks a contiguous range of the round's pairs (once into a
        // small buffer; again only if a thread found more triplets than it
        // holds), a block scan placing the triplets in order in the round's
        // triplet buffer; the triplets then become candidates.
        for (int b1 = 0; b1 < n_items; b1 += T) {
            const int i = b1 + tid;
            int np = 0, lo3 = 0, tag = 0;
            if (i < n_items) {
                int it = it_lo, k1 = i;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (it + 1 < it_hi) {
                        const int n1 = szl[P.it[it].s1 + 1] - szl[P.it[it].s1];
                        if (k1 >= n1) {
                            k1 -= n1;
                            ++it;
                        }
                    }
                }
                const IterP& I = P.it[it];
                const float x1 = X[szl[I.s1] + k1];
                const float xc = I.scale3 * x1;
                const int st3 = szl[I.s3], n3 = szl[I.s3 + 1] - st3;
                const uint16_t* l3 = lut + I.s3 * kLutBins;
                lo3 = zlo(X + st3, l3, n3, xc - I.dx3);
                np = zhi(X + st3, l3, n3, xc + I.dx3) - lo3;
                if (is_used(used, szl[I.s1] + k1)) np = 0;
                tag = (it << 20) | k1;
            }
            int tot_p;
            const int ps = block_exscan1(np, tmp, spar, tot_p);
            if (tid == 0) s_ctr[0] += tot_p;
            sPS[tid] = ps;
            sA[tid] = lo3;
            sB[tid] = tag;
            __syncthreads();
            int ntrip = 0;
            const int pb = static_cast<int>((int64_t(tot_p) * tid) / T);
            const int pe = static_cast<int>((int64_t(tot_p) * (tid + 1)) / T);
            // walk [pb, pe) once, buffering up to kTripLocal triplets per
            // thread; only if some thread found more is the walk repeated to
            // write them in place
            auto walk = [&](bool direct, int wofs) {
                int w = 0;
                if (pb >= pe) return 0;
                int o = owner_of(sPS, T, pb);
                int nxt = o + 1 < T ? sPS[o + 1] : tot_p;
                int k3 = sA[o] + (pb - sPS[o]);
                int tg = sB[o];
                int it = tg >> 20, k1 = tg & 0xFFFFF;
                // the owner's iteration's slot starts, kept while the owner lasts
                int st3 = szl[P.it[it].s3], st2 = szl[P.it[it].s2], n2 = szl[P.it[it].s2 + 1] - st2;
                float x1 = X[szl[P.it[it].s1] + k1];
                for (int p = pb; p < pe; ++p) {
                    while (p >= nxt) {
                        ++o;
                        nxt = o + 1 < T ? sPS[o + 1] : tot_p;
                        k3 = sA[o];
                        tg = sB[o];
                        it = tg >> 20;
                        k1 = tg & 0xFFFFF;
                        st3 = szl[P.it[it].s3];
                        st2 = szl[P.it[it].s2];
                        n2 = szl[P.it[it].s2 + 1] - st2;
                        x1 = X[szl[P.it[it].s1] + k1];
                    }
                    const IterP& I = P.it[it];
                    int lo2 = 0, c = 0;
                    if (!is_used(used, st3 + k3))
                        c = pair_window(P, I, X + st2, lut + I.s2 * kLutBins, n2, x1, X[st3 + k3], lo2);
                    for (int q = 0; q < c; ++q) {
                        if (is_used(used, st2 + lo2 + q)) continue;
                        const ull key = pack_trip(it, k1, k3, lo2 + q);
                        if (direct) trip[wofs + w] = key;
                        else if (w < kTripLocal) tloc[w * T] = key;
                        ++w;
                    }
                    ++k3;
                }
                return w;
            };
            const int nt = walk(false, 0);
            int tot_t;
            bool again;
            int wofs = block_exscan1_any(nt, nt > kTripLocal, tmp, spar, tot_t, again);
            if (tid == 0) s_ctr[1] += tot_t;
            if (ntrip + tot_t > TC) overflow = true;
            if (!overflow) {
                wofs += ntrip;
                ntrip += tot_t;
                if (again) {
                    walk(true, wofs);
                } else {
                    for (int q = 0; q < nt; ++q) trip[wofs + q] = tloc[q * T];
                }
            }
            __syncthreads();
            if (overflow) break;

            // this round's triplets -> candidates, in order
            for (int b = 0; b < ntrip; b += T) {
                const int t = b + tid;
                Trip o;
                int code = -1;
                if (t < ntrip) {
                    const ull tk = trip[t];
                    const int it = static_cast<int>(tk >> 60);
                    const int k1 = static_cast<int>((tk >> 40) & 0xFFFFF), k2 = static_cast<int>(tk & 0xFFFFF);
                    const int k3 = static_cast<int>((tk >> 20) & 0xFFFFF);
                    if constexpr (kOut)
                        code = do_triplet_out(P, P.it[it], X, szl, lut, sG, sMask, used, k1, k2, k3, o);
                    else
                        code = do_triplet(P, P.it[it], X, szl, lut, sG, sMask, used, k1, k2, k3, o);
                }
                // candidates in the low 16 bits, extended triplets (code >= 1)
                // in the high ones: at most one each per thread, so no carry
                int tot;
                const int co = block_exscan1((code == 2 ? 1 : 0) | (code >= 1 ? 0x10000 : 0), tmp, spar, tot) & 0xFFFF;
                if (tid == 0) s_ctr[2] += tot >> 16;
                tot &= 0xFFFF;
                if (code == 2) {
                    const int ci = ncand + co;
                    if (ci < CC) {
#pragma unroll
                        for (int s = 0; s < 6; ++s) c_pos[s * CC + ci] = o.pos[s];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            c_f[q * CC + ci] = o.th[q];
                            c_f[(3 + q) * CC + ci] = o.dth[q];
                        }
                        c_f[6 * CC + ci] = o.chi2;
                        c_f[7 * CC + ci] = o.score;
                        c_nx[ci] = o.nx;
                    }
                }
                ncand += tot;
            }
        }
        if (overflow || ncand > CC) {
            overflow = true;
            break;
        }

        // ------------------------------------------------------------ clone kill
        const int nxh = szl[6];
        ull* tbl = nxh <= A.tbl_smem ? stab : g_tbl;
        for (int i = tid; i < nxh; i += T) tbl[i] = ~0ull;
        __syncthreads();
        for (int k = cb0 + tid; k < ncand; k += T) {
            const ull key = (ull(__float_as_uint(c_f[7 * CC + k])) << 32) | unsigned(k);
#pragma unroll
            for (int s = 0; s < 6; ++s) {
                const int p = c_pos[s * CC + k];
                if (p >= 0) atomicMin(&tbl[p], key);
            }
        }
        __syncthreads();
        const int kb = nk;
        for (int b = cb0; b < ncand; b += T) {
            const int k = b + tid;
            int keep = 0;
            if (k < ncand) {
                const ull key = (ull(__float_as_uint(c_f[7 * CC + k])) << 32) | unsigned(k);
                int owned = 0;
#pragma unroll
                for (int s = 0; s < 6; ++s) {
                    const int p = c_pos[s * CC + k];
                    owned += p >= 0 && tbl[p] == key;
                }
                keep = owned >= 3 || (owned >= 2 && c_nx[k] == 6);
            }
            int tot;
            const int o = block_exscan1(keep, tmp, spar, tot);
            if (keep) kept[nk + o] = k;
            nk += tot;
        }
        if (tid == 0) s_ctr[4] += nk - kb;
        __syncthreads();

        // ------------------------------------------------------------ UV
        // (kept seeds [kb, nk) of this pass; with several passes the keys and
        // stereo positions live in global scratch)
        ull* ukey = (!seq && nk <= A.key_smem) ? skey : g_key;
        float* Xs = (!seq && nk <= A.key_smem) ? sXs : g_xs;
        const int nkp = nk - kb;
        const int nvs0 = min(s_nvalid, kUvStore);
        for (int j = kb + tid; j < nk; j += T) {
            ukey[j] = ~0ull;
            const int k = kept[j];
            const float th[3] = {c_f[k], c_f[CC + k], c_f[2 * CC + k]};
            const float dth[3] = {c_f[3 * CC + k], c_f[4 * CC + k], c_f[5 * CC + k]};
#pragma unroll
            for (int u = 0; u < 6; ++u) Xs[6 * j + u] = x_at_uv(P, th, dth, u);
        }
        __syncthreads();
        if (hough) {
            for (int j = kb + tid; j < nk; j += T)
                if constexpr (kOut)
                    hn[j] = static_cast<uint8_t>(hough_select_out(P, X, szl, lut, used, Xs + 6 * j, h, hcl + 8 * j));
                else
                    hn[j] = static_cast<uint8_t>(hough_select_in(P, X, szl, lut, used, Xs + 6 * j, h, hcl + 8 * j));
            __syncthreads();
        }
        // iterative: one item per (seed, pass), numbered pass-major (all pass
        // A chains, then pass B) so that a warp's chains mostly share their
        // initial layer; Hough: one item per seed with its hypotheses
        const int nuv = hough ? nkp : 2 * nkp;
        for (int b = 0; b < nuv; b += T) {
            const int i = b + tid;
            int cntc = 0, lo = 0;
            if (i < nuv && hough) {
                cntc = hn[kb + i] * P.h_fine;
            } else if (i < nuv) {
                const int pass = i >= nkp, j = kb + i - (pass ? nkp : 0);
                const int ui = P.uv_init[pass];
                const float Xi = Xs[6 * j + ui];
                const float t = P.ut[ui];
                const float xa = fmaf(-P.uv_yhi[h], t, Xi), xb = fmaf(-P.uv_ylo[h], t, Xi);
                const int st = szl[6 + ui], n = szl[7 + ui] - st;
                // the window holds a few hits: its end by a forward scan
                const float wlo = fminf(xa, xb), whi = fmaxf(xa, xb);
                const float* xs = X + st;
                lo = zlo(xs, lut + (6 + ui) * kLutBins, n, wlo);
                int e = lo;
                while (e < n && !(whi < xs[e])) ++e;
                cntc = e - lo;
            }
            int tot;
            const int ps = block_exscan1(cntc, tmp, spar, tot);
            if (tid == 0) s_ctr[5] += tot;
            sPS[tid] = ps;
            sA[tid] = lo;
            sB[tid] = i;
            __syncthreads();
            const int cb = static_cast<int>((int64_t(tot) * tid) / T);
            const int ce = static_cast<int>((int64_t(tot) * (tid + 1)) / T);
            if (cb < ce) {
                int o = owner_of(sPS, T, cb);
                int nxt = o + 1 < T ? sPS[o + 1] : tot;
                int kinit = sA[o] + (cb - sPS[o]);
                for (int c = cb; c < ce; ++c) {
                    while (c >= nxt) {
                        ++o;
                        nxt = o + 1 < T ? sPS[o + 1] : tot;
                        kinit = sA[o];
                    }
                    const int i2 = sB[o];
                    const int pass = hough ? 0 : i2 >= nkp, j = kb + i2 - (pass ? nkp : 0);
                    UV u;
                    if (hough) {
                        const int r = kinit / P.h_fine;
                        const float ty = hough_ty(P, h, hcl[8 * j + r], kinit - r * P.h_fine);
                        if constexpr (kOut)
                            uv_hough_out(P, X, szl, lut, used, Xs + 6 * j, ty, u);
                        else
                            uv_hough_in(P, X, szl, lut, used, Xs + 6 * j, ty, u);
                    } else if (is_used(used, szl[6 + P.uv_init[pass]] + kinit)) {
                        u.n = 0;  // initial hit taken by an earlier iteration
                    } else {
                        uv_chain(P, X, szl, lut, used, Xs + 6 * j, pass, kinit, u);
                    }
                    if (u.n >= P.n_uv_min) {
                        const int sidx = atomicAdd(&s_nvalid, 1);
                        if (sidx < kUvStore) {
                            uint4 r;
                            r.x = (unsigned(u.pos[0] + 1) & 0xFFFFu) | (unsigned(u.pos[1] + 1) << 16);
                            r.y = (unsigned(u.pos[2] + 1) & 0xFFFFu) | (unsigned(u.pos[3] + 1) << 16);
                            r.z = (unsigned(u.pos[4] + 1) & 0xFFFFu) | (unsigned(u.pos[5] + 1) << 16);
                            r.w = __float_as_uint(u.tyr);
                            vstore[sidx] = r;
                            vmeta[sidx] = make_uint2(unsigned(j), unsigned(pass) | (unsigned(kinit) << 1));
                        } else {
                            // store full: fit here; the winner is searched again at output
                            if constexpr (kOut)
                                uv_fit_unstored_out(P, X, c_f, CC, kept[j], u, &ukey[j], pass, kinit);
                            else
                                uv_fit_unstored_in(P, X, c_f, CC, kept[j], u, &ukey[j], pass, kinit);
                        }
                    }
                    ++kinit;
                }
            }
            __syncthreads();
        }
        // the stored chains' fits, one per thread
        const int nvs = min(s_nvalid, kUvStore);
        for (int q = nvs0 + tid; q < nvs; q += T) {
            const uint4 v = vstore[q];
            const uint2 mt = vmeta[q];
            const unsigned w[3] = {v.x, v.y, v.z};
            UV u;
            u.n = 0;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                u.pos[r] = static_cast<int>((w[r >> 1] >> (16 * (r & 1))) & 0xFFFFu) - 1;
                u.n += u.pos[r] >= 0;
            }
            u.tyr = __uint_as_float(v.w);
            const int j = static_cast<int>(mt.x);
            const int k = kept[j];
            const float th[3] = {c_f[k], c_f[CC + k], c_f[2 * CC + k]};
            const float dth[3] = {c_f[3 * CC + k], c_f[4 * CC + k], c_f[5 * CC + k]};
            uv_fit(P, X, th, dth, u);
            vfit[q] = make_float4(u.chi2, u.beta, u.wm, u.zm);
            atomicMin(&ukey[j], uv_key(u.n, u.chi2, static_cast<int>(mt.y & 1u), static_cast<int>(mt.y >> 1), q));
        }
        __syncthreads();
        if (seq && ipass + 1 < n_pass) {
            // hit cleanup: this pass's seeds give their hits to no later pass.
            // Their stereo hits come from the chain store; a pass whose store
            // overflowed cannot be cleaned up and counts as an overflow.
            if (s_nvalid > kUvStore) {
                overflow = true;
                break;
            }
            for (int j = kb + tid; j < nk; j += T) {
                const ull key = ukey[j];
                if (key == ~0ull) continue;
                const int k = kept[j];
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const int p = c_pos[q * CC + k];
                    if (p >= 0) atomicOr(&g_used[p >> 5], 1u << (p & 31));
                }
                const uint4 v = vstore[key & 0x1FFFu];
                const unsigned w[3] = {v.x, v.y, v.z};
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const int p = static_cast<int>((w[q >> 1] >> (16 * (q & 1))) & 0xFFFFu) - 1;
                    if (p >= 0) atomicOr(&g_used[p >> 5], 1u << (p & 31));
                }
            }
            __syncthreads();
        }
        }  // passes
        if (tid == 0) {
            s_ctr[3] += ncand;
            s_ctr[6] += s_nvalid;  // every valid UV chain of the item's passes
        }
        if (overflow || (seq && s_nvalid > kUvStore)) {
            if (tid == 0) {
                A.status[e] = -3;  // ST_OVERFLOW
                A.item_count[item] = 0;
            }
            continue;
        }
        ull* ukey = (!seq && nk <= A.key_smem) ? skey : g_key;
        float* Xs = (!seq && nk <= A.key_smem) ? sXs : g_xs;


        // ------------------------------------------------------------ seeds
        int nseed = 0;
        for (int b = 0; b < nk; b += T) {
            const int j = b + tid;
            const int has = j < nk && ukey[j] != ~0ull;
            nseed += __syncthreads_count(has);
        }
        if (tid == 0) {
            ull st = ~0ull;
            if (nseed > 0) {
                st = atomicAdd(A.pool_ctr, ull(nseed));
                if (st + nseed > ull(A.pool_cap)) {
                    A.status[e] = -3;
                    st = ~0ull;
                }
            }
            s_start = st;
            A.item_start[item] = st == ~0ull ? 0 : static_cast<int32_t>(st);
            A.item_count[item] = st == ~0ull ? 0 : nseed;
            s_ctr[7] += st == ~0ull ? 0 : nseed;
        }
        __syncthreads();
        if (s_start == ~0ull) continue;
        int wbase = 0;
        for (int b = 0; b < nk; b += T) {
            const int j = b + tid;
            const int has = j < nk && ukey[j] != ~0ull;
            int tot;
            const int o = block_exscan1(has, tmp, spar, tot);
            if (has) {
                const int64_t r = int64_t(s_start) + wbase + o;
                const ull key = ukey[j];
                const int sidx = static_cast<int>(key & 0x1FFFu);
                const int k = kept[j];
                const float th[3] = {c_f[k], c_f[CC + k], c_f[2 * CC + k]};
                const float dth[3] = {c_f[3 * CC + k], c_f[4 * CC + k], c_f[5 * CC + k]};
                UV u;
                if (sidx != kUvNotStored) {
                    const uint4 v = vstore[sidx];
                    const unsigned w[3] = {v.x, v.y, v.z};
                    u.n = 0;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        u.pos[q] = static_cast<int>((w[q >> 1] >> (16 * (q & 1))) & 0xFFFFu) - 1;
                        u.n += u.pos[q] >= 0;
                    }
                    u.tyr = __uint_as_float(v.w);
                    const float4 f = vfit[sidx];
                    u.chi2 = f.x;
                    u.beta = f.y;
                    u.wm = f.z;
                    u.zm = f.w;
                } else {
                    if constexpr (kOut)
                        u = uv_redo_out(P, X, szl, lut, used, Xs + 6 * j, c_f, CC, k, h, hcl + 8 * j, key);
                    else
                        u = uv_redo_in(P, X, szl, lut, used, Xs + 6 * j, c_f, CC, k, h, hcl + 8 * j, key);
                }
                // the record goes out as 16-byte stores (pool rows are 48 /
                // 32 / 16 bytes long and the pool is 256-byte aligned)
                // layers 0..11 are x u v x | x u v x | x u v x: x slot q and
                // stereo slot q in layer order
                auto hx = [&](int q) {
                    const int p = c_pos[q * CC + k];
                    return p >= 0 ? A.corig[cbh + p] : -1;
                };
                auto hu = [&](int q) { return u.pos[q] >= 0 ? A.corig[cbh + u.pos[q]] : -1; };
                int4* ho = reinterpret_cast<int4*>(A.pool_hits + r * 12);
                ho[0] = make_int4(hx(0), hu(0), hu(1), hx(1));
                ho[1] = make_int4(hx(2), hu(2), hu(3), hx(3));
                ho[2] = make_int4(hx(4), hu(4), hu(5), hx(5));
                const float a = th[0] + dth[0], bb = th[1] + dth[1], cc = th[2] + dth[2];
                // y(z) = tyr z + wm + beta (z - zc - zm)
                const float ty = u.tyr + u.beta;
                const float y0 = fmaf(-u.beta, P.zc_uv + u.zm, u.wm);
                const float yS = fmaf(u.tyr, P.zS, fmaf(u.beta, (P.zS - P.zc_uv) - u.zm, u.wm));
                float4* po = reinterpret_cast<float4*>(A.pool_params + r * 8);
                po[0] = make_float4(a, bb, cc, c_f[6 * CC + k]);
                po[1] = make_float4(y0, ty, u.chi2, 0.f);
                reinterpret_cast<float4*>(A.pool_state)[r] =
                    make_float4(fmaf(th[2], P.fS, fmaf(th[1], P.zbS, th[0])) +
                                    fmaf(dth[2], P.fS, fmaf(dth[1], P.zbS, dth[0])),
                                yS, fmaf(cc, P.dfS, bb), ty);
                const unsigned short nn = static_cast<unsigned short>((c_nx[k] & 0xFF) | ((u.n & 0xFF) << 8));
                reinterpret_cast<unsigned short*>(A.pool_n)[r] = nn;
            }
            wbase += tot;
        }
    }
    __syncthreads();
    // a copy given up on may still land: wait for it (bounded) before the
    // CTA's shared memory goes away
    if (!stage_ok) mbar_wait(&s_mbar, mphase ^ 1u, kStagePolls);
    if (tid < 8 && s_ctr[tid]) atomicAdd(A.counters + C_PAIRS + tid, s_ctr[tid]);
    if (kFuse && tid < 3 && s_mctr[tid]) atomicAdd(A.counters + C_MATCH_PAIRS + tid, s_mctr[tid]);
    if (kFuse && tid == 3 && s_mctr[3]) atomicAdd(A.counters + C_MATCH_EVAL, s_mctr[3]);
}

// ===========================================================================
// per-event CSR of the seed records
// ===========================================================================

__global__ void __launch_bounds__(1024) k_scan(const __grid_constant__ GatherArgs A) {
    __shared__ int tmp[36];
    pdl_signal();
    pdl_wait();  // the seeding kernel's item counts
    int64_t carry = 0;
    for (int64_t b = 0; b < A.n_events; b += blockDim.x) {
        const int64_t e = b + threadIdx.x;
        const int c = e < A.n_events ? A.item_count[2 * e] + A.item_count[2 * e + 1] : 0;
        int tot;
        const int ex = block_exscan(c, tmp, tot);
        if (e < A.n_events) A.ev_off[e] = static_cast<int32_t>(carry + ex);
        carry += tot;
    }
    if (threadIdx.x == 0) A.ev_off[A.n_events] = static_cast<int32_t>(carry);
}

// One block per event: the event's records come from the pool ranges of its
// two (event, half) items and go to one contiguous range of each output
// array, so every array is copied as a flat run (16-byte words when all
// output arrays allow it).
// (at most 32 registers: eight CTAs per SM, a 1000-event batch in one round)
template <bool kVec>
__global__ void __launch_bounds__(256, 8) k_gather(const __grid_constant__ GatherArgs A) {
    pdl_wait();  // the event offsets (and, through k_scan, the seed records)
    const bool fault = A.fault && *A.fault;
    for (int64_t e = blockIdx.x; e < A.n_events; e += gridDim.x) {
        if (fault && threadIdx.x == 0) A.status[e] = -4;  // ST_TIMEOUT: the fused matching gave up a wait
        const int c0 = A.item_count[2 * e], c1 = A.item_count[2 * e + 1];
        const int n = c0 + c1;
        if (n == 0) continue;
        const int64_t s0 = A.item_start[2 * e], s1 = A.item_start[2 * e + 1];
        const int64_t d0 = A.ev_off[e];
        auto src = [&](int k) { return k < c0 ? s0 + k : s1 + (k - c0); };
        const int T = blockDim.x;
        if (kVec) {
            // the event's 16-byte words as one range: hits (3 per record),
            // params (2), state (1); a thread loads four words before it stores
            // them, so their latencies overlap
            const uint4* ph = reinterpret_cast<const uint4*>(A.pool_hits);
            const uint4* pp = reinterpret_cast<const uint4*>(A.pool_params);
            const uint4* ps = reinterpret_cast<const uint4*>(A.pool_state);
            uint4* oh = reinterpret_cast<uint4*>(A.hits);
            uint4* op = reinterpret_cast<uint4*>(A.params);
            uint4* os = reinterpret_cast<uint4*>(A.state);
            const int W = 6 * n;
            for (int w0 = threadIdx.x; w0 < W; w0 += 4 * T) {
                uint4 v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int w = w0 + j * T;
                    if (w < 3 * n) {
                        const int k = w / 3;
                        v[j] = ph[src(k) * 3 + (w - 3 * k)];
                    } else if (w < 5 * n) {
                        const int u = w - 3 * n;
                        v[j] = pp[src(u >> 1) * 2 + (u & 1)];
                    } else if (w < W) {
                        v[j] = ps[src(w - 5 * n)];
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int w = w0 + j * T;
                    if (w < 3 * n) {
                        oh[d0 * 3 + w] = v[j];
                    } else if (w < 5 * n) {
                        op[d0 * 2 + (w - 3 * n)] = v[j];
                    } else if (w < W) {
                        os[d0 + (w - 5 * n)] = v[j];
                    }
                }
            }
            const uint16_t* pn = reinterpret_cast<const uint16_t*>(A.pool_n);
            uint16_t* on = reinterpret_cast<uint16_t*>(A.n_hits);
            for (int k = threadIdx.x; k < n; k += T) {
                const int64_t r = src(k);
                const uint16_t c = pn[r];
                if (A.pool_velo) {
                    const int32_t vi = A.pool_velo[r];
                    const float ch = A.pool_chi2[r];
                    A.velo_idx[d0 + k] = vi;
                    A.chi2[d0 + k] = ch;
                }
                on[d0 + k] = c;
            }
        } else {
            if (A.pool_velo) {
                for (int k = threadIdx.x; k < n; k += T) {
                    A.velo_idx[d0 + k] = A.pool_velo[src(k)];
                    A.chi2[d0 + k] = A.pool_chi2[src(k)];
                }
            }
            for (int i = threadIdx.x; i < 12 * n; i += blockDim.x) {
                const int k = i / 12, q = i - 12 * k;
                A.hits[(d0 + k) * 12 + q] = A.pool_hits[src(k) * 12 + q];
            }
            for (int i = threadIdx.x; i < 8 * n; i += blockDim.x) {
                const int k = i >> 3, q = i & 7;
                A.params[(d0 + k) * 8 + q] = A.pool_params[src(k) * 8 + q];
            }
            for (int i = threadIdx.x; i < 4 * n; i += blockDim.x) {
                const int k = i >> 2, q = i & 3;
                A.state[(d0 + k) * 4 + q] = A.pool_state[src(k) * 4 + q];
            }
            for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
                const int k = i >> 1, q = i & 1;
                A.n_hits[(d0 + k) * 2 + q] = A.pool_n[src(k) * 2 + q];
            }
        }
    }
}

// ===========================================================================
// matching
// ===========================================================================

constexpr int kTyBins = 64;
constexpr float kTyRange = 0.32f;  // buckets of 0.01 over [-0.32, 0.32); outside values go to the end buckets

size_t match_smem_bytes(int velo_smem) {
    return sizeof(float) * 7 * size_t(velo_smem) + sizeof(int) * (2 * size_t(velo_smem) + 2 * kTyBins + 8);
}

__device__ __forceinline__ int ty_bin(float ty) {
    const int b = __float2int_rd((ty + kTyRange) * (kTyBins / (2.f * kTyRange)));
    return min(max(b, 0), kTyBins - 1);  // NaN maps to bucket 0 and never passes the cuts
}

// One (VELO, seed) pair of Section 4: preselection, then chi2_match; updates
// the best (chi2, VELO index).  Position differences are formed from
// float-float extrapolations to z = A_x and z = z_match_y.
__device__ __forceinline__ int match_pair(const DevParams& P, float vxh, float vxl, float vyh, float vyl,
                                          float vtx, float vty, float vit, int vg, float xh, float xl,
                                          float yh, float yl, float txS, float tyS, float dzx, float& best,
                                          int& bv) {
    const float dtx = vtx - txS, dty = vty - tyS;
    if (!(fabsf(dty) < P.cut_ty) || !(fabsf(dtx) < P.cut_tx)) return 0;
    const float dy = (vyh - yh) + (vyl - yl);
    if (!(fabsf(dy) < P.cut_y)) return 0;
    const float dz = fmaf(P.Bx, fabsf(dtx), fmaf(P.Cx, dtx * dtx, fmaf(P.Ex * vtx, vtx, dzx)));
    const float dx = fmaf(dz, dtx, (vxh - xh) + (vxl - xl));
    if (!(fabsf(dx) < P.cut_x)) return 0;
    const float tolx = fmaf(P.tolx_b, dtx * dtx, P.tolx_a);
    const float c2 = dx * dx / tolx + dy * dy * vit + dtx * dtx * P.inv_toltx + dty * dty * P.inv_tolty;
    if (c2 < P.chi2m_max && (c2 < best || (c2 == best && vg < bv))) {
        best = c2;
        bv = vg;
    }
    return 1;
}

// The eight inputs of the ghost network (Section 4.4) for one pair: z_match_x,
// dx, dy, dtx, dty (formed like match_pair's), slot 5 left for chi2_match,
// the VELO segment's pseudorapidity asinh(1/|slope|) (= -ln tan(theta/2)),
// slot 7 left for the seed's hit count.
__device__ void pair_features(const DevParams& P, const float* vs, const float* ss, float f[8]) {
    const float x = vs[0], y = vs[1], tx = vs[2], ty = vs[3];
    float p, pe, s, se;
    two_prod(P.dAV_hi, tx, p, pe);
    two_sum(x, p, s, se);
    const float vxh = s, vxl = se + fmaf(P.dAV_lo, tx, pe);
    two_prod(P.dMV_hi, ty, p, pe);
    two_sum(y, p, s, se);
    const float vyh = s, vyl = se + fmaf(P.dMV_lo, ty, pe);
    const float xS = ss[0], yS = ss[1], txS = ss[2], tyS = ss[3];
    float xh, xl, yh, yl;
    two_prod(P.dAS_hi, txS, p, pe);
    two_sum(xS, p, xh, xl);
    xl += fmaf(P.dAS_lo, txS, pe);
    two_prod(P.dMS_hi, tyS, p, pe);
    two_sum(yS, p, yh, yl);
    yl += fmaf(P.dMS_lo, tyS, pe);
    const float dtx = tx - txS, dty = ty - tyS;
    const float dz = fmaf(P.Bx, fabsf(dtx), fmaf(P.Cx, dtx * dtx, fmaf(P.Ex * tx, tx, P.Dx * fabsf(xS))));
    f[0] = P.A_hi + (P.A_lo + dz);
    f[1] = fmaf(dz, dtx, (vxh - xh) + (vxl - xl));
    f[2] = (vyh - yh) + (vyl - yl);
    f[3] = dtx;
    f[4] = dty;
    f[6] = asinhf(1.f / fmaxf(sqrtf(fmaf(tx, tx, ty * ty)), 1e-6f));
}

// The ghost network: standardised inputs, 32 ReLU nodes, sigmoid output.
// Every lane reads the same weight at the same time (uniform constant reads).
__device__ float ghost_nn(const DevParams& P, const float f[8]) {
    float in[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) in[i] = (f[i] - P.nn[i]) * P.nn[8 + i];
    float z = P.nn[336];
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        float a = P.nn[272 + k];
#pragma unroll
        for (int i = 0; i < 8; ++i) a = fmaf(P.nn[16 + 8 * k + i], in[i], a);
        if (a > 0.f) z = fmaf(P.nn[304 + k], a, z);
    }
    return 1.f / (1.f + expf(-z));
}

// Matching of one event (Section 4), one thread per seed: the event's VELO
// segments are staged in shared memory (msm, match_smem_bytes(VS) bytes) with
// their float-float extrapolations and bucketed by ty, so a seed only visits
// the buckets its |dty| cut can reach (every other pair fails that cut).
// Events with more segments than fit are processed in chunks, each scanned in
// full.  Seed s (0 .. ns-1, in the event's canonical seed order) reads its
// state and hit counts and writes its pair at index row(s) of M's arrays.
// Returns the event's Long-track count; n_grid / n_presel accumulate this
// thread's pair counts.
template <bool kFinal, class Row>
__device__ int match_event(const DevParams& P, const MatchIO& M, int VS, unsigned char* msm, int64_t v0, int nv,
                           int ns, Row row, int* s_cnt, ull& n_grid, ull& n_presel, ull& n_eval) {
    const int T = blockDim.x, tid = threadIdx.x;
    float* vxh = reinterpret_cast<float*>(msm);
    float* vxl = vxh + VS;
    float* vyh = vxl + VS;
    float* vyl = vyh + VS;
    float* vtx = vyl + VS;
    float* vty = vtx + VS;
    float* vit = vty + VS;
    int* bidx = reinterpret_cast<int*>(vit + VS);  // VELO indices grouped by ty bucket
    int* bcnt = bidx + VS;                         // [kTyBins]
    int* boff = bcnt + kTyBins;                    // [kTyBins + 1]
    unsigned* vmin = reinterpret_cast<unsigned*>(boff + kTyBins + 8);  // final selection: lowest ghost
                                                                       // probability per VELO segment
    if (tid == 0) *s_cnt = 0;
    const bool bucketed = nv <= VS;
    for (int vc = 0; vc < nv; vc += VS) {
        const int m = min(VS, nv - vc);
        for (int k = tid; k < kTyBins; k += T) bcnt[k] = 0;
        __syncthreads();
        for (int v = tid; v < m; v += T) {
            const float* st = M.velo + (v0 + vc + v) * 4;
            const float x = st[0], y = st[1], tx = st[2], ty = st[3];
            float p, pe, s, se;
            two_prod(P.dAV_hi, tx, p, pe);
            two_sum(x, p, s, se);
            vxh[v] = s;
            vxl[v] = se + fmaf(P.dAV_lo, tx, pe);
            two_prod(P.dMV_hi, ty, p, pe);
            two_sum(y, p, s, se);
            vyh[v] = s;
            vyl[v] = se + fmaf(P.dMV_lo, ty, pe);
            vtx[v] = tx;
            vty[v] = ty;
            vit[v] = 1.f / fmaf(P.toly_b, fmaf(tx, tx, ty * ty), P.toly_a);
            if (bucketed) atomicAdd(&bcnt[ty_bin(ty)], 1);
        }
        __syncthreads();
        if (bucketed) {
            if (tid < 32) {  // exclusive scan of the bucket counts by one warp
                int c0 = bcnt[2 * tid], c1 = bcnt[2 * tid + 1];
                int x = c0 + c1;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (tid >= o) x += y;
                }
                const int ex = x - c0 - c1;
                boff[2 * tid] = ex;
                boff[2 * tid + 1] = ex + c0;
                if (tid == 31) boff[kTyBins] = x;
            }
            __syncthreads();
            for (int q = tid; q < kTyBins; q += T) bcnt[q] = boff[q];  // reuse as fill cursors
            __syncthreads();
            for (int v = tid; v < m; v += T) bidx[atomicAdd(&bcnt[ty_bin(vty[v])], 1)] = v;
            __syncthreads();
        }
        for (int s = tid; s < ns; s += T) {
            // read past L1: in the fused kernel other CTAs wrote the rows during this launch
            const float* st = M.seed_state + row(s) * 4;
            const float xS = __ldcg(st), yS = __ldcg(st + 1), txS = __ldcg(st + 2), tyS = __ldcg(st + 3);
            float p, pe, xh, xl, yh, yl;
            two_prod(P.dAS_hi, txS, p, pe);
            two_sum(xS, p, xh, xl);
            xl += fmaf(P.dAS_lo, txS, pe);
            two_prod(P.dMS_hi, tyS, p, pe);
            two_sum(yS, p, yh, yl);
            yl += fmaf(P.dMS_lo, tyS, pe);
            const float dzx = P.Dx * fabsf(xS);
            float best = FLT_MAX;
            int bv = 0x7fffffff;
            if (vc > 0) {
                const int pv = M.velo_idx[row(s)];
                if (pv >= 0) {
                    bv = pv;
                    best = M.chi2[row(s)];
                }
            }
            int npre = 0;
            if (bucketed) {
                // buckets that can hold |ty - tyS| < cut_ty (slightly widened;
                // the exact cut is applied per pair)
                const float w = P.cut_ty + 1e-6f * (fabsf(tyS) + P.cut_ty);
                const int k0 = boff[ty_bin(tyS - w)], k1 = boff[ty_bin(tyS + w) + 1];
                n_eval += k1 - k0;
                for (int k = k0; k < k1; ++k) {
                    const int v = bidx[k];
                    npre += match_pair(P, vxh[v], vxl[v], vyh[v], vyl[v], vtx[v], vty[v], vit[v], vc + v,
                                       xh, xl, yh, yl, txS, tyS, dzx, best, bv);
                }
            } else {
                n_eval += m;
                for (int v = 0; v < m; ++v)
                    npre += match_pair(P, vxh[v], vxl[v], vyh[v], vyl[v], vtx[v], vty[v], vit[v], vc + v,
                                       xh, xl, yh, yl, txS, tyS, dzx, best, bv);
            }
            n_presel += npre;
            n_grid += m;
            const bool found = best < FLT_MAX;
            M.velo_idx[row(s)] = found ? bv : -1;
            M.chi2[row(s)] = found ? best : 0.f;
        }
        __syncthreads();
    }
    if (nv == 0) {
        for (int s = tid; s < ns; s += T) {
            M.velo_idx[row(s)] = -1;
            M.chi2[row(s)] = 0.f;
        }
    }
    __syncthreads();
    if (P.velo_unique) {
        // a VELO segment keeps its best seed (lowest chi2, then lower seed
        // index); losers are marked -2 - v so that concurrent readers still
        // see which segment they held
        for (int s = tid; s < ns; s += T) {
            const int v = M.velo_idx[row(s)];
            if (v < 0) continue;
            const float c = M.chi2[row(s)];
            for (int t = 0; t < ns; ++t) {
                if (t == s) continue;
                int vt = M.velo_idx[row(t)];
                if (vt <= -2) vt = -2 - vt;
                if (vt != v) continue;
                const float ct = M.chi2[row(t)];
                if (ct < c || (ct == c && t < s)) {
                    M.velo_idx[row(s)] = -2 - v;
                    break;
                }
            }
        }
        __syncthreads();
        for (int s = tid; s < ns; s += T) {
            if (M.velo_idx[row(s)] <= -2) {
                M.velo_idx[row(s)] = -1;
                M.chi2[row(s)] = 0.f;
            }
        }
        __syncthreads();
    }
    if (kFinal && P.final_sel) {
        // Section 4.4: ghost probability of each best pair and the cut
        for (int s = tid; s < ns; s += T) {
            const int v = M.velo_idx[row(s)];
            float p = 1.f;
            if (v >= 0) {
                float f[8];
                pair_features(P, M.velo + (v0 + v) * 4, M.seed_state + row(s) * 4, f);
                f[5] = M.chi2[row(s)];
                f[7] = static_cast<float>(M.seed_n[2 * row(s)] + M.seed_n[2 * row(s) + 1]);
                p = ghost_nn(P, f);
                if (!(p < P.ghost_max)) {
                    M.velo_idx[row(s)] = -1;
                    M.chi2[row(s)] = 0.f;
                }
            }
            M.ghost_prob[row(s)] = p;
        }
        __syncthreads();
        // clones: a kept pair whose VELO segment another kept pair holds
        // with a ghost probability lower by at least clone_margin (one
        // pair per seed, so no two pairs share a seed); marked -2 - v.
        // With clone_margin > 0 that is p - (lowest p on the segment) >=
        // clone_margin; the lowest p per segment is an atomicMin of the
        // probabilities' bits (non-negative floats order as unsigned).
        if (nv <= VS) {
            for (int v = tid; v < nv; v += T) vmin[v] = 0x7f800000u;
            __syncthreads();
            for (int s = tid; s < ns; s += T) {
                const int v = M.velo_idx[row(s)];
                if (v >= 0) atomicMin(&vmin[v], __float_as_uint(M.ghost_prob[row(s)]));
            }
            __syncthreads();
            for (int s = tid; s < ns; s += T) {
                const int v = M.velo_idx[row(s)];
                if (v >= 0 && M.ghost_prob[row(s)] - __uint_as_float(vmin[v]) >= P.clone_margin)
                    M.velo_idx[row(s)] = -2 - v;
            }
        } else {
            for (int s = tid; s < ns; s += T) {
                const int v = M.velo_idx[row(s)];
                if (v < 0) continue;
                const float p = M.ghost_prob[row(s)];
                for (int t = 0; t < ns; ++t) {
                    if (t == s) continue;
                    int vt = M.velo_idx[row(t)];
                    if (vt <= -2) vt = -2 - vt;
                    if (vt == v && p - M.ghost_prob[row(t)] >= P.clone_margin) {
                        M.velo_idx[row(s)] = -2 - v;
                        break;
                    }
                }
            }
        }
        __syncthreads();
        for (int s = tid; s < ns; s += T) {
            if (M.velo_idx[row(s)] <= -2) {
                M.velo_idx[row(s)] = -1;
                M.chi2[row(s)] = 0.f;
            }
        }
        __syncthreads();
    }
    int nl = 0;
    for (int s = tid; s < ns; s += T) nl += M.velo_idx[row(s)] >= 0;
    nl = warp_sum(nl);
    if ((tid & 31) == 0 && nl) atomicAdd(s_cnt, nl);
    __syncthreads();
    return *s_cnt;
}

// One event per work item (match_event), for matching_run on seeds in the
// per-event CSR layout.
// kFinal: compiled with the final selection of Section 4.4 (the plain
// instantiation does not carry its registers).
template <bool kFinal>
__global__ void __launch_bounds__(kMaxThreads)
k_match(const __grid_constant__ DevParams P, const __grid_constant__ MatchArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    __shared__ int s_item, s_cnt;
    ull ctr[4] = {0, 0, 0, 0};  // grid pairs, preselected pairs, Long tracks, evaluated pairs
    const MatchIO M{A.velo, A.seed_state, A.seed_n, A.velo_idx, A.chi2, A.ghost_prob};

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(A.queue, 1);
        __syncthreads();
        const int64_t e = s_item;
        if (e >= A.n_events) break;
        const int64_t v0 = A.velo_off[e];
        const int nv = static_cast<int>(A.velo_off[e + 1] - v0);
        const int64_t s0 = A.seed_off[e];
        const int ns = A.seed_off[e + 1] - static_cast<int>(s0);
        const int nl = match_event<kFinal>(P, M, A.velo_smem, smem, v0, nv, ns,
                                           [&](int s) { return s0 + s; }, &s_cnt, ctr[0], ctr[1], ctr[3]);
        if (tid == 0) {
            if (A.n_long) A.n_long[e] = nl;
            ctr[2] += nl;
        }
    }
    flush_counters(A.counters + C_MATCH_PAIRS, ctr, 3);
    flush_counters(A.counters + C_MATCH_EVAL, ctr + 3, 1);
}

// ===========================================================================
// launchers
// ===========================================================================

// Raise each kernel's dynamic shared-memory ceiling to what the device allows
// next to the kernel's own static shared memory (opt-in maximum - static).
cudaError_t set_smem_limits(size_t optin) {
    const void* fns[] = {reinterpret_cast<const void*>(k_build),
                         reinterpret_cast<const void*>(k_seed<256, kSeedBlocks256, false, false>),
                         reinterpret_cast<const void*>(k_seed<kMaxThreads, 2, false, false>),
                         reinterpret_cast<const void*>(k_seed<256, kSeedBlocks256, true, false>),
                         reinterpret_cast<const void*>(k_seed<kMaxThreads, 2, true, false>),
                         reinterpret_cast<const void*>(k_seed<256, kSeedBlocks256, false, true>),
                         reinterpret_cast<const void*>(k_match<false>), reinterpret_cast<const void*>(k_match<true>)};
    for (const void* f : fns) {
        cudaFuncAttributes fa;
        cudaError_t err = cudaFuncGetAttributes(&fa, f);
        if (err != cudaSuccess) return err;
        const int dyn = static_cast<int>(optin) - static_cast<int>(fa.sharedSizeBytes);
        if ((err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess)
            return err;
    }
    return cudaSuccess;
}

// Whether the ceilings set_smem_limits raises are still in place (a
// cudaDeviceReset drops them with the context): checked on the container
// kernel, the first one set_smem_limits raises.
cudaError_t smem_limits_hold(size_t optin, bool& hold) {
    cudaFuncAttributes fa;
    const cudaError_t err = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(k_build));
    hold = err == cudaSuccess &&
           fa.maxDynamicSharedSizeBytes >= static_cast<int>(optin) - static_cast<int>(fa.sharedSizeBytes);
    return err;
}

int build_blocks_per_sm(int threads, size_t smem) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_build, threads, smem);
    return n;
}
int seed_blocks_per_sm(int threads, size_t smem) {
    int n = 0;
    if (threads <= 256)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_seed<256, kSeedBlocks256, false, false>, threads, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_seed<kMaxThreads, 2, false, false>, threads, smem);
    return n;
}
int match_blocks_per_sm(int threads, size_t smem) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_match<false>, threads, smem);
    return n;
}

// A launch as a programmatic dependent of the stream's previous kernel
// (chained), or a plain one.
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*k)(KArgs...), unsigned grid, unsigned threads, size_t smem, cudaStream_t s,
                            bool chained, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = chained ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

cudaError_t launch_build(const DevParams& P, const BuildArgs& a, int grid, int threads, cudaStream_t s, bool chained) {
    k_build<<<grid, threads, build_smem_bytes(a.bins, a.smem_hits), s>>>(P, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t items = 2 * a.n_events;
    if (items <= 0) return cudaSuccess;
    return launch_k(k_order, static_cast<unsigned>((items + kOrderThreads - 1) / kOrderThreads), kOrderThreads, 0, s,
                    chained, a);
}

cudaError_t launch_seed(const DevParams& P, const SeedArgs& a, int grid, int threads, cudaStream_t s, bool chained) {
    const size_t smem = seed_smem_bytes(threads, a.smem_hits, a.tbl_smem, a.key_smem);
    const bool sq = P.iter_mode == 1;
    void (*k)(const DevParams, const SeedArgs);
    if (a.velo) {  // fused matching: the runtime only asks for it where this instantiation applies
        if (threads > 256 || sq) return cudaErrorInvalidValue;
        k = k_seed<256, kSeedBlocks256, false, true>;
    } else if (threads <= 256) {
        k = sq ? k_seed<256, kSeedBlocks256, true, false> : k_seed<256, kSeedBlocks256, false, false>;
    } else {
        k = sq ? k_seed<kMaxThreads, 2, true, false> : k_seed<kMaxThreads, 2, false, false>;
    }
    return launch_k(k, static_cast<unsigned>(grid), static_cast<unsigned>(threads), smem, s, chained, P, a);
}

cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s, bool chained) {
    cudaError_t err = launch_k(k_scan, 1, 1024, 0, s, chained, a);
    if (err != cudaSuccess) return err;
    const int grid = static_cast<int>(std::min<int64_t>(a.n_events, 8192));
    if (grid <= 0) return cudaSuccess;
    // pool arrays are 256-byte aligned; the caller's output arrays may not be
    const uintptr_t mis = (reinterpret_cast<uintptr_t>(a.hits) | reinterpret_cast<uintptr_t>(a.params) |
                           reinterpret_cast<uintptr_t>(a.state)) & 15u;
    const bool vec = mis == 0 && (reinterpret_cast<uintptr_t>(a.n_hits) & 1u) == 0;
    return launch_k(vec ? k_gather<true> : k_gather<false>, static_cast<unsigned>(grid), 256, 0, s, true, a);
}

cudaError_t launch_match(const DevParams& P, const MatchArgs& a, int grid, int threads, cudaStream_t s) {
    if (P.final_sel)
        k_match<true><<<grid, threads, match_smem_bytes(a.velo_smem), s>>>(P, a);
    else
        k_match<false><<<grid, threads, match_smem_bytes(a.velo_smem), s>>>(P, a);
    return cudaGetLastError();
}

}  // namespace st
