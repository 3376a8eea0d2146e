// st_static.cu -- seeding_run_static: the seeding chain with all of its
// scratch in one array compiled into the library, for callers that cannot
// allocate device memory.
//
// Who cannot allocate: a process whose device memory is owned by a host
// framework's own allocator (every cudaMalloc outside it breaks its
// accounting), or a real-time event loop that forbids allocation once it has
// started, because cudaMalloc / cudaFree can synchronise the device and stall
// the loop for milliseconds.  Such callers still own their inputs and
// outputs; this entry point only needs a place for its intermediate data.
//
// The array g_scratch below is a `__device__` variable: every GPU that loads
// the library holds ST_STATIC_SCRATCH_BYTES of it until the process exits.
// In host code its name is only a host-side stand-in, so the device address is
// obtained with cudaGetSymbolAddress (with that device current) on the first
// call per device, checked again on later calls made outside stream capture,
// and passed to the kernels as a pointer.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "st.h"
#include "st_host.h"
#include "st_kernels.cuh"

using namespace st;

static __device__ __align__(256) unsigned char g_scratch[ST_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
constexpr int kStaticMaxHits = 6144;  // every event's per-hit sort arrays fit in shared memory

struct DeviceSetup {
    bool done = false;
    unsigned char* base = nullptr;  // device address of g_scratch on this device
    int n_sms = 0;
    int optin = 0;                  // opt-in shared memory per CTA
};

std::mutex g_mu;
DeviceSetup g_setup[kMaxDevices];

int fail(char* err, int err_len, int code, const char* fmt, ...) {
    if (err && err_len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, static_cast<size_t>(err_len), fmt, ap);
        va_end(ap);
    }
    return code;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// With `dev` current.  The first call on a device looks up the array's
// device address and raises the kernels' shared-memory ceilings.  Later calls
// outside stream capture check both again, since a cudaDeviceReset in between
// ends the context that held them: the address is looked up anew and the
// ceilings raised again if they are gone.  Inside a capture the cached values
// are used (the first call must come before any capture).
int setup_device(int dev, bool capturing, DeviceSetup*& out, char* err, int err_len) {
    std::lock_guard<std::mutex> g(g_mu);
    DeviceSetup& S = g_setup[dev];
    if (S.done && capturing) {
        out = &S;
        return ST_OK;
    }
    if (!S.done) {
        cudaError_t e = cudaDeviceGetAttribute(&S.n_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return fail(err, err_len, ST_ECUDA, "device set-up: %s", cudaGetErrorString(e));
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess)
        return fail(err, err_len, ST_ECUDA, "cudaGetSymbolAddress(g_scratch): %s", cudaGetErrorString(e));
    bool hold = false;
    e = smem_limits_hold(size_t(S.optin), hold);
    if (e == cudaSuccess && !hold) e = set_smem_limits(size_t(S.optin));
    if (e != cudaSuccess) return fail(err, err_len, ST_ECUDA, "device set-up: %s", cudaGetErrorString(e));
    S.base = static_cast<unsigned char*>(p);
    S.done = true;
    out = &S;
    return ST_OK;
}

}  // namespace

extern "C" int seeding_run_static(const st_config* cfg, const st_hits* H, st_seeds* S, void* stream,
                                  char* err, int32_t err_len) {
    if (err && err_len > 0) err[0] = '\0';
    if (!cfg || !H || !S) return fail(err, err_len, ST_EINVAL, "null argument");
    if (H->n_events < 0 || (H->n_events > 0 && (!H->ev_off || !H->x || !H->zone)))
        return fail(err, err_len, ST_EINVAL, "st_hits: null array or negative n_events");
    if (H->max_hits_per_event < 1 || H->max_hits_per_event > kStaticMaxHits)
        return fail(err, err_len, ST_OVERFLOW, "max_hits_per_event must be in [1, %d] for the static scratch",
                    kStaticMaxHits);
    if (S->cap < 0 || S->cap > INT32_MAX || !S->ev_off || !S->status ||
        (S->cap > 0 && (!S->hits || !S->params || !S->state || !S->n_hits)))
        return fail(err, err_len, ST_EINVAL, "st_seeds: null array or bad cap");
    DevParams P;
    std::string msg;
    if (!derive_params(*cfg, P, msg)) return fail(err, err_len, ST_EINVAL, "config: %s", msg.c_str());
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(err, err_len, ST_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(err, err_len, ST_EINVAL, "device index %d out of range", dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap_st);
    if (e != cudaSuccess) return fail(err, err_len, ST_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    DeviceSetup* D = nullptr;
    int rc = setup_device(dev, cap_st != cudaStreamCaptureStatusNone, D, err, err_len);
    if (rc != ST_OK) return rc;

    // carve the static array for this batch
    const int64_t ne = H->n_events, mh = H->max_hits_per_event, items = 2 * ne;
    const int64_t cont = ne * mh + 3 * ne + 8;  // container entries for events within max_hits
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += up256(bytes);
        return o;
    };
    const size_t o_q = take(64 + 2 * 128 * sizeof(int32_t));  // queues, pool counter, item-class counts
    const size_t o_cnt = take(sizeof(unsigned long long) * C_N);
    const size_t o_zoff = take(sizeof(int32_t) * size_t(ne) * kZoffStride + 4);
    const size_t o_cx = take(sizeof(float) * size_t(cont));
    const size_t o_co = take(sizeof(int32_t) * size_t(cont));
    const size_t o_is = take(sizeof(int32_t) * size_t(items) + 4);
    const size_t o_ic = take(sizeof(int32_t) * size_t(items) + 4);
    const size_t o_icl = take(sizeof(int32_t) * size_t(items) + 4);
    const size_t o_ord = take(sizeof(int32_t) * size_t(items) + 4);
    const size_t o_ph = take(sizeof(int32_t) * 12 * size_t(S->cap) + 4);
    const size_t o_pp = take(sizeof(float) * 8 * size_t(S->cap) + 4);
    const size_t o_ps = take(sizeof(float) * 4 * size_t(S->cap) + 4);
    const size_t o_pn = take(2 * size_t(S->cap) + 4);
    const size_t slot_stride = up256(seed_slot_bytes(cfg->cand_cap, static_cast<int>(mh)));
    const size_t fixed = off;
    if (fixed + slot_stride > size_t(ST_STATIC_SCRATCH_BYTES))
        return fail(err, err_len, ST_OVERFLOW,
                    "batch needs %zu bytes of scratch (%lld events, max %lld hits/event, %lld seeds) but the "
                    "static scratch holds %zu; split the batch or lower seeds cap / cand_cap",
                    fixed + slot_stride, (long long)ne, (long long)mh, (long long)S->cap,
                    size_t(ST_STATIC_SCRATCH_BYTES));
    const int64_t slots_fit = int64_t((size_t(ST_STATIC_SCRATCH_BYTES) - fixed) / slot_stride);
    unsigned char* b = D->base;

    // what must start at zero each call: work queues, the pool counter and the
    // (discarded) work counters; everything else is written before it is read
    e = cudaMemsetAsync(b + o_q, 0, o_cnt + sizeof(unsigned long long) * C_N - o_q, s);
    if (e != cudaSuccess) return fail(err, err_len, ST_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    if (ne == 0) {
        e = cudaMemsetAsync(S->ev_off, 0, sizeof(int32_t), s);
        return e == cudaSuccess ? ST_OK : fail(err, err_len, ST_ECUDA, "%s", cudaGetErrorString(e));
    }
    int32_t* queues = reinterpret_cast<int32_t*>(b + o_q);
    unsigned long long* pool_ctr = reinterpret_cast<unsigned long long*>(b + o_q + 32);
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(b + o_cnt);

    int bins = 8;
    while (bins < 512 && bins * 96 < mh) bins <<= 1;
    const size_t bsmem = build_smem_bytes(bins, static_cast<int>(mh));
    const int tbl_smem = cfg->smem_hits / 2, key_smem = std::max(64, cfg->smem_hits / 8);  // as st_create
    const size_t ssmem = seed_smem_bytes(cfg->threads_seed, cfg->smem_hits, tbl_smem, key_smem);
    // the shared-memory check of st_create (2 KB left for static shared memory)
    if (ssmem + 2048 > size_t(D->optin) || bsmem + 2048 > size_t(D->optin))
        return fail(err, err_len, ST_EINVAL,
                    "config needs %zu (seeding) / %zu (containers) bytes of shared memory per CTA; the device "
                    "allows %d", ssmem, bsmem, D->optin);
    int bbps = std::max(1, build_blocks_per_sm(cfg->threads_build, bsmem));
    int sbps = std::max(1, seed_blocks_per_sm(cfg->threads_seed, ssmem));
    if (cfg->ctas_per_sm > 0) {  // as seeding_run
        bbps = std::min(bbps, cfg->ctas_per_sm);
        sbps = std::min(sbps, cfg->ctas_per_sm);
    }
    const int g_build = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ne, int64_t(D->n_sms) * bbps)));
    const int g_seed = static_cast<int>(
        std::max<int64_t>(1, std::min<int64_t>({items, int64_t(D->n_sms) * sbps, slots_fit})));

    BuildArgs ba;
    ba.n_events = ne;
    ba.ev_off = H->ev_off;
    ba.x = H->x;
    ba.zone = H->zone;
    ba.z = H->z;
    ba.dxdy = H->dxdy;
    ba.max_hits = static_cast<int32_t>(mh);
    ba.bins = bins;
    ba.smem_hits = static_cast<int32_t>(mh);
    ba.cont_cap = cont;
    ba.cx = reinterpret_cast<float*>(b + o_cx);
    ba.corig = reinterpret_cast<int32_t*>(b + o_co);
    ba.zoff = reinterpret_cast<int32_t*>(b + o_zoff);
    ba.status = S->status;
    ba.big = nullptr;
    ba.big_stride = 0;
    ba.item_class = reinterpret_cast<int32_t*>(b + o_icl);
    ba.class_count = queues + 16;
    ba.class_fill = queues + 16 + 128;
    ba.order = reinterpret_cast<int32_t*>(b + o_ord);
    ba.queue = queues + 0;
    ba.counters = counters;
    e = launch_build(P, ba, g_build, cfg->threads_build, s);
    if (e != cudaSuccess) return fail(err, err_len, ST_ECUDA, "k_build: %s", cudaGetErrorString(e));

    SeedArgs sa;
    sa.n_events = ne;
    sa.ev_off = H->ev_off;
    sa.cx = ba.cx;
    sa.corig = ba.corig;
    sa.zoff = ba.zoff;
    sa.status = S->status;
    sa.smem_hits = cfg->smem_hits;
    sa.cand_cap = cfg->cand_cap;
    sa.tbl_smem = tbl_smem;
    sa.key_smem = key_smem;
    sa.slot = b + fixed;
    sa.slot_stride = static_cast<int64_t>(slot_stride);
    sa.max_xhits = static_cast<int32_t>(mh);
    sa.pool_hits = reinterpret_cast<int32_t*>(b + o_ph);
    sa.pool_params = reinterpret_cast<float*>(b + o_pp);
    sa.pool_state = reinterpret_cast<float*>(b + o_ps);
    sa.pool_n = reinterpret_cast<int8_t*>(b + o_pn);
    sa.pool_cap = S->cap;
    sa.pool_ctr = pool_ctr;
    sa.item_start = reinterpret_cast<int32_t*>(b + o_is);
    sa.item_count = reinterpret_cast<int32_t*>(b + o_ic);
    sa.order = ba.order;
    sa.queue = queues + 1;
    sa.counters = counters;
    sa.fault = queues + 4;  // set if a staging copy was given up on
    e = launch_seed(P, sa, g_seed, cfg->threads_seed, s);
    if (e != cudaSuccess) return fail(err, err_len, ST_ECUDA, "k_seed: %s", cudaGetErrorString(e));

    GatherArgs ga;
    ga.n_events = ne;
    ga.item_start = sa.item_start;
    ga.item_count = sa.item_count;
    ga.pool_hits = sa.pool_hits;
    ga.pool_params = sa.pool_params;
    ga.pool_state = sa.pool_state;
    ga.pool_n = sa.pool_n;
    ga.cap = S->cap;
    ga.ev_off = S->ev_off;
    ga.hits = S->hits;
    ga.params = S->params;
    ga.state = S->state;
    ga.n_hits = S->n_hits;
    ga.status = S->status;
    ga.fault = sa.fault;
    e = launch_gather(ga, s);
    if (e != cudaSuccess) return fail(err, err_len, ST_ECUDA, "gather: %s", cudaGetErrorString(e));
    return ST_OK;
}
