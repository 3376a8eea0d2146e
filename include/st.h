/*
 * st.h -- C ABI of libst: GB300 (sm_103a) SciFi Seeding and VELO-SciFi
 * Matching, the hot path of the backward long-track reconstruction described
 * in "Seeding and Matching algorithms for the first GPU-based High Level
 * Trigger of the LHCb experiment" (Sections 3 and 4).
 *
 * Problem statement (Abstract, Section 4): from the hits of the SciFi tracker
 * build T-track segments ("seeds"), then link each seed to the VELO segment
 * whose straight-line extrapolation matches it best, forming a Long track.
 *
 * Conventions for every entry point
 *  - Return value is an st_status; nothing aborts, traps or exits.
 *  - Device pointers are owned by the caller (e.g. torch tensors) and are never
 *    freed or retained beyond the call's stream work.  Host pointers are read
 *    during the call only, unless stated otherwise.
 *  - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *    void*; NULL = legacy default stream) and is asynchronous unless stated.
 *  - Indices of hits are event-local: 0 .. hits-of-the-event-1, in the
 *    caller's order.  Seeds and VELO states are likewise event-local.
 *  - Per-event problems (invalid hit, capacity exceeded) are reported in the
 *    per-event status array, never by writing out of bounds.
 *  - A context is used by one host thread at a time, except the pipeline_*
 *    calls, which are thread-safe.
 */
#ifndef ST_H
#define ST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ST_OK = 0,
    ST_PENDING = 1,     /* pipeline_poll: result not ready yet */
    ST_EINVAL = -1,     /* invalid argument / input */
    ST_ENOMEM = -2,     /* device or pinned allocation failed */
    ST_OVERFLOW = -3,   /* a capacity was exceeded (per event, or call-level) */
    ST_TIMEOUT = -4,    /* pipeline_poll: the wait ran out; per event: a bounded device wait gave up */
    ST_ECUDA = -5,      /* a CUDA runtime call failed; see st_last_error */
    ST_ESTATE = -6      /* call not valid in the context's current state */
} st_status;

#define ST_NLAYER 12

/*
 * Method parameters and launch tuning.  All geometry in mm.  Fill with
 * st_config_default() and override fields.  Layers: 12 SciFi layers, three
 * stations of four layers ordered x,u,v,x (Section 1); zone = 2*layer + half,
 * half 1 holding the hits of particles at y >= 0 (Section 5.2).
 */
typedef struct {
    double z[ST_NLAYER];       /* layer z */
    double dxdy[ST_NLAYER];    /* tan of the stereo angle: 0 (x), +tan5 (u), -tan5 (v) */
    double z_ref;              /* reference z of the track model, Eq. (trackequation) */
    double d_ratio;            /* fixed cubic-correction coefficient of Eq. (trackequation) */
    /* XZ seeding (Section 3.3) */
    double invp_a, invp_b;     /* Eq. (invp): 1/p = a|x0| + b x0^2 (1/p in (MeV/c)^-1) */
    double p_min;              /* MeV/c, both iterations (Section 3.2) */
    double alpha0, alpha1;     /* Eq. (alphacorr), MeV/c */
    double dx3_scale;          /* scales Delta x3^max of Eq. (tolHp); 1 = paper */
    int32_t n_iter;            /* XZ iterations (2 in HLT1, up to 3) */
    int32_t iter_layers[3][3]; /* initial x-layers (T1, T2, T3) of each iteration */
    double kappa_c;            /* third-hit band centre: -sign(x0)*c_x = kappa_c * (1/p) */
    double m_lo, m_hi;         /* band edges as multiples of the centre */
    double c_nsigma;           /* band widening, in units of the c_x resolution */
    double sigma_x;            /* x resolution (mm) used in the band and in chi2_x */
    double ext_tol;            /* x-layer extension tolerance (Section 3.2): 1 mm */
    double chi2x_max;          /* x-z fit cut on chi2/ndf */
    double score_w_chi2;       /* Eq. (seed_clone_score): 1000 */
    double score_w5;           /* Eq. (seed_clone_score): 10 for five-hit tracks */
    /* UV seeding (Section 3.4) */
    int32_t uv_init[2];        /* initial stereo layer of pass A and pass B */
    int32_t n_uv_min;          /* stereo hits a seed needs (2..6) */
    int32_t pad1;
    double uv_tol;             /* closest stereo hit within 2 mm */
    double uv_y_overlap;       /* first-layer window reaches this far into the other half */
    double uv_y_max;           /* |y| limit of the first-layer window */
    double sigma_y;            /* y resolution used in chi2_y */
    double z_state;            /* z of the seed state handed to matching */
    /* Matching (Section 4) */
    double z_velo;             /* z of the VELO states */
    double z_match_y;          /* y matching plane: 10 m */
    double zmx[5];             /* A_x..E_x of Eq. (z_match) */
    double presel[4];          /* |dx|, |dy|, |dtx|, |dty| preselection cuts (Section 4.2) */
    double presel_scale;       /* multiplies the four preselection cuts */
    double tol_scale;          /* multiplies tol_x, tol_y, tol_tx, tol_ty */
    double tolx[3];            /* tol_x = tolx0 (tolx1^2 + tolx2^2 dtx^2) */
    double toly[3];            /* tol_y = toly0 (toly1^2 + toly2^2 (tx^2 + ty^2)) */
    double tol_tx, tol_ty;
    double chi2_match_max;     /* chi2_match < 2 */
    int32_t velo_unique;       /* 1: a VELO segment keeps only its best seed */
    /* launch tuning (no effect on results) */
    int32_t threads_seed;      /* threads per CTA of the seeding kernel: 64, 128, 256, 512 */
    int32_t threads_build;     /* threads per CTA of the container kernel */
    int32_t threads_match;     /* threads per CTA of the matching kernel */
    int32_t ctas_per_sm;       /* persistent CTAs per SM (0 = occupancy maximum) */
    int32_t smem_hits;         /* hits of one detector half staged in shared memory */
    int32_t cand_cap;          /* x-z candidates per (event, half) work item */
    int32_t pad2;
    /* UV seeding, Hough-cluster variant (Section 3.4, second approach; bin
     * counts and ranges are not given in the paper) */
    int32_t uv_mode;           /* 0: iterative over an initial layer (default), 1: Hough clusters */
    int32_t hough_bins;        /* coarse t_y bins (2..64); a cluster is two adjacent bins */
    int32_t hough_fine;        /* t_y hypotheses per kept cluster, at sub-bin centres (1..8) */
    int32_t hough_clusters;    /* clusters kept per seed, most populated first (1..8) */
    double hough_ty_max;       /* coarse t_y range [-hough_ty_in, hough_ty_max] for half 1, */
    double hough_ty_in;        /* mirrored for half 0 */
    /* Matching final selection (Section 4.4): ghost network, cut, clone removal */
    int32_t final_sel;         /* 1: apply it in matching_run (weights from st_set_ghost_nn) */
    int32_t pad3;
    double ghost_max;          /* keep pairs with ghost probability below 0.8 */
    double clone_margin;       /* drop a pair sharing a segment with one at least 0.05 less ghost-like (> 0) */
    /* UT hits of the Long tracks (Section 4.3, ut_run) */
    double ut_z[4];            /* UT layers UTaX, UTaU, UTbV, UTbX (not given in the paper) */
    double ut_dxdy[4];         /* stereo slopes of the UT layers (x, u, v, x) */
    double ut_gamma[2];        /* Eq. (gamma_parametrisation): A_gamma, B_gamma (per MeV) */
    double ut_kick;            /* a pair's q/p = (tx_SciFi - tx_VELO) / ut_kick (MeV) */
    double ut_loose[16];       /* per UT layer: A_L (mm), B_L (mm GeV/c), x_min, x_max; zeros = none */
    double ut_tight[16];       /* per UT layer: A_T, B_T, x_min, x_max; zeros = none */
    int32_t ut_min_hits;       /* Long tracks need this many UT hits in ut_run (0 = no requirement) */
    /* Iteration scheme (Section 3.1): 0 = HLT1, independent iterations and one
     * clone kill at the end; 1 = HLT2-style, iterations in sequence, each with
     * its own clone kill and UV step, the hits of its seeds removed before
     * the next iteration */
    int32_t iter_mode;
    double p_min_iter[3];      /* per-iteration p_min (MeV/c); 0 = p_min */
} st_config;

/* Hits of a batch of events (CSR).  All arrays are DEVICE memory.
 * ev_off[n_events+1] (int64, non-decreasing) indexes x / zone / z / dxdy;
 * ev_off[0] need not be 0.  z and dxdy may be NULL; when given, each hit's
 * value must equal the configured value of its layer within 1e-3 mm / 1e-6,
 * else the event's status is ST_EINVAL.  max_hits_per_event is a host-side
 * bound; larger events get ST_OVERFLOW.  Events with a zone outside [0, 24)
 * or a non-finite x get ST_EINVAL. */
typedef struct {
    int64_t n_events;
    const int64_t* ev_off;
    const float* x;
    const int32_t* zone;
    const float* z;
    const float* dxdy;
    int32_t max_hits_per_event;
    int32_t pad;
} st_hits;

/* Seeding output (T tracks).  All arrays DEVICE memory, caller-allocated.
 *   ev_off  [n_events+1] int32: seeds of event e are [ev_off[e], ev_off[e+1])
 *   hits    [cap*12]     int32: event-local hit index per layer, -1 = none
 *   params  [cap*8]      float: a, b, c (x-z model), chi2_x, y0, ty, chi2_y, 0
 *   state   [cap*4]      float: x, y, tx, ty at z_state
 *   n_hits  [cap*2]      int8 : x-layer hits, stereo hits
 *   status  [n_events]   int32: ST_OK, ST_EINVAL or ST_OVERFLOW
 * Within an event, seeds of half 0 precede those of half 1, each in the
 * deterministic order of the search (iteration, T1 hit, T3 hit, T2 hit). */
typedef struct {
    int64_t cap;
    int32_t* ev_off;
    int32_t* hits;
    float* params;
    float* state;
    int8_t* n_hits;
    int32_t* status;
} st_seeds;

/* VELO segments (CSR), DEVICE memory: state[4*i] = x, y, tx, ty at z_velo. */
typedef struct {
    int64_t n_events;
    const int64_t* ev_off;
    const float* state;
} st_velo;

/* Matching output, one entry per seed (same indexing as st_seeds), DEVICE:
 *   velo_idx   [cap] int32: event-local VELO index of the Long track, -1 = none
 *   chi2       [cap] float: chi2_match of that pair (0 if none)
 *   n_long     [n_events] int32 (may be NULL): Long tracks per event
 *   ghost_prob [cap] float: with final_sel (required then; may be NULL
 *              otherwise) the ghost network's output for the seed's best
 *              pair, 1 if the seed had none */
typedef struct {
    int32_t* velo_idx;
    float* chi2;
    int32_t* n_long;
    float* ghost_prob;
} st_long;

/* Per-stage work counters, summed over the calls since the last reset.
 * match_pairs is the full VELO x seed grid of Section 4.2; match_eval the
 * pairs the matching kernel actually evaluates (those in the ty buckets the
 * |dty| preselection cut can reach; every other pair fails that cut). */
typedef struct {
    int64_t pairs, triplets, ext_ok, cands, kept, uv_init, uv_cands, seeds;
    int64_t match_pairs, match_presel, matched;
    int64_t hits, events;
    int64_t match_eval;
} st_counters;

typedef struct st_ctx st_ctx;
typedef struct st_graph st_graph;

/* Fill *cfg with the paper's constants (Sections 3-4), this library's
 * readings of the values the paper leaves open, and default tuning. */
void st_config_default(st_config* cfg);

/* Create a context on CUDA device `device` (made current for the call).
 * Validates cfg (ST_EINVAL), derives the device constants and allocates the
 * counters.  Scratch memory is allocated on first use or by st_reserve.
 * *out receives the context; destroy it with st_destroy. */
int st_create(const st_config* cfg, int device, st_ctx** out);

/* Waits for the context's pipeline work, frees its memory and the context.
 * NULL is accepted. */
void st_destroy(st_ctx* ctx);

/* Message of the last failing call on this context (owned by the context,
 * valid until the next call).  Never NULL. */
const char* st_last_error(const st_ctx* ctx);

/* Pre-allocate scratch for batches of up to n_events events, n_hits hits,
 * max_hits_per_event hits per event and seeds_cap seeds, so that later
 * seeding_run / matching_run calls allocate nothing (required before CUDA
 * graph capture).  Synchronous. */
int st_reserve(st_ctx* ctx, int64_t n_events, int64_t n_hits, int32_t max_hits_per_event,
               int64_t seeds_cap);

/* SciFi Seeding (Section 3): per event, hit containers sorted by (layer
 * zone, x); XZ iterations of two-hit (Eqs. tolHp, alphacorr) and three-hit
 * (Section 3.3.3) searches; extension to the other x-layers (1 mm) keeping
 * >= 5 hits; least-squares x-z fit with d_ratio fixed and a chi2/ndf cut;
 * O(n) clone killing (Eq. seed_clone_score and the two-pass vote of Section
 * 3.3.4); UV seeding (Section 3.4, iterative or Hough clusters by uv_mode).
 * iter_mode 0 (HLT1): the iterations run independently and one clone kill
 * follows; iter_mode 1: each iteration in turn with its own clone kill and
 * UV step, the hits of its seeds removed before the next (an event whose
 * store of UV combinations overflows in this mode gets ST_OVERFLOW).
 * Output `seeds` as described at st_seeds.  Returns ST_EINVAL for a bad
 * argument (NULL array, cap < 0, n_events < 0), ST_ENOMEM / ST_ECUDA for
 * allocation or launch failures; per-event problems go to seeds->status.
 * Each (event, half) work item's hits are staged in shared memory by one
 * bulk copy whose completion the kernel waits for with a bound; a copy that
 * never lands (which a working device cannot produce) gives every event of
 * the launch ST_TIMEOUT.
 * Allocates scratch if st_reserve was not called for this size. */
int seeding_run(st_ctx* ctx, const st_hits* hits, st_seeds* seeds, void* cuda_stream);

/* VELO-SciFi Matching (Section 4): for every seed, every VELO segment of
 * the same event is extrapolated with the seed to the kink plane z_match_x
 * (Eq. z_match) and to z_match_y; pairs passing the preselection (Section
 * 4.2) get chi2_match; the seed's Long track is the pair with the lowest
 * chi2_match below chi2_match_max (ties: lower VELO index).  `seeds` must be
 * a seeding_run output for the same events (velo->n_events events).  With
 * cfg.final_sel = 1 the final selection of Section 4.4 follows: the ghost
 * network (weights from st_set_ghost_nn) evaluates every best pair from its
 * z_match_x, dx, dy, dtx, dty, chi2_match, the VELO segment's pseudorapidity
 * and the seed's SciFi hit count; pairs with a ghost probability >= ghost_max
 * are dropped, and a pair sharing its VELO segment with a kept pair whose
 * ghost probability is lower by >= clone_margin is dropped as a clone
 * (velo_idx = -1, chi2 = 0).  ST_ESTATE if final_sel is set and no weights
 * were given.  The UT-hit search of Section 4.3 is not part of this call.
 * Errors as seeding_run. */
int matching_run(st_ctx* ctx, const st_velo* velo, const st_seeds* seeds, st_long* out,
                 void* cuda_stream);

/* UT hits of a batch (CSR), DEVICE memory: x is the measured coordinate at
 * y = 0 along the strip, layer 0..3 = UTaX, UTaU, UTbV, UTbX. */
typedef struct {
    int64_t n_events;
    const int64_t* ev_off;  /* [n_events + 1] into x / layer */
    const float* x;
    const int32_t* layer;
} st_ut_hits;

/* UT search output, one entry per seed (st_seeds indexing), DEVICE:
 *   hits  [cap*4] int32: event-local UT hit index per UT layer, -1 = none
 *   n_hits[cap]   int8:  UT hits attached
 *   gamma [cap]   float: the final gamma_x of Eq. (velo_ut_extrapolation) */
typedef struct {
    int32_t* hits;
    int8_t* n_hits;
    float* gamma;
} st_ut_out;

/* UT hits of the Long tracks (Section 4.3), after matching_run on the same
 * seeds: for every seed with out->velo_idx >= 0 the VELO segment is
 * extrapolated with Eq. (velo_ut_extrapolation), gamma_x from Eq.
 * (gamma_parametrisation) at the pair's q/p = (tx_SciFi - tx_VELO) / ut_kick,
 * through the UT layers in order: until a hit is found a layer is searched in
 * its loose window min(max(A_L + B_L/p, x_min), x_max) and the closest hit in
 * it is attached and refits gamma_x through itself; later layers use their
 * tight windows (closest hit attached).  Ties go to the smaller x, then the
 * smaller hit index.  A Long track with fewer than cfg.ut_min_hits UT hits is
 * dropped (velo_idx = -1, chi2 = 0) and n_long (if given) is recounted.  An
 * event with a UT layer outside [0, 4) or a non-finite x gets
 * seeds->status = ST_EINVAL and no UT hits.  Errors as seeding_run. */
int ut_run(st_ctx* ctx, const st_velo* velo, const st_seeds* seeds, const st_ut_hits* ut, st_long* out,
           st_ut_out* ut_out, void* cuda_stream);

/* Weights of the ghost network (Section 4.4): ST_GHOST_NN_SIZE floats, HOST
 * memory, copied.  Layout: input mean[8] and inverse scale[8] (each input is
 * standardised as (f - mean) * inv_scale), W1[32][8], b1[32] (hidden layer,
 * ReLU), w2[32], b2 (output, sigmoid).  The trained weights of the paper are
 * not published; any set may be given.  Call before the matching work that
 * should use it.  ST_EINVAL for a wrong size or a non-finite value. */
#define ST_GHOST_NN_SIZE 337
int st_set_ghost_nn(st_ctx* ctx, const float* weights, int32_t n);

/* Capture seeding_run + matching_run for these exact buffers and sizes into a
 * CUDA graph (persistent, work-queue kernels).  Scratch must be reserved
 * first (st_reserve).  The arguments' pointers must stay valid while the
 * graph exists.  *out receives the graph; launch with st_graph_launch.
 * With threads_seed <= 256, iter_mode 0 and no final selection the matching
 * runs inside the seeding kernel (each event as soon as its two halves are
 * seeded); the outputs are those of the two calls.  If that kernel ever gave
 * up a (bounded) wait for an event being seeded, which a correct run cannot
 * do, every event of the launch gets status ST_TIMEOUT.  The serving pipeline
 * runs batches the same way. */
int st_graph_create(st_ctx* ctx, const st_hits* hits, const st_velo* velo, st_seeds* seeds,
                    st_long* out, st_graph** graph);
int st_graph_launch(st_graph* graph, void* cuda_stream);
void st_graph_destroy(st_graph* graph);

/* Kernel timing (a tracing aid).  When enabled, seeding_run, matching_run
 * and graphs created afterwards record CUDA events around each kernel on the
 * launch stream.  st_kernel_ms waits for the last recorded work and returns
 * the durations (ms) of its kernels: [0] hit containers, [1] seeding,
 * [2] seed gather, [3] matching (0 for kernels not run). */
int st_set_timing(st_ctx* ctx, int enable);
int st_kernel_ms(st_ctx* ctx, float ms[4]);

/* Longest time (nanoseconds of the device's global timer) a CTA of the fused
 * seeding kernel (st_graph_create, the serving pipeline) waits for an event
 * that another running CTA is still seeding.  Default 200 ms; a correct run
 * waits for microseconds.  A wait that runs out sets a fault word and every
 * event of that launch gets status ST_TIMEOUT; the kernel returns normally
 * and the context stays usable.  0 makes every such wait give up at once (to
 * exercise that path).  Applies to launches prepared after the call (a graph
 * keeps the limit it was captured with).  ST_EINVAL for ns < 0.  Section 5.3
 * describes the batch of events this kernel runs; the limit itself has no
 * counterpart in the paper. */
int st_set_wait_limit(st_ctx* ctx, int64_t ns);

/* Counters of the work done since the last reset (synchronises the device).
 * reset != 0 zeroes them afterwards. */
int st_read_counters(st_ctx* ctx, st_counters* out, int reset);

/* ---------------------------------------------------------------------- */
/* Seeding without allocation.  The paper has no counterpart to this entry   */
/* point; it exists for callers that cannot allocate device memory.          */
/* ---------------------------------------------------------------------- */

/* Size of the scratch array compiled into the library: every GPU that loads
 * libst holds this much device memory until the process exits. */
#define ST_STATIC_SCRATCH_BYTES (16u << 20)

/* seeding_run without a context and without any allocation: the same
 * kernels, with all intermediate data (hit containers, per-event slot
 * offsets, work queues, per-CTA candidate storage, seed pool) in one fixed
 * array of ST_STATIC_SCRATCH_BYTES inside the library.  For callers that
 * cannot call cudaMalloc: a process whose device memory belongs to a host
 * framework's own allocator, or a real-time event loop that forbids
 * allocation after start-up because cudaMalloc / cudaFree can synchronise the
 * device and stall it.
 *
 * Arguments and output are those of seeding_run (DEVICE pointers owned by the
 * caller), cfg replaces the context, and the work runs on the device that is
 * current for the calling thread.  The results equal seeding_run's.
 * Limits: max_hits_per_event <= 6144, and the batch must fit the array:
 * (8*max_hits_per_event + 156) bytes per event plus 98*seeds->cap bytes plus
 * one candidate store of about 121*cand_cap + 8*max_hits_per_event + 377 KB
 * (e.g. 128 events of up to 4096 hits with 40 000 seeds fit); otherwise it
 * returns ST_OVERFLOW, writes nothing, and the message gives the exact byte
 * count the batch needs.  A configuration whose shared-memory needs exceed
 * the device's (the check st_create makes) gives ST_EINVAL.  Launch shapes
 * follow cfg as in seeding_run, ctas_per_sm included.  A NUL-terminated
 * message goes to err (may be NULL) on every failure.
 *
 * The first call on a device sets that device up (looks up the array's device
 * address and raises the kernels' shared-memory limits); make that first call
 * before any stream capture.  Later calls outside a capture check that set-up
 * again, so a call after cudaDeviceReset sets the device up anew; calls inside
 * a capture use what the last call outside one found.  Every call reuses the
 * same array: work queues and counters are cleared at the start of each call,
 * and calls that overlap on the GPU (different streams or host threads at
 * once) race on it, so serialise them.  Returns ST_OK, ST_EINVAL, ST_OVERFLOW
 * or ST_ECUDA. */
int seeding_run_static(const st_config* cfg, const st_hits* hits, st_seeds* seeds, void* cuda_stream,
                       char* err, int32_t err_len);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of host-side event batches.                */
/* ---------------------------------------------------------------------- */

/* Serving limits; set before the first pipeline_submit. */
typedef struct {
    int32_t n_slots;             /* batches in flight on the device (streams) */
    int32_t max_events_per_slot; /* events packed into one launch */
    int64_t max_hits_per_slot;   /* hits packed into one launch */
    int32_t max_hits_per_event;
    int32_t max_velo_per_event;
    int64_t mem_cap_bytes;       /* device + pinned memory the pipeline may hold */
    int64_t max_velo_per_slot;   /* VELO segments packed into one launch */
} st_pipeline_config;

void st_pipeline_config_default(st_pipeline_config* pc);
int st_pipeline_configure(st_ctx* ctx, const st_pipeline_config* pc);

/* Queue one batch given in HOST memory (hits->x, zone, ev_off etc. and
 * velo->state, ev_off are host pointers; z/dxdy ignored).  The hits and VELO
 * states are copied by DMA into device-resident input rings before the call
 * returns, so the caller may reuse its buffers; if the rings are full the
 * call waits (up to 60 s, then ST_TIMEOUT) until earlier batches have run.
 * Waiting batches that follow each other in the rings are packed into one
 * launch on a free slot; slots run on their own streams and overlap on the
 * device.  *ticket identifies the batch.  ST_OVERFLOW if the batch can never
 * fit a slot; ST_ESTATE after st_destroy has begun.  Results stay in a device
 * output ring until polled: poll every ticket.  A launch runs seeding_run and
 * matching_run with the context's configuration (so also the final
 * selection when final_sel is set); UT hits are not part of the pipeline
 * (ut_run on device buffers). */
int pipeline_submit(st_ctx* ctx, const st_hits* host_hits, const st_velo* host_velo,
                    uint64_t* ticket);

/* Timing of a finished request (host steady clock, nanoseconds): submitted,
 * launched on the device, results complete on the device, results copied
 * into the caller's buffers by pipeline_poll. */
typedef struct {
    int64_t t_submit_ns, t_launch_ns, t_done_ns, t_returned_ns;
    int32_t n_events, n_seeds;
} st_request_info;

/* Wait up to timeout_us (0 = do not wait, < 0 = forever) for the batch of
 * `ticket`.  On ST_OK its seeds and Long tracks are copied by DMA from the
 * device output ring into the HOST buffers host_seeds (cap, ev_off, hits,
 * params, state, n_hits, status) and host_long (velo_idx, chi2, n_long,
 * ghost_prob; each may be NULL, as may host_long), info (may be NULL) is
 * filled, and the ticket is released.
 * ST_PENDING (timeout_us == 0) or ST_TIMEOUT if not ready; ST_OVERFLOW if
 * host_seeds->cap is too small (ticket kept); ST_EINVAL for an unknown
 * ticket. */
int pipeline_poll(st_ctx* ctx, uint64_t ticket, st_seeds* host_seeds, st_long* host_long,
                  int64_t timeout_us, st_request_info* info);

#ifdef __cplusplus
}
#endif
#endif
