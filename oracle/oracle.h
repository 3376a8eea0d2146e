/*
 * oracle.h -- FP64 CPU reference of the SciFi Seeding + VELO-SciFi Matching
 * hot path (test infrastructure only).
 *
 * This library is the slow, obviously-correct statement of what the method
 * computes, used by the test-suite, the smoke check and the CPU baseline of the
 * benchmark.  The product path never links, loads or calls it.  It shares no
 * code, header or constant table with the CUDA library.
 *
 * Every function works on ONE event, single-threaded, in double precision, on
 * host memory.  Hit indices are event-local (0 .. n_hits-1, the caller's order).
 * Sections and equations cited are those of the paper "Seeding and Matching
 * algorithms for the first GPU-based High Level Trigger of the LHCb experiment".
 */
#ifndef ST_ORACLE_H
#define ST_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NLAYER 12

/* Method parameters.  Geometry: 12 SciFi layers, ordered x,u,v,x per station
 * (Section 1); zone = 2*layer + half (half 1 = y >= 0). */
typedef struct {
    double z[OR_NLAYER];          /* layer z (mm) */
    double dxdy[OR_NLAYER];       /* stereo slope tan(alpha); 0 for x-layers */
    double z_ref;                 /* track-model reference z (Eq. trackequation) */
    double d_ratio;               /* fixed cubic-correction coefficient (1/mm) */
    /* XZ seeding, Section 3.3 */
    double invp_a, invp_b;        /* Eq. invp: 1/p = a|x0| + b x0^2, per MeV */
    double p_min;                 /* MeV/c */
    double alpha0, alpha1;        /* Eq. alphacorr (MeV/c) */
    double dx3_scale;             /* multiplies Delta x3^max (1 = paper) */
    int32_t n_iter;               /* 2 in HLT1 (up to 3) */
    int32_t iter_layers[3][3];    /* (T1, T2, T3) initial x-layers per iteration */
    double kappa_c;               /* -s*c_x = kappa_c / p (mm^-1 MeV) */
    double m_lo, m_hi;            /* third-hit band multipliers */
    double c_nsigma;              /* band half-width in units of the c_x resolution */
    double sigma_x;               /* x-hit resolution (mm) */
    double ext_tol;               /* x-layer extension tolerance (mm), 1.0 */
    double chi2x_max;             /* chi2/ndf cut of the XZ fit */
    double score_w_chi2;          /* 1000 in Eq. seed_clone_score */
    double score_w5;              /* 10   in Eq. seed_clone_score */
    /* UV seeding, Section 3.4 */
    int32_t uv_init[2];           /* initial stereo layer of pass A and pass B */
    int32_t n_uv_min;             /* minimum stereo hits of a kept seed (>= 2) */
    int32_t pad1;
    double uv_tol;                /* stereo tolerance (mm), 2.0 */
    double uv_y_overlap;          /* y window reaches this far into the other half */
    double uv_y_max;              /* |y| acceptance of the first-layer window */
    double sigma_y;               /* y resolution used in chi2_y */
    double z_state;               /* z of the seed state handed to matching */
    /* Matching, Section 4 */
    double z_velo;                /* z of the VELO states */
    double z_match_y;             /* 10 m */
    double zmx[5];                /* A_x..E_x of Eq. z_match */
    double presel[4];             /* |dx| |dy| |dtx| |dty| preselection cuts */
    double presel_scale;          /* multiplies the four preselection cuts */
    double tol_scale;             /* multiplies tol_x, tol_y, tol_tx, tol_ty */
    double tolx[3];               /* tol_x = tolx0 * (tolx1^2 + tolx2^2 dtx^2) */
    double toly[3];               /* tol_y = toly0 * (toly1^2 + toly2^2 rho) */
    double tol_tx, tol_ty;
    double chi2_match_max;        /* 2 */
    int32_t velo_unique;          /* 1: a VELO segment serves at most one seed */
    int32_t pad2;
    /* UV seeding, Hough-cluster variant (Section 3.4, second approach) */
    int32_t uv_mode;              /* 0: iterative over an initial layer, 1: Hough clusters */
    int32_t hough_bins;           /* coarse t_y bins (2..64) */
    int32_t hough_fine;           /* t_y hypotheses per selected cluster (1..8) */
    int32_t hough_clusters;       /* clusters kept per seed, best first (1..8) */
    double hough_ty_max;          /* coarse range [-hough_ty_in, hough_ty_max] for half 1, */
    double hough_ty_in;           /* mirrored for half 0 */
    /* Matching final selection, Section 4.4 */
    int32_t final_sel;            /* 1: ghost network, ghost_prob < ghost_max, clone removal */
    int32_t pad3;
    double ghost_max;             /* 0.8 */
    double clone_margin;          /* 0.05 */
    /* UT hits of a Long track, Section 4.3 */
    double ut_z[4];               /* UT layers UTaX, UTaU, UTbV, UTbX */
    double ut_dxdy[4];            /* their stereo slopes (x, u, v, x) */
    double ut_gamma[2];           /* Eq. gamma_parametrisation: A_gamma, B_gamma (per MeV) */
    double ut_kick;               /* q/p of a pair = (tx_S - tx_V) / ut_kick (MeV) */
    double ut_loose[16];          /* per layer A_L, B_L (mm GeV), x_min, x_max; zeros: no loose search */
    double ut_tight[16];          /* per layer A_T, B_T, x_min, x_max; zeros: no tight search */
    int32_t ut_min_hits;          /* keep Long tracks with at least this many UT hits (0: keep all) */
    /* HLT2-style iterations (Section 3.1): 0 = independent iterations with one
     * clone kill at the end (HLT1); 1 = iterations in sequence, each with its
     * own clone kill and UV step, hits of its seeds removed before the next */
    int32_t iter_mode;
    double p_min_iter[3];         /* per-iteration p_min (MeV/c); 0: use p_min */
} or_config;

typedef struct {
    int32_t hits[OR_NLAYER];      /* event-local hit index per layer, -1 = none */
    int32_t half, nx, nuv, cand_id;
    int32_t pass, pad;            /* iteration that found it in the HLT2-style mode (else 0) */
    double a, b, c, chi2x;        /* x-z parameters (Eq. trackequation) and chi2 */
    double y0, ty, chi2y;         /* y(z) = y0 + ty z */
    double x_s, y_s, tx_s, ty_s;  /* state at z_state */
} or_seed;

typedef struct {
    int32_t hits[6];              /* per x-layer slot (layers 0,3,4,7,8,11) */
    int32_t half, iter, nx, keep;
    int32_t h1, h2, h3, id;
    double a, b, c, chi2, score;
} or_cand;

/* Decisions that came within `tau` (relative) of flipping. */
enum {
    OR_L_PAIR_WIN = 1, OR_L_TRIP_WIN = 2, OR_L_EXT_TOL = 3, OR_L_EXT_TIE = 4,
    OR_L_CHI2X = 5, OR_L_CLONE = 6, OR_L_UV_WIN = 7, OR_L_UV_TOL = 8,
    OR_L_UV_TIE = 9, OR_L_UV_SEL = 10, OR_L_M_PRESEL = 11, OR_L_M_CHI2 = 12,
    OR_L_M_TIE = 13, OR_L_HOUGH_BIN = 14, OR_L_GHOST = 15, OR_L_M_CLONE = 16, OR_L_UT_WIN = 17,
    OR_L_UT_TIE = 18
};
typedef struct {
    int32_t kind, half;
    int32_t hits[12];             /* hits involved (-1 padded); matching: {seed, velo, velo2} */
    double margin;                /* |q - t| / scale */
} or_ledger;

typedef struct {
    int64_t pairs, triplets, ext_ok, cands, kept, uv_init, uv_cands, seeds;
    int64_t match_pairs, match_presel, matched;
} or_counters;

void or_config_default(or_config* c);

/* Closed-form window constants (exposed for the pins). */
double or_x0max(const or_config* c);
double or_dx3max(const or_config* c, int32_t iter);
double or_alpha_corr(const or_config* c, int32_t iter);
double or_k3(const or_config* c, int32_t iter);
double or_invp(const or_config* c, double x0);

/* Seeding of one event.  x[i], zone[i] for i < n_hits.  Returns 0, or -1 on
 * invalid input/config.  Each optional output (NULL allowed) reports its full
 * count in *n_* and stores at most *_cap records.  trips: 5 int32 per triplet
 * (half, iter, h1, h2, h3). */
int32_t or_seeding_event(const or_config* c, int32_t n_hits, const double* x,
                         const int32_t* zone,
                         or_seed* seeds, int32_t seeds_cap, int32_t* n_seeds,
                         or_cand* cands, int32_t cands_cap, int32_t* n_cands,
                         int32_t* trips, int32_t trips_cap, int32_t* n_trips,
                         or_ledger* ledger, int32_t ledger_cap, int32_t* n_ledger,
                         double tau, or_counters* counters);

/* Matching of one event.  velo: n_velo x (x, y, tx, ty) at z_velo; seed_state:
 * n_seeds x (x, y, tx, ty) at z_state.  Outputs per seed: velo_idx (-1 = no
 * match) and chi2 (chi2_match of the chosen pair, 0 if none). */
int32_t or_matching_event(const or_config* c, int32_t n_velo, const double* velo,
                          int32_t n_seeds, const double* seed_state,
                          int32_t* velo_idx, double* chi2,
                          or_ledger* ledger, int32_t ledger_cap, int32_t* n_ledger,
                          double tau, or_counters* counters);

/* Ghost network of Section 4.4: 8 inputs, one hidden layer of 32 ReLU nodes,
 * a sigmoid output.  Weight layout (float32, OR_GHOST_NN_SIZE values):
 * mean[8], inv_scale[8] (inputs are standardised as (f - mean) * inv_scale),
 * W1[32][8], b1[32], w2[32], b2.  Inputs, in the paper's order: z_match_x,
 * dx, dy, dtx, dty, chi2_match, eta of the VELO segment, SciFi hits. */
#define OR_GHOST_NN_SIZE 337
double or_ghost_nn(const float* nn, const double f[8]);

/* Final selection of the matched pairs of one event (Section 4.4), applied to
 * the output of or_matching_event: for every seed with a match the eight
 * inputs are formed from its VELO segment and seed state, the ghost
 * probability is evaluated (ghost_prob[s]; 1 for seeds without a match),
 * pairs with ghost_prob >= ghost_max are dropped, and a pair is dropped as a
 * clone when another kept pair shares its VELO segment (or its seed) with a
 * ghost probability lower by at least clone_margin.  velo_idx is updated in
 * place (-1 = dropped).  seed_nhits: SciFi hits per seed. */
int32_t or_final_selection(const or_config* c, int32_t n_velo, const double* velo, int32_t n_seeds,
                           const double* seed_state, const int32_t* seed_nhits, const float* nn,
                           int32_t* velo_idx, const double* chi2, double* ghost_prob,
                           or_ledger* ledger, int32_t ledger_cap, int32_t* n_ledger, double tau);

/* UT hits of one event's Long tracks (Section 4.3).  For every seed with
 * velo_idx[s] >= 0 the VELO segment is extrapolated with Eq.
 * velo_ut_extrapolation, gamma_x from Eq. gamma_parametrisation at the pair's
 * q/p, through the four UT layers in order.  Until a hit is found a layer is
 * searched in its loose window, and the closest hit in it is attached and
 * refits gamma_x through that hit; later layers are searched in their tight
 * windows (closest hit attached).  Windows: min(max(A + B/p, x_min), x_max),
 * p in GeV/c.  ut_x / ut_layer: the event's UT hits (measured x at y = 0,
 * layer 0..3).  Outputs per seed: ut_hits[4] (event-local UT index, -1),
 * n_ut, gamma (the final gamma_x); velo_idx is set to -1 where n_ut <
 * ut_min_hits. */
int32_t or_ut_search(const or_config* c, int32_t n_velo, const double* velo, int32_t n_seeds,
                     const double* seed_state, int32_t* velo_idx, int32_t n_ut, const double* ut_x,
                     const int32_t* ut_layer, int32_t* ut_hits, int32_t* n_ut_out, double* gamma,
                     or_ledger* ledger, int32_t ledger_cap, int32_t* n_ledger, double tau);

#ifdef __cplusplus
}
#endif
#endif
