/*
 * oracle.c -- FP64 reference of SciFi Seeding + VELO-SciFi Matching.
 *
 * TEST INFRASTRUCTURE ONLY: the product path never loads this library.
 *
 * It follows the paper step by step (Section 3: XZ seeding with two- and
 * three-hit windows, x-layer extension, x-z least-squares fit, O(n) clone
 * killing, iterative UV seeding; Section 4: kink-point extrapolation,
 * preselection, chi2_match and best-pair choice).  Where the paper leaves a
 * detail open, the reading used is stated at that step.  Searches are plain
 * scans over every hit of a layer, in ascending (x, index) order; fits are
 * normal equations solved by Gaussian elimination with partial pivoting.
 *
 * Alongside the result it can write a ledger: every decision whose margin to
 * flipping, relative to the size of the numbers it is made from, is at most
 * `tau`.  Tests use it to trace differences to near-threshold decisions.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NZONE 24

static const int X_LAYERS[6] = {0, 3, 4, 7, 8, 11};
static const int UV_LAYERS[6] = {1, 2, 5, 6, 9, 10};

static int xslot_of_layer(int L) {
    for (int k = 0; k < 6; ++k)
        if (X_LAYERS[k] == L) return k;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* configuration                                                            */
/* ------------------------------------------------------------------------ */

void or_config_default(or_config* c) {
    memset(c, 0, sizeof(*c));
    static const double zl[OR_NLAYER] = {7826, 7896, 7966, 8036, 8508, 8578,
                                         8648, 8718, 9193, 9263, 9333, 9403};
    const double t5 = tan(5.0 * M_PI / 180.0); /* stereo angle +-5 deg, Section 1 */
    static const int sgn[OR_NLAYER] = {0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, 0};
    for (int l = 0; l < OR_NLAYER; ++l) {
        c->z[l] = zl[l];
        c->dxdy[l] = sgn[l] * t5;
    }
    c->z_ref = 8520.0;       /* benchmark generator's reference point */
    c->d_ratio = -2.6e-4;    /* "fixed from simulation"; value of the generator */
    c->invp_a = 1.6322e-7;   /* Eq. invp, per MeV (see the unit pin) */
    c->invp_b = -5.0217e-12;
    c->p_min = 3000.0;       /* p_min = 3 GeV/c, both iterations */
    c->alpha0 = 2.180e6;     /* Eq. alphacorr */
    c->alpha1 = -1073.0;
    c->dx3_scale = 1.0;
    c->n_iter = 2;
    c->iter_layers[0][0] = 0; c->iter_layers[0][1] = 4; c->iter_layers[0][2] = 11;
    c->iter_layers[1][0] = 3; c->iter_layers[1][1] = 7; c->iter_layers[1][2] = 8;
    /* a third iteration (HLT2-style use only): T1 and T3 from the first,
     * the other T2 x-layer */
    c->iter_layers[2][0] = 0; c->iter_layers[2][1] = 7; c->iter_layers[2][2] = 11;
    c->kappa_c = 1.0e-2;
    c->m_lo = 0.5;
    c->m_hi = 1.5;
    c->c_nsigma = 5.0;
    c->sigma_x = 0.07;
    c->ext_tol = 1.0;        /* Section 3.2: hits within 1 mm */
    c->chi2x_max = 10.0;
    c->score_w_chi2 = 1000.0;/* Eq. seed_clone_score */
    c->score_w5 = 10.0;
    c->uv_init[0] = 1;       /* pass A: u layer of T1 */
    c->uv_init[1] = 2;       /* pass B: v layer of T1 */
    c->n_uv_min = 4;
    c->uv_tol = 2.0;         /* Section 3.4: 2 mm */
    c->uv_y_overlap = 50.0;
    c->uv_y_max = 2500.0;
    c->sigma_y = 0.07 / t5;
    c->z_state = 7826.0;
    c->z_velo = 770.0;
    c->z_match_y = 10000.0;  /* Section 4: z_match_y = 10 m */
    c->zmx[0] = 5287.6;      /* Table mag_params */
    c->zmx[1] = -7.98878;
    c->zmx[2] = 317.683;
    c->zmx[3] = 0.0119379;
    c->zmx[4] = -1418.42;
    c->presel[0] = 20.0;     /* Section 4.2 preselection */
    c->presel[1] = 150.0;
    c->presel[2] = 1.5;
    c->presel[3] = 0.02;
    c->presel_scale = 1.0;
    c->tol_scale = 1.0;
    c->tolx[0] = 0.8; c->tolx[1] = 10.12; c->tolx[2] = 101.0;
    c->toly[0] = 0.2; c->toly[1] = 1.59;  c->toly[2] = 212.1;
    c->tol_tx = 0.5;
    c->tol_ty = 1.0 / 937.5;
    c->chi2_match_max = 2.0;
    c->velo_unique = 0;
    c->uv_mode = 0;          /* the paper's default UV approach */
    c->hough_bins = 64;      /* Hough variant: not given in the paper (readings) */
    c->hough_fine = 4;
    c->hough_clusters = 8;   /* "up to eight of the best bins" */
    c->hough_ty_max = 0.33;
    c->hough_ty_in = 0.01;
    c->final_sel = 0;
    c->ghost_max = 0.8;      /* Section 4.4 */
    c->clone_margin = 0.05;
    /* UT (Section 4.3): layer z not given in the paper (reading); x-u-v-x */
    static const double uz[4] = {2327.5, 2372.5, 2597.5, 2642.5};
    static const int us[4] = {0, 1, -1, 0};
    for (int l = 0; l < 4; ++l) {
        c->ut_z[l] = uz[l];
        c->ut_dxdy[l] = us[l] * t5;
    }
    c->ut_gamma[0] = 7.707063e-11;  /* Table mag_params */
    c->ut_gamma[1] = -7.817364e-3;
    c->ut_kick = 1200.0;
    /* Table ut_search_window_values: loose windows of UTaX, UTaU, UTbV */
    static const double lw[16] = {0.8333, 3.3333, 1.2, 8.5, 0.8333, 3.3333, 1.2, 8.5,
                                  1.3333, 3.3333, 1.5, 9.5, 0, 0, 0, 0};
    /* tight windows of UTaU, UTbV, UTbX */
    static const double tw[16] = {0, 0, 0, 0, 0.2, 0.6, 0.5, 2.0, 0.4, 1.2, 1.0, 4.0, 0.4, 1.2, 1.0, 4.0};
    memcpy(c->ut_loose, lw, sizeof(lw));
    memcpy(c->ut_tight, tw, sizeof(tw));
    c->ut_min_hits = 3;      /* "more than two associated UT hits" */
    c->iter_mode = 0;
    for (int it = 0; it < 3; ++it) c->p_min_iter[it] = 0.0;
}

static int config_ok(const or_config* c) {
    if (c->n_iter < 1 || c->n_iter > 3 || c->iter_mode < 0 || c->iter_mode > 1) return 0;
    for (int it = 0; it < 3; ++it)
        if (c->p_min_iter[it] < 0) return 0;
    for (int it = 0; it < c->n_iter; ++it)
        for (int k = 0; k < 3; ++k)
            if (xslot_of_layer(c->iter_layers[it][k]) < 0) return 0;
    for (int p = 0; p < 2; ++p) {
        int ok = 0;
        for (int k = 0; k < 6; ++k) ok |= (UV_LAYERS[k] == c->uv_init[p]);
        if (!ok) return 0;
    }
    if (c->n_uv_min < 2 || c->n_uv_min > 6) return 0;
    if (!(c->p_min > 0) || !(c->sigma_x > 0) || !(c->sigma_y > 0)) return 0;
    if (c->uv_mode < 0 || c->uv_mode > 1) return 0;
    if (c->hough_bins < 2 || c->hough_bins > 64 || c->hough_fine < 1 || c->hough_fine > 8 ||
        c->hough_clusters < 1 || c->hough_clusters > 8 || !(c->hough_ty_max + c->hough_ty_in > 0))
        return 0;
    if (c->final_sel < 0 || c->final_sel > 1 || (c->final_sel && c->velo_unique) || !(c->ghost_max > 0) ||
        !(c->clone_margin > 0))
        return 0;
    if (c->ut_min_hits < 0 || c->ut_min_hits > 4 || !(c->ut_kick > 0)) return 0;
    for (int l = 0; l < 4; ++l)
        if (!(fabs(c->ut_z[l] - c->z_velo) > 0)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* track model, Eq. (trackequation): x(z) = a + b zb + c zb^2 (1 + d zb)    */
/* ------------------------------------------------------------------------ */

/* p_min of an iteration (Section 3.2; HLT2-style runs may set one per iteration) */
static double pmin_of(const or_config* c, int it) {
    return it >= 0 && it < 3 && c->p_min_iter[it] > 0 ? c->p_min_iter[it] : c->p_min;
}

static double fcub(const or_config* c, double z) {
    double zb = z - c->z_ref;
    return zb * zb * (1.0 + c->d_ratio * zb);
}

static double xmodel(const or_config* c, const double th[3], double z) {
    return th[0] + th[1] * (z - c->z_ref) + th[2] * fcub(c, z);
}

/* Largest magnitude among the terms that form xmodel: the scale against which
 * a margin on a predicted position is measured. */
static double xscale(const or_config* c, const double th[3], double z) {
    double s = fabs(th[0]);
    double t1 = fabs(th[1] * (z - c->z_ref)), t2 = fabs(th[2] * fcub(c, z));
    if (t1 > s) s = t1;
    if (t2 > s) s = t2;
    return s;
}

/* Solve the n x n system A y = r (n <= 3) by Gaussian elimination with
 * partial pivoting. */
static int gauss_solve(int n, double A[3][3], double r[3], double y[3]) {
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (fabs(A[i][col]) > fabs(A[piv][col])) piv = i;
        if (A[piv][col] == 0.0) return 0;
        if (piv != col) {
            for (int j = 0; j < n; ++j) {
                double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t;
            }
            double t = r[col]; r[col] = r[piv]; r[piv] = t;
        }
        for (int i = col + 1; i < n; ++i) {
            double f = A[i][col] / A[col][col];
            for (int j = col; j < n; ++j) A[i][j] -= f * A[col][j];
            r[i] -= f * r[col];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = r[i];
        for (int j = i + 1; j < n; ++j) s -= A[i][j] * y[j];
        y[i] = s / A[i][i];
    }
    return 1;
}

/* Least-squares fit of (a, b, c) of the track model, d fixed, to m points
 * (m >= 3; m = 3 is the exact interpolation).  The basis is evaluated with zb
 * in metres and f in m^3 so that the normal matrix is well scaled; the
 * solution is scaled back.  Returns the unweighted sum of squared residuals. */
static double fit_xz(const or_config* c, int m, const double* z, const double* x,
                     double th[3]) {
    static const double sc[3] = {1.0, 1e-3, 1e-6};
    double A[3][3] = {{0}}, r[3] = {0}, y[3] = {0};
    for (int i = 0; i < m; ++i) {
        double phi[3] = {sc[0], (z[i] - c->z_ref) * sc[1], fcub(c, z[i]) * sc[2]};
        for (int j = 0; j < 3; ++j) {
            r[j] += phi[j] * x[i];
            for (int k = 0; k < 3; ++k) A[j][k] += phi[j] * phi[k];
        }
    }
    if (!gauss_solve(3, A, r, y)) {
        th[0] = th[1] = th[2] = 0.0;
        return INFINITY;
    }
    for (int j = 0; j < 3; ++j) th[j] = y[j] * sc[j];
    double s2 = 0.0;
    for (int i = 0; i < m; ++i) {
        double res = x[i] - xmodel(c, th, z[i]);
        s2 += res * res;
    }
    return s2;
}

/* Straight-line least squares y = y0 + ty z over m >= 2 points; returns the
 * sum of squared residuals. */
static double fit_line(int m, const double* z, const double* y, double* y0, double* ty) {
    double A[3][3] = {{0}}, r[3] = {0}, s[3] = {0};
    double zm = 0.0;
    for (int i = 0; i < m; ++i) zm += z[i];
    zm /= m;
    for (int i = 0; i < m; ++i) {
        double phi[2] = {1.0, z[i] - zm};
        for (int j = 0; j < 2; ++j) {
            r[j] += phi[j] * y[i];
            for (int k = 0; k < 2; ++k) A[j][k] += phi[j] * phi[k];
        }
    }
    if (!gauss_solve(2, A, r, s)) {
        *y0 = 0; *ty = 0;
        return INFINITY;
    }
    *ty = s[1];
    *y0 = s[0] - s[1] * zm;
    double s2 = 0.0;
    for (int i = 0; i < m; ++i) {
        double res = y[i] - (*y0 + *ty * z[i]);
        s2 += res * res;
    }
    return s2;
}

/* ------------------------------------------------------------------------ */
/* closed-form window constants, Section 3.3                                */
/* ------------------------------------------------------------------------ */

double or_invp(const or_config* c, double x0) {
    return c->invp_a * fabs(x0) + c->invp_b * x0 * x0; /* Eq. invp */
}

/* x0 at which the momentum estimate equals p_min: b x0^2 + a x0 = 1/p_min,
 * smaller root. */
double or_x0max(const or_config* c) {
    double a = c->invp_a, b = c->invp_b;
    return (-a + sqrt(a * a + 4.0 * b / c->p_min)) / (2.0 * b);
}

/* Eq. tolHp: Delta x3^max = (z3 - z1)/z1 * x0max. */
double or_dx3max(const or_config* c, int32_t it) {
    double z1 = c->z[c->iter_layers[it][0]], z3 = c->z[c->iter_layers[it][2]];
    return c->dx3_scale * (z3 - z1) / (2.0 * z1 * c->invp_b) *
           (-c->invp_a + sqrt(c->invp_a * c->invp_a + 4.0 * c->invp_b / pmin_of(c, it)));
}

/* Eq. alphacorr with k = z1 / (z3 - z1); a z offset (mm) added to z3. */
double or_alpha_corr(const or_config* c, int32_t it) {
    double z1 = c->z[c->iter_layers[it][0]], z3 = c->z[c->iter_layers[it][2]];
    double k = z1 / (z3 - z1);
    return c->alpha0 / (k * (pmin_of(c, it) - c->alpha1));
}

/* k3 of Section 3.3.3: deviation of the track model at z2 from the chord
 * through (z1, z3), per unit c_x, d_ratio included.  (The printed closed
 * form is garbled; this is the quantity the text defines.) */
double or_k3(const or_config* c, int32_t it) {
    double z1 = c->z[c->iter_layers[it][0]], z2 = c->z[c->iter_layers[it][1]],
           z3 = c->z[c->iter_layers[it][2]];
    return fcub(c, z2) - fcub(c, z1) - (z2 - z1) / (z3 - z1) * (fcub(c, z3) - fcub(c, z1));
}

/* ------------------------------------------------------------------------ */
/* event context                                                            */
/* ------------------------------------------------------------------------ */

typedef struct { double x; int32_t i; } xi_t;

static int cmp_xi(const void* pa, const void* pb) {
    const xi_t* a = (const xi_t*)pa;
    const xi_t* b = (const xi_t*)pb;
    if (a->x < b->x) return -1;
    if (a->x > b->x) return 1;
    return (a->i > b->i) - (a->i < b->i);
}

typedef struct {
    const or_config* c;
    const double* x;
    xi_t* zl[NZONE];
    int zn[NZONE];
    or_ledger* led;
    int32_t led_cap;
    int32_t n_led;
    double tau;
    or_counters cnt;
    const unsigned char* used; /* hits taken by earlier iterations (HLT2-style mode), or NULL */
} ev_t;

static void ledger_add(ev_t* E, int kind, int half, double margin, const int32_t* hits, int nh) {
    if (!(margin <= E->tau)) return;
    if (E->led && E->n_led < E->led_cap) {
        or_ledger* L = &E->led[E->n_led];
        L->kind = kind;
        L->half = half;
        L->margin = margin;
        for (int k = 0; k < 12; ++k) L->hits[k] = k < nh ? hits[k] : -1;
    }
    E->n_led++;
}

static double dmax2(double a, double b) { return a > b ? a : b; }

/* candidate of the x-z search (one per triplet that survives) */
typedef struct {
    int32_t hits[6];
    int32_t iter, nx, h1, h2, h3, id, keep;
    double th[3];
    double chi2, score;
} cand_t;

typedef struct {
    cand_t* v;
    int n, cap;
} cvec_t;

static cand_t* cvec_push(cvec_t* cv) {
    if (cv->n == cv->cap) {
        int nc = cv->cap ? 2 * cv->cap : 64;
        cand_t* nv = (cand_t*)realloc(cv->v, (size_t)nc * sizeof(cand_t));
        if (!nv) return NULL;
        cv->v = nv;
        cv->cap = nc;
    }
    return &cv->v[cv->n++];
}

/* Closest hit of zone `zi` to position xp within tol (inclusive); ties go to
 * the smaller x (the first one met in ascending order).  Records near-edge and
 * near-tie decisions.  `scale` is the magnitude of the terms forming xp. */
static int closest_hit(ev_t* E, int zi, double xp, double tol, double scale, int kind_tol,
                       int kind_tie, int half, const int32_t* ctx_hits, int nctx) {
    int best = -1;
    double bestd = INFINITY, second = INFINITY;
    int second_i = -1;
    int32_t hh[12];
    for (int k = 0; k < nctx && k < 10; ++k) hh[k] = ctx_hits[k];
    int nh = nctx < 10 ? nctx : 10;
    for (int k = 0; k < E->zn[zi]; ++k) {
        if (E->used && E->used[E->zl[zi][k].i]) continue;
        double xh = E->zl[zi][k].x;
        double d = fabs(xh - xp);
        double S = dmax2(scale, fabs(xh));
        hh[nh] = E->zl[zi][k].i;
        ledger_add(E, kind_tol, half, fabs(d - tol) / S, hh, nh + 1);
        if (d <= tol) {
            if (d < bestd) {
                second = bestd; second_i = best;
                bestd = d; best = E->zl[zi][k].i;
            } else if (d < second) {
                second = d; second_i = E->zl[zi][k].i;
            }
        }
    }
    if (best >= 0 && second_i >= 0) {
        hh[nh] = best;
        hh[nh + 1] = second_i;
        ledger_add(E, kind_tie, half, fabs(second - bestd) / dmax2(scale, 1.0), hh, nh + 2);
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* XZ seeding, Section 3.2-3.3                                              */
/* ------------------------------------------------------------------------ */

static void xz_search(ev_t* E, int half, cvec_t* cv, int32_t* trips, int32_t trips_cap,
                      int32_t* n_trips, int it0, int it1) {
    const or_config* c = E->c;
    for (int it = it0; it < it1; ++it) {
        const int L1 = c->iter_layers[it][0], L2 = c->iter_layers[it][1], L3 = c->iter_layers[it][2];
        const double z1 = c->z[L1], z2 = c->z[L2], z3 = c->z[L3];
        const double alpha = or_alpha_corr(c, it);
        const double dx3 = or_dx3max(c, it);
        const double k3 = or_k3(c, it);
        const double w1 = (z3 - z2) / (z3 - z1), w3 = (z2 - z1) / (z3 - z1);
        /* third-hit band half-width: c_nsigma resolutions of dx2, in c_x units */
        const double c0 = c->c_nsigma * c->sigma_x * sqrt(1.0 + w1 * w1 + w3 * w3) / fabs(k3);
        const int zi1 = 2 * L1 + half, zi2 = 2 * L2 + half, zi3 = 2 * L3 + half;
        /* the x-layers not used by the triplet, in slot order */
        int ext[3], ne = 0;
        for (int k = 0; k < 6; ++k) {
            int L = X_LAYERS[k];
            if (L != L1 && L != L2 && L != L3) ext[ne++] = L;
        }
        for (int k1 = 0; k1 < E->zn[zi1]; ++k1) {
            const double x1 = E->zl[zi1][k1].x;
            const int32_t h1 = E->zl[zi1][k1].i;
            if (E->used && E->used[h1]) continue;
            /* two-hit window (Eqs. tolHp, alphacorr and the window limits) */
            const double xc = (z3 + alpha) / z1 * x1;
            const double lo = xc - dx3, hi = xc + dx3;
            const double S3 = fabs(xc) + dx3;
            for (int k3i = 0; k3i < E->zn[zi3]; ++k3i) {
                const double x3 = E->zl[zi3][k3i].x;
                const int32_t h3 = E->zl[zi3][k3i].i;
                if (E->used && E->used[h3]) continue;
                {
                    int32_t hh[2] = {h1, h3};
                    double m = fmin(fabs(x3 - lo), fabs(x3 - hi)) / dmax2(S3, fabs(x3));
                    ledger_add(E, OR_L_PAIR_WIN, half, m, hh, 2);
                }
                if (x3 < lo || x3 > hi) continue;
                E->cnt.pairs++;
                /* back-propagated x0 and momentum estimate (Eqs. x0, t13, invp) */
                const double t13 = (x3 - x1) / (z3 - z1);
                const double x0 = x1 - z1 * t13;
                const double invp = or_invp(c, x0);
                if (!(invp > 0.0)) continue;
                const double s = x0 > 0.0 ? 1.0 : -1.0;
                /* band of -s*c_x around kappa_c/p, mapped to x2 through
                 * dx2 = k3 * c_x (Section 3.3.3) */
                const double u_lo = c->m_lo * c->kappa_c * invp - c0;
                const double u_hi = c->m_hi * c->kappa_c * invp + c0;
                const double base = x1 + (z2 - z1) * t13;
                const double xa = base + k3 * (-s * u_lo);
                const double xb = base + k3 * (-s * u_hi);
                const double lo2 = fmin(xa, xb), hi2 = fmax(xa, xb);
                const double S2 = fabs(base) + fabs(k3) * dmax2(fabs(u_lo), fabs(u_hi));
                for (int k2 = 0; k2 < E->zn[zi2]; ++k2) {
                    const double x2 = E->zl[zi2][k2].x;
                    const int32_t h2 = E->zl[zi2][k2].i;
                    if (E->used && E->used[h2]) continue;
                    {
                        int32_t hh[3] = {h1, h3, h2};
                        double m = fmin(fabs(x2 - lo2), fabs(x2 - hi2)) / dmax2(S2, fabs(x2));
                        ledger_add(E, OR_L_TRIP_WIN, half, m, hh, 3);
                    }
                    if (x2 < lo2 || x2 > hi2) continue;
                    if (trips && *n_trips < trips_cap) {
                        int32_t* t = &trips[5 * (*n_trips)];
                        t[0] = half; t[1] = it; t[2] = h1; t[3] = h2; t[4] = h3;
                    }
                    (*n_trips)++;
                    E->cnt.triplets++;
                    /* exact model through the three hits */
                    double zz[3] = {z1, z2, z3}, xx[3] = {x1, x2, x3}, th3[3];
                    fit_xz(c, 3, zz, xx, th3);
                    int32_t hits[6] = {-1, -1, -1, -1, -1, -1};
                    hits[xslot_of_layer(L1)] = h1;
                    hits[xslot_of_layer(L2)] = h2;
                    hits[xslot_of_layer(L3)] = h3;
                    /* extension to the remaining x-layers, 1 mm (Section 3.2) */
                    int32_t ctx[3] = {h1, h2, h3};
                    for (int e = 0; e < ne; ++e) {
                        const int L = ext[e];
                        const double xp = xmodel(c, th3, c->z[L]);
                        const double sc = xscale(c, th3, c->z[L]);
                        hits[xslot_of_layer(L)] = closest_hit(E, 2 * L + half, xp, c->ext_tol, sc,
                                                              OR_L_EXT_TOL, OR_L_EXT_TIE, half, ctx, 3);
                    }
                    int nx = 0;
                    double fz[6], fx[6];
                    for (int k = 0; k < 6; ++k)
                        if (hits[k] >= 0) {
                            fz[nx] = c->z[X_LAYERS[k]];
                            fx[nx] = E->x[hits[k]];
                            nx++;
                        }
                    if (nx < 5) continue;
                    E->cnt.ext_ok++;
                    /* least-squares x-z fit, d_ratio fixed; chi2 filter */
                    double th[3];
                    double chi2 = fit_xz(c, nx, fz, fx, th) / (c->sigma_x * c->sigma_x);
                    double q = chi2 / (nx - 3);
                    {
                        int32_t hh[6];
                        int m = 0;
                        for (int k = 0; k < 6; ++k)
                            if (hits[k] >= 0) hh[m++] = hits[k];
                        ledger_add(E, OR_L_CHI2X, half, fabs(q - c->chi2x_max) / c->chi2x_max, hh, m);
                    }
                    if (q > c->chi2x_max) continue;
                    cand_t* cd = cvec_push(cv);
                    if (!cd) return;
                    memcpy(cd->hits, hits, sizeof(hits));
                    cd->iter = it;
                    cd->nx = nx;
                    cd->h1 = h1; cd->h2 = h2; cd->h3 = h3;
                    cd->id = cv->n - 1;
                    cd->keep = 0;
                    memcpy(cd->th, th, sizeof(th));
                    cd->chi2 = chi2;
                    /* Eq. seed_clone_score, with |c_x| (reading: the score is
                     * non-negative and prefers high momentum) */
                    double sc = c->score_w_chi2 * chi2 + fabs(th[2]);
                    cd->score = nx == 6 ? sc : c->score_w5 * sc;
                    E->cnt.cands++;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* O(n) clone killing, Section 3.3.4                                        */
/* ------------------------------------------------------------------------ */

static int same_hits(const cand_t* a, const cand_t* b) {
    return memcmp(a->hits, b->hits, sizeof(a->hits)) == 0;
}

static void clone_kill(ev_t* E, int half, cvec_t* cv, int n_hits) {
    /* table indexed by hit: (best score, id of its candidate); a smaller
     * (score, id) pair is better.  Pass 1 keeps the minimum per hit, pass 2
     * counts how many hits of each candidate still carry its own pair. */
    double* bs = (double*)malloc(sizeof(double) * (size_t)(n_hits > 0 ? n_hits : 1));
    int32_t* bid = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_hits > 0 ? n_hits : 1));
    for (int h = 0; h < n_hits; ++h) {
        bs[h] = INFINITY;
        bid[h] = -1;
    }
    for (int k = 0; k < cv->n; ++k) {
        const cand_t* cd = &cv->v[k];
        for (int s = 0; s < 6; ++s) {
            int h = cd->hits[s];
            if (h < 0) continue;
            if (cd->score < bs[h] || (cd->score == bs[h] && (bid[h] < 0 || cd->id < bid[h]))) {
                bs[h] = cd->score;
                bid[h] = cd->id;
            }
        }
    }
    for (int k = 0; k < cv->n; ++k) {
        cand_t* cd = &cv->v[k];
        int owned = 0;
        for (int s = 0; s < 6; ++s) {
            int h = cd->hits[s];
            if (h >= 0 && bs[h] == cd->score && bid[h] == cd->id) owned++;
        }
        cd->keep = owned >= 3 || (owned >= 2 && cd->nx == 6);
        if (cd->keep) E->cnt.kept++;
    }
    /* ledger: a hit whose winning score is nearly tied with a candidate of a
     * different hit set */
    if (E->tau > 0) {
        for (int k = 0; k < cv->n; ++k) {
            const cand_t* a = &cv->v[k];
            for (int s = 0; s < 6; ++s) {
                int h = a->hits[s];
                if (h < 0 || bid[h] == a->id) continue;
                const cand_t* w = &cv->v[bid[h]];
                if (same_hits(a, w)) continue;
                double m = fabs(a->score - w->score) / dmax2(a->score, w->score);
                if (m <= E->tau) {
                    int32_t hh[12];
                    for (int q = 0; q < 6; ++q) {
                        hh[q] = a->hits[q];
                        hh[6 + q] = w->hits[q];
                    }
                    ledger_add(E, OR_L_CLONE, half, m, hh, 12);
                }
            }
        }
    }
    free(bs);
    free(bid);
}

/* ------------------------------------------------------------------------ */
/* UV seeding (iterative variant), Section 3.4                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t hits[6]; /* per stereo slot (layers 1,2,5,6,9,10) */
    int n;
    double chi2, y0, ty;
} uvc_t;

static int uv_slot(int L) {
    for (int k = 0; k < 6; ++k)
        if (UV_LAYERS[k] == L) return k;
    return -1;
}

static int uv_seed(ev_t* E, int half, const cand_t* cd, uvc_t* best_out) {
    const or_config* c = E->c;
    const double ylo = half ? -c->uv_y_overlap : -c->uv_y_max;
    const double yhi = half ? c->uv_y_max : c->uv_y_overlap;
    uvc_t* all = NULL;
    int nall = 0, cap = 0;
    int32_t ctx[6];
    int nctx = 0;
    for (int s = 0; s < 6; ++s)
        if (cd->hits[s] >= 0) ctx[nctx++] = cd->hits[s];
    for (int pass = 0; pass < 2; ++pass) {
        const int Li = c->uv_init[pass];
        const int zi = 2 * Li + half;
        const double zI = c->z[Li], tI = c->dxdy[Li];
        const double XI = xmodel(c, cd->th, zI);
        const double SI = xscale(c, cd->th, zI);
        for (int k = 0; k < E->zn[zi]; ++k) {
            const double xh = E->zl[zi][k].x;
            const int32_t h = E->zl[zi][k].i;
            if (E->used && E->used[h]) continue;
            /* the stereo hit's y (Section 3.4) */
            const double y = (XI - xh) / tI;
            {
                int32_t hh[7];
                for (int q = 0; q < nctx; ++q) hh[q] = ctx[q];
                hh[nctx] = h;
                double m = fmin(fabs(y - ylo), fabs(y - yhi)) * fabs(tI) /
                           dmax2(dmax2(SI, fabs(xh)), fabs(yhi * tI));
                ledger_add(E, OR_L_UV_WIN, half, m, hh, nctx + 1);
            }
            if (y < ylo || y > yhi) continue;
            E->cnt.uv_init++;
            uvc_t u;
            for (int q = 0; q < 6; ++q) u.hits[q] = -1;
            u.hits[uv_slot(Li)] = h;
            int n = 1;
            double ty = y / zI; /* slope from the origin */
            int32_t cx[7];
            for (int q = 0; q < nctx; ++q) cx[q] = ctx[q];
            cx[nctx] = h;
            for (int q = 0; q < 6; ++q) {
                const int L = UV_LAYERS[q];
                if (L == Li) continue; /* remaining layers in increasing z */
                const double zL = c->z[L], tL = c->dxdy[L];
                const double XL = xmodel(c, cd->th, zL);
                const double xp = XL - tL * ty * zL;
                const double sc = dmax2(xscale(c, cd->th, zL), fabs(tL * ty * zL));
                int hb = closest_hit(E, 2 * L + half, xp, c->uv_tol, sc, OR_L_UV_TOL, OR_L_UV_TIE,
                                     half, cx, nctx + 1);
                if (hb >= 0) {
                    const double yL = (XL - E->x[hb]) / tL;
                    ty = 0.5 * (ty + yL / zL); /* averaging refinement */
                    u.hits[q] = hb;
                    n++;
                }
            }
            if (n < c->n_uv_min) continue;
            E->cnt.uv_cands++;
            double y0f, tyf;
            /* fit in increasing z for a canonical summation order */
            double zs2[6], ys2[6];
            int m = 0;
            for (int q = 0; q < 6; ++q) {
                int hq = u.hits[q];
                if (hq < 0) continue;
                const int L = UV_LAYERS[q];
                zs2[m] = c->z[L];
                ys2[m] = (xmodel(c, cd->th, c->z[L]) - E->x[hq]) / c->dxdy[L];
                m++;
            }
            u.chi2 = fit_line(m, zs2, ys2, &y0f, &tyf) / (c->sigma_y * c->sigma_y);
            u.n = m;
            u.y0 = y0f;
            u.ty = tyf;
            if (nall == cap) {
                cap = cap ? 2 * cap : 16;
                all = (uvc_t*)realloc(all, sizeof(uvc_t) * (size_t)cap);
            }
            all[nall++] = u;
        }
    }
    /* most hits, then smallest chi2_y; first in (pass, x) order on ties */
    int b = -1;
    for (int k = 0; k < nall; ++k)
        if (b < 0 || all[k].n > all[b].n || (all[k].n == all[b].n && all[k].chi2 < all[b].chi2)) b = k;
    if (b >= 0 && E->tau > 0) {
        for (int k = 0; k < nall; ++k) {
            if (k == b || all[k].n != all[b].n) continue;
            if (memcmp(all[k].hits, all[b].hits, sizeof(all[k].hits)) == 0) continue;
            double m = fabs(all[k].chi2 - all[b].chi2) / dmax2(dmax2(all[k].chi2, all[b].chi2), 1e-300);
            int32_t hh[12];
            for (int q = 0; q < 6; ++q) {
                hh[q] = all[b].hits[q];
                hh[6 + q] = all[k].hits[q];
            }
            ledger_add(E, OR_L_UV_SEL, half, m, hh, 12);
        }
    }
    if (b >= 0) *best_out = all[b];
    free(all);
    return b >= 0;
}

/* ------------------------------------------------------------------------ */
/* UV seeding, Hough-cluster variant, Section 3.4                           */
/* ------------------------------------------------------------------------ */
/* Every stereo hit of the seed's half whose y lies in the same window as the
 * iterative variant's first layer is mapped to t_y = y / z (a straight line
 * from the origin) and to a coarse bin of [ty_lo, ty_hi) (hough_bins bins;
 * half 1: [-ty_in, ty_max], half 0 mirrored).  A cluster b is the pair of
 * bins (b, b+1); its population is the number of stereo LAYERS with a hit in
 * either bin.  The clusters with the largest populations (at least n_uv_min;
 * ties to the smaller b) are kept, up to hough_clusters of them, and each is
 * divided into hough_fine t_y hypotheses at the centres of equal sub-bins.
 * For each hypothesis the closest hit within uv_tol is attached in every
 * stereo layer; combinations with at least n_uv_min hits are fitted as in the
 * iterative variant and the best is chosen by the same rule (most hits, then
 * smallest chi2_y), ties to the earlier hypothesis (cluster rank, then
 * sub-bin). */
static int uv_seed_hough(ev_t* E, int half, const cand_t* cd, uvc_t* best_out) {
    const or_config* c = E->c;
    const double ylo = half ? -c->uv_y_overlap : -c->uv_y_max;
    const double yhi = half ? c->uv_y_max : c->uv_y_overlap;
    const double ty_lo = half ? -c->hough_ty_in : -c->hough_ty_max;
    const double ty_hi = half ? c->hough_ty_max : c->hough_ty_in;
    const int NB = c->hough_bins, F = c->hough_fine;
    const double w = (ty_hi - ty_lo) / NB;
    int32_t ctx[7];
    int nctx = 0;
    for (int s = 0; s < 6; ++s)
        if (cd->hits[s] >= 0) ctx[nctx++] = cd->hits[s];
    /* hits of every stereo layer in every coarse bin */
    int occ[6][64];
    memset(occ, 0, sizeof(occ));
    for (int q = 0; q < 6; ++q) {
        const int L = UV_LAYERS[q];
        const int zi = 2 * L + half;
        const double zL = c->z[L], tL = c->dxdy[L];
        const double XL = xmodel(c, cd->th, zL);
        const double SL = xscale(c, cd->th, zL);
        for (int k = 0; k < E->zn[zi]; ++k) {
            if (E->used && E->used[E->zl[zi][k].i]) continue;
            const double xh = E->zl[zi][k].x;
            ctx[nctx] = E->zl[zi][k].i;
            const double y = (XL - xh) / tL;
            const double S = dmax2(dmax2(SL, fabs(xh)), fabs(yhi * tL));
            ledger_add(E, OR_L_UV_WIN, half, fmin(fabs(y - ylo), fabs(y - yhi)) * fabs(tL) / S, ctx, nctx + 1);
            if (y < ylo || y > yhi) continue;
            const double u = (y / zL - ty_lo) / w;
            int b = (int)floor(u);
            /* distance to the nearer bin edge, as an x distance in the layer */
            const double du = fmin(u - floor(u), ceil(u) - u);
            ledger_add(E, OR_L_HOUGH_BIN, half, du * w * zL * fabs(tL) / S, ctx, nctx + 1);
            if (b < 0) b = 0;
            if (b > NB - 1) b = NB - 1;
            occ[q][b]++;
        }
    }
    /* cluster populations and the kept clusters, best first */
    int pop[64], sel[8], nsel = 0;
    for (int b = 0; b + 1 < NB; ++b) {
        pop[b] = 0;
        for (int q = 0; q < 6; ++q) pop[b] += occ[q][b] + occ[q][b + 1] > 0;
    }
    for (int p = 6; p >= c->n_uv_min && nsel < c->hough_clusters; --p)
        for (int b = 0; b + 1 < NB && nsel < c->hough_clusters; ++b)
            if (pop[b] == p) sel[nsel++] = b;
    /* hypotheses */
    uvc_t best;
    int have = 0;
    nctx = 0;
    for (int s = 0; s < 6; ++s)
        if (cd->hits[s] >= 0) ctx[nctx++] = cd->hits[s];
    uvc_t all[64];
    int nall = 0;
    for (int r = 0; r < nsel; ++r) {
        for (int f = 0; f < F; ++f) {
            const double ty = ty_lo + w * (sel[r] + (f + 0.5) * 2.0 / F);
            E->cnt.uv_init++;
            uvc_t u;
            int n = 0;
            for (int q = 0; q < 6; ++q) {
                const int L = UV_LAYERS[q];
                const double zL = c->z[L], tL = c->dxdy[L];
                const double XL = xmodel(c, cd->th, zL);
                const double xp = XL - tL * ty * zL;
                const double sc = dmax2(xscale(c, cd->th, zL), fabs(tL * ty * zL));
                u.hits[q] = closest_hit(E, 2 * L + half, xp, c->uv_tol, sc, OR_L_UV_TOL, OR_L_UV_TIE, half,
                                        ctx, nctx);
                n += u.hits[q] >= 0;
            }
            if (n < c->n_uv_min) continue;
            E->cnt.uv_cands++;
            double zs2[6], ys2[6], y0f, tyf;
            int m = 0;
            for (int q = 0; q < 6; ++q) {
                if (u.hits[q] < 0) continue;
                const int L = UV_LAYERS[q];
                zs2[m] = c->z[L];
                ys2[m] = (xmodel(c, cd->th, c->z[L]) - E->x[u.hits[q]]) / c->dxdy[L];
                m++;
            }
            u.chi2 = fit_line(m, zs2, ys2, &y0f, &tyf) / (c->sigma_y * c->sigma_y);
            u.n = m;
            u.y0 = y0f;
            u.ty = tyf;
            all[nall++] = u;
            if (!have || u.n > best.n || (u.n == best.n && u.chi2 < best.chi2)) {
                best = u;
                have = 1;
            }
        }
    }
    if (have && E->tau > 0) {
        for (int k = 0; k < nall; ++k) {
            if (all[k].n != best.n || memcmp(all[k].hits, best.hits, sizeof(best.hits)) == 0) continue;
            double m = fabs(all[k].chi2 - best.chi2) / dmax2(dmax2(all[k].chi2, best.chi2), 1e-300);
            int32_t hh[12];
            for (int q = 0; q < 6; ++q) {
                hh[q] = best.hits[q];
                hh[6 + q] = all[k].hits[q];
            }
            ledger_add(E, OR_L_UV_SEL, half, m, hh, 12);
        }
    }
    if (have) *best_out = best;
    return have;
}

/* ------------------------------------------------------------------------ */
/* event driver                                                             */
/* ------------------------------------------------------------------------ */

int32_t or_seeding_event(const or_config* c, int32_t n_hits, const double* x,
                         const int32_t* zone,
                         or_seed* seeds, int32_t seeds_cap, int32_t* n_seeds,
                         or_cand* cands, int32_t cands_cap, int32_t* n_cands,
                         int32_t* trips, int32_t trips_cap, int32_t* n_trips,
                         or_ledger* ledger, int32_t ledger_cap, int32_t* n_ledger,
                         double tau, or_counters* counters) {
    int32_t ns = 0, nc = 0, nt = 0;
    if (n_seeds) *n_seeds = 0;
    if (n_cands) *n_cands = 0;
    if (n_trips) *n_trips = 0;
    if (n_ledger) *n_ledger = 0;
    if (!config_ok(c) || n_hits < 0) return -1;
    for (int i = 0; i < n_hits; ++i)
        if (zone[i] < 0 || zone[i] >= NZONE || !isfinite(x[i])) return -1;

    ev_t E;
    memset(&E, 0, sizeof(E));
    E.c = c;
    E.x = x;
    E.led = ledger;
    E.led_cap = ledger ? ledger_cap : 0;
    E.tau = (ledger || n_ledger) ? tau : -1.0;
    /* per-zone hit lists in ascending (x, index) order */
    for (int i = 0; i < n_hits; ++i) E.zn[zone[i]]++;
    for (int z = 0; z < NZONE; ++z) {
        E.zl[z] = (xi_t*)malloc(sizeof(xi_t) * (size_t)(E.zn[z] > 0 ? E.zn[z] : 1));
        E.zn[z] = 0;
    }
    for (int i = 0; i < n_hits; ++i) {
        xi_t* p = &E.zl[zone[i]][E.zn[zone[i]]++];
        p->x = x[i];
        p->i = i;
    }
    for (int z = 0; z < NZONE; ++z) qsort(E.zl[z], (size_t)E.zn[z], sizeof(xi_t), cmp_xi);

    /* HLT1: both iterations, one clone kill, UV (Sections 3.2-3.4).  HLT2-style
     * (iter_mode 1): one iteration at a time, each with its own clone kill and
     * UV step; the hits of its seeds are removed before the next iteration. */
    unsigned char* used = NULL;
    if (c->iter_mode == 1) {
        used = (unsigned char*)calloc((size_t)(n_hits > 0 ? n_hits : 1), 1);
        E.used = used;
    }
    const int n_pass = c->iter_mode == 1 ? c->n_iter : 1;
    for (int half = 0; half < 2; ++half) {
        for (int pass = 0; pass < n_pass; ++pass) {
            cvec_t cv = {0};
            const int it0 = c->iter_mode == 1 ? pass : 0, it1 = c->iter_mode == 1 ? pass + 1 : c->n_iter;
            xz_search(&E, half, &cv, trips, trips_cap, &nt, it0, it1);
            clone_kill(&E, half, &cv, n_hits);
            int32_t* taken = (int32_t*)malloc(sizeof(int32_t) * 12 * (size_t)(cv.n > 0 ? cv.n : 1));
            int n_taken = 0;
            for (int k = 0; k < cv.n; ++k) {
                const cand_t* cd = &cv.v[k];
                if (cands && nc < cands_cap) {
                    or_cand* o = &cands[nc];
                    memcpy(o->hits, cd->hits, sizeof(o->hits));
                    o->half = half; o->iter = cd->iter; o->nx = cd->nx; o->keep = cd->keep;
                    o->h1 = cd->h1; o->h2 = cd->h2; o->h3 = cd->h3; o->id = cd->id;
                    o->a = cd->th[0]; o->b = cd->th[1]; o->c = cd->th[2];
                    o->chi2 = cd->chi2; o->score = cd->score;
                }
                nc++;
                if (!cd->keep) continue;
                uvc_t u;
                if (!(c->uv_mode == 1 ? uv_seed_hough(&E, half, cd, &u) : uv_seed(&E, half, cd, &u))) continue;
                E.cnt.seeds++;
                for (int q = 0; q < 6; ++q) {
                    if (cd->hits[q] >= 0) taken[n_taken++] = cd->hits[q];
                    if (u.hits[q] >= 0) taken[n_taken++] = u.hits[q];
                }
                if (seeds && ns < seeds_cap) {
                    or_seed* s = &seeds[ns];
                    for (int l = 0; l < OR_NLAYER; ++l) s->hits[l] = -1;
                    for (int q = 0; q < 6; ++q) {
                        s->hits[X_LAYERS[q]] = cd->hits[q];
                        s->hits[UV_LAYERS[q]] = u.hits[q];
                    }
                    s->half = half;
                    s->nx = cd->nx;
                    s->nuv = u.n;
                    s->cand_id = cd->id;
                    s->pass = pass;
                    s->pad = 0;
                    s->a = cd->th[0]; s->b = cd->th[1]; s->c = cd->th[2];
                    s->chi2x = cd->chi2;
                    s->y0 = u.y0; s->ty = u.ty; s->chi2y = u.chi2;
                    /* state for matching (reading of Section 4.1's z_ref for SciFi) */
                    const double zS = c->z_state, zb = zS - c->z_ref;
                    s->x_s = xmodel(c, cd->th, zS);
                    s->tx_s = cd->th[1] + cd->th[2] * (2.0 * zb + 3.0 * c->d_ratio * zb * zb);
                    s->y_s = u.y0 + u.ty * zS;
                    s->ty_s = u.ty;
                }
                ns++;
            }
            /* hit cleanup: the next iteration does not see this one's seeds' hits */
            if (used)
                for (int k = 0; k < n_taken; ++k) used[taken[k]] = 1;
            free(taken);
            free(cv.v);
        }
    }
    free(used);
    for (int z = 0; z < NZONE; ++z) free(E.zl[z]);
    if (n_seeds) *n_seeds = ns;
    if (n_cands) *n_cands = nc;
    if (n_trips) *n_trips = nt;
    if (n_ledger) *n_ledger = E.n_led;
    if (counters) {
        counters->pairs += E.cnt.pairs;
        counters->triplets += E.cnt.triplets;
        counters->ext_ok += E.cnt.ext_ok;
        counters->cands += E.cnt.cands;
        counters->kept += E.cnt.kept;
        counters->uv_init += E.cnt.uv_init;
        counters->uv_cands += E.cnt.uv_cands;
        counters->seeds += E.cnt.seeds;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Matching, Section 4                                                      */
/* ------------------------------------------------------------------------ */

int32_t or_matching_event(const or_config* c, int32_t n_velo, const double* velo,
                          int32_t n_seeds, const double* seed_state,
                          int32_t* velo_idx, double* chi2_out,
                          or_ledger* ledger, int32_t ledger_cap, int32_t* n_ledger,
                          double tau, or_counters* counters) {
    ev_t E;
    memset(&E, 0, sizeof(E));
    E.c = c;
    E.led = ledger;
    E.led_cap = ledger ? ledger_cap : 0;
    E.tau = (ledger || n_ledger) ? tau : -1.0;
    if (n_ledger) *n_ledger = 0;
    if (n_velo < 0 || n_seeds < 0) return -1;
    const double ps = c->presel_scale, ts = c->tol_scale;
    for (int s = 0; s < n_seeds; ++s) {
        const double xS = seed_state[4 * s + 0], yS = seed_state[4 * s + 1];
        const double txS = seed_state[4 * s + 2], tyS = seed_state[4 * s + 3];
        int best = -1, second = -1;
        double bchi = INFINITY, schi = INFINITY;
        for (int v = 0; v < n_velo; ++v) {
            const double xV = velo[4 * v + 0], yV = velo[4 * v + 1];
            const double txV = velo[4 * v + 2], tyV = velo[4 * v + 3];
            E.cnt.match_pairs++;
            const double dtx = txV - txS, dty = tyV - tyS;
            /* kink position, Eq. z_match */
            const double zmx = c->zmx[0] + c->zmx[1] * fabs(dtx) + c->zmx[2] * dtx * dtx +
                               c->zmx[3] * fabs(xS) + c->zmx[4] * txV * txV;
            /* both segments as straight lines to z_match_x and to z_match_y */
            const double dx = (xV + (zmx - c->z_velo) * txV) - (xS + (zmx - c->z_state) * txS);
            const double dy = (yV + (c->z_match_y - c->z_velo) * tyV) -
                              (yS + (c->z_match_y - c->z_state) * tyS);
            const double cut[4] = {c->presel[0] * ps, c->presel[1] * ps, c->presel[2] * ps,
                                   c->presel[3] * ps};
            const double val[4] = {fabs(dx), fabs(dy), fabs(dtx), fabs(dty)};
            int pass = 1;
            for (int q = 0; q < 4; ++q) {
                int32_t hh[2] = {s, v};
                ledger_add(&E, OR_L_M_PRESEL, 0, fabs(val[q] - cut[q]) / cut[q], hh, 2);
                if (!(val[q] < cut[q])) pass = 0;
            }
            if (!pass) continue;
            E.cnt.match_presel++;
            /* chi2_match with the tolerances of Section 4.2 */
            const double tolx = ts * c->tolx[0] * (c->tolx[1] * c->tolx[1] + c->tolx[2] * c->tolx[2] * dtx * dtx);
            const double rho = txV * txV + tyV * tyV;
            const double toly = ts * c->toly[0] * (c->toly[1] * c->toly[1] + c->toly[2] * c->toly[2] * rho);
            const double toltx = ts * c->tol_tx, tolty = ts * c->tol_ty;
            const double chi2 = dx * dx / tolx + dy * dy / toly + dtx * dtx / toltx + dty * dty / tolty;
            {
                int32_t hh[2] = {s, v};
                ledger_add(&E, OR_L_M_CHI2, 0, fabs(chi2 - c->chi2_match_max) / c->chi2_match_max, hh, 2);
            }
            if (!(chi2 < c->chi2_match_max)) continue;
            if (chi2 < bchi) {
                second = best; schi = bchi;
                best = v; bchi = chi2;
            } else if (chi2 < schi) {
                second = v; schi = chi2;
            }
        }
        if (best >= 0 && second >= 0) {
            int32_t hh[3] = {s, best, second};
            ledger_add(&E, OR_L_M_TIE, 0, fabs(schi - bchi) / dmax2(schi, 1e-300), hh, 3);
        }
        velo_idx[s] = best;
        chi2_out[s] = best >= 0 ? bchi : 0.0;
        if (best >= 0) E.cnt.matched++;
    }
    if (c->velo_unique) {
        /* a VELO segment keeps only its best seed: lowest chi2, then lower
         * seed index; the other seeds lose their match */
        for (int s = 0; s < n_seeds; ++s) {
            int v = velo_idx[s];
            if (v < 0) continue;
            for (int t = 0; t < n_seeds; ++t) {
                if (t == s || velo_idx[t] != v) continue;
                if (chi2_out[t] < chi2_out[s] || (chi2_out[t] == chi2_out[s] && t < s)) {
                    int32_t hh[3] = {s, t, v};
                    ledger_add(&E, OR_L_M_TIE, 0,
                               fabs(chi2_out[t] - chi2_out[s]) / dmax2(chi2_out[s], 1e-300), hh, 3);
                    velo_idx[s] = -2; /* marked; cleared below */
                    break;
                }
            }
        }
        for (int s = 0; s < n_seeds; ++s)
            if (velo_idx[s] == -2) {
                velo_idx[s] = -1;
                chi2_out[s] = 0.0;
                E.cnt.matched--;
            }
    }
    if (n_ledger) *n_ledger = E.n_led;
    if (counters) {
        counters->match_pairs += E.cnt.match_pairs;
        counters->match_presel += E.cnt.match_presel;
        counters->matched += E.cnt.matched;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Final selection, Section 4.4                                             */
/* ------------------------------------------------------------------------ */

double or_ghost_nn(const float* nn, const double f[8]) {
    const float* mean = nn;
    const float* inv_scale = nn + 8;
    const float* W1 = nn + 16;
    const float* b1 = nn + 16 + 256;
    const float* w2 = nn + 16 + 256 + 32;
    const double b2 = nn[16 + 256 + 64];
    double in[8];
    for (int i = 0; i < 8; ++i) in[i] = (f[i] - mean[i]) * inv_scale[i];
    double z = b2;
    for (int k = 0; k < 32; ++k) {
        double a = b1[k];
        for (int i = 0; i < 8; ++i) a += W1[8 * k + i] * in[i];
        if (a > 0) z += w2[k] * a;
    }
    return 1.0 / (1.0 + exp(-z));
}

int32_t or_final_selection(const or_config* c, int32_t n_velo, const double* velo, int32_t n_seeds,
                           const double* seed_state, const int32_t* seed_nhits, const float* nn,
                           int32_t* velo_idx, const double* chi2, double* ghost_prob,
                           or_ledger* ledger, int32_t ledger_cap, int32_t* n_ledger, double tau) {
    ev_t E;
    memset(&E, 0, sizeof(E));
    E.c = c;
    E.led = ledger;
    E.led_cap = ledger ? ledger_cap : 0;
    E.tau = (ledger || n_ledger) ? tau : -1.0;
    if (n_ledger) *n_ledger = 0;
    if (!config_ok(c) || n_velo < 0 || n_seeds < 0 || !nn) return -1;
    for (int s = 0; s < n_seeds; ++s) {
        const int v = velo_idx[s];
        ghost_prob[s] = 1.0;
        if (v < 0 || v >= n_velo) continue;
        const double xS = seed_state[4 * s + 0], yS = seed_state[4 * s + 1];
        const double txS = seed_state[4 * s + 2], tyS = seed_state[4 * s + 3];
        const double xV = velo[4 * v + 0], yV = velo[4 * v + 1];
        const double txV = velo[4 * v + 2], tyV = velo[4 * v + 3];
        const double dtx = txV - txS, dty = tyV - tyS;
        const double zmx = c->zmx[0] + c->zmx[1] * fabs(dtx) + c->zmx[2] * dtx * dtx + c->zmx[3] * fabs(xS) +
                           c->zmx[4] * txV * txV;
        /* the two segments at z_match_x and z_match_y, as in the matching */
        const double xv_m = xV + (zmx - c->z_velo) * txV, xs_m = xS + (zmx - c->z_state) * txS;
        const double yv_m = yV + (c->z_match_y - c->z_velo) * tyV, ys_m = yS + (c->z_match_y - c->z_state) * tyS;
        const double dx = xv_m - xs_m, dy = yv_m - ys_m;
        /* pseudorapidity of the VELO segment: tan(theta) = |slope|, eta =
         * -ln tan(theta/2) = asinh(1/|slope|); slopes below 1e-6 count as 1e-6 */
        const double rho = fmax(sqrt(txV * txV + tyV * tyV), 1e-6);
        const double f[8] = {zmx, dx, dy, dtx, dty, chi2[s], asinh(1.0 / rho), (double)seed_nhits[s]};
        const double p = or_ghost_nn(nn, f);
        ghost_prob[s] = p;
        int32_t hh[2] = {s, v};
        ledger_add(&E, OR_L_GHOST, 0, fabs(p - c->ghost_max) / c->ghost_max, hh, 2);
        if (!(p < c->ghost_max)) velo_idx[s] = -1;
    }
    /* clone removal among the kept pairs: one pair per seed here, so only a
     * shared VELO segment can make a clone */
    int* drop = (int*)calloc((size_t)(n_seeds > 0 ? n_seeds : 1), sizeof(int));
    for (int s = 0; s < n_seeds; ++s) {
        if (velo_idx[s] < 0) continue;
        for (int t = 0; t < n_seeds; ++t) {
            if (t == s || velo_idx[t] != velo_idx[s]) continue;
            const double d = ghost_prob[s] - ghost_prob[t];
            int32_t hh[3] = {s, t, velo_idx[s]};
            ledger_add(&E, OR_L_M_CLONE, 0, fabs(d - c->clone_margin) / c->clone_margin, hh, 3);
            if (d >= c->clone_margin) drop[s] = 1;
        }
    }
    for (int s = 0; s < n_seeds; ++s)
        if (drop[s]) velo_idx[s] = -1;
    free(drop);
    if (n_ledger) *n_ledger = E.n_led;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* UT hits of the Long tracks, Section 4.3                                  */
/* ------------------------------------------------------------------------ */

int32_t or_ut_search(const or_config* c, int32_t n_velo, const double* velo, int32_t n_seeds,
                     const double* seed_state, int32_t* velo_idx, int32_t n_ut, const double* ut_x,
                     const int32_t* ut_layer, int32_t* ut_hits, int32_t* n_ut_out, double* gamma,
                     or_ledger* ledger, int32_t ledger_cap, int32_t* n_ledger, double tau) {
    ev_t E;
    memset(&E, 0, sizeof(E));
    E.c = c;
    E.led = ledger;
    E.led_cap = ledger ? ledger_cap : 0;
    E.tau = (ledger || n_ledger) ? tau : -1.0;
    if (n_ledger) *n_ledger = 0;
    if (!config_ok(c) || n_velo < 0 || n_seeds < 0 || n_ut < 0) return -1;
    for (int i = 0; i < n_ut; ++i)
        if (ut_layer[i] < 0 || ut_layer[i] > 3 || !isfinite(ut_x[i])) return -1;
    for (int s = 0; s < n_seeds; ++s) {
        for (int l = 0; l < 4; ++l) ut_hits[4 * s + l] = -1;
        n_ut_out[s] = 0;
        gamma[s] = 0.0;
        const int v = velo_idx[s];
        if (v < 0 || v >= n_velo) continue;
        const double xV = velo[4 * v + 0], yV = velo[4 * v + 1];
        const double txV = velo[4 * v + 2], tyV = velo[4 * v + 3];
        const double txS = seed_state[4 * s + 2];
        /* the pair's q/p from its kink, and 1/p in (GeV/c)^-1 for the windows */
        const double qop = (txS - txV) / c->ut_kick;
        const double inv_p_gev = 1000.0 * fabs(qop);
        double g = c->ut_gamma[0] + c->ut_gamma[1] * qop; /* Eq. gamma_parametrisation */
        int found = 0, n = 0;
        for (int l = 0; l < 4; ++l) {
            const double* w = found ? &c->ut_tight[4 * l] : &c->ut_loose[4 * l];
            if (!(w[3] > 0)) continue; /* no window of this kind in this layer */
            const double win = fmin(fmax(w[0] + w[1] * inv_p_gev, w[2]), w[3]);
            const double dz = c->ut_z[l] - c->z_velo;
            /* Eq. velo_ut_extrapolation, then the layer's measured coordinate */
            const double xt = xV + txV * dz + g * dz * dz;
            const double yt = yV + tyV * dz;
            const double xm = xt - yt * c->ut_dxdy[l];
            int best = -1;
            double bd = INFINITY, bx = 0;
            for (int i = 0; i < n_ut; ++i) {
                if (ut_layer[i] != l) continue;
                const double d = fabs(ut_x[i] - xm);
                const double S = dmax2(dmax2(fabs(xm), fabs(ut_x[i])), 1.0);
                int32_t hh[3] = {s, v, i};
                ledger_add(&E, OR_L_UT_WIN, 0, fabs(d - win) / S, hh, 3);
                if (d > win) continue;
                if (best >= 0) {
                    int32_t h2[4] = {s, v, best, i};
                    ledger_add(&E, OR_L_UT_TIE, 0, fabs(d - bd) / S, h2, 4);
                }
                if (best < 0 || d < bd || (d == bd && (ut_x[i] < bx || (ut_x[i] == bx && i < best)))) {
                    best = i;
                    bd = d;
                    bx = ut_x[i];
                }
            }
            if (best < 0) continue;
            ut_hits[4 * s + l] = best;
            n++;
            if (!found) {
                /* gamma_x through the loose-window hit */
                g = (ut_x[best] + yt * c->ut_dxdy[l] - xV - txV * dz) / (dz * dz);
                found = 1;
            }
        }
        n_ut_out[s] = n;
        gamma[s] = g;
        if (n < c->ut_min_hits) velo_idx[s] = -1;
    }
    if (n_ledger) *n_ledger = E.n_led;
    return 0;
}
