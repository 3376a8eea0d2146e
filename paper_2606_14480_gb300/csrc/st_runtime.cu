// st_runtime.cu -- host side of libst: the C ABI declared in include/st.h.
//
// Configuration and its device constants, per-call scratch (one arena per
// workspace), the seeding / matching launch sequences, CUDA-graph capture,
// work counters, and the continuous-batching pipeline (submit / poll).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "st.h"
#include "st_host.h"
#include "st_kernels.cuh"
#include "st_ut.cuh"

using namespace st;

namespace {

const int kXL[6] = {0, 3, 4, 7, 8, 11};
const int kUL[6] = {1, 2, 5, 6, 9, 10};

int xslot(int L) {
    for (int k = 0; k < 6; ++k)
        if (kXL[k] == L) return k;
    return -1;
}
int uslot(int L) {
    for (int k = 0; k < 6; ++k)
        if (kUL[k] == L) return k;
    return -1;
}

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

void split(double v, float& hi, float& lo) {
    hi = static_cast<float>(v);
    lo = static_cast<float>(v - static_cast<double>(hi));
}

// Solve the n x n system A X = R (columns of R) by Gauss-Jordan elimination
// with partial pivoting, in place.  Returns false if singular.
bool gauss_jordan(int n, double A[3][3], double R[3][6], int ncol) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int i = c + 1; i < n; ++i)
            if (std::fabs(A[i][c]) > std::fabs(A[piv][c])) piv = i;
        if (A[piv][c] == 0.0) return false;
        std::swap(A[c], A[piv]);
        std::swap(R[c], R[piv]);
        const double d = A[c][c];
        for (int j = 0; j < n; ++j) A[c][j] /= d;
        for (int j = 0; j < ncol; ++j) R[c][j] /= d;
        for (int i = 0; i < n; ++i) {
            if (i == c) continue;
            const double f = A[i][c];
            for (int j = 0; j < n; ++j) A[i][j] -= f * A[c][j];
            for (int j = 0; j < ncol; ++j) R[i][j] -= f * R[c][j];
        }
    }
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// configuration
// ---------------------------------------------------------------------------

extern "C" void st_config_default(st_config* c) {
    std::memset(c, 0, sizeof(*c));
    const double zl[12] = {7826, 7896, 7966, 8036, 8508, 8578, 8648, 8718, 9193, 9263, 9333, 9403};
    const double t5 = std::tan(5.0 * M_PI / 180.0);  // stereo angle (Section 1)
    for (int l = 0; l < 12; ++l) {
        c->z[l] = zl[l];
        const int u = uslot(l);
        c->dxdy[l] = u < 0 ? 0.0 : ((u & 1) ? -t5 : t5);  // u layers +5 deg, v layers -5 deg
    }
    c->z_ref = 8520.0;
    c->d_ratio = -2.6e-4;
    c->invp_a = 1.6322e-7;     // Eq. (invp)
    c->invp_b = -5.0217e-12;
    c->p_min = 3000.0;         // 3 GeV/c
    c->alpha0 = 2.180e6;       // Eq. (alphacorr)
    c->alpha1 = -1073.0;
    c->dx3_scale = 1.0;
    c->n_iter = 2;
    // the third row is only used by HLT2-style runs with three iterations
    const int il[3][3] = {{0, 4, 11}, {3, 7, 8}, {0, 7, 11}};
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) c->iter_layers[i][k] = il[i][k];
    c->kappa_c = 1.0e-2;
    c->m_lo = 0.5;
    c->m_hi = 1.5;
    c->c_nsigma = 5.0;
    c->sigma_x = 0.07;
    c->ext_tol = 1.0;
    c->chi2x_max = 10.0;
    c->score_w_chi2 = 1000.0;  // Eq. (seed_clone_score)
    c->score_w5 = 10.0;
    c->uv_init[0] = 1;
    c->uv_init[1] = 2;
    c->n_uv_min = 4;
    c->uv_tol = 2.0;
    c->uv_y_overlap = 50.0;
    c->uv_y_max = 2500.0;
    c->sigma_y = 0.07 / t5;
    c->z_state = 7826.0;
    c->z_velo = 770.0;
    c->z_match_y = 10000.0;
    const double zmx[5] = {5287.6, -7.98878, 317.683, 0.0119379, -1418.42};  // Table (mag_params)
    for (int k = 0; k < 5; ++k) c->zmx[k] = zmx[k];
    c->presel[0] = 20.0;
    c->presel[1] = 150.0;
    c->presel[2] = 1.5;
    c->presel[3] = 0.02;
    c->presel_scale = 1.0;
    c->tol_scale = 1.0;
    c->tolx[0] = 0.8;
    c->tolx[1] = 10.12;
    c->tolx[2] = 101.0;
    c->toly[0] = 0.2;
    c->toly[1] = 1.59;
    c->toly[2] = 212.1;
    c->tol_tx = 0.5;
    c->tol_ty = 1.0 / 937.5;
    c->chi2_match_max = 2.0;
    c->velo_unique = 0;
    c->uv_mode = 0;
    c->hough_bins = 64;
    c->hough_fine = 4;
    c->hough_clusters = 8;  // "up to eight of the best bins"
    c->hough_ty_max = 0.33;
    c->hough_ty_in = 0.01;
    c->final_sel = 0;
    c->ghost_max = 0.8;     // Section 4.4
    c->clone_margin = 0.05;
    {
        // UT (Section 4.3); the layer z are not given in the paper
        const double uz[4] = {2327.5, 2372.5, 2597.5, 2642.5};
        const int us[4] = {0, 1, -1, 0};
        for (int l = 0; l < 4; ++l) {
            c->ut_z[l] = uz[l];
            c->ut_dxdy[l] = us[l] * t5;
        }
        c->ut_gamma[0] = 7.707063e-11;  // Table (mag_params)
        c->ut_gamma[1] = -7.817364e-3;
        c->ut_kick = 1200.0;
        // Table (ut_search_window_values): loose windows of UTaX, UTaU, UTbV;
        // tight windows of UTaU, UTbV, UTbX
        const double lw[16] = {0.8333, 3.3333, 1.2, 8.5, 0.8333, 3.3333, 1.2, 8.5,
                               1.3333, 3.3333, 1.5, 9.5, 0, 0, 0, 0};
        const double tw[16] = {0, 0, 0, 0, 0.2, 0.6, 0.5, 2.0, 0.4, 1.2, 1.0, 4.0, 0.4, 1.2, 1.0, 4.0};
        for (int k = 0; k < 16; ++k) {
            c->ut_loose[k] = lw[k];
            c->ut_tight[k] = tw[k];
        }
        c->ut_min_hits = 3;  // "more than two associated UT hits"
    }
    c->iter_mode = 0;
    for (int it = 0; it < 3; ++it) c->p_min_iter[it] = 0.0;
    c->threads_seed = 256;
    c->threads_build = 512;
    c->threads_match = 256;
    c->ctas_per_sm = 0;
    c->smem_hits = 1536;
    c->cand_cap = 4096;
}

bool derive_params(const st_config& c, DevParams& P, std::string& err) {
    std::memset(&P, 0, sizeof(P));
    auto fail = [&](const char* m) {
        err = m;
        return false;
    };
    for (int l = 0; l + 1 < 12; ++l)
        if (!(c.z[l] < c.z[l + 1])) return fail("layer z must increase strictly");
    for (int k = 0; k < 6; ++k) {
        if (c.dxdy[kXL[k]] != 0.0) return fail("x-layers must have dxdy = 0");
        if (!(std::fabs(c.dxdy[kUL[k]]) > 0.0)) return fail("stereo layers need dxdy != 0");
    }
    if (c.n_iter < 1 || c.n_iter > 3) return fail("n_iter must be 1, 2 or 3");
    if (c.iter_mode < 0 || c.iter_mode > 1) return fail("iter_mode must be 0 or 1");
    for (int it = 0; it < 3; ++it)
        if (c.p_min_iter[it] < 0) return fail("p_min_iter must be >= 0");
    if (!(c.p_min > 0) || !(c.sigma_x > 0) || !(c.sigma_y > 0) || !(c.ext_tol > 0) || !(c.uv_tol > 0))
        return fail("p_min, sigma_x, sigma_y, ext_tol and uv_tol must be positive");
    if (c.n_uv_min < 2 || c.n_uv_min > 6) return fail("n_uv_min must be in [2, 6]");
    if (c.uv_mode < 0 || c.uv_mode > 1) return fail("uv_mode must be 0 or 1");
    if (c.hough_bins < 2 || c.hough_bins > 64 || c.hough_fine < 1 || c.hough_fine > 8 || c.hough_clusters < 1 ||
        c.hough_clusters > 8 || !(c.hough_ty_max + c.hough_ty_in > 0))
        return fail("Hough parameters: bins in [2, 64], fine and clusters in [1, 8], non-empty t_y range");
    if (c.final_sel < 0 || c.final_sel > 1 || (c.final_sel && c.velo_unique) || !(c.ghost_max > 0) ||
        !(c.clone_margin > 0))
        return fail("final_sel must be 0 or 1 and excludes velo_unique; ghost_max and clone_margin > 0");
    if (c.ut_min_hits < 0 || c.ut_min_hits > 4 || !(c.ut_kick > 0))
        return fail("ut_min_hits must be in [0, 4] and ut_kick > 0");
    for (int l = 0; l < 4; ++l)
        if (!(std::fabs(c.ut_z[l] - c.z_velo) > 0)) return fail("UT layers must not sit at z_velo");
    if (!(c.invp_b != 0.0) || !(c.invp_a * c.invp_a + 4 * c.invp_b / c.p_min >= 0))
        return fail("Eq. invp parameters give no momentum limit");
    if (c.threads_seed < 64 || c.threads_seed > kMaxThreads || c.threads_seed % 32 ||
        c.threads_build < 64 || c.threads_build > kMaxThreads || c.threads_build % 32 ||
        c.threads_match < 32 || c.threads_match > kMaxThreads || c.threads_match % 32)
        return fail("thread counts must be multiples of 32 in [64, 512]");
    if (c.smem_hits < 0 || c.smem_hits > 32768 || c.cand_cap < 16 || c.cand_cap > (1 << 20) || c.ctas_per_sm < 0)
        return fail("bad tuning value (smem_hits, cand_cap or ctas_per_sm)");

    auto F = [&](double z) {
        const double zb = z - c.z_ref;
        return zb * zb * (1.0 + c.d_ratio * zb);
    };
    for (int s = 0; s < 6; ++s) {
        const double z = c.z[kXL[s]];
        P.xzb[s] = static_cast<float>(z - c.z_ref);
        split(F(z), P.xf_hi[s], P.xf_lo[s]);
    }
    double zc = 0;
    for (int u = 0; u < 6; ++u) zc += c.z[kUL[u]];
    zc = std::rint(zc / 6.0);
    P.zc_uv = static_cast<float>(zc);
    for (int u = 0; u < 6; ++u) {
        const double z = c.z[kUL[u]];
        P.uz[u] = static_cast<float>(z);
        P.uzb[u] = static_cast<float>(z - c.z_ref);
        split(F(z), P.uf_hi[u], P.uf_lo[u]);
        P.ut[u] = static_cast<float>(c.dxdy[kUL[u]]);
        P.uzt[u] = static_cast<float>(z - zc);
        P.uinv_t[u] = static_cast<float>(1.0 / c.dxdy[kUL[u]]);
        P.uinv_z[u] = static_cast<float>(1.0 / z);
    }
    P.n_iter = c.n_iter;
    P.iter_mode = c.iter_mode;
    for (int it = 0; it < c.n_iter; ++it) {
        const double pmin = c.p_min_iter[it] > 0 ? c.p_min_iter[it] : c.p_min;
        if (!(c.invp_a * c.invp_a + 4 * c.invp_b / pmin >= 0))
            return fail("Eq. invp parameters give no momentum limit for an iteration's p_min");
        const int L1 = c.iter_layers[it][0], L2 = c.iter_layers[it][1], L3 = c.iter_layers[it][2];
        IterP& I = P.it[it];
        I.s1 = xslot(L1);
        I.s2 = xslot(L2);
        I.s3 = xslot(L3);
        if (I.s1 < 0 || I.s2 < 0 || I.s3 < 0 || L1 == L2 || L1 == L3 || L2 == L3)
            return fail("iteration layers must be three different x-layers");
        int ne = 0;
        for (int s = 0; s < 6; ++s)
            if (s != I.s1 && s != I.s2 && s != I.s3) I.ext[ne++] = s;
        const double z1 = c.z[L1], z2 = c.z[L2], z3 = c.z[L3];
        // two-hit window: Eqs. (tolHp) and (alphacorr)
        const double k = z1 / (z3 - z1);
        const double alpha = c.alpha0 / (k * (pmin - c.alpha1));
        I.scale3 = static_cast<float>((z3 + alpha) / z1);
        I.dx3 = static_cast<float>(c.dx3_scale * (z3 - z1) / (2.0 * z1 * c.invp_b) *
                                   (-c.invp_a + std::sqrt(c.invp_a * c.invp_a + 4.0 * c.invp_b / pmin)));
        I.inv_dz31 = static_cast<float>(1.0 / (z3 - z1));
        I.dz21 = static_cast<float>(z2 - z1);
        I.z1 = static_cast<float>(z1);
        // three-hit window: dx2 = k3 c_x, k3 from the track model
        const double k3 = F(z2) - F(z1) - (z2 - z1) / (z3 - z1) * (F(z3) - F(z1));
        if (k3 == 0.0) return fail("degenerate three-hit geometry");
        I.k3 = static_cast<float>(k3);
        I.inv_k3 = static_cast<float>(1.0 / k3);
        const double w1 = (z3 - z2) / (z3 - z1), w3 = (z2 - z1) / (z3 - z1);
        I.c0 = static_cast<float>(c.c_nsigma * c.sigma_x * std::sqrt(1.0 + w1 * w1 + w3 * w3) / std::fabs(k3));
        I.mlo_k = static_cast<float>(c.m_lo * c.kappa_c);
        I.mhi_k = static_cast<float>(c.m_hi * c.kappa_c);
        I.q31 = static_cast<float>((F(z3) - F(z1)) / (z3 - z1));
        I.zb1 = static_cast<float>(z1 - c.z_ref);
        I.f1 = static_cast<float>(F(z1));
    }
    P.invp_a = static_cast<float>(c.invp_a);
    P.invp_b = static_cast<float>(c.invp_b);
    P.ext_tol = static_cast<float>(c.ext_tol);
    P.chi2x_max = static_cast<float>(c.chi2x_max);
    P.inv_sx2 = static_cast<float>(1.0 / (c.sigma_x * c.sigma_x));
    P.w_chi2 = static_cast<float>(c.score_w_chi2);
    P.w5 = static_cast<float>(c.score_w5);
    // least-squares gain G = (Phi^T Phi)^-1 Phi^T per x-hit pattern with one
    // or no missing layer; basis (1, zb, f), solved in metres for conditioning
    for (int m = 0; m < 64; ++m) P.mask_index[m] = -1;
    for (int mi = 0; mi < kMasks; ++mi) {
        const int missing = mi < 6 ? mi : -1;
        const double sc[3] = {1.0, 1e-3, 1e-9};
        double N[3][3] = {{0}}, R[3][6] = {{0}};
        for (int s = 0; s < 6; ++s) {
            if (s == missing) continue;
            const double z = c.z[kXL[s]];
            const double phi[3] = {sc[0], (z - c.z_ref) * sc[1], F(z) * sc[2]};
            for (int a = 0; a < 3; ++a) {
                R[a][s] = phi[a];
                for (int b = 0; b < 3; ++b) N[a][b] += phi[a] * phi[b];
            }
        }
        if (!gauss_jordan(3, N, R, 6)) return fail("singular x-z fit");
        for (int a = 0; a < 3; ++a)
            for (int s = 0; s < 6; ++s) P.G[mi][a][s] = static_cast<float>(R[a][s] * sc[a]);
        P.mask_index[missing < 0 ? 63 : (63 ^ (1 << missing))] = mi;
    }
    for (int p = 0; p < 2; ++p) {
        const int u = uslot(c.uv_init[p]);
        if (u < 0) return fail("uv_init must name stereo layers");
        P.uv_init[p] = u;
        int q = 0;
        for (int v = 0; v < 6; ++v)
            if (v != u) P.uv_rem[p][q++] = v;
    }
    P.n_uv_min = c.n_uv_min;
    P.uv_tol = static_cast<float>(c.uv_tol);
    P.uv_ylo[0] = static_cast<float>(-c.uv_y_max);
    P.uv_yhi[0] = static_cast<float>(c.uv_y_overlap);
    P.uv_ylo[1] = static_cast<float>(-c.uv_y_overlap);
    P.uv_yhi[1] = static_cast<float>(c.uv_y_max);
    P.inv_sy2 = static_cast<float>(1.0 / (c.sigma_y * c.sigma_y));
    P.uv_mode = c.uv_mode;
    P.h_bins = c.hough_bins;
    P.h_fine = c.hough_fine;
    P.h_clusters = c.hough_clusters;
    {
        const double w = (c.hough_ty_max + c.hough_ty_in) / c.hough_bins;
        P.h_lo[0] = static_cast<float>(-c.hough_ty_max);
        P.h_lo[1] = static_cast<float>(-c.hough_ty_in);
        P.h_w = static_cast<float>(w);
        P.h_inv_w = static_cast<float>(1.0 / w);
        P.h_step = static_cast<float>(2.0 / c.hough_fine);
    }
    {
        const double zb = c.z_state - c.z_ref;
        P.zS = static_cast<float>(c.z_state);
        P.zbS = static_cast<float>(zb);
        P.fS = static_cast<float>(F(c.z_state));
        P.dfS = static_cast<float>(2.0 * zb + 3.0 * c.d_ratio * zb * zb);
    }
    P.zV = static_cast<float>(c.z_velo);
    P.zMY = static_cast<float>(c.z_match_y);
    split(c.zmx[0], P.A_hi, P.A_lo);
    P.Bx = static_cast<float>(c.zmx[1]);
    P.Cx = static_cast<float>(c.zmx[2]);
    P.Dx = static_cast<float>(c.zmx[3]);
    P.Ex = static_cast<float>(c.zmx[4]);
    split(c.zmx[0] - c.z_velo, P.dAV_hi, P.dAV_lo);
    split(c.zmx[0] - c.z_state, P.dAS_hi, P.dAS_lo);
    split(c.z_match_y - c.z_velo, P.dMV_hi, P.dMV_lo);
    split(c.z_match_y - c.z_state, P.dMS_hi, P.dMS_lo);
    const double ps = c.presel_scale, ts = c.tol_scale;
    if (!(ps > 0) || !(ts > 0)) return fail("presel_scale and tol_scale must be positive");
    P.cut_x = static_cast<float>(c.presel[0] * ps);
    P.cut_y = static_cast<float>(c.presel[1] * ps);
    P.cut_tx = static_cast<float>(c.presel[2] * ps);
    P.cut_ty = static_cast<float>(c.presel[3] * ps);
    P.tolx_a = static_cast<float>(ts * c.tolx[0] * c.tolx[1] * c.tolx[1]);
    P.tolx_b = static_cast<float>(ts * c.tolx[0] * c.tolx[2] * c.tolx[2]);
    P.toly_a = static_cast<float>(ts * c.toly[0] * c.toly[1] * c.toly[1]);
    P.toly_b = static_cast<float>(ts * c.toly[0] * c.toly[2] * c.toly[2]);
    P.inv_toltx = static_cast<float>(1.0 / (ts * c.tol_tx));
    P.inv_tolty = static_cast<float>(1.0 / (ts * c.tol_ty));
    P.chi2m_max = static_cast<float>(c.chi2_match_max);
    P.velo_unique = c.velo_unique ? 1 : 0;
    P.final_sel = c.final_sel;
    P.ghost_max = static_cast<float>(c.ghost_max);
    P.clone_margin = static_cast<float>(c.clone_margin);
    for (int l = 0; l < 12; ++l) {
        P.zl[l] = static_cast<float>(c.z[l]);
        P.tl[l] = static_cast<float>(c.dxdy[l]);
    }
    for (int zn = 0; zn < 24; ++zn) {
        const int L = zn >> 1, h = zn & 1;
        P.slot_of_zone[zn] = 12 * h + (xslot(L) >= 0 ? xslot(L) : 6 + uslot(L));
    }
    return true;
}

// ---------------------------------------------------------------------------
// workspace: one scratch arena and its launch shapes
// ---------------------------------------------------------------------------

struct Workspace {
    char* base = nullptr;
    size_t bytes = 0;
    // capacity
    int64_t cap_events = -1, cap_hits = -1, cap_seeds = -1;
    int32_t cap_max_hits = -1;
    int build_ctas = 0, seed_ctas = 0;  // CTAs the per-CTA scratch is sized for
    // carved pointers
    // [0] build, [1] seed, [2] match queues; fused matching: [3] announced, [4] fault,
    // [5] claimed, [6] done; [16, 144) item classes, [144, 272) their fill
    int32_t* queues = nullptr;
    unsigned long long* pool_ctr = nullptr;
    float* cx = nullptr;
    int32_t* corig = nullptr;
    int32_t* zoff = nullptr;
    uint8_t* big = nullptr;
    int64_t big_stride = 0;
    uint8_t* slot = nullptr;
    int64_t slot_stride = 0;
    int32_t* pool_hits = nullptr;
    float* pool_params = nullptr;
    float* pool_state = nullptr;
    int8_t* pool_n = nullptr;
    int32_t* item_start = nullptr;
    int32_t* item_count = nullptr;
    int32_t* item_class = nullptr;
    int32_t* order = nullptr;
    int32_t* ev_done = nullptr;    // fused matching: [events] halves done, then [events] announced
    int32_t* pool_velo = nullptr;  // fused matching: per seed record
    float* pool_chi2 = nullptr;
};

struct Pipeline;

constexpr int64_t kDefaultWaitNs = 200000000;  // 200 ms

struct st_ctx {
    st_config cfg;
    DevParams P;
    int device = 0;
    int n_sms = 0;
    size_t smem_optin = 0;
    std::string err;
    unsigned long long* counters = nullptr;
    Workspace ws;
    int tbl_smem = 0, key_smem = 0, velo_smem = 0;
    size_t seed_smem = 0, match_smem = 0, build_smem_max = 0;
    int seed_bps = 0, match_bps = 0;
    Pipeline* pipe = nullptr;
    std::mutex pipe_mu;
    bool timing = false;
    bool has_nn = false;  // ghost network weights given
    int64_t wait_ns = kDefaultWaitNs;  // fused seeding kernel: longest wait for an announced event
    cudaEvent_t tev[4][2] = {};
    bool tused[4] = {};
};

struct st_graph {
    st_ctx* ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static int set_err(st_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

#define ST_CUDA(ctx, call)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return set_err(ctx, e_ == cudaErrorMemoryAllocation ? ST_ENOMEM : ST_ECUDA,       \
                           "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// kernel timing marks on the launch stream (only for the context's own workspace)
static void tmark(st_ctx* ctx, const Workspace& w, int k, int end, cudaStream_t s) {
    if (!ctx->timing || &w != &ctx->ws) return;
    // external: inside a stream capture the record becomes a graph node that
    // records the event on every launch of the graph
    cudaEventRecordWithFlags(ctx->tev[k][end], s, cudaEventRecordExternal);
    ctx->tused[k] = true;
}

// work queues, the pool counter and the item-class counts, zeroed per launch
constexpr size_t kQueueBytes = 64 + 2 * 128 * sizeof(int32_t);
constexpr int kBuildSmemHits = 6144;  // larger events keep their per-hit arrays in scratch
constexpr int kBuildCtasPerSm = 8;

// buckets per container slot for a batch: about four hits per bucket (the
// rank sort inside a bucket is quadratic but tiny; fewer buckets mean less
// to clear and scan per event)
static int bins_for(int64_t n_events, int64_t n_hits) {
    const double avg = n_events > 0 ? double(n_hits) / double(n_events) : 0.0;
    int b = 8;
    while (b < 512 && b * 96 < avg) b <<= 1;
    return b;
}

// Arena layout for the given capacities; assigns pointers if `base`.
static size_t carve(st_ctx* ctx, Workspace& w, int64_t ne, int64_t nh, int32_t mh, int64_t sc, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += al256(bytes);
        return base ? base + o : nullptr;
    };
    const int build_ctas = ctx->n_sms * kBuildCtasPerSm;
    const int seed_ctas = ctx->n_sms * std::max(1, ctx->seed_bps);
    const int64_t items = 2 * ne;
    char* q = take(kQueueBytes);
    char* cx = take(sizeof(float) * size_t(nh + 3 * ne + 8));
    char* co = take(sizeof(int32_t) * size_t(nh + 3 * ne + 8));
    char* zo = take(sizeof(int32_t) * size_t(ne) * kZoffStride + 4);
    const int64_t big_stride = mh > kBuildSmemHits ? int64_t(al256(size_t(10) * mh)) : 0;
    char* big = take(size_t(big_stride) * build_ctas + 16);
    const int64_t slot_stride = int64_t(al256(seed_slot_bytes(ctx->cfg.cand_cap, mh)));
    char* slot = take(size_t(slot_stride) * seed_ctas);
    char* ph = take(sizeof(int32_t) * 12 * size_t(sc) + 4);
    char* pp = take(sizeof(float) * 8 * size_t(sc) + 4);
    char* pst = take(sizeof(float) * 4 * size_t(sc) + 4);
    char* pn = take(2 * size_t(sc) + 4);
    char* is = take(sizeof(int32_t) * size_t(items) + 4);
    char* ic = take(sizeof(int32_t) * size_t(items) + 4);
    char* icl = take(sizeof(int32_t) * size_t(items) + 4);
    char* ord = take(sizeof(int32_t) * size_t(items) + 4);
    char* evd = take(sizeof(int32_t) * size_t(items) + 4);
    char* pv = take(sizeof(int32_t) * size_t(sc) + 4);
    char* pc = take(sizeof(float) * size_t(sc) + 4);
    if (base) {
        w.queues = reinterpret_cast<int32_t*>(q);
        w.pool_ctr = reinterpret_cast<unsigned long long*>(q + 32);
        w.cx = reinterpret_cast<float*>(cx);
        w.corig = reinterpret_cast<int32_t*>(co);
        w.zoff = reinterpret_cast<int32_t*>(zo);
        w.big = reinterpret_cast<uint8_t*>(big);
        w.big_stride = big_stride;
        w.slot = reinterpret_cast<uint8_t*>(slot);
        w.slot_stride = slot_stride;
        w.pool_hits = reinterpret_cast<int32_t*>(ph);
        w.pool_params = reinterpret_cast<float*>(pp);
        w.pool_state = reinterpret_cast<float*>(pst);
        w.pool_n = reinterpret_cast<int8_t*>(pn);
        w.item_start = reinterpret_cast<int32_t*>(is);
        w.item_count = reinterpret_cast<int32_t*>(ic);
        w.item_class = reinterpret_cast<int32_t*>(icl);
        w.order = reinterpret_cast<int32_t*>(ord);
        w.ev_done = reinterpret_cast<int32_t*>(evd);
        w.pool_velo = reinterpret_cast<int32_t*>(pv);
        w.pool_chi2 = reinterpret_cast<float*>(pc);
        w.cap_events = ne;
        w.cap_hits = nh;
        w.cap_max_hits = mh;
        w.cap_seeds = sc;
        w.build_ctas = build_ctas;
        w.seed_ctas = seed_ctas;
    }
    return off;
}

// Make sure `w` can run a batch of this shape; (re)allocates if allowed.
static int ensure(st_ctx* ctx, Workspace& w, int64_t ne, int64_t nh, int32_t mh, int64_t sc, bool may_alloc) {
    if (w.base && ne <= w.cap_events && nh <= w.cap_hits && mh <= w.cap_max_hits && sc <= w.cap_seeds)
        return ST_OK;
    if (!may_alloc)
        return set_err(ctx, ST_ESTATE, "scratch too small for this batch during graph capture; call st_reserve first");
    ne = std::max(ne, w.cap_events);
    nh = std::max(nh, w.cap_hits);
    mh = std::max(mh, w.cap_max_hits);
    sc = std::max(sc, w.cap_seeds);
    const size_t need = carve(ctx, w, ne, nh, mh, sc, nullptr);
    if (w.base) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return set_err(ctx, ST_ECUDA, "cudaDeviceSynchronize: %s", cudaGetErrorString(e));
        cudaFree(w.base);
        w = Workspace();
    }
    char* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) return set_err(ctx, ST_ENOMEM, "cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
    w.base = p;
    w.bytes = need;
    carve(ctx, w, ne, nh, mh, sc, p);
    return ST_OK;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

extern "C" int st_create(const st_config* cfg, int device, st_ctx** out) {
    if (!cfg || !out) return ST_EINVAL;
    *out = nullptr;
    st_ctx* ctx = new (std::nothrow) st_ctx();
    if (!ctx) return ST_ENOMEM;
    ctx->cfg = *cfg;
    std::string err;
    if (!derive_params(*cfg, ctx->P, err)) {
        delete ctx;
        return ST_EINVAL;
    }
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sms, cudaDevAttrMultiProcessorCount, device);
    int optin = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) {
        delete ctx;
        return ST_ECUDA;
    }
    ctx->smem_optin = optin;
    const st_config& c = *cfg;
    ctx->tbl_smem = c.smem_hits / 2;
    ctx->key_smem = std::max(64, c.smem_hits / 8);  // kept seeds whose UV keys and stereo x stay in shared memory
    ctx->velo_smem = 512;
    ctx->seed_smem = seed_smem_bytes(c.threads_seed, c.smem_hits, ctx->tbl_smem, ctx->key_smem);
    ctx->match_smem = match_smem_bytes(ctx->velo_smem);
    ctx->build_smem_max = build_smem_bytes(512, kBuildSmemHits);
    // 2 KB of margin for the kernels' static shared memory
    if (ctx->seed_smem + 2048 > ctx->smem_optin || ctx->build_smem_max + 2048 > ctx->smem_optin) {
        delete ctx;
        return ST_EINVAL;
    }
    // a permission ceiling, not a reservation: set it to the device maximum so
    // that contexts with different configurations never lower each other's
    e = set_smem_limits(ctx->smem_optin);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->counters, sizeof(unsigned long long) * C_N);
    if (e == cudaSuccess) e = cudaMemset(ctx->counters, 0, sizeof(unsigned long long) * C_N);
    if (e != cudaSuccess) {
        if (ctx->counters) cudaFree(ctx->counters);
        delete ctx;
        return ST_ECUDA;
    }
    ctx->seed_bps = seed_blocks_per_sm(c.threads_seed, ctx->seed_smem);
    ctx->match_bps = match_blocks_per_sm(c.threads_match, ctx->match_smem);
    *out = ctx;
    return ST_OK;
}

static void pipeline_shutdown(st_ctx* ctx);

extern "C" void st_destroy(st_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    pipeline_shutdown(ctx);
    cudaDeviceSynchronize();
    if (ctx->ws.base) cudaFree(ctx->ws.base);
    if (ctx->counters) cudaFree(ctx->counters);
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < 2; ++j)
            if (ctx->tev[k][j]) cudaEventDestroy(ctx->tev[k][j]);
    delete ctx;
}

extern "C" const char* st_last_error(const st_ctx* ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" int st_reserve(st_ctx* ctx, int64_t n_events, int64_t n_hits, int32_t max_hits, int64_t seeds_cap) {
    if (!ctx) return ST_EINVAL;
    if (n_events < 0 || n_hits < 0 || max_hits < 1 || max_hits > 65535 || seeds_cap < 0 || seeds_cap > INT32_MAX)
        return set_err(ctx, ST_EINVAL, "st_reserve: bad sizes");
    ST_CUDA(ctx, cudaSetDevice(ctx->device));
    return ensure(ctx, ctx->ws, n_events, n_hits, max_hits, seeds_cap, true);
}

// ---------------------------------------------------------------------------
// seeding / matching
// ---------------------------------------------------------------------------

// With V and L (fused): the seeding kernel also matches each event once its
// two halves are done, and the gather writes the Long tracks too.
static int run_seeding(st_ctx* ctx, Workspace& w, const st_hits& H, st_seeds& S, cudaStream_t s,
                       int64_t n_hits_total, bool may_alloc, const st_velo* V = nullptr, st_long* L = nullptr,
                       bool defer = false) {
    int rc = ensure(ctx, w, H.n_events, n_hits_total, H.max_hits_per_event, S.cap, may_alloc);
    if (rc != ST_OK) return rc;
    const st_config& c = ctx->cfg;
    const int bins = bins_for(H.n_events, n_hits_total);
    const int build_cap = std::min<int>(H.max_hits_per_event, kBuildSmemHits);
    int bbps = std::max(1, build_blocks_per_sm(c.threads_build, build_smem_bytes(bins, build_cap)));
    if (c.ctas_per_sm > 0) bbps = std::min(bbps, c.ctas_per_sm);
    const int g_build = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>({H.n_events, int64_t(ctx->n_sms) * bbps, int64_t(w.build_ctas)})));
    int sbps = std::max(1, ctx->seed_bps);
    if (c.ctas_per_sm > 0) sbps = std::min(sbps, c.ctas_per_sm);
    const int g_seed = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>({2 * H.n_events, int64_t(ctx->n_sms) * sbps, int64_t(w.seed_ctas)})));
    ST_CUDA(ctx, cudaMemsetAsync(w.queues, 0, kQueueBytes, s));
    if (H.n_events == 0) {
        ST_CUDA(ctx, cudaMemsetAsync(S.ev_off, 0, sizeof(int32_t), s));
        return ST_OK;
    }
    const bool fused = V && L;
    BuildArgs b;
    b.n_events = H.n_events;
    b.ev_off = H.ev_off;
    b.x = H.x;
    b.zone = H.zone;
    b.z = H.z;
    b.dxdy = H.dxdy;
    b.max_hits = H.max_hits_per_event;
    b.bins = bins;
    b.smem_hits = build_cap;
    b.cont_cap = w.cap_hits + 3 * w.cap_events + 8;
    b.cx = w.cx;
    b.corig = w.corig;
    b.zoff = w.zoff;
    b.status = S.status;
    b.big = w.big;
    b.big_stride = w.big_stride;
    b.item_class = w.item_class;
    b.class_count = w.queues + 16;
    b.class_fill = w.queues + 16 + 128;
    b.order = w.order;
    b.zero2 = fused ? w.ev_done : nullptr;  // halves done + announcements, cleared before k_seed
    b.queue = w.queues + 0;
    b.counters = ctx->counters;
    // k_order, the seeding kernel and the scan follow their predecessors as
    // programmatic dependents on the context's own workspace, except where
    // timing marks come between.  Not on the serving pipeline's slot
    // streams: CTAs waiting there for their predecessor hold SMs that the
    // other slots' kernels could use (measured: 24% less served throughput
    // at saturation).
    const bool marks = ctx->timing && &w == &ctx->ws;
    const bool chain = &w == &ctx->ws;
    tmark(ctx, w, 0, 0, s);
    ST_CUDA(ctx, launch_build(ctx->P, b, g_build, c.threads_build, s, chain));
    tmark(ctx, w, 0, 1, s);

    SeedArgs a;
    a.n_events = H.n_events;
    a.ev_off = H.ev_off;
    a.cx = w.cx;
    a.corig = w.corig;
    a.zoff = w.zoff;
    a.status = S.status;
    a.smem_hits = ctx->cfg.smem_hits;
    a.cand_cap = ctx->cfg.cand_cap;
    a.tbl_smem = ctx->tbl_smem;
    a.key_smem = ctx->key_smem;
    a.slot = w.slot;
    a.slot_stride = w.slot_stride;
    a.max_xhits = w.cap_max_hits;
    a.pool_hits = w.pool_hits;
    a.pool_params = w.pool_params;
    a.pool_state = w.pool_state;
    a.pool_n = w.pool_n;
    a.pool_cap = S.cap;
    a.pool_ctr = w.pool_ctr;
    a.item_start = w.item_start;
    a.item_count = w.item_count;
    a.order = w.order;
    a.queue = w.queues + 1;
    a.counters = ctx->counters;
    a.fault = w.queues + 4;  // a wait that gave up (staging copy, announced event)
    if (fused) {
        a.velo_off = V->ev_off;
        a.velo = V->state;
        a.velo_smem = ctx->velo_smem;
        a.defer_match = defer ? 1 : 0;
        a.ev_done = w.ev_done;
        a.ready = w.ev_done + H.n_events;
        a.ready_ctr = w.queues + 3;
        a.wait_ns = static_cast<unsigned long long>(ctx->wait_ns);
        a.m_claim = w.queues + 5;
        a.done_ctr = w.queues + 6;
        a.pool_velo = w.pool_velo;
        a.pool_chi2 = w.pool_chi2;
        a.n_long = L->n_long;
        if (ctx->timing && &w == &ctx->ws) ctx->tused[3] = false;  // matching runs inside k_seed
    }
    tmark(ctx, w, 1, 0, s);
    ST_CUDA(ctx, launch_seed(ctx->P, a, g_seed, c.threads_seed, s, chain && !marks));
    tmark(ctx, w, 1, 1, s);

    GatherArgs g;
    g.n_events = H.n_events;
    g.item_start = w.item_start;
    g.item_count = w.item_count;
    g.pool_hits = w.pool_hits;
    g.pool_params = w.pool_params;
    g.pool_state = w.pool_state;
    g.pool_n = w.pool_n;
    g.cap = S.cap;
    g.ev_off = S.ev_off;
    g.hits = S.hits;
    g.params = S.params;
    g.state = S.state;
    g.n_hits = S.n_hits;
    g.status = S.status;
    g.fault = w.queues + 4;
    if (fused) {
        g.pool_velo = w.pool_velo;
        g.pool_chi2 = w.pool_chi2;
        g.velo_idx = L->velo_idx;
        g.chi2 = L->chi2;
    }
    tmark(ctx, w, 2, 0, s);
    ST_CUDA(ctx, launch_gather(g, s, chain && !marks));
    tmark(ctx, w, 2, 1, s);
    return ST_OK;
}

static int run_matching(st_ctx* ctx, Workspace& w, const st_velo& V, const st_seeds& S, st_long& L,
                        cudaStream_t s) {
    if (V.n_events == 0) return ST_OK;
    if (!w.base) return set_err(ctx, ST_ESTATE, "matching_run before any seeding_run on this context");
    ST_CUDA(ctx, cudaMemsetAsync(w.queues + 2, 0, sizeof(int32_t), s));
    MatchArgs m;
    m.n_events = V.n_events;
    m.velo_off = V.ev_off;
    m.velo = V.state;
    m.seed_off = S.ev_off;
    m.seed_state = S.state;
    if (ctx->cfg.final_sel && !ctx->has_nn)
        return set_err(ctx, ST_ESTATE, "final_sel needs the ghost network weights (st_set_ghost_nn)");
    if (ctx->cfg.final_sel && !L.ghost_prob)
        return set_err(ctx, ST_EINVAL, "final_sel needs an st_long.ghost_prob array");
    m.velo_idx = L.velo_idx;
    m.chi2 = L.chi2;
    m.n_long = L.n_long;
    m.seed_n = S.n_hits;
    m.ghost_prob = L.ghost_prob;
    m.velo_smem = ctx->velo_smem;
    m.queue = w.queues + 2;
    m.counters = ctx->counters;
    int mbps = std::max(1, ctx->match_bps);
    if (ctx->cfg.ctas_per_sm > 0) mbps = std::min(mbps, ctx->cfg.ctas_per_sm);
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(V.n_events, int64_t(ctx->n_sms) * mbps)));
    tmark(ctx, w, 3, 0, s);
    ST_CUDA(ctx, launch_match(ctx->P, m, grid, ctx->cfg.threads_match, s));
    tmark(ctx, w, 3, 1, s);
    return ST_OK;
}

// Seeding then matching of one batch.  The fused kernel (matching inside the
// seeding kernel) serves the HLT1 configuration with 256-thread seeding CTAs
// and no final selection; every other configuration runs the two steps apart.
static bool fusable(const st_ctx* ctx, const st_hits& H, const st_velo& V) {
    const st_config& c = ctx->cfg;
    return c.threads_seed <= 256 && c.iter_mode == 0 && !c.final_sel && V.n_events == H.n_events &&
           match_smem_bytes(ctx->velo_smem) <= ctx->seed_smem;
}

// defer: the kernel has the GPU to itself (a graph replay), so CTAs without
// seeding work may wait for the last events (see k_seed).
static int run_batch(st_ctx* ctx, Workspace& w, const st_hits& H, st_seeds& S, const st_velo& V, st_long& L,
                     cudaStream_t s, int64_t n_hits_total, bool may_alloc, bool defer) {
    if (fusable(ctx, H, V)) return run_seeding(ctx, w, H, S, s, n_hits_total, may_alloc, &V, &L, defer);
    int rc = run_seeding(ctx, w, H, S, s, n_hits_total, may_alloc);
    if (rc == ST_OK) rc = run_matching(ctx, w, V, S, L, s);
    return rc;
}

static int check_hits(st_ctx* ctx, const st_hits* h) {
    if (!h || h->n_events < 0 || (h->n_events > 0 && (!h->ev_off || !h->x || !h->zone)))
        return set_err(ctx, ST_EINVAL, "st_hits: null array or negative n_events");
    if (h->max_hits_per_event < 1 || h->max_hits_per_event > 65535)
        return set_err(ctx, ST_EINVAL, "st_hits: max_hits_per_event must be in [1, 65535]");
    if (h->n_events > (int64_t(1) << 30)) return set_err(ctx, ST_EINVAL, "st_hits: too many events");
    return ST_OK;
}

static int check_seeds(st_ctx* ctx, const st_seeds* s) {
    if (!s || s->cap < 0 || s->cap > INT32_MAX || !s->ev_off || !s->status ||
        (s->cap > 0 && (!s->hits || !s->params || !s->state || !s->n_hits)))
        return set_err(ctx, ST_EINVAL, "st_seeds: null array or bad cap");
    return ST_OK;
}

extern "C" int seeding_run(st_ctx* ctx, const st_hits* hits, st_seeds* seeds, void* stream) {
    if (!ctx) return ST_EINVAL;
    int rc = check_hits(ctx, hits);
    if (rc) return rc;
    if ((rc = check_seeds(ctx, seeds))) return rc;
    ST_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    ST_CUDA(ctx, cudaStreamIsCapturing(s, &cs));
    // the hit total is only known on the device: size the containers by the
    // bound n_events * max_hits_per_event
    const int64_t use = hits->n_events * int64_t(hits->max_hits_per_event);
    return run_seeding(ctx, ctx->ws, *hits, *seeds, s, use, cs == cudaStreamCaptureStatusNone);
}

extern "C" int matching_run(st_ctx* ctx, const st_velo* velo, const st_seeds* seeds, st_long* out, void* stream) {
    if (!ctx) return ST_EINVAL;
    if (!velo || velo->n_events < 0 || (velo->n_events > 0 && (!velo->ev_off || !velo->state)))
        return set_err(ctx, ST_EINVAL, "st_velo: null array or negative n_events");
    if (!seeds || !seeds->ev_off || !seeds->state || !out || !out->velo_idx || !out->chi2)
        return set_err(ctx, ST_EINVAL, "matching_run: null seeds or output array");
    ST_CUDA(ctx, cudaSetDevice(ctx->device));
    return run_matching(ctx, ctx->ws, *velo, *seeds, *out, static_cast<cudaStream_t>(stream));
}

extern "C" int ut_run(st_ctx* ctx, const st_velo* velo, const st_seeds* seeds, const st_ut_hits* ut, st_long* out,
                      st_ut_out* uo, void* stream) {
    if (!ctx) return ST_EINVAL;
    if (!velo || !seeds || !ut || !out || !uo || !seeds->ev_off || !seeds->state || !seeds->status ||
        !out->velo_idx || !out->chi2 || !uo->hits || !uo->n_hits || !uo->gamma)
        return set_err(ctx, ST_EINVAL, "ut_run: null argument or array");
    if (ut->n_events != velo->n_events || ut->n_events < 0 ||
        (ut->n_events > 0 && (!ut->ev_off || !ut->x || !ut->layer || !velo->ev_off || !velo->state)))
        return set_err(ctx, ST_EINVAL, "ut_run: event counts differ or null hit arrays");
    if (ut->n_events == 0) return ST_OK;
    ST_CUDA(ctx, cudaSetDevice(ctx->device));
    const st_config& c = ctx->cfg;
    UtParams U;
    U.z_velo = static_cast<float>(c.z_velo);
    for (int l = 0; l < 4; ++l) {
        const double dz = c.ut_z[l] - c.z_velo;
        U.dz[l] = static_cast<float>(dz);
        U.dz2[l] = static_cast<float>(dz * dz);
        U.t[l] = static_cast<float>(c.ut_dxdy[l]);
    }
    U.gA = static_cast<float>(c.ut_gamma[0]);
    U.gB = static_cast<float>(c.ut_gamma[1]);
    U.inv_kick = static_cast<float>(1.0 / c.ut_kick);
    for (int k = 0; k < 16; ++k) {
        U.loose[k] = static_cast<float>(c.ut_loose[k]);
        U.tight[k] = static_cast<float>(c.ut_tight[k]);
    }
    U.min_hits = c.ut_min_hits;
    UtArgs a;
    a.n_events = ut->n_events;
    a.ut_off = ut->ev_off;
    a.ut_x = ut->x;
    a.ut_layer = ut->layer;
    a.velo_off = velo->ev_off;
    a.velo = velo->state;
    a.seed_off = seeds->ev_off;
    a.seed_state = seeds->state;
    a.velo_idx = out->velo_idx;
    a.chi2 = out->chi2;
    a.n_long = out->n_long;
    a.status = seeds->status;
    a.ut_hits = uo->hits;
    a.ut_n = uo->n_hits;
    a.gamma = uo->gamma;
    const int grid = static_cast<int>(std::min<int64_t>(ut->n_events, int64_t(ctx->n_sms) * 6));
    ST_CUDA(ctx, launch_ut(U, a, grid, static_cast<cudaStream_t>(stream)));
    return ST_OK;
}

extern "C" int st_set_ghost_nn(st_ctx* ctx, const float* weights, int32_t n) {
    if (!ctx) return ST_EINVAL;
    if (!weights || n != ST_GHOST_NN_SIZE)
        return set_err(ctx, ST_EINVAL, "st_set_ghost_nn: expected %d weights", ST_GHOST_NN_SIZE);
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(weights[i])) return set_err(ctx, ST_EINVAL, "st_set_ghost_nn: weight %d not finite", i);
    std::memcpy(ctx->P.nn, weights, sizeof(float) * ST_GHOST_NN_SIZE);
    ctx->has_nn = true;
    return ST_OK;
}

extern "C" int st_set_timing(st_ctx* ctx, int enable) {
    if (!ctx) return ST_EINVAL;
    ST_CUDA(ctx, cudaSetDevice(ctx->device));
    if (enable && !ctx->tev[0][0]) {
        for (int k = 0; k < 4; ++k)
            for (int j = 0; j < 2; ++j) ST_CUDA(ctx, cudaEventCreate(&ctx->tev[k][j]));
    }
    ctx->timing = enable != 0;
    for (int k = 0; k < 4; ++k) ctx->tused[k] = false;
    return ST_OK;
}

extern "C" int st_set_wait_limit(st_ctx* ctx, int64_t ns) {
    if (!ctx) return ST_EINVAL;
    if (ns < 0) return set_err(ctx, ST_EINVAL, "st_set_wait_limit: negative limit %lld", (long long)ns);
    ctx->wait_ns = ns;
    return ST_OK;
}

extern "C" int st_kernel_ms(st_ctx* ctx, float ms[4]) {
    if (!ctx || !ms) return ST_EINVAL;
    ST_CUDA(ctx, cudaSetDevice(ctx->device));
    for (int k = 0; k < 4; ++k) {
        ms[k] = 0.f;
        if (!ctx->timing || !ctx->tused[k]) continue;
        ST_CUDA(ctx, cudaEventSynchronize(ctx->tev[k][1]));
        ST_CUDA(ctx, cudaEventElapsedTime(&ms[k], ctx->tev[k][0], ctx->tev[k][1]));
    }
    return ST_OK;
}

extern "C" int st_read_counters(st_ctx* ctx, st_counters* out, int reset) {
    if (!ctx || !out) return ST_EINVAL;
    ST_CUDA(ctx, cudaSetDevice(ctx->device));
    ST_CUDA(ctx, cudaDeviceSynchronize());
    unsigned long long h[C_N];
    ST_CUDA(ctx, cudaMemcpy(h, ctx->counters, sizeof(h), cudaMemcpyDeviceToHost));
    int64_t* o = reinterpret_cast<int64_t*>(out);
    for (int k = 0; k < C_N; ++k) o[k] = static_cast<int64_t>(h[k]);
    if (reset) ST_CUDA(ctx, cudaMemset(ctx->counters, 0, sizeof(h)));
    return ST_OK;
}

// ---------------------------------------------------------------------------
// CUDA graph of one batch
// ---------------------------------------------------------------------------

extern "C" int st_graph_create(st_ctx* ctx, const st_hits* hits, const st_velo* velo, st_seeds* seeds,
                               st_long* out, st_graph** graph) {
    if (!ctx || !graph) return ST_EINVAL;
    *graph = nullptr;
    int rc = check_hits(ctx, hits);
    if (rc) return rc;
    if ((rc = check_seeds(ctx, seeds))) return rc;
    if (!velo || !out || !out->velo_idx || !out->chi2) return set_err(ctx, ST_EINVAL, "st_graph_create: null argument");
    if (velo->n_events != hits->n_events) return set_err(ctx, ST_EINVAL, "hits and velo event counts differ");
    ST_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t bound = hits->n_events * int64_t(hits->max_hits_per_event);
    rc = ensure(ctx, ctx->ws, hits->n_events, bound, hits->max_hits_per_event, seeds->cap, true);
    if (rc) return rc;
    cudaStream_t cs;
    ST_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    st_graph* g = new st_graph();
    g->ctx = ctx;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = run_batch(ctx, ctx->ws, *hits, *seeds, *velo, *out, cs, bound, false, true);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
        if (rc == ST_OK && e2 != cudaSuccess) rc = set_err(ctx, ST_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
        if (rc == ST_OK) {
            e2 = cudaGraphInstantiate(&g->exec, g->graph, 0);
            if (e2 != cudaSuccess) rc = set_err(ctx, ST_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e2));
        }
    } else {
        rc = set_err(ctx, ST_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    cudaStreamDestroy(cs);
    if (rc != ST_OK) {
        st_graph_destroy(g);
        return rc;
    }
    *graph = g;
    return ST_OK;
}

extern "C" int st_graph_launch(st_graph* g, void* stream) {
    if (!g || !g->exec) return ST_EINVAL;
    ST_CUDA(g->ctx, cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
    return ST_OK;
}

extern "C" void st_graph_destroy(st_graph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

// ---------------------------------------------------------------------------
// serving pipeline
// ---------------------------------------------------------------------------
// What the pipeline keeps between calls lives in device memory:
//  * input rings (hits: x and zone side by side; VELO states), filled by DMA
//    straight from the caller's memory inside pipeline_submit;
//  * an output ring, one block per launch, written by the kernels and read
//    by DMA straight into the caller's memory inside pipeline_poll.
// The host never copies event data.  A dispatcher thread packs waiting
// requests that follow each other in the input rings into one launch on a
// free slot (stream + workspace); a completer thread retires launches in
// order.

// FIFO ring allocator over `cap` units; blocks are released by id in any
// order and their space is reclaimed from the oldest block on.  Blocks are
// exact (no padding), so consecutive blocks are contiguous unless the ring
// wrapped.  Zero-size blocks take no space.
struct Ring {
    size_t cap = 0, head = 0;
    uint64_t next_id = 1;
    struct B {
        uint64_t id;
        size_t off, size;
        bool released;
    };
    std::deque<B> live;

    bool alloc(size_t n, size_t& off, uint64_t& id) {
        if (n > cap) return false;
        const B* oldest = nullptr;
        for (const auto& b : live)
            if (b.size > 0) {
                oldest = &b;
                break;
            }
        if (!oldest) {
            if (head + n > cap) head = 0;
            off = head;
        } else {
            const size_t tail = oldest->off;
            if (head > tail) {  // occupied: [tail, head)
                if (head + n <= cap) off = head;
                else if (n <= tail) off = 0;
                else return false;
            } else {            // occupied: [tail, cap) and [0, head)
                if (head + n <= tail) off = head;
                else return false;
            }
        }
        id = next_id++;
        live.push_back({id, off, n, false});
        head = off + n;
        return true;
    }
    void release(uint64_t id) {
        for (auto& b : live)
            if (b.id == id) {
                b.released = true;
                break;
            }
        while (!live.empty() && live.front().released) live.pop_front();
        if (live.empty()) head = 0;
    }
};

struct OutBlock {
    uint64_t ring_id = 0;
    int64_t events = 0, cap = 0;
    int refs = 0;
    int32_t *ev_off, *status, *n_long, *hits, *vidx;
    float *params, *state, *chi2, *gp;
    int8_t* n;
};

struct Request {
    uint64_t id = 0;
    int64_t n_events = 0, n_hits = 0, n_velo = 0;
    size_t h_off = 0, v_off = 0;           // offsets in the hit / VELO rings
    uint64_t h_id = 0, v_id = 0;           // ring blocks
    std::vector<int64_t> ev_off, velo_off;  // rebased to 0
    std::shared_ptr<OutBlock> out;         // results
    int64_t e0 = 0, s0 = 0, s1 = 0;
    int status = ST_PENDING;
    bool done = false;
    int64_t t_submit = 0, t_launch = 0, t_done = 0;
};

struct Slot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int64_t *d_ev_off = nullptr, *d_velo_off = nullptr;
    int64_t *h_ev_off = nullptr, *h_velo_off = nullptr;  // pinned
    int32_t* h_counts = nullptr;                          // pinned: the launch's seed offsets
    std::vector<std::shared_ptr<Request>> reqs;
    std::shared_ptr<OutBlock> out;
    int64_t n_events = 0;
    bool busy = false;
    int rc = ST_OK;
};

struct Pipeline {
    st_pipeline_config pc;
    std::vector<Slot> slots;
    Ring hr, vr, orr;  // hits, VELO states, outputs (bytes)
    float* d_x = nullptr;
    int32_t* d_zone = nullptr;
    float* d_velo = nullptr;
    char* d_out = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_space;
    std::deque<std::shared_ptr<Request>> pending;
    std::deque<int> launched;
    std::map<uint64_t, std::shared_ptr<Request>> all;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread dispatcher, completer;
    std::mutex in_mu, out_mu;  // serialise use of the two DMA streams
    cudaStream_t in_stream = nullptr, out_stream = nullptr;
};

extern "C" void st_pipeline_config_default(st_pipeline_config* pc) {
    if (!pc) return;
    pc->n_slots = 4;
    pc->max_events_per_slot = 4096;
    pc->max_hits_per_slot = 4096ll * 3000;
    pc->max_hits_per_event = 16384;
    pc->max_velo_per_event = 2048;
    pc->mem_cap_bytes = 40ll << 30;
    pc->max_velo_per_slot = 1ll << 20;
}

static int64_t out_cap_for(int64_t hits) { return std::max<int64_t>(1024, hits / 8); }

static size_t out_block_bytes(int64_t events, int64_t cap) {
    return al256(4 * size_t(events + 1)) + 2 * al256(4 * size_t(events)) + al256(48 * size_t(cap)) +
           al256(32 * size_t(cap)) + al256(16 * size_t(cap)) + al256(2 * size_t(cap)) + 3 * al256(4 * size_t(cap));
}

static void carve_out(OutBlock& o, char* p) {
    size_t k = 0;
    auto take = [&](size_t b) {
        char* r = p + k;
        k += al256(b);
        return r;
    };
    o.ev_off = reinterpret_cast<int32_t*>(take(4 * size_t(o.events + 1)));
    o.status = reinterpret_cast<int32_t*>(take(4 * size_t(o.events)));
    o.n_long = reinterpret_cast<int32_t*>(take(4 * size_t(o.events)));
    o.hits = reinterpret_cast<int32_t*>(take(48 * size_t(o.cap)));
    o.params = reinterpret_cast<float*>(take(32 * size_t(o.cap)));
    o.state = reinterpret_cast<float*>(take(16 * size_t(o.cap)));
    o.n = reinterpret_cast<int8_t*>(take(2 * size_t(o.cap)));
    o.vidx = reinterpret_cast<int32_t*>(take(4 * size_t(o.cap)));
    o.chi2 = reinterpret_cast<float*>(take(4 * size_t(o.cap)));
    o.gp = reinterpret_cast<float*>(take(4 * size_t(o.cap)));
}

static int slot_alloc(st_ctx* ctx, Slot& S, const st_pipeline_config& pc) {
    ST_CUDA(ctx, cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking));
    ST_CUDA(ctx, cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming));
    const int64_t E = pc.max_events_per_slot;
    ST_CUDA(ctx, cudaMalloc(&S.d_ev_off, 8 * (E + 1)));
    ST_CUDA(ctx, cudaMalloc(&S.d_velo_off, 8 * (E + 1)));
    ST_CUDA(ctx, cudaMallocHost(&S.h_ev_off, 8 * (E + 1)));
    ST_CUDA(ctx, cudaMallocHost(&S.h_velo_off, 8 * (E + 1)));
    ST_CUDA(ctx, cudaMallocHost(&S.h_counts, 4 * (E + 1)));
    return ensure(ctx, S.ws, E, pc.max_hits_per_slot, pc.max_hits_per_event, out_cap_for(pc.max_hits_per_slot), true);
}

static void slot_free(Slot& S) {
    if (S.stream) cudaStreamSynchronize(S.stream);
    if (S.d_ev_off) cudaFree(S.d_ev_off);
    if (S.d_velo_off) cudaFree(S.d_velo_off);
    if (S.ws.base) cudaFree(S.ws.base);
    if (S.h_ev_off) cudaFreeHost(S.h_ev_off);
    if (S.h_velo_off) cudaFreeHost(S.h_velo_off);
    if (S.h_counts) cudaFreeHost(S.h_counts);
    if (S.ev) cudaEventDestroy(S.ev);
    if (S.stream) cudaStreamDestroy(S.stream);
}

// Pack waiting requests into slot `si` and launch; called with the lock held.
static void launch_slot(st_ctx* ctx, Pipeline& pl, int si, std::unique_lock<std::mutex>& lk) {
    Slot& S = pl.slots[si];
    S.reqs.clear();
    int64_t ne = 0, nh = 0, nv = 0;
    size_t next_h = 0, next_v = 0;
    while (!pl.pending.empty()) {
        auto& r = pl.pending.front();
        if (!S.reqs.empty()) {
            // only a request that continues the previous one in both rings
            // extends the launch's CSR without gaps
            const bool contiguous = r->h_off == next_h && r->v_off == next_v;
            if (!contiguous || ne + r->n_events > pl.pc.max_events_per_slot ||
                nh + r->n_hits > pl.pc.max_hits_per_slot || nv + r->n_velo > pl.pc.max_velo_per_slot)
                break;
        }
        ne += r->n_events;
        nh += r->n_hits;
        nv += r->n_velo;
        next_h = r->h_off + size_t(r->n_hits);
        next_v = r->v_off + size_t(r->n_velo);
        S.reqs.push_back(r);
        pl.pending.pop_front();
    }
    auto ob = std::make_shared<OutBlock>();
    ob->events = ne;
    ob->cap = out_cap_for(std::max<int64_t>(nh, 1));
    size_t ob_off = 0;
    while (!pl.stop && !pl.orr.alloc(out_block_bytes(ne, ob->cap), ob_off, ob->ring_id)) pl.cv_space.wait(lk);
    if (pl.stop) {
        for (auto it = S.reqs.rbegin(); it != S.reqs.rend(); ++it) pl.pending.push_front(*it);
        S.reqs.clear();
        return;
    }
    carve_out(*ob, pl.d_out + ob_off);
    ob->refs = static_cast<int>(S.reqs.size());
    S.out = ob;
    S.busy = true;
    S.n_events = ne;
    lk.unlock();
    const int64_t t0 = now_ns();
    // the launch's CSR: absolute positions in the rings
    int64_t e = 0;
    S.h_ev_off[0] = int64_t(S.reqs.front()->h_off);
    S.h_velo_off[0] = int64_t(S.reqs.front()->v_off);
    for (auto& r : S.reqs) {
        r->t_launch = t0;
        r->e0 = e;
        r->out = ob;
        for (int64_t k = 0; k < r->n_events; ++k) {
            S.h_ev_off[e + k + 1] = int64_t(r->h_off) + r->ev_off[k + 1];
            S.h_velo_off[e + k + 1] = int64_t(r->v_off) + r->velo_off[k + 1];
        }
        e += r->n_events;
    }
    cudaStream_t st = S.stream;
    int rc = ST_OK;
    auto ck = [&](cudaError_t err) {
        if (err != cudaSuccess && rc == ST_OK) rc = set_err(nullptr, ST_ECUDA, "%s", cudaGetErrorString(err));
    };
    ck(cudaMemcpyAsync(S.d_ev_off, S.h_ev_off, 8 * (ne + 1), cudaMemcpyHostToDevice, st));
    ck(cudaMemcpyAsync(S.d_velo_off, S.h_velo_off, 8 * (ne + 1), cudaMemcpyHostToDevice, st));
    st_hits H{ne, S.d_ev_off, pl.d_x, pl.d_zone, nullptr, nullptr, pl.pc.max_hits_per_event, 0};
    st_seeds Sd{ob->cap, ob->ev_off, ob->hits, ob->params, ob->state, ob->n, ob->status};
    st_velo V{ne, S.d_velo_off, pl.d_velo};
    st_long L{ob->vidx, ob->chi2, ob->n_long, ob->gp};
    if (rc == ST_OK) rc = run_batch(ctx, S.ws, H, Sd, V, L, st, pl.pc.max_hits_per_slot, false, false);
    ck(cudaMemcpyAsync(S.h_counts, ob->ev_off, 4 * (ne + 1), cudaMemcpyDeviceToHost, st));
    ck(cudaEventRecord(S.ev, st));
    S.rc = rc;
    lk.lock();
    pl.launched.push_back(si);
    pl.cv_done.notify_all();
}

static void dispatcher_main(st_ctx* ctx, Pipeline* pl) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(pl->mu);
    for (;;) {
        pl->cv_work.wait(lk, [&] {
            if (pl->stop) return true;
            if (pl->pending.empty()) return false;
            for (auto& s : pl->slots)
                if (!s.busy) return true;
            return false;
        });
        if (pl->stop) return;
        int si = -1;
        for (size_t k = 0; k < pl->slots.size(); ++k)
            if (!pl->slots[k].busy) {
                si = static_cast<int>(k);
                break;
            }
        if (si >= 0) launch_slot(ctx, *pl, si, lk);
    }
}

static void completer_main(st_ctx* ctx, Pipeline* pl) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(pl->mu);
    for (;;) {
        pl->cv_done.wait(lk, [&] { return pl->stop || !pl->launched.empty(); });
        if (pl->launched.empty() && pl->stop) return;
        const int si = pl->launched.front();
        pl->launched.pop_front();
        Slot& S = pl->slots[si];
        lk.unlock();
        int rc = S.rc;
        if (cudaEventSynchronize(S.ev) != cudaSuccess && rc == ST_OK) rc = ST_ECUDA;
        const int64_t tdone = now_ns();
        lk.lock();
        for (auto& r : S.reqs) {
            r->s0 = rc == ST_OK ? S.h_counts[r->e0] : 0;
            r->s1 = rc == ST_OK ? S.h_counts[r->e0 + r->n_events] : 0;
            r->t_done = tdone;
            r->status = rc;
            r->done = true;
            // the inputs are no longer needed
            pl->hr.release(r->h_id);
            pl->vr.release(r->v_id);
        }
        S.reqs.clear();
        S.out.reset();
        S.busy = false;
        pl->cv_done.notify_all();
        pl->cv_work.notify_all();
        pl->cv_space.notify_all();
    }
}

static int pipeline_configure_locked(st_ctx* ctx, const st_pipeline_config* pcin);

static int pipeline_start(st_ctx* ctx) {
    std::lock_guard<std::mutex> g(ctx->pipe_mu);
    if (ctx->pipe) return ST_OK;
    st_pipeline_config pc;
    st_pipeline_config_default(&pc);
    return pipeline_configure_locked(ctx, &pc);
}

extern "C" int st_pipeline_configure(st_ctx* ctx, const st_pipeline_config* pcin) {
    if (!ctx || !pcin) return ST_EINVAL;
    std::lock_guard<std::mutex> g(ctx->pipe_mu);
    return pipeline_configure_locked(ctx, pcin);
}

static void pipeline_free(Pipeline* pl) {
    for (auto& S : pl->slots) slot_free(S);
    if (pl->d_x) cudaFree(pl->d_x);
    if (pl->d_zone) cudaFree(pl->d_zone);
    if (pl->d_velo) cudaFree(pl->d_velo);
    if (pl->d_out) cudaFree(pl->d_out);
    if (pl->in_stream) cudaStreamDestroy(pl->in_stream);
    if (pl->out_stream) cudaStreamDestroy(pl->out_stream);
    delete pl;
}

static int pipeline_configure_locked(st_ctx* ctx, const st_pipeline_config* pcin) {
    if (ctx->pipe) return set_err(ctx, ST_ESTATE, "pipeline already configured");
    st_pipeline_config pc = *pcin;
    if (pc.n_slots < 1 || pc.max_events_per_slot < 1 || pc.max_hits_per_slot < 1 || pc.max_hits_per_event < 1 ||
        pc.max_hits_per_event > 65535 || pc.max_velo_per_event < 1 || pc.mem_cap_bytes <= 0 ||
        pc.max_velo_per_slot < 1)
        return set_err(ctx, ST_EINVAL, "bad pipeline config");
    ST_CUDA(ctx, cudaSetDevice(ctx->device));
    // device memory: per slot a workspace; shared input rings holding two
    // slots' worth of hits and VELO states per slot; an output ring holding
    // two launches' worth of results per slot
    Workspace t;
    const int64_t ocap = out_cap_for(pc.max_hits_per_slot);
    const size_t ws_bytes = carve(ctx, t, pc.max_events_per_slot, pc.max_hits_per_slot, pc.max_hits_per_event,
                                  ocap, nullptr);
    const size_t in_bytes = 2 * (8 * size_t(pc.max_hits_per_slot) + 16 * size_t(pc.max_velo_per_slot));
    const size_t out_bytes = 2 * out_block_bytes(pc.max_events_per_slot, ocap);
    const size_t per_slot = ws_bytes + in_bytes + out_bytes;
    const int64_t fit = pc.mem_cap_bytes / int64_t(per_slot);
    if (fit < 1) return set_err(ctx, ST_ENOMEM, "one pipeline slot (%zu bytes) exceeds mem_cap_bytes", per_slot);
    pc.n_slots = static_cast<int32_t>(std::min<int64_t>(pc.n_slots, fit));
    Pipeline* pl = new Pipeline();
    pl->pc = pc;
    pl->hr.cap = 2 * size_t(pc.max_hits_per_slot) * pc.n_slots;
    pl->vr.cap = 2 * size_t(pc.max_velo_per_slot) * pc.n_slots;
    pl->orr.cap = out_bytes * pc.n_slots;
    cudaError_t e = cudaMalloc(&pl->d_x, 4 * pl->hr.cap);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_zone, 4 * pl->hr.cap);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_velo, 16 * pl->vr.cap);
    if (e == cudaSuccess) e = cudaMalloc(&pl->d_out, pl->orr.cap);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->in_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->out_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        pipeline_free(pl);
        return set_err(ctx, e == cudaErrorMemoryAllocation ? ST_ENOMEM : ST_ECUDA, "pipeline memory: %s",
                       cudaGetErrorString(e));
    }
    pl->slots.resize(pc.n_slots);
    for (auto& S : pl->slots) {
        int rc = slot_alloc(ctx, S, pc);
        if (rc != ST_OK) {
            pipeline_free(pl);
            return rc;
        }
    }
    pl->dispatcher = std::thread(dispatcher_main, ctx, pl);
    pl->completer = std::thread(completer_main, ctx, pl);
    ctx->pipe = pl;
    return ST_OK;
}

static void pipeline_shutdown(st_ctx* ctx) {
    Pipeline* pl = ctx->pipe;
    if (!pl) return;
    {
        std::unique_lock<std::mutex> lk(pl->mu);
        // let launched work finish, drop what has not started
        pl->pending.clear();
        pl->cv_done.wait(lk, [&] {
            for (auto& s : pl->slots)
                if (s.busy) return false;
            return true;
        });
        pl->stop = true;
        pl->cv_work.notify_all();
        pl->cv_done.notify_all();
        pl->cv_space.notify_all();
    }
    pl->dispatcher.join();
    pl->completer.join();
    pipeline_free(pl);
    ctx->pipe = nullptr;
}

extern "C" int pipeline_submit(st_ctx* ctx, const st_hits* hh, const st_velo* hv, uint64_t* ticket) {
    if (!ctx || !hh || !hv || !ticket) return ST_EINVAL;
    if (!ctx->pipe) {
        int rc = pipeline_start(ctx);
        if (rc != ST_OK) return rc;
    }
    Pipeline& pl = *ctx->pipe;
    const int64_t n = hh->n_events;
    if (n < 1 || hv->n_events != n || !hh->ev_off || !hv->ev_off ||
        (hh->ev_off[n] > hh->ev_off[0] && (!hh->x || !hh->zone)) || (hv->ev_off[n] > hv->ev_off[0] && !hv->state))
        return set_err(ctx, ST_EINVAL, "pipeline_submit: bad batch");
    auto r = std::make_shared<Request>();
    r->t_submit = now_ns();
    r->n_events = n;
    const int64_t h0 = hh->ev_off[0], v0 = hv->ev_off[0];
    r->n_hits = hh->ev_off[n] - h0;
    r->n_velo = hv->ev_off[n] - v0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t dh = hh->ev_off[k + 1] - hh->ev_off[k], dv = hv->ev_off[k + 1] - hv->ev_off[k];
        if (dh < 0 || dv < 0) return set_err(ctx, ST_EINVAL, "pipeline_submit: decreasing offsets");
        if (dh > pl.pc.max_hits_per_event || dv > pl.pc.max_velo_per_event)
            return set_err(ctx, ST_OVERFLOW, "pipeline_submit: event larger than the pipeline limits");
    }
    if (n > pl.pc.max_events_per_slot || r->n_hits > pl.pc.max_hits_per_slot || r->n_velo > pl.pc.max_velo_per_slot)
        return set_err(ctx, ST_OVERFLOW, "pipeline_submit: batch larger than a pipeline slot");
    r->ev_off.resize(n + 1);
    r->velo_off.resize(n + 1);
    for (int64_t k = 0; k <= n; ++k) {
        r->ev_off[k] = hh->ev_off[k] - h0;
        r->velo_off[k] = hv->ev_off[k] - v0;
    }
    {
        // admission: wait (bounded) until the input rings have room
        std::unique_lock<std::mutex> lk(pl.mu);
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(60);
        for (;;) {
            if (pl.stop) return set_err(ctx, ST_ESTATE, "pipeline stopping");
            size_t ho, vo;
            uint64_t hid, vid;
            if (pl.hr.alloc(size_t(r->n_hits), ho, hid)) {
                if (pl.vr.alloc(size_t(r->n_velo), vo, vid)) {
                    r->h_off = ho;
                    r->h_id = hid;
                    r->v_off = vo;
                    r->v_id = vid;
                    break;
                }
                pl.hr.release(hid);
            }
            if (pl.cv_space.wait_until(lk, deadline) == std::cv_status::timeout)
                return set_err(ctx, ST_TIMEOUT, "pipeline_submit: no room in the input rings for 60 s");
        }
    }
    {
        // DMA straight from the caller's memory; the caller may reuse its
        // buffers when this returns
        std::lock_guard<std::mutex> g(pl.in_mu);
        cudaError_t e = cudaSuccess;
        if (r->n_hits) {
            e = cudaMemcpyAsync(pl.d_x + r->h_off, hh->x + h0, 4 * size_t(r->n_hits), cudaMemcpyHostToDevice,
                                pl.in_stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(pl.d_zone + r->h_off, hh->zone + h0, 4 * size_t(r->n_hits),
                                    cudaMemcpyHostToDevice, pl.in_stream);
        }
        if (e == cudaSuccess && r->n_velo)
            e = cudaMemcpyAsync(pl.d_velo + 4 * r->v_off, hv->state + 4 * v0, 16 * size_t(r->n_velo),
                                cudaMemcpyHostToDevice, pl.in_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(pl.in_stream);
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> g2(pl.mu);
            pl.hr.release(r->h_id);
            pl.vr.release(r->v_id);
            pl.cv_space.notify_all();
            return set_err(ctx, ST_ECUDA, "pipeline_submit: copy: %s", cudaGetErrorString(e));
        }
    }
    std::lock_guard<std::mutex> g(pl.mu);
    r->id = pl.next_id++;
    pl.all[r->id] = r;
    pl.pending.push_back(r);
    *ticket = r->id;
    pl.cv_work.notify_one();
    return ST_OK;
}

extern "C" int pipeline_poll(st_ctx* ctx, uint64_t ticket, st_seeds* hs, st_long* hl, int64_t timeout_us,
                             st_request_info* info) {
    if (!ctx) return ST_EINVAL;
    if (!ctx->pipe) return set_err(ctx, ST_EINVAL, "pipeline_poll: unknown ticket");
    Pipeline& pl = *ctx->pipe;
    std::unique_lock<std::mutex> lk(pl.mu);
    auto it = pl.all.find(ticket);
    if (it == pl.all.end()) return set_err(ctx, ST_EINVAL, "pipeline_poll: unknown ticket");
    std::shared_ptr<Request> r = it->second;
    if (!r->done) {
        if (timeout_us == 0) return ST_PENDING;
        auto pred = [&] { return r->done; };
        if (timeout_us < 0) {
            pl.cv_done.wait(lk, pred);
        } else if (!pl.cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) {
            return ST_TIMEOUT;
        }
    }
    auto finish = [&](std::unique_lock<std::mutex>& l) {
        pl.all.erase(ticket);
        if (r->out && --r->out->refs == 0) {
            pl.orr.release(r->out->ring_id);
            pl.cv_space.notify_all();
        }
        r->out.reset();
        (void)l;
    };
    if (r->status != ST_OK) {
        finish(lk);
        return set_err(ctx, r->status, "pipeline batch failed");
    }
    const int64_t n = r->n_events, ns = r->s1 - r->s0;
    if (!hs || !hs->ev_off || !hs->status || (ns > 0 && (!hs->hits || !hs->params || !hs->state || !hs->n_hits)))
        return set_err(ctx, ST_EINVAL, "pipeline_poll: null output");
    if (hs->cap < ns)
        return set_err(ctx, ST_OVERFLOW, "pipeline_poll: host_seeds cap %lld < %lld", (long long)hs->cap, (long long)ns);
    std::shared_ptr<OutBlock> ob = r->out;
    lk.unlock();
    cudaError_t e = cudaSuccess;
    {
        // DMA straight into the caller's memory
        std::lock_guard<std::mutex> g(pl.out_mu);
        cudaStream_t st = pl.out_stream;
        auto cp = [&](void* dst, const void* src, size_t bytes) {
            if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
        };
        const int64_t s0 = r->s0;
        cp(hs->ev_off, ob->ev_off + r->e0, 4 * size_t(n + 1));
        cp(hs->status, ob->status + r->e0, 4 * size_t(n));
        cp(hs->hits, ob->hits + 12 * s0, 48 * size_t(ns));
        cp(hs->params, ob->params + 8 * s0, 32 * size_t(ns));
        cp(hs->state, ob->state + 4 * s0, 16 * size_t(ns));
        cp(hs->n_hits, ob->n + 2 * s0, 2 * size_t(ns));
        if (hl) {
            if (hl->velo_idx) cp(hl->velo_idx, ob->vidx + s0, 4 * size_t(ns));
            if (hl->chi2) cp(hl->chi2, ob->chi2 + s0, 4 * size_t(ns));
            if (hl->n_long) cp(hl->n_long, ob->n_long + r->e0, 4 * size_t(n));
            if (hl->ghost_prob) cp(hl->ghost_prob, ob->gp + s0, 4 * size_t(ns));
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e == cudaSuccess) {
        const int32_t base = hs->ev_off[0];
        for (int64_t k = 0; k <= n; ++k) hs->ev_off[k] -= base;
    }
    const int64_t tret = now_ns();
    lk.lock();
    finish(lk);
    if (e != cudaSuccess) return set_err(ctx, ST_ECUDA, "pipeline_poll: copy: %s", cudaGetErrorString(e));
    if (info) {
        info->t_submit_ns = r->t_submit;
        info->t_launch_ns = r->t_launch;
        info->t_done_ns = r->t_done;
        info->t_returned_ns = tret;
        info->n_events = static_cast<int32_t>(n);
        info->n_seeds = static_cast<int32_t>(ns);
    }
    return ST_OK;
}
