"""Each pin set must catch a plausible mistake planted in the oracle.

A copy of oracle.c is edited in a temporary directory (one mistake per copy:
a dropped term, a wrong sign, a transposed operand, a wrong index), compiled,
and the pin checks of test_oracle_pins.py and test_ledger_pins.py are run
against it.  At least one check must fail for every mutant.  The real oracle
is never modified.  The "ledger_*" mutants plant mistakes in the cut ledger
(a margin left unnormalised or measured to the wrong edge, the wrong hits
named, entries dropped): the ledger decides which GPU/oracle differences are
excused, so a mistake there must not pass unseen.
"""

import os

import pytest

import oracle
import test_ledger_pins as ledger_pins
import test_oracle_pins as pins

MUTATIONS = {
    "drop_d_ratio": ("return zb * zb * (1.0 + c->d_ratio * zb);", "return zb * zb;"),
    "alpha_sign": ("const double xc = (z3 + alpha) / z1 * x1;", "const double xc = (z3 - alpha) / z1 * x1;"),
    "k_transposed": ("double k = z1 / (z3 - z1);\n    return c->alpha0",
                     "double k = (z3 - z1) / z1;\n    return c->alpha0"),
    "dx3_wrong_layer": ("double z1 = c->z[c->iter_layers[it][0]], z3 = c->z[c->iter_layers[it][2]];\n    return c->dx3_scale",
                        "double z1 = c->z[c->iter_layers[it][0]], z3 = c->z[c->iter_layers[it][1]];\n    return c->dx3_scale"),
    "fit_unscale": ("for (int j = 0; j < 3; ++j) th[j] = y[j] * sc[j];",
                    "for (int j = 0; j < 3; ++j) th[j] = y[j] / sc[j];"),
    "chi2_sigma": ("fit_xz(c, nx, fz, fx, th) / (c->sigma_x * c->sigma_x)", "fit_xz(c, nx, fz, fx, th) / c->sigma_x"),
    "ext_tol_half": ("hits[xslot_of_layer(L)] = closest_hit(E, 2 * L + half, xp, c->ext_tol, sc,",
                     "hits[xslot_of_layer(L)] = closest_hit(E, 2 * L + half, xp, 0.5 * c->ext_tol, sc,"),
    "clone_rule": ("cd->keep = owned >= 3 || (owned >= 2 && cd->nx == 6);", "cd->keep = owned >= 2;"),
    "uv_y_sign": ("const double y = (XI - xh) / tI;", "const double y = (xh - XI) / tI;"),
    "match_dropped_E": (" + c->zmx[4] * txV * txV;", ";"),
    "match_wrong_z": ("(xS + (zmx - c->z_state) * txS)", "(xS + (zmx - c->z_velo) * txS)"),
    "toly_no_ty": ("const double rho = txV * txV + tyV * tyV;", "const double rho = txV * txV;"),
    "hough_single_bin": ("for (int q = 0; q < 6; ++q) pop[b] += occ[q][b] + occ[q][b + 1] > 0;",
                         "for (int q = 0; q < 6; ++q) pop[b] += occ[q][b] > 0;"),
    "hough_counts_hits": ("for (int q = 0; q < 6; ++q) pop[b] += occ[q][b] + occ[q][b + 1] > 0;",
                          "for (int q = 0; q < 6; ++q) pop[b] += occ[q][b] + occ[q][b + 1];"),
    "hough_worst_first": ("for (int p = 6; p >= c->n_uv_min && nsel < c->hough_clusters; --p)",
                          "for (int p = c->n_uv_min; p <= 6 && nsel < c->hough_clusters; ++p)"),
    "hough_bin_edge": ("const double ty = ty_lo + w * (sel[r] + (f + 0.5) * 2.0 / F);",
                       "const double ty = ty_lo + w * (sel[r] + f * 2.0 / F);"),
    "hough_y_sign": ("const double y = (XL - xh) / tL;\n            const double S = dmax2(dmax2(SL",
                     "const double y = (xh - XL) / tL;\n            const double S = dmax2(dmax2(SL"),
    "nn_no_relu": ("        if (a > 0) z += w2[k] * a;", "        z += w2[k] * a;"),
    "nn_standardise_sign": ("for (int i = 0; i < 8; ++i) in[i] = (f[i] - mean[i]) * inv_scale[i];",
                            "for (int i = 0; i < 8; ++i) in[i] = (f[i] + mean[i]) * inv_scale[i];"),
    "eta_inverted": ("asinh(1.0 / rho)", "asinh(rho)"),
    "ghost_cut_reversed": ("if (!(p < c->ghost_max)) velo_idx[s] = -1;", "if (p < c->ghost_max) velo_idx[s] = -1;"),
    "clone_margin_sign": ("if (d >= c->clone_margin) drop[s] = 1;", "if (-d >= c->clone_margin) drop[s] = 1;"),
    "nn_hits_feature": ("chi2[s], asinh(1.0 / rho), (double)seed_nhits[s]};", "chi2[s], asinh(1.0 / rho), chi2[s]};"),
    "ut_refit_sign": ("g = (ut_x[best] + yt * c->ut_dxdy[l] - xV - txV * dz) / (dz * dz);",
                      "g = (ut_x[best] - yt * c->ut_dxdy[l] - xV - txV * dz) / (dz * dz);"),
    "ut_window_p": ("w[0] + w[1] * inv_p_gev", "w[0] + w[1] / inv_p_gev"),
    "ut_no_refit": ("                g = (ut_x[best] + yt * c->ut_dxdy[l] - xV - txV * dz) / (dz * dz);\n", ""),
    "ut_min_hits": ("if (n < c->ut_min_hits) velo_idx[s] = -1;", "if (n <= c->ut_min_hits) velo_idx[s] = -1;"),
    "ut_windows_swapped": ("found ? &c->ut_tight[4 * l] : &c->ut_loose[4 * l]",
                           "found ? &c->ut_loose[4 * l] : &c->ut_tight[4 * l]"),
    "cleanup_missing": ("for (int k = 0; k < n_taken; ++k) used[taken[k]] = 1;",
                        "for (int k = 0; k < n_taken; ++k) (void)taken[k];"),
    "pmin_iter_ignored": ("return it >= 0 && it < 3 && c->p_min_iter[it] > 0 ? c->p_min_iter[it] : c->p_min;",
                          "return c->p_min;"),
    "used_t3_ignored": ("                if (E->used && E->used[h3]) continue;\n", ""),
    "ledger_pair_unscaled": ("double m = fmin(fabs(x3 - lo), fabs(x3 - hi)) / dmax2(S3, fabs(x3));",
                             "double m = fmin(fabs(x3 - lo), fabs(x3 - hi));"),
    "ledger_pair_far_edge": ("double m = fmin(fabs(x3 - lo), fabs(x3 - hi)) / dmax2(S3, fabs(x3));",
                             "double m = fmax(fabs(x3 - lo), fabs(x3 - hi)) / dmax2(S3, fabs(x3));"),
    "ledger_trip_unscaled": ("double m = fmin(fabs(x2 - lo2), fabs(x2 - hi2)) / dmax2(S2, fabs(x2));",
                             "double m = fmin(fabs(x2 - lo2), fabs(x2 - hi2));"),
    "ledger_trip_hit_order": ("int32_t hh[3] = {h1, h3, h2};", "int32_t hh[3] = {h1, h2, h3};"),
    "ledger_tol_unscaled": ("ledger_add(E, kind_tol, half, fabs(d - tol) / S, hh, nh + 1);",
                            "ledger_add(E, kind_tol, half, fabs(d - tol), hh, nh + 1);"),
    "ledger_tol_wrong_hit": ("hh[nh] = E->zl[zi][k].i;", "hh[nh] = -1;"),
    "ledger_tie_unscaled": ("fabs(second - bestd) / dmax2(scale, 1.0)", "fabs(second - bestd)"),
    "ledger_chi2_unnormalised": ("fabs(q - c->chi2x_max) / c->chi2x_max", "fabs(q - c->chi2x_max)"),
    "ledger_clone_absolute": ("double m = fabs(a->score - w->score) / dmax2(a->score, w->score);",
                              "double m = fabs(a->score - w->score);"),
    "ledger_clone_wrong_hits": ("hh[6 + q] = w->hits[q];", "hh[6 + q] = a->hits[q];"),
    "ledger_uv_win_in_y": ("double m = fmin(fabs(y - ylo), fabs(y - yhi)) * fabs(tI) /",
                           "double m = fmin(fabs(y - ylo), fabs(y - yhi)) /"),
    "ledger_uv_sel_absolute": (
        "double m = fabs(all[k].chi2 - all[b].chi2) / dmax2(dmax2(all[k].chi2, all[b].chi2), 1e-300);",
        "double m = fabs(all[k].chi2 - all[b].chi2);"),
    "ledger_presel_absolute": ("fabs(val[q] - cut[q]) / cut[q]", "fabs(val[q] - cut[q])"),
    "ledger_m_chi2_absolute": ("fabs(chi2 - c->chi2_match_max) / c->chi2_match_max",
                               "fabs(chi2 - c->chi2_match_max)"),
    "ledger_m_tie_absolute": ("fabs(schi - bchi) / dmax2(schi, 1e-300)", "fabs(schi - bchi)"),
    "ledger_drops_entries": ("if (!(margin <= E->tau)) return;", "if (!(margin <= 0.01 * E->tau)) return;"),
    "state_slope": ("s->tx_s = cd->th[1] + cd->th[2] * (2.0 * zb + 3.0 * c->d_ratio * zb * zb);",
                    "s->tx_s = cd->th[1];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path, zmx_calibrated):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    mpath = tmp_path / "oracle_mut.c"
    mpath.write_text(src.replace(old, new))
    so = oracle.build(force=True, src=str(mpath), out=str(tmp_path / "liboracle_mut.so"))
    L = oracle.lib(so)
    failed = []
    for chk in pins.ALL_CHECKS + ledger_pins.ALL_CHECKS:
        kw = {"zmx": zmx_calibrated} if chk is pins.check_noise_free_recovery else {}
        try:
            chk(L, **kw)
        except AssertionError:
            failed.append(chk.__name__)
    assert failed, f"no pin caught mutation {name}"
