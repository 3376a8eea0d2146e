"""Each pin set must catch a plausible mistake planted in the oracle.

A copy of oracle.c is edited in a temporary directory (one mistake per copy:
a dropped term, a wrong sign, a transposed operand, a wrong index), compiled,
and the pin checks of test_oracle_pins.py are run against it.  At least one
check must fail for every mutant.  The real oracle is never modified.
"""

import os

import pytest

import oracle
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
    for chk in pins.ALL_CHECKS:
        kw = {"zmx": zmx_calibrated} if chk is pins.check_noise_free_recovery else {}
        try:
            chk(L, **kw)
        except AssertionError:
            failed.append(chk.__name__)
    assert failed, f"no pin caught mutation {name}"
