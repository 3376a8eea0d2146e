"""Pins of the FP64 oracle to things other than itself.

Each check compares the oracle with what the paper prints, a closed form, a
library routine applied to a special case, generator truth, or a brute-force
enumeration on tiny inputs.  The `check_*` functions take the oracle library
handle so that test_oracle_mutations.py can run them against copies of the
oracle with a planted mistake.
"""

import math

import numpy as np
import pytest

import oracle
from conftest import read_golden_constants, truth_track_of, workload
from synth import Detector, make_events

DET = Detector()
X_LAYERS = (0, 3, 4, 7, 8, 11)
UV_LAYERS = (1, 2, 5, 6, 9, 10)


# ---------------------------------------------------------------------------
# reusable checks
# ---------------------------------------------------------------------------

def check_paper_constants(L=None):
    cfg = oracle.default_config(_lib=L)
    for (f, i), v in read_golden_constants().items():
        cur = getattr(cfg, f)
        got = cur[i] if i is not None else cur
        assert got == pytest.approx(v, rel=1e-12, abs=1e-15), (f, i, got, v)


def check_window_closed_forms(L=None):
    cfg = oracle.default_config(_lib=L)
    # x0max: the momentum limit solves b x0^2 + a x0 = 1/p_min (Eq. invp);
    # its smaller positive root, from numpy's polynomial root finder.
    r = np.roots([cfg.invp_b, cfg.invp_a, -1.0 / cfg.p_min])
    r = np.sort(r[np.isreal(r) & (r.real > 0)].real)
    assert oracle.x0max(cfg, _lib=L) == pytest.approx(r[0], rel=1e-12)
    assert oracle.invp(cfg, r[0], _lib=L) == pytest.approx(1.0 / cfg.p_min, rel=1e-12)
    assert oracle.invp(cfg, -r[0], _lib=L) == pytest.approx(1.0 / cfg.p_min, rel=1e-12)
    for it in range(2):
        z1 = cfg.z[cfg.iter_layers[it][0]]
        z3 = cfg.z[cfg.iter_layers[it][2]]
        # Eq. tolHp must equal Eq. delta3 evaluated at the momentum limit
        assert oracle.dx3max(cfg, it, _lib=L) == pytest.approx((z3 - z1) / z1 * r[0], rel=1e-12)
        # Eq. alphacorr as an offset in z: k * alpha_corr * (p_min - alpha1) = alpha0
        k = z1 / (z3 - z1)
        assert k * oracle.alpha_corr(cfg, it, _lib=L) * (cfg.p_min - cfg.alpha1) == \
            pytest.approx(cfg.alpha0, rel=1e-12)


def check_k3_chord(L=None):
    # d_ratio = 0: deviation of a parabola from its chord is c (z2-z1)(z2-z3)
    cfg0 = oracle.default_config(_lib=L, d_ratio=0.0)
    for it in range(2):
        z1, z2, z3 = (cfg0.z[cfg0.iter_layers[it][k]] for k in range(3))
        assert oracle.k3(cfg0, it, _lib=L) == pytest.approx((z2 - z1) * (z2 - z3), rel=1e-12)
    # d_ratio != 0: dx2 = x2 - (x1 + (z2-z1) t13) equals k3 * c for exact model
    # positions produced by the generator's track model
    cfg = oracle.default_config(_lib=L)
    rng = np.random.default_rng(5)
    for it in range(2):
        z1, z2, z3 = (cfg.z[cfg.iter_layers[it][k]] for k in range(3))
        for _ in range(20):
            a, b, c = rng.uniform(-2000, 2000), rng.uniform(-0.3, 0.3), rng.uniform(-5e-6, 5e-6)
            x1, x2, x3 = (DET.x_model(a, b, c, zz) for zz in (z1, z2, z3))
            dx2 = x2 - (x1 + (z2 - z1) * (x3 - x1) / (z3 - z1))
            assert dx2 == pytest.approx(oracle.k3(cfg, it, _lib=L) * c, rel=1e-7, abs=1e-9)


def check_noise_free_recovery(L=None, zmx=None, n_events=6, **overrides):
    """North-star pin: noise-free, unsmeared, fully efficient tracks above
    3.5 GeV are all found, with no ghost or clone, each seed holds exactly its
    track's 12 hits, the fit returns the generating parameters to FP64
    rounding, and matching picks the track's own VELO segment."""
    b = workload("noise_free", n_events=n_events)
    cfg = oracle.default_config(_lib=L, **overrides)
    if zmx is not None:
        oracle.apply(cfg, {"zmx": zmx})
    for e in range(b.n_events):
        x, z = b.exact_hits_of(e)
        r = oracle.seeding_event(cfg, x, z, _lib=L)
        tr = b.tracks_of(e)
        seeds = r["seeds"]
        assert len(seeds) == len(tr["p"]), (e, len(seeds), len(tr["p"]))
        found = set()
        for s in seeds:
            t, purity = truth_track_of(b, e, s["hits"])
            assert purity == 1.0 and t >= 0
            k = t - b.trk_off[e]
            assert t not in found
            found.add(t)
            assert list(s["hits"]) == list(tr["layer_hit"][k])
            assert s["a"] == pytest.approx(tr["a"][k], rel=1e-9, abs=1e-9)
            assert s["b"] == pytest.approx(tr["b"][k], rel=1e-9, abs=1e-12)
            assert s["c"] == pytest.approx(tr["c"][k], rel=1e-7, abs=1e-15)
            assert s["ty"] == pytest.approx(tr["ty"][k], rel=1e-9, abs=1e-12)
            assert s["y0"] == pytest.approx(0.0, abs=1e-6)
            assert s["chi2x"] < 1e-12 and s["chi2y"] < 1e-12
            zs = cfg.z_state
            assert s["x_s"] == pytest.approx(DET.x_model(tr["a"][k], tr["b"][k], tr["c"][k], zs),
                                             rel=1e-9, abs=1e-9)
            assert s["tx_s"] == pytest.approx(DET.x_slope(tr["b"][k], tr["c"][k], zs), abs=1e-11)
        if zmx is not None:
            st = np.stack([seeds["x_s"], seeds["y_s"], seeds["tx_s"], seeds["ty_s"]], 1)
            m = oracle.matching_event(cfg, b.velo_of(e), st, _lib=L)
            vt = b.velo_track[b.velo_off[e]:b.velo_off[e + 1]]
            for k, s in enumerate(seeds):
                t, _ = truth_track_of(b, e, s["hits"])
                assert m["velo_idx"][k] >= 0 and vt[m["velo_idx"][k]] == t


def _tiny_event(seed, ntr=6, noise=3.0):
    return make_events(1, seed=seed, tracks=("fixed", ntr), noise_frac=noise, eff=0.9,
                       sigma_x=0.07, velo_ghosts_per_track=0.0, velo_sigma=(0, 0))


def check_triplets_brute_force(L=None, n_events=8):
    """Every (T1, T2, T3) hit triple is tested with the window predicates of
    Section 3.3 directly (no sorting, no scan order); the set must equal the
    oracle's triplet list, and for each triplet the candidate built by brute
    force (closest hit within 1 mm in each remaining x-layer, numpy least
    squares, chi2/ndf cut) must equal the oracle's candidate."""
    cfg = oracle.default_config(_lib=L)
    a, bb, pmin = cfg.invp_a, cfg.invp_b, cfg.p_min
    for ev in range(n_events):
        b = _tiny_event(900 + ev)
        x, zone = b.hits_of(0)
        x = x.astype(np.float64)
        r = oracle.seeding_event(cfg, x, zone, trips=True, cands=True, _lib=L)
        got = {tuple(t) for t in r["trips"]}
        want = set()
        want_cands = {}
        n_pairs = 0
        for half in range(2):
            for it in range(cfg.n_iter):
                L1, L2, L3 = (cfg.iter_layers[it][k] for k in range(3))
                z1, z2, z3 = cfg.z[L1], cfg.z[L2], cfg.z[L3]
                H1, H2, H3 = (np.nonzero(zone == 2 * Lx + half)[0] for Lx in (L1, L2, L3))
                x0max = (-a + math.sqrt(a * a + 4 * bb / pmin)) / (2 * bb)
                dx3 = (z3 - z1) / z1 * x0max
                alpha = cfg.alpha0 * (z3 - z1) / (z1 * (pmin - cfg.alpha1))
                f = lambda zz: (zz - cfg.z_ref) ** 2 * (1 + cfg.d_ratio * (zz - cfg.z_ref))
                k3v = f(z2) - f(z1) - (z2 - z1) / (z3 - z1) * (f(z3) - f(z1))
                w1, w3 = (z3 - z2) / (z3 - z1), (z2 - z1) / (z3 - z1)
                c0 = cfg.c_nsigma * cfg.sigma_x * math.sqrt(1 + w1 ** 2 + w3 ** 2) / abs(k3v)
                for h1 in H1:
                    for h3 in H3:
                        centre = (z3 + alpha) / z1 * x[h1]
                        if not (centre - dx3 <= x[h3] <= centre + dx3):
                            continue
                        n_pairs += 1
                        t13 = (x[h3] - x[h1]) / (z3 - z1)
                        x0 = x[h1] - z1 * t13
                        ip = a * abs(x0) + bb * x0 * x0
                        if ip <= 0:
                            continue
                        s = 1.0 if x0 > 0 else -1.0
                        cands = [-s * (cfg.m_lo * cfg.kappa_c * ip - c0), -s * (cfg.m_hi * cfg.kappa_c * ip + c0)]
                        xs = [x[h1] + (z2 - z1) * t13 + k3v * cc for cc in cands]
                        for h2 in H2:
                            if min(xs) <= x[h2] <= max(xs):
                                want.add((half, it, h1, h2, h3))
                                # candidate by brute force
                                Z = np.array([z1, z2, z3])
                                A3 = np.stack([np.ones(3), Z - cfg.z_ref, f(Z)], 1)
                                th3 = np.linalg.solve(A3, x[[h1, h2, h3]])
                                hits = {L1: h1, L2: h2, L3: h3}
                                for Lx in X_LAYERS:
                                    if Lx in hits:
                                        continue
                                    HL = np.nonzero(zone == 2 * Lx + half)[0]
                                    xp = th3 @ [1.0, cfg.z[Lx] - cfg.z_ref, f(cfg.z[Lx])]
                                    d = np.abs(x[HL] - xp)
                                    ok = d <= cfg.ext_tol
                                    if ok.any():
                                        dm = d[ok].min()
                                        best = HL[ok][d[ok] == dm]
                                        hits[Lx] = best[np.argmin(x[best])]
                                if len(hits) < 5:
                                    continue
                                Ls = sorted(hits)
                                Zs = np.array([cfg.z[l] for l in Ls])
                                Af = np.stack([np.ones(len(Ls)), (Zs - cfg.z_ref) / 1e3, f(Zs) / 1e9], 1)
                                xv = x[[hits[l] for l in Ls]]
                                th, *_ = np.linalg.lstsq(Af, xv, rcond=None)
                                chi2 = np.sum((xv - Af @ th) ** 2) / cfg.sigma_x ** 2
                                if chi2 / (len(Ls) - 3) > cfg.chi2x_max:
                                    continue
                                key = (half, it, h1, h2, h3)
                                want_cands[key] = (tuple(hits.get(l, -1) for l in X_LAYERS), chi2,
                                                   th * [1, 1e-3, 1e-9])
        assert r["counters"]["pairs"] == n_pairs, ev
        assert got == want, (ev, sorted(got ^ want)[:5])
        got_c = {(int(c["half"]), int(c["iter"]), int(c["h1"]), int(c["h2"]), int(c["h3"])): c
                 for c in r["cands"]}
        assert set(got_c) == set(want_cands), ev
        for key, (hits, chi2, th) in want_cands.items():
            c = got_c[key]
            assert tuple(c["hits"]) == hits
            assert c["chi2"] == pytest.approx(chi2, rel=1e-6, abs=1e-9)
            assert c["a"] == pytest.approx(th[0], rel=1e-9, abs=1e-9)
            assert c["c"] == pytest.approx(th[2], rel=1e-6, abs=1e-14)


def check_clone_kill_pairwise(L=None, n_events=8):
    """The O(n) table-and-vote of Section 3.3.4 against a pairwise statement
    of the same rule: a candidate owns a hit iff no other candidate holding
    that hit is better by (score, id); kept iff it owns >= 3 hits, or >= 2
    with 6 hits.  Dense events (280 tracks, 40% noise) so that every branch
    of the rule occurs."""
    cfg = oracle.default_config(_lib=L)
    b = workload("match_stress", n_events=n_events)
    n_five_two = 0
    for e in range(b.n_events):
        r = oracle.seeding_event(cfg, *b.hits_of(e), cands=True, _lib=L)
        cands = r["cands"]
        for half in range(2):
            cs = cands[cands["half"] == half]
            if len(cs) == 0:
                continue
            H = cs["hits"]                                     # (n, 6)
            better = (cs["score"][None, :] < cs["score"][:, None]) | (
                (cs["score"][None, :] == cs["score"][:, None]) & (cs["id"][None, :] < cs["id"][:, None]))
            # holds[i, s, j]: hit s of candidate i is one of candidate j's hits
            holds = (H[:, :, None, None] == H[None, None, :, :]).any(-1).transpose(0, 1, 2)
            holds &= (H >= 0)[:, :, None]
            beaten = (holds & better[:, None, :]).any(-1)      # (n, 6)
            owned = ((H >= 0) & ~beaten).sum(1)
            keep = (owned >= 3) | ((owned >= 2) & (cs["nx"] == 6))
            n_five_two += int(np.sum((owned == 2) & (cs["nx"] == 5)))
            assert np.array_equal(cs["keep"].astype(bool), keep)
            kept = [tuple(h) for h in H[keep]]
            assert len(kept) == len(set(kept))
    assert n_five_two > 0


def check_tolerance_boundaries(L=None):
    """A noise-free track with one hit moved to 0.9x or 1.1x of a tolerance from
    its exact prediction: the x-layer extension (1 mm, Section 3.2) and the
    stereo search (2 mm, Section 3.4) take the hit only inside the tolerance."""
    cfg = oracle.default_config(_lib=L, chi2x_max=1e12)
    b = make_events(1, seed=321, tracks=("fixed", 1), noise_frac=0.0, eff=1.0, sigma_x=0.0,
                    p_range=(5.0, 50.0), velo_ghosts_per_track=0.0, velo_sigma=(0, 0))
    x0, zone = b.exact_hits_of(0)
    lh = b.tracks_of(0)["layer_hit"][0]
    for frac, inside in ((0.9, True), (1.1, False)):
        for sign in (1.0, -1.0):
            # x-layer 8 is extended from the iteration-0 triplet (layers 0, 4, 11)
            x = x0.copy()
            x[lh[8]] += sign * frac * cfg.ext_tol
            r = oracle.seeding_event(cfg, x, zone, cands=True, _lib=L)
            c0 = [c for c in r["cands"] if c["iter"] == 0 and c["h1"] == lh[0] and c["h2"] == lh[4]
                  and c["h3"] == lh[11]]
            assert len(c0) == 1
            assert (c0[0]["hits"][4] == lh[8]) == inside
            # stereo layer 10 is the last one searched in both passes
            x = x0.copy()
            x[lh[10]] += sign * frac * cfg.uv_tol
            r = oracle.seeding_event(cfg, x, zone, _lib=L)
            assert len(r["seeds"]) == 1
            sd = r["seeds"][0]
            assert (sd["hits"][10] == lh[10]) == inside
            assert sd["nuv"] == (6 if inside else 5)


def check_matching_grid(L=None, zmx=None, n_events=8):
    """Matching against a vectorised evaluation of Section 4 over the full
    VELO x seed grid, plus two constructed special cases."""
    cfg = oracle.default_config(_lib=L)
    if zmx is not None:
        oracle.apply(cfg, {"zmx": zmx})
    b = workload("run3", n_events=n_events)
    rng = np.random.default_rng(3)
    for e in range(b.n_events):
        velo = b.velo_of(e).astype(np.float64)
        tr = b.tracks_of(e)
        # seed states: true SciFi states plus random ones
        st = np.stack([DET.x_model(tr["a"], tr["b"], tr["c"], cfg.z_state), tr["ty"] * cfg.z_state,
                       DET.x_slope(tr["b"], tr["c"], cfg.z_state), tr["ty"]], 1)
        st = np.concatenate([st, st[rng.permutation(len(st))] + rng.normal(0, [5, 20, 0.01, 0.002], st.shape)])
        m = oracle.matching_event(cfg, velo, st, _lib=L)
        xv, yv, txv, tyv = (velo[:, k][None, :] for k in range(4))
        xs, ys, txs, tys = (st[:, k][:, None] for k in range(4))
        dtx, dty = txv - txs, tyv - tys
        A, B, Cc, D, E = (cfg.zmx[k] for k in range(5))
        zm = A + B * np.abs(dtx) + Cc * dtx ** 2 + D * np.abs(xs) + E * txv ** 2
        dx = (xv + (zm - cfg.z_velo) * txv) - (xs + (zm - cfg.z_state) * txs)
        dy = (yv + (cfg.z_match_y - cfg.z_velo) * tyv) - (ys + (cfg.z_match_y - cfg.z_state) * tys)
        pres = (np.abs(dx) < 20) & (np.abs(dy) < 150) & (np.abs(dtx) < 1.5) & (np.abs(dty) < 0.02)
        tolx = 0.8 * (10.12 ** 2 + 101.0 ** 2 * dtx ** 2)
        toly = 0.2 * (1.59 ** 2 + 212.1 ** 2 * (txv ** 2 + tyv ** 2))
        chi2 = dx ** 2 / tolx + dy ** 2 / toly + dtx ** 2 / 0.5 + dty ** 2 * 937.5
        chi2 = np.where(pres & (chi2 < 2.0), chi2, np.inf)
        want = np.where(np.isfinite(chi2.min(1)), chi2.argmin(1), -1)
        assert np.array_equal(m["velo_idx"], want)
        ok = want >= 0
        assert np.allclose(m["chi2"][ok], chi2[ok, want[ok]], rtol=1e-12)
    # collinear VELO and SciFi segments: all four differences vanish
    tx, ty = 0.1, 0.05
    velo = np.array([[tx * cfg.z_velo + 3.0, ty * cfg.z_velo - 1.0, tx, ty]])
    seed = np.array([[tx * cfg.z_state + 3.0, ty * cfg.z_state - 1.0, tx, ty]])
    m = oracle.matching_event(cfg, velo, seed, _lib=L)
    assert m["velo_idx"][0] == 0 and m["chi2"][0] == pytest.approx(0.0, abs=1e-18)
    # pure y offset at the matching plane: chi2 = dy^2 / tol_y
    dyo = 1.0
    velo2 = velo.copy()
    velo2[0, 1] += dyo
    m = oracle.matching_event(cfg, velo2, seed, _lib=L)
    tol_y = 0.2 * (1.59 ** 2 + 212.1 ** 2 * (tx * tx + ty * ty))
    assert m["chi2"][0] == pytest.approx(dyo ** 2 / tol_y, rel=1e-12)


# ---------------------------------------------------------------------------
# Hough-cluster UV variant (Section 3.4, second approach)
# ---------------------------------------------------------------------------

def check_hough_noise_free(L=None, n_events=4):
    """The noise-free recovery pin with the Hough-cluster UV variant: every
    track found with its exact twelve hits and its generating t_y."""
    check_noise_free_recovery(L, None, n_events=n_events, uv_mode=1)


def _stereo_event(seed, ty_of_layer, extra=()):
    """One noise-free track whose six stereo hits are placed at the given
    t_y per stereo layer (y = t_y z), plus extra hits (layer, t_y); x-layer
    hits are the generator's exact ones.  Returns x, zone, the track's layer
    hits and its half."""
    b = make_events(1, seed=seed, tracks=("fixed", 1), noise_frac=0.0, eff=1.0, sigma_x=0.0,
                    p_range=(5.0, 50.0), velo_ghosts_per_track=0.0, velo_sigma=(0, 0))
    x, zone = b.exact_hits_of(0)
    x, zone = x.copy(), zone.copy()
    tr = b.tracks_of(0)
    lh = tr["layer_hit"][0]
    half = int(zone[lh[0]] % 2)
    sgn = 1.0 if half else -1.0
    a, bb, c = tr["a"][0], tr["b"][0], tr["c"][0]
    zl, t = DET.z_arr, DET.dxdy
    for L, ty in ty_of_layer.items():
        if ty is None:
            x[lh[L]] += 500.0  # moved far from the track: acts as a noise hit
        else:
            x[lh[L]] = DET.x_model(a, bb, c, zl[L]) - t[L] * sgn * ty * zl[L]
    xs, zs = [x], [zone]
    for L, ty in extra:
        xs.append(np.array([DET.x_model(a, bb, c, zl[L]) - t[L] * sgn * ty * zl[L]]))
        zs.append(np.array([2 * L + half], np.int32))
    return np.concatenate(xs), np.concatenate(zs).astype(np.int32), lh, half


def check_hough_clusters(L=None):
    """Constructed cases that fix each part of the Hough-cluster reading:
    a track whose stereo hits straddle a coarse bin edge is one cluster (two
    bins); populations count stereo LAYERS, not hits; clusters are taken best
    first; the t_y hypotheses are the centres of the fine sub-bins."""
    base = oracle.default_config(_lib=L, uv_mode=1)
    NB, F = base.hough_bins, base.hough_fine
    # half 1 range [-ty_in, ty_max]; the constructions use |t_y| of the track
    lo = -base.hough_ty_in
    w = (base.hough_ty_max + base.hough_ty_in) / NB
    layers = UV_LAYERS
    for seed in (401, 402, 403, 404):
        # (a) edge straddle: alternate layers 0.1 bin below / above an edge
        edge = lo + 11 * w
        x, zone, lh, half = _stereo_event(seed, {L: edge + (0.1 if k % 2 else -0.1) * w
                                                 for k, L in enumerate(layers)})
        if half == 0:  # the mirrored range of half 0 puts the edge elsewhere
            continue
        r = oracle.seeding_event(base, x, zone, _lib=L)
        assert len(r["seeds"]) == 1 and r["seeds"][0]["nuv"] == 6
        assert [r["seeds"][0]["hits"][q] for q in layers] == [lh[q] for q in layers]
        # (b) layers, not hits: 4 true stereo layers at 0.05 against 2 layers
        # holding 4 decoy hits each at 0.15; one cluster kept
        one = oracle.default_config(_lib=L, uv_mode=1, hough_clusters=1)
        spec = {L: 0.05 for L in layers}
        spec[9] = spec[10] = None
        x, zone, lh, half = _stereo_event(seed, spec, extra=[(9, 0.15)] * 4 + [(10, 0.15)] * 4)
        r = oracle.seeding_event(one, x, zone, _lib=L)
        assert len(r["seeds"]) == 1 and r["seeds"][0]["nuv"] == 4
        assert [r["seeds"][0]["hits"][q] for q in (1, 2, 5, 6)] == [lh[q] for q in (1, 2, 5, 6)]
        # (c) best first: the true 6-layer cluster against a 5-layer decoy
        x, zone, lh, half = _stereo_event(seed, {L: 0.05 for L in layers},
                                          extra=[(L, 0.15) for L in layers[:5]])
        r = oracle.seeding_event(one, x, zone, _lib=L)
        assert len(r["seeds"]) == 1 and r["seeds"][0]["nuv"] == 6
        assert [r["seeds"][0]["hits"][q] for q in layers] == [lh[q] for q in layers]
        # (d) hypothesis grid: t_y at a sub-bin centre, tolerance 1 um
        ty = lo + w * (11 + 1.5 * 2.0 / F)
        tight = oracle.default_config(_lib=L, uv_mode=1, uv_tol=1e-3)
        x, zone, lh, half = _stereo_event(seed, {L: ty for L in layers})
        r = oracle.seeding_event(tight, x, zone, _lib=L)
        assert len(r["seeds"]) == 1 and r["seeds"][0]["nuv"] == 6
        assert r["seeds"][0]["ty"] == pytest.approx(ty, rel=1e-9)
        return
    raise AssertionError("no upper-half track among the constructed events")


# ---------------------------------------------------------------------------
# matching final selection (Section 4.4)
# ---------------------------------------------------------------------------

def _torch_mlp(nn, F):
    """The 8-32-1 ghost network evaluated with torch's linear / relu /
    sigmoid in float64 (a library statement of the same network)."""
    import torch
    w = torch.as_tensor(np.asarray(nn, np.float64))
    mean, inv = w[:8], w[8:16]
    W1, b1, w2, b2 = w[16:272].reshape(32, 8), w[272:304], w[304:336].reshape(1, 32), w[336:337]
    x = (torch.as_tensor(np.asarray(F, np.float64)) - mean) * inv
    h = torch.nn.functional.relu(torch.nn.functional.linear(x, W1, b1))
    return torch.sigmoid(torch.nn.functional.linear(h, w2, b2))[:, 0].numpy()


def _probe_weights(k, scale=1.0):
    """Weights whose output is sigmoid(scale * f_k) for input k (two hidden
    ReLU units carry +f_k and -f_k)."""
    nn = np.zeros(337, np.float32)
    nn[8:16] = 1.0
    W1 = np.zeros((32, 8), np.float32)
    W1[0, k], W1[1, k] = scale, -scale
    nn[16:272] = W1.ravel()
    nn[304], nn[305] = 1.0, -1.0
    return nn


def check_final_selection(L=None, zmx=None, n_events=6):
    """(1) The network equals torch's evaluation on random inputs; (2) each
    of the eight inputs, read back through probe weights, equals its
    definition (the vectorised matching quantities of Section 4, eta =
    -ln tan(theta/2) with tan(theta) the VELO slope, the SciFi hit count);
    (3) with the seeded stand-in weights the kept pairs follow the two rules
    of Section 4.4 (ghost probability below 0.8; a pair sharing its VELO
    segment with a pair whose probability is lower by at least 0.05 is
    dropped), checked pair by pair."""
    from synth import ghost_nn_weights
    rng = np.random.default_rng(5)
    nn = ghost_nn_weights()
    F = np.column_stack([rng.normal(5200, 300, 64), rng.normal(0, 10, 64), rng.normal(0, 60, 64),
                         rng.normal(0, 0.2, 64), rng.normal(0, 0.01, 64), rng.uniform(0, 2, 64),
                         rng.uniform(1, 6, 64), rng.integers(9, 13, 64)])
    got = np.array([oracle.ghost_nn(nn, f, _lib=L) for f in F])
    assert np.allclose(got, _torch_mlp(nn, F), rtol=1e-12, atol=1e-15)
    cfg = oracle.default_config(_lib=L, final_sel=1)
    if zmx is not None:
        oracle.apply(cfg, {"zmx": zmx})
    b = workload("match_stress", n_events=n_events)
    res = oracle.seeding_batch(cfg, b, _lib=L)
    nshared = ndropped = 0
    for e, r in enumerate(res):
        s = r["seeds"]
        st = np.stack([s["x_s"], s["y_s"], s["tx_s"], s["ty_s"]], 1)
        velo = b.velo_of(e).astype(np.float64)
        nh = (s["nx"] + s["nuv"]).astype(np.int32)
        m = oracle.matching_event(cfg, velo, st, _lib=L)
        vi = m["velo_idx"]
        ok = vi >= 0
        if not ok.any():
            continue
        # the inputs by definition
        V, S = velo[vi[ok]], st[ok]
        dtx, dty = V[:, 2] - S[:, 2], V[:, 3] - S[:, 3]
        A, B, Cc, D, E = (cfg.zmx[k] for k in range(5))
        zm = A + B * np.abs(dtx) + Cc * dtx ** 2 + D * np.abs(S[:, 0]) + E * V[:, 2] ** 2
        dx = (V[:, 0] + (zm - cfg.z_velo) * V[:, 2]) - (S[:, 0] + (zm - cfg.z_state) * S[:, 2])
        dy = (V[:, 1] + (cfg.z_match_y - cfg.z_velo) * V[:, 3]) - (S[:, 1] + (cfg.z_match_y - cfg.z_state) * S[:, 3])
        theta = np.arctan(np.hypot(V[:, 2], V[:, 3]))
        eta = -np.log(np.tan(theta / 2))
        want = np.column_stack([zm, dx, dy, dtx, dty, m["chi2"][ok], eta, nh[ok]])
        for k, sc in enumerate((2.0 ** -10, 0.125, 2.0 ** -6, 1.0, 8.0, 1.0, 0.25, 0.125)):  # exact in float32
            f = oracle.final_selection(cfg, velo, st, nh, _probe_weights(k, sc), vi, m["chi2"], _lib=L)
            p = f["ghost_prob"][ok]
            assert np.allclose(np.log(p / (1 - p)) / sc, want[:, k], rtol=1e-9, atol=1e-9), k
        # the selection rules with the stand-in weights
        f = oracle.final_selection(cfg, velo, st, nh, nn, vi, m["chi2"], _lib=L)
        p = _torch_mlp(nn, want)
        assert np.allclose(f["ghost_prob"][ok], p, rtol=1e-12, atol=1e-15)
        idx = np.nonzero(ok)[0]
        kept = {int(i): int(vi[i]) for i, pi in zip(idx, p) if pi < cfg.ghost_max}
        pp = dict(zip(idx.tolist(), p.tolist()))
        expect = np.full(len(vi), -1, np.int32)
        for i, v in kept.items():
            others = [j for j, w in kept.items() if w == v and j != i]
            nshared += bool(others)
            if all(pp[i] - pp[j] < cfg.clone_margin for j in others):
                expect[i] = v
            else:
                ndropped += 1
        assert np.array_equal(f["velo_idx"], expect)
        assert np.all(f["ghost_prob"][~ok] == 1.0)
    assert nshared > 0 and ndropped > 0


# ---------------------------------------------------------------------------
# UT hits of the Long tracks (Section 4.3)
# ---------------------------------------------------------------------------

def _ut_case(seed, n_tracks=6):
    """Noise-free, unsmeared, fully efficient tracks with UT hits; the true
    seed states at z_state and the true VELO segment of each track."""
    b = make_events(1, seed=seed, tracks=("fixed", n_tracks), noise_frac=0.0, eff=1.0, sigma_x=0.0,
                    p_range=(3.5, 100.0), velo_ghosts_per_track=0.0, velo_sigma=(0, 0), ut_sigma=0.0,
                    ut_eff=1.0)
    tr = b.tracks_of(0)
    zs = 7826.0
    st = np.stack([DET.x_model(tr["a"], tr["b"], tr["c"], zs), tr["ty"] * zs, DET.x_slope(tr["b"], tr["c"], zs),
                   tr["ty"]], 1)
    # the true VELO states in float64 (the batch stores them as float32), one per track
    velo = np.stack([tr["tx_velo"] * DET.z_velo, tr["ty"] * DET.z_velo, tr["tx_velo"], tr["ty"]], 1)
    vidx = np.arange(len(tr["p"]), dtype=np.int32)
    ux, ul = b.ut_x_exact[b.ut_off[0]:b.ut_off[1]], b.ut_layer[b.ut_off[0]:b.ut_off[1]]
    gam_true = DET.ut_gamma_a + DET.ut_gamma_b * tr["q"] / (tr["p"] * 1000.0)
    return velo, tr, st, vidx, ux.copy(), ul.copy(), gam_true


def check_ut_search(L=None):
    """(1) noise-free tracks get their four UT hits and, once a hit has been
    attached, gamma_x equals the generating value (also when the first hit is
    a stereo one); (2) a hit 0.9x / 1.1x the printed window (Table
    ut_search_window_values, 1/p from the pair) from its prediction is taken
    / not taken, for the loose window of UTaX and the tight one of UTbX;
    (3) Long tracks with fewer than three UT hits are dropped."""
    const = read_golden_constants()
    cfg = oracle.default_config(_lib=L)
    for seed in (501, 502):
        velo, tr, st, vidx, ux, ul, gt = _ut_case(seed)
        r = oracle.ut_search(cfg, velo, st, vidx, ux, ul, _lib=L)
        assert np.array_equal(r["ut_hits"], tr["ut_hit"]), (r["ut_hits"], tr["ut_hit"])
        assert np.all(r["n_ut"] == 4) and np.array_equal(r["velo_idx"], vidx)
        assert np.allclose(r["gamma"], gt, rtol=1e-9, atol=1e-18)
        # without the UTaX hits the first hit is on the u layer (stereo)
        keep = ul != 0
        remap = -np.ones(len(ux), np.int64)
        remap[keep] = np.arange(keep.sum())
        r2 = oracle.ut_search(cfg, velo, st, vidx, ux[keep], ul[keep], _lib=L)
        want = np.where(tr["ut_hit"] >= 0, remap[np.maximum(tr["ut_hit"], 0)], -1)
        want[:, 0] = -1
        assert np.array_equal(r2["ut_hits"], want)
        assert np.allclose(r2["gamma"], gt, rtol=1e-9, atol=1e-18)
        # (2) window edges
        k = 0
        dz = np.array(cfg.ut_z[:]) - cfg.z_velo
        xV, yV, txV, tyV = (float(v) for v in velo[vidx[k]])
        qop = (st[k, 2] - txV) / cfg.ut_kick
        inv_p = 1000.0 * abs(qop)
        lo = [const[("ut_loose", 4 * 0 + i)] for i in range(4)]
        win_l = min(max(lo[0] + lo[1] * inv_p, lo[2]), lo[3])
        g0 = const[("ut_gamma", 0)] + const[("ut_gamma", 1)] * qop
        x_pred0 = xV + txV * dz[0] + g0 * dz[0] ** 2
        ti = [const[("ut_tight", 4 * 3 + i)] for i in range(4)]
        win_t = min(max(ti[0] + ti[1] * inv_p, ti[2]), ti[3])
        h0, h3 = tr["ut_hit"][k, 0], tr["ut_hit"][k, 3]
        for frac, inside in ((0.9, True), (1.1, False)):
            for sgn in (1.0, -1.0):
                x = ux.copy()
                x[h0] = x_pred0 + sgn * frac * win_l
                r = oracle.ut_search(cfg, velo, st[k:k + 1], vidx[k:k + 1], x, ul, _lib=L)
                assert (r["ut_hits"][0, 0] == h0) == inside
                x = ux.copy()
                x[h3] += sgn * frac * win_t  # the prediction there is exact once UTaX is attached
                r = oracle.ut_search(cfg, velo, st[k:k + 1], vidx[k:k + 1], x, ul, _lib=L)
                assert r["ut_hits"][0, 0] == h0 and (r["ut_hits"][0, 3] == h3) == inside
        # (3) the hit-count requirement: drop two or one of track k's hits
        for n_drop, kept in ((2, False), (1, True)):
            keep = np.ones(len(ux), bool)
            keep[tr["ut_hit"][k, :n_drop]] = False
            r = oracle.ut_search(cfg, velo, st[k:k + 1], vidx[k:k + 1], ux[keep], ul[keep], _lib=L)
            assert r["n_ut"][0] == 4 - n_drop and (r["velo_idx"][0] >= 0) == kept


# ---------------------------------------------------------------------------
# HLT2-style iterations in sequence with hit cleanup (Section 3.1)
# ---------------------------------------------------------------------------

SEQ3 = dict(iter_mode=1, n_iter=3, p_min_iter=[5000.0, 3000.0, 1500.0])


def check_sequential_iterations(L=None):
    """(1) noise-free tracks are found once each with their exact hits, for
    two and three iterations in sequence; (2) on Run-3-like events no hit of
    a seed is used by a seed of a later iteration (the cleanup) and every
    pass finds something; (3) one iteration in sequence equals one HLT1
    iteration; (4) each iteration's two-hit window is Eq. tolHp at its own
    p_min (numpy's root of b x0^2 + a x0 = 1/p_min)."""
    for ov in (dict(iter_mode=1), SEQ3):
        check_noise_free_recovery(L, None, n_events=3, **ov)
    cfg = oracle.default_config(_lib=L, **SEQ3)
    b = workload("run3", n_events=6)
    res = oracle.seeding_batch(cfg, b, _lib=L)
    per_pass = np.zeros(3, int)
    for r in res:
        s = r["seeds"]
        for half in (0, 1):
            taken = set()
            for p in range(3):
                sel = s[(s["half"] == half) & (s["pass"] == p)]
                per_pass[p] += len(sel)
                hs = {int(h) for h in sel["hits"].ravel() if h >= 0}
                assert not (hs & taken), (half, p)
                taken |= hs
    assert (per_pass > 0).all(), per_pass
    one_seq = oracle.default_config(_lib=L, iter_mode=1, n_iter=1)
    one = oracle.default_config(_lib=L, n_iter=1)
    for e in range(3):
        x, z = b.hits_of(e)
        a = oracle.seeding_event(one_seq, x, z, _lib=L)["seeds"]
        c = oracle.seeding_event(one, x, z, _lib=L)["seeds"]
        assert sorted(map(tuple, a["hits"])) == sorted(map(tuple, c["hits"]))
    const = read_golden_constants()
    aa, bb = const[("invp_a", None)], const[("invp_b", None)]
    for it, pm in enumerate(SEQ3["p_min_iter"]):
        roots = np.roots([bb, aa, -1.0 / pm])
        x0 = min(r.real for r in roots if r.real > 0)
        z1, z3 = cfg.z[cfg.iter_layers[it][0]], cfg.z[cfg.iter_layers[it][2]]
        assert oracle.dx3max(cfg, it, _lib=L) == pytest.approx((z3 - z1) / z1 * x0, rel=1e-12)


ALL_CHECKS = (check_paper_constants, check_window_closed_forms, check_k3_chord,
              check_noise_free_recovery, check_triplets_brute_force, check_clone_kill_pairwise,
              check_tolerance_boundaries, check_matching_grid, check_hough_noise_free,
              check_hough_clusters, check_final_selection, check_ut_search, check_sequential_iterations)


# ---------------------------------------------------------------------------
# tests
# ---------------------------------------------------------------------------

def test_paper_constants():
    check_paper_constants()


def test_window_closed_forms():
    check_window_closed_forms()


def test_k3_chord_identity():
    check_k3_chord()


def test_noise_free_recovery(zmx_calibrated):
    check_noise_free_recovery(zmx=zmx_calibrated)


def test_triplets_and_candidates_brute_force():
    check_triplets_brute_force()


def test_clone_kill_pairwise():
    check_clone_kill_pairwise()


def test_tolerance_boundaries():
    check_tolerance_boundaries()


@pytest.mark.parametrize("preset", ["paper_table", "calibrated"])
def test_matching_grid(preset, zmx_calibrated):
    check_matching_grid(zmx=None if preset == "paper_table" else zmx_calibrated)


def test_unit_reading_of_invp(ocfg):
    """1/p of Eq. invp is per MeV/c: for this generator's kick (dtx = 1.2/p[GeV]
    at z = 5200 mm) a 3 GeV/c track has x0 = 5200 * 1.2 / 3 = 2080 mm, and
    the fit then returns p within 5% of 3000 MeV/c; reading it per GeV/c would
    be off by a factor 1000."""
    x0 = DET.z_kink * DET.kick_gev / 3.0
    p = 1.0 / oracle.invp(ocfg, x0)
    assert abs(p / 3000.0 - 1.0) < 0.05


def test_two_hit_window_containment(ocfg):
    """Section 3.3.2: the two-hit window holds more than 99% of true (T1, T3)
    hit pairs of tracks above p_min."""
    b = workload("run3", n_events=40)
    inside = total = 0
    for it in range(2):
        L1, L3 = ocfg.iter_layers[it][0], ocfg.iter_layers[it][2]
        z1, z3 = ocfg.z[L1], ocfg.z[L3]
        alpha, dx3 = oracle.alpha_corr(ocfg, it), oracle.dx3max(ocfg, it)
        for e in range(b.n_events):
            tr = b.tracks_of(e)
            x = b.hits_of(e)[0].astype(np.float64)
            sel = (tr["p"] > 3.0) & (tr["layer_hit"][:, L1] >= 0) & (tr["layer_hit"][:, L3] >= 0)
            x1 = x[tr["layer_hit"][sel, L1]]
            x3 = x[tr["layer_hit"][sel, L3]]
            c = (z3 + alpha) / z1 * x1
            inside += np.sum((x3 >= c - dx3) & (x3 <= c + dx3))
            total += len(x1)
    assert inside / total > 0.99


def test_uv_recovers_true_stereo_hits(ocfg):
    """A single noise-free track among noise hits of the other half: the UV step
    attaches exactly its six stereo hits and the line fit returns its ty."""
    for s in range(10):
        b = make_events(1, seed=300 + s, tracks=("fixed", 1), noise_frac=0.0, eff=1.0, sigma_x=0.0,
                        p_range=(3.5, 100), velo_ghosts_per_track=0.0, velo_sigma=(0, 0))
        x, zone = b.exact_hits_of(0)
        tr = b.tracks_of(0)
        r = oracle.seeding_event(ocfg, x, zone)
        assert len(r["seeds"]) == 1
        sd = r["seeds"][0]
        for Lx in UV_LAYERS:
            assert sd["hits"][Lx] == tr["layer_hit"][0, Lx]
        assert sd["nuv"] == 6
        assert sd["ty"] == pytest.approx(tr["ty"][0], rel=1e-10, abs=1e-13)


def test_final_selection(zmx_calibrated):
    check_final_selection(zmx=zmx_calibrated)


def test_sequential_iterations():
    check_sequential_iterations()


def test_sequential_iterations_reach_lower_momentum():
    """Section 3.1: later iterations with wider windows find lower-momentum
    tracks in a cleaned-up event.  Three iterations in sequence (p_min 5, 3,
    1.5 GeV/c) find more tracks between 2 and 3 GeV/c than HLT1's two, keep
    the efficiency above 3 GeV/c within 0.5%, and form fewer pairs."""
    b = workload("run3", n_events=30)
    out = {}
    for name, ov in (("hlt1", {}), ("seq3", SEQ3)):
        res = oracle.seeding_batch(oracle.default_config(**ov), b)
        eff = {}
        for lo, hi in ((2.0, 3.0), (3.0, 1e9)):
            nt = nf = 0
            for e, r in enumerate(res):
                tr = b.tracks_of(e)
                seen = set()
                for s in r["seeds"]:
                    t, pur = truth_track_of(b, e, s["hits"])
                    if t >= 0 and pur >= 0.7:
                        seen.add(t)
                good = (tr["p"] > lo) & (tr["p"] <= hi) & ((tr["layer_hit"] >= 0).sum(1) >= 10)
                nt += good.sum()
                nf += sum((b.trk_off[e] + k) in seen for k in np.nonzero(good)[0])
            eff[lo] = nf / nt
        out[name] = (eff, sum(r["counters"]["pairs"] for r in res))
    assert out["seq3"][0][2.0] > out["hlt1"][0][2.0] + 0.05, out
    assert out["seq3"][0][3.0] > out["hlt1"][0][3.0] - 0.005, out
    assert out["seq3"][1] < out["hlt1"][1], out


def test_ut_search():
    check_ut_search()


def test_ut_efficiency_on_synthetic_events(zmx_calibrated):
    """On the Run-3-like sample almost every true Long track keeps at least
    three UT hits, and the attached hits are mostly the track's own."""
    b = workload("run3", n_events=20)
    cfg = oracle.default_config(zmx=zmx_calibrated)
    res = oracle.seeding_batch(cfg, b)
    n_true = n_kept = n_hit = n_own = 0
    for e, r in enumerate(res):
        s = r["seeds"]
        st = np.stack([s["x_s"], s["y_s"], s["tx_s"], s["ty_s"]], 1)
        m = oracle.matching_event(cfg, b.velo_of(e), st)
        ux, ul = b.ut_of(e)
        u = oracle.ut_search(cfg, b.velo_of(e), st, m["velo_idx"], ux, ul)
        vt = b.velo_track[b.velo_off[e]:b.velo_off[e + 1]]
        utt = b.ut_track[b.ut_off[e]:b.ut_off[e + 1]]
        for k in np.nonzero(m["velo_idx"] >= 0)[0]:
            t = vt[m["velo_idx"][k]]
            if t < 0 or truth_track_of(b, e, s["hits"][k])[0] != t:
                continue
            n_true += 1
            n_kept += u["velo_idx"][k] >= 0
            hs = u["ut_hits"][k][u["ut_hits"][k] >= 0]
            n_hit += len(hs)
            n_own += int(np.sum(utt[hs] == t))
    assert n_kept / n_true > 0.98 and n_own / n_hit > 0.9, (n_kept / n_true, n_own / n_hit)


def test_hough_noise_free():
    check_hough_noise_free()


def test_hough_cluster_cases():
    check_hough_clusters()


def test_hough_similar_to_iterative():
    """Section 3.4: the two UV approaches have similar tracking performance.
    On the Run-3-like sample the Hough-cluster variant's efficiency above
    5 GeV/c is within 1% of the iterative one's, with few ghosts."""
    b = workload("run3", n_events=30)
    eff = {}
    for mode in (0, 1):
        cfg = oracle.default_config(uv_mode=mode)
        res = oracle.seeding_batch(cfg, b)
        ntrue = nfound = nseed = nghost = 0
        for e, r in enumerate(res):
            tr = b.tracks_of(e)
            seen = set()
            for sd in r["seeds"]:
                nseed += 1
                t, pur = truth_track_of(b, e, sd["hits"])
                if t < 0 or pur < 0.7:
                    nghost += 1
                else:
                    seen.add(t)
            good = (tr["p"] > 5.0) & ((tr["layer_hit"] >= 0).sum(1) >= 10)
            ntrue += good.sum()
            nfound += sum((b.trk_off[e] + k) in seen for k in np.nonzero(good)[0])
        eff[mode] = nfound / ntrue
        assert nghost / nseed < 0.02
    assert abs(eff[1] - eff[0]) < 0.01, eff


def test_synthetic_efficiency_targets(ocfg, zmx_calibrated):
    """Section 5 targets on the synthetic Run-3-like sample: seeding efficiency
    above 95% for tracks above 5 GeV/c, about half the x-z candidates are
    duplicates before clone killing and at most 2% after, few ghosts, and
    matching picks the true VELO segment for more than 90% of true seeds."""
    b = workload("run3", n_events=40)
    cfg = oracle.default_config(zmx=zmx_calibrated)
    res = oracle.seeding_batch(cfg, b, cands=True)
    ntrue = nfound = nseed = nghost = nclone = 0
    ncand = ndup = 0
    nmatch_ok = nmatch_tot = 0
    for e, r in enumerate(res):
        tr = b.tracks_of(e)
        seen = set()
        for s in r["seeds"]:
            nseed += 1
            t, pur = truth_track_of(b, e, s["hits"])
            if t < 0 or pur < 0.7:
                nghost += 1
                continue
            nclone += t in seen
            seen.add(t)
        good = (tr["p"] > 5.0) & ((tr["layer_hit"] >= 0).sum(1) >= 10)
        ntrue += good.sum()
        nfound += sum((b.trk_off[e] + k) in seen for k in np.nonzero(good)[0])
        hs = [tuple(c["hits"]) for c in r["cands"]]
        ncand += len(hs)
        ndup += len(hs) - len(set(hs))
        s = r["seeds"]
        st = np.stack([s["x_s"], s["y_s"], s["tx_s"], s["ty_s"]], 1).astype(np.float32)
        m = oracle.matching_event(cfg, b.velo_of(e), st)
        vt = b.velo_track[b.velo_off[e]:b.velo_off[e + 1]]
        for k, sd in enumerate(s):
            t, pur = truth_track_of(b, e, sd["hits"])
            if t < 0 or pur < 0.7:
                continue
            nmatch_tot += 1
            nmatch_ok += m["velo_idx"][k] >= 0 and vt[m["velo_idx"][k]] == t
    assert nfound / ntrue > 0.95
    assert 0.3 < ndup / ncand < 0.7
    assert nclone / nseed < 0.02
    assert nghost / nseed < 0.05
    assert nmatch_ok / nmatch_tot > 0.9


def test_invalid_input_rejected(ocfg):
    x = np.array([1.0, 2.0])
    assert oracle.seeding_event(ocfg, x, np.array([0, 24], np.int32))["status"] == -1
    assert oracle.seeding_event(ocfg, np.array([np.nan, 1.0]), np.array([0, 1], np.int32))["status"] == -1
    bad = oracle.default_config(n_uv_min=1)
    assert oracle.seeding_event(bad, x, np.array([0, 1], np.int32))["status"] == -1


def test_empty_event(ocfg):
    r = oracle.seeding_event(ocfg, np.zeros(0), np.zeros(0, np.int32), cands=True, trips=True)
    assert r["status"] == 0 and len(r["seeds"]) == 0 and len(r["cands"]) == 0
    m = oracle.matching_event(ocfg, np.zeros((0, 4)), np.zeros((3, 4)))
    assert list(m["velo_idx"]) == [-1, -1, -1]
