"""Pins of the oracle's cut ledger.

GPU/oracle differences are excused only by ledger entries within a margin tau
of their thresholds, so the ledger itself needs a pin: for every kind of
decision the GPU and the oracle can take differently, an event is built in
which that decision sits at a KNOWN relative margin m (1e-6 and 1e-4), and the
check asserts that

  * the ledger holds an entry of that kind naming the hits (or the seed and
    VELO indices) the decision is made on, with a margin within 1% of m, and
  * the decision itself flips where the construction says it does: the input
    moved to the other side of the threshold by the same distance changes the
    observable result (a pair, a triplet, a chosen hit, a seed, a match).

A margin is the distance of the decisive quantity to its threshold, relative to
the magnitude of the numbers the decision is made from: for a window in x the
largest of the hit position and the terms that form the bound; for a cut on a
chi2 the threshold; for a tie the larger of the two values (position ties: the
prediction's magnitude, at least 1 mm).  The events are built from the track
model of Section 3.1 (x = a + b zb + c zb^2 (1 + d zb)) and the stereo hit model
(x_hit = x(z) - y(z) dxdy), independently of the oracle's arithmetic; the
window constants the constructions use (Eq. tolHp, Eq. alphacorr, k3, Eq.
invp) are themselves pinned by test_oracle_pins.py's closed forms.

The checks take the oracle library handle so that test_oracle_mutations.py can
run them against copies of the oracle with a planted mistake.
"""

import math

import numpy as np
import pytest

import oracle
from synth import Detector

DET = Detector()
Z = DET.z_arr
T = DET.dxdy
X_LAYERS = (0, 3, 4, 7, 8, 11)
UV_LAYERS = (1, 2, 5, 6, 9, 10)
KIND = {v: k for k, v in oracle.LEDGER_KINDS.items()}
MARGINS = (1e-6, 1e-4)
TAU_RECORD = 1e-3


def track(p_gev=10.0, q=1, txv=0.05, ty=0.1):
    """(a, b, c, ty) of a track from the origin with the benchmark
    generator's kink: slope txv up to z_kink, txv + q * kick / p after it,
    SciFi curvature kappa_c q / p."""
    b = txv + q * DET.kick_gev / p_gev
    a = txv * DET.z_kink + b * (DET.z_ref - DET.z_kink)
    c = DET.kappa_c * q / (p_gev * 1000.0)
    return (a, b, c, ty)


def fcub(z):
    zb = z - DET.z_ref
    return zb * zb * (1.0 + DET.d_ratio * zb)


def x_track(trk, z):
    a, b, c, _ = trk
    return a + b * (z - DET.z_ref) + c * fcub(z)


def hit_x(trk, L):
    """Measured coordinate of the track in layer L (x at y = 0 along the fibre)."""
    return x_track(trk, Z[L]) - trk[3] * Z[L] * T[L]


def xscale(trk, z):
    """Largest of the terms that form the track's x at z."""
    a, b, c, _ = trk
    return max(abs(a), abs(b * (z - DET.z_ref)), abs(c * fcub(z)))


class Ev:
    """A hand-built event: hits are appended in order, a hit's index is its
    position."""

    def __init__(self):
        self.x, self.zone = [], []

    def add(self, L, x, half=1):
        self.x.append(float(x))
        self.zone.append(2 * L + half)
        return len(self.x) - 1

    def add_track(self, trk, skip=()):
        half = 1 if trk[3] >= 0 else 0
        return {L: self.add(L, hit_x(trk, L), half) for L in range(12) if L not in skip}

    def copy(self):
        e = Ev()
        e.x, e.zone = list(self.x), list(self.zone)
        return e

    def run(self, cfg, L, **kw):
        return oracle.seeding_event(cfg, np.array(self.x), np.array(self.zone, np.int32), ledger_tau=TAU_RECORD,
                                    cands=True, _lib=L, **kw)


def entries(led, kind, hits):
    """Ledger entries of `kind` whose hit list starts with `hits`."""
    sel = led[led["kind"] == KIND[kind]]
    n = len(hits)
    return [e for e in sel if [int(h) for h in e["hits"][:n]] == [int(h) for h in hits]]


def assert_margin(led, kind, hits, m, what=""):
    es = entries(led, kind, hits)
    assert es, f"no {kind} entry for hits {list(hits)} {what}"
    got = [float(e["margin"]) for e in es]
    assert any(abs(g - m) <= 0.01 * m for g in got), (kind, what, m, got)


def slot_hits(H):
    """A track's x-layer hits in x-slot order (layers 0, 3, 4, 7, 8, 11)."""
    return [H[L] for L in X_LAYERS]


def base_config(L, **ov):
    return oracle.default_config(_lib=L, **ov)


# ---------------------------------------------------------------------------
# the checks
# ---------------------------------------------------------------------------

def check_ledger_xz_windows(L=None):
    """Two-hit window (Eqs. tolHp, alphacorr) and third-hit band (Section
    3.3.3): a hit at relative distance m inside the window edge."""
    cfg = base_config(L)
    A = track()
    for m in MARGINS:
        ev = Ev()
        H = ev.add_track(A)
        # --- two-hit window of iteration 0: (T1, T2, T3) = layers (0, 4, 11)
        z1, z3 = Z[0], Z[11]
        x1 = hit_x(A, 0)
        xc = (z3 + oracle.alpha_corr(cfg, 0, _lib=L)) / z1 * x1
        dx3 = oracle.dx3max(cfg, 0, _lib=L)
        assert xc > 0
        S3 = abs(xc) + dx3  # the window's upper edge is xc + dx3 = S3 > |x3|
        hi = xc + dx3
        pairs = {}
        for side in (-1.0, 1.0):
            e2 = ev.copy()
            hn = e2.add(11, hi + side * m * S3)
            r = e2.run(cfg, L)
            pairs[side] = r["counters"]["pairs"]
            assert_margin(r["ledger"], "pair_win", [H[0], hn], m, f"side {side}")
        assert pairs[-1.0] == pairs[1.0] + 1  # inside: one pair more
        # --- third-hit band of the true pair (layer-0 hit, layer-11 hit)
        x3 = hit_x(A, 11)
        z2 = Z[4]
        t13 = (x3 - x1) / (z3 - z1)
        x0 = x1 - z1 * t13
        invp = oracle.invp(cfg, x0, _lib=L)
        s = 1.0 if x0 > 0 else -1.0
        k3 = oracle.k3(cfg, 0, _lib=L)
        w1, w3 = (z3 - z2) / (z3 - z1), (z2 - z1) / (z3 - z1)
        c0 = cfg.c_nsigma * cfg.sigma_x * math.sqrt(1 + w1 * w1 + w3 * w3) / abs(k3)
        ulo = cfg.m_lo * cfg.kappa_c * invp - c0
        uhi = cfg.m_hi * cfg.kappa_c * invp + c0
        base = x1 + (z2 - z1) * t13
        xa, xb = base + k3 * (-s * ulo), base + k3 * (-s * uhi)
        hi2 = max(xa, xb)
        S2 = abs(base) + abs(k3) * max(abs(ulo), abs(uhi))
        assert abs(hi2) <= S2
        trips = {}
        for side in (-1.0, 1.0):
            e2 = ev.copy()
            hn = e2.add(4, hi2 + side * m * S2)
            r = e2.run(cfg, L)
            trips[side] = r["counters"]["triplets"]
            assert_margin(r["ledger"], "trip_win", [H[0], H[11], hn], m, f"side {side}")
        assert trips[-1.0] == trips[1.0] + 1


def check_ledger_extension(L=None):
    """Extension to the other x-layers (1 mm, Section 3.2): the hit of layer 8
    at relative distance m inside / outside the tolerance of the exact 3-hit
    prediction, and two hits whose distances to it differ by m."""
    cfg = base_config(L, chi2x_max=1e12)  # keep every candidate to see the chosen hit
    A = track()
    xp = hit_x(A, 8)
    for m in MARGINS:
        # tolerance
        got = {}
        for side in (-1.0, 1.0):
            ev = Ev()
            H = ev.add_track(A, skip=(8,))
            S = max(xscale(A, Z[8]), abs(xp + cfg.ext_tol))
            h8 = ev.add(8, xp + cfg.ext_tol + side * m * S)
            r = ev.run(cfg, L)
            assert_margin(r["ledger"], "ext_tol", [H[0], H[4], H[11], h8], m, f"side {side}")
            c = [c for c in r["cands"] if c["iter"] == 0 and c["h1"] == H[0] and c["h2"] == H[4]
                 and c["h3"] == H[11]]
            assert len(c) == 1
            got[side] = int(c[0]["hits"][4])
        assert got[-1.0] == h8 and got[1.0] == -1
        # tie between two hits 0.3 mm either side of the prediction
        got = {}
        for side in (-1.0, 1.0):
            ev = Ev()
            H = ev.add_track(A, skip=(8,))
            d = 0.3
            sc = max(xscale(A, Z[8]), 1.0)
            ha = ev.add(8, xp - d)
            hb = ev.add(8, xp + d + side * m * sc)
            r = ev.run(cfg, L)
            best, second = (ha, hb) if side > 0 else (hb, ha)
            assert_margin(r["ledger"], "ext_tie", [H[0], H[4], H[11], best, second], m, f"side {side}")
            c = [c for c in r["cands"] if c["iter"] == 0 and c["h1"] == H[0] and c["h2"] == H[4]
                 and c["h3"] == H[11]]
            got[side] = int(c[0]["hits"][4])
        assert got[1.0] == ha and got[-1.0] == hb


def check_ledger_chi2x(L=None):
    """The chi2/ndf cut (Section 3.3): one hit of a noise-free 6-hit track
    moved by D; for the unweighted 6-point least-squares fit on the basis
    (1, zb, f(zb)) the chi2 is D^2 (1 - H_kk) / sigma^2, with H the hat
    matrix (numpy), so D puts chi2/ndf at (1 -/+ m) of the threshold."""
    cfg = base_config(L)
    A = track()
    zs = np.array([Z[Lx] for Lx in X_LAYERS])
    Bm = np.stack([np.ones(6), zs - DET.z_ref, fcub(zs)], 1)
    Hat = Bm @ np.linalg.solve(Bm.T @ Bm, Bm.T)
    k = X_LAYERS.index(8)
    for m in MARGINS:
        got = {}
        for side in (-1.0, 1.0):
            q = cfg.chi2x_max * (1.0 + side * m)
            D = cfg.sigma_x * math.sqrt(3.0 * q / (1.0 - Hat[k, k]))
            ev = Ev()
            H = ev.add_track(A, skip=(8,))
            H[8] = ev.add(8, hit_x(A, 8) + D)
            r = ev.run(cfg, L)
            assert_margin(r["ledger"], "chi2x", slot_hits(H), m, f"side {side}")
            got[side] = any(sorted(int(h) for h in c["hits"]) == sorted(slot_hits(H)) for c in r["cands"])
        assert got[-1.0] and not got[1.0]


def check_ledger_clone(L=None):
    """Clone-killing score tie (Eq. seed_clone_score): two noise-free tracks
    crossing at their layer-7 hit, with curvatures in the ratio 1 : 1 + e so
    that their scores (|c_x|, chi2 = 0) differ by the relative margin m; the
    loser's entry names both hit sets."""
    cfg = base_config(L)
    A = track()
    for m in MARGINS:
        eps = m / (1.0 - m)  # |sA - sB| / max(sA, sB) = eps / (1 + eps) = m
        a, b, c, _ = A
        zb7 = Z[7] - DET.z_ref
        bB, cB = b - 0.02, c * (1.0 + eps)
        aB = a + (b - bB) * zb7 + (c - cB) * fcub(Z[7])
        B = (aB, bB, cB, 0.12)
        assert abs(x_track(B, Z[7]) - x_track(A, Z[7])) < 1e-9
        ev = Ev()
        HA = ev.add_track(A)
        HB = ev.add_track(B, skip=(7,))
        HB[7] = HA[7]
        r = ev.run(cfg, L)
        found = {tuple(sorted(int(h) for h in s["hits"] if h >= 0)) for s in r["seeds"]}
        assert tuple(sorted(HA.values())) in found and tuple(sorted(HB.values())) in found
        assert_margin(r["ledger"], "clone", slot_hits(HB) + slot_hits(HA), m)
        # the better score owns the shared hit: swap the curvatures and the
        # entry names the other candidate as the loser
        cA2 = c * (1.0 + eps) ** 2
        A2 = (a + (c - cA2) * fcub(Z[7]), b, cA2, A[3])
        ev = Ev()
        HA = ev.add_track(A2)
        HB = ev.add_track(B, skip=(7,))
        HB[7] = HA[7]
        r = ev.run(cfg, L)
        # |sA2 - sB| / max = (cA2 - cB) / cA2 = eps / (1 + eps) = m
        assert_margin(r["ledger"], "clone", slot_hits(HA) + slot_hits(HB), m, "swapped")


def check_ledger_uv(L=None):
    """UV seeding (Section 3.4): the first-layer y window, the 2 mm tolerance,
    a closest-hit tie, and the choice between two complete chains whose
    chi2_y are in the ratio (1 + e)^2."""
    cfg = base_config(L)
    A = track()
    a, b, c, ty = A
    half = 1
    ylo, yhi = -cfg.uv_y_overlap, cfg.uv_y_max
    Lu = UV_LAYERS[0]  # pass A starts on layer 1
    XI, tI = x_track(A, Z[Lu]), T[Lu]
    for m in MARGINS:
        # --- first-layer window: a hit of layer 1 whose y sits m inside / outside y_max
        S = max(xscale(A, Z[Lu]), abs(XI - yhi * tI), abs(yhi * tI))
        n_init = {}
        for side in (-1.0, 1.0):
            ev = Ev()
            H = ev.add_track(A)
            y = yhi + side * m * S / abs(tI)
            hn = ev.add(Lu, XI - y * tI, half)
            r = ev.run(cfg, L)
            n_init[side] = r["counters"]["uv_init"]
            assert_margin(r["ledger"], "uv_win", slot_hits(H) + [hn], m, f"side {side}")
        assert n_init[-1.0] == n_init[1.0] + 1
        # --- tolerance on the last stereo layer (10): prediction exact for a
        # noise-free track (every ty step averages exact values)
        Lt = UV_LAYERS[5]
        xp = hit_x(A, Lt)
        sc = max(xscale(A, Z[Lt]), abs(T[Lt] * ty * Z[Lt]))
        nuv = {}
        for side in (-1.0, 1.0):
            ev = Ev()
            H = ev.add_track(A, skip=(Lt,))
            S = max(sc, abs(xp + cfg.uv_tol))
            h10 = ev.add(Lt, xp + cfg.uv_tol + side * m * S, half)
            r = ev.run(cfg, L)
            assert_margin(r["ledger"], "uv_tol", slot_hits(H) + [H[Lu], h10], m, f"side {side}")
            assert len(r["seeds"]) == 1
            nuv[side] = int(r["seeds"][0]["nuv"])
        assert nuv[-1.0] == 6 and nuv[1.0] == 5
        # --- tie on layer 10: hits 0.5 mm either side of the prediction
        got = {}
        for side in (-1.0, 1.0):
            ev = Ev()
            H = ev.add_track(A, skip=(Lt,))
            ha = ev.add(Lt, xp - 0.5, half)
            hb = ev.add(Lt, xp + 0.5 + side * m * max(sc, 1.0), half)
            r = ev.run(cfg, L)
            best, second = (ha, hb) if side > 0 else (hb, ha)
            assert_margin(r["ledger"], "uv_tie", slot_hits(H) + [H[Lu], best, second], m, f"side {side}")
            got[side] = int(r["seeds"][0]["hits"][Lt])
        assert got[1.0] == ha and got[-1.0] == hb
        # --- chain choice: the layer-1 hit moved by +D and a second layer-1 hit
        # at -D (1 + e): the two pass-A chains share the other five exact hits,
        # so their chi2_y are in the ratio (1 + e)^2 and the relative margin is
        # 1 - (1 + e)^-2 = m
        D = 0.2
        e1 = (1.0 - m) ** -0.5 - 1.0
        for side in (1.0, -1.0):
            ev = Ev()
            H = ev.add_track(A, skip=(Lu,))
            x1t = hit_x(A, Lu)
            hp = ev.add(Lu, x1t + D * (1.0 if side > 0 else (1.0 + e1)), half)
            hm = ev.add(Lu, x1t - D * ((1.0 + e1) if side > 0 else 1.0), half)
            r = ev.run(cfg, L)
            best, other = (hp, hm) if side > 0 else (hm, hp)
            rest = [H[Lx] for Lx in UV_LAYERS[1:]]
            assert_margin(r["ledger"], "uv_sel", [best] + rest + [other] + rest, m, f"side {side}")
            assert len(r["seeds"]) == 1 and int(r["seeds"][0]["hits"][Lu]) == best


def check_ledger_matching(L=None, zmx=None):
    """Matching (Section 4.2): preselection cut, chi2_match cut and the
    best-pair argmin, on a seed state and VELO segments that are collinear
    in x (dx = dtx = dty = 0) and offset in y at the y matching plane, so
    that chi2_match = dy^2 / tol_y with tol_y = 0.2 (1.59^2 + 212.1^2 rho)."""
    cfg = base_config(L)
    if zmx is not None:
        oracle.apply(cfg, {"zmx": zmx})
    tx, ty = 0.1, 0.05
    seed = np.array([[tx * cfg.z_state + 3.0, ty * cfg.z_state - 1.0, tx, ty]])

    def velo_dy(dy):
        return [tx * cfg.z_velo + 3.0, ty * cfg.z_velo - 1.0 + dy, tx, ty]

    tol_y = 0.2 * (1.59 ** 2 + 212.1 ** 2 * (tx * tx + ty * ty))
    cut_y = cfg.presel[1] * cfg.presel_scale
    for m in MARGINS:
        npre, idx = {}, {}
        for side in (-1.0, 1.0):
            r = oracle.matching_event(cfg, np.array([velo_dy(cut_y * (1.0 + side * m))]), seed,
                                      ledger_tau=TAU_RECORD, _lib=L)
            npre[side] = r["counters"]["match_presel"]
            assert_margin(r["ledger"], "m_presel", [0, 0], m, f"side {side}")
            dy = math.sqrt(cfg.chi2_match_max * (1.0 + side * m) * tol_y)
            r = oracle.matching_event(cfg, np.array([velo_dy(dy)]), seed, ledger_tau=TAU_RECORD, _lib=L)
            idx[side] = int(r["velo_idx"][0])
            assert_margin(r["ledger"], "m_chi2", [0, 0], m, f"side {side}")
        assert npre[-1.0] == 1 and npre[1.0] == 0
        assert idx[-1.0] == 0 and idx[1.0] == -1
        # argmin: chi2 0.2 and 0.2 (1 + e) with e / (1 + e) = m
        eps = m / (1.0 - m)
        dy1 = math.sqrt(0.2 * tol_y)
        for side in (1.0, -1.0):
            dy2 = dy1 * math.sqrt(1.0 + eps) if side > 0 else dy1 / math.sqrt(1.0 + eps)
            r = oracle.matching_event(cfg, np.array([velo_dy(dy1), velo_dy(dy2)]), seed,
                                      ledger_tau=TAU_RECORD, _lib=L)
            best, second = (0, 1) if side > 0 else (1, 0)
            assert int(r["velo_idx"][0]) == best
            assert_margin(r["ledger"], "m_tie", [0, best, second], m, f"side {side}")


ALL_CHECKS = (check_ledger_xz_windows, check_ledger_extension, check_ledger_chi2x, check_ledger_clone,
              check_ledger_uv, check_ledger_matching)


# ---------------------------------------------------------------------------
# tests
# ---------------------------------------------------------------------------

def test_ledger_xz_windows():
    check_ledger_xz_windows()


def test_ledger_extension():
    check_ledger_extension()


def test_ledger_chi2x():
    check_ledger_chi2x()


def test_ledger_clone():
    check_ledger_clone()


def test_ledger_uv():
    check_ledger_uv()


@pytest.mark.parametrize("preset", ["calibrated", "paper_table"])
def test_ledger_matching(preset, zmx_calibrated):
    check_ledger_matching(zmx=None if preset == "paper_table" else zmx_calibrated)
