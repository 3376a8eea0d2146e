"""Seeded synthetic LHCb-like events with known truth.

Physics model of the toy detector (all lengths in mm, momenta in GeV/c unless
stated):

* A charged particle leaves the origin with slopes (tx_V, ty).  In the VELO it
  is a straight line; its state is recorded at z = z_velo.
* The dipole is a single kink at z = z_kink that changes the x slope by
  dtx = q * kick_gev / p.
* Downstream of the kink the x-z trajectory is the post-kink line plus a small
  curvature term from the residual field inside the SciFi:
      x(z) = a + b*dz + c*dz^2*(1 + d_ratio*dz),  dz = z - z_ref,
  where (a, b) is the post-kink line at z_ref and c = kappa_c * q / p[MeV].
  This is the track model of the paper's Eq. (trackequation); the generator
  only samples from it.
* The y-z trajectory is the straight line y(z) = ty * z (no bending in y).
* A SciFi layer at z_l with stereo slope dxdy_l measures the x at which the
  fibre through the particle crosses y = 0: x_hit = x(z_l) - y(z_l)*dxdy_l,
  smeared by N(0, sigma_x) and kept with probability `eff`.
* Noise hits are uniform in x over the acceptance, on a random layer and half.
* Hits of an event are shuffled, so the event-local hit index carries no
  information.

The detector half of a hit is 1 when the particle is at y >= 0 and 0 below.
A hit's zone id is 2*layer + half.

Nothing in this module reconstructs anything: it contains no search window, fit
or selection of the method.  The z_match calibration at the bottom follows the
paper's own prescription (Section 4.1: fit the kink-position model to the
intersections of true VELO and true SciFi straight-line segments) and produces
input constants for the matching step.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, Optional

import numpy as np

N_LAYERS = 12


@dataclass(frozen=True)
class Detector:
    """Toy SciFi + VELO geometry.

    Layer z positions and the x-u-v-x ordering are those of the benchmark
    workloads (three stations of four layers, stereo +-5 degrees); z_ref and
    d_ratio are the track-model reference point and cubic-correction
    coefficient the events are generated with.
    """

    z: tuple = (7826.0, 7896.0, 7966.0, 8036.0,
                8508.0, 8578.0, 8648.0, 8718.0,
                9193.0, 9263.0, 9333.0, 9403.0)
    stereo_sign: tuple = (0, +1, -1, 0, 0, +1, -1, 0, 0, +1, -1, 0)
    stereo_angle_deg: float = 5.0
    z_ref: float = 8520.0
    d_ratio: float = -2.6e-4
    z_velo: float = 770.0
    z_kink: float = 5200.0
    kick_gev: float = 1.2
    kappa_c: float = 1.0e-2
    x_acc: float = 3200.0
    y_acc: float = 2500.0
    tx_max: float = 0.3
    ty_max: float = 0.25
    # UT (four layers x-u-v-x in front of the magnet).  Between the VELO and
    # the UT a track bends as x(z) = x_V + tx_V dz + gamma dz^2 (dz = z -
    # z_velo) with gamma = ut_gamma_a + ut_gamma_b * q/p (per MeV), the
    # parametrisation the reconstruction uses; the SciFi segment is not
    # affected (the bend is folded into the kink).
    ut_z: tuple = (2327.5, 2372.5, 2597.5, 2642.5)
    ut_stereo_sign: tuple = (0, +1, -1, 0)
    ut_gamma_a: float = 7.707063e-11
    ut_gamma_b: float = -7.817364e-3
    ut_x_acc: float = 900.0

    @property
    def z_arr(self) -> np.ndarray:
        return np.asarray(self.z, dtype=np.float64)

    @property
    def dxdy(self) -> np.ndarray:
        t = math.tan(math.radians(self.stereo_angle_deg))
        return np.asarray([s * t for s in self.stereo_sign], dtype=np.float64)

    def x_model(self, a, b, c, z):
        dz = np.asarray(z, dtype=np.float64) - self.z_ref
        return a + b * dz + c * dz * dz * (1.0 + self.d_ratio * dz)

    def x_slope(self, b, c, z):
        dz = np.asarray(z, dtype=np.float64) - self.z_ref
        return b + c * (2.0 * dz + 3.0 * self.d_ratio * dz * dz)


DEFAULT_DETECTOR = Detector()


@dataclass
class EventBatch:
    """Flat, CSR-organised batch of events.

    Hits (length N):      x (float32), z (float32), dxdy (float32), zone (int32),
                          x_exact (float64, the measured x before rounding to
                          float32), hit_track (int32, global track id or -1).
    Events:               ev_off (int64, n_events+1) into the hit arrays.
    Tracks (length T):    trk_ev, a, b, c, ty, y0, p, q, tx_velo, half,
                          layer_hit (T x 12, event-local hit index or -1).
                          trk_off (int64, n_events+1).
    VELO states (len M):  velo (float32, M x 4: x, y, tx, ty at z_velo),
                          velo_track (int32, global track id or -1 for ghosts),
                          velo_off (int64, n_events+1).
    """

    det: Detector
    ev_off: np.ndarray
    x: np.ndarray
    z: np.ndarray
    dxdy: np.ndarray
    zone: np.ndarray
    x_exact: np.ndarray
    hit_track: np.ndarray
    trk_off: np.ndarray
    trk: Dict[str, np.ndarray]
    velo_off: np.ndarray
    velo: np.ndarray
    velo_track: np.ndarray
    meta: Dict[str, object] = field(default_factory=dict)
    # UT hits (CSR per event): measured x at y = 0 along the strip, layer 0..3,
    # truth track id (-1 noise), and the float64 value before rounding
    ut_off: Optional[np.ndarray] = None
    ut_x: Optional[np.ndarray] = None
    ut_layer: Optional[np.ndarray] = None
    ut_track: Optional[np.ndarray] = None
    ut_x_exact: Optional[np.ndarray] = None

    @property
    def n_events(self) -> int:
        return int(self.ev_off.shape[0] - 1)

    @property
    def n_hits(self) -> int:
        return int(self.ev_off[-1])

    def hits_of(self, e: int):
        s, t = int(self.ev_off[e]), int(self.ev_off[e + 1])
        return self.x[s:t], self.zone[s:t]

    def exact_hits_of(self, e: int):
        s, t = int(self.ev_off[e]), int(self.ev_off[e + 1])
        return self.x_exact[s:t], self.zone[s:t]

    def ut_of(self, e: int):
        s, t = int(self.ut_off[e]), int(self.ut_off[e + 1])
        return self.ut_x[s:t], self.ut_layer[s:t]

    def velo_of(self, e: int) -> np.ndarray:
        s, t = int(self.velo_off[e]), int(self.velo_off[e + 1])
        return self.velo[s:t]

    def tracks_of(self, e: int) -> Dict[str, np.ndarray]:
        s, t = int(self.trk_off[e]), int(self.trk_off[e + 1])
        return {k: v[s:t] for k, v in self.trk.items()}

    def subset(self, events) -> "EventBatch":
        """A new batch made of the listed events (in the given order)."""
        events = np.asarray(events, dtype=np.int64)

        def gather(off, *arrays):
            parts = [np.arange(off[e], off[e + 1]) for e in events]
            idx = np.concatenate(parts) if parts else np.zeros(0, np.int64)
            counts = np.array([off[e + 1] - off[e] for e in events], dtype=np.int64)
            new_off = np.zeros(len(events) + 1, dtype=np.int64)
            np.cumsum(counts, out=new_off[1:])
            return new_off, [a[idx] for a in arrays], idx

        ev_off, (x, z, dxdy, zone, xe, ht), _ = gather(
            self.ev_off, self.x, self.z, self.dxdy, self.zone, self.x_exact, self.hit_track)
        trk_off, tv, tidx = gather(self.trk_off, *self.trk.values())
        trk = dict(zip(self.trk.keys(), tv))
        # renumber global track ids
        remap = -np.ones(self.trk_off[-1] + 1, dtype=np.int64)
        remap[tidx] = np.arange(len(tidx))
        ht = np.where(ht >= 0, remap[ht], -1).astype(np.int32)
        trk["trk_ev"] = np.repeat(np.arange(len(events)), np.diff(trk_off)).astype(np.int32)
        velo_off, (velo, vt), _ = gather(self.velo_off, self.velo, self.velo_track)
        vt = np.where(vt >= 0, remap[vt], -1).astype(np.int32)
        ut = {}
        if self.ut_off is not None:
            ut_off, (ux, ul, ut_t, uxe), _ = gather(self.ut_off, self.ut_x, self.ut_layer, self.ut_track,
                                                     self.ut_x_exact)
            ut = dict(ut_off=ut_off, ut_x=ux, ut_layer=ul, ut_track=np.where(ut_t >= 0, remap[ut_t], -1).astype(np.int32),
                      ut_x_exact=uxe)
        return EventBatch(self.det, ev_off, x, z, dxdy, zone, xe, ht, trk_off, trk,
                          velo_off, velo, vt, dict(self.meta), **ut)


# ---------------------------------------------------------------------------
# sampling helpers
# ---------------------------------------------------------------------------

def _tracks_per_event(rng, n_events, spec) -> np.ndarray:
    kind = spec[0]
    if kind == "fixed":
        return np.full(n_events, int(spec[1]), dtype=np.int64)
    if kind == "poisson":
        return rng.poisson(float(spec[1]), size=n_events).astype(np.int64)
    if kind == "lognormal":
        _, median, sigma, lo, hi = spec
        v = np.exp(rng.normal(math.log(median), sigma, size=n_events))
        return np.clip(np.rint(v), lo, hi).astype(np.int64)
    raise ValueError(f"unknown track-count spec {spec!r}")


def _sample_tracks(rng, n, det: Detector, p_range):
    """n accepted tracks (rejection sampling on slope and acceptance)."""
    out = {k: np.empty(n) for k in ("p", "q", "txv", "ty", "a", "b", "c")}
    z = det.z_arr
    dxdy = det.dxdy
    filled = 0
    lp0, lp1 = math.log(p_range[0]), math.log(p_range[1])
    while filled < n:
        m = max(2 * (n - filled), 1024)
        p = np.exp(rng.uniform(lp0, lp1, m))
        q = np.where(rng.random(m) < 0.5, -1.0, 1.0)
        txv = rng.uniform(-det.tx_max, det.tx_max, m)
        ty = rng.uniform(-det.ty_max, det.ty_max, m)
        dtx = q * det.kick_gev / p
        b = txv + dtx
        a = txv * det.z_kink + b * (det.z_ref - det.z_kink)
        c = det.kappa_c * q / (p * 1000.0)
        X = det.x_model(a[:, None], b[:, None], c[:, None], z[None, :])
        Y = ty[:, None] * z[None, :]
        Xh = X - Y * dxdy[None, :]
        ok = (np.abs(b) < det.tx_max) & np.all(np.abs(X) < det.x_acc, axis=1) \
            & np.all(np.abs(Y) < det.y_acc, axis=1) & np.all(np.abs(Xh) < det.x_acc, axis=1)
        idx = np.nonzero(ok)[0][: n - filled]
        for k, v in (("p", p), ("q", q), ("txv", txv), ("ty", ty), ("a", a), ("b", b), ("c", c)):
            out[k][filled:filled + len(idx)] = v[idx]
        filled += len(idx)
    return out


def make_events(n_events: int, *, seed: int, tracks=("poisson", 150.0),
                p_range=(2.0, 100.0), noise_frac: float = 0.3, eff: float = 0.98,
                sigma_x: float = 0.07, velo_ghosts_per_track: float = 0.2,
                velo_sigma=(0.015, 2.0e-4), det: Detector = DEFAULT_DETECTOR,
                ntracks: Optional[np.ndarray] = None, ut_sigma: float = 0.05,
                ut_eff: float = 0.99) -> EventBatch:
    """Generate `n_events` events.

    tracks: ("fixed", n) | ("poisson", mean) | ("lognormal", median, sigma, lo, hi)
    noise_frac: noise hits per event = round(noise_frac * signal hits of the event)
    velo_ghosts_per_track: VELO ghosts per event = round(g * tracks of the event)
    velo_sigma: (position mm, slope) Gaussian smearing of true VELO states
    ut_sigma, ut_eff: UT hit smearing (mm) and layer efficiency; UT noise hits
        are noise_frac of the event's UT signal hits, uniform in x and layer
    """
    rng = np.random.default_rng(seed)
    nt = _tracks_per_event(rng, n_events, tracks) if ntracks is None else np.asarray(ntracks, np.int64)
    T = int(nt.sum())
    trk_ev = np.repeat(np.arange(n_events), nt)
    tr = _sample_tracks(rng, T, det, p_range)
    z = det.z_arr
    dxdy = det.dxdy
    half = (tr["ty"] >= 0.0).astype(np.int32)

    # signal hits
    X = det.x_model(tr["a"][:, None], tr["b"][:, None], tr["c"][:, None], z[None, :])
    Y = tr["ty"][:, None] * z[None, :]
    xh = X - Y * dxdy[None, :]
    if sigma_x > 0:
        xh = xh + rng.normal(0.0, sigma_x, size=xh.shape)
    keep = rng.random(xh.shape) < eff if eff < 1.0 else np.ones(xh.shape, bool)
    ti, li = np.nonzero(keep)
    s_x = xh[ti, li]
    s_layer = li.astype(np.int32)
    s_half = half[ti]
    s_ev = trk_ev[ti]
    s_trk = ti.astype(np.int64)

    # noise hits
    n_sig_ev = np.bincount(s_ev, minlength=n_events)
    n_noise_ev = np.rint(noise_frac * n_sig_ev).astype(np.int64)
    NN = int(n_noise_ev.sum())
    n_ev = np.repeat(np.arange(n_events), n_noise_ev)
    n_x = rng.uniform(-det.x_acc, det.x_acc, NN)
    n_layer = rng.integers(0, N_LAYERS, NN).astype(np.int32)
    n_half = rng.integers(0, 2, NN).astype(np.int32)

    ev_all = np.concatenate([s_ev, n_ev])
    x_all = np.concatenate([s_x, n_x])
    layer_all = np.concatenate([s_layer, n_layer])
    half_all = np.concatenate([s_half, n_half])
    trk_all = np.concatenate([s_trk, -np.ones(NN, np.int64)])
    key = rng.random(len(ev_all))
    order = np.lexsort((key, ev_all))
    ev_all, x_all, layer_all, half_all, trk_all = (
        ev_all[order], x_all[order], layer_all[order], half_all[order], trk_all[order])

    counts = np.bincount(ev_all, minlength=n_events)
    ev_off = np.zeros(n_events + 1, np.int64)
    np.cumsum(counts, out=ev_off[1:])
    local = np.arange(len(ev_all)) - ev_off[ev_all]

    layer_hit = -np.ones((T, N_LAYERS), np.int64)
    sig = trk_all >= 0
    layer_hit[trk_all[sig], layer_all[sig]] = local[sig]

    # VELO states
    g = np.rint(velo_ghosts_per_track * nt).astype(np.int64)
    G = int(g.sum())
    sp, ss = velo_sigma
    tv = np.stack([tr["txv"] * det.z_velo, tr["ty"] * det.z_velo, tr["txv"], tr["ty"]], axis=1)
    if sp > 0 or ss > 0:
        tv = tv + rng.normal(0.0, 1.0, size=tv.shape) * np.array([sp, sp, ss, ss])
    gtx = rng.uniform(-det.tx_max, det.tx_max, G)
    gty = rng.uniform(-det.ty_max, det.ty_max, G)
    gv = np.stack([gtx * det.z_velo + rng.normal(0, 1.0, G),
                   gty * det.z_velo + rng.normal(0, 1.0, G), gtx, gty], axis=1)
    v_ev = np.concatenate([trk_ev, np.repeat(np.arange(n_events), g)])
    v_all = np.concatenate([tv, gv]) if G else tv
    v_trk = np.concatenate([np.arange(T), -np.ones(G, np.int64)])
    vkey = rng.random(len(v_ev))
    vorder = np.lexsort((vkey, v_ev))
    v_ev, v_all, v_trk = v_ev[vorder], v_all[vorder], v_trk[vorder]
    vcounts = np.bincount(v_ev, minlength=n_events)
    velo_off = np.zeros(n_events + 1, np.int64)
    np.cumsum(vcounts, out=velo_off[1:])

    trk_off = np.zeros(n_events + 1, np.int64)
    np.cumsum(nt, out=trk_off[1:])

    # UT hits, from their own random stream (the SciFi and VELO outputs do not
    # depend on whether UT hits are made)
    urng = np.random.default_rng([seed, 7])
    uz = np.asarray(det.ut_z, np.float64)
    ut_t = np.tan(np.radians(det.stereo_angle_deg)) * np.asarray(det.ut_stereo_sign, np.float64)
    dz = uz - det.z_velo
    gam = det.ut_gamma_a + det.ut_gamma_b * tr["q"] / (tr["p"] * 1000.0)
    UX = tr["txv"][:, None] * uz[None, :] + gam[:, None] * dz[None, :] ** 2
    UY = tr["ty"][:, None] * uz[None, :]
    uxm = UX - UY * ut_t[None, :]
    if ut_sigma > 0:
        uxm = uxm + urng.normal(0.0, ut_sigma, size=uxm.shape)
    ukeep = (urng.random(uxm.shape) < ut_eff) & (np.abs(uxm) < det.ut_x_acc)
    uti, uli = np.nonzero(ukeep)
    u_ev = np.concatenate([trk_ev[uti], np.repeat(np.arange(n_events), np.rint(noise_frac * np.bincount(
        trk_ev[uti], minlength=n_events)).astype(np.int64))])
    n_un = len(u_ev) - len(uti)
    u_x = np.concatenate([uxm[uti, uli], urng.uniform(-det.ut_x_acc, det.ut_x_acc, n_un)])
    u_l = np.concatenate([uli, urng.integers(0, 4, n_un)]).astype(np.int32)
    u_trk = np.concatenate([uti, -np.ones(n_un, np.int64)])
    uorder = np.lexsort((urng.random(len(u_ev)), u_ev))
    u_ev, u_x, u_l, u_trk = u_ev[uorder], u_x[uorder], u_l[uorder], u_trk[uorder]
    ut_off = np.zeros(n_events + 1, np.int64)
    np.cumsum(np.bincount(u_ev, minlength=n_events), out=ut_off[1:])
    ut_hit = -np.ones((T, 4), np.int64)
    usig = u_trk >= 0
    ut_hit[u_trk[usig], u_l[usig]] = (np.arange(len(u_ev)) - ut_off[u_ev])[usig]

    trk = {
        "trk_ev": trk_ev.astype(np.int32), "a": tr["a"], "b": tr["b"], "c": tr["c"],
        "ty": tr["ty"], "y0": np.zeros(T), "p": tr["p"], "q": tr["q"],
        "tx_velo": tr["txv"], "half": half, "layer_hit": layer_hit, "ut_hit": ut_hit,
    }
    zf = z.astype(np.float32)
    return EventBatch(
        det=det, ev_off=ev_off,
        x=x_all.astype(np.float32), z=zf[layer_all], dxdy=dxdy.astype(np.float32)[layer_all],
        zone=(2 * layer_all + half_all).astype(np.int32), x_exact=x_all.astype(np.float64),
        hit_track=trk_all.astype(np.int32), trk_off=trk_off, trk=trk,
        velo_off=velo_off, velo=v_all.astype(np.float32), velo_track=v_trk.astype(np.int32),
        meta={"seed": seed, "tracks": tracks, "noise_frac": noise_frac, "eff": eff,
              "sigma_x": sigma_x, "p_range": p_range},
        ut_off=ut_off, ut_x=u_x.astype(np.float32), ut_layer=u_l, ut_track=u_trk.astype(np.int32),
        ut_x_exact=u_x.astype(np.float64),
    )


# ---------------------------------------------------------------------------
# Named workloads.  Each entry is a recipe; sizes follow the benchmark
# configurations (tiny oracle run, Run-3-like batch, uneven occupancy,
# matching stress).  Seeds are fixed per workload.
# ---------------------------------------------------------------------------

WORKLOADS: Dict[str, Dict[str, object]] = {
    # 10 events x 50 tracks, 10% noise, 50 matching VELO states, no VELO smearing
    "tiny": dict(n_events=10, seed=1001, tracks=("fixed", 50), noise_frac=0.10, eff=0.98,
                 sigma_x=0.07, velo_ghosts_per_track=0.0, velo_sigma=(0.0, 0.0)),
    # 1000 events, Poisson(150) tracks, 30% noise (~2000 hits/event), VELO truth + 20% ghosts
    "run3": dict(n_events=1000, seed=1002, tracks=("poisson", 150.0), noise_frac=0.30,
                 eff=0.98, sigma_x=0.07, velo_ghosts_per_track=0.2, velo_sigma=(0.015, 2.0e-4)),
    # 10000 events, log-normal occupancy (median 120 tracks, clipped to [5, 800])
    "uneven": dict(n_events=10000, seed=1003, tracks=("lognormal", 120.0, 0.65, 5, 800),
                   noise_frac=0.30, eff=0.98, sigma_x=0.07, velo_ghosts_per_track=0.2,
                   velo_sigma=(0.015, 2.0e-4)),
    # 2000 events, 280 true tracks + 120 VELO ghosts (400 VELO/event, 30% ghosts), 40% noise
    "match_stress": dict(n_events=2000, seed=1004, tracks=("fixed", 280), noise_frac=0.40,
                         eff=0.98, sigma_x=0.07, velo_ghosts_per_track=120.0 / 280.0,
                         velo_sigma=(0.015, 2.0e-4)),
    # noise-free, unsmeared, fully efficient tracks above 3.5 GeV (oracle pins)
    "noise_free": dict(n_events=20, seed=1006, tracks=("fixed", 20), noise_frac=0.0, eff=1.0,
                       sigma_x=0.0, p_range=(3.5, 100.0), velo_ghosts_per_track=0.2,
                       velo_sigma=(0.0, 0.0)),
}


def make_workload(name: str, n_events: Optional[int] = None, seed: Optional[int] = None,
                  **overrides) -> EventBatch:
    spec = dict(WORKLOADS[name])
    if n_events is not None:
        spec["n_events"] = n_events
    if seed is not None:
        spec["seed"] = seed
    spec.update(overrides)
    n = spec.pop("n_events")
    b = make_events(n, **spec)
    b.meta["workload"] = name
    return b


def serving_requests(n_events_total: int, *, seed: int = 1005, batch_lo: int = 1,
                     batch_hi: int = 4096) -> np.ndarray:
    """Batch sizes of a request stream: log-uniform over [batch_lo, batch_hi],
    drawn until they add up to n_events_total (the last one is trimmed)."""
    rng = np.random.default_rng(seed)
    sizes = []
    tot = 0
    while tot < n_events_total:
        s = int(np.exp(rng.uniform(math.log(batch_lo), math.log(batch_hi + 1))))
        s = max(batch_lo, min(batch_hi, s, n_events_total - tot))
        sizes.append(s)
        tot += s
    return np.asarray(sizes, dtype=np.int64)


def poisson_arrivals(n: int, rate_per_s: float, *, seed: int) -> np.ndarray:
    """Arrival times (s) of n requests from a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


# ---------------------------------------------------------------------------
# z_match calibration (matching input constants)
# ---------------------------------------------------------------------------

def calibrate_zmatch(z_state: float, *, det: Detector = DEFAULT_DETECTOR, n_tracks: int = 200000,
                     seed: int = 77, p_range=(2.0, 100.0)) -> np.ndarray:
    """Fit (A, B, C, D, E) of  z_match_x = A + B|dtx| + C dtx^2 + D|x_S| + E tx_V^2
    to the intersection of each true VELO line with the tangent line of its true
    SciFi trajectory at z_state, over `n_tracks` generated tracks.

    This is the paper's calibration recipe for the kink-position parameters
    (Section 4.1), applied to this toy detector; the paper's table values are
    tuned to the real LHCb field map and do not describe this generator.
    """
    rng = np.random.default_rng(seed)
    tr = _sample_tracks(rng, n_tracks, det, p_range)
    txv = tr["txv"]
    x_s = det.x_model(tr["a"], tr["b"], tr["c"], z_state)
    tx_s = det.x_slope(tr["b"], tr["c"], z_state)
    # VELO line: x = txv * z ; SciFi tangent: x = x_s + tx_s (z - z_state)
    dtx = txv - tx_s
    ok = np.abs(dtx) > 1e-3
    zint = (x_s[ok] - tx_s[ok] * z_state) / dtx[ok]
    A = np.stack([np.ones(ok.sum()), np.abs(dtx[ok]), dtx[ok] ** 2, np.abs(x_s[ok]), txv[ok] ** 2], axis=1)
    coef, *_ = np.linalg.lstsq(A, zint, rcond=None)
    return coef


def ghost_nn_weights(seed: int = 1009) -> np.ndarray:
    """Seeded stand-in weights for the ghost network of the matching's final
    selection (8 inputs, 32 hidden nodes, 1 output; the trained weights are
    not published).  Layout (float32, 337 values): input mean[8],
    inverse scale[8], W1[32][8], b1[32], w2[32], b2.  The standardisation
    constants are the rough centre and spread of each input on these
    synthetic events, so the standardised inputs are of order one and the
    output spreads over (0, 1)."""
    rng = np.random.default_rng(seed)
    mean = np.array([5200.0, 0.0, 0.0, 0.0, 0.0, 1.0, 2.0, 10.0])
    scale = np.array([200.0, 10.0, 50.0, 0.1, 0.005, 1.0, 1.0, 1.0])
    w1 = rng.normal(0.0, 1.0 / np.sqrt(8.0), (32, 8))
    b1 = rng.normal(0.0, 0.3, 32)
    w2 = rng.normal(0.0, 4.0 / np.sqrt(32.0), 32)
    b2 = np.array([1.5])
    return np.concatenate([mean, 1.0 / scale, w1.ravel(), b1, w2, b2]).astype(np.float32)
