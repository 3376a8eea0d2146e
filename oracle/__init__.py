"""FP64 CPU oracle of SciFi Seeding + VELO-SciFi Matching.

TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package.  The product path (the CUDA library
and its binding) never imports, loads or calls it, and shares no code with it.

The arithmetic lives in `oracle.c` (plain C, double precision, one event per
call).  This module compiles it on demand and marshals numpy arrays.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Dict, List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: Optional[str] = None, out: Optional[str] = None,
          defines=()) -> str:
    """Compile oracle.c (or `src`) into a shared library (gcc, -O2)."""
    src = src or os.path.join(_HERE, "oracle.c")
    out = out or _LIB_PATH
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall",
                           "-I", _HERE, *[f"-D{d}" for d in defines], src, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


class OrConfig(C.Structure):
    _fields_ = [
        ("z", C.c_double * 12), ("dxdy", C.c_double * 12), ("z_ref", C.c_double),
        ("d_ratio", C.c_double), ("invp_a", C.c_double), ("invp_b", C.c_double),
        ("p_min", C.c_double), ("alpha0", C.c_double), ("alpha1", C.c_double),
        ("dx3_scale", C.c_double), ("n_iter", C.c_int32), ("iter_layers", (C.c_int32 * 3) * 3),
        ("kappa_c", C.c_double), ("m_lo", C.c_double), ("m_hi", C.c_double),
        ("c_nsigma", C.c_double), ("sigma_x", C.c_double), ("ext_tol", C.c_double),
        ("chi2x_max", C.c_double), ("score_w_chi2", C.c_double), ("score_w5", C.c_double),
        ("uv_init", C.c_int32 * 2), ("n_uv_min", C.c_int32), ("pad1", C.c_int32),
        ("uv_tol", C.c_double), ("uv_y_overlap", C.c_double), ("uv_y_max", C.c_double),
        ("sigma_y", C.c_double), ("z_state", C.c_double), ("z_velo", C.c_double),
        ("z_match_y", C.c_double), ("zmx", C.c_double * 5), ("presel", C.c_double * 4),
        ("presel_scale", C.c_double), ("tol_scale", C.c_double), ("tolx", C.c_double * 3),
        ("toly", C.c_double * 3), ("tol_tx", C.c_double), ("tol_ty", C.c_double),
        ("chi2_match_max", C.c_double), ("velo_unique", C.c_int32), ("pad2", C.c_int32),
        ("uv_mode", C.c_int32), ("hough_bins", C.c_int32), ("hough_fine", C.c_int32),
        ("hough_clusters", C.c_int32), ("hough_ty_max", C.c_double), ("hough_ty_in", C.c_double),
        ("final_sel", C.c_int32), ("pad3", C.c_int32), ("ghost_max", C.c_double), ("clone_margin", C.c_double),
        ("ut_z", C.c_double * 4), ("ut_dxdy", C.c_double * 4), ("ut_gamma", C.c_double * 2),
        ("ut_kick", C.c_double), ("ut_loose", C.c_double * 16), ("ut_tight", C.c_double * 16),
        ("ut_min_hits", C.c_int32), ("iter_mode", C.c_int32), ("p_min_iter", C.c_double * 3),
    ]


SEED_DTYPE = np.dtype([
    ("hits", "<i4", 12), ("half", "<i4"), ("nx", "<i4"), ("nuv", "<i4"), ("cand_id", "<i4"),
    ("pass", "<i4"), ("pad", "<i4"), ("a", "<f8"), ("b", "<f8"), ("c", "<f8"), ("chi2x", "<f8"), ("y0", "<f8"), ("ty", "<f8"),
    ("chi2y", "<f8"), ("x_s", "<f8"), ("y_s", "<f8"), ("tx_s", "<f8"), ("ty_s", "<f8"),
], align=True)
CAND_DTYPE = np.dtype([
    ("hits", "<i4", 6), ("half", "<i4"), ("iter", "<i4"), ("nx", "<i4"), ("keep", "<i4"),
    ("h1", "<i4"), ("h2", "<i4"), ("h3", "<i4"), ("id", "<i4"),
    ("a", "<f8"), ("b", "<f8"), ("c", "<f8"), ("chi2", "<f8"), ("score", "<f8"),
], align=True)
LEDGER_DTYPE = np.dtype([("kind", "<i4"), ("half", "<i4"), ("hits", "<i4", 12), ("margin", "<f8")],
                        align=True)
COUNTER_NAMES = ("pairs", "triplets", "ext_ok", "cands", "kept", "uv_init", "uv_cands", "seeds",
                 "match_pairs", "match_presel", "matched")


class OrCounters(C.Structure):
    _fields_ = [(n, C.c_int64) for n in COUNTER_NAMES]


LEDGER_KINDS = {1: "pair_win", 2: "trip_win", 3: "ext_tol", 4: "ext_tie", 5: "chi2x", 6: "clone",
                7: "uv_win", 8: "uv_tol", 9: "uv_tie", 10: "uv_sel", 11: "m_presel", 12: "m_chi2",
                13: "m_tie", 14: "hough_bin", 15: "ghost", 16: "m_clone", 17: "ut_win", 18: "ut_tie"}
GHOST_NN_SIZE = 337

_P = C.c_void_p


_libs: Dict[str, C.CDLL] = {}


def lib(path: Optional[str] = None):
    """The ctypes handle of the oracle library at `path` (default: the
    in-tree build, compiled on first use)."""
    with _lock:
        key = path or _LIB_PATH
        if key not in _libs:
            if path is None:
                build()
            L = C.CDLL(key)
            L.or_config_default.argtypes = [C.POINTER(OrConfig)]
            for name in ("or_dx3max", "or_alpha_corr", "or_k3"):
                getattr(L, name).argtypes = [C.POINTER(OrConfig), C.c_int32]
                getattr(L, name).restype = C.c_double
            L.or_x0max.argtypes = [C.POINTER(OrConfig)]
            L.or_x0max.restype = C.c_double
            L.or_invp.argtypes = [C.POINTER(OrConfig), C.c_double]
            L.or_invp.restype = C.c_double
            L.or_seeding_event.argtypes = [
                C.POINTER(OrConfig), C.c_int32, _P, _P,
                _P, C.c_int32, C.POINTER(C.c_int32),
                _P, C.c_int32, C.POINTER(C.c_int32),
                _P, C.c_int32, C.POINTER(C.c_int32),
                _P, C.c_int32, C.POINTER(C.c_int32), C.c_double, C.POINTER(OrCounters)]
            L.or_seeding_event.restype = C.c_int32
            L.or_matching_event.argtypes = [
                C.POINTER(OrConfig), C.c_int32, _P, C.c_int32, _P, _P, _P,
                _P, C.c_int32, C.POINTER(C.c_int32), C.c_double, C.POINTER(OrCounters)]
            L.or_matching_event.restype = C.c_int32
            L.or_ghost_nn.argtypes = [_P, _P]
            L.or_ghost_nn.restype = C.c_double
            L.or_final_selection.argtypes = [
                C.POINTER(OrConfig), C.c_int32, _P, C.c_int32, _P, _P, _P, _P, _P, _P,
                _P, C.c_int32, C.POINTER(C.c_int32), C.c_double]
            L.or_final_selection.restype = C.c_int32
            L.or_ut_search.argtypes = [
                C.POINTER(OrConfig), C.c_int32, _P, C.c_int32, _P, _P, C.c_int32, _P, _P, _P, _P, _P,
                _P, C.c_int32, C.POINTER(C.c_int32), C.c_double]
            L.or_ut_search.restype = C.c_int32
            _libs[key] = L
    return _libs[key]


def default_config(_lib=None, **overrides) -> OrConfig:
    """The oracle's own defaults (the paper's constants and the readings of
    its gaps), with keyword overrides (arrays accepted for array fields)."""
    cfg = OrConfig()
    (_lib or lib()).or_config_default(C.byref(cfg))
    apply(cfg, overrides)
    return cfg


def apply(cfg: OrConfig, overrides: Dict[str, object]) -> OrConfig:
    for k, v in overrides.items():
        cur = getattr(cfg, k)
        if isinstance(cur, C.Array):
            flat = np.asarray(v).ravel()
            rows = [cur[i] for i in range(len(cur))] if isinstance(cur[0], C.Array) else [cur]
            pos = 0
            for row in rows:
                conv = float if row._type_ is C.c_double else int
                for j in range(len(row)):
                    row[j] = conv(flat[pos])
                    pos += 1
        else:
            setattr(cfg, k, v)
    return cfg


def config_dict(cfg: OrConfig) -> Dict[str, object]:
    out = {}
    for name, _ in OrConfig._fields_:
        if name.startswith("pad"):
            continue
        v = getattr(cfg, name)
        if isinstance(v, C.Array):
            out[name] = np.array([list(r) if isinstance(r, C.Array) else r for r in v])
        else:
            out[name] = v
    return out


def x0max(cfg, _lib=None) -> float:
    return (_lib or lib()).or_x0max(C.byref(cfg))


def dx3max(cfg, it: int, _lib=None) -> float:
    return (_lib or lib()).or_dx3max(C.byref(cfg), it)


def alpha_corr(cfg, it: int, _lib=None) -> float:
    return (_lib or lib()).or_alpha_corr(C.byref(cfg), it)


def k3(cfg, it: int, _lib=None) -> float:
    return (_lib or lib()).or_k3(C.byref(cfg), it)


def invp(cfg, x0: float, _lib=None) -> float:
    return (_lib or lib()).or_invp(C.byref(cfg), x0)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_P)


def seeding_event(cfg: OrConfig, x, zone, *, cands: bool = False, trips: bool = False,
                  ledger_tau: Optional[float] = None, _lib=None) -> Dict[str, object]:
    """Seed one event.  x: hit x positions (converted to float64), zone: int32.

    Returns dict(seeds, cands?, trips?, ledger?, counters, status)."""
    L = _lib or lib()
    x = np.ascontiguousarray(x, dtype=np.float64)
    zone = np.ascontiguousarray(zone, dtype=np.int32)
    n = int(x.shape[0])
    caps = {"s": max(64, n // 4), "c": max(256, n) if cands else 0,
            "t": max(1024, 4 * n) if trips else 0, "l": 4096 if ledger_tau is not None else 0}
    while True:
        seeds = np.zeros(caps["s"], SEED_DTYPE)
        cbuf = np.zeros(caps["c"], CAND_DTYPE) if cands else None
        tbuf = np.zeros((caps["t"], 5), np.int32) if trips else None
        lbuf = np.zeros(caps["l"], LEDGER_DTYPE) if ledger_tau is not None else None
        ns, nc, nt, nl = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        cnt = OrCounters()
        st = L.or_seeding_event(
            C.byref(cfg), n, _ptr(x), _ptr(zone),
            _ptr(seeds), caps["s"], C.byref(ns),
            _ptr(cbuf), caps["c"], C.byref(nc),
            _ptr(tbuf), caps["t"], C.byref(nt),
            _ptr(lbuf), caps["l"], C.byref(nl),
            float(ledger_tau) if ledger_tau is not None else -1.0, C.byref(cnt))
        grow = False
        if ns.value > caps["s"]:
            caps["s"] = ns.value; grow = True
        if cands and nc.value > caps["c"]:
            caps["c"] = nc.value; grow = True
        if trips and nt.value > caps["t"]:
            caps["t"] = nt.value; grow = True
        if ledger_tau is not None and nl.value > caps["l"]:
            caps["l"] = nl.value; grow = True
        if not grow:
            break
    out = {"status": int(st), "seeds": seeds[: ns.value],
           "counters": {k: int(getattr(cnt, k)) for k in COUNTER_NAMES}}
    if cands:
        out["cands"] = cbuf[: nc.value]
    if trips:
        out["trips"] = tbuf[: nt.value]
    if ledger_tau is not None:
        out["ledger"] = lbuf[: nl.value]
    return out


def matching_event(cfg: OrConfig, velo, seed_state, *, ledger_tau: Optional[float] = None,
                   _lib=None):
    """Match one event.  velo: (n_velo, 4), seed_state: (n_seeds, 4), both
    converted to float64.  Returns dict(velo_idx, chi2, ledger?, counters)."""
    L = _lib or lib()
    velo = np.ascontiguousarray(velo, dtype=np.float64).reshape(-1, 4)
    ss = np.ascontiguousarray(seed_state, dtype=np.float64).reshape(-1, 4)
    nv, ns = velo.shape[0], ss.shape[0]
    vidx = np.zeros(ns, np.int32)
    chi2 = np.zeros(ns, np.float64)
    cap = 4096 if ledger_tau is not None else 0
    while True:
        lbuf = np.zeros(cap, LEDGER_DTYPE) if ledger_tau is not None else None
        nl = C.c_int32()
        cnt = OrCounters()
        st = L.or_matching_event(C.byref(cfg), nv, _ptr(velo), ns, _ptr(ss), _ptr(vidx), _ptr(chi2),
                                 _ptr(lbuf), cap, C.byref(nl),
                                 float(ledger_tau) if ledger_tau is not None else -1.0, C.byref(cnt))
        if ledger_tau is not None and nl.value > cap:
            cap = nl.value
            continue
        break
    out = {"status": int(st), "velo_idx": vidx, "chi2": chi2,
           "counters": {k: int(getattr(cnt, k)) for k in COUNTER_NAMES}}
    if ledger_tau is not None:
        out["ledger"] = lbuf[: nl.value]
    return out


def ghost_nn(nn, features, _lib=None) -> float:
    """The ghost network (Section 4.4) on one input vector of 8 features."""
    L = _lib or lib()
    nn = np.ascontiguousarray(nn, dtype=np.float32)
    assert nn.shape == (GHOST_NN_SIZE,)
    f = np.ascontiguousarray(features, dtype=np.float64)
    return float(L.or_ghost_nn(_ptr(nn), _ptr(f)))


def final_selection(cfg: OrConfig, velo, seed_state, seed_nhits, nn, velo_idx, chi2, *,
                    ledger_tau: Optional[float] = None, _lib=None):
    """Section 4.4 on one event's matching result.  Returns dict(velo_idx
    (after selection), ghost_prob, ledger?)."""
    L = _lib or lib()
    velo = np.ascontiguousarray(velo, dtype=np.float64).reshape(-1, 4)
    ss = np.ascontiguousarray(seed_state, dtype=np.float64).reshape(-1, 4)
    nh = np.ascontiguousarray(seed_nhits, dtype=np.int32)
    nn = np.ascontiguousarray(nn, dtype=np.float32)
    assert nn.shape == (GHOST_NN_SIZE,)
    vidx = np.ascontiguousarray(velo_idx, dtype=np.int32).copy()
    c2 = np.ascontiguousarray(chi2, dtype=np.float64)
    gp = np.zeros(ss.shape[0], np.float64)
    cap = 4096 if ledger_tau is not None else 0
    while True:
        lbuf = np.zeros(cap, LEDGER_DTYPE) if ledger_tau is not None else None
        nl = C.c_int32()
        st = L.or_final_selection(C.byref(cfg), velo.shape[0], _ptr(velo), ss.shape[0], _ptr(ss), _ptr(nh),
                                  _ptr(nn), _ptr(vidx), _ptr(c2), _ptr(gp), _ptr(lbuf), cap, C.byref(nl),
                                  float(ledger_tau) if ledger_tau is not None else -1.0)
        if ledger_tau is not None and nl.value > cap:
            cap = nl.value
            continue
        break
    out = {"status": int(st), "velo_idx": vidx, "ghost_prob": gp}
    if ledger_tau is not None:
        out["ledger"] = lbuf[: nl.value]
    return out


def ut_search(cfg: OrConfig, velo, seed_state, velo_idx, ut_x, ut_layer, *, ledger_tau: Optional[float] = None,
              _lib=None):
    """Section 4.3 on one event's Long tracks.  Returns dict(ut_hits (n, 4),
    n_ut, gamma, velo_idx (after the UT hit requirement), ledger?)."""
    L = _lib or lib()
    velo = np.ascontiguousarray(velo, dtype=np.float64).reshape(-1, 4)
    ss = np.ascontiguousarray(seed_state, dtype=np.float64).reshape(-1, 4)
    vidx = np.ascontiguousarray(velo_idx, dtype=np.int32).copy()
    ux = np.ascontiguousarray(ut_x, dtype=np.float64)
    ul = np.ascontiguousarray(ut_layer, dtype=np.int32)
    ns = ss.shape[0]
    hits = np.zeros((ns, 4), np.int32)
    nut = np.zeros(ns, np.int32)
    gam = np.zeros(ns, np.float64)
    cap = 8192 if ledger_tau is not None else 0
    while True:
        lbuf = np.zeros(cap, LEDGER_DTYPE) if ledger_tau is not None else None
        nl = C.c_int32()
        st = L.or_ut_search(C.byref(cfg), velo.shape[0], _ptr(velo), ns, _ptr(ss), _ptr(vidx), len(ux), _ptr(ux),
                            _ptr(ul), _ptr(hits), _ptr(nut), _ptr(gam), _ptr(lbuf), cap, C.byref(nl),
                            float(ledger_tau) if ledger_tau is not None else -1.0)
        if ledger_tau is not None and nl.value > cap:
            cap = nl.value
            continue
        break
    out = {"status": int(st), "ut_hits": hits, "n_ut": nut, "gamma": gam, "velo_idx": vidx}
    if ledger_tau is not None:
        out["ledger"] = lbuf[: nl.value]
    return out


def seeding_batch(cfg: OrConfig, batch, events=None, *, threads: Optional[int] = None,
                  exact: bool = False, **kw) -> List[Dict[str, object]]:
    """Seed many events of a synth.EventBatch, one event per task on a thread
    pool (the C calls release the GIL).  exact=True feeds the float64 positions
    the float32 hits were rounded from."""
    events = range(batch.n_events) if events is None else events
    threads = threads or os.cpu_count() or 1

    def one(e):
        x, z = batch.exact_hits_of(e) if exact else batch.hits_of(e)
        return seeding_event(cfg, x, z, **kw)

    if threads == 1:
        return [one(e) for e in events]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, events))
