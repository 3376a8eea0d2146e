"""Python binding of libst (include/st.h): argument marshalling only.

Every step of the seeding / matching path runs in the CUDA library; this
module loads it with ctypes, mirrors its structs, and moves torch tensors'
pointers and streams across the boundary.  There is no CPU fallback: if the
library cannot be loaded the import of the functions raises.
"""

from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Dict, Optional, Tuple

import numpy as np

from . import build as _build

_P = C.c_void_p


class StConfig(C.Structure):
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
        ("chi2_match_max", C.c_double), ("velo_unique", C.c_int32),
        ("threads_seed", C.c_int32), ("threads_build", C.c_int32), ("threads_match", C.c_int32),
        ("ctas_per_sm", C.c_int32), ("smem_hits", C.c_int32), ("cand_cap", C.c_int32),
        ("pad2", C.c_int32),
        ("uv_mode", C.c_int32), ("hough_bins", C.c_int32), ("hough_fine", C.c_int32),
        ("hough_clusters", C.c_int32), ("hough_ty_max", C.c_double), ("hough_ty_in", C.c_double),
        ("final_sel", C.c_int32), ("pad3", C.c_int32), ("ghost_max", C.c_double), ("clone_margin", C.c_double),
        ("ut_z", C.c_double * 4), ("ut_dxdy", C.c_double * 4), ("ut_gamma", C.c_double * 2),
        ("ut_kick", C.c_double), ("ut_loose", C.c_double * 16), ("ut_tight", C.c_double * 16),
        ("ut_min_hits", C.c_int32), ("iter_mode", C.c_int32), ("p_min_iter", C.c_double * 3),
    ]


class StHits(C.Structure):
    _fields_ = [("n_events", C.c_int64), ("ev_off", _P), ("x", _P), ("zone", _P), ("z", _P),
                ("dxdy", _P), ("max_hits_per_event", C.c_int32), ("pad", C.c_int32)]


class StSeeds(C.Structure):
    _fields_ = [("cap", C.c_int64), ("ev_off", _P), ("hits", _P), ("params", _P), ("state", _P),
                ("n_hits", _P), ("status", _P)]


class StVelo(C.Structure):
    _fields_ = [("n_events", C.c_int64), ("ev_off", _P), ("state", _P)]


class StLong(C.Structure):
    _fields_ = [("velo_idx", _P), ("chi2", _P), ("n_long", _P), ("ghost_prob", _P)]


class StUtHits(C.Structure):
    _fields_ = [("n_events", C.c_int64), ("ev_off", _P), ("x", _P), ("layer", _P)]


class StUtOut(C.Structure):
    _fields_ = [("hits", _P), ("n_hits", _P), ("gamma", _P)]


COUNTER_NAMES = ("pairs", "triplets", "ext_ok", "cands", "kept", "uv_init", "uv_cands", "seeds",
                 "match_pairs", "match_presel", "matched", "hits", "events", "match_eval")


class StCounters(C.Structure):
    _fields_ = [(n, C.c_int64) for n in COUNTER_NAMES]


class StPipelineConfig(C.Structure):
    _fields_ = [("n_slots", C.c_int32), ("max_events_per_slot", C.c_int32),
                ("max_hits_per_slot", C.c_int64), ("max_hits_per_event", C.c_int32),
                ("max_velo_per_event", C.c_int32), ("mem_cap_bytes", C.c_int64),
                ("max_velo_per_slot", C.c_int64)]


class StRequestInfo(C.Structure):
    _fields_ = [("t_submit_ns", C.c_int64), ("t_launch_ns", C.c_int64), ("t_done_ns", C.c_int64),
                ("t_returned_ns", C.c_int64), ("n_events", C.c_int32), ("n_seeds", C.c_int32)]


ST_OK, ST_PENDING, ST_EINVAL, ST_ENOMEM, ST_OVERFLOW, ST_TIMEOUT, ST_ECUDA, ST_ESTATE = 0, 1, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "ST_OK", 1: "ST_PENDING", -1: "ST_EINVAL", -2: "ST_ENOMEM", -3: "ST_OVERFLOW",
                -4: "ST_TIMEOUT", -5: "ST_ECUDA", -6: "ST_ESTATE"}

# exported symbol -> (argtypes, restype)
SIGNATURES = {
    "st_config_default": ([C.POINTER(StConfig)], None),
    "st_create": ([C.POINTER(StConfig), C.c_int, C.POINTER(_P)], C.c_int),
    "st_destroy": ([_P], None),
    "st_last_error": ([_P], C.c_char_p),
    "st_reserve": ([_P, C.c_int64, C.c_int64, C.c_int32, C.c_int64], C.c_int),
    "seeding_run": ([_P, C.POINTER(StHits), C.POINTER(StSeeds), _P], C.c_int),
    "matching_run": ([_P, C.POINTER(StVelo), C.POINTER(StSeeds), C.POINTER(StLong), _P], C.c_int),
    "st_graph_create": ([_P, C.POINTER(StHits), C.POINTER(StVelo), C.POINTER(StSeeds),
                         C.POINTER(StLong), C.POINTER(_P)], C.c_int),
    "st_graph_launch": ([_P, _P], C.c_int),
    "st_graph_destroy": ([_P], None),
    "st_read_counters": ([_P, C.POINTER(StCounters), C.c_int], C.c_int),
    "st_set_timing": ([_P, C.c_int], C.c_int),
    "st_set_wait_limit": ([_P, C.c_int64], C.c_int),
    "st_set_ghost_nn": ([_P, _P, C.c_int32], C.c_int),
    "ut_run": ([_P, C.POINTER(StVelo), C.POINTER(StSeeds), C.POINTER(StUtHits), C.POINTER(StLong),
                C.POINTER(StUtOut), _P], C.c_int),
    "st_kernel_ms": ([_P, C.POINTER(C.c_float * 4)], C.c_int),
    "seeding_run_static": ([C.POINTER(StConfig), C.POINTER(StHits), C.POINTER(StSeeds), _P, C.c_char_p,
                            C.c_int32], C.c_int),
    "st_pipeline_config_default": ([C.POINTER(StPipelineConfig)], None),
    "st_pipeline_configure": ([_P, C.POINTER(StPipelineConfig)], C.c_int),
    "pipeline_submit": ([_P, C.POINTER(StHits), C.POINTER(StVelo), C.POINTER(C.c_uint64)], C.c_int),
    "pipeline_poll": ([_P, C.c_uint64, C.POINTER(StSeeds), C.POINTER(StLong), C.c_int64,
                       C.POINTER(StRequestInfo)], C.c_int),
}

_lock = threading.Lock()
_lib = None


def library(build_if_missing: bool = True):
    """Load libst.so (building it in-tree first if allowed).  Raises if the
    library cannot be built or loaded."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libst.so not found at {path}; run paper_2606_14480_gb300.build")
            L = C.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


class StError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _apply(cfg, overrides):
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


def st_config_default(**overrides) -> StConfig:
    cfg = StConfig()
    library().st_config_default(C.byref(cfg))
    return _apply(cfg, overrides)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class Context:
    """Owns an st_ctx.  Methods carry the C entry points' names."""

    def __init__(self, cfg: Optional[StConfig] = None, device: int = 0):
        self.lib = library()
        self.cfg = cfg if cfg is not None else st_config_default()
        h = _P()
        rc = self.lib.st_create(C.byref(self.cfg), device, C.byref(h))
        if rc != ST_OK:
            raise StError(rc, "st_create failed (invalid config or CUDA error)")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self.lib.st_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc not in (ST_OK, ST_PENDING):
            raise StError(rc, f"{what}: {self.lib.st_last_error(self.h).decode()}")
        return rc

    def last_error(self) -> str:
        return self.lib.st_last_error(self.h).decode()

    def st_reserve(self, n_events, n_hits, max_hits, seeds_cap):
        return self._check(self.lib.st_reserve(self.h, n_events, n_hits, max_hits, seeds_cap), "st_reserve")

    def seeding_run(self, hits: StHits, seeds: StSeeds, stream=None, check=True):
        rc = self.lib.seeding_run(self.h, C.byref(hits), C.byref(seeds), _stream_handle(stream))
        return self._check(rc, "seeding_run") if check else rc

    def matching_run(self, velo: StVelo, seeds: StSeeds, out: StLong, stream=None, check=True):
        rc = self.lib.matching_run(self.h, C.byref(velo), C.byref(seeds), C.byref(out), _stream_handle(stream))
        return self._check(rc, "matching_run") if check else rc

    def ut_run(self, velo: StVelo, seeds: StSeeds, ut: StUtHits, out: StLong, ut_out: StUtOut, stream=None,
               check=True):
        rc = self.lib.ut_run(self.h, C.byref(velo), C.byref(seeds), C.byref(ut), C.byref(out), C.byref(ut_out),
                             _stream_handle(stream))
        return self._check(rc, "ut_run") if check else rc

    def st_graph_create(self, hits, velo, seeds, out):
        g = _P()
        self._check(self.lib.st_graph_create(self.h, C.byref(hits), C.byref(velo), C.byref(seeds),
                                             C.byref(out), C.byref(g)), "st_graph_create")
        return Graph(self, g)

    def st_set_ghost_nn(self, weights):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        return self._check(self.lib.st_set_ghost_nn(self.h, w.ctypes.data, int(w.size)), "st_set_ghost_nn")

    def st_set_timing(self, enable=True):
        return self._check(self.lib.st_set_timing(self.h, int(enable)), "st_set_timing")

    def st_set_wait_limit(self, ns):
        return self._check(self.lib.st_set_wait_limit(self.h, int(ns)), "st_set_wait_limit")

    def st_kernel_ms(self):
        ms = (C.c_float * 4)()
        self._check(self.lib.st_kernel_ms(self.h, C.byref(ms)), "st_kernel_ms")
        return {"build": ms[0], "seed": ms[1], "gather": ms[2], "match": ms[3]}

    def st_read_counters(self, reset=False) -> Dict[str, int]:
        c = StCounters()
        self._check(self.lib.st_read_counters(self.h, C.byref(c), int(reset)), "st_read_counters")
        return {n: int(getattr(c, n)) for n in COUNTER_NAMES}

    def st_pipeline_configure(self, **kw):
        pc = StPipelineConfig()
        self.lib.st_pipeline_config_default(C.byref(pc))
        for k, v in kw.items():
            setattr(pc, k, v)
        return self._check(self.lib.st_pipeline_configure(self.h, C.byref(pc)), "st_pipeline_configure")

    def pipeline_submit(self, hits: StHits, velo: StVelo) -> int:
        t = C.c_uint64()
        self._check(self.lib.pipeline_submit(self.h, C.byref(hits), C.byref(velo), C.byref(t)),
                    "pipeline_submit")
        return t.value

    def pipeline_poll(self, ticket: int, seeds: StSeeds, out: Optional[StLong], timeout_us: int):
        info = StRequestInfo()
        rc = self.lib.pipeline_poll(self.h, ticket, C.byref(seeds), C.byref(out) if out is not None else None,
                                    timeout_us, C.byref(info))
        if rc in (ST_PENDING, ST_TIMEOUT):
            return rc, None
        self._check(rc, "pipeline_poll")
        return rc, info


class Graph:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def st_graph_launch(self, stream=None):
        return self.ctx._check(self.ctx.lib.st_graph_launch(self.h, _stream_handle(stream)), "st_graph_launch")

    def close(self):
        if self.h:
            self.ctx.lib.st_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# torch marshalling helpers
# ---------------------------------------------------------------------------

class DeviceBatch:
    """Device copies of a batch (hits + VELO) and the argument structs that
    point at them.  Inputs: numpy arrays (CSR, as produced by synth)."""

    def __init__(self, ev_off, x, zone, velo_off, velo, *, device="cuda", max_hits=None, z=None, dxdy=None):
        import torch
        dev = torch.device(device)

        def t(a, dt):
            # never hand a null pointer across the boundary for an empty array
            a = np.ascontiguousarray(a)
            if a.size == 0:
                a = np.zeros((1,) + a.shape[1:], dtype=a.dtype if a.dtype != object else np.float32)
            return torch.as_tensor(a, dtype=dt).to(dev)
        self.ev_off = t(ev_off, torch.int64)
        self.x = t(x, torch.float32)
        self.zone = t(zone, torch.int32)
        self.z = None if z is None else t(z, torch.float32)
        self.dxdy = None if dxdy is None else t(dxdy, torch.float32)
        self.velo_off = t(velo_off, torch.int64)
        self.velo = t(np.asarray(velo, np.float32).reshape(-1, 4), torch.float32)
        n = len(ev_off) - 1
        if max_hits is None:
            max_hits = int(np.max(np.diff(ev_off))) if n > 0 else 1
        self.n_events = n
        self.max_hits = max(1, int(max_hits))
        self.hits = StHits(n, _ptr(self.ev_off), _ptr(self.x), _ptr(self.zone), _ptr(self.z), _ptr(self.dxdy),
                           self.max_hits, 0)
        self.velo_s = StVelo(n, _ptr(self.velo_off), _ptr(self.velo))

    def add_ut(self, ut_off, ut_x, ut_layer):
        """Device copies of the batch's UT hits; sets self.ut (st_ut_hits)."""
        import torch
        dev = self.x.device

        def t(a, dt):
            a = np.ascontiguousarray(a)
            if a.size == 0:
                a = np.zeros(1, dtype=a.dtype)
            return torch.as_tensor(a, dtype=dt).to(dev)
        self.ut_off = t(ut_off, torch.int64)
        self.ut_x = t(ut_x, torch.float32)
        self.ut_layer = t(ut_layer, torch.int32)
        self.ut = StUtHits(self.n_events, _ptr(self.ut_off), _ptr(self.ut_x), _ptr(self.ut_layer))
        return self

    @classmethod
    def from_synth(cls, batch, device="cuda", **kw):
        db = cls(batch.ev_off, batch.x, batch.zone, batch.velo_off, batch.velo, device=device, **kw)
        if getattr(batch, "ut_off", None) is not None:
            db.add_ut(batch.ut_off, batch.ut_x, batch.ut_layer)
        return db


class DeviceOutputs:
    """Caller-owned device output buffers for seeding and matching."""

    def __init__(self, n_events: int, cap: int, device="cuda"):
        import torch
        dev = torch.device(device)
        self.cap = cap
        self.ev_off = torch.zeros(n_events + 1, dtype=torch.int32, device=dev)
        self.hits = torch.zeros((max(cap, 1), 12), dtype=torch.int32, device=dev)
        self.params = torch.zeros((max(cap, 1), 8), dtype=torch.float32, device=dev)
        self.state = torch.zeros((max(cap, 1), 4), dtype=torch.float32, device=dev)
        self.n_hits = torch.zeros((max(cap, 1), 2), dtype=torch.int8, device=dev)
        self.status = torch.zeros(max(n_events, 1), dtype=torch.int32, device=dev)
        self.velo_idx = torch.zeros(max(cap, 1), dtype=torch.int32, device=dev)
        self.chi2 = torch.zeros(max(cap, 1), dtype=torch.float32, device=dev)
        self.n_long = torch.zeros(max(n_events, 1), dtype=torch.int32, device=dev)
        self.ghost_prob = torch.zeros(max(cap, 1), dtype=torch.float32, device=dev)
        self.ut_hits = torch.zeros((max(cap, 1), 4), dtype=torch.int32, device=dev)
        self.ut_n = torch.zeros(max(cap, 1), dtype=torch.int8, device=dev)
        self.ut_gamma = torch.zeros(max(cap, 1), dtype=torch.float32, device=dev)
        self.ut_out = StUtOut(_ptr(self.ut_hits), _ptr(self.ut_n), _ptr(self.ut_gamma))
        self.seeds = StSeeds(cap, _ptr(self.ev_off), _ptr(self.hits), _ptr(self.params), _ptr(self.state),
                             _ptr(self.n_hits), _ptr(self.status))
        self.long = StLong(_ptr(self.velo_idx), _ptr(self.chi2), _ptr(self.n_long), _ptr(self.ghost_prob))

    def to_numpy(self) -> Dict[str, np.ndarray]:
        ev = self.ev_off.cpu().numpy()
        ns = int(ev[-1])
        return {"ev_off": ev, "hits": self.hits[:ns].cpu().numpy(), "params": self.params[:ns].cpu().numpy(),
                "state": self.state[:ns].cpu().numpy(), "n_hits": self.n_hits[:ns].cpu().numpy(),
                "status": self.status[: len(ev) - 1].cpu().numpy(),
                "velo_idx": self.velo_idx[:ns].cpu().numpy(), "chi2": self.chi2[:ns].cpu().numpy(),
                "n_long": self.n_long[: len(ev) - 1].cpu().numpy(),
                "ghost_prob": self.ghost_prob[:ns].cpu().numpy(), "ut_hits": self.ut_hits[:ns].cpu().numpy(),
                "ut_n": self.ut_n[:ns].cpu().numpy(), "ut_gamma": self.ut_gamma[:ns].cpu().numpy()}


def _host_array(a_or_shape, dtype, pinned: bool, keep: list):
    """A numpy array in host memory, page-locked (through a pinned torch
    tensor kept in `keep`) if `pinned`; a copy of `a_or_shape` when it is an
    array, else zero-filled of that shape."""
    src = None if isinstance(a_or_shape, tuple) else np.ascontiguousarray(a_or_shape, dtype)
    shape = a_or_shape if src is None else src.shape
    if not pinned:
        return np.zeros(shape, dtype) if src is None else src
    import torch
    t = torch.zeros(shape, dtype=torch.from_numpy(np.zeros(0, dtype)).dtype, pin_memory=True)
    keep.append(t)
    a = t.numpy()
    if src is not None:
        a[...] = src
    return a


class HostBuffers:
    """Host (numpy) buffers for the pipeline: inputs of pipeline_submit and
    outputs of pipeline_poll; page-locked with pinned=True (the copies then
    run at the link's full rate)."""

    @staticmethod
    def inputs(ev_off, x, zone, velo_off, velo, max_hits=65535, pinned=False):
        pins = []
        keep = [_host_array(ev_off, np.int64, pinned, pins), _host_array(x, np.float32, pinned, pins),
                _host_array(zone, np.int32, pinned, pins), _host_array(velo_off, np.int64, pinned, pins),
                _host_array(np.asarray(velo, np.float32).reshape(-1, 4), np.float32, pinned, pins)]
        keep += pins
        n = len(ev_off) - 1
        p = lambda a: a.ctypes.data
        hits = StHits(n, p(keep[0]), p(keep[1]), p(keep[2]), None, None, max_hits, 0)
        velo_s = StVelo(n, p(keep[3]), p(keep[4]))
        return hits, velo_s, keep

    def __init__(self, n_events: int, cap: int, pinned: bool = False):
        # filled by pipeline_poll up to the returned counts
        self._pins = []
        h = lambda shape, dt: _host_array(shape, dt, pinned, self._pins)
        self.ev_off = h((n_events + 1,), np.int32)
        self.hits = h((max(cap, 1), 12), np.int32)
        self.params = h((max(cap, 1), 8), np.float32)
        self.state = h((max(cap, 1), 4), np.float32)
        self.n_hits = h((max(cap, 1), 2), np.int8)
        self.status = h((max(n_events, 1),), np.int32)
        self.velo_idx = h((max(cap, 1),), np.int32)
        self.chi2 = h((max(cap, 1),), np.float32)
        self.n_long = h((max(n_events, 1),), np.int32)
        self.ghost_prob = h((max(cap, 1),), np.float32)
        p = lambda a: a.ctypes.data
        self.seeds = StSeeds(cap, p(self.ev_off), p(self.hits), p(self.params), p(self.state), p(self.n_hits),
                             p(self.status))
        self.long = StLong(p(self.velo_idx), p(self.chi2), p(self.n_long), p(self.ghost_prob))

    def to_numpy(self):
        ns = int(self.ev_off[-1])
        n = len(self.ev_off) - 1
        return {"ev_off": self.ev_off.copy(), "hits": self.hits[:ns].copy(), "params": self.params[:ns].copy(),
                "state": self.state[:ns].copy(), "n_hits": self.n_hits[:ns].copy(), "status": self.status[:n].copy(),
                "velo_idx": self.velo_idx[:ns].copy(), "chi2": self.chi2[:ns].copy(), "n_long": self.n_long[:n].copy(),
                "ghost_prob": self.ghost_prob[:ns].copy()}


def seeding_run_static(cfg: StConfig, hits: StHits, seeds: StSeeds, stream=None) -> Tuple[int, str]:
    """The allocation-free seeding entry point; returns (status, message)."""
    buf = C.create_string_buffer(512)
    rc = library().seeding_run_static(C.byref(cfg), C.byref(hits), C.byref(seeds), _stream_handle(stream), buf,
                                      len(buf))
    return rc, buf.value.decode()


def run_batch(ctx: Context, db: DeviceBatch, cap: Optional[int] = None, stream=None) -> DeviceOutputs:
    """seeding_run then matching_run on one device batch; returns the outputs."""
    cap = cap if cap is not None else max(1024, int(db.x.shape[0]) // 4)
    out = DeviceOutputs(db.n_events, cap, device=db.x.device)
    ctx.seeding_run(db.hits, out.seeds, stream)
    ctx.matching_run(db.velo_s, out.seeds, out.long, stream)
    return out
