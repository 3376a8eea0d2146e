"""The batch path with matching fused into the seeding kernel (the CUDA graph
and the serving pipeline take it for the HLT1 configuration) against the two
separate steps (seeding_run then matching_run) and against the oracle.

The two paths run the same per-event matching code on the same seed records,
so every output array must be equal bit for bit: seeds, Long tracks, chi2,
per-event counts and statuses."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import parity  # noqa: E402
from conftest import workload  # noqa: E402
from paper_2606_14480_gb300 import st  # noqa: E402
from synth import calibrate_zmatch  # noqa: E402


@pytest.fixture(scope="module")
def zmx():
    return calibrate_zmatch(7826.0)


def two_step(gcfg, ev_off, x, zone, velo_off, velo, cap):
    ctx = st.Context(gcfg)
    db = st.DeviceBatch(ev_off, x, zone, velo_off, velo)
    out = st.run_batch(ctx, db, cap=cap)
    torch.cuda.synchronize()
    res = out.to_numpy()
    ctx.close()
    return res


def fused(gcfg, ev_off, x, zone, velo_off, velo, cap, replays=2):
    """Through a CUDA graph of the batch (the fused kernel), replayed."""
    ctx = st.Context(gcfg)
    db = st.DeviceBatch(ev_off, x, zone, velo_off, velo)
    out = st.DeviceOutputs(len(ev_off) - 1, cap)
    ctx.st_reserve(len(ev_off) - 1, (len(ev_off) - 1) * db.max_hits, db.max_hits, cap)
    g = ctx.st_graph_create(db.hits, db.velo_s, out.seeds, out.long)
    for _ in range(replays):
        out.velo_idx.fill_(-7)
        out.n_long.fill_(-7)
        g.st_graph_launch()
    torch.cuda.synchronize()
    res = out.to_numpy()
    cnt = ctx.st_read_counters()
    g.close()
    ctx.close()
    return res, cnt


def doubled_velo(b):
    """Every event's VELO segments twice (more than one shared-memory chunk of
    512 in the stress workload)."""
    parts = [np.concatenate([b.velo_of(e), b.velo_of(e)]) for e in range(b.n_events)]
    off = np.zeros(b.n_events + 1, np.int64)
    off[1:] = np.cumsum([len(p) for p in parts])
    return off, np.concatenate(parts).astype(np.float32)


CASES = [("run3", 200, {}), ("uneven", 300, {}), ("match_stress", 40, {}),
         ("match_stress", 30, {"velo_unique": 1}), ("run3", 100, {"tol_scale": 2.0})]


@pytest.mark.parametrize("name,n,over", CASES, ids=[f"{c[0]}-{c[1]}-{len(c[2])}" for c in CASES])
def test_fused_equals_two_step(name, n, over, zmx):
    b = workload(name, n_events=n)
    _, gcfg = parity.config_pair(zmx, **over)
    cap = max(1024, b.n_hits // 4)
    args = (b.ev_off, b.x, b.zone, b.velo_off, b.velo, cap)
    ref = two_step(gcfg, *args)
    got, cnt = fused(gcfg, *args)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
    assert cnt["matched"] == int((got["velo_idx"] >= 0).sum()) * 2  # two replays
    assert (got["n_long"] >= 0).all()


def test_fused_chunked_velo(zmx):
    b = workload("match_stress", n_events=20)
    voff, velo = doubled_velo(b)
    assert np.diff(voff).max() > 512
    _, gcfg = parity.config_pair(zmx)
    cap = max(1024, b.n_hits // 4)
    args = (b.ev_off, b.x, b.zone, voff, velo, cap)
    ref = two_step(gcfg, *args)
    got, _ = fused(gcfg, *args)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k


def test_fused_with_empty_and_invalid_events(zmx):
    """Events without hits, without VELO segments, and one with an invalid
    zone: statuses, empty seed ranges and zero Long-track counts agree."""
    b = workload("tiny")
    x, zone = b.x.copy(), b.zone.copy()
    zone[b.ev_off[2]] = 99
    keep = np.ones(len(x), bool)
    keep[b.ev_off[5]:b.ev_off[6]] = False  # event 5 without hits
    ev_off = np.zeros(b.n_events + 1, np.int64)
    ev_off[1:] = np.cumsum([keep[b.ev_off[e]:b.ev_off[e + 1]].sum() for e in range(b.n_events)])
    parts = [b.velo_of(e) if e != 7 else b.velo_of(e)[:0] for e in range(b.n_events)]
    voff = np.zeros(b.n_events + 1, np.int64)
    voff[1:] = np.cumsum([len(p) for p in parts])
    velo = np.concatenate(parts).astype(np.float32)
    _, gcfg = parity.config_pair(zmx)
    args = (ev_off, x[keep], zone[keep], voff, velo, 1024)
    ref = two_step(gcfg, *args)
    got, _ = fused(gcfg, *args)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
    assert got["status"][2] == st.ST_EINVAL and got["n_long"][7] == 0 and got["n_long"][5] == 0


def test_fused_full_size_run3_against_oracle(zmx):
    """The benchmark's 1000-event batch through the graph (fused kernel); the
    oracle recomputes seeding and matching of a sample of events."""
    b = workload("run3")
    ocfg, gcfg = parity.config_pair(zmx)
    got, _ = fused(gcfg, b.ev_off, b.x, b.zone, b.velo_off, b.velo, max(1024, b.n_hits // 4), replays=1)
    rng = np.random.default_rng(21)
    ev = np.sort(rng.choice(b.n_events, 40, replace=False))
    rep = parity.compare_seeding(got, ocfg, b, ev)
    parity.assert_seeding(rep)
    _, untraced, _, _ = parity.compare_matching(got, ocfg, b, ev)
    assert not untraced, untraced[:5]


def test_fused_full_size_uneven_equals_two_step(zmx):
    """10000 events of 100-15000 hits, as the uneven benchmark line runs them."""
    b = workload("uneven")
    _, gcfg = parity.config_pair(zmx)
    cap = max(1024, b.n_hits // 4)
    args = (b.ev_off, b.x, b.zone, b.velo_off, b.velo, cap)
    ref = two_step(gcfg, *args)
    got, _ = fused(gcfg, *args, replays=1)
    assert (got["status"] == 0).all()
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k
