"""Edge cases of the widened method (Hough-cluster UV, HLT2-style iterations,
final selection, UT hits): empty events and batches, events without UT hits
or VELO segments, the allocation-free entry point and the serving pipeline
in the HLT2-style mode, and determinism across launch shapes."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import parity  # noqa: E402
from conftest import workload  # noqa: E402
from paper_2606_14480_gb300 import st  # noqa: E402
from synth import calibrate_zmatch, ghost_nn_weights  # noqa: E402

SEQ3 = dict(iter_mode=1, n_iter=3, p_min_iter=[5000.0, 3000.0, 1500.0])
MODES = [dict(uv_mode=1), SEQ3, dict(SEQ3, uv_mode=1), dict(final_sel=1)]


@pytest.fixture(scope="module")
def zmx():
    return calibrate_zmatch(7826.0)


def _with_empty_events(b):
    """The batch with events 1 and 4 emptied (hits, VELO segments, UT hits)."""
    def rebuild(off, arrays, empty):
        parts = [[a[off[e]:off[e + 1]] if e not in empty else a[off[e]:off[e]] for e in range(b.n_events)]
                 for a in arrays]
        new_off = np.zeros(b.n_events + 1, np.int64)
        new_off[1:] = np.cumsum([len(p) for p in parts[0]])
        return new_off, [np.concatenate(p) for p in parts]
    empty = {1, 4}
    ev, (x, zone) = rebuild(b.ev_off, [b.x, b.zone], empty)
    vo, (velo,) = rebuild(b.velo_off, [b.velo], empty)
    uo, (ux, ul) = rebuild(b.ut_off, [b.ut_x, b.ut_layer], empty)
    return ev, x, zone, vo, velo, uo, ux, ul, empty


@pytest.mark.parametrize("mode", MODES, ids=["hough", "seq3", "seq3_hough", "final_sel"])
def test_empty_events_in_every_mode(mode, zmx):
    b = workload("tiny")
    ev, x, zone, vo, velo, uo, ux, ul, empty = _with_empty_events(b)
    _, gcfg = parity.config_pair(zmx, **mode)
    ctx = st.Context(gcfg)
    if mode.get("final_sel"):
        ctx.st_set_ghost_nn(ghost_nn_weights())
    db = st.DeviceBatch(ev, x, zone, vo, velo)
    db.add_ut(uo, ux, ul)
    out = st.run_batch(ctx, db)
    ctx.ut_run(db.velo_s, out.seeds, db.ut, out.long, out.ut_out)
    torch.cuda.synchronize()
    res = out.to_numpy()
    ctx.close()
    assert (res["status"] == 0).all()
    for e in range(b.n_events):
        n = res["ev_off"][e + 1] - res["ev_off"][e]
        assert (n == 0) == (e in empty), (e, n)
        assert res["n_long"][e] == int((res["velo_idx"][res["ev_off"][e]:res["ev_off"][e + 1]] >= 0).sum())


@pytest.mark.parametrize("mode", MODES, ids=["hough", "seq3", "seq3_hough", "final_sel"])
def test_empty_batch_every_mode(mode):
    cfg = st.st_config_default(**mode)
    ctx = st.Context(cfg)
    if mode.get("final_sel"):
        ctx.st_set_ghost_nn(ghost_nn_weights())
    db = st.DeviceBatch(np.zeros(1, np.int64), np.zeros(0, np.float32), np.zeros(0, np.int32),
                        np.zeros(1, np.int64), np.zeros((0, 4), np.float32), max_hits=16)
    db.add_ut(np.zeros(1, np.int64), np.zeros(0, np.float32), np.zeros(0, np.int32))
    out = st.run_batch(ctx, db, cap=16)
    ctx.ut_run(db.velo_s, out.seeds, db.ut, out.long, out.ut_out)
    torch.cuda.synchronize()
    assert out.ev_off.cpu().tolist() == [0]
    ctx.close()


def test_static_entry_in_hlt2_mode(zmx):
    """seeding_run_static takes the configuration's iteration scheme and
    returns seeding_run's result."""
    cfg = st.st_config_default(zmx=zmx, **SEQ3)
    b = workload("run3", n_events=40)
    ctx = st.Context(cfg)
    db = st.DeviceBatch.from_synth(b)
    cap = max(1024, b.n_hits // 4)
    ref = st.DeviceOutputs(b.n_events, cap)
    ctx.seeding_run(db.hits, ref.seeds)
    out = st.DeviceOutputs(b.n_events, cap)
    rc, msg = st.seeding_run_static(cfg, db.hits, out.seeds)
    assert rc == st.ST_OK, msg
    torch.cuda.synchronize()
    r, g = ref.to_numpy(), out.to_numpy()
    for k in ("ev_off", "hits", "params", "state", "n_hits", "status"):
        assert np.array_equal(g[k], r[k]), k
    ctx.close()


def test_pipeline_in_hlt2_mode_equals_direct(zmx):
    b = workload("run3", n_events=64)
    _, gcfg = parity.config_pair(zmx, **SEQ3)
    ctx = st.Context(gcfg)
    direct = st.run_batch(ctx, st.DeviceBatch.from_synth(b)).to_numpy()
    ctx.st_pipeline_configure(n_slots=2, max_events_per_slot=128, max_hits_per_slot=b.n_hits + 16,
                              max_hits_per_event=int(np.diff(b.ev_off).max()), max_velo_per_event=1024,
                              max_velo_per_slot=int(b.velo.shape[0]) + 16)
    hh, hv, keep = st.HostBuffers.inputs(b.ev_off, b.x, b.zone, b.velo_off, b.velo)
    hb = st.HostBuffers(b.n_events, b.n_hits // 4 + 1024)
    t = ctx.pipeline_submit(hh, hv)
    rc, _ = ctx.pipeline_poll(t, hb.seeds, hb.long, 60_000_000)
    assert rc == st.ST_OK
    got = hb.to_numpy()
    ctx.close()
    for k in ("ev_off", "hits", "params", "state", "velo_idx", "chi2"):
        assert np.array_equal(got[k], direct[k]), k


@pytest.mark.parametrize("mode", [dict(uv_mode=1), SEQ3], ids=["hough", "seq3"])
def test_widened_modes_deterministic_across_launch_shapes(mode, zmx):
    b = workload("uneven", n_events=200)
    res = []
    for shape in (dict(), dict(threads_seed=512), dict(threads_seed=128, smem_hits=512, ctas_per_sm=1)):
        _, gcfg = parity.config_pair(zmx, **mode, **shape)
        ctx = st.Context(gcfg)
        res.append(st.run_batch(ctx, st.DeviceBatch.from_synth(b)).to_numpy())
        ctx.close()
    for r in res[1:]:
        for k in ("ev_off", "hits", "params", "state", "velo_idx"):
            assert np.array_equal(r[k], res[0][k]), k
