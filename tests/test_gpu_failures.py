"""Failure paths on the GPU, made to happen without a fault.

* The fused seeding kernel's wait for an event that another CTA is still
  seeding is bounded by the device's global timer.  With the limit set to 0
  every such wait gives up: the kernel must return promptly, every event of
  the launch must carry ST_TIMEOUT, and the next launch on the same context
  (with the default limit) must give the right result.
* pipeline_poll's own wait on the host: 0 us on a pending ticket returns
  ST_PENDING, a short timeout returns ST_TIMEOUT and keeps the ticket, and a
  later poll returns the batch's result, equal to the batch run alone.
"""

import time

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


def _graph_run(ctx, b, db, out):
    g = ctx.st_graph_create(db.hits, db.velo_s, out.seeds, out.long)
    out.status.fill_(123)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.st_graph_launch()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    g.close()
    return out.to_numpy(), dt


def test_fused_wait_runs_out_and_context_recovers(zmx):
    b = workload("run3", n_events=300)
    _, gcfg = parity.config_pair(zmx)
    ctx = st.Context(gcfg)
    direct = st.run_batch(ctx, st.DeviceBatch.from_synth(b))
    torch.cuda.synchronize()
    want = direct.to_numpy()
    db = st.DeviceBatch.from_synth(b)
    cap = int(want["ev_off"][-1]) + 1024
    out = st.DeviceOutputs(b.n_events, cap)
    ctx.st_reserve(b.n_events, b.n_events * db.max_hits, db.max_hits, cap)
    with pytest.raises(st.StError):
        ctx.st_set_wait_limit(-1)
    ctx.st_set_wait_limit(0)
    res, dt = _graph_run(ctx, b, db, out)
    assert (res["status"] == st.ST_TIMEOUT).all(), np.unique(res["status"])
    assert dt < 5.0, dt
    ctx.st_set_wait_limit(200_000_000)
    res, _ = _graph_run(ctx, b, db, out)
    assert (res["status"] == 0).all()
    for k in ("ev_off", "hits", "params", "state", "n_hits", "velo_idx", "chi2", "n_long"):
        assert np.array_equal(res[k], want[k]), k
    ctx.close()


def test_pipeline_poll_timeouts(zmx):
    _, gcfg = parity.config_pair(zmx)
    b = workload("uneven", n_events=2400)
    cuts = list(range(0, 2401, 300))
    ctx = st.Context(gcfg)
    last = b.subset(range(cuts[-2], cuts[-1]))
    alone = st.run_batch(ctx, st.DeviceBatch.from_synth(last, max_hits=16000))
    torch.cuda.synchronize()
    alone = alone.to_numpy()
    ctx.st_pipeline_configure(n_slots=2, max_events_per_slot=300, max_hits_per_slot=300 * 16000,
                              max_hits_per_event=16000, max_velo_per_event=4096)
    keep, tickets = [], []
    for a, c in zip(cuts[:-1], cuts[1:]):
        sub = b.subset(range(a, c))
        hits, velo, k = st.HostBuffers.inputs(sub.ev_off, sub.x, sub.zone, sub.velo_off, sub.velo)
        keep.append(k)
        tickets.append(ctx.pipeline_submit(hits, velo))
    n_ev = cuts[-1] - cuts[-2]
    hb = st.HostBuffers(n_ev, 400 * n_ev + 64)
    # the last of eight batches of 300 uneven events is behind the others
    rc, info = ctx.pipeline_poll(tickets[-1], hb.seeds, hb.long, 0)
    assert rc == st.ST_PENDING and info is None
    rc, info = ctx.pipeline_poll(tickets[-1], hb.seeds, hb.long, 1)
    assert rc == st.ST_TIMEOUT and info is None
    for t, (a, c) in zip(tickets[:-1], zip(cuts[:-2], cuts[1:-1])):
        h2 = st.HostBuffers(c - a, 400 * (c - a) + 64)
        rc, _ = ctx.pipeline_poll(t, h2.seeds, h2.long, 60_000_000)
        assert rc == st.ST_OK
    rc, info = ctx.pipeline_poll(tickets[-1], hb.seeds, hb.long, 60_000_000)
    assert rc == st.ST_OK and info.n_events == n_ev
    got = hb.to_numpy()
    for k in ("ev_off", "hits", "params", "state", "n_hits", "status", "velo_idx", "chi2", "n_long"):
        assert np.array_equal(got[k], alone[k]), k
    ctx.close()
