"""seeding_run_static: seeding without any device allocation.

Some callers cannot call cudaMalloc (a process whose device memory belongs to a
host framework's allocator, or a real-time loop that forbids allocation after
start-up because it can synchronise the device).  seeding_run_static serves
them with all of its scratch in a fixed array inside the library.  This test
calls it through the C ABI twice in a row, on two different batches, and checks
each output against seeding_run's (the existing entry point) for the same
batch; the second call also shows that what the first call left in the shared
array does not leak into the next result.  A batch beyond the array's limit is
rejected with ST_OVERFLOW and a message.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2606_14480_gb300 import st  # noqa: E402
from synth import calibrate_zmatch, make_workload  # noqa: E402


def _outputs_equal(a, b):
    for k in ("ev_off", "hits", "params", "state", "n_hits", "status"):
        assert np.array_equal(a[k], b[k]), k


def test_static_scratch_seeding_equals_seeding_run():
    cfg = st.st_config_default(zmx=calibrate_zmatch(7826.0, n_tracks=20000))
    batches = [make_workload("run3", n_events=48, seed=2001), make_workload("tiny", n_events=10, seed=2002)]
    ctx = st.Context(cfg)
    for call, b in enumerate(batches):
        db = st.DeviceBatch.from_synth(b)
        cap = max(1024, b.n_hits // 4)
        ref = st.DeviceOutputs(b.n_events, cap)
        ctx.seeding_run(db.hits, ref.seeds)
        out = st.DeviceOutputs(b.n_events, cap)
        out.hits.fill_(-5)
        out.params.fill_(7.0)
        rc, msg = st.seeding_run_static(cfg, db.hits, out.seeds)
        assert rc == st.ST_OK, (call, msg)
        torch.cuda.synchronize()
        r, g = ref.to_numpy(), out.to_numpy()
        assert (r["status"] == 0).all() and r["ev_off"][-1] > 0
        _outputs_equal(g, r)
    ctx.close()


def test_static_scratch_call_allocates_nothing():
    """After a first call (which may load the kernels' code on the device), a
    further call leaves the device's free memory unchanged: nothing is
    allocated, by the library or by anything it calls.  Every buffer the
    calls use is made before the first reading."""
    cfg = st.st_config_default()
    b = make_workload("run3", n_events=32, seed=2004)
    db = st.DeviceBatch.from_synth(b)
    outs = [st.DeviceOutputs(b.n_events, max(1024, b.n_hits // 4)) for _ in range(2)]
    rc, msg = st.seeding_run_static(cfg, db.hits, outs[0].seeds)
    assert rc == st.ST_OK, msg
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc, msg = st.seeding_run_static(cfg, db.hits, outs[1].seeds)
        assert rc == st.ST_OK, msg
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    _outputs_equal(outs[0].to_numpy(), outs[1].to_numpy())


def test_static_scratch_checks_shared_memory_and_launch_shape():
    """A configuration that st_create refuses for its shared memory is refused
    here too, before anything runs; ctas_per_sm changes the launch shape, not
    the result."""
    b = make_workload("tiny", n_events=10, seed=2005)
    db = st.DeviceBatch.from_synth(b)
    out = st.DeviceOutputs(b.n_events, 2048)
    rc, msg = st.seeding_run_static(st.st_config_default(smem_hits=32768), db.hits, out.seeds)
    assert rc == st.ST_EINVAL and "shared memory" in msg, (rc, msg)
    res = []
    for cps in (0, 1):
        o = st.DeviceOutputs(b.n_events, 2048)
        rc, msg = st.seeding_run_static(st.st_config_default(ctas_per_sm=cps), db.hits, o.seeds)
        assert rc == st.ST_OK, msg
        torch.cuda.synchronize()
        res.append(o.to_numpy())
    _outputs_equal(res[0], res[1])


def test_static_scratch_rejects_oversized_batch():
    cfg = st.st_config_default()
    b = make_workload("tiny", n_events=10, seed=2003)
    db = st.DeviceBatch.from_synth(b)
    # a seed capacity whose pool alone exceeds the array
    big = st.DeviceOutputs(b.n_events, 1)
    seeds = st.StSeeds(1 << 20, big.seeds.ev_off, big.seeds.hits, big.seeds.params, big.seeds.state,
                       big.seeds.n_hits, big.seeds.status)
    rc, msg = st.seeding_run_static(cfg, db.hits, seeds)
    assert rc == st.ST_OVERFLOW and "static scratch" in msg
    # an event size above the limit
    h = st.StHits(db.hits.n_events, db.hits.ev_off, db.hits.x, db.hits.zone, None, None, 20000, 0)
    rc, msg = st.seeding_run_static(cfg, h, big.seeds)
    assert rc == st.ST_OVERFLOW and "max_hits_per_event" in msg
    torch.cuda.synchronize()
