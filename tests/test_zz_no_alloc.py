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
