"""Full-size GPU runs of the matching-stress batch and of the serving path.

* Matching stress: the whole 2000-event batch (280 tracks and 120 ghost VELO
  segments per event, so 400 VELO segments, 40% noise hits) is seeded once;
  matching then runs at each of the ten sweep points (the chi2 tolerances,
  and separately the preselection cuts, scaled 0.5x-2x).  The oracle matches
  a sample of 64 events per point on the GPU's own seed states (the events
  with the most seeds and a random draw).  Seeding is compared on a sample of
  64 events, the largest included.
* Serving: a stream of requests of log-uniform size 1-4096 events (the
  largest size included) from the benchmark's 8192-event serving pool goes
  through pipeline_submit / pipeline_poll with a collector polling in
  completion order; a sample of the results, the largest requests included,
  must equal the same batch run alone through run_batch, byte for byte.
"""

import threading
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
from synth import calibrate_zmatch, make_workload  # noqa: E402
from synth.events import poisson_arrivals, serving_requests  # noqa: E402

SWEEP = [(w, s) for w in ("tol_scale", "presel_scale") for s in (0.5, 0.71, 1.0, 1.41, 2.0)]


@pytest.fixture(scope="module")
def zmx():
    return calibrate_zmatch(7826.0)


@pytest.fixture(scope="module")
def stress(zmx):
    """The matching-stress batch seeded once on the GPU (default config)."""
    b = workload("match_stress")
    ocfg, gcfg = parity.config_pair(zmx)
    ctx = st.Context(gcfg)
    db = st.DeviceBatch.from_synth(b)
    out = st.DeviceOutputs(b.n_events, max(1024, b.n_hits // 4))
    ctx.seeding_run(db.hits, out.seeds)
    torch.cuda.synchronize()
    seeds = out.to_numpy()
    ctx.close()
    assert (seeds["status"] == 0).all()
    return b, db, out, seeds


def test_match_stress_full_size_seeding_sampled(zmx, stress):
    b, db, out, seeds = stress
    ocfg, _ = parity.config_pair(zmx)
    sizes = np.diff(b.ev_off)
    rng = np.random.default_rng(41)
    ev = np.unique(np.concatenate([np.argsort(sizes)[-16:], rng.choice(b.n_events, 48, replace=False)]))
    assert len(ev) >= 60
    rep = parity.compare_seeding(seeds, ocfg, b, ev)
    print(rep.summary())
    parity.assert_seeding(rep)


@pytest.mark.parametrize("which,s", SWEEP)
def test_match_stress_full_size_sweep(which, s, zmx, stress):
    b, db, out, seeds = stress
    ocfg, gcfg = parity.config_pair(zmx, **{which: s})
    ctx = st.Context(gcfg)
    ctx.seeding_run(db.hits, out.seeds)  # matching needs this context's seeding (the seeds do not change)
    ctx.matching_run(db.velo_s, out.seeds, out.long)
    torch.cuda.synchronize()
    got = out.to_numpy()
    cnt = ctx.st_read_counters()
    ctx.close()
    for k in ("ev_off", "hits", "params", "state", "n_hits"):
        assert np.array_equal(got[k], seeds[k]), k
    assert cnt["match_pairs"] == sum(int(b.velo_off[e + 1] - b.velo_off[e]) * int(seeds["ev_off"][e + 1] -
                                     seeds["ev_off"][e]) for e in range(b.n_events))
    assert 0 < cnt["match_eval"] <= cnt["match_pairs"]
    n_seeds = np.diff(got["ev_off"])
    rng = np.random.default_rng(int(100 * s) + (0 if which == "tol_scale" else 7))
    ev = np.unique(np.concatenate([np.argsort(n_seeds)[-16:], rng.choice(b.n_events, 56, replace=False)]))
    assert len(ev) >= 64
    assert np.all(np.diff(b.velo_off)[ev] == 400)
    n, untraced, traced, chi_rel = parity.compare_matching(got, ocfg, b, ev)
    print(which, s, "seeds", n, "traced", traced, "evaluated/grid", cnt["match_eval"] / cnt["match_pairs"])
    assert n > 0 and not untraced, (untraced[:5], traced)
    assert traced <= (1.0 - parity.AGREE_MIN) * n
    assert chi_rel <= 1e-5


def test_served_results_equal_alone(zmx):
    _, gcfg = parity.config_pair(zmx)
    pool = make_workload("uneven", n_events=8192, seed=1005)
    ev_off = np.ascontiguousarray(pool.ev_off, np.int64)
    velo_off = np.ascontiguousarray(pool.velo_off, np.int64)
    x = np.ascontiguousarray(pool.x, np.float32)
    zone = np.ascontiguousarray(pool.zone, np.int32)
    velo = np.ascontiguousarray(pool.velo, np.float32)
    mh = int(np.max(np.diff(ev_off)))
    sizes = list(serving_requests(24000, seed=1011))
    sizes[len(sizes) // 2] = 4096  # the largest request size, in the middle of the stream
    sizes = np.array(sizes)
    rng = np.random.default_rng(1012)
    starts = [int(rng.integers(0, pool.n_events - n + 1)) for n in sizes]
    arr = poisson_arrivals(len(sizes), 200.0, seed=1013)
    ctx = st.Context(gcfg)
    ctx.st_pipeline_configure(n_slots=4, max_events_per_slot=4096, max_hits_per_slot=4096 * 4000,
                              max_hits_per_event=mh, max_velo_per_event=4096, max_velo_per_slot=4096 * 1024)
    n_req = len(sizes)
    tickets = [None] * n_req
    got = [None] * n_req
    errs = []

    def collector():
        try:
            pending, nxt, done, bufs = [], 0, 0, {}
            while done < n_req:
                while nxt < n_req and tickets[nxt] is not None:
                    n = int(sizes[nxt])
                    nh = int(ev_off[starts[nxt] + n] - ev_off[starts[nxt]])
                    bufs[nxt] = st.HostBuffers(n, max(1024, nh // 4))
                    pending.append(nxt)
                    nxt += 1
                hit = False
                for i in list(pending[:32]):
                    hb = bufs[i]
                    rc, _ = ctx.pipeline_poll(tickets[i], hb.seeds, hb.long, 0)
                    if rc == st.ST_OK:
                        got[i] = hb.to_numpy()
                        del bufs[i]
                        pending.remove(i)
                        done += 1
                        hit = True
                if not hit:
                    time.sleep(0.0002)
        except Exception as exc:
            errs.append(exc)

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for i in range(n_req):
        w = arr[i] - (time.perf_counter() - t0)
        if w > 0:
            time.sleep(w)
        s0, n = starts[i], int(sizes[i])
        hits = st.StHits(n, ev_off[s0:].ctypes.data, x.ctypes.data, zone.ctypes.data, None, None, mh, 0)
        vel = st.StVelo(n, velo_off[s0:].ctypes.data, velo.ctypes.data)
        tickets[i] = ctx.pipeline_submit(hits, vel)
    th.join(timeout=300)
    assert not th.is_alive() and not errs, errs
    order = np.argsort(sizes)
    sample = np.unique(np.concatenate([order[-4:], order[:6], rng.choice(n_req, 8, replace=False)]))
    assert sizes[sample].max() == 4096
    alone_ctx = st.Context(gcfg)
    for i in sample:
        sub = pool.subset(range(starts[i], starts[i] + int(sizes[i])))
        ref = st.run_batch(alone_ctx, st.DeviceBatch.from_synth(sub, max_hits=mh))
        torch.cuda.synchronize()
        ref = ref.to_numpy()
        for k in ("ev_off", "hits", "params", "state", "n_hits", "status", "velo_idx", "chi2", "n_long"):
            assert np.array_equal(got[i][k], ref[k]), (i, int(sizes[i]), k)
    alone_ctx.close()
    ctx.close()
