"""GPU path (through the C ABI) against the FP64 oracle.

Element-by-element comparisons on seeded synthetic events at sizes the oracle
finishes in seconds (several hundred events, many CTA rounds, every zone
populated), sampled comparisons at the benchmark's full batch sizes in the
benchmark's launch configuration, and edge cases.  Acceptance rules and
tolerances are in tests/parity.py.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import parity  # noqa: E402
from conftest import workload  # noqa: E402
from paper_2606_14480_gb300 import st  # noqa: E402
from synth import calibrate_zmatch, make_events  # noqa: E402


@pytest.fixture(scope="module")
def zmx():
    return calibrate_zmatch(7826.0)


def run_gpu(batch, gcfg, cap=None, **kw):
    ctx = st.Context(gcfg)
    db = st.DeviceBatch.from_synth(batch, **kw)
    out = st.run_batch(ctx, db, cap=cap)
    torch.cuda.synchronize()
    res = out.to_numpy()
    cnt = ctx.st_read_counters()
    ctx.close()
    return res, cnt


def assert_seeding_parity(rep: parity.Report):
    parity.assert_seeding(rep)


@pytest.mark.parametrize("name,n", [("tiny", None), ("run3", 200), ("match_stress", 40), ("uneven", 200)])
def test_seeding_parity(name, n, zmx):
    b = workload(name, n_events=n) if n else workload(name)
    ocfg, gcfg = parity.config_pair(zmx)
    gpu, cnt = run_gpu(b, gcfg)
    assert (gpu["status"] == 0).all()
    rep = parity.compare_seeding(gpu, ocfg, b)
    print(name, rep.summary())
    assert_seeding_parity(rep)


def test_counters_match_oracle(zmx):
    b = workload("run3", n_events=100)
    ocfg, gcfg = parity.config_pair(zmx)
    gpu, cnt = run_gpu(b, gcfg)
    refs = oracle.seeding_batch(ocfg, b)
    tot = {k: sum(r["counters"][k] for r in refs) for k in refs[0]["counters"]}
    # pair and triplet counts may differ only by window-edge flips
    for k in ("pairs", "triplets", "ext_ok", "cands", "kept", "uv_init", "uv_cands", "seeds"):
        assert abs(cnt[k] - tot[k]) <= max(2, 1e-4 * tot[k]), (k, cnt[k], tot[k])
    assert cnt["events"] == b.n_events and cnt["hits"] == b.n_hits


@pytest.mark.parametrize("preset", ["calibrated", "paper_table"])
def test_matching_parity(preset, zmx):
    b = workload("run3", n_events=200)
    ocfg, gcfg = parity.config_pair(zmx if preset == "calibrated" else None)
    gpu, cnt = run_gpu(b, gcfg)
    n, untraced, traced, chi_rel = parity.compare_matching(gpu, ocfg, b)
    assert n > 0 and not untraced, (untraced[:5], traced)
    assert chi_rel <= 1e-5
    assert (gpu["velo_idx"] >= 0).sum() > 0.5 * n


@pytest.mark.parametrize("s", [0.5, 0.71, 1.0, 1.41, 2.0])
@pytest.mark.parametrize("which", ["tol_scale", "presel_scale"])
def test_matching_window_sweep(s, which, zmx):
    """Matching stress: 400 VELO segments per event (30% ghosts); the chi2
    tolerances, and separately the preselection cuts, scaled 0.5x-2x."""
    b = workload("match_stress", n_events=30)
    ocfg, gcfg = parity.config_pair(zmx, **{which: s})
    gpu, cnt = run_gpu(b, gcfg)
    n, untraced, traced, chi_rel = parity.compare_matching(gpu, ocfg, b)
    assert n > 0 and not untraced, (untraced[:5], traced)
    assert chi_rel <= 1e-5


def test_velo_unique(zmx):
    b = workload("match_stress", n_events=20)
    ocfg, gcfg = parity.config_pair(zmx, velo_unique=1, tol_scale=2.0)
    gpu, cnt = run_gpu(b, gcfg)
    n, untraced, traced, chi_rel = parity.compare_matching(gpu, ocfg, b)
    assert not untraced, untraced[:5]
    for e in range(b.n_events):
        s0, s1 = gpu["ev_off"][e], gpu["ev_off"][e + 1]
        v = gpu["velo_idx"][s0:s1]
        v = v[v >= 0]
        assert len(v) == len(set(v))


def test_full_size_run3_sampled(zmx):
    """The benchmark's batch (1000 events) in its launch configuration; the
    oracle recomputes a sample of events one by one."""
    b = workload("run3")
    ocfg, gcfg = parity.config_pair(zmx)
    gpu, cnt = run_gpu(b, gcfg)
    rng = np.random.default_rng(11)
    ev = np.sort(rng.choice(b.n_events, 48, replace=False))
    rep = parity.compare_seeding(gpu, ocfg, b, ev)
    print(rep.summary())
    assert_seeding_parity(rep)
    n, untraced, traced, _ = parity.compare_matching(gpu, ocfg, b, ev)
    assert not untraced


def test_full_size_uneven_sampled(zmx):
    """10000 events with 100-15000 hits each in one launch; the sample takes
    the largest events (which exceed the shared-memory staging and use the
    global-memory path) and random ones."""
    b = workload("uneven")
    ocfg, gcfg = parity.config_pair(zmx)
    gpu, cnt = run_gpu(b, gcfg)
    assert (gpu["status"] == 0).all()
    sizes = np.diff(b.ev_off)
    rng = np.random.default_rng(12)
    ev = np.unique(np.concatenate([np.argsort(sizes)[-6:], rng.choice(b.n_events, 24, replace=False)]))
    rep = parity.compare_seeding(gpu, ocfg, b, ev)
    print(rep.summary(), "max hits", sizes.max())
    assert_seeding_parity(rep)


def test_deterministic_across_launch_shapes(zmx):
    """Results do not depend on threads per CTA, CTAs per SM or staging size."""
    b = workload("run3", n_events=150)
    ref = None
    for tune in (dict(), dict(threads_seed=128, threads_build=128, threads_match=64, ctas_per_sm=2),
                 dict(threads_seed=512, smem_hits=0), dict(threads_seed=64, ctas_per_sm=1, smem_hits=512)):
        _, gcfg = parity.config_pair(zmx, **tune)
        gpu, _ = run_gpu(b, gcfg)
        if ref is None:
            ref = gpu
            continue
        for k in ref:
            assert np.array_equal(ref[k], gpu[k]), (tune, k)


def test_staging_boundary(zmx):
    """A half is staged in shared memory by one bulk copy of the 16-byte words
    that hold it (up to three floats more on each side) when those fit the
    staging budget, else read from global memory.  Budgets around one half's
    size (below it, at it, and up to seven hits above it) flip that choice for
    it and for halves of nearby sizes; every result equals the default
    budget's, which equals the oracle's (test_seeding_parity)."""
    b = workload("run3", n_events=40)
    half1 = np.array([int(np.count_nonzero(b.hits_of(e)[1] & 1)) for e in range(b.n_events)])
    n = int(np.median(half1))
    _, gcfg = parity.config_pair(zmx)
    ref, _ = run_gpu(b, gcfg)
    for s in (n - 1, n, n + 1, n + 3, n + 6, n + 7):
        _, gcfg = parity.config_pair(zmx, smem_hits=s)
        gpu, _ = run_gpu(b, gcfg)
        for k in ref:
            assert np.array_equal(ref[k], gpu[k]), (s, k)


def test_graph_replay_matches_direct_run(zmx):
    b = workload("run3", n_events=100)
    _, gcfg = parity.config_pair(zmx)
    direct, _ = run_gpu(b, gcfg)
    ctx = st.Context(gcfg)
    db = st.DeviceBatch.from_synth(b)
    out = st.DeviceOutputs(b.n_events, max(1024, b.n_hits // 4))
    ctx.st_reserve(b.n_events, b.n_events * db.max_hits, db.max_hits, out.cap)
    g = ctx.st_graph_create(db.hits, db.velo_s, out.seeds, out.long)
    for _ in range(3):
        out.velo_idx.fill_(-7)
        g.st_graph_launch()
    torch.cuda.synchronize()
    res = out.to_numpy()
    for k in direct:
        assert np.array_equal(direct[k], res[k]), k
    g.close()
    ctx.close()


def test_edge_cases(zmx):
    """Empty events, invalid zones and positions, oversized events, a layer
    z that disagrees with the geometry, and a seed capacity that is too small
    are reported per event without touching the other events."""
    b = workload("tiny")
    ocfg, gcfg = parity.config_pair(zmx)
    good, _ = run_gpu(b, gcfg)
    # rebuild the batch with special events inserted
    ev = b.ev_off
    xs, zs, zz = [], [], []
    offs = [0]
    kinds = []
    for e in range(b.n_events):
        x = b.x[ev[e]:ev[e + 1]].copy()
        zn = b.zone[ev[e]:ev[e + 1]].copy()
        z = b.z[ev[e]:ev[e + 1]].copy()
        kind = "ok"
        if e == 1:
            x, zn, z = x[:0], zn[:0], z[:0]
            kind = "empty"
        elif e == 3:
            zn[5] = 24
            kind = "bad_zone"
        elif e == 5:
            x[7] = np.nan
            kind = "nan"
        elif e == 7:
            z[2] += 0.5
            kind = "bad_z"
        xs.append(x); zs.append(zn); zz.append(z)
        offs.append(offs[-1] + len(x))
        kinds.append(kind)
    x = np.concatenate(xs); zn = np.concatenate(zs); z = np.concatenate(zz)
    dxdy = np.asarray(list(ocfg.dxdy), np.float32)[zn.clip(0, 23) >> 1]
    db = st.DeviceBatch(np.array(offs), x, zn, b.velo_off, b.velo, z=z, dxdy=dxdy)
    ctx = st.Context(gcfg)
    out = st.run_batch(ctx, db)
    torch.cuda.synchronize()
    res = out.to_numpy()
    for e, kind in enumerate(kinds):
        want = {"ok": 0, "empty": 0, "bad_zone": -1, "nan": -1, "bad_z": -1}[kind]
        assert res["status"][e] == want, (e, kind, res["status"][e])
        n = res["ev_off"][e + 1] - res["ev_off"][e]
        if kind == "ok":
            g0, g1 = good["ev_off"][e], good["ev_off"][e + 1]
            assert np.array_equal(res["hits"][res["ev_off"][e]:res["ev_off"][e + 1]], good["hits"][g0:g1])
        else:
            assert n == 0
    # max_hits smaller than some events: those report ST_OVERFLOW
    sizes = np.diff(b.ev_off)
    mh = int(np.sort(sizes)[len(sizes) // 2])
    db2 = st.DeviceBatch.from_synth(b, max_hits=mh)
    out2 = st.run_batch(ctx, db2)
    torch.cuda.synchronize()
    r2 = out2.to_numpy()
    for e in range(b.n_events):
        assert r2["status"][e] == (-3 if sizes[e] > mh else 0)
    # seed capacity too small: status ST_OVERFLOW, nothing written past cap
    db3 = st.DeviceBatch.from_synth(b)
    out3 = st.DeviceOutputs(b.n_events, 60)
    out3.hits.fill_(-9)
    ctx.seeding_run(db3.hits, out3.seeds)
    torch.cuda.synchronize()
    r3 = out3.to_numpy()
    assert r3["ev_off"][-1] <= 60 and (r3["status"] == -3).any()
    ok = r3["status"] == 0
    for e in np.nonzero(ok)[0]:
        g0, g1 = good["ev_off"][e], good["ev_off"][e + 1]
        s0, s1 = r3["ev_off"][e], r3["ev_off"][e + 1]
        assert np.array_equal(r3["hits"][s0:s1], good["hits"][g0:g1])
    ctx.close()


def test_bad_events_among_many(zmx):
    """More events than the container-build CTAs (608 on a GB300) with
    invalid and oversized events spread among them, so that CTAs take further
    events after rejecting one: every good event's seeds and Long tracks equal
    those of the same event in a batch without the bad ones, directly and
    through the CUDA graph (the fused matching)."""
    b = workload("tiny", n_events=1500)
    _, gcfg = parity.config_pair(zmx)
    ev = b.ev_off
    mh = int(np.diff(ev).max())
    xs, zs, offs, kinds = [], [], [0], []
    for e in range(b.n_events):
        x = b.x[ev[e]:ev[e + 1]].copy()
        zn = b.zone[ev[e]:ev[e + 1]].copy()
        kind = "ok"
        if len(x) and e % 7 == 3:
            zn[len(zn) // 2] = 24
            kind = "bad_zone"
        elif len(x) and e % 11 == 5:
            x[-1] = np.inf
            kind = "inf"
        elif len(x) and e % 13 == 8:
            reps = mh // len(x) + 1
            x, zn = np.tile(x, reps)[:mh + 1], np.tile(zn, reps)[:mh + 1]
            kind = "oversized"
        xs.append(x)
        zs.append(zn)
        offs.append(offs[-1] + len(x))
        kinds.append(kind)
    assert kinds.count("ok") > 1000
    want = {"ok": 0, "bad_zone": -1, "inf": -1, "oversized": -3}

    ctx = st.Context(gcfg)
    clean = st.run_batch(ctx, st.DeviceBatch.from_synth(b, max_hits=mh))
    torch.cuda.synchronize()
    ref = clean.to_numpy()
    assert (ref["status"] == 0).all()
    db = st.DeviceBatch(np.array(offs), np.concatenate(xs), np.concatenate(zs), b.velo_off, b.velo, max_hits=mh)
    direct = st.run_batch(ctx, db)
    torch.cuda.synchronize()
    res_direct = direct.to_numpy()
    cap = int(ref["ev_off"][-1]) + 1024
    out = st.DeviceOutputs(b.n_events, cap)
    ctx.st_reserve(b.n_events, b.n_events * mh, mh, cap)
    g = ctx.st_graph_create(db.hits, db.velo_s, out.seeds, out.long)
    g.st_graph_launch()
    torch.cuda.synchronize()
    res_graph = out.to_numpy()
    g.close()
    ctx.close()
    for res in (res_direct, res_graph):
        for e, kind in enumerate(kinds):
            assert res["status"][e] == want[kind], (e, kind, res["status"][e])
            s0, s1 = res["ev_off"][e], res["ev_off"][e + 1]
            if kind != "ok":
                assert s1 == s0 and res["n_long"][e] == 0
                continue
            r0, r1 = ref["ev_off"][e], ref["ev_off"][e + 1]
            assert np.array_equal(res["hits"][s0:s1], ref["hits"][r0:r1]), e
            assert np.array_equal(res["velo_idx"][s0:s1], ref["velo_idx"][r0:r1]), e
            assert res["n_long"][e] == ref["n_long"][e], e


def test_empty_batch():
    ctx = st.Context(st.st_config_default())
    db = st.DeviceBatch(np.zeros(1, np.int64), np.zeros(0, np.float32), np.zeros(0, np.int32),
                        np.zeros(1, np.int64), np.zeros((0, 4), np.float32), max_hits=16)
    out = st.run_batch(ctx, db, cap=16)
    torch.cuda.synchronize()
    assert out.ev_off.cpu().tolist() == [0]
    ctx.close()


def test_single_track_events_and_noise_only(zmx):
    """Degenerate events: one noise-free track, only noise hits."""
    ocfg, gcfg = parity.config_pair(zmx)
    b1 = make_events(8, seed=77, tracks=("fixed", 1), noise_frac=0.0, eff=1.0, sigma_x=0.0,
                     p_range=(3.5, 100), velo_ghosts_per_track=1.0, velo_sigma=(0, 0))
    gpu, _ = run_gpu(b1, gcfg)
    assert (np.diff(gpu["ev_off"]) == 1).all()
    assert_seeding_parity(parity.compare_seeding(gpu, ocfg, b1))
    # noise-only events
    rng = np.random.default_rng(5)
    n = 400
    x = rng.uniform(-3200, 3200, 8 * n).astype(np.float32)
    zn = rng.integers(0, 24, 8 * n).astype(np.int32)
    db = st.DeviceBatch(np.arange(9) * n, x, zn, np.zeros(9, np.int64), np.zeros((0, 4), np.float32))
    ctx = st.Context(gcfg)
    out = st.run_batch(ctx, db)
    torch.cuda.synchronize()
    res = out.to_numpy()
    for e in range(8):
        ref = oracle.seeding_event(ocfg, x[e * n:(e + 1) * n], zn[e * n:(e + 1) * n])["seeds"]
        s0, s1 = res["ev_off"][e], res["ev_off"][e + 1]
        assert {tuple(h) for h in res["hits"][s0:s1]} == {tuple(h) for h in ref["hits"]}
        assert (res["velo_idx"][s0:s1] == -1).all()
    ctx.close()


def test_pipeline_alone_and_in_the_mix(zmx):
    """Serving: batches submitted together are packed into shared launches and
    overlap on the device; each batch's result equals its result alone."""
    _, gcfg = parity.config_pair(zmx)
    b = workload("run3", n_events=300)
    cuts = [0, 7, 8, 60, 61, 140, 300]
    alone = []
    ctx = st.Context(gcfg)
    for a, c in zip(cuts[:-1], cuts[1:]):
        sub = b.subset(range(a, c))
        out = st.run_batch(ctx, st.DeviceBatch.from_synth(sub, max_hits=8000))
        torch.cuda.synchronize()
        alone.append(out.to_numpy())
    ctx.st_pipeline_configure(n_slots=3, max_events_per_slot=256, max_hits_per_slot=256 * 4000,
                              max_hits_per_event=8000, max_velo_per_event=1024)
    tickets, keep = [], []
    for a, c in zip(cuts[:-1], cuts[1:]):
        sub = b.subset(range(a, c))
        hits, velo, k = st.HostBuffers.inputs(sub.ev_off, sub.x, sub.zone, sub.velo_off, sub.velo)
        keep.append(k)
        tickets.append(ctx.pipeline_submit(hits, velo))
    for i, t in enumerate(tickets):
        n_ev = cuts[i + 1] - cuts[i]
        hb = st.HostBuffers(n_ev, 200 * n_ev + 16)
        rc, info = ctx.pipeline_poll(t, hb.seeds, hb.long, 30_000_000)
        assert rc == st.ST_OK
        got = hb.to_numpy()
        for k in ("ev_off", "hits", "params", "state", "n_hits", "status", "velo_idx", "chi2", "n_long"):
            assert np.array_equal(got[k], alone[i][k]), (i, k)
        assert info.n_events == n_ev and info.t_returned_ns >= info.t_done_ns >= info.t_launch_ns >= info.t_submit_ns
    # unknown ticket, and a poll that times out on nothing pending is an error
    assert ctx.lib.pipeline_poll(ctx.h, 123456789, None, None, 0, None) == st.ST_EINVAL
    ctx.close()


def _alone(ctx, b, a, c):
    sub = b.subset(range(a, c))
    out = st.run_batch(ctx, st.DeviceBatch.from_synth(sub, max_hits=8000))
    torch.cuda.synchronize()
    return out.to_numpy()


def _poll_ok(ctx, t, n_ev):
    hb = st.HostBuffers(n_ev, 300 * n_ev + 64)
    rc, info = ctx.pipeline_poll(t, hb.seeds, hb.long, 60_000_000)
    assert rc == st.ST_OK
    return hb.to_numpy()


def _same(got, want):
    for k in ("ev_off", "hits", "params", "state", "n_hits", "status", "velo_idx", "chi2", "n_long"):
        assert np.array_equal(got[k], want[k]), k


def test_pipeline_ring_wraps(zmx):
    """Small input rings (two slots' worth of hits) wrap many times while a
    poller thread collects results; packing stops at every wrap."""
    import threading
    _, gcfg = parity.config_pair(zmx)
    b = workload("run3", n_events=120)
    rng = np.random.default_rng(21)
    cuts = [0]
    while cuts[-1] < b.n_events:
        cuts.append(min(b.n_events, cuts[-1] + int(rng.integers(1, 8))))
    ctx = st.Context(gcfg)
    alone = [_alone(ctx, b, a, c) for a, c in zip(cuts[:-1], cuts[1:])]
    ctx.st_pipeline_configure(n_slots=2, max_events_per_slot=16, max_hits_per_slot=20000,
                              max_hits_per_event=8000, max_velo_per_event=1024, max_velo_per_slot=4000)
    tickets = [None] * (len(cuts) - 1)
    got = [None] * len(tickets)
    err = []

    def poller():
        try:
            for i in range(len(tickets)):
                while tickets[i] is None:
                    time.sleep(0.0005)
                got[i] = _poll_ok(ctx, tickets[i], cuts[i + 1] - cuts[i])
        except Exception as exc:
            err.append(exc)

    import time
    th = threading.Thread(target=poller)
    th.start()
    keep = []
    for i, (a, c) in enumerate(zip(cuts[:-1], cuts[1:])):
        sub = b.subset(range(a, c))
        hits, velo, k = st.HostBuffers.inputs(sub.ev_off, sub.x, sub.zone, sub.velo_off, sub.velo)
        keep.append(k)
        tickets[i] = ctx.pipeline_submit(hits, velo)
    th.join(timeout=120)
    assert not th.is_alive() and not err, err
    for g, a in zip(got, alone):
        _same(g, a)
    ctx.close()


def test_pipeline_threads_and_shuffled_polls(zmx):
    """Four host threads submit concurrently; results are polled in a
    shuffled order and each equals its batch run alone."""
    import threading
    _, gcfg = parity.config_pair(zmx)
    b = workload("run3", n_events=160)
    cuts = list(range(0, 161, 10))
    ctx = st.Context(gcfg)
    alone = [_alone(ctx, b, a, c) for a, c in zip(cuts[:-1], cuts[1:])]
    ctx.st_pipeline_configure(n_slots=3, max_events_per_slot=64, max_hits_per_slot=64 * 4000,
                              max_hits_per_event=8000, max_velo_per_event=1024)
    tickets = [None] * len(alone)
    errs = []

    def submitter(idx):
        try:
            for i in idx:
                sub = b.subset(range(cuts[i], cuts[i + 1]))
                hits, velo, k = st.HostBuffers.inputs(sub.ev_off, sub.x, sub.zone, sub.velo_off, sub.velo)
                tickets[i] = ctx.pipeline_submit(hits, velo)
                del k
        except Exception as exc:
            errs.append(exc)

    ths = [threading.Thread(target=submitter, args=(list(range(j, len(alone), 4)),)) for j in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join(timeout=120)
    assert not errs, errs
    order = np.random.default_rng(5).permutation(len(alone))
    for i in order:
        _same(_poll_ok(ctx, tickets[i], 10), alone[i])
    ctx.close()
