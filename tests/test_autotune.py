"""The autotuner: its truth scoring (CPU), its search spaces, and on the GPU
that every window-grid point agrees with the oracle at the same configuration
values and that launch-shape tuning never changes the outputs."""

import numpy as np
import pytest

from conftest import truth_track_of, workload
from paper_2606_14480_gb300 import autotune


def _outputs_from_lists(per_event):
    """Outputs dict (ev_off, hits) from per-event lists of hit lists."""
    ev = [0]
    rows = []
    for seeds in per_event:
        for h in seeds:
            rows.append(list(h) + [-1] * (12 - len(h)))
        ev.append(len(rows))
    return {"ev_off": np.array(ev, np.int32), "hits": np.array(rows, np.int32).reshape(-1, 12)}


def test_quality_against_a_loop_over_seeds():
    """Vectorised purity / efficiency equals a plain loop over seeds with the
    majority-track rule, on seeds assembled from truth with planted impurities."""
    b = workload("tiny")
    calib = autotune.calibration_from_synth(b, p_min_gev=0.0, min_layers=8)
    rng = np.random.default_rng(3)
    per_event = []
    for e in range(b.n_events):
        n = int(b.ev_off[e + 1] - b.ev_off[e])
        tr = b.tracks_of(e)
        seeds = []
        for k in range(len(tr["p"])):
            h = [int(v) for v in tr["layer_hit"][k] if v >= 0]
            if not h or rng.random() < 0.2:
                continue  # a missed track
            r = rng.random()
            if r < 0.2:  # replace hits by random ones: purity drops
                for j in rng.choice(len(h), size=min(len(h), int(rng.integers(1, 6))), replace=False):
                    h[j] = int(rng.integers(0, n))
            seeds.append(h)
        seeds.append([int(v) for v in rng.choice(n, size=8, replace=False)])  # a ghost
        per_event.append(seeds)
    out = _outputs_from_lists(per_event)
    eff, ghost = autotune.quality(calib, out)
    # the same numbers by a loop
    found, nghost, nseed = set(), 0, 0
    for e, seeds in enumerate(per_event):
        for h in seeds:
            nseed += 1
            t, pur = truth_track_of(b, e, h)
            if t < 0 or pur < 0.7:
                nghost += 1
            else:
                found.add(t)
    want_eff = len(found & set(calib.reconstructible.tolist())) / len(calib.reconstructible)
    assert eff == pytest.approx(want_eff, abs=1e-12)
    assert ghost == pytest.approx(nghost / nseed, abs=1e-12)
    assert 0.3 < eff < 1.0 and ghost > 0


def test_quality_perfect_seeds():
    b = workload("tiny")
    calib = autotune.calibration_from_synth(b, p_min_gev=0.0, min_layers=1)
    per_event = [[[int(v) for v in b.tracks_of(e)["layer_hit"][k] if v >= 0]
                  for k in range(len(b.tracks_of(e)["p"])) if (b.tracks_of(e)["layer_hit"][k] >= 0).any()]
                 for e in range(b.n_events)]
    eff, ghost = autotune.quality(calib, _outputs_from_lists(per_event))
    assert eff == 1.0 and ghost == 0.0


def test_search_spaces_hold_the_defaults():
    from paper_2606_14480_gb300 import st
    cfg = st.st_config_default()
    for k, values in autotune.LAUNCH_SPACE.items():
        assert getattr(cfg, k) in values, k
    first = autotune.WINDOW_GRID[0]
    for k, v in first.items():
        assert getattr(cfg, k) == v, k
    assert len({tuple(sorted(p.items())) for p in autotune.WINDOW_GRID}) == len(autotune.WINDOW_GRID)


def test_tuned_windows_record():
    """The committed window pick is a grid point within the tuner's budget,
    and the benchmark's arms read it the same way."""
    rec = autotune.tuned_windows_record()
    if rec is None:
        pytest.skip("no tuned_windows.json")
    w = autotune.tuned_windows()
    assert set(w) <= set(autotune.WINDOW_KEYS)
    assert any(all(abs(p[k] - w[k]) < 1e-12 for k in w) for p in autotune.WINDOW_GRID)
    ref = rec["paper_widths"]
    assert ref["overrides"] == autotune.WINDOW_GRID[0]
    assert rec["eff"] >= ref["eff"] - rec["budget"]["eff_drop"]
    assert rec["ghost"] <= ref["ghost"] + rec["budget"]["ghost_rise"]
    picked = [p for p in rec["grid"] if p["overrides"] == rec["overrides"]]
    assert len(picked) == 1 and picked[0]["ok"]
    assert all(p["ms"] >= rec["ms"] for p in rec["grid"] if p["ok"])


# ------------------------------------------------------------------- GPU

def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.gpu
@pytest.mark.parametrize("point", range(len(autotune.WINDOW_GRID)))
def test_window_grid_point_parity(point):
    """Each window-grid point the tuner may pick, on the GPU and in the oracle
    at the same configuration values."""
    _gpu()
    import parity
    from paper_2606_14480_gb300 import st
    from synth import calibrate_zmatch
    b = workload("run3", n_events=40)
    zmx = calibrate_zmatch(7826.0)
    ocfg, gcfg = parity.config_pair(zmx, **autotune.WINDOW_GRID[point])
    ctx = st.Context(gcfg)
    out = st.run_batch(ctx, st.DeviceBatch.from_synth(b))
    gpu = out.to_numpy()
    ctx.close()
    assert (gpu["status"] == 0).all()
    rep = parity.compare_seeding(gpu, ocfg, b)
    assert rep.agreement >= parity.AGREE_MIN, rep.summary()
    assert not rep.untraced and not rep.bad_params, rep.summary()


@pytest.mark.gpu
def test_launch_tuning_keeps_outputs():
    _gpu()
    from synth import calibrate_zmatch
    b = workload("uneven", n_events=300)
    calib = autotune.calibration_from_synth(b)
    base = {"zmx": calibrate_zmatch(7826.0)}
    space = {"threads_seed": (128, 256, 512), "ctas_per_sm": (0, 1), "smem_hits": (1536, 2048)}
    r = autotune.tune_launch(base, calib, space=space, passes=1, reps=2, flush_mb=64)
    assert all(p.ok for p in r.points), [p.note for p in r.points if not p.ok]
    assert len(r.points) >= 4
    assert r.best_ms <= r.start_ms


@pytest.mark.gpu
def test_window_tuning_picks_within_budget():
    _gpu()
    from synth import calibrate_zmatch
    b = workload("run3", n_events=200)
    calib = autotune.calibration_from_synth(b)
    base = {"zmx": calibrate_zmatch(7826.0)}
    grid = autotune.WINDOW_GRID[:1] + autotune.WINDOW_GRID[-2:]
    r = autotune.tune_windows(base, calib, grid=grid, reps=2, flush_mb=64)
    ref = r.points[0]
    assert 0.9 < ref.eff <= 1.0 and 0.0 <= ref.ghost < 0.1
    pick = next(p for p in r.points if p.overrides == r.best)
    assert pick.eff >= ref.eff - 0.002 and pick.ghost <= ref.ghost + 0.002


@pytest.mark.gpu
def test_applied_windows_full_size_parity():
    """The benchmark's configuration: the full 1000-event Run-3-like batch at
    the applied (tuned) window widths, the oracle at the same values on a
    sample of 48 events, seeding and matching."""
    _gpu()
    import parity
    from paper_2606_14480_gb300 import st
    from synth import calibrate_zmatch
    w = autotune.tuned_windows()
    b = workload("run3")
    zmx = calibrate_zmatch(7826.0)
    ocfg, gcfg = parity.config_pair(zmx, **w)
    ctx = st.Context(gcfg)
    out = st.run_batch(ctx, st.DeviceBatch.from_synth(b))
    gpu = out.to_numpy()
    ctx.close()
    assert (gpu["status"] == 0).all()
    rng = np.random.default_rng(17)
    ev = np.sort(rng.choice(b.n_events, 48, replace=False))
    rep = parity.compare_seeding(gpu, ocfg, b, ev)
    print(w, rep.summary())
    parity.assert_seeding(rep)
    n, untraced, traced, _ = parity.compare_matching(gpu, ocfg, b, ev)
    assert not untraced, untraced[:5]
