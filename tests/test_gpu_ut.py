"""UT hits of the Long tracks (Section 4.3) on the GPU against the oracle.

The oracle runs on the GPU's own seed states and matching result (as in the
matching parity tests) with the same float32 UT hits; per seed the attached
UT hits and the hit-count decision must be equal unless a window or tie
decision of that seed lies within TAU of flipping, and gamma_x must agree
within GAMMA_TOL: a gamma difference moves the UT prediction by
dgamma * dz^2, and the position bar of 1e-3 mm at the farthest UT layer
(dz = 1872.5 mm) gives 1e-3 / 1872.5^2 = 2.85e-10 per mm."""

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
from synth import calibrate_zmatch  # noqa: E402

GAMMA_TOL = 1e-3 / 1872.5 ** 2


@pytest.fixture(scope="module")
def zmx():
    return calibrate_zmatch(7826.0)


def run_ut(batch, gcfg):
    ctx = st.Context(gcfg)
    db = st.DeviceBatch.from_synth(batch)
    out = st.run_batch(ctx, db)
    torch.cuda.synchronize()
    pre = out.velo_idx.cpu().numpy().copy()
    ctx.ut_run(db.velo_s, out.seeds, db.ut, out.long, out.ut_out)
    torch.cuda.synchronize()
    res = out.to_numpy()
    ctx.close()
    return res, pre


def compare_ut(gpu, pre, ocfg, batch, tau=parity.TAU):
    n_long = n_hits = 0
    untraced, traced, max_d = [], 0, 0.0
    for e in range(batch.n_events):
        s0, s1 = int(gpu["ev_off"][e]), int(gpu["ev_off"][e + 1])
        ux, ul = batch.ut_of(e)
        r = oracle.ut_search(ocfg, batch.velo_of(e), gpu["state"][s0:s1], pre[s0:s1], ux, ul, ledger_tau=1e-4)
        assert r["status"] == 0
        led = r["ledger"]
        near = {int(h[0]) for h in led[led["margin"] <= tau]["hits"]} if len(led) else set()
        gh, gn, gv = gpu["ut_hits"][s0:s1], gpu["ut_n"][s0:s1].astype(np.int32), gpu["velo_idx"][s0:s1]
        for k in range(s1 - s0):
            if pre[s0 + k] < 0:
                continue
            n_long += 1
            same = np.array_equal(gh[k], r["ut_hits"][k]) and gn[k] == r["n_ut"][k] and gv[k] == r["velo_idx"][k]
            if not same:
                if k in near:
                    traced += 1
                else:
                    untraced.append((e, k, gh[k].tolist(), r["ut_hits"][k].tolist()))
                continue
            n_hits += int(gn[k])
            max_d = max(max_d, abs(float(gpu["ut_gamma"][s0 + k]) - float(r["gamma"][k])))
    return n_long, n_hits, untraced, traced, max_d


@pytest.mark.parametrize("name,n", [("run3", 200), ("match_stress", 40), ("uneven", 150)])
def test_ut_parity(name, n, zmx):
    b = workload(name, n_events=n)
    ocfg, gcfg = parity.config_pair(zmx)
    gpu, pre = run_ut(b, gcfg)
    n_long, n_hits, untraced, traced, max_d = compare_ut(gpu, pre, ocfg, b)
    print(name, n_long, n_hits, traced, max_d)
    assert n_long > 0 and n_hits > 3 * n_long * 0.9
    assert not untraced, untraced[:5]
    assert max_d <= GAMMA_TOL
    for e in range(b.n_events):
        s0, s1 = int(gpu["ev_off"][e]), int(gpu["ev_off"][e + 1])
        assert gpu["n_long"][e] == int((gpu["velo_idx"][s0:s1] >= 0).sum())


def test_ut_no_requirement_keeps_matches(zmx):
    """ut_min_hits = 0: UT hits are attached, no Long track is dropped."""
    b = workload("run3", n_events=50)
    _, gcfg = parity.config_pair(zmx, ut_min_hits=0)
    gpu, pre = run_ut(b, gcfg)
    assert np.array_equal(gpu["velo_idx"], pre[: len(gpu["velo_idx"])])
    assert (gpu["ut_n"][pre[: len(gpu["velo_idx"])] >= 0] >= 3).mean() > 0.98


def test_ut_invalid_hit_marks_event(zmx):
    b = workload("tiny")
    _, gcfg = parity.config_pair(zmx)
    ctx = st.Context(gcfg)
    db = st.DeviceBatch.from_synth(b)
    layer = b.ut_layer.copy()
    e_bad = 3
    layer[b.ut_off[e_bad]] = 7
    db.add_ut(b.ut_off, b.ut_x, layer)
    out = st.run_batch(ctx, db)
    ctx.ut_run(db.velo_s, out.seeds, db.ut, out.long, out.ut_out)
    torch.cuda.synchronize()
    res = out.to_numpy()
    ctx.close()
    assert res["status"][e_bad] == -1
    assert all(res["status"][e] == 0 for e in range(b.n_events) if e != e_bad)
    s0, s1 = res["ev_off"][e_bad], res["ev_off"][e_bad + 1]
    assert (res["ut_n"][s0:s1] == 0).all() and (res["velo_idx"][s0:s1] == -1).all()
