"""The matching's final selection (Section 4.4: ghost network, ghost
probability cut, clone removal) on the GPU against the oracle.

The oracle matches the GPU's own float32 seed states (as in the matching
parity tests) and applies its final selection with the GPU's seed hit
counts and the same seeded weights; per seed the kept VELO segment must be
equal unless a matching or selection decision of that seed lies within TAU
of its threshold, and the ghost probabilities must agree within 2e-5."""

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
from synth import calibrate_zmatch, ghost_nn_weights  # noqa: E402

GP_TOL = 2e-5


@pytest.fixture(scope="module")
def zmx():
    return calibrate_zmatch(7826.0)


def run_final(batch, gcfg, nn):
    ctx = st.Context(gcfg)
    ctx.st_set_ghost_nn(nn)
    db = st.DeviceBatch.from_synth(batch)
    out = st.run_batch(ctx, db)
    torch.cuda.synchronize()
    res = out.to_numpy()
    ctx.close()
    return res


def compare_final(gpu, ocfg, batch, nn, tau=parity.TAU):
    n = n_kept = n_gp = 0
    untraced, traced, max_gp = [], 0, 0.0
    for e in range(batch.n_events):
        s0, s1 = int(gpu["ev_off"][e]), int(gpu["ev_off"][e + 1])
        st_ = gpu["state"][s0:s1]
        nh = gpu["n_hits"][s0:s1].astype(np.int32).sum(1)
        velo = batch.velo_of(e)
        m = oracle.matching_event(ocfg, velo, st_, ledger_tau=1e-4)
        f = oracle.final_selection(ocfg, velo, st_, nh, nn, m["velo_idx"], m["chi2"], ledger_tau=1e-4)
        # seeds and VELO segments of decisions within tau of flipping; a
        # flipped cut of one pair can change the clone decision of another
        # pair on the same segment, so segments count too
        near, near_v = set(), set()
        if len(m["ledger"]):
            near |= {int(h[0]) for h in m["ledger"][m["ledger"]["margin"] <= tau]["hits"]}
        if len(f["ledger"]):
            for h in f["ledger"][f["ledger"]["margin"] <= tau]["hits"]:
                near.add(int(h[0]))
                if h[2] >= 0:  # clone decision (seed, other seed, segment)
                    near.add(int(h[1]))
                    near_v.add(int(h[2]))
                else:          # ghost cut (seed, segment)
                    near_v.add(int(h[1]))
        gv = gpu["velo_idx"][s0:s1]
        n += s1 - s0
        n_kept += int((gv >= 0).sum())
        for k in np.nonzero(gv != f["velo_idx"])[0]:
            if k in near or int(m["velo_idx"][k]) in near_v:
                traced += 1
            else:
                untraced.append((e, int(k), int(gv[k]), int(f["velo_idx"][k])))
        same = m["velo_idx"] >= 0
        d = np.abs(gpu["ghost_prob"][s0:s1][same] - f["ghost_prob"][same])
        n_gp += int(same.sum())
        if d.size:
            max_gp = max(max_gp, float(d.max()))
    return n, n_kept, n_gp, untraced, traced, max_gp


@pytest.mark.parametrize("name,n,over", [("run3", 200, {}), ("match_stress", 40, {"tol_scale": 2.0}),
                                         ("uneven", 150, {})])
def test_final_selection_parity(name, n, over, zmx):
    b = workload(name, n_events=n)
    nn = ghost_nn_weights()
    ocfg, gcfg = parity.config_pair(zmx, final_sel=1, **over)
    gpu = run_final(b, gcfg, nn)
    n_seeds, n_kept, n_gp, untraced, traced, max_gp = compare_final(gpu, ocfg, b, nn)
    print(name, n_seeds, n_kept, n_gp, traced, max_gp)
    assert n_gp > 0 and 0 < n_kept < n_gp
    assert not untraced, untraced[:5]
    assert max_gp <= GP_TOL
    # the per-event Long-track counts are those of the kept pairs
    for e in range(b.n_events):
        s0, s1 = int(gpu["ev_off"][e]), int(gpu["ev_off"][e + 1])
        assert gpu["n_long"][e] == int((gpu["velo_idx"][s0:s1] >= 0).sum())


def test_final_selection_needs_weights(zmx):
    _, gcfg = parity.config_pair(zmx, final_sel=1)
    ctx = st.Context(gcfg)
    db = st.DeviceBatch.from_synth(workload("tiny"))
    with pytest.raises(st.StError) as ei:
        st.run_batch(ctx, db)
    assert ei.value.code == st.ST_ESTATE
    with pytest.raises(st.StError):
        ctx.st_set_ghost_nn(np.zeros(10, np.float32))
    bad = ghost_nn_weights().copy()
    bad[20] = np.nan
    with pytest.raises(st.StError):
        ctx.st_set_ghost_nn(bad)
    ctx.close()


def test_final_selection_through_pipeline(zmx):
    """pipeline_poll returns the selection and the ghost probabilities equal
    to a direct run of the same batch."""
    b = workload("run3", n_events=64)
    nn = ghost_nn_weights()
    _, gcfg = parity.config_pair(zmx, final_sel=1)
    direct = run_final(b, gcfg, nn)
    ctx = st.Context(gcfg)
    ctx.st_set_ghost_nn(nn)
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
    for k in ("velo_idx", "chi2", "ghost_prob", "n_long"):
        assert np.array_equal(got[k], direct[k]), k
