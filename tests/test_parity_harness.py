"""The GPU/oracle comparison harness (tests/parity.py) on CPU.

A stand-in "GPU" result is made from the oracle's own output for a few events;
seeds are then dropped or altered on purpose, and the harness must classify
each difference: untraced when no ledger decision within tau is involved,
traced (directly) when the seed shares a hit with such a decision, and a
parameter error when a fitted value moves beyond its tolerance.  The matching
trace must require an entry that names the seed and one of the two chosen
VELO segments.
"""

import numpy as np
import pytest

import oracle
import parity
from conftest import workload


def fake_gpu(refs):
    """The oracle's seeds of several events in the library's output layout."""
    n = [len(r["seeds"]) for r in refs]
    ev_off = np.concatenate([[0], np.cumsum(n)]).astype(np.int32)
    seeds = np.concatenate([r["seeds"] for r in refs])
    params = np.stack([seeds[k] for k in ("a", "b", "c", "chi2x", "y0", "ty", "chi2y")] +
                      [np.zeros(len(seeds))], 1).astype(np.float32)
    state = np.stack([seeds[k] for k in ("x_s", "y_s", "tx_s", "ty_s")], 1).astype(np.float32)
    return {"ev_off": ev_off, "hits": seeds["hits"].copy(), "params": params, "state": state,
            "n_hits": np.stack([seeds["nx"], seeds["nuv"]], 1).astype(np.int8)}


def drop_seed(g, i):
    out = dict(g)
    for k in ("hits", "params", "state", "n_hits"):
        out[k] = np.delete(g[k], i, axis=0)
    ev = np.searchsorted(g["ev_off"], i, side="right") - 1
    out["ev_off"] = g["ev_off"].copy()
    out["ev_off"][ev + 1:] -= 1
    return out


@pytest.fixture(scope="module")
def sample(ocfg):
    b = workload("run3", n_events=6)
    refs = oracle.seeding_batch(ocfg, b, list(range(b.n_events)), cands=True, ledger_tau=1e-4)
    return b, refs


def test_identical_results_agree(sample):
    b, refs = sample
    g = fake_gpu(refs)
    rep = parity.Report()
    for e, r in enumerate(refs):
        rep.merge(parity.compare_seeding_event(e, g, r))
    assert rep.agreement == 1.0 and rep.traced == 0 and not rep.untraced and not rep.bad_params
    parity.assert_seeding(rep)


def test_dropped_seed_classified(sample):
    """A seed whose hits touch no ledger decision within tau is untraced when
    missing; with tau raised until a decision on one of its hits is within
    it, the same difference is traced directly."""
    b, refs = sample
    g = fake_gpu(refs)
    e = 0
    r = refs[e]
    led = r["ledger"]
    for i, s in enumerate(r["seeds"]):
        hs = {int(h) for h in s["hits"] if h >= 0}
        on = led[[bool(hs & {int(h) for h in row["hits"] if h >= 0}) for row in led]]
        if len(on) and on["margin"].min() > parity.TAU:
            break
    else:
        pytest.skip("every seed touches a near decision")
    gd = drop_seed(g, int(g["ev_off"][e]) + i)
    rep = parity.compare_seeding_event(e, gd, r)
    assert len(rep.untraced) == 1 and rep.traced == 0
    assert rep.untraced[0][2] == "oracle"
    rep = parity.compare_seeding_event(e, gd, r, tau=float(on["margin"].min()))
    assert not rep.untraced and rep.traced == 1 and rep.traced_kinds


def test_parameter_beyond_tolerance(sample):
    b, refs = sample
    g = fake_gpu(refs)
    g["params"] = g["params"].copy()
    g["params"][3, 0] += 2e-3  # a: 2e-3 mm against a tolerance of 1e-3 mm
    e = int(np.searchsorted(g["ev_off"], 3, side="right") - 1)
    rep = parity.compare_seeding_event(e, g, refs[e])
    assert [p[2] for p in rep.bad_params] == ["a"]


def test_matching_trace_needs_the_pair(ocfg):
    """A changed VELO choice is traced only by an entry of that seed naming
    one of the two VELO segments."""
    b = workload("run3", n_events=2)
    e = 0
    velo = b.velo_of(e)
    # a stand-in GPU result: the oracle's matching on the oracle's seed states
    r = oracle.seeding_event(ocfg, *b.hits_of(e))
    st = np.stack([r["seeds"][k] for k in ("x_s", "y_s", "tx_s", "ty_s")], 1).astype(np.float32)
    m = oracle.matching_event(ocfg, velo, st, ledger_tau=1e-4)
    k = int(np.nonzero(m["velo_idx"] >= 0)[0][0])
    other = int((m["velo_idx"][k] + 1) % len(velo))
    g = {"ev_off": np.array([0, len(st), len(st)], np.int32), "state": st,
         "velo_idx": m["velo_idx"].astype(np.int32).copy(), "chi2": m["chi2"].astype(np.float32)}
    n, untraced, traced, _ = parity.compare_matching(g, ocfg, b, [e])
    assert not untraced and traced == 0
    g["velo_idx"][k] = other
    led = m["ledger"]
    names_pair = [bool(int(row["hits"][0]) == k and {int(row["hits"][1]), int(row["hits"][2])} &
                       {other, int(m["velo_idx"][k])}) for row in led]
    n, untraced, traced, _ = parity.compare_matching(g, ocfg, b, [e])
    if any(names_pair[i] and led["margin"][i] <= parity.TAU for i in range(len(led))):
        assert traced == 1
    else:
        assert len(untraced) == 1 and untraced[0][1] == k
