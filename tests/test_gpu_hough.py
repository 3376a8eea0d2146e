"""The Hough-cluster UV variant (Section 3.4, second approach) on the GPU
against the oracle at the same configuration: element by element on small
batches, the oracle's work counters, non-default Hough parameters, and the
largest events of the uneven-occupancy mix (global-memory staging, long
hypothesis lists)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import parity  # noqa: E402
from conftest import workload  # noqa: E402
from synth import calibrate_zmatch  # noqa: E402
from test_gpu_parity import assert_seeding_parity, run_gpu  # noqa: E402


@pytest.fixture(scope="module")
def zmx():
    return calibrate_zmatch(7826.0)


@pytest.mark.parametrize("name,n", [("tiny", None), ("run3", 200), ("match_stress", 40), ("uneven", 200)])
def test_hough_seeding_parity(name, n, zmx):
    b = workload(name, n_events=n) if n else workload(name)
    ocfg, gcfg = parity.config_pair(zmx, uv_mode=1)
    gpu, cnt = run_gpu(b, gcfg)
    assert (gpu["status"] == 0).all()
    rep = parity.compare_seeding(gpu, ocfg, b)
    print(name, rep.summary())
    assert rep.n_common > 0
    assert_seeding_parity(rep)


def test_hough_counters_match_oracle(zmx):
    b = workload("run3", n_events=100)
    ocfg, gcfg = parity.config_pair(zmx, uv_mode=1)
    gpu, cnt = run_gpu(b, gcfg)
    refs = oracle.seeding_batch(ocfg, b)
    tot = {k: sum(r["counters"][k] for r in refs) for k in refs[0]["counters"]}
    for k in ("pairs", "triplets", "ext_ok", "cands", "kept", "uv_init", "uv_cands", "seeds"):
        assert abs(cnt[k] - tot[k]) <= max(2, 1e-4 * tot[k]), (k, cnt[k], tot[k])


@pytest.mark.parametrize("params", [dict(hough_bins=32, hough_fine=2, hough_clusters=4),
                                    dict(hough_bins=64, hough_fine=8, hough_clusters=1),
                                    dict(hough_bins=48, hough_fine=3, hough_clusters=8, n_uv_min=5)])
def test_hough_parameters(params, zmx):
    b = workload("run3", n_events=60)
    ocfg, gcfg = parity.config_pair(zmx, uv_mode=1, **params)
    gpu, cnt = run_gpu(b, gcfg)
    rep = parity.compare_seeding(gpu, ocfg, b)
    print(params, rep.summary())
    assert rep.n_common > 0
    assert_seeding_parity(rep)


def test_hough_largest_uneven_events(zmx):
    """The largest events of a 3000-event uneven batch, run in one launch."""
    b = workload("uneven", n_events=3000)
    ocfg, gcfg = parity.config_pair(zmx, uv_mode=1)
    gpu, cnt = run_gpu(b, gcfg)
    assert (gpu["status"] == 0).all()
    sizes = np.diff(b.ev_off)
    ev = np.sort(np.argsort(sizes)[-8:])
    rep = parity.compare_seeding(gpu, ocfg, b, ev)
    print(rep.summary(), "max hits", sizes.max())
    assert_seeding_parity(rep)
