"""HLT2-style iterations in sequence with hit cleanup (iter_mode = 1) on the
GPU against the oracle at the same configuration, element by element."""

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import parity  # noqa: E402
from conftest import workload  # noqa: E402
from synth import calibrate_zmatch  # noqa: E402
from test_gpu_parity import assert_seeding_parity, run_gpu  # noqa: E402

SEQ2 = dict(iter_mode=1)
SEQ3 = dict(iter_mode=1, n_iter=3, p_min_iter=[5000.0, 3000.0, 1500.0])


@pytest.fixture(scope="module")
def zmx():
    return calibrate_zmatch(7826.0)


@pytest.mark.parametrize("name,n,over", [
    ("tiny", None, SEQ2), ("tiny", None, SEQ3), ("run3", 150, SEQ2), ("run3", 150, SEQ3),
    ("uneven", 150, SEQ3), ("match_stress", 30, SEQ3), ("run3", 80, dict(SEQ3, uv_mode=1)),
    ("run3", 80, dict(n_iter=3, p_min_iter=[5000.0, 3000.0, 1500.0])),
])
def test_sequential_iterations_parity(name, n, over, zmx):
    b = workload(name, n_events=n) if n else workload(name)
    ocfg, gcfg = parity.config_pair(zmx, **over)
    gpu, cnt = run_gpu(b, gcfg)
    assert (gpu["status"] == 0).all()
    rep = parity.compare_seeding(gpu, ocfg, b)
    print(name, over, rep.summary())
    assert rep.n_common > 0
    assert_seeding_parity(rep)
