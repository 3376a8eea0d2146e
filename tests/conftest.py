import os
import re
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def read_golden_constants(path=os.path.join(GOLDEN, "paper_constants.txt")):
    """Parse `field[idx] = value  # citation` lines into {(field, idx): value}."""
    out = {}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        lhs, rhs = [s.strip() for s in line.split("=", 1)]
        m = re.fullmatch(r"(\w+)(?:\[(\d+)\])?", lhs)
        out[(m.group(1), None if m.group(2) is None else int(m.group(2)))] = float(rhs)
    return out


@pytest.fixture(scope="session")
def ocfg():
    import oracle
    return oracle.default_config()


@pytest.fixture(scope="session")
def zmx_calibrated(ocfg):
    from synth import calibrate_zmatch
    return calibrate_zmatch(ocfg.z_state)


_CACHE = {}


def workload(name, **kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in _CACHE:
        from synth import make_workload
        _CACHE[key] = make_workload(name, **kw)
    return _CACHE[key]


def truth_track_of(batch, e, hits):
    """Majority truth track (global id) of a hit list, with its purity."""
    ht = batch.hit_track[batch.ev_off[e]:batch.ev_off[e + 1]]
    hs = [h for h in hits if h >= 0]
    ids = ht[hs]
    ids = ids[ids >= 0]
    if len(ids) == 0:
        return -1, 0.0
    v, c = np.unique(ids, return_counts=True)
    return int(v[c.argmax()]), c.max() / len(hs)
