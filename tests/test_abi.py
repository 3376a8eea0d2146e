"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point declared in include/st.h, and its defaults equal the paper's
printed constants and the oracle's defaults (two independent transcriptions)."""

import os
import re

import numpy as np
import pytest

from conftest import ROOT, read_golden_constants


def declared_functions():
    src = open(os.path.join(ROOT, "include", "st.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "for", "sizeof", "defined")))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("seeding_run", "matching_run", "pipeline_submit", "pipeline_poll", "st_create", "st_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2606_14480_gb300 import st
    L = st.library()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in st.SIGNATURES, name


def test_library_defaults_equal_paper_constants():
    from paper_2606_14480_gb300 import st
    cfg = st.st_config_default()
    for (f, i), v in read_golden_constants().items():
        cur = getattr(cfg, f)
        got = cur[i] if i is not None else cur
        assert got == pytest.approx(v, rel=1e-12, abs=1e-15), (f, i)


def test_library_and_oracle_defaults_agree():
    import oracle
    from paper_2606_14480_gb300 import st
    g = st.st_config_default()
    o = oracle.default_config()
    for name, _ in oracle.OrConfig._fields_:
        if name.startswith("pad"):
            continue
        a, b = getattr(g, name), getattr(o, name)
        if hasattr(a, "__len__"):
            assert np.allclose(np.array([list(r) if hasattr(r, "__len__") else r for r in a], dtype=float),
                               np.array([list(r) if hasattr(r, "__len__") else r for r in b], dtype=float),
                               rtol=1e-15, atol=0), name
        else:
            assert a == b, name


def test_invalid_config_rejected_without_gpu():
    """st_create validates the configuration before touching the device."""
    import ctypes as C
    from paper_2606_14480_gb300 import st
    L = st.library()
    for bad in (dict(n_uv_min=1), dict(n_iter=4), dict(threads_seed=100), dict(sigma_x=0.0),
                dict(iter_layers=[[0, 1, 11], [3, 7, 8], [0, 7, 11]]), dict(iter_mode=2),
                dict(p_min_iter=[0.0, -1.0, 0.0]), dict(uv_mode=2), dict(final_sel=1, velo_unique=1),
                dict(hough_bins=65), dict(ut_min_hits=5)):
        cfg = st.st_config_default(**bad)
        h = C.c_void_p()
        assert L.st_create(C.byref(cfg), 0, C.byref(h)) == st.ST_EINVAL, bad
        assert not h.value
    assert L.seeding_run(None, None, None, None) == st.ST_EINVAL
    assert L.st_last_error(None) == b"null context"


def test_struct_sizes_match_header():
    """ctypes mirrors have the C layout (compiled probe of sizeof/offsetof)."""
    import ctypes as C
    import subprocess
    import tempfile
    from paper_2606_14480_gb300 import st
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "st.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(st_config), sizeof(st_hits), sizeof(st_seeds),
         sizeof(st_velo), sizeof(st_long), sizeof(st_counters), sizeof(st_pipeline_config),
         sizeof(st_request_info), offsetof(st_config, threads_seed), offsetof(st_config, velo_unique));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    want = [C.sizeof(st.StConfig), C.sizeof(st.StHits), C.sizeof(st.StSeeds), C.sizeof(st.StVelo),
            C.sizeof(st.StLong), C.sizeof(st.StCounters), C.sizeof(st.StPipelineConfig),
            C.sizeof(st.StRequestInfo), st.StConfig.threads_seed.offset, st.StConfig.velo_unique.offset]
    assert got == want
