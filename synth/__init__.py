"""Seeded synthetic event generator shared by the tests, the benchmark and
the oracle harness.

This package simulates a toy LHCb-like tracking system (VELO straight-line
segments, a dipole kink, a 12-layer SciFi tracker with x-u-v-x stations) and
returns hits, VELO states and the truth behind them.  It contains no part of
the reconstruction method: no search windows, no fits, no cuts.
"""

from .events import (  # noqa: F401
    Detector,
    EventBatch,
    WORKLOADS,
    calibrate_zmatch,
    ghost_nn_weights,
    make_events,
    make_workload,
)
