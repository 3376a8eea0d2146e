"""The container layout bounds the seeding kernel's staging copies.

The seeding kernel stages each (event, half) slice of the hit containers in
shared memory with one bulk copy of whole 16-byte words: it rounds the
slice's start down and its end up to a multiple of four floats.  That is safe
only because of the container layout: event e starts at
round4((ev_off[e] - ev_off[0]) + 3 e) floats, so every event starts 16-byte
aligned and is followed by at least three spare entries up to the next
event's start, and the allocation holds n_hits + 3 n_events + 8 floats.
These tests restate that layout and check, for many batch shapes and every
split of an event into its two halves, that the rounded copy never leaves
the event's own region nor the allocation.  No GPU is needed.
"""

import numpy as np


def cont_base(ev_off, e):
    b = int(ev_off[e] - ev_off[0]) + 3 * e
    return (b + 3) & ~3


def copy_range(cbh, nh):
    """Start (rounded down) and end (rounded up) of the staged words, in floats."""
    w0 = cbh & ~3
    lead = cbh - w0
    return w0, w0 + ((lead + nh + 3) & ~3)


def check_batch(sizes, rng):
    ev_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n_events = len(sizes)
    cap = int(ev_off[-1]) + 3 * n_events + 8  # the library's container allocation
    for e in range(n_events):
        n = int(sizes[e])
        start = cont_base(ev_off, e)
        limit = cont_base(ev_off, e + 1) if e + 1 < n_events else cap
        assert start % 4 == 0
        assert start + n <= limit
        for k in {0, n, int(rng.integers(0, n + 1)), n // 2}:
            for cbh, nh in ((start, k), (start + k, n - k)):
                if nh == 0:
                    continue
                w0, w1 = copy_range(cbh, nh)
                assert w0 % 4 == 0 and (w1 - w0) % 4 == 0
                assert start <= w0 <= cbh and cbh + nh <= w1 <= limit, (e, k, cbh, nh, w0, w1, limit)


def test_staging_copy_stays_in_its_event():
    rng = np.random.default_rng(7)
    for trial in range(200):
        n_events = int(rng.integers(1, 60))
        if trial % 4 == 0:
            sizes = rng.integers(0, 8, n_events)  # tiny and empty events
        else:
            sizes = rng.integers(0, 7000, n_events)
        check_batch(sizes, rng)


def test_staging_copy_single_and_aligned_events():
    rng = np.random.default_rng(11)
    for sizes in ([1], [0], [4], [3, 5], [4, 4, 4], [1] * 9, [6144] * 3, [0, 0, 7, 0]):
        check_batch(np.asarray(sizes, dtype=np.int64), rng)
