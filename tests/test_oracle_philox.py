"""Pins of the oracle's Philox4x32-10 and of its counter layout."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answer_vectors(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, expect in rows:
        assert list(orc.philox(ctr, key)) == expect


def test_init_counter_layout_matches_kat(orc):
    # seed 0, individual 0, genes 0..3 use counter (0, 0, 0, INIT=0) under key (0, 0):
    # the first known-answer vector; label = high word of u * N.
    _, _, words = _kat()[0]
    for N in (10, 16, 500, 65535):
        pop = orc.ga_init(1, N, seed=0)
        got = pop[0, :4].tolist()
        assert got == [(w * N) >> 32 for w in words]


def test_threshold_exact(orc):
    assert orc.threshold(0.0) == 0
    assert orc.threshold(-1.0) == 0
    assert orc.threshold(1.0) == 1 << 32
    assert orc.threshold(0.5) == 1 << 31
    assert orc.threshold(0.9) == int(np.floor(0.9 * 2**32))
    assert orc.threshold(0.01) == 42949672  # floor(0.01 * 2^32) = 42949672.96 -> 42949672
