"""Pins for the oracle's random() (reading A12 of Fig. 1's random()).

The oracle's Philox4x64-10 is checked against (1) the published known-answer
vectors and (2) numpy's independent Philox implementation (numpy.random.Philox
is Philox4x64-10; it increments the counter before producing each block, so
its first block for counter c is the block of c+1).  The 16-bit draw layout
is checked by slicing numpy's words directly.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_10_kat.txt")


def kat_rows():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", kat_rows())
def test_philox_known_answers(ctr, key, want):
    assert O.philox4x64_10(ctr, key) == want


def numpy_block(ctr, key):
    c = list(ctr)
    # numpy bumps the 256-bit counter before each block: start one below.
    v = (c[0] | (c[1] << 64) | (c[2] << 128) | (c[3] << 192)) - 1
    v %= 2**256
    start = [(v >> (64 * i)) & (2**64 - 1) for i in range(4)]
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(start, dtype=np.uint64))
    return [int(x) for x in g.random_raw(4)]


def test_philox_matches_numpy_random_counters():
    rng = np.random.default_rng(1234)
    for _ in range(200):
        ctr = [int(x) for x in rng.integers(0, 2**64, 4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2**64, 2, dtype=np.uint64)]
        assert O.philox4x64_10(ctr, key) == numpy_block(ctr, key)


def test_philox_matches_numpy_small_counters():
    for d in [0, 1, 7, 569_999]:
        for r in [0, 1, 19]:
            for b in [0, 1, 2]:
                for seed in [0, 1, 2**63 + 5]:
                    assert O.philox4x64_10([d, r, b, 0], [seed, 0]) == numpy_block([d, r, b, 0], [seed, 0])


def test_draw16_layout_from_numpy_words():
    """Draw i = 16-bit field (i % 4), most significant first, of word
    (i % 16) // 4 of block i // 16 for counter (d, r, i // 16, 0), key (seed, 0)."""
    for seed, d, r in [(0, 0, 0), (99, 1234, 0), (2**40 + 3, 7, 3)]:
        for i in range(0, 40):
            blk = numpy_block([d, r, i // 16, 0], [seed, 0])
            w = blk[(i % 16) // 4]
            want = (w >> (48 - 16 * (i % 4))) & 0xFFFF
            assert O.draw16(seed, d, r, i) == want


def test_draw16_is_roughly_uniform():
    vals = np.array([O.draw16(5, d, 0, i) for d in range(40) for i in range(50)])
    assert 0 <= vals.min() and vals.max() < 65536
    assert abs(vals.mean() / 65536 - 0.5) < 0.03
