"""Pins for the oracle's exact dynamic programmes.

* The periphery-gap DP (the optimum under the paper's gap model, Sec. III.B.1)
  equals the best SCORE over every alignment of two short sequences,
  enumerated exhaustively.
* With PGP = 0 the same DP reduces to textbook Smith-Waterman with affine
  gaps (the prior work of Sec. II), so the two must agree exactly.
"""
import numpy as np
import pytest

import oracle as O
from paper_1508_06561_gb300 import synth


def all_alignments(x, y):
    """Every alignment of x and y (no gap-gap column), as (row_x, row_y)."""
    out = []

    def rec(i, j, rx, ry):
        if i == len(x) and j == len(y):
            out.append((list(rx), list(ry)))
            return
        if i < len(x) and j < len(y):
            rec(i + 1, j + 1, rx + [x[i]], ry + [y[j]])
        if i < len(x):
            rec(i + 1, j, rx + [x[i]], ry + [O.GAP])
        if j < len(y):
            rec(i, j + 1, rx + [O.GAP], ry + [y[j]])

    rec(0, 0, [], [])
    return out


def test_enumeration_counts_are_delannoy_numbers():
    # D(m, n): 1, 3, 13, 63, 321 on the diagonal
    assert [len(all_alignments([0] * n, [1] * n)) for n in range(5)] == [1, 3, 13, 63, 321]


@pytest.mark.parametrize("case", range(60))
def test_periphery_dp_equals_exhaustive_best(case):
    rng = np.random.default_rng(100 + case)
    nx, ny = int(rng.integers(0, 6)), int(rng.integers(0, 6))
    if case % 3 == 0:
        M = O.blosum62()
        x = rng.integers(0, 20, nx).astype(np.uint8)
        y = rng.integers(0, 20, ny).astype(np.uint8)
    else:
        M = synth.random_symmetric_matrix(rng, -6, 9)
        x = rng.integers(0, 24, nx).astype(np.uint8)
        y = rng.integers(0, 24, ny).astype(np.uint8)
    pgp, gop, gep = int(rng.integers(0, 6)), int(rng.integers(0, 12)), int(rng.integers(0, 6))
    best = max(O.score_rows(a, b, M, pgp, gop, gep) for a, b in all_alignments(list(x), list(y)))
    assert O.periphery_opt(x, y, M, pgp, gop, gep) == best


@pytest.mark.parametrize("case", range(40))
def test_periphery_dp_with_free_ends_is_smith_waterman(case):
    rng = np.random.default_rng(500 + case)
    nx, ny = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    M = O.blosum62() if case % 2 else synth.random_symmetric_matrix(rng, -5, 8)
    x = rng.integers(0, 20, nx).astype(np.uint8)
    y = rng.integers(0, 20, ny).astype(np.uint8)
    gop, gep = int(rng.integers(1, 14)), int(rng.integers(0, 6))
    assert O.periphery_opt(x, y, M, 0, gop, gep) == O.smith_waterman(x, y, M, gop, gep)


def test_smith_waterman_textbook_values():
    M = O.blosum62()
    enc = O.encode
    # identical sequences: the ungapped diagonal sum
    s = enc("HEAGAWGHEE")
    assert O.smith_waterman(s, s, M, 10, 1) == sum(int(M[c, c]) for c in s)
    # one inserted letter in a long identical run: the gap costs GOP once
    a = enc("WWWWWCWWWWW")
    b = enc("WWWWWWWWWW")
    assert O.smith_waterman(a, b, M, 8, 1) == 10 * 11 - 8
