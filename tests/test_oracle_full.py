"""Pins for the oracle's full-slide mode (Fig. 1 as printed: small slides
from overlapping large's first letter with its last to overlapping large's
last letter with its first; readings F1-F4)."""
import numpy as np
import pytest

import oracle as O
from paper_1508_06561_gb300 import synth

FULL = O.paper_params(mode=O.MODE_FULL)


def numpy_full_slide(A, B, M):
    ns, nl = len(B), len(A)
    best, bk = None, None
    for k in range(-(ns - 1), nl):
        j = np.arange(max(0, -k), min(ns, nl - k))
        v = int(M.astype(np.int64)[A[k + j], B[j]].sum())
        if best is None or v > best:
            best, bk = v, k
    return bk, best


@pytest.mark.parametrize("case", range(40))
def test_full_slide_shift_matches_numpy(case):
    rng = np.random.default_rng(case)
    A = rng.integers(0, 24, int(rng.integers(1, 80))).astype(np.uint8)
    B = rng.integers(0, 24, int(rng.integers(1, 80))).astype(np.uint8)   # may be longer than A
    M = O.blosum62() if case % 2 else synth.random_symmetric_matrix(rng, -9, 9)
    assert O.best_shift_full(A, B, M) == numpy_full_slide(A, B, M)


def degap(row):
    row = np.asarray(row)
    return row[row != O.GAP]


@pytest.mark.parametrize("case", range(80))
def test_full_mode_alignment_valid_and_bounded(case):
    rng = np.random.default_rng(3000 + case)
    q = rng.integers(0, 20, int(rng.integers(0, 40))).astype(np.uint8)
    t = rng.integers(0, 20, int(rng.integers(0, 40))).astype(np.uint8)
    M = O.blosum62() if case % 2 else synth.random_symmetric_matrix(rng, -5, 9)
    p = O.paper_params(mode=O.MODE_FULL, pgp=int(rng.integers(0, 3)), rounds=int(rng.integers(1, 21)),
                       lfactor_q16=int(rng.integers(1, 65537)), sfactor_q16=int(rng.integers(1, 65537)),
                       minfactor_q16=int(rng.integers(0, 65537)))
    s, rq, rt, r, cells = O.align_pair(q, t, M, p, case, case)
    assert len(rq) == len(rt) and not np.any((rq == O.GAP) & (rt == O.GAP))
    assert np.array_equal(degap(rq), q) and np.array_equal(degap(rt), t)
    assert O.score_rows(rq, rt, M, p.pgp, p.gop, p.gep) == s
    assert s <= O.periphery_opt(q, t, M, p.pgp, p.gop, p.gep)
    if p.pgp == 0 and len(q) and len(t):
        assert s <= O.smith_waterman(q, t, M, p.gop, p.gep)


def test_full_mode_self_alignment_is_identity():
    M = O.blosum62()
    rng = np.random.default_rng(9)
    for n in [1, 3, 50, 400]:
        q = synth.residues(rng, n)
        s, rq, rt, _, _ = O.align_pair(q, q, M, O.paper_params(mode=O.MODE_FULL, rounds=3), 1, 2)
        assert s == int(M[q, q].astype(np.int64).sum()) and np.array_equal(rq, q)


def test_one_letter_query_full_equals_database_mode():
    """With |small| = 1 no overhang is possible (F1 gives shifts 0..ls-1), so
    both modes take identical steps."""
    M = O.blosum62()
    rng = np.random.default_rng(4)
    for n in [1, 2, 9, 100]:
        t = synth.residues(rng, n)
        q = synth.residues(rng, 1)
        a = O.align_pair(q, t, M, O.paper_params(), 5, 6)
        b = O.align_pair(q, t, M, FULL, 5, 6)
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_full_mode_can_overhang():
    """Some pairs must use a shift outside 0..ls-ss (gaps in large's row)."""
    M = O.blosum62()
    rng = np.random.default_rng(12)
    seen = False
    for trial in range(200):
        q = synth.residues(rng, int(rng.integers(20, 60)))
        t = synth.residues(rng, int(rng.integers(20, 60)))
        s, rq, rt, _, _ = O.align_pair(q, t, M, FULL, trial, trial)
        big = rt if len(t) >= len(q) else rq
        letters = np.nonzero(big != O.GAP)[0]
        if len(letters) and np.any(big[: letters[-1]] == O.GAP):
            seen = True
            break
    assert seen
