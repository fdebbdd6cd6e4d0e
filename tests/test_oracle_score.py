"""Closed-form pins for SCORE (Fig. 1's final scoring, reading A2/A3).

Gap model of Sec. III.B.1: leading and trailing gaps cost PGP each; inside the
alignment a run of n gaps in one row costs GOP + (n-1)*GEP.  Every expected
value below is written from those rules and BLOSUM62 entries by hand.
"""
import pytest

import oracle as O

GAP = "-"


def rows(a: str, b: str):
    enc = lambda s: [O.GAP if c == GAP else O.LETTERS.index(c) for c in s]
    return enc(a), enc(b)


M = O.blosum62()
L = O.LETTERS


def m(a, b):
    return int(M[L.index(a), L.index(b)])


def sc(a, b, pgp=0, gop=10, gep=5):
    ra, rb = rows(a, b)
    return O.score_rows(ra, rb, M, pgp, gop, gep)


def test_ungapped_is_sum_of_matrix_entries():
    assert sc("ACD", "ACD") == 4 + 9 + 6
    assert sc("WYV", "FHI") == m("W", "F") + m("Y", "H") + m("V", "I")


def test_single_internal_gap_in_query_row():
    # one gap: GOP only
    assert sc("A-CD", "AWCD") == m("A", "A") + m("C", "C") + m("D", "D") - 10
    # run of two: GOP + GEP
    assert sc("A--CD", "AWWCD") == 19 - (10 + 5)
    # run of four: GOP + 3 GEP, other penalties
    assert sc("A----CD", "AWWWWCD", gop=7, gep=2) == 19 - (7 + 3 * 2)


def test_single_internal_gap_in_target_row():
    assert sc("AWWWCD", "A---CD", gop=11, gep=1) == 19 - (11 + 2 * 1)


def test_adjacent_runs_in_different_rows_are_two_runs():
    assert sc("AW-D", "A-CD") == m("A", "A") + m("D", "D") - 10 - 10


def test_two_separate_runs_in_one_row():
    assert sc("A-C--D", "AWCYYD") == m("A", "A") + m("C", "C") + m("D", "D") - 10 - (10 + 5)


def test_leading_and_trailing_gaps_are_periphery():
    assert sc("--ACD", "WWACD", pgp=3) == 19 - 2 * 3
    assert sc("ACD--", "ACDWW", pgp=3) == 19 - 2 * 3
    # periphery in both rows: first/last letter pair bound the core
    assert sc("WACD-", "-ACDW", pgp=3) == 19 - 2 * 3
    # PGP = 0: free ends (Sec. III.B.1 a, local-like behaviour)
    assert sc("----ACD", "WWWWACD", pgp=0) == 19


def test_no_letter_pair_is_all_periphery():
    assert sc("AC--", "--DE", pgp=4) == -4 * 4
    assert sc("A", "-", pgp=2) == -2


def test_gap_gap_column_is_rejected():
    with pytest.raises(ValueError):
        sc("A-C", "A-C")


def test_matrix_orientation_query_first():
    # an asymmetric matrix: M[q][t] is used, never M[t][q]
    import numpy as np
    A = np.zeros((24, 24), np.int8)
    A[0, 1] = 7
    A[1, 0] = -3
    assert O.score_rows([0], [1], A, 0, 10, 5) == 7
    assert O.score_rows([1], [0], A, 0, 10, 5) == -3
