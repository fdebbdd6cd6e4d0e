"""Pins for the oracle's alphabet and substitution-matrix parser.

BLOSUM62 (Sec. III.A, Sec. III.B.5) is transcribed from Henikoff & Henikoff
(1992); its values are pinned by the invariants the published table has:
24x24, symmetric, integer range [-4, 11], and each amino acid scores highest
against itself.  The parser is checked on a column-permuted copy of the file
and on malformed input.
"""
import numpy as np
import pytest

import oracle as O


def test_blosum62_shape_symmetry_range():
    M = O.blosum62()
    assert M.shape == (24, 24)
    assert (M == M.T).all()
    assert M.min() == -4 and M.max() == 11


def test_blosum62_diagonal_dominates_each_column():
    M = O.blosum62().astype(int)
    for a in range(20):
        col = M[:20, a]
        assert col[a] == col.max()
        assert (col[np.arange(20) != a] < col[a]).all()


def test_blosum62_landmarks():
    M = O.blosum62()
    L = O.LETTERS
    assert M[L.index("W"), L.index("W")] == 11
    assert M[L.index("C"), L.index("C")] == 9
    assert M[L.index("*"), L.index("*")] == 1
    assert M[L.index("A"), L.index("*")] == -4
    diag20 = [int(M[i, i]) for i in range(20)]
    assert diag20 == [4, 5, 6, 6, 9, 5, 5, 6, 8, 4, 4, 5, 5, 6, 7, 4, 5, 11, 7, 4]


def test_parser_is_order_independent():
    M = O.blosum62()
    rng = np.random.default_rng(0)
    perm = rng.permutation(24)
    L = O.LETTERS
    lines = ["# permuted", "  " + "  ".join(L[p] for p in perm)]
    for r in rng.permutation(24):
        lines.append(L[r] + " " + " ".join("%3d" % M[r, p] for p in perm))
    assert (O.parse_matrix("\n".join(lines) + "\n") == M).all()


def test_parser_rejects_malformed():
    good = open(O.BLOSUM62_TXT).read()
    with pytest.raises(ValueError):
        O.parse_matrix("\n".join(good.splitlines()[:-3]))      # missing rows
    bad = good.replace("W -3 -3 -4 -4 -2", "W -3 -3 -4 -4 999")
    with pytest.raises(ValueError):
        O.parse_matrix(bad)


def test_encode():
    assert O.encode("ARNDCQEGHILKMFPSTWYVBZX*").tolist() == list(range(24))
    assert O.encode("arnd").tolist() == [0, 1, 2, 3]
    assert O.encode("J1Uo").tolist() == [22, 22, 22, 22]   # unknown letters read as X
