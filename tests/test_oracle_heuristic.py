"""Pins for the oracle's heuristic (Fig. 1 in database mode, Sec. III.B.3).

What fixes the heuristic without a reference implementation:
* the shift scan equals an independent numpy sliding-window argmax;
* every output is a valid alignment of the two full sequences, with no gap
  in the large sequence's row before its last letter (Sec. III.B.3 b);
* its score never exceeds the exact optimum under the same gap model, nor
  (PGP = 0) the Smith-Waterman optimum;
* closed forms: a sequence against itself aligns ungapped with the diagonal
  sum; a one-letter small sequence scores the best letter in large's first
  max(1, floor(|large|*lf)) positions;
* best-of-rounds behaves as Fig. 1's AlignSequences (strict '>').
"""
import numpy as np
import pytest
from numpy.lib.stride_tricks import sliding_window_view

import oracle as O
from paper_1508_06561_gb300 import synth

PAPER = O.paper_params()


def rand_params(rng):
    return O.paper_params(pgp=int(rng.integers(0, 4)), gop=int(rng.integers(0, 15)),
                          gep=int(rng.integers(0, 6)), rounds=int(rng.integers(1, 4)),
                          lfactor_q16=int(rng.integers(0, 65537)),
                          sfactor_q16=int(rng.integers(0, 65537)),
                          minfactor_q16=int(rng.integers(0, 65537)))


def degap(row):
    row = np.asarray(row)
    return row[row != O.GAP]


@pytest.mark.parametrize("case", range(50))
def test_best_shift_matches_numpy_sliding_window(case):
    rng = np.random.default_rng(case)
    nl = int(rng.integers(1, 300))
    ns = int(rng.integers(1, nl + 1))
    M = O.blosum62() if case % 2 else synth.random_symmetric_matrix(rng, -9, 9)
    A = rng.integers(0, 24, nl).astype(np.uint8)
    B = rng.integers(0, 24, ns).astype(np.uint8)
    win = sliding_window_view(A, ns)                         # (nl-ns+1, ns)
    V = M.astype(np.int64)[win, B[None, :]].sum(axis=1)
    k, v = O.best_shift(A, B, M)
    assert k == int(np.argmax(V)) and v == int(V.max())      # argmax: first maximum


def check_alignment(q, t, rq, rt):
    assert len(rq) == len(rt)
    assert not np.any((rq == O.GAP) & (rt == O.GAP))
    assert np.array_equal(degap(rq), q) and np.array_equal(degap(rt), t)
    # database mode: the larger sequence's row has no gap before its last letter
    big = rt if len(t) >= len(q) else rq
    letters = np.nonzero(big != O.GAP)[0]
    if len(letters):
        assert not np.any(big[: letters[-1]] == O.GAP)


@pytest.mark.parametrize("case", range(120))
def test_alignment_valid_and_bounded_by_optimum(case):
    rng = np.random.default_rng(1000 + case)
    nq, nt = int(rng.integers(0, 45)), int(rng.integers(0, 45))
    if case % 2:
        M, p = O.blosum62(), PAPER
    else:
        M, p = synth.random_symmetric_matrix(rng, -5, 9), rand_params(rng)
    q = rng.integers(0, 20, nq).astype(np.uint8)
    t = rng.integers(0, 20, nt).astype(np.uint8)
    s, rq, rt, r, cells = O.align_pair(q, t, M, p, seed=case, dbidx=case * 7)
    check_alignment(q, t, rq, rt)
    assert O.score_rows(rq, rt, M, p.pgp, p.gop, p.gep) == s
    assert s <= O.periphery_opt(q, t, M, p.pgp, p.gop, p.gep)
    if p.pgp == 0 and nq and nt:
        assert s <= O.smith_waterman(q, t, M, p.gop, p.gep)
    assert 0 <= r < p.rounds
    # work bounds: every step scores at least its ss cells, and the steps of a
    # round tile part of the |large| x |small| matrix (ls <= Lrem, sum ss <= |small|)
    assert min(nq, nt) * p.rounds <= cells <= p.rounds * nq * nt


def test_self_alignment_is_ungapped_diagonal_sum():
    M = O.blosum62()
    rng = np.random.default_rng(7)
    for n in [1, 2, 5, 64, 300, 1000]:
        q = synth.residues(rng, n)
        for seed in range(3):
            s, rq, rt, _, _ = O.align_pair(q, q, M, PAPER, seed, seed * 11)
            assert s == int(M[q, q].astype(np.int64).sum())
            assert np.array_equal(rq, q) and np.array_equal(rt, q)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 40, 333])
def test_one_letter_small_sequence_closed_form(n):
    """|small| = 1: one step with ss = 1 and ls = max(1, floor(n * lf)); the
    letter lands at the best of large's first ls positions (first on ties)
    and every other letter of large is periphery."""
    M = O.blosum62()
    rng = np.random.default_rng(n)
    for pgp in [0, 2]:
        p = O.paper_params(pgp=pgp)                          # lf = 0.5 exactly
        for trial in range(5):
            t = synth.residues(rng, n)
            q = synth.residues(rng, 1)
            ls = max(1, n // 2)
            col = M[t[:ls], q[0]].astype(int)
            k = int(np.argmax(col))
            s, rq, rt, _, cells = O.align_pair(q, t, M, p, trial, trial)
            assert s == col[k] - pgp * (n - 1)
            assert cells == ls
            assert rq.tolist() == [O.GAP] * k + [int(q[0])] + [O.GAP] * (n - 1 - k)


def test_hand_worked_examples():
    """Q = W against short targets, paper parameters (PGP=0, LFactor=0.5).
    T = AWA: ls = floor(3/2) = 1, only shift 0 -> M[W][A] = -3.
    T = AWAA: ls = 2, shift 1 puts W on W -> 11.
    With PGP = 2 the three unused target letters cost 6 -> 5."""
    M = O.blosum62()
    q = O.encode("W")
    assert O.align_pair(q, O.encode("AWA"), M, PAPER, 0, 0)[0] == -3
    assert O.align_pair(q, O.encode("AWAA"), M, PAPER, 0, 0)[0] == 11
    assert O.align_pair(q, O.encode("AWAA"), M, O.paper_params(pgp=2), 0, 0)[0] == 5
    assert O.align_pair(q, O.encode("AAAW"), M, PAPER, 0, 0)[0] == -3   # W beyond ls


def test_empty_sequences():
    M = O.blosum62()
    q = O.encode("ACDEF")
    s, rq, rt, _, cells = O.align_pair(q, np.zeros(0, np.uint8), M, O.paper_params(pgp=3), 0, 0)
    assert s == -15 and cells == 0 and rt.tolist() == [O.GAP] * 5


def test_rounds_best_of_and_first_wins():
    M = O.blosum62()
    rng = np.random.default_rng(11)
    for trial in range(30):
        q = synth.residues(rng, int(rng.integers(5, 60)))
        t = synth.residues(rng, int(rng.integers(5, 90)))
        prev = None
        for R in [1, 2, 5, 20]:
            p = O.paper_params(rounds=R, lfactor_q16=65536, sfactor_q16=32768, minfactor_q16=16384)
            s, _, _, r, _ = O.align_pair(q, t, M, p, trial, trial)
            if prev is not None:
                assert s >= prev
            prev = s
            # the winning round alone reproduces the score: rounds 0..r only
            p2 = O.paper_params(rounds=r + 1, lfactor_q16=65536, sfactor_q16=32768, minfactor_q16=16384)
            s2, _, _, r2, _ = O.align_pair(q, t, M, p2, trial, trial)
            assert (s2, r2) == (s, r)
            if r > 0:   # strictly better than every earlier round
                p3 = O.paper_params(rounds=r, lfactor_q16=65536, sfactor_q16=32768, minfactor_q16=16384)
                assert O.align_pair(q, t, M, p3, trial, trial)[0] < s


def test_search_is_thread_count_independent_and_topk_order():
    rng = np.random.default_rng(3)
    db = synth.db_from_lengths(rng, synth.lognormal_lengths(rng, 300, 120, 0.6, 1, 600))
    q = synth.residues(rng, 50)
    M = O.blosum62()
    s1, c1, _ = O.search_scores(db.codes, db.offsets, q, M, PAPER, 9, nthreads=1)
    s4, c4, used = O.search_scores(db.codes, db.offsets, q, M, PAPER, 9, nthreads=4)
    assert used == 4 and np.array_equal(s1, s4) and np.array_equal(c1, c4)
    idx = np.arange(0, 300, 7)
    s5, _, _ = O.search_scores(db.codes, db.offsets, q, M, PAPER, 9, idx=idx, nthreads=3)
    assert np.array_equal(s5, s1[idx])
    top = O.topk(s1, 25)
    want = np.lexsort((np.arange(len(s1)), -s1))[:25]
    assert np.array_equal(top, want)


def test_seed_and_index_change_the_draws():
    M = O.blosum62()
    rng = np.random.default_rng(5)
    q = synth.residues(rng, 100)
    t = synth.residues(rng, 400)
    a = [O.align_pair(q, t, M, PAPER, seed, 0)[4] for seed in range(6)]
    b = [O.align_pair(q, t, M, PAPER, 0, d)[4] for d in range(6)]
    assert len(set(a)) > 1 and len(set(b)) > 1
