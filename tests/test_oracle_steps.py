"""Pins for the oracle's step sizing and step layout (Fig. 1's Align and
getBestSubsequenceAlignment, readings A4, A6, A9, A12, A17 and F1-F3).

Each pair is traced here step by step, by a route that shares nothing with
the oracle's C: the 16-bit draws are sliced out of numpy's own Philox4x64-10
blocks, the piece sizes are Python integers following the paper's
ls = |large rest| * lf and ss = |small rest| * sf * random() (floors, A6), and
the best shift is a numpy sliding-window argmax.  The trace predicts, per
round, every step's (ls, ss, k*), so it predicts

* the alignment rows column by column (a step writes k* letters of large
  against gaps, then its ss letter pairs; full mode adds the overhangs),
* the cell count, which is sum((ls - ss + 1) * ss) in database mode and
  sum(ls * ss) in full mode -- it sees every ls and ss even where k* = 0,
* the score, from the same steps (A17: the first step's leading gap run is
  periphery; every later k* > 0 is one interior run),

and the oracle must match all three.  The last tests plant plausible
mistakes into copies of the oracle (a draw taken from the wrong index, a
wrong fixed-point shift, the clamp applied before the product, rounding
instead of the floor, the last shift winning ties, and in full mode a wrong
overlap end or shift range) and check that these pins catch every one.
"""
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1508_06561_gb300 import synth

GAP = O.GAP


# --------------------------------------------------------------------------
# random(): numpy's Philox4x64-10 (reading A12)
# --------------------------------------------------------------------------
def philox_block(ctr, key):
    """numpy's Philox4x64-10 block for a counter; numpy increments its
    256-bit counter before each block, so it starts one below."""
    v = (ctr[0] | (ctr[1] << 64) | (ctr[2] << 128) | (ctr[3] << 192)) - 1
    v %= 2**256
    start = [(v >> (64 * i)) & (2**64 - 1) for i in range(4)]
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(start, dtype=np.uint64))
    return [int(x) for x in g.random_raw(4)]


class Draws:
    """The pair's 16-bit draws D_i: field i % 4 (most significant first) of
    word (i % 16) // 4 of the block for counter (d, r, i // 16, 0), key (seed, 0)."""

    def __init__(self, seed, d, r):
        self.seed, self.d, self.r, self.blocks = seed, d, r, {}

    def __call__(self, i):
        b = i // 16
        if b not in self.blocks:
            self.blocks[b] = philox_block([self.d, self.r, b, 0], [self.seed, 0])
        w = self.blocks[b][(i % 16) // 4]
        return (w >> (48 - 16 * (i % 4))) & 0xFFFF


# --------------------------------------------------------------------------
# The trace
# --------------------------------------------------------------------------
def trace_round(q, t, M, p, seed, d, r):
    """One round of Align: (rows as (large row, small row), steps, cells, score)."""
    q_is_large = not (len(t) >= len(q))                    # A13: the target is large on ties
    large, small = (q, t) if q_is_large else (t, q)
    nl, ns = len(large), len(small)
    D = Draws(seed, d, r)
    lf = max(p.minfactor_q16, (p.lfactor_q16 * D(0)) >> 16)   # A4 in Q16: LFactor * U1, at least MinFactor
    sf = max(p.minfactor_q16, (p.sfactor_q16 * D(1)) >> 16)
    full = p.mode == O.MODE_FULL
    Mq = M.astype(np.int64) if q_is_large else M.astype(np.int64).T   # Mq[large letter, small letter]
    rl, rs, steps = [], [], []
    Lp = Sp = t_ = 0
    cells = score = 0
    while Lp < nl and Sp < ns:
        Lrem, Srem = nl - Lp, ns - Sp
        ls = max(1, (Lrem * lf) // 65536)                  # |large rest| * lf, floored, at least 1
        ss = (Srem * sf * D(2 + t_)) // 2**32              # |small rest| * sf * random(), floored
        ss = max(1, min(ss, Srem if full else min(Srem, ls)))
        win, piece = large[Lp:Lp + ls], small[Sp:Sp + ss]
        if not full:
            # shifts 0 .. ls - ss, small wholly inside the window
            V = np.array([Mq[win[k:k + ss], piece].sum() for k in range(ls - ss + 1)])
            k = int(np.argmax(V))                          # first maximum: the lowest shift
            cells += (ls - ss + 1) * ss
            if k > 0:
                score -= p.pgp * k if t_ == 0 else p.gop + (k - 1) * p.gep     # A17
            score += int(V[k])
            rl += list(win[:k]) + list(win[k:k + ss])
            rs += [GAP] * k + list(piece)
            Lp += k + ss
        else:
            # shifts -(ss - 1) .. ls - 1, each scored over its overlap
            best, k = None, None
            for kk in range(-(ss - 1), ls):
                j = np.arange(max(0, -kk), min(ss, ls - kk))
                v = int(Mq[win[kk + j], piece[j]].sum())
                if best is None or v > best:
                    best, k = v, kk
            cells += ls * ss                               # every (large, small) letter pair once
            j0, j1 = max(0, -k), min(ss, ls - k)
            rl += [GAP] * j0 + list(win[:max(k, 0)]) + list(win[k + j0:k + j1]) + [GAP] * (ss - j1)
            rs += list(piece[:j0]) + [GAP] * max(k, 0) + list(piece[j0:j1]) + list(piece[j1:])
            Lp += k + j1
        Sp += ss
        steps.append((ls, ss, k))
        t_ += 1
    rl += list(large[Lp:]) + [GAP] * (ns - Sp)
    rs += [GAP] * (nl - Lp) + list(small[Sp:])
    if not full:
        score -= p.pgp * ((nl - Lp) + (ns - Sp))           # trailing periphery
    rq, rt = (rl, rs) if q_is_large else (rs, rl)
    return np.array(rq, np.uint8), np.array(rt, np.uint8), steps, cells, score


def trace_pair(q, t, M, p, seed, d):
    """AlignSequences: the first best of the rounds (strict '>')."""
    best = None
    cells = 0
    for r in range(p.rounds):
        rq, rt, steps, c, s = trace_round(q, t, M, p, seed, d, r)
        cells += c
        if p.mode == O.MODE_FULL:
            s = O.score_rows(rq, rt, M, p.pgp, p.gop, p.gep)   # F4: SCORE over the finished rows
        if best is None or s > best[0]:
            best = (s, rq, rt, r, steps)
    s, rq, rt, r, steps = best
    return s, rq, rt, r, cells, steps


def check_against_trace(q, t, M, p, seed, d, using=None):
    """True when the oracle (or a build of it) matches the trace in score,
    rows, winning round and cell count."""
    s, rq, rt, r, cells, steps = trace_pair(q, t, M, p, seed, d)
    os_, orq, ort, orr, oc = O.align_pair(q, t, M, p, seed, d, using=using)
    return (os_ == s and np.array_equal(orq, rq) and np.array_equal(ort, rt) and orr == r and oc == cells), steps


# --------------------------------------------------------------------------
# Cases
# --------------------------------------------------------------------------
def marker_matrix():
    """One letter pair (W, W) scores +11, every other pair -4: a window's best
    shift is wherever small's Ws meet large's, so the trace's k* values are
    spread over the whole shift range and every step boundary is visible."""
    M = np.full((24, 24), -4, np.int8)
    M[17, 17] = 11
    return M


def asymmetric_matrix(rng):
    return rng.integers(-7, 12, (24, 24)).astype(np.int8)


def cases():
    """(name, q, t, M, params, seed, d): database mode with the paper's
    parameters and others, both roles, several rounds, and full mode."""
    rng = np.random.default_rng(20240)
    out = []
    B = O.blosum62()
    for i in range(24):
        nq, nt = int(rng.integers(20, 160)), int(rng.integers(20, 200))
        q, t = synth.residues(rng, nq), synth.residues(rng, nt)
        out.append(("paper-%d" % i, q, t, B, O.paper_params(), int(rng.integers(0, 2**63)), int(rng.integers(0, 10**6))))
    for i in range(12):
        nq, nt = int(rng.integers(5, 120)), int(rng.integers(5, 120))
        # sparse Ws: windows hold one or two, so k* lands anywhere
        q = np.where(rng.random(nq) < 0.15, 17, rng.integers(0, 17, nq)).astype(np.uint8)
        t = np.where(rng.random(nt) < 0.15, 17, rng.integers(0, 17, nt)).astype(np.uint8)
        p = O.paper_params(pgp=int(rng.integers(0, 3)), rounds=int(rng.integers(1, 4)),
                           lfactor_q16=int(rng.integers(16384, 65537)), sfactor_q16=int(rng.integers(16384, 65537)),
                           minfactor_q16=int(rng.integers(0, 40000)))
        out.append(("marker-%d" % i, q, t, marker_matrix(), p, i * 977, i))
    for i in range(8):
        q, t = synth.residues(rng, int(rng.integers(10, 90))), synth.residues(rng, int(rng.integers(10, 90)))
        p = O.paper_params(lfactor_q16=65536, sfactor_q16=32768, rounds=2)     # Sec. III.B.1's example set
        out.append(("asym-%d" % i, q, t, asymmetric_matrix(rng), p, i, 31 * i))
    for i in range(16):
        nq, nt = int(rng.integers(5, 70)), int(rng.integers(5, 70))
        q = np.where(rng.random(nq) < 0.2, 17, rng.integers(0, 17, nq)).astype(np.uint8)
        t = np.where(rng.random(nt) < 0.2, 17, rng.integers(0, 17, nt)).astype(np.uint8)
        M = marker_matrix() if i % 2 else B
        p = O.paper_params(mode=O.MODE_FULL, pgp=int(rng.integers(0, 3)), rounds=int(rng.integers(1, 6)),
                           lfactor_q16=int(rng.integers(16384, 65537)), sfactor_q16=int(rng.integers(16384, 65537)),
                           minfactor_q16=int(rng.integers(0, 40000)))
        out.append(("full-%d" % i, q, t, M, p, 5 * i + 1, 7 * i))
    return out


CASES = cases()


def test_draws_from_numpy_match_the_oracle_layout_at_large_indices():
    D = Draws(2**63 + 11, 569_999, 2)
    for i in [0, 1, 2, 15, 16, 17, 63, 64, 200]:
        assert D(i) == O.draw16(2**63 + 11, 569_999, 2, i)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_oracle_matches_the_step_trace(case):
    name, q, t, M, p, seed, d = case
    ok, steps = check_against_trace(q, t, M, p, seed, d)
    assert ok, name
    assert len(steps) >= 1


def test_traces_cover_the_interesting_steps():
    """The cases above exercise what the pins are for: multi-step rounds,
    steps whose best shift is not 0, steps whose piece is clamped by the
    window (ss = ls), and in full mode negative and overhanging shifts."""
    seen = dict(multi=0, kpos=0, clamp=0, neg=0, over=0)
    for name, q, t, M, p, seed, d in CASES:
        for r in range(p.rounds):
            _, _, steps, _, _ = trace_round(q, t, M, p, seed, d, r)
            seen["multi"] += len(steps) >= 3
            for ls, ss, k in steps:
                seen["kpos"] += k > 0
                seen["clamp"] += p.mode == O.MODE_DB and ss == ls and ls > 1
                seen["neg"] += k < 0
                seen["over"] += p.mode == O.MODE_FULL and k > ls - ss
    assert seen["multi"] >= 20 and seen["kpos"] >= 50 and seen["clamp"] >= 3, seen
    assert seen["neg"] >= 3 and seen["over"] >= 3, seen


def test_hand_worked_first_step():
    """Q = WCWHKLMN (8 letters) against T = AAWCWHKLMNPQ (12), paper
    parameters, seed 3, database index 5, round 0.  numpy's Philox gives
    D_0 = 60587, D_1 = 14299, D_2 = 35381.  lf = max(0.5, 0.5 * D_0 / 2^16) =
    0.5 and sf = max(0.5, D_1 / 2^16) = 0.5, so step 0 has
    ls = floor(12 * 0.5) = 6 (window AAWCWH) and
    ss = floor(8 * 0.5 * 35381 / 2^16) = floor(2.16) = 2 (piece WC).
    BLOSUM62: V(0) = A.W + A.C = -3 + 0, V(1) = A.W + W.C = -3 - 2,
    V(2) = W.W + C.C = 11 + 9, V(3) = C.W + W.C = -2 - 2,
    V(4) = W.W + H.C = 11 - 3; so k* = 2 and the step scores 20 after a
    leading periphery run of 2 (PGP = 0), with (6 - 2 + 1) * 2 = 10 cells."""
    M = O.blosum62()
    q, t = O.encode("WCWHKLMN"), O.encode("AAWCWHKLMNPQ")
    D = Draws(3, 5, 0)
    assert (D(0), D(1), D(2)) == (60587, 14299, 35381)
    W, C, A, H = (int(O.encode(x)[0]) for x in "WCAH")
    V = [M[A, W] + M[A, C], M[A, W] + M[W, C], M[W, W] + M[C, C], M[C, W] + M[W, C], M[W, W] + M[H, C]]
    assert [int(v) for v in V] == [-3, -5, 20, -4, 8]
    _, _, steps, cells, _ = trace_round(q, t, M, O.paper_params(), 3, 5, 0)
    assert steps[0] == (6, 2, 2)
    assert cells == sum((ls - ss + 1) * ss for ls, ss, _ in steps) and cells >= 10
    s, rq, rt, _, oc = O.align_pair(q, t, M, O.paper_params(), 3, 5)
    assert rq[:4].tolist() == [GAP, GAP, W, C] and rt[:4].tolist() == t[:4].tolist()
    assert oc == cells and check_against_trace(q, t, M, O.paper_params(), 3, 5)[0]


# --------------------------------------------------------------------------
# Planted mistakes: each must fail the pins above
# --------------------------------------------------------------------------
MUTANTS = {
    "step draw from D_(1+t)": ("draw16(seed, d, r, 2 + (uint64_t)t)", "draw16(seed, d, r, 1 + (uint64_t)t)"),
    "step draw from D_(3+t)": ("draw16(seed, d, r, 2 + (uint64_t)t)", "draw16(seed, d, r, 3 + (uint64_t)t)"),
    "ss shifted by 31": ("((uint64_t)Srem * sf * u) >> 32", "((uint64_t)Srem * sf * u) >> 31"),
    "ss shifted by 33": ("((uint64_t)Srem * sf * u) >> 32", "((uint64_t)Srem * sf * u) >> 33"),
    "clamp before the product": ("((uint64_t)Srem * sf * u) >> 32",
                                 "((uint64_t)(Srem < ls ? Srem : ls) * sf * u) >> 32"),
    "ls rounded": ("((uint64_t)Lrem * lf) >> 16", "((uint64_t)Lrem * lf + 32768) >> 16"),
    "lf and sf draws swapped": ("u1 = draw16(seed, dbidx, (uint64_t)r, 0), u2 = draw16(seed, dbidx, (uint64_t)r, 1)",
                                "u1 = draw16(seed, dbidx, (uint64_t)r, 1), u2 = draw16(seed, dbidx, (uint64_t)r, 0)"),
    "last shift wins ties": ("if (score > best) { best = score; *best_k = k; }",
                             "if (score >= best) { best = score; *best_k = k; }"),
    "full: overlap end ignores the window": ("const int64_t j1 = (ls - kstar < ss) ? ls - kstar : ss;",
                                             "const int64_t j1 = ss;"),
    "full: large advances by ss": ("Lp += kstar + j1;", "Lp += kstar + ss;"),
    "full: last shift dropped": ("int64_t start = 0, end = n - 1;", "int64_t start = 0, end = n - 2;"),
}


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    src = open(O.SRC).read()
    d = tmp_path_factory.mktemp("mutants")
    libs = {}
    for i, (name, (old, new)) in enumerate(MUTANTS.items()):
        assert src.count(old) >= 1, "mutation site not found: %s" % name
        path = str(d / ("m%d.so" % i))
        c = str(d / ("m%d.c" % i))
        with open(c, "w") as f:
            f.write(src.replace(old, new))
        subprocess.check_call([gcc, "-O1", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-o", path, c])
        libs[name] = O.load(path)
    return libs


@pytest.mark.parametrize("name", list(MUTANTS))
def test_each_planted_mistake_is_caught(mutant_libs, name):
    L = mutant_libs[name]
    caught = [c[0] for c in CASES if not check_against_trace(*c[1:], using=L)[0]]
    assert caught, "the step pins did not notice: %s" % name
