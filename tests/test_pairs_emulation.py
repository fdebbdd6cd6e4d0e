"""The scan's whole pair loop on the CPU, checked against the oracle.

run_pairs -- the loop every scan kernel's warps run: queue refill, the two
schedule phases, step planning from the Philox draws, the ranked and
flattened unit list with its pass owners and key folding, the lane grid for
the remaining steps, consume, score and settle -- is cut out of
csrc/hs_scan.cu as it stands and compiled as plain C++ into
tests/emu/pairs_emu.cpp, which runs each warp as 32 threads in lockstep (the
stub cuda_runtime.h turns every warp intrinsic into a post-and-wait
exchange).  Per-pair scores and cell counts must equal the oracle's exactly,
for both accumulator forms, several warps sharing one queue, long targets
(the one-per-warp phase), empty targets, several rounds and shard offsets.
The one-warp-per-pair path (align_pair: full-slide mode, replay) and the
one-CTA-per-pair path (align_round_cta, with a CTA barrier) run the same
way, and so does the replay's emission of run-length ops, whose rows must
equal the oracle's alignment.  A change to the kernel's bookkeeping can so be checked without a
GPU.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1508_06561_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1508_06561_gb300", "csrc")


def pair_loop_source():
    """run_pairs and its helpers, verbatim from the kernel source."""
    with open(os.path.join(CSRC, "hs_scan.cu")) as f:
        s = f.read()
    a = s.find("constexpr int kLocalIters")
    b = s.find("// Plain scan: a persistent grid over one queue")
    assert a >= 0 and b > a, "pair-loop markers not found in hs_scan.cu"
    b = s.rfind("// ----", 0, b)
    region = s[a:b]
    assert "void run_pairs(" in region
    return region


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("pairs_emu")
    with open(d / "hs_pairs_region.inc", "w") as f:
        f.write(pair_loop_source())
    exe = str(d / "pairs_emu")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", "-Wno-unknown-pragmas",
                           "-I", os.path.join(ROOT, "tests", "emu"), "-I", str(d), "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(ROOT, "tests", "emu", "pairs_emu.cpp")])
    return exe, d


def run_emu(emu, codes, offsets, q, M, p, seed, warps=2, index_base=0, how="", flat=None, lanes=None,
            help_min=None):
    exe, d = emu
    n = len(offsets) - 1
    hdr = struct.pack("<qqiiiiiiiIIIQq", n, len(codes), len(q), warps, p.pgp, p.gop, p.gep, p.rounds, p.mode,
                      p.lfactor_q16, p.sfactor_q16, p.minfactor_q16, seed, index_base)
    inp, out = str(d / "in.bin"), str(d / "out.bin")
    with open(inp, "wb") as f:
        f.write(hdr)
        f.write(np.ascontiguousarray(M, np.int8).tobytes())
        f.write(np.ascontiguousarray(codes, np.uint8).tobytes())
        f.write(np.ascontiguousarray(offsets, np.int64).tobytes())
        f.write(np.ascontiguousarray(q, np.uint8).tobytes())
    env = dict(os.environ)
    if flat is not None:            # (flat_min_chunks, flat_max_iters), as a batch tuning sets them
        env["HS_EMU_FLAT_MIN_CHUNKS"], env["HS_EMU_FLAT_MAX_ITERS"] = str(flat[0]), str(flat[1])
    if lanes is not None:           # lanes a warp fills with pairs
        env["HS_EMU_LANES"] = str(lanes)
    if help_min is not None:        # units from which a lone flat step is shared with idle warps
        env["HS_EMU_HELP_MIN"] = str(help_min)
    subprocess.run([exe, inp, out] + ([how] if how else []), check=True, timeout=600, env=env)
    with open(out, "rb") as f:
        b = f.read()
    scores = np.frombuffer(b, np.int32, n)
    cells = np.frombuffer(b, np.int64, n, 4 * n)
    pair16, long_end = struct.unpack("<iq", b[12 * n:12 * n + 12])
    return scores, cells, pair16, long_end


def oracle_scores(db, q, M, p, seed, index_base=0):
    if index_base == 0:
        s, c, _ = O.search_scores(db.codes, db.offsets, q, M, p, seed)
        return np.asarray(s), np.asarray(c)
    s, c = [], []
    for d in range(db.n):
        r = O.align_pair(q, db.seq(d), M, p, seed, d + index_base)
        s.append(r[0])
        c.append(r[4])
    return np.array(s), np.array(c)


def mixed_db(rng, n_short, long_lens, extra=(0, 1, 2, 3)):
    lengths = np.concatenate([rng.integers(1, 400, n_short), list(extra), list(long_lens)]).astype(np.int64)
    rng.shuffle(lengths)
    return synth.db_from_lengths(rng, lengths)


def check(emu, db, q, M, p, seed, warps=2, index_base=0, want_pair16=None, want_long=None, how="", flat=None,
          lanes=None, help_min=None):
    s, c, pair16, long_end = run_emu(emu, db.codes, db.offsets, q, M, p, seed, warps, index_base, how, flat, lanes,
                                     help_min)
    ref, refc = oracle_scores(db, q, M, p, seed, index_base)
    bad = np.nonzero(s != ref)[0]
    assert bad.size == 0, "scores differ at %s: %s vs oracle %s" % (bad[:5], s[bad[:5]], ref[bad[:5]])
    assert np.array_equal(c, refc)
    if want_pair16 is not None:
        assert pair16 == want_pair16
    if want_long is not None:
        assert long_end == want_long


def test_paper_parameters_with_long_and_empty_targets(emu):
    rng = np.random.default_rng(7)
    db = mixed_db(rng, 250, [2048, 2900, 3999])
    check(emu, db, synth.residues(rng, 120), O.blosum62(), O.paper_params(), 5, want_pair16=1, want_long=3)


@pytest.mark.parametrize("qlen", [1, 3, 17, 600])
def test_query_lengths_and_three_warps_on_one_queue(emu, qlen):
    rng = np.random.default_rng(100 + qlen)
    db = mixed_db(rng, 120, [2100])
    check(emu, db, synth.residues(rng, qlen), O.blosum62(), O.paper_params(), qlen, warps=3)


def test_32_bit_accumulators(emu):
    """A full-range matrix with a 300-letter query: 16-bit pair sums could
    overflow, so the loop takes its 32-bit form (lane-local and lane-grid
    steps, byte lanes widened after every cell)."""
    rng = np.random.default_rng(11)
    M = synth.random_symmetric_matrix(rng, -128, 127)
    db = mixed_db(rng, 120, [2300])
    check(emu, db, synth.residues(rng, 300), M, O.paper_params(), 3, want_pair16=0)


def test_narrow_flush_matrix(emu):
    rng = np.random.default_rng(12)
    M = synth.random_symmetric_matrix(rng, -40, 50)         # widen every 2 cells, 16-bit pairs
    db = mixed_db(rng, 150, [])
    check(emu, db, synth.residues(rng, 90), M, O.paper_params(gop=3, gep=1), 9, want_pair16=1, want_long=0)


def test_rounds_factors_and_periphery(emu):
    """Best of several rounds with the Sec. III.B.1 example factors (LFactor 1,
    SFactor 0.5) and a periphery penalty."""
    rng = np.random.default_rng(13)
    db = mixed_db(rng, 150, [2500])
    p = O.paper_params(rounds=3, lfactor_q16=65536, sfactor_q16=32768, minfactor_q16=16384, pgp=2)
    check(emu, db, synth.residues(rng, 70), O.blosum62(), p, 21)


def test_shard_offset_keys_the_draws(emu):
    rng = np.random.default_rng(14)
    db = mixed_db(rng, 60, [], extra=())
    check(emu, db, synth.residues(rng, 80), O.blosum62(), O.paper_params(), 4, index_base=123456)


@pytest.mark.parametrize("mode", ["db", "full"])
def test_one_warp_per_pair(emu, mode):
    """The full-slide scan's loop (run_full_items: one (pair, round) item per
    warp, rounds folded by atomics; readings F1-F4, several rounds) and, in
    database mode, align_pair one warp per pair, the path the one-warp replay
    and hs_get_alignment run."""
    rng = np.random.default_rng(15 if mode == "db" else 16)
    db = mixed_db(rng, 80, [2200])
    if mode == "db":
        p = O.paper_params(rounds=2)
    else:
        p = O.paper_params(rounds=4, mode=O.MODE_FULL, sfactor_q16=65536, lfactor_q16=65536, minfactor_q16=16384)
    check(emu, db, synth.residues(rng, 60), O.blosum62(), p, 8, warps=3, how="whole")


@pytest.mark.parametrize("matrix,qlen", [("blosum62", 300), ("full-range", 120)])
def test_full_slide_items_both_roles(emu, matrix, qlen):
    """Full-slide mode (F1-F4) with the query long enough that many targets
    are shorter (the query is then the large sequence), high size factors
    (steps whose piece of small is longer than large's window, so every
    shift overhangs) and, for the full int8 range, byte sums widened every
    cell."""
    rng = np.random.default_rng(19 if matrix == "blosum62" else 20)
    M = O.blosum62() if matrix == "blosum62" else synth.random_symmetric_matrix(rng, -128, 127)
    db = mixed_db(rng, 70, [900])
    p = O.paper_params(rounds=5, mode=O.MODE_FULL, sfactor_q16=65536, lfactor_q16=40000, minfactor_q16=8192)
    check(emu, db, synth.residues(rng, qlen), M, p, 21, warps=3, how="whole")


@pytest.mark.parametrize("matrix,qlen,lanes,flat", [("blosum62", 60, None, None), ("blosum62", 300, 5, None),
                                                    ("wide", 90, None, (1, 100000)), ("blosum62", 40, None, (100000, 1)),
                                                    ("blosum62", 1, 3, None)])
def test_full_slide_lane_owned_items(emu, matrix, qlen, lanes, flat):
    """Full-slide mode with every lane holding one (pair, round) item and the
    warp's flat steps dealt as units (run_full_pairs, F1-F4): both roles,
    overhanging steps, several rounds of a long pair in neighbouring lanes,
    warps filling only some lanes, every step flat and none flat, a wide
    matrix (byte sums widened every few cells)."""
    rng = np.random.default_rng(90 + qlen)
    M = O.blosum62() if matrix == "blosum62" else synth.random_symmetric_matrix(rng, -40, 50)
    db = mixed_db(rng, 60, [2300])
    p = O.paper_params(rounds=6, mode=O.MODE_FULL, sfactor_q16=65536, lfactor_q16=45000, minfactor_q16=10000,
                       pgp=1)
    check(emu, db, synth.residues(rng, qlen), M, p, 31, warps=3, how="lanes", lanes=lanes, flat=flat)


@pytest.mark.parametrize("matrix", ["blosum62", "full-range"])
def test_one_cta_per_pair(emu, matrix):
    """align_round_cta: every step of a pair scanned by all warps of a CTA,
    their best shifts reduced through shared memory (the replay's path for
    one-round searches), for both accumulator forms and several rounds."""
    rng = np.random.default_rng(17 if matrix == "blosum62" else 18)
    M = O.blosum62() if matrix == "blosum62" else synth.random_symmetric_matrix(rng, -128, 127)
    db = mixed_db(rng, 60, [2400])
    check(emu, db, synth.residues(rng, 280), M, O.paper_params(rounds=2), 6, warps=4, how="cta")


def run_replay(emu, db, q, M, p, seed, warps, how):
    exe, d = emu
    hdr = struct.pack("<qqiiiiiiiIIIQq", db.n, len(db.codes), len(q), warps, p.pgp, p.gop, p.gep, p.rounds, p.mode,
                      p.lfactor_q16, p.sfactor_q16, p.minfactor_q16, seed, 0)
    inp, out = str(d / "in.bin"), str(d / "out.bin")
    with open(inp, "wb") as f:
        f.write(hdr)
        f.write(np.ascontiguousarray(M, np.int8).tobytes())
        f.write(np.ascontiguousarray(db.codes, np.uint8).tobytes())
        f.write(np.ascontiguousarray(db.offsets, np.int64).tobytes())
        f.write(np.ascontiguousarray(q, np.uint8).tobytes())
    subprocess.run([exe, inp, out, how], check=True, timeout=600)
    with open(out, "rb") as f:
        b = f.read()
    res, at = [], 0
    for _ in range(db.n):
        score, nops, qb, qe, tb, te = struct.unpack_from("<6i", b, at)
        at += 24
        res.append((score, (qb, qe, tb, te), np.frombuffer(b, np.uint32, nops, at)))
        at += 4 * nops
    assert at == len(b)
    return res


@pytest.mark.parametrize("how,mode,rounds", [("ops", "db", 3), ("ops", "full", 2), ("ops_cta", "db", 1)])
def test_replayed_alignments(emu, how, mode, rounds):
    """The replay's emission -- run-length ops and core span of the best
    round, by one warp, or by one CTA for one-round searches -- expands to
    the oracle's alignment rows, rescores to the score, and spans the first
    to the last letter pair."""
    from paper_1508_06561_gb300 import ops_to_rows
    rng = np.random.default_rng(19 + rounds)
    db = mixed_db(rng, 40, [2100])
    q = synth.residues(rng, 70)
    M = O.blosum62()
    p = O.paper_params(rounds=rounds, pgp=1, mode=O.MODE_FULL if mode == "full" else O.MODE_DB)
    for d, (score, span, ops) in enumerate(run_replay(emu, db, q, M, p, 2, 3, how)):
        t = db.seq(d)
        s, oq, ot, _, _ = O.align_pair(q, t, M, p, 2, d)
        rq, rt = ops_to_rows(ops, q, t)
        assert score == s and np.array_equal(rq, oq) and np.array_equal(rt, ot), d
        assert O.score_rows(rq, rt, M, p.pgp, p.gop, p.gep) == s
        m = (rq != 255) & (rt != 255)
        if m.any():
            cols = np.nonzero(m)[0]
            qpos, tpos = np.cumsum(rq != 255) - 1, np.cumsum(rt != 255) - 1
            assert span == (qpos[cols[0]], qpos[cols[-1]] + 1, tpos[cols[0]], tpos[cols[-1]] + 1)


@pytest.fixture(scope="module")
def emu_tsan(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("pairs_emu_tsan")
    with open(d / "hs_pairs_region.inc", "w") as f:
        f.write(pair_loop_source())
    exe = str(d / "pairs_emu")
    r = subprocess.run([gxx, "-O1", "-g", "-fsanitize=thread", "-std=c++17", "-pthread", "-Wno-unknown-pragmas",
                        "-I", os.path.join(ROOT, "tests", "emu"), "-I", str(d), "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), "-o", exe,
                        os.path.join(ROOT, "tests", "emu", "pairs_emu.cpp")], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no ThreadSanitizer runtime: " + r.stderr[-200:])
    return exe, d


@pytest.mark.parametrize("how", ["", "help", "lanes", "cta", "ops_cta"])
def test_shared_memory_traffic_is_ordered(emu_tsan, how):
    """Under ThreadSanitizer every read of a slot another lane or warp wrote
    (plans, flat-step descriptors and keys, the CTA's reduction words, the
    boards of steps shared with idle warps) must be ordered by the warp or
    CTA barrier or the atomics the device code places; an unordered one is
    reported as a race."""
    exe, d = emu_tsan
    env = dict(os.environ)
    if how == "help":               # every lone flat step shared
        env["HS_EMU_HELP_MIN"] = "1"
        how = ""
    rng = np.random.default_rng(3)
    db = mixed_db(rng, 60, [2100], extra=(0, 2))
    q = synth.residues(rng, 50)
    p = O.paper_params(rounds=3, mode=O.MODE_FULL) if how == "lanes" else O.paper_params()
    hdr = struct.pack("<qqiiiiiiiIIIQq", db.n, len(db.codes), len(q), 2, p.pgp, p.gop, p.gep, p.rounds, p.mode,
                      p.lfactor_q16, p.sfactor_q16, p.minfactor_q16, 1, 0)
    inp, out = str(d / "in.bin"), str(d / "out.bin")
    with open(inp, "wb") as f:
        f.write(hdr)
        f.write(O.blosum62().tobytes())
        f.write(np.ascontiguousarray(db.codes, np.uint8).tobytes())
        f.write(np.ascontiguousarray(db.offsets, np.int64).tobytes())
        f.write(np.ascontiguousarray(q, np.uint8).tobytes())
    r = subprocess.run([exe, inp, out] + ([how] if how else []), capture_output=True, text=True, timeout=900,
                       env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "WARNING: ThreadSanitizer" not in r.stderr, r.stderr[:4000]


@pytest.mark.parametrize("case", range(8))
def test_random_configurations(emu, case):
    """Seeded random databases, queries, matrices and parameters: lengths
    around the role switch and the one-per-warp threshold, matrix ranges
    from 1 to 255, every factor and penalty in its accepted range, and in
    two cases of three random flat-list thresholds (every step flat, every
    step on the lane grid, and between)."""
    rng = np.random.default_rng(1000 + case)
    qlen = int(rng.choice([1, 2, 5, 31, 64, 129, 256, 511, 1000]))
    lengths = np.concatenate([rng.integers(0, 2 * qlen + 8, 40), [qlen - 1, qlen, qlen + 1],
                              rng.integers(2000, 2200, int(rng.integers(0, 3)))]).clip(0)
    db = synth.db_from_lengths(rng, lengths)
    lo = int(rng.integers(-128, 0))
    hi = int(rng.integers(lo + 1, 128))
    M = synth.random_symmetric_matrix(rng, lo, hi)
    p = O.paper_params(pgp=int(rng.integers(0, 6)), gop=int(rng.integers(0, 20)), gep=int(rng.integers(0, 8)),
                       rounds=int(rng.integers(1, 4)), lfactor_q16=int(rng.integers(0, 65537)),
                       sfactor_q16=int(rng.integers(0, 65537)), minfactor_q16=int(rng.integers(0, 65537)))
    flat = None if case % 3 == 0 else (int(rng.choice([1, 4, 16, 64, 100000])), int(rng.choice([1, 32, 128, 100000])))
    check(emu, db, synth.residues(rng, qlen), M, p, int(rng.integers(0, 2**63)), warps=int(rng.integers(1, 4)),
          flat=flat)


@pytest.mark.parametrize("help_min,warps,qlen", [(1, 3, 60), (16, 4, 200), (64, 2, 20), (1, 4, 1)])
def test_idle_warps_share_lone_steps(emu, help_min, warps, qlen):
    """The end of a scan: a warp left with one pair publishes each of its
    flat steps with at least help_min units, the CTA's warps that ran out
    of pairs take passes of it, and the owner waits for them before it
    consumes the step.  Scores and cell counts must equal the oracle's,
    every warp must leave, and no wait may run out."""
    rng = np.random.default_rng(70 + help_min + warps)
    db = mixed_db(rng, 50, [3100])              # one long pair outlasts the short ones
    check(emu, db, synth.residues(rng, qlen), O.blosum62(), O.paper_params(rounds=2), 5, warps=warps,
          help_min=help_min)


@pytest.mark.parametrize("lanes", [1, 3, 17])
def test_warps_filling_only_some_lanes(emu, lanes):
    """A small database spreads one or a few pairs per warp: the warp's
    other lanes hold no pair but still score units of its steps."""
    rng = np.random.default_rng(60 + lanes)
    db = mixed_db(rng, 120, [2048, 2100])
    check(emu, db, synth.residues(rng, 70), O.blosum62(), O.paper_params(rounds=2), 3, warps=3, lanes=lanes)


@pytest.fixture(scope="module")
def help_emu(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("help_emu")
    with open(d / "hs_pairs_region.inc", "w") as f:
        f.write(pair_loop_source())
    exe = str(d / "help_emu")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", "-Wno-unknown-pragmas",
                           "-I", os.path.join(ROOT, "tests", "emu"), "-I", str(d), "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), "-o", exe,
                           os.path.join(ROOT, "tests", "emu", "help_emu.cpp")])
    return exe


def run_help(exe, how, seed):
    r = subprocess.run([exe, how, str(seed)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    f = r.stdout.split()
    return {f[i]: float(f[i + 1]) for i in range(0, len(f), 2)}


@pytest.mark.parametrize("seed", [1, 2])
def test_shared_step_key_with_a_helper(help_emu, seed):
    """A step shared by its owner and one helper warp: the folded key is the
    maximum of the units' keys, both warps leave, the status stays OK."""
    r = run_help(help_emu, "ok", seed)
    assert r["key"] == r["want"] and r["status"] == 0 and r["live"] == 0


def test_owner_gives_up_on_a_pass_that_never_finishes(help_emu):
    """A helper that claims a pass and never finishes it (made on the host:
    a stand-in thread that stops after its claim): the owner's wait runs out
    after its 2 s limit, it records HS_ETIMEOUT (5) and returns."""
    for seed in range(5):                       # the stand-in must win a claim before the owner takes them all
        r = run_help(help_emu, "stuck", seed)
        if r["claimed"]:
            break
    assert r["claimed"] == 1
    assert r["status"] == 5
    assert 2000 <= r["ms"] < 20000
