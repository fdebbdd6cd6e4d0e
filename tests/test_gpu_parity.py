"""GPU path vs the CPU oracle, bit for bit (all arithmetic is integer).

Every test calls the library through its C ABI (via the ctypes binding) and
compares with ``oracle`` on the same seeded inputs: every pair's score and
cell count, the ranked hits, and every hit's alignment rows.
"""
import numpy as np
import pytest

import oracle as O
import paper_1508_06561_gb300 as P
from paper_1508_06561_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_06561_gb300 import build
    build.build()
    O.build()
    torch.cuda.set_device(0)


from gpu_checks import check_hits, oparams, run_device  # noqa: E402


def full_parity(db, q, k, params, seed, M=None):
    M = O.blosum62() if params.matrix is None else params.matrix
    op = oparams(params)
    D = P.Database(db.codes, db.offsets)
    hits, ops, scores, cells = run_device(D, q, k, params, seed)
    ref, ref_cells, _ = O.search_scores(db.codes, db.offsets, q, M, op, seed)
    bad = np.nonzero(scores != ref)[0]
    assert len(bad) == 0, "score mismatch at %s: gpu %s oracle %s" % (bad[:5], scores[bad[:5]], ref[bad[:5]])
    assert np.array_equal(cells, ref_cells)
    check_hits(db, q, M, op, seed, hits, ops, ref, min(k, db.n))
    # the host-buffer entry point returns the same hits and ops
    h2, o2 = P.search(D, q, k, params, seed)
    assert np.array_equal(h2, hits) and np.array_equal(o2, ops)
    D.close()
    return scores


def test_plain_small_workload():
    db, q, k = synth.plain_small(0)
    full_parity(db, q, k, P.Params(), seed=0)


EDGE_QLENS = [1, 2, 3, 4, 5, 7, 31, 64, 127, 255, 256, 257, 600]


@pytest.mark.parametrize("case", range(len(EDGE_QLENS)))
def test_random_databases(case):
    rng = np.random.default_rng(9000 + case)
    qlen = EDGE_QLENS[case]
    n = int(rng.integers(1, 400))
    lengths = np.concatenate([
        rng.integers(0, 4, n // 8 + 1),                       # empty and tiny targets
        rng.integers(max(1, qlen - 3), qlen + 4, n // 8 + 1),  # around the role switch
        synth.lognormal_lengths(rng, n, 250, 0.8, 1, 3000),
    ])
    rng.shuffle(lengths)
    db = synth.db_from_lengths(rng, lengths)
    q = synth.residues(rng, qlen)
    kind = case % 4
    if kind == 0:
        params = P.Params()
    elif kind == 1:
        params = P.Params(pgp=int(rng.integers(0, 4)), gop=int(rng.integers(0, 20)), gep=int(rng.integers(0, 7)),
                          rounds=int(rng.integers(1, 4)), lfactor_q16=int(rng.integers(1, 65537)),
                          sfactor_q16=int(rng.integers(1, 65537)), minfactor_q16=int(rng.integers(0, 65537)))
    elif kind == 2:   # a wide matrix: flush every 3 cells
        params = P.Params(matrix=synth.random_symmetric_matrix(rng, -40, 50), rounds=2)
    else:             # the widest int8 range: flush every cell
        params = P.Params(matrix=synth.random_symmetric_matrix(rng, -128, 127), pgp=1)
    full_parity(db, q, int(rng.integers(1, 40)), params, seed=int(rng.integers(0, 2**63)))


def test_paper_example_factor_setting():
    """Sec. III.B.1's suggested setting (SFactor=0.5 < LFactor=1)."""
    rng = np.random.default_rng(77)
    db = synth.db_from_lengths(rng, synth.lognormal_lengths(rng, 300, 300, 0.6, 1, 2000))
    q = synth.residues(rng, 120)
    full_parity(db, q, 20, P.Params(lfactor_q16=65536, sfactor_q16=32768), seed=5)


def test_long_targets_and_long_query():
    rng = np.random.default_rng(31)
    lengths = np.array([35_000, 20_000, 9000, 5000, 2048, 2047, 2100, 1999, 300, 17, 0, 1] + [400] * 30)
    db = synth.db_from_lengths(rng, lengths)
    for qlen in [2048, 1500, 64]:
        q = synth.residues(rng, qlen)
        full_parity(db, q, 10, P.Params(), seed=qlen)


def test_k_edge_cases():
    rng = np.random.default_rng(5)
    db = synth.db_from_lengths(rng, [50, 0, 120, 7])
    q = synth.residues(rng, 30)
    D = P.Database(db.codes, db.offsets)
    hits, ops = P.search(D, q, 0)
    assert len(hits) == 0 and len(ops) == 0
    hits, ops = P.search(D, q, 100)            # k > n: every target, ranked
    ref, _, _ = O.search_scores(db.codes, db.offsets, q, O.blosum62(), O.paper_params(), 0)
    assert hits["db_index"].tolist() == O.topk(ref, 4).tolist()
    D.close()
    one = synth.db_from_lengths(rng, [0])
    D1 = P.Database(one.codes, one.offsets)
    hits, ops = P.search(D1, q, 3)
    assert len(hits) == 1 and hits[0]["score"] == 0 and hits[0]["q_begin"] == -1
    assert P.ops_to_rows(ops, q, one.seq(0))[1].tolist() == [255] * 30
    D1.close()


def test_get_alignment_matches_search():
    rng = np.random.default_rng(12)
    db = synth.db_from_lengths(rng, synth.lognormal_lengths(rng, 200, 300, 0.6, 1, 2000))
    q = synth.residues(rng, 90)
    D = P.Database(db.codes, db.offsets)
    params = P.Params(pgp=2, rounds=3, lfactor_q16=50000)
    hits, ops = P.search(D, q, 8, params, seed=44)
    for h in hits:
        s, o, rec = P.get_alignment(D, q, int(h["db_index"]), params, seed=44)
        assert s == h["score"]
        assert o.tolist() == ops[h["ops_offset"]:h["ops_offset"] + h["ops_len"]].tolist()
    # any pair, not only hits
    for d in [0, 1, 57, 199]:
        s, o, _ = P.get_alignment(D, q, d, params, seed=44)
        ref = O.align_pair(q, db.seq(d), O.blosum62(), oparams(params), 44, d)
        assert s == ref[0]
        rq, rt = P.ops_to_rows(o, q, db.seq(d))
        assert np.array_equal(rq, ref[1]) and np.array_equal(rt, ref[2])
    D.close()


def test_repeatable_across_runs_and_streams():
    rng = np.random.default_rng(3)
    db = synth.db_from_lengths(rng, synth.lognormal_lengths(rng, 1000, 300, 0.6, 1, 4000))
    q = synth.residues(rng, 100)
    D = P.Database(db.codes, db.offsets)
    a = P.search(D, q, 50, seed=8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = P.search(D, q, 50, seed=8, stream=s)
    c = P.search(D, q, 50, seed=9)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0]["score"], c[0]["score"]) or not np.array_equal(a[1], c[1])
    D.close()


def test_swissprot_scale_full():
    """The plain database-scale workload (256-residue query, ~570k targets,
    ~205M residues, top-100) in the benchmark's launch configuration (seed 1),
    compared in full: every one of the 570,000 pair scores and cell counts
    equals the oracle's, the top 100 is the oracle's ranking, and every hit's
    alignment rows and core span are the oracle's."""
    db, q, k = synth.plain_large()
    D = P.Database(db.codes, db.offsets)
    params = P.Params()
    hits, ops, scores, cells = run_device(D, q, k, params, 1)
    M, op = O.blosum62(), O.paper_params()
    ref, ref_cells, _ = O.search_scores(db.codes, db.offsets, q, M, op, 1)
    bad = np.nonzero(scores != ref)[0]
    assert len(bad) == 0, "score mismatch at %s: gpu %s oracle %s" % (bad[:5], scores[bad[:5]], ref[bad[:5]])
    assert np.array_equal(cells, ref_cells)
    assert int(ref_cells.sum()) == 7_889_671_540           # the work count the roofline is quoted on
    check_hits(db, q, M, op, 1, hits, ops, ref, k)
    D.close()


def oparams_full(p: P.Params):
    op = oparams(p)
    op.mode = O.MODE_FULL
    return op


@pytest.mark.parametrize("case", range(7))
def test_full_slide_mode(case):
    """Fig. 1 as printed (pair-wise form): every score, cell count, ranked
    hit and alignment equals the oracle's, overhanging pieces included;
    the last case takes the full int8 matrix range (byte sums widened every
    cell)."""
    rng = np.random.default_rng(4200 + case)
    qlen = [1, 7, 40, 130, 300, 700, 90][case]
    lengths = np.concatenate([rng.integers(0, 4, 5), synth.lognormal_lengths(rng, 250, 150, 0.7, 1, 2500)])
    db = synth.db_from_lengths(rng, lengths)
    q = synth.residues(rng, qlen)
    p = P.Params(pgp=int(rng.integers(0, 3)), gop=int(rng.integers(1, 15)), gep=int(rng.integers(0, 6)),
                 rounds=[1, 20, 3, 20, 2, 5, 4][case], lfactor_q16=int(rng.integers(20000, 65537)),
                 sfactor_q16=int(rng.integers(20000, 65537)), minfactor_q16=int(rng.integers(0, 40000)),
                 matrix=synth.random_symmetric_matrix(rng, -128, 127) if case == 6 else
                 None if case % 2 else synth.random_symmetric_matrix(rng, -7, 9))
    M = O.blosum62() if p.matrix is None else p.matrix
    op = oparams_full(p)
    seed = int(rng.integers(0, 2**62))
    D = P.Database(db.codes, db.offsets)
    hits, ops, scores, cells = run_device(D, q, 15, p_full(p), seed)
    ref, ref_cells, _ = O.search_scores(db.codes, db.offsets, q, M, op, seed)
    assert np.array_equal(scores, ref)
    assert np.array_equal(cells, ref_cells)
    check_hits(db, q, M, op, seed, hits, ops, ref, min(15, db.n))
    s, o, _ = P.get_alignment(D, q, int(hits[0]["db_index"]), p_full(p), seed)
    assert s == hits[0]["score"]
    D.close()


def p_full(p: P.Params):
    f = P.Params(**p.__dict__)
    f.mode = 1
    return f


def test_batched_rejects_full_mode():
    rng = np.random.default_rng(1)
    db = synth.db_from_lengths(rng, [50, 60])
    D = P.Database(db.codes, db.offsets)
    with pytest.raises(P.HsError):
        P.search_batch(D, [synth.residues(rng, 10)], 2, p_full(P.Params()))
    D.close()


def test_trace_hook_packs_shift_counts():
    """With the trace hook's pack_shifts set, a database-mode search that
    counts cells stores per pair cells + (shifts << 40), shifts being the
    shifts whose virtual score was taken (sum of ls - ss + 1 over the steps
    of every round).  Both parts equal the independent step trace's
    (tests/test_oracle_steps.py, Fig. 1); without the flag the plain cell
    counts come back."""
    import ctypes as C

    from paper_1508_06561_gb300 import _lib
    from test_oracle_steps import trace_round
    rng = np.random.default_rng(77)
    db = synth.db_from_lengths(rng, np.concatenate([[0, 1, 3], synth.lognormal_lengths(rng, 300, 200, 0.7, 1, 3000)]))
    q = synth.residues(rng, 90)
    M = O.blosum62()
    for params, op in ((P.Params(), O.paper_params()),
                       (P.Params(rounds=2, lfactor_q16=50000), O.paper_params(rounds=2, lfactor_q16=50000))):
        D = P.Database(db.codes, db.offsets)
        tr = _lib.hs_trace()
        tr.pack_shifts = 1
        _lib.lib().hs_db_set_trace(D.handle, C.byref(tr))
        out = P.search_device(D, torch.from_numpy(q).cuda(), 5, params, seed=21, want_cells=True)
        torch.cuda.synchronize()
        packed = out["cells"].cpu().numpy()[: D.n]
        _lib.lib().hs_db_set_trace(D.handle, None)
        _, _, _, plain = run_device(D, q, 5, params, 21)
        for d in range(db.n):
            cells = shifts = 0
            for r in range(op.rounds):
                _, _, steps, c, _ = trace_round(q, db.seq(d), M, op, 21, d, r)
                cells += c
                shifts += sum(ls - ss + 1 for ls, ss, _ in steps)
            assert int(packed[d]) & ((1 << 40) - 1) == cells == int(plain[d])
            assert int(packed[d]) >> 40 == shifts
        D.close()
