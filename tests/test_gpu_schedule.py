"""The scan's work schedule changes only speed: longest-first (length-binned)
and database-order schedules give identical results, for plain, batched
and full-slide searches, on a bimodal database like the load-balance
workload (most targets short, a tenth very long)."""
import numpy as np
import pytest

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


def test_schedules_agree():
    rng = np.random.default_rng(44)
    n = 3000
    long_ = rng.random(n) < 0.1
    lengths = np.where(long_, rng.integers(3000, 9000, n), rng.integers(50, 151, n))
    db = synth.db_from_lengths(rng, lengths)
    D = P.Database(db.codes, db.offsets)
    qs = [synth.residues(rng, L) for L in (50, 500, 2000)]
    res = {}
    for sched in (P.Database.SCHEDULE_LENGTH, P.Database.SCHEDULE_INPUT):
        D.set_schedule(sched)
        res[sched] = ([P.search(D, q, 50, seed=3) for q in qs],
                      P.search_batch(D, qs, 50, seeds=[3, 3, 3]),
                      P.search(D, qs[0], 20, P.Params(mode=1, rounds=2), seed=5))
    a, b = res[0], res[1]
    for (h0, o0), (h1, o1) in zip(a[0], b[0]):
        assert np.array_equal(h0, h1) and np.array_equal(o0, o1)
    for (h0, o0), (h1, o1) in zip(a[1], b[1]):
        assert np.array_equal(h0, h1) and np.array_equal(o0, o1)
    assert np.array_equal(a[2][0], b[2][0]) and np.array_equal(a[2][1], b[2][1])
    for (h0, _), (hb, _) in zip(a[0], a[1]):
        assert np.array_equal(h0, hb)
    D.close()


@pytest.mark.slow
def test_load_balance_workload_matches_oracle_under_both_schedules():
    """The load-balance workload itself (100k targets, 90% of 50-150 letters
    and 10% of 5,000-35,000; 16 queries of 50, 500 and 2,000 letters; top
    50): under the length-binned schedule and in database order, every
    pair's score and cell count, the ranked hits and every hit's alignment
    equal the oracle's, for the plain searches and for the batched search of
    all 16 queries (Sec. III.B.3 search, Fig. 1 per pair)."""
    import oracle as O
    from gpu_checks import check_hits, run_device
    O.build()
    db, qs, k = synth.bimodal()
    D = P.Database(db.codes, db.offsets)
    M, op = O.blosum62(), O.paper_params()
    seeds = [1000 + i for i in range(len(qs))]
    refs = [O.search_scores(db.codes, db.offsets, q, M, op, s) for q, s in zip(qs, seeds)]
    for sched in (P.Database.SCHEDULE_LENGTH, P.Database.SCHEDULE_INPUT):
        D.set_schedule(sched)
        batch = P.search_batch(D, qs, k, seeds=seeds)
        for i, (q, s) in enumerate(zip(qs, seeds)):
            ref, ref_cells, _ = refs[i]
            hits, ops, scores, cells = run_device(D, q, k, P.Params(), s)
            bad = np.nonzero(scores != ref)[0]
            assert len(bad) == 0, "schedule %d query %d: score mismatch at %s" % (sched, i, bad[:5])
            assert np.array_equal(cells, ref_cells)
            check_hits(db, q, M, op, s, hits, ops, ref, k)
            check_hits(db, q, M, op, s, batch[i][0], batch[i][1], ref, k)
    D.close()


def host_order(lengths):
    """The schedule the scan needs: longest first, equal lengths in database
    order (a stable sort of -length)."""
    return np.argsort(-np.asarray(lengths, np.int64), kind="stable")


def check_schedule(D, lengths):
    L = np.asarray(lengths, np.int64)
    order, cumres = D.schedule()
    want = host_order(L)
    assert np.array_equal(order, want)
    assert np.array_equal(cumres, np.concatenate([[0], np.cumsum(L[want])]))
    D.set_schedule(P.Database.SCHEDULE_INPUT)
    order, cumres = D.schedule()
    assert np.array_equal(order, np.arange(len(L))) and np.array_equal(cumres, np.concatenate([[0], np.cumsum(L)]))
    D.set_schedule(P.Database.SCHEDULE_LENGTH)
    order, _ = D.schedule()
    assert np.array_equal(order, want)


def test_length_order_is_built_on_the_device_and_stable():
    """The length-binned schedule comes from the device radix sort: it equals
    a stable host sort on the database-scale workload (570k sequences), on a
    database made almost only of ties, on lengths that need all three 8-bit
    digit passes (up to 300,000 letters), and on the degenerate cases."""
    db, _, _ = synth.plain_large()
    D = P.Database(db.codes, db.offsets)
    check_schedule(D, db.lengths())
    D.close()
    rng = np.random.default_rng(9)
    cases = [
        rng.choice([0, 1, 7, 300, 301, 2048], 50_000),                          # ties everywhere
        np.concatenate([rng.integers(0, 400, 20_000), [300_000, 65_536, 65_535, 256, 255, 300_000]]),
        np.zeros(10, np.int64),                                                  # all empty
        np.array([5]),
        np.array([], np.int64),
    ]
    for lengths in cases:
        d = synth.db_from_lengths(rng, lengths)
        D = P.Database(d.codes, d.offsets)
        check_schedule(D, d.lengths())
        if d.n:
            q = synth.residues(rng, 40)
            h0, o0 = P.search(D, q, 5, seed=2)
            D.set_schedule(P.Database.SCHEDULE_INPUT)
            h1, o1 = P.search(D, q, 5, seed=2)
            assert np.array_equal(h0, h1) and np.array_equal(o0, o1)
        D.close()
