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
