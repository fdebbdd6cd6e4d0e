"""Failure paths without a GPU fault: with HS_FAIL_ALLOC set, every
allocation the library makes is refused (host-side injection).  Loading a
database and the first search that needs buffers must then return
HS_ENOMEM, release what they took, and work again once allocations are
allowed -- with the same results as an untouched database."""
import os

import numpy as np
import pytest

import paper_1508_06561_gb300 as P
from paper_1508_06561_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HS_ENOMEM = 2


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_06561_gb300 import build
    build.build()
    torch.cuda.set_device(0)


class refused:
    def __enter__(self):
        os.environ["HS_FAIL_ALLOC"] = "1"

    def __exit__(self, *exc):
        del os.environ["HS_FAIL_ALLOC"]


def status_of(fn, *args):
    try:
        fn(*args)
    except _lib.HsError as e:
        return e.status
    return 0


def test_refused_allocations_and_recovery():
    rng = np.random.default_rng(41)
    db = synth.db_from_lengths(rng, rng.integers(1, 400, 800))
    q = synth.residues(rng, 90)
    with refused():
        assert status_of(P.Database, db.codes, db.offsets) == HS_ENOMEM
    D = P.Database(db.codes, db.offsets)
    with refused():
        assert status_of(P.search, D, q, 7, None, 3) == HS_ENOMEM            # buffers are made on first use
        assert status_of(P.search_batch, D, [q, q[:40]], 7) == HS_ENOMEM
    hits, ops = P.search(D, q, 7, seed=3)
    D2 = P.Database(db.codes, db.offsets)
    h2, o2 = P.search(D2, q, 7, seed=3)
    assert np.array_equal(hits, h2) and np.array_equal(ops, o2)
    res = P.search_batch(D, [q, q[:40]], 7, seeds=[3, 4])
    assert np.array_equal(res[0][0], h2)
    D.close()
    D2.close()
