"""Edges of the C ABI on the GPU: an empty database, query lengths at and
past the supported bounds, output and workspace buffers that are too small,
and bad parameters.  Every case must come back as a status code (never a
fault), and a too-small ops buffer must still leave the hits written."""
import ctypes as C

import numpy as np
import pytest

import paper_1508_06561_gb300 as P
from paper_1508_06561_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HS_EINVAL, HS_ETOOLONG, HS_ETRUNC = 1, 4, 6


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_06561_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def small_db():
    rng = np.random.default_rng(31)
    db = synth.db_from_lengths(rng, rng.integers(1, 300, 500))
    D = P.Database(db.codes, db.offsets)
    yield db, D
    D.close()


def status_of(fn, *args):
    try:
        fn(*args)
    except _lib.HsError as e:
        return e.status
    return 0


def test_empty_database():
    D = P.Database(np.zeros(0, np.uint8), np.zeros(1, np.int64))
    q = synth.residues(np.random.default_rng(1), 50)
    hits, ops = P.search(D, q, 10)
    assert len(hits) == 0 and len(ops) == 0
    res = P.search_batch(D, [q, q[:7]], 5)
    assert all(len(h) == 0 and len(o) == 0 for h, o in res)
    hits, ops, above = P.search_threshold(D, q, -1000, 10)
    assert len(hits) == 0 and above == 0
    assert status_of(P.get_alignment, D, q, 0) == HS_EINVAL
    D.close()


def test_query_length_bounds(small_db):
    db, D = small_db
    rng = np.random.default_rng(2)
    assert status_of(P.search, D, synth.residues(rng, 2049), 5) == HS_ETOOLONG
    assert status_of(P.search, D, np.zeros(0, np.uint8), 5) == HS_EINVAL
    hits, _ = P.search(D, synth.residues(rng, 1), 5)           # one-letter query
    assert len(hits) == 5


def test_bad_parameters_are_rejected(small_db):
    db, D = small_db
    q = synth.residues(np.random.default_rng(3), 40)
    assert status_of(P.search, D, q, 5, P.Params(gep=-1)) == HS_EINVAL
    assert status_of(P.search, D, q, 5, P.Params(rounds=0)) == HS_EINVAL
    assert status_of(P.search, D, q, 5, P.Params(gop=1001)) == HS_EINVAL
    assert status_of(P.search, D, q, 4097) == HS_EINVAL
    assert status_of(P.get_alignment, D, q, db.n) == HS_EINVAL


def test_small_ops_buffer_reports_trunc_and_keeps_hits(small_db):
    db, D = small_db
    q = synth.residues(np.random.default_rng(4), 120)
    want, _ = P.search(D, q, 8, seed=5)
    L = _lib.lib()
    p, _keep = P.Params().to_c()
    hits = np.zeros(8, P.HIT_DTYPE)
    nh = C.c_int32()
    ops = np.zeros(4, np.uint32)
    used = C.c_int64()
    rc = L.hs_search(D.handle, q.ctypes.data, len(q), C.byref(p), 8, 5, None, hits.ctypes.data, C.byref(nh),
                     ops.ctypes.data, len(ops), C.byref(used))
    assert rc == HS_ETRUNC
    assert nh.value == 8
    assert hits["db_index"].tolist() == want["db_index"].tolist()
    assert hits["score"].tolist() == want["score"].tolist()
    assert used.value > len(ops)


def test_small_workspace_is_rejected_before_launch(small_db):
    db, D = small_db
    L = _lib.lib()
    qlen, k = 64, 10
    q = torch.from_numpy(synth.residues(np.random.default_rng(6), qlen)).cuda()
    need = P.workspace_size(D, qlen, k)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    hits = torch.zeros(k * P.HIT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cap = L.hs_ops_capacity(qlen, k)
    ops = torch.zeros(cap, dtype=torch.int32, device="cuda")
    meta = torch.zeros(2, dtype=torch.int64, device="cuda")
    p, _keep = P.Params().to_c()

    def call(ws_bytes):
        return L.hs_search_device(D.handle, q.data_ptr(), qlen, C.byref(p), k, 0, None, ws.data_ptr(), ws_bytes,
                                  hits.data_ptr(), ops.data_ptr(), cap, meta.data_ptr(), None, None,
                                  meta.data_ptr() + 8)

    assert call(need - 1) == HS_ETRUNC
    assert call(need) == 0
    torch.cuda.synchronize()
    assert int(meta[1].item()) & 0xFFFFFFFF == 0


def test_bad_letter_codes_on_device_report_einval(small_db):
    """A device-resident query holding a code outside the 24-letter alphabet
    (the host cannot look at it) comes back as HS_EINVAL in the status word
    of every device entry point, reads nothing out of range, and leaves the
    context usable: the next search of a good query equals the host search."""
    db, D = small_db
    rng = np.random.default_rng(9)
    good = synth.residues(rng, 40)
    for bad_code in (24, 65, 255):
        q = good.copy()
        q[17] = bad_code
        qd = torch.from_numpy(q).cuda()
        out = P.search_device(D, qd, 5)
        torch.cuda.synchronize()
        assert int(out["status"].item()) == HS_EINVAL
        P.search_device_noalloc(D, qd, 5, out)
        torch.cuda.synchronize()
        assert int(out["status"].item()) == HS_EINVAL
        cat = torch.from_numpy(np.concatenate([good, q])).cuda()
        off = torch.tensor([0, len(good), 2 * len(good)], dtype=torch.int64, device="cuda")
        seeds = torch.zeros(2, dtype=torch.int64, device="cuda")
        bo = P.search_batch_device(D, cat, off, seeds, len(good), 5)
        torch.cuda.synchronize()
        assert int(bo["status"].item()) == HS_EINVAL
    out = P.search_device(D, torch.from_numpy(good).cuda(), 5)
    torch.cuda.synchronize()
    hits, ops = P.device_result_to_host(out)
    hh, ho = P.search(D, good, 5)
    assert np.array_equal(hits, hh) and np.array_equal(ops, ho)
