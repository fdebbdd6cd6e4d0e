"""Batched search (many queries, one persistent scan launch) on the GPU.

Every query's hits and alignments must be exactly those of the plain
single-query search with the same seed -- which the plain parity tests tie
to the oracle -- whatever the work split (chunks per query, CTAs per SM)."""
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


def uneven_queries(rng, n):
    lens = [1, 2, 5, 31, 64, 255, 256, 700, 2048] + list(rng.integers(30, 1001, max(0, n - 9)))
    return [synth.residues(rng, int(L)) for L in lens[:n]]


@pytest.mark.parametrize("tuning", [None, {"chunks": 1}, {"chunks": 7, "warps": 12}, {"chunks": 8192},
                                    {"flat_min_chunks": 1, "flat_max_iters": 1},
                                    {"flat_min_chunks": 100000, "flat_max_iters": 100000, "long_len": 1},
                                    {"warps": 12, "flat_min_chunks": 64, "flat_max_iters": 32, "long_len": 8192}])
def test_batch_equals_plain_per_query(tuning):
    rng = np.random.default_rng(77)
    lengths = np.concatenate([synth.lognormal_lengths(rng, 4000, 300, 0.6, 1, 4000), [0, 1, 6000, 2500]])
    db = synth.db_from_lengths(rng, lengths)
    D = P.Database(db.codes, db.offsets)
    qs = uneven_queries(rng, 12)
    seeds = rng.integers(0, 2**62, len(qs))
    params = P.Params(pgp=1, rounds=2)
    res = P.search_batch(D, qs, 25, params, seeds, tuning)
    for q, s, (h, o) in zip(qs, seeds, res):
        h0, o0 = P.search(D, q, 25, params, int(s))
        assert np.array_equal(h, h0) and np.array_equal(o, o0)
    D.close()


def test_batch_device_api_and_oracle_spot_check():
    rng = np.random.default_rng(3)
    db = synth.db_from_lengths(rng, synth.lognormal_lengths(rng, 1500, 250, 0.6, 1, 3000))
    D = P.Database(db.codes, db.offsets)
    qs = [synth.residues(rng, int(L)) for L in rng.integers(30, 600, 9)]
    seeds = np.arange(9, dtype=np.uint64) * 1000 + 1
    cat = np.concatenate(qs)
    off = np.zeros(10, np.int64)
    np.cumsum([len(q) for q in qs], out=off[1:])
    out = P.search_batch_device(D, torch.from_numpy(cat).cuda(), torch.from_numpy(off).cuda(),
                                torch.from_numpy(seeds.view(np.int64)).cuda(), int(max(len(q) for q in qs)), 10)
    torch.cuda.synchronize()
    assert int(out["status"].item()) == 0
    hits = np.frombuffer(out["hits"].cpu().numpy().tobytes(), dtype=P.HIT_DTYPE)
    ops = out["ops"].cpu().numpy().view(np.uint32)
    for i, q in enumerate(qs):
        h = hits[i * 10:(i + 1) * 10]
        ref, _, _ = O.search_scores(db.codes, db.offsets, q, O.blosum62(), O.paper_params(), int(seeds[i]))
        assert h["db_index"].tolist() == O.topk(ref, 10).tolist()
        x = h[0]
        rq, rt = P.ops_to_rows(ops[x["ops_offset"]:x["ops_offset"] + x["ops_len"]], q, db.seq(x["db_index"]))
        s, oq, ot, _, _ = O.align_pair(q, db.seq(x["db_index"]), O.blosum62(), O.paper_params(), int(seeds[i]),
                                       int(x["db_index"]))
        assert s == x["score"] and np.array_equal(rq, oq) and np.array_equal(rt, ot)
    D.close()
