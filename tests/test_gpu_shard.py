"""Sharded and threshold searches on the GPU.

Shards of one database (hs_db_load_shard, global indices), searched one by
one on the same GPU and merged on the host, must give exactly the hits and
alignments of the unsharded search; the threshold search (Sec. IV) must
return every pair at or above the threshold, ranked, as the oracle does."""
import numpy as np
import pytest

import oracle as O
import paper_1508_06561_gb300 as P
from paper_1508_06561_gb300 import shard, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_06561_gb300 import build
    build.build()
    O.build()


def test_shards_merge_to_the_unsharded_result():
    rng = np.random.default_rng(21)
    db = synth.db_from_lengths(rng, synth.lognormal_lengths(rng, 3000, 300, 0.6, 1, 9000))
    q = synth.residues(rng, 150)
    whole = P.Database(db.codes, db.offsets)
    for params, seed, k in [(P.Params(), 3, 40), (P.Params(pgp=2, rounds=2), 9, 200)]:
        h0, o0 = P.search(whole, q, k, params, seed)
        for nsh in [2, 3, 5]:
            S = shard.ShardedDatabase(db.codes, db.offsets, [0] * nsh)
            h1, o1 = S.search(q, k, params, seed)
            assert np.array_equal(h1, h0) and np.array_equal(o1, o0)
            # a hit's alignment from its own shard, by global index
            lo = [r[0] for r in S.ranges]
            d = int(h0[0]["db_index"])
            owner = S.shards[int(np.searchsorted(lo, d, side="right")) - 1]
            s, ops, _ = P.get_alignment(owner, q, d, params, seed)
            assert s == h0[0]["score"]
            assert ops.tolist() == o0[h0[0]["ops_offset"]:h0[0]["ops_offset"] + h0[0]["ops_len"]].tolist()
            S.close()
    whole.close()


def test_threshold_search_matches_oracle():
    rng = np.random.default_rng(5)
    db = synth.db_from_lengths(rng, synth.lognormal_lengths(rng, 2000, 250, 0.6, 1, 3000))
    q = synth.residues(rng, 80)
    D = P.Database(db.codes, db.offsets)
    ref, _, _ = O.search_scores(db.codes, db.offsets, q, O.blosum62(), O.paper_params(), 4)
    ranked = np.lexsort((np.arange(db.n), -ref))
    for thr in [int(np.percentile(ref, 99)), int(np.percentile(ref, 90)), int(ref.max()) + 1]:
        above = int((ref >= thr).sum())
        for max_hits in [5, 50, 4096]:
            hits, ops, n_above = P.search_threshold(D, q, thr, max_hits, seed=4)
            assert n_above == above
            want = ranked[:min(above, max_hits)]
            assert hits["db_index"].tolist() == want.tolist()
            assert (hits["score"] >= thr).all()
            assert sum(hits["ops_len"]) == len(ops)
            for h in hits[:5]:
                rq, rt = P.ops_to_rows(ops[h["ops_offset"]:h["ops_offset"] + h["ops_len"]], q, db.seq(h["db_index"]))
                assert O.score_rows(rq, rt, O.blosum62(), 0, 10, 5) == h["score"]
    S = shard.ShardedDatabase(db.codes, db.offsets, [0, 0])
    thr = int(np.percentile(ref, 95))
    h1, o1, a1 = S.search_threshold(q, thr, 4096, seed=4)
    h0, o0, a0 = P.search_threshold(D, q, thr, 4096, seed=4)
    assert a1 == a0 and np.array_equal(h1, h0) and np.array_equal(o1, o0)
    S.close()
    D.close()
