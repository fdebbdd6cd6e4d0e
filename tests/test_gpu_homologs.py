"""The batched workload's planted homologs: 64 queries (lengths uniform in
30-1000) against the ~570k-sequence database in which 500 sequences are
query copies mutated to 20-40% identity with indels, embedded in background
flanks.  For every one of the 64 queries the oracle scores every pair, so
every GPU score and cell count, the rank of every planted homolog, the whole
top 100 and every hit's alignment must be the oracle's exactly -- from the
plain search and from the batched search of all 64 queries in one launch
(Sec. III.B.3 search, Fig. 1 per pair)."""
import numpy as np
import pytest

import oracle as O
import paper_1508_06561_gb300 as P
from paper_1508_06561_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")

from gpu_checks import check_hits, run_device  # noqa: E402


def rank_of(scores, d):
    s = scores[d]
    return int(np.sum(scores > s) + np.sum((scores == s) & (np.arange(len(scores)) < d)))


def test_all_64_queries_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_06561_gb300 import build
    build.build()
    O.build()
    db, queries, planted = synth.batched_homologs()
    D = P.Database(db.codes, db.offsets)
    k = 100
    seeds = np.arange(len(queries), dtype=np.uint64) + 11
    batch = P.search_batch(D, queries, k, seeds=seeds)
    by_query = {}
    for d, qi in planted.items():
        by_query.setdefault(qi, []).append(d)
    M, op = O.blosum62(), O.paper_params()
    checked = 0
    for qi, q in enumerate(queries):
        seed = int(seeds[qi])
        hits, ops, gpu, cells = run_device(D, q, k, P.Params(), seed)
        ref, ref_cells, _ = O.search_scores(db.codes, db.offsets, q, M, op, seed)
        bad = np.nonzero(gpu != ref)[0]
        assert len(bad) == 0, "query %d: score mismatch at %s" % (qi, bad[:5])
        assert np.array_equal(cells, ref_cells), "query %d: cell counts differ" % qi
        for d in by_query.get(qi, []):
            assert rank_of(gpu, d) == rank_of(ref, d)
            checked += 1
        check_hits(db, q, M, op, seed, hits, ops, ref, k)
        bh, bo = batch[qi]
        check_hits(db, q, M, op, seed, bh, bo, ref, k)
    assert checked == len(planted) == 500
    D.close()
