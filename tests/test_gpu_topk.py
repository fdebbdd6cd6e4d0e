"""Ranking of the scanned pairs (score descending, database index ascending)
on the GPU, for the score distributions that take the selection's different
paths: many equal scores (ties at the k-th score), slices holding fewer keys
than k, score ranges needing more than one histogram pass, and more
candidates than the final sort holds.  Scores are checked against the
oracle on small databases and the ranking against the GPU's own score array
at database scale."""
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


def ranked(scores, k):
    return np.lexsort((np.arange(len(scores)), -np.asarray(scores)))[:k]


def test_ties_and_short_slices():
    """4,000 targets, most of them copies of four sequences (so thousands of
    equal scores); k from 1 to beyond a slice's size."""
    rng = np.random.default_rng(21)
    base = [synth.residues(rng, L) for L in (40, 90, 150, 60)]
    seqs = []
    for i in range(4000):
        seqs.append(base[i % 4] if rng.random() < 0.8 else synth.residues(rng, int(rng.integers(5, 200))))
    lengths = [len(s) for s in seqs]
    offsets = np.zeros(len(seqs) + 1, np.int64)
    np.cumsum(lengths, out=offsets[1:])
    codes = np.concatenate(seqs).astype(np.uint8)
    q = synth.residues(rng, 70)
    ref, _, _ = O.search_scores(codes, offsets, q, O.blosum62(), O.paper_params(), 9)
    assert len(np.unique(ref)) < len(ref) // 4          # many ties
    D = P.Database(codes, offsets)
    for k in (1, 10, 26, 27, 100, 500, 4000):
        hits, _ = P.search(D, q, k, seed=9)
        assert hits["db_index"].tolist() == O.topk(ref, k).tolist(), k
        assert hits["score"].tolist() == ref[O.topk(ref, k)].tolist()
    D.close()


def test_wide_score_range():
    """Scores spanning more than 4096 values (near-copies of a 1,500-residue
    query among random targets): the threshold takes two digit passes."""
    rng = np.random.default_rng(22)
    q = synth.residues(rng, 1500)
    seqs = [synth.residues(rng, int(rng.integers(20, 400))) for _ in range(1500)]
    for i in range(0, 1500, 100):
        seqs[i] = synth.mutate_homolog(rng, q, identity=0.5 + 0.03 * (i // 100))
    lengths = [len(s) for s in seqs]
    offsets = np.zeros(len(seqs) + 1, np.int64)
    np.cumsum(lengths, out=offsets[1:])
    codes = np.concatenate(seqs).astype(np.uint8)
    ref, _, _ = O.search_scores(codes, offsets, q, O.blosum62(), O.paper_params(), 4)
    assert ref.max() - ref.min() >= 4096
    D = P.Database(codes, offsets)
    for k in (5, 15, 16, 40):
        hits, _ = P.search(D, q, k, seed=4)
        assert hits["db_index"].tolist() == O.topk(ref, k).tolist(), k
    D.close()


@pytest.mark.parametrize("k", [100, 3000, 4096])
def test_database_scale_large_k(k):
    """The 570k-target database: k = 3000 leaves more candidates above the
    slices' bound than the final sort holds; k = 4096 exceeds every slice."""
    db, q, _ = synth.plain_large()
    D = P.Database(db.codes, db.offsets)
    qd = torch.from_numpy(q).cuda()
    out = P.search_device(D, qd, k, P.Params(), seed=1, want_scores=True)
    torch.cuda.synchronize()
    hits, _ = P.device_result_to_host(out)
    scores = out["scores"].cpu().numpy()[: D.n].astype(np.int64)
    want = ranked(scores, k)
    assert hits["db_index"].tolist() == want.tolist()
    assert hits["score"].tolist() == scores[want].tolist()
    D.close()
