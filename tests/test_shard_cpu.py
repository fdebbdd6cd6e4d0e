"""Host side of database sharding (no GPU): the residue-balanced split, the
ranked merge, and a two-rank gloo run in which each rank scores its shard
with the oracle (draws keyed by global index), the k best are gathered and
merged, and the result must equal the unsharded oracle ranking."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1508_06561_gb300 import shard, synth


def test_split_is_contiguous_and_balanced():
    rng = np.random.default_rng(0)
    lengths = synth.lognormal_lengths(rng, 5000, 300, 0.6, 1, 35000)
    off = synth.offsets_from_lengths(lengths)
    for s in [1, 2, 3, 8]:
        r = shard.split_offsets(off, s)
        assert r[0][0] == 0 and r[-1][1] == len(lengths)
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        res = [off[hi] - off[lo] for lo, hi in r]
        assert max(res) - min(res) <= 2 * lengths.max()


def test_merge_ranked_equals_global_sort():
    rng = np.random.default_rng(1)
    scores = rng.integers(-50, 50, 1000)
    idx = np.arange(1000)
    cuts = [0, 300, 301, 1000]
    parts_s, parts_i = [], []
    for a, b in zip(cuts, cuts[1:]):
        top = np.lexsort((idx[a:b], -scores[a:b]))[:20]
        parts_s.append(scores[a:b][top]); parts_i.append(idx[a:b][top])
    _, ms, mi = shard.merge_ranked(parts_s, parts_i, 20)
    want = np.lexsort((idx, -scores))[:20]
    assert mi.tolist() == want.tolist() and ms.tolist() == scores[want].tolist()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(42)
    db = synth.db_from_lengths(rng, synth.lognormal_lengths(rng, 400, 200, 0.6, 1, 2000))
    qs = synth.residues(rng, 60)
    lo, hi = shard.split_offsets(db.offsets, world)[rank]
    idx = np.arange(lo, hi)
    s, _, _ = O.search_scores(db.codes, db.offsets, qs, O.blosum62(), O.paper_params(), 7, idx=idx, nthreads=2)
    top = O.topk(s, 15)
    parts = [None] * world
    dist.all_gather_object(parts, (s[top].tolist(), idx[top].tolist()))
    _, ms, mi = shard.merge_ranked([p[0] for p in parts], [p[1] for p in parts], 15)
    if rank == 0:
        full, _, _ = O.search_scores(db.codes, db.offsets, qs, O.blosum62(), O.paper_params(), 7, nthreads=2)
        want = O.topk(full, 15)
        q.put((mi.tolist() == want.tolist(), ms.tolist() == full[want].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_merge_equals_unsharded():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs)
    same_idx, same_scores = q.get(timeout=10)
    assert same_idx and same_scores
