"""Checks shared by the GPU tests: run a search through the C ABI with every
pair's score and cell count, and compare ranked hits and their alignments
with the oracle (Sec. III.B.3 search, Fig. 1 per pair)."""
import numpy as np
import torch

import oracle as O
import paper_1508_06561_gb300 as P


def oparams(p: P.Params):
    return O.paper_params(pgp=p.pgp, gop=p.gop, gep=p.gep, rounds=p.rounds, lfactor_q16=p.lfactor_q16,
                          sfactor_q16=p.sfactor_q16, minfactor_q16=p.minfactor_q16)


def run_device(D, q, k, params, seed):
    qd = torch.from_numpy(np.ascontiguousarray(q, np.uint8)).cuda()
    out = P.search_device(D, qd, k, params, seed=seed, want_scores=True, want_cells=True)
    torch.cuda.synchronize()
    hits, ops = P.device_result_to_host(out)
    scores = out["scores"].cpu().numpy()[: D.n].astype(np.int64)
    cells = out["cells"].cpu().numpy()[: D.n]
    return hits, ops, scores, cells


def check_hits(db, q, M, op, seed, hits, ops, ref_scores, k):
    want = O.topk(ref_scores, k)
    assert hits["db_index"].tolist() == want.tolist()
    assert hits["score"].tolist() == ref_scores[want].tolist()
    for h in hits:
        t = db.seq(int(h["db_index"]))
        seg = ops[h["ops_offset"]:h["ops_offset"] + h["ops_len"]]
        rq, rt = P.ops_to_rows(seg, q, t)
        s, oq, ot, _, _ = O.align_pair(q, t, M, op, seed, int(h["db_index"]))
        assert s == h["score"]
        assert np.array_equal(rq, oq) and np.array_equal(rt, ot)
        assert O.score_rows(rq, rt, M, op.pgp, op.gop, op.gep) == h["score"]
        m = (rq != 255) & (rt != 255)
        if m.any():
            cols = np.nonzero(m)[0]
            qpos = np.cumsum(rq != 255) - 1
            tpos = np.cumsum(rt != 255) - 1
            assert (h["q_begin"], h["q_end"]) == (qpos[cols[0]], qpos[cols[-1]] + 1)
            assert (h["t_begin"], h["t_end"]) == (tpos[cols[0]], tpos[cols[-1]] + 1)
