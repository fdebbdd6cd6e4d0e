"""The allocation-free search entry point, hs_search_device_noalloc.

It exists for callers that cannot allocate device memory at search time (a
process whose memory manager reserved all device memory up front, a serving
loop that cannot afford cudaMalloc's synchronisation, a host that forbids
allocation after start-up).  It must give exactly what hs_search_device
gives, call after call, although every call reuses the same fixed scratch
area and finds the previous call's data in it.  The file name makes pytest
collect it last.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1508_06561_gb300 as P
from paper_1508_06561_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_06561_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return _lib.lib()


def fresh_outputs(n, qlen, k):
    nh = min(k, n)
    cap = _lib.lib().hs_ops_capacity(qlen, k)
    return {
        "hits": torch.zeros(max(nh, 1) * P.HIT_DTYPE.itemsize, dtype=torch.uint8, device="cuda"),
        "ops": torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda"),
        "ops_used": torch.zeros(1, dtype=torch.int64, device="cuda"),
        "status": torch.zeros(1, dtype=torch.int32, device="cuda"),
        "scores": torch.zeros(max(n, 1), dtype=torch.int32, device="cuda"),
        "cells": torch.zeros(max(n, 1), dtype=torch.int64, device="cuda"),
    }


def call_noalloc(L, D, qd, k, params, seed, out):
    p, _keep = params.to_c()
    st = torch.cuda.current_stream()
    rc = L.hs_search_device_noalloc(
        D.handle, qd.data_ptr(), int(qd.numel()), C.byref(p), k, seed, st.cuda_stream,
        out["hits"].data_ptr(), out["ops"].data_ptr(), int(out["ops"].numel()), out["ops_used"].data_ptr(),
        out["scores"].data_ptr(), out["cells"].data_ptr(), out["status"].data_ptr())
    return rc


def test_noalloc_matches_device_search_on_consecutive_calls(L):
    rng = np.random.default_rng(2024)
    db = synth.db_from_lengths(rng, synth.lognormal_lengths(rng, 5000, 300, 0.6, 1, 6000))
    D = P.Database(db.codes, db.offsets)
    cases = [(synth.residues(rng, 64), 10, 3, P.Params()),
             (synth.residues(rng, 300), 40, 4, P.Params(pgp=1, rounds=2)),
             (synth.residues(rng, 64), 10, 3, P.Params())]
    out = fresh_outputs(D.n, 300, 40)
    for q, k, seed, params in cases:                 # consecutive calls share the scratch
        qd = torch.from_numpy(q).cuda()
        ref = P.search_device(D, qd, k, params, seed=seed, want_scores=True, want_cells=True)
        torch.cuda.synchronize()
        ref_hits, ref_ops = P.device_result_to_host(ref)
        assert call_noalloc(L, D, qd, k, params, seed, out) == 0
        torch.cuda.synchronize()
        assert int(out["status"].item()) == 0
        nh = min(k, D.n)
        hits = np.frombuffer(out["hits"].cpu().numpy().tobytes(), dtype=P.HIT_DTYPE)[:nh]
        used = int(out["ops_used"].item())
        ops = out["ops"][:used].cpu().numpy().view(np.uint32)
        assert np.array_equal(hits, ref_hits)
        assert np.array_equal(ops, ref_ops)
        assert torch.equal(out["scores"][: D.n], ref["scores"][: D.n])
        assert torch.equal(out["cells"][: D.n], ref["cells"][: D.n])
    D.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(L):
    rng = np.random.default_rng(5)
    db = synth.db_from_lengths(rng, [100, 200, 300])
    D = P.Database(db.codes, db.offsets)
    qd = torch.from_numpy(synth.residues(rng, 2048)).cuda()
    need = P.workspace_size(D, 2048, 4096)
    assert need > _lib.HS_NOALLOC_SCRATCH_BYTES
    out = fresh_outputs(D.n, 64, 3)
    assert call_noalloc(L, D, qd, 4096, P.Params(), 0, out) == _lib.HS_ETRUNC
    D.close()
