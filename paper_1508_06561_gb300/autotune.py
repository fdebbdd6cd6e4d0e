"""Autotuner for the batched search's launch shape.

The batched scan splits the length-ordered database into `chunks` work items
per query and runs `ctas_per_sm` resident CTAs per SM.  Results never depend
on either; speed does (fewer chunks: less per-item overhead, longer tails;
more CTAs: more warps to hide latency, less shared memory each).  The tuner
times every candidate on a sample of the batch's queries with CUDA events on
the search stream and keeps the fastest, caching the choice per database
size, query-length class and GPU.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import Database, Params, search_batch_device

CANDIDATES = [{"chunks": c, "ctas_per_sm": t} for c in (256, 1024, 4096) for t in (0, 1)]
_CACHE: dict = {}


def _key(db: Database, queries, k):
    import torch
    L = np.array([len(q) for q in queries])
    qclass = int(2 ** np.ceil(np.log2(max(int(L.max()), 1))))
    return "%s|n=%d|r=%d|qmax<=%d|k=%d" % (torch.cuda.get_device_name(), db.n, db.residues, qclass, k)


def tune(db: Database, queries, k: int, params: Params | None = None, sample: int = 8, reps: int = 2,
         candidates=None, cache_path: str | None = None):
    """Returns (best tuning dict, {candidate: seconds}) for this batch shape."""
    import torch
    key = _key(db, queries, k)
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                _CACHE.update(json.load(f))
        except (OSError, ValueError):
            pass
    if key in _CACHE:
        return _CACHE[key], {}
    rng = np.random.default_rng(0)
    pick = rng.choice(len(queries), min(sample, len(queries)), replace=False)
    qs = [np.asarray(queries[i], dtype=np.uint8) for i in pick]
    cat = torch.from_numpy(np.concatenate(qs)).cuda()
    off = np.zeros(len(qs) + 1, np.int64)
    np.cumsum([len(q) for q in qs], out=off[1:])
    offd = torch.from_numpy(off).cuda()
    seeds = torch.zeros(len(qs), dtype=torch.int64, device="cuda")
    mq = int(max(len(q) for q in qs))
    st = torch.cuda.Stream()
    times = {}
    out = None
    ws = None
    for cand in candidates or CANDIDATES:
        with torch.cuda.stream(st):
            out = search_batch_device(db, cat, offd, seeds, mq, k, params, cand, st, ws, out)   # warm
            ws = out["workspace"]
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                search_batch_device(db, cat, offd, seeds, mq, k, params, cand, st, ws, out)
            b.record(st)
        st.synchronize()
        times[json.dumps(cand, sort_keys=True)] = a.elapsed_time(b) / 1000.0 / reps
    best = json.loads(min(times, key=times.get))
    _CACHE[key] = best
    if cache_path:
        try:
            with open(cache_path, "w") as f:
                json.dump(_CACHE, f, indent=1)
        except OSError:
            pass
    return best, times
