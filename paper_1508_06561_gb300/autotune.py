"""Autotuner for the batched search's launch shape.

The batched scan's speed, never its results, depends on five knobs
(hs_batch_tuning):

* chunks -- chunks per query over the length-ordered database (fewer:
  less per-item overhead, longer tails; 0 lets the library pick one per ~256
  targets, at most 1024);
* warps -- warps per scan CTA, 24 or 12 (more warps hide more latency;
  fewer leave each warp more registers and the profile more room);
* flat_min_chunks, flat_max_iters -- which steps go to the flat unit list
  and which to a warp's lane grid (long narrow steps fill a pass badly as
  units, but the lane grid pays a whole warp for one step);
* long_len -- the length from which a target gets a warp to itself.

The tuner times the batch's own shape (a sample of its queries) with CUDA
events on the search stream, one knob at a time from the defaults
(coordinate descent, two sweeps), keeps the fastest and caches it per
database size, query-length class and GPU.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import Database, Params, search_batch_device

# chunks 0: the library's default (one chunk per ~256 targets, at most 1024)
DEFAULT = {"chunks": 0, "warps": 24, "flat_min_chunks": 16, "flat_max_iters": 128, "long_len": 2048}
SPACE = {
    "chunks": (256, 512, 1024, 2048, 4096),
    "warps": (24, 12),
    "flat_min_chunks": (8, 16, 32, 64),
    "flat_max_iters": (32, 64, 128, 256),
    "long_len": (1024, 2048, 4096, 8192),
}
_CACHE: dict = {}


def _key(db: Database, queries, k):
    import torch
    L = np.array([len(q) for q in queries])
    qclass = int(2 ** np.ceil(np.log2(max(int(L.max()), 1))))
    return "%s|n=%d|r=%d|qmax<=%d|k=%d" % (torch.cuda.get_device_name(), db.n, db.residues, qclass, k)


def tune(db: Database, queries, k: int, params: Params | None = None, sample: int = 8, reps: int = 2,
         sweeps: int = 2, space=None, cache_path: str | None = None, margin: float = 0.005):
    """Returns (best tuning dict, {candidate json: seconds}) for this batch shape."""
    import torch
    key = _key(db, queries, k)
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                _CACHE.update(json.load(f))
        except (OSError, ValueError):
            pass
    if key in _CACHE:
        return dict(_CACHE[key]), {}
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
    state = {"out": None, "ws": None}

    def timed(cand):
        name = json.dumps(cand, sort_keys=True)
        if name in times:
            return times[name]
        with torch.cuda.stream(st):
            state["out"] = search_batch_device(db, cat, offd, seeds, mq, k, params, cand, st, state["ws"],
                                               state["out"])     # warm-up
            state["ws"] = state["out"]["workspace"]
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                search_batch_device(db, cat, offd, seeds, mq, k, params, cand, st, state["ws"], state["out"])
            b.record(st)
        st.synchronize()
        times[name] = a.elapsed_time(b) / 1000.0 / reps
        return times[name]

    best = dict(DEFAULT)
    best_t = timed(best)
    for _ in range(sweeps):
        changed = False
        for knob, values in (space or SPACE).items():
            for v in values:
                cand = dict(best, **{knob: v})
                t = timed(cand)
                if t < best_t * (1.0 - margin):      # a real gain, not timing noise
                    best, best_t, changed = cand, t, True
        if not changed:
            break
    _CACHE[key] = best
    if cache_path:
        try:
            with open(cache_path, "w") as f:
                json.dump(_CACHE, f, indent=1)
        except OSError:
            pass
    return dict(best), times
