"""Database sharding: one contiguous, residue-balanced range of sequences per
GPU, each searched on its own, then one exchange -- the k best (score,
index) records of every shard -- merged on the host.

Pairs are independent (Sec. III.B.3: one query against every sequence), and
a shard keeps the global database indices of its sequences (hs_db_load_shard),
so every pair draws the same random numbers as in a single-GPU search and the
merge by (score desc, index asc) reproduces the unsharded top k exactly.
Alignments come from the shard that owns the hit.
"""
from __future__ import annotations

import numpy as np

from . import HIT_DTYPE, Database, Params, device_result_to_host, search, search_device, search_threshold


def split_offsets(offsets, nshards: int):
    """Contiguous sequence ranges [(lo, hi), ...] with about equal residues."""
    offsets = np.asarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    total = int(offsets[-1])
    cuts = [0]
    for s in range(1, nshards):
        c = int(np.searchsorted(offsets, total * s / nshards, side="left"))
        cuts.append(min(max(c, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[i], cuts[i + 1]) for i in range(nshards)]


def shard_arrays(codes, offsets, lo: int, hi: int):
    """(codes, offsets rebased to 0, index_base) of sequences [lo, hi)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    a, b = int(offsets[lo]), int(offsets[hi])
    return np.asarray(codes[a:b]), offsets[lo:hi + 1] - a, lo


def merge_ranked(scores_list, index_list, k: int):
    """Merge per-shard ranked lists: the k best by (score desc, index asc).
    Returns (positions, scores, indices) where positions index the
    concatenation of the inputs."""
    scores = np.concatenate([np.asarray(s, dtype=np.int64) for s in scores_list]) if scores_list else np.zeros(0, np.int64)
    index = np.concatenate([np.asarray(x, dtype=np.int64) for x in index_list]) if index_list else np.zeros(0, np.int64)
    order = np.lexsort((index, -scores))[:k]
    return order, scores[order], index[order]


def merge_hits(parts, k: int):
    """parts: [(hits, ops), ...] from each shard (global db_index).  Returns
    the merged (hits, ops) with ops offsets rewritten for the new buffer."""
    if not parts:
        return np.zeros(0, HIT_DTYPE), np.zeros(0, np.uint32)
    hits_all = np.concatenate([h for h, _ in parts])
    owner = np.concatenate([np.full(len(h), i) for i, (h, _) in enumerate(parts)])
    order, _, _ = merge_ranked([hits_all["score"]], [hits_all["db_index"]], k)
    out = hits_all[order].copy()
    ops_out, off = [], 0
    for j, pos in enumerate(order):
        h = hits_all[pos]
        seg = parts[owner[pos]][1][h["ops_offset"]:h["ops_offset"] + h["ops_len"]]
        out[j]["ops_offset"] = off
        ops_out.append(seg)
        off += len(seg)
    ops = np.concatenate(ops_out) if ops_out else np.zeros(0, np.uint32)
    return out, ops.astype(np.uint32)


class ShardedDatabase:
    """A database split over several devices (or several handles on one).

    devices: CUDA device ordinals, one shard each."""

    def __init__(self, codes, offsets, devices):
        import torch
        self.devices = list(devices)
        self.ranges = split_offsets(offsets, len(self.devices))
        self.shards, self.streams = [], []
        self._bufs = [None] * len(self.devices)      # per shard: device buffers of the last search
        prev = torch.cuda.current_device()
        try:
            for dev, (lo, hi) in zip(self.devices, self.ranges):
                torch.cuda.set_device(dev)
                c, o, base = shard_arrays(codes, offsets, lo, hi)
                self.shards.append(Database(c, o, index_base=base))
                self.streams.append(torch.cuda.Stream(dev))
        finally:
            torch.cuda.set_device(prev)
        self.n = sum(s.n for s in self.shards)

    def search(self, query, k: int, params: Params | None = None, seed: int = 0):
        """Every shard's search is enqueued on its own stream (and device)
        before any is waited for, so the shards run at the same time; then
        the k best records are merged on the host."""
        import torch
        q = np.ascontiguousarray(query, dtype=np.uint8)
        qh = torch.from_numpy(q).pin_memory()
        prev = torch.cuda.current_device()
        outs = []
        try:
            for i, (dev, db, st) in enumerate(zip(self.devices, self.shards, self.streams)):
                torch.cuda.set_device(dev)
                with torch.cuda.stream(st):
                    qd = qh.to(torch.device("cuda", dev), non_blocking=True)
                    b = self._bufs[i]
                    fits = b is not None and b["k"] == k and b["qlen"] == len(q)
                    out = search_device(db, qd, k, params, seed, stream=st,
                                        workspace=b["out"]["workspace"] if fits else None,
                                        out=b["out"] if fits else None)
                    self._bufs[i] = {"k": k, "qlen": len(q), "out": out, "q": qd}
                outs.append(out)
            parts = []
            for dev, st, out in zip(self.devices, self.streams, outs):
                torch.cuda.set_device(dev)
                st.synchronize()
                parts.append(device_result_to_host(out))
        finally:
            torch.cuda.set_device(prev)
        return merge_hits(parts, k)

    def search_threshold(self, query, threshold: int, max_hits: int, params: Params | None = None, seed: int = 0):
        """One host thread per shard (the library call releases the GIL), so
        the shards' searches run at the same time; then the merge."""
        import concurrent.futures as cf

        import torch

        def one(i):
            torch.cuda.set_device(self.devices[i])
            return search_threshold(self.shards[i], query, threshold, max_hits, params, seed, stream=self.streams[i])

        with cf.ThreadPoolExecutor(len(self.shards)) as ex:
            res = list(ex.map(one, range(len(self.shards))))
        hits, ops = merge_hits([(h, o) for h, o, _ in res], max_hits)
        return hits, ops, sum(a for _, _, a in res)

    def close(self):
        for s in self.shards:
            s.close()


def search_distributed(local_db: Database, query, k: int, params: Params | None = None, seed: int = 0, group=None):
    """One shard per rank: every rank searches its shard, the k best records
    (with their alignments) are gathered to every rank and merged."""
    import torch.distributed as dist
    part = search(local_db, query, k, params, seed)
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, (part[0].tobytes(), part[1]), group=group)
    parts = [(np.frombuffer(h, dtype=HIT_DTYPE), o) for h, o in parts]
    return merge_hits(parts, k)
