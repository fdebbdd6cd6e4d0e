"""Serving: continuous batching of search requests against a resident database.

Requests (a query and its seed) arrive at any time and wait in a FIFO queue.
The server owns `slots` CUDA streams, each with device buffers allocated once
at start-up (workspace, queries, hits, ops).  Whenever a slot is free, the
scheduler admits requests from the head of the queue into a batch as long as
the batch's device memory need (hs_search_batch_workspace_size and the
query/ops buffers) fits the slot's budget and the batch has at most
`max_batch` queries, then launches the batched search on that slot's stream.
Requests that arrive while other batches run are admitted as soon as a slot
and its memory free up, and several batches overlap on the device.  A batch
of one query (the common case at low load) runs the plain search entry point
on the slot's buffers instead: its scan is faster for a single query.  Results
are the same as a search of the query alone with the same seed (every pair's
random draws are keyed by its database index, never by its batch), which the
tests check.

Latency is measured from submit() to the moment the result is ready on the
host.
"""
from __future__ import annotations

import ctypes as C
import threading
import time
from collections import deque
from concurrent.futures import Future

import numpy as np

from . import HIT_DTYPE, Database, Params, _lib, _tuning, check, lib


class _Req:
    __slots__ = ("query", "seed", "future", "t_submit", "t_done")

    def __init__(self, query, seed):
        self.query = np.ascontiguousarray(query, dtype=np.uint8)
        self.seed = int(seed) & (2**64 - 1)
        self.future = Future()
        self.t_submit = time.perf_counter()
        self.t_done = None


class _Slot:
    def __init__(self, db, k, max_batch, max_qlen, max_total_qlen, device):
        import torch
        self.stream = torch.cuda.Stream(device)
        b = C.c_size_t()
        check(lib().hs_search_batch_workspace_size(db.handle, max_batch, max_total_qlen, max_qlen, k, C.byref(b)),
              "hs_search_batch_workspace_size")
        self.ws_bytes = b.value
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.ops_cap = lib().hs_batch_ops_capacity(max_batch, max_total_qlen, k)
        self.d_q = torch.empty(max_total_qlen, dtype=torch.uint8, device=device)
        self.d_off = torch.empty(max_batch + 1, dtype=torch.int64, device=device)
        self.d_seed = torch.empty(max_batch, dtype=torch.int64, device=device)
        self.d_hits = torch.empty(max_batch * k * HIT_DTYPE.itemsize, dtype=torch.uint8, device=device)
        self.d_ops = torch.empty(max(self.ops_cap, 1), dtype=torch.int32, device=device)
        self.d_meta = torch.zeros(2, dtype=torch.int64, device=device)          # ops_used, status
        self.h_q = torch.empty(max_total_qlen, dtype=torch.uint8, pin_memory=True)
        self.h_off = torch.empty(max_batch + 1, dtype=torch.int64, pin_memory=True)
        self.h_seed = torch.empty(max_batch, dtype=torch.int64, pin_memory=True)
        self.h_hits = torch.empty(max_batch * k * HIT_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        self.h_meta = torch.zeros(2, dtype=torch.int64, pin_memory=True)
        self.event = torch.cuda.Event()
        # device-time bounds of the batch in flight (for the overlap record)
        self.ev_start = torch.cuda.Event(enable_timing=True)
        self.ev_end = torch.cuda.Event(enable_timing=True)
        self.batch = None


class Server:
    """Continuous-batching search server on one GPU.

    k: hits per request; params: shared search parameters; max_batch: most
    queries per launch; slots: launches in flight (CUDA streams);
    max_total_qlen: per-slot budget of query letters, which with max_batch
    and k sizes each slot's device memory (the admission gate); None sizes
    it from free device memory at start-up: the largest budget whose slot
    buffers, one per slot, fit `memory_fraction` of the free memory."""

    def __init__(self, db: Database, k: int = 100, params: Params | None = None, max_batch: int = 64,
                 slots: int = 2, max_qlen: int = 2048, max_total_qlen: int | None = 32768, tuning=None, device=None,
                 memory_fraction: float = 0.5):
        import torch
        if max_total_qlen is None:
            dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
            free, _ = torch.cuda.mem_get_info(dev)
            max_total_qlen = slot_budget(db, k, max_batch, max_qlen, free * memory_fraction / max(slots, 1))
        if max_total_qlen < max_qlen:
            raise ValueError("max_total_qlen (%d) must be at least max_qlen (%d): a request of max_qlen letters "
                             "must fit a batch alone" % (max_total_qlen, max_qlen))
        self.db, self.k, self.params = db, k, params or Params()
        self.max_batch, self.max_qlen, self.max_total = max_batch, max_qlen, max_total_qlen
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.tuning = _tuning(tuning)
        self._p, self._keep = self.params.to_c()
        self.slots = [_Slot(db, k, max_batch, max_qlen, max_total_qlen, self.device) for _ in range(slots)]
        self.queue: deque = deque()
        self.cv = threading.Condition()
        self.running = True
        self.batches = []                       # (queries, letters) of every batch launched
        self.latencies = []                     # seconds from submit to result, per request
        self.errors = []
        self.cancelled = 0                      # requests dropped because their caller cancelled them
        self.intervals = []                     # (start, end) of every batch on the device, ms from t_ref
        self.t_ref = torch.cuda.Event(enable_timing=True)
        self.t_ref.record(torch.cuda.current_stream(self.device))
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    # ------------------------------------------------------------------
    def submit(self, query, seed: int = 0) -> Future:
        q = np.asarray(query)
        if q.ndim != 1 or len(q) < 1 or len(q) > self.max_qlen:
            raise ValueError("query length must be in [1, %d]" % self.max_qlen)
        if q.dtype.kind not in "ui" or int(q.min()) < 0 or int(q.max()) >= 24:
            raise ValueError("query letters must be alphabet codes 0..23 (see encode())")
        r = _Req(q, seed)
        with self.cv:
            self.queue.append(r)
            self.cv.notify()
        return r.future

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify()
        self.thread.join()

    # ------------------------------------------------------------------
    def _fits(self, nq, total, mq):
        if nq > self.max_batch or total > self.max_total or mq > self.max_qlen:
            return False
        b = C.c_size_t()
        if lib().hs_search_batch_workspace_size(self.db.handle, nq, total, mq, self.k, C.byref(b)) != 0:
            return False
        return b.value <= self.slots[0].ws_bytes

    def _admit(self):
        """Requests from the head of the queue that fit one slot's memory;
        requests their callers cancelled are dropped here."""
        batch, total, mq = [], 0, 0
        with self.cv:
            while self.queue:
                r = self.queue[0]
                if r.future.cancelled():
                    self.queue.popleft()
                    self.cancelled += 1
                    continue
                L = len(r.query)
                if not self._fits(len(batch) + 1, total + L, max(mq, L)):
                    if batch:
                        break
                    # it does not fit even alone: fail it rather than stall the queue
                    self.queue.popleft()
                    if r.future.set_running_or_notify_cancel():
                        r.future.set_exception(ValueError("request does not fit one slot's device memory"))
                    else:
                        self.cancelled += 1
                    continue
                self.queue.popleft()
                if not r.future.set_running_or_notify_cancel():     # cancelled just now
                    self.cancelled += 1
                    continue
                batch.append(r)
                total += L
                mq = max(mq, L)
        return batch, total, mq

    def _plain_fits(self, s: _Slot, qlen):
        b = C.c_size_t()
        if lib().hs_search_workspace_size(self.db.handle, qlen, self.k, C.byref(b)) != 0:
            return False
        return b.value <= s.ws_bytes and lib().hs_ops_capacity(qlen, self.k) <= s.ops_cap

    def _launch(self, s: _Slot, batch, total, mq):
        import torch
        nq = len(batch)
        off = np.zeros(nq + 1, np.int64)
        np.cumsum([len(r.query) for r in batch], out=off[1:])
        s.h_q[:total].copy_(torch.from_numpy(np.concatenate([r.query for r in batch])))
        s.h_off[:nq + 1].copy_(torch.from_numpy(off))
        s.h_seed[:nq].copy_(torch.from_numpy(np.array([r.seed for r in batch], dtype=np.uint64).view(np.int64)))
        with torch.cuda.stream(s.stream):
            s.ev_start.record(s.stream)
            s.d_q[:total].copy_(s.h_q[:total], non_blocking=True)
            s.d_off[:nq + 1].copy_(s.h_off[:nq + 1], non_blocking=True)
            s.d_seed[:nq].copy_(s.h_seed[:nq], non_blocking=True)
            meta = s.d_meta.data_ptr()
            if nq == 1 and self._plain_fits(s, total):
                check(lib().hs_search_device(
                    self.db.handle, s.d_q.data_ptr(), total, C.byref(self._p), self.k, batch[0].seed,
                    s.stream.cuda_stream, s.ws.data_ptr(), s.ws_bytes, s.d_hits.data_ptr(), s.d_ops.data_ptr(),
                    lib().hs_ops_capacity(total, self.k), meta, None, None, meta + 8), "hs_search_device")
            else:
                cap = lib().hs_batch_ops_capacity(nq, total, self.k)
                check(lib().hs_search_batch_device(
                    self.db.handle, nq, s.d_q.data_ptr(), s.d_off.data_ptr(), s.d_seed.data_ptr(), total, mq,
                    C.byref(self._p), self.k, C.byref(self.tuning) if self.tuning is not None else None,
                    s.stream.cuda_stream, s.ws.data_ptr(), s.ws_bytes, s.d_hits.data_ptr(), s.d_ops.data_ptr(),
                    cap, meta, meta + 8), "hs_search_batch_device")
            nh = min(self.k, self.db.n)
            nbytes = nq * self.k * HIT_DTYPE.itemsize
            s.h_hits[:nbytes].copy_(s.d_hits[:nbytes], non_blocking=True)
            s.h_meta.copy_(s.d_meta, non_blocking=True)
            s.ev_end.record(s.stream)
            s.event.record(s.stream)
        s.batch = (batch, nq, nh)
        self.batches.append((nq, total))

    def _harvest(self, s: _Slot):
        batch = s.batch[0]
        s.batch = None
        ref = getattr(self, "t_ref", None)
        if ref is not None:
            try:
                self.intervals.append((ref.elapsed_time(s.ev_start), ref.elapsed_time(s.ev_end)))
            except RuntimeError:            # timing unavailable: the record is informational only
                pass
        try:
            self._deliver(s, batch)
        except Exception as e:
            # every caller of the batch learns of the failure; none waits forever
            self.errors.append(e)
            for r in batch:
                if not r.future.done():
                    r.future.set_exception(e)

    def _deliver(self, s: _Slot, batch):
        import torch
        nq, nh = len(batch), min(self.k, self.db.n)
        used = int(s.h_meta[0].item())
        status = int(s.h_meta[1].item()) & 0xFFFFFFFF
        if status != 0:
            err = _lib.HsError(status, "batched search (device status)")
            for r in batch:
                r.future.set_exception(err)
            return
        ops = np.zeros(0, np.uint32)
        if used > 0 and nh > 0:
            with torch.cuda.stream(s.stream):
                ops = s.d_ops[:used].cpu().numpy().view(np.uint32)
        hits = np.frombuffer(s.h_hits[:nq * self.k * HIT_DTYPE.itemsize].numpy().tobytes(), dtype=HIT_DTYPE)
        now = time.perf_counter()
        for i, r in enumerate(batch):
            h = hits[i * self.k:i * self.k + nh].copy()
            # the replay packs every query's ops contiguously, in hit order
            if nh > 0:
                first = int(h["ops_offset"][0])
                end = int(h["ops_offset"][-1] + h["ops_len"][-1])
                o = ops[first:end].astype(np.uint32)
                h["ops_offset"] -= first
            else:
                o = np.zeros(0, np.uint32)
            r.t_done = now
            self.latencies.append(now - r.t_submit)
            r.future.set_result((h, o))

    def _loop(self):
        import torch
        torch.cuda.set_device(self.device)
        while True:
            progressed = False
            for s in self.slots:
                if s.batch is not None and s.event.query():
                    self._harvest(s)
                    progressed = True
            for s in self.slots:
                if s.batch is None:
                    batch, total, mq = self._admit()
                    if batch:
                        try:
                            self._launch(s, batch, total, mq)
                        except Exception as e:      # pragma: no cover
                            for r in batch:
                                r.future.set_exception(e)
                        progressed = True
            with self.cv:
                if not self.running and not self.queue and all(s.batch is None for s in self.slots):
                    return
                if not progressed:
                    busy = any(s.batch is not None for s in self.slots)
                    self.cv.wait(timeout=0.0002 if busy else 0.01)


def slot_bytes(db: Database, k: int, max_batch: int, max_qlen: int, max_total_qlen: int) -> int:
    """Device bytes one slot holds: the batched workspace, the query,
    offset and seed buffers, the hits and the ops."""
    b = C.c_size_t()
    check(lib().hs_search_batch_workspace_size(db.handle, max_batch, max_total_qlen, max_qlen, k, C.byref(b)),
          "hs_search_batch_workspace_size")
    ops = lib().hs_batch_ops_capacity(max_batch, max_total_qlen, k)
    return int(b.value) + max_total_qlen + 16 * (max_batch + 1) + max_batch * k * HIT_DTYPE.itemsize + 4 * ops + 16


def slot_budget(db: Database, k: int, max_batch: int, max_qlen: int, bytes_per_slot: float) -> int:
    """The largest per-slot letter budget (at least max_qlen, at most
    max_batch * max_qlen) whose slot fits bytes_per_slot."""
    lo, hi = max_qlen, max_batch * max_qlen
    if slot_bytes(db, k, max_batch, max_qlen, lo) > bytes_per_slot:
        raise MemoryError("one slot for a %d-letter query does not fit the device memory budget" % max_qlen)
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if slot_bytes(db, k, max_batch, max_qlen, mid) <= bytes_per_slot:
            lo = mid
        else:
            hi = mid - 1
    return lo


def overlap_stats(intervals_ms):
    """From the device-time (start, end) of every batch: the time the device
    had at least one batch in flight, the time it had two or more (batches on
    different slots overlapping), that fraction, and the most batches in
    flight at once."""
    ev = sorted([(a, 1) for a, _ in intervals_ms] + [(b, -1) for _, b in intervals_ms], key=lambda x: (x[0], x[1]))
    busy = over = 0.0
    depth = peak = 0
    last = None
    for t, d in ev:
        if last is not None:
            if depth >= 1:
                busy += t - last
            if depth >= 2:
                over += t - last
        depth += d
        peak = max(peak, depth)
        last = t
    return {"device_busy_ms": busy, "overlap_ms": over, "overlap_frac": over / busy if busy > 0 else 0.0,
            "max_in_flight": peak}


def latency_stats(requests_latency_s):
    x = np.sort(np.asarray(requests_latency_s))
    if len(x) == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None}
    return {"p50_ms": float(np.percentile(x, 50) * 1000), "p99_ms": float(np.percentile(x, 99) * 1000),
            "mean_ms": float(x.mean() * 1000)}
