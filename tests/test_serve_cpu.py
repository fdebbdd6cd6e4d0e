"""Host logic of the serving loop, without a GPU: admission from the head of
the queue under the memory gate, cancelled requests dropped (and admitted
ones marked running, so a late cancel cannot race the result), and the
latency summary."""
import threading
from collections import deque

import numpy as np

from paper_1508_06561_gb300 import serve


def fake_server(fits):
    srv = serve.Server.__new__(serve.Server)
    srv.queue = deque()
    srv.cv = threading.Condition()
    srv.cancelled = 0
    srv._fits = fits
    return srv


def test_admission_follows_the_gate_and_drops_cancelled():
    srv = fake_server(lambda nq, total, mq: nq <= 3 and total <= 100)
    reqs = [serve._Req(np.zeros(L, np.uint8), i) for i, L in enumerate([10, 20, 30, 40, 5, 7])]
    assert reqs[1].future.cancel()
    srv.queue.extend(reqs)
    batch, total, mq = srv._admit()
    assert [r.seed for r in batch] == [0, 2, 3]          # 10 + 30 + 40 letters, three queries
    assert (total, mq) == (80, 40)
    assert srv.cancelled == 1
    assert all(r.future.running() for r in batch)
    assert not batch[0].future.cancel()                  # admitted: too late to cancel
    batch, total, mq = srv._admit()
    assert [r.seed for r in batch] == [4, 5] and total == 12
    assert not srv.queue


def test_head_of_queue_blocks_when_it_does_not_fit():
    srv = fake_server(lambda nq, total, mq: total <= 50)
    reqs = [serve._Req(np.zeros(L, np.uint8), i) for i, L in enumerate([40, 30, 5])]
    srv.queue.extend(reqs)
    batch, _, _ = srv._admit()
    assert [r.seed for r in batch] == [0]                # FIFO: the 5-letter request waits its turn
    batch, _, _ = srv._admit()
    assert [r.seed for r in batch] == [1, 2]


def test_latency_stats():
    st = serve.latency_stats([0.001 * i for i in range(1, 101)])
    assert abs(st["p50_ms"] - 50.5) < 1e-9 and abs(st["p99_ms"] - 99.01) < 1e-6
    assert serve.latency_stats([])["p50_ms"] is None


def test_a_request_that_never_fits_fails_instead_of_stalling_the_queue():
    srv = fake_server(lambda nq, total, mq: total <= 50)
    reqs = [serve._Req(np.zeros(L, np.uint8), i) for i, L in enumerate([60, 30, 5])]
    srv.queue.extend(reqs)
    batch, total, _ = srv._admit()
    assert [r.seed for r in batch] == [1, 2] and total == 35
    assert isinstance(reqs[0].future.exception(timeout=0), ValueError)
    assert not srv.queue


def test_a_failed_harvest_resolves_every_future_of_the_batch():
    """An error while results are copied out reaches every caller of the
    batch (as its exception) and the server's error list."""
    srv = serve.Server.__new__(serve.Server)
    srv.errors = []

    class Boom(RuntimeError):
        pass

    def deliver(slot, batch):
        batch[0].future.set_result("first one done")
        raise Boom("copy failed")

    srv._deliver = deliver
    slot = type("S", (), {})()
    reqs = [serve._Req(np.zeros(4, np.uint8), i) for i in range(3)]
    for r in reqs:
        r.future.set_running_or_notify_cancel()
    slot.batch = (reqs, 3, 3)
    srv._harvest(slot)
    assert slot.batch is None
    assert reqs[0].future.result(timeout=0) == "first one done"
    for r in reqs[1:]:
        assert isinstance(r.future.exception(timeout=0), Boom)
    assert len(srv.errors) == 1


def test_submit_rejects_codes_outside_the_alphabet():
    srv = fake_server(lambda nq, total, mq: True)
    srv.max_qlen = 100
    import pytest
    with pytest.raises(ValueError):
        srv.submit(np.array([1, 2, 24], np.uint8))
    with pytest.raises(ValueError):
        srv.submit(np.array([65, 66], np.uint8))
    with pytest.raises(ValueError):
        srv.submit(np.zeros(101, np.uint8))
    f = srv.submit(np.array([0, 23], np.uint8))
    assert not f.done() and len(srv.queue) == 1


def test_slot_budget_below_the_longest_request_is_refused():
    import pytest
    with pytest.raises(ValueError):
        serve.Server(None, max_qlen=2048, max_total_qlen=1000)


def test_overlap_stats_of_batch_intervals():
    st = serve.overlap_stats([(0.0, 10.0), (5.0, 12.0), (20.0, 25.0)])
    assert st["device_busy_ms"] == 17.0 and st["overlap_ms"] == 5.0 and st["max_in_flight"] == 2
    assert abs(st["overlap_frac"] - 5.0 / 17.0) < 1e-12
    assert serve.overlap_stats([])["overlap_frac"] == 0.0
    st = serve.overlap_stats([(0.0, 4.0), (1.0, 2.0), (1.5, 3.0)])
    assert st["max_in_flight"] == 3 and st["overlap_ms"] == 2.0
