"""Host-side completion logic of the server, with fake CUDA events (no GPU).

Batches on different streams can finish in any order; the completion
thread must resolve each batch's futures as soon as its own event is done,
and any failure must reach every outstanding future instead of leaving them
pending.
"""
import collections
import queue
import threading
from concurrent.futures import Future

import numpy as np

from paper_2203_11100_gb300 import serve


class _Event:
    def __init__(self):
        self.ready = False

    def query(self):
        return self.ready


class _Hits:
    def __init__(self, arr):
        self.arr = arr

    def numpy(self):
        return self.arr


def _server_shell(top_k=3):
    s = serve.SearchServer.__new__(serve.SearchServer)
    s.inflight = queue.Queue()
    s.cv = threading.Condition()
    s.free_workers = queue.Queue()
    s.pending = collections.deque()
    s.latencies, s.batch_sizes = [], []
    s.completed = s.cells = s.batches = 0
    s.in_flight_bytes = 0
    s.t_last = None
    s.top_k = top_k
    s.error = None
    return s


def _batch(n_req, worker, score, length):
    reqs = [serve._Request(np.zeros(length + i, np.uint8), Future(), 0.0, 10) for i in range(n_req)]
    h = np.zeros((n_req, 3, 2), np.int64)
    h[:, :, 0] = score
    h[:, :, 1] = np.arange(3)
    return serve._Batch(reqs, None, _Event(), None, _Hits(h), worker, 10 * n_req, 0.0, 100)


def test_out_of_order_completion():
    s = _server_shell()
    b1, b2 = _batch(2, 0, 7, 367), _batch(3, 1, 9, 133)
    t = threading.Thread(target=s._complete)
    t.start()
    s.inflight.put(b1)
    s.inflight.put(b2)
    b2.event.ready = True                     # the later batch finishes first
    r = b2.requests[0].future.result(timeout=5)
    assert list(r["score"]) == [9, 9, 9]
    assert not b1.requests[0].future.done()
    b1.event.ready = True
    assert list(b1.requests[1].future.result(timeout=5)["score"]) == [7, 7, 7]
    s.inflight.put(serve._POISON)
    t.join(timeout=5)
    assert not t.is_alive()
    assert s.completed == 5 and s.batches == 2 and s.error is None


def test_failure_reaches_every_future():
    s = _server_shell()
    bad = _batch(2, 0, 1, 10)
    bad.hits_host = None                      # completing this batch raises
    other = _batch(1, 1, 2, 20)
    t = threading.Thread(target=s._complete)
    t.start()
    s.inflight.put(other)
    s.inflight.put(bad)
    bad.event.ready = True
    for r in bad.requests + other.requests:
        try:
            r.future.result(timeout=5)
        except Exception:
            pass
        assert r.future.done()
    t.join(timeout=5)
    assert s.error is not None


def test_failed_launch_resolves_its_requests():
    """A batch whose launch raises gets the exception on its own futures and
    the server goes on with the next batch."""
    s = _server_shell()
    s.max_batch = 4
    s.mem_budget = 1 << 40
    s.closed = False
    s.error = None
    calls = []

    def launch(worker, batch, nbytes):
        calls.append(len(batch))
        if len(calls) == 1:
            raise RuntimeError("workspace too small")
        for r in batch:
            r.future.set_result("ok")
        with s.cv:
            s.in_flight_bytes -= nbytes
        s.free_workers.put(worker)

    s._launch = launch
    s.free_workers.put(0)
    reqs = [serve._Request(np.zeros(5, np.uint8), Future(), 0.0, 10) for _ in range(6)]
    s.pending.extend(reqs[:4])
    t = threading.Thread(target=s._dispatch)
    s.torch = type("T", (), {"cuda": type("C", (), {"set_device": staticmethod(lambda d: None)})})
    s.device = None
    t.start()
    for r in reqs[:4]:
        try:
            r.future.result(timeout=5)
        except RuntimeError:
            pass
    assert all(isinstance(r.future.exception(timeout=1), RuntimeError) for r in reqs[:4])
    with s.cv:
        s.pending.extend(reqs[4:])
        s.cv.notify_all()
    assert [r.future.result(timeout=5) for r in reqs[4:]] == ["ok", "ok"]
    with s.cv:
        s.closed = True
        s.cv.notify_all()
    t.join(timeout=5)
    assert not t.is_alive()
