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


class _Status:
    def __init__(self, v=0):
        self.v = v

    def numpy(self):
        return np.array([self.v], np.int32)


def _server_shell(top_k=3, budget=1 << 40):
    s = serve.SearchServer.__new__(serve.SearchServer)
    s.pool = serve._Pool(budget)
    s.mem_budget = budget
    s.peak_in_flight_bytes = 0
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


def _batch(s, n_req, worker, score, length, status=0):
    reqs = [serve._Request(np.zeros(length + i, np.uint8), Future(), 0.0) for i in range(n_req)]
    h = np.zeros((n_req, 3, 2), np.int64)
    h[:, :, 0] = score
    h[:, :, 1] = np.arange(3)
    off, n = s.pool.reserve(1000 * n_req)
    s.in_flight_bytes += n
    return serve._Batch(reqs, None, _Event(), None, _Hits(h), _Status(status), worker, off, n, 0.0, 100)


def test_out_of_order_completion():
    s = _server_shell()
    b1, b2 = _batch(s, 2, 0, 7, 367), _batch(s, 3, 1, 9, 133)
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
    assert s.pool.used == 0 and s.in_flight_bytes == 0 and s.pool.free == [(0, 1 << 40)]


def test_failure_reaches_every_future():
    s = _server_shell()
    bad = _batch(s, 2, 0, 1, 10)
    bad.hits_host = None                      # completing this batch raises
    other = _batch(s, 1, 1, 2, 20)
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
    s.closed = False
    s.error = None
    s._workspace_bytes = lambda q_off: 1000 * (len(q_off) - 1)
    calls = []

    def launch(worker, batch, ext):
        calls.append(len(batch))
        if len(calls) == 1:
            raise RuntimeError("workspace too small")
        for r in batch:
            r.future.set_result("ok")
        with s.cv:
            s.in_flight_bytes -= ext[1]
            s.pool.release(*ext)
        s.free_workers.put(worker)

    s._launch = launch
    s.free_workers.put(0)
    reqs = [serve._Request(np.zeros(5, np.uint8), Future(), 0.0) for _ in range(6)]
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
    assert s.pool.used == 0


def test_status_word_fails_the_batch():
    """A batch whose device-side status reports a bounded wait that gave up
    resolves its futures with SW_ERR_TIMEOUT instead of returning its hits."""
    from paper_2203_11100_gb300 import binding
    s = _server_shell()
    bad = _batch(s, 2, 0, 5, 10, status=4)
    good = _batch(s, 1, 1, 6, 20)
    t = threading.Thread(target=s._complete)
    t.start()
    s.inflight.put(bad)
    s.inflight.put(good)
    bad.event.ready = good.event.ready = True
    for r in bad.requests:
        e = r.future.exception(timeout=5)
        assert isinstance(e, binding.SwError) and e.code == 4
    assert list(good.requests[0].future.result(timeout=5)["score"]) == [6, 6, 6]
    s.inflight.put(serve._POISON)
    t.join(timeout=5)
    assert s.pool.used == 0


def test_pool_first_fit_and_coalescing():
    p = serve._Pool(4096)
    a = p.reserve(1)            # rounded up to 256
    b = p.reserve(1000)         # 1024
    c = p.reserve(256)
    assert a == (0, 256) and b == (256, 1024) and c == (1280, 256)
    assert p.reserve(4096) is None
    p.release(*b)
    assert p.reserve(512) == (256, 512)       # first fit, inside the freed hole
    p.release(256, 512)
    p.release(*a)
    p.release(*c)
    assert p.free == [(0, 4096)] and p.used == 0


def _admission_shell(budget, per_query, max_batch=8):
    s = _server_shell(budget=budget)
    s.max_batch = max_batch
    s._workspace_bytes = lambda q_off: per_query * (len(q_off) - 1)
    return s


def test_admission_takes_the_longest_prefix_that_fits():
    s = _admission_shell(budget=5 * 1024, per_query=1024)
    reqs = [serve._Request(np.zeros(5, np.uint8), Future(), 0.0) for _ in range(8)]
    s.pending.extend(reqs)
    batch, ext = s._take_batch()
    assert len(batch) == 4 and ext == (0, 4096)           # 8 do not fit, 4 do
    batch2, ext2 = s._take_batch()
    assert len(batch2) == 1 and ext2 == (4096, 1024)      # what is left holds one
    assert s._take_batch() == ([], None)                   # full: wait for completions
    s.pool.release(*ext)
    batch3, _ = s._take_batch()
    assert len(batch3) == 3 and not s.pending


def test_request_larger_than_the_budget_fails():
    s = _admission_shell(budget=1000, per_query=4096)
    r = serve._Request(np.zeros(5, np.uint8), Future(), 0.0)
    s.pending.append(r)
    assert s._take_batch() == ([], None)
    assert isinstance(r.future.exception(timeout=1), MemoryError)
    assert not s.pending and s.pool.used == 0
