"""Continuous-batching search server over a database resident in HBM.

Requests (one query each) arrive at any time through ``submit``.  A
dispatcher thread admits waiting requests into the next batch as long as the
device memory the batch needs fits what is left of a fixed budget, and
launches it on the next free worker stream with ``sw_search`` in the batched
form while earlier batches are still running on other streams.  A completion
thread waits on each batch's CUDA event, copies nothing but the top-k hits
and the batch's status word back, and resolves the requests' futures,
recording arrival-to-hits latency.

Memory admission: the server allocates one device pool of ``mem_budget``
bytes at start-up.  A batch's device memory is the workspace
``sw_search_workspace_size`` reports for exactly its queries (the query
codes, one int32 score row over the whole database per query, its top-k
hits, the int32 profile, the overflow lists and the strip-boundary rows);
the batch is admitted only when that many bytes are free in the pool, is
carved out of it, and is returned when the batch completes.  So the bytes
of all batches in flight never exceed the budget, and the number of worker
streams caps how many batches run at once.  A request that needs more than
the whole budget on its own fails instead of being admitted.  The library
allocates nothing per call.

All scoring runs in libswdb's kernels; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import queue
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import binding

_POISON = object()


@dataclasses.dataclass(eq=False)        # identity equality: fields hold arrays
class _Request:
    codes: np.ndarray
    future: Future
    t_arrival: float


@dataclasses.dataclass(eq=False)
class _Batch:
    requests: list
    stream: object
    event: object
    hits_dev: object
    hits_host: object
    status_host: object
    worker: int
    ws_offset: int
    nbytes: int
    t_launch: float
    cells: int


class _Pool:
    """First-fit bookkeeping of byte extents in one device buffer (host side
    only; extents are 256-byte aligned)."""

    ALIGN = 256

    def __init__(self, size: int):
        self.size = int(size)
        self.free = [(0, self.size)]        # (offset, length), sorted by offset
        self.used = 0

    def reserve(self, nbytes: int):
        n = -(-int(nbytes) // self.ALIGN) * self.ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                self.used += n
                return off, n
        return None

    def release(self, off: int, n: int):
        self.used -= n
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged


class SearchServer:
    """Serve top-k searches of single queries against one loaded database.

    db          a binding.Database (resident database)
    matrix      substitution matrix (A x A int32), gap_open / gap_extend, top_k
    max_batch   most queries per launch
    streams     worker streams (batches in flight at once)
    mem_budget  bytes of the device pool the batches in flight are carved from
                (default: room for every stream to run a full batch of the
                longest admissible queries)
    launch      extra sw_search keyword arguments (launch parameters, e.g.
                from autotune.autotune); they never change the results
    """

    def __init__(self, db, matrix, gap_open: int, gap_extend: int, top_k: int = 10, max_batch: int = 32,
                 streams: int = 2, mem_budget: int | None = None, max_query_len: int = 8000,
                 mode: int = binding.SW_MODE_BATCHED, launch: dict | None = None):
        import torch
        self.torch = torch
        self.db = db
        self.matrix = np.ascontiguousarray(matrix, dtype=np.int32)
        self.gap_open, self.gap_extend, self.top_k = int(gap_open), int(gap_extend), int(top_k)
        self.max_batch = int(max_batch)
        self.max_query_len = int(max_query_len)
        self.mode = mode
        self.launch_kw = dict(launch or {})
        self.launch_kw.pop("mode", None)
        self.n_seqs = db.n_seqs
        info = db.info()
        self.db_residues = info["residues"]
        self.device = torch.device("cuda", db.device)
        if mem_budget is None:
            q_off = np.arange(self.max_batch + 1, dtype=np.int64) * self.max_query_len
            mem_budget = streams * (self._workspace_bytes(q_off) + _Pool.ALIGN)
        self.mem_budget = int(mem_budget)
        self.pool = _Pool(self.mem_budget)
        self.pool_dev = torch.empty(max(self.mem_budget, 1), dtype=torch.uint8, device=self.device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.status_dev = [torch.zeros(1, dtype=torch.int32, device=self.device) for _ in range(streams)]
        self.free_workers = queue.Queue()
        for i in range(streams):
            self.free_workers.put(i)
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.in_flight_bytes = 0
        self.peak_in_flight_bytes = 0
        self.inflight = queue.Queue()
        self.latencies = []
        self.completed = 0
        self.cells = 0
        self.batches = 0
        self.batch_sizes = []
        self.t_first = None
        self.t_last = None
        self.closed = False
        self.error = None
        self.dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self.completer = threading.Thread(target=self._complete, daemon=True)
        self.dispatcher.start()
        self.completer.start()

    def _workspace_bytes(self, q_off) -> int:
        kw = {k: v for k, v in self.launch_kw.items()
              if k in ("precision", "long_cutoff", "lanes", "rows_per_lane", "long_rows_per_lane")}
        return binding.sw_search_workspace_size(self.db.handle, q_off, self.top_k, mode=self.mode, **kw)

    # -- public -------------------------------------------------------------
    def submit(self, codes) -> Future:
        """Queue one query (uint8 codes); the future resolves to its top-k hits
        (HIT_DTYPE array, best first)."""
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        if len(codes) > self.max_query_len:
            raise ValueError(f"query longer than max_query_len={self.max_query_len}")
        fut = Future()
        req = _Request(codes, fut, time.perf_counter())
        with self.cv:
            if self.closed:
                raise RuntimeError("server closed")
            if self.t_first is None:
                self.t_first = req.t_arrival
            self.pending.append(req)
            self.cv.notify_all()
        return fut

    def close(self, timeout: float = 600.0):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        self.dispatcher.join(timeout)
        self.inflight.put(_POISON)
        self.completer.join(timeout)
        if self.error:
            raise self.error
        if self.dispatcher.is_alive() or self.completer.is_alive():
            raise TimeoutError("server threads did not finish")

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.zeros(1)
        span = (self.t_last - self.t_first) if (self.t_first and self.t_last) else 0.0
        return {"completed": self.completed, "batches": self.batches,
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "gcups": self.cells / span / 1e9 if span > 0 else 0.0,
                "span_s": span, "mem_budget": self.mem_budget, "peak_in_flight_bytes": self.peak_in_flight_bytes}

    # -- threads ------------------------------------------------------------
    def _take_batch(self):
        """Admit waiting requests (FIFO, at most max_batch) whose workspace fits
        the free part of the pool: the longest prefix that fits, found by
        halving.  Returns (requests, (offset, bytes)) or ([], None).  A lone
        request that cannot fit even an empty pool gets an error instead."""
        n = min(len(self.pending), self.max_batch)
        while n > 0:
            lens = np.array([len(self.pending[i].codes) for i in range(n)], dtype=np.int64)
            q_off = np.zeros(n + 1, dtype=np.int64)
            np.cumsum(lens, out=q_off[1:])
            need = self._workspace_bytes(q_off)
            got = self.pool.reserve(need)
            if got is not None:
                return [self.pending.popleft() for _ in range(n)], got
            if n == 1 and self.pool.used == 0:
                r = self.pending.popleft()
                r.future.set_exception(MemoryError(
                    f"query of length {len(r.codes)} needs {need} device bytes, more than the "
                    f"whole budget of {self.mem_budget}"))
                return [], None
            n //= 2
        return [], None

    def _dispatch(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        try:
            while True:
                worker = None
                while worker is None:           # a failed completer never returns workers
                    try:
                        worker = self.free_workers.get(timeout=0.1)
                    except queue.Empty:
                        if self.error is not None:
                            return
                        with self.cv:
                            if self.closed and not self.pending:
                                return
                with self.cv:
                    while True:
                        while not self.pending and not self.closed:
                            self.cv.wait()
                        if not self.pending and self.closed:
                            self.free_workers.put(worker)
                            return
                        batch, ext = self._take_batch()
                        if batch:
                            break
                        if self.error is not None:
                            return
                        if self.pending:                   # memory budget: wait for completions
                            self.cv.wait(timeout=0.05)
                    self.in_flight_bytes += ext[1]
                    self.peak_in_flight_bytes = max(self.peak_in_flight_bytes, self.in_flight_bytes)
                try:
                    self._launch(worker, batch, ext)
                except Exception as e:   # this batch fails; the server keeps serving
                    for r in batch:
                        if not r.future.done():
                            r.future.set_exception(e)
                    with self.cv:
                        self.in_flight_bytes -= ext[1]
                        self.pool.release(*ext)
                        self.cv.notify_all()
                    self.free_workers.put(worker)
        except Exception as e:  # surface errors to close()
            self.error = e
            with self.cv:
                for r in self.pending:
                    r.future.set_exception(e)
                self.pending.clear()

    def _launch(self, worker, batch, ext):
        torch = self.torch
        stream = self.streams[worker]
        lens = np.array([len(r.codes) for r in batch], dtype=np.int64)
        q_off = np.zeros(len(batch) + 1, dtype=np.int64)
        np.cumsum(lens, out=q_off[1:])
        q_host = torch.from_numpy(np.concatenate([r.codes for r in batch]) if q_off[-1] else
                                  np.zeros(1, np.uint8)).pin_memory()
        ws = self.pool_dev[ext[0]:ext[0] + ext[1]]
        with torch.cuda.stream(stream):
            q_dev = q_host.to(self.device, non_blocking=True)
            hits_dev = torch.empty((len(batch), max(self.top_k, 1), 2), dtype=torch.int64, device=self.device)
            binding.sw_search(self.db.handle, q_dev[:int(q_off[-1])], q_off, self.matrix, self.gap_open,
                              self.gap_extend, self.top_k, None, hits_dev, mode=self.mode, workspace=ws,
                              stream=stream.cuda_stream, status_out=self.status_dev[worker], **self.launch_kw)
            hits_host = torch.empty(hits_dev.shape, dtype=torch.int64).pin_memory()
            hits_host.copy_(hits_dev, non_blocking=True)
            status_host = torch.empty(1, dtype=torch.int32).pin_memory()
            status_host.copy_(self.status_dev[worker], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.inflight.put(_Batch(batch, stream, ev, hits_dev, hits_host, status_host, worker, ext[0], ext[1],
                                 time.perf_counter(), int(lens.sum()) * self.db_residues))

    def _complete(self):
        """Resolve batches as their events complete (in any order across streams).
        If anything fails, every outstanding future gets the exception."""
        live = []
        try:
            self._complete_loop(live)
        except BaseException as e:  # noqa: BLE001 - surfaced through the futures and close()
            self.error = e
            for b in live:
                for r in b.requests:
                    if not r.future.done():
                        r.future.set_exception(e)
            while True:
                try:
                    b = self.inflight.get_nowait()
                except queue.Empty:
                    break
                if b is not _POISON:
                    for r in b.requests:
                        if not r.future.done():
                            r.future.set_exception(e)
            with self.cv:
                for r in self.pending:
                    if not r.future.done():
                        r.future.set_exception(e)
                self.pending.clear()
                self.cv.notify_all()

    def _complete_loop(self, live):
        done = False
        while not done or live:
            try:
                while True:
                    b = self.inflight.get(block=not live and not done, timeout=None)
                    if b is _POISON:
                        done = True
                    else:
                        live.append(b)
                    if self.inflight.empty():
                        break
            except queue.Empty:
                pass
            finished = [b for b in live if b.event.query()]
            if not finished:
                time.sleep(50e-6)
                continue
            now = time.perf_counter()
            for b in finished:
                h = b.hits_host.numpy()
                status = int(b.status_host.numpy()[0])
                for i, r in enumerate(b.requests):
                    if status != 0:     # a bounded wait gave up: this batch's hits are not valid
                        r.future.set_exception(binding.SwError(status, "the search's device-side status "
                                                                       "reports a bounded wait that gave up"))
                        continue
                    out = np.empty(self.top_k, dtype=binding.HIT_DTYPE)
                    out["score"] = (h[i, :, 0] & 0xffffffff).astype(np.int64).astype(np.int32)
                    out["reserved"] = 0
                    out["db_index"] = h[i, :, 1]
                    self.latencies.append(now - r.t_arrival)
                    r.future.set_result(out)
                with self.cv:
                    self.in_flight_bytes -= b.nbytes
                    self.pool.release(b.ws_offset, b.nbytes)
                    self.completed += len(b.requests)
                    self.cells += b.cells
                    self.batches += 1
                    self.batch_sizes.append(len(b.requests))
                    self.t_last = now
                    self.cv.notify_all()
                live[:] = [x for x in live if x is not b]   # only once its futures are resolved
                self.free_workers.put(b.worker)
