"""Autotuner for the search's launch parameters.

The paper's SW#db takes its launch shape from fixed per-architecture tables
(Section 3.2) and its GCUPS depend on the work-group size (Section 4.2).
Here the library picks, per query (plain form) or per query pair (batched
form), the launch shape -- lanes per subwarp, which sets the sequences per
256-thread block, and query rows per lane -- with the least predicted time
ceil(m / (lanes*rows)) * lanes*rows / rate, from a table of shapes and
their cell rates.  This module measures that table on the caller's GPU and
database and installs it on the handle (sw_db_set_tuning), together with:

- the lane packing: sequence pairs in the int16x2 halves with one launch per
  query (the plain form), or query pairs with one persistent launch for the
  whole batch (the batched form) -- what SW_MODE_AUTO then means;
- the length above which database sequences go to the intra-task kernel.

Measurements use the library's own CUDA-event kernel times (the median of
several repeats after a warm-up):

- shape rates: a query of 3,072 residues taken from the batch itself (a
  whole number of strips of every shape, so no padding enters the rate)
  against the whole resident database, one search per candidate shape,
  rate = the scoring kernel's cells / its event time; on a database so large
  that one such search would exceed about 2e12 cells the query is halved (to
  1,536 or 768 rows) and the shapes whose strip does not divide it are left
  out;
- cutoff and form: the whole search of a sample of the batch (queries spread
  over its length range), bracketed by CUDA events on its stream.

The result is cached in a JSON file keyed by GPU, database, substitution
matrix, penalties, the arithmetic the library chose, library version and the
batch's length profile, so the next batch of the same kind reuses it.  The
launch parameters never change the scores; only the time does.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import time

import numpy as np

from . import binding

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "swdb", "autotune.json")

# The 4-lane shapes (4, 24) and (4, 32) are left out: their padding-free probe
# rate is the highest (6,278 GCUPS for (4, 32) against 6,193 for (8, 32) on the
# default database), but a table holding them made the 20-query default
# workload slower (5,598 against 5,877 GCUPS), so the probe misranks them.
PLAIN_SHAPES = ((8, 16), (16, 16), (32, 16), (8, 24), (8, 32), (16, 32), (32, 32))
BATCH_SHAPES = ((8, 16), (8, 24), (8, 32), (16, 16), (16, 24), (16, 32))
CUTOFFS = (0, 1024, 2048, 3072, 6144)   # 0: the library's balanced default for this database
RATE_ROWS = 3072          # a whole number of strips of every candidate shape
MAX_PROBE_CELLS = 2e12    # cells of one rate-probe search (about a third of a second)


def probe_rows(residues: int) -> int:
    """Rows of the rate-probe query for a database of this many residues."""
    rows = RATE_ROWS
    while rows > 768 and float(residues) * rows > MAX_PROBE_CELLS:
        rows //= 2
    return rows


def _device_key(device: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|sm{p.multi_processor_count}"


def _batch_key(db_info: dict, lengths: np.ndarray) -> str:
    q = np.percentile(lengths, [10, 50, 90]).astype(int) if len(lengths) else [0, 0, 0]
    nq_bucket = int(2 ** np.ceil(np.log2(max(len(lengths), 1))))
    return (f"db{db_info['n_seqs']}:{db_info['residues']}:{db_info['max_length']}"
            f"|nq{nq_bucket}|len{q[0]}-{q[1]}-{q[2]}")


def _search_key(matrix, gap_open: int, gap_extend: int, precision: int) -> str:
    h = hashlib.sha256(np.ascontiguousarray(matrix, dtype=np.int32).tobytes()).hexdigest()[:16]
    return f"S{h}|o{int(gap_open)}e{int(gap_extend)}|prec{int(precision)}|{binding.sw_version()}"


def _sample(queries, offsets, k: int):
    """Up to k queries spread over the length range (by length rank)."""
    lens = np.diff(offsets)
    order = np.argsort(lens, kind="stable")
    pick = order[np.unique(np.linspace(0, len(order) - 1, min(k, len(order))).round().astype(int))]
    pick = np.sort(pick)
    res = np.concatenate([queries[offsets[i]:offsets[i + 1]] for i in pick]) if len(pick) else np.zeros(0, np.uint8)
    off = np.zeros(len(pick) + 1, dtype=np.int64)
    np.cumsum(lens[pick], out=off[1:])
    return res, off


def _probe_queries(queries, n: int, rows: int = RATE_ROWS):
    """n queries of `rows` residues cut from the batch's own residues (tiled
    when the batch is shorter)."""
    src = np.ascontiguousarray(queries, dtype=np.uint8)
    if len(src) == 0:
        src = np.zeros(1, np.uint8)
    reps = -(-(n * rows) // len(src))
    res = np.tile(src, reps)[:n * rows].copy()
    return res, np.arange(n + 1, dtype=np.int64) * rows


def _median_rate(db, q_res, q_off, matrix, o, e, stream, repeats: int, **kw) -> float:
    """Median over repeats of the scoring kernel's own cell rate (GCUPS) in
    one search, after a warm-up search."""
    import torch
    q_dev = torch.from_numpy(q_res).cuda(db.device)
    call = lambda: binding.sw_search(db.handle, q_dev, q_off, matrix, o, e, 0, None, None, stats=True,
                                     stream=stream.cuda_stream, **kw)
    call()
    rates = []
    for _ in range(repeats):
        st = call()
        if st["inter_ms"] <= 0 or st["inter_cells"] <= 0:
            continue
        rates.append(st["inter_cells"] / (st["inter_ms"] * 1e-3) / 1e9)
    return statistics.median(rates) if rates else 0.0


def _median_search_ms(db, q_res, q_off, matrix, o, e, top_k, stream, repeats: int, **kw) -> float:
    """Median over repeats of a whole search's time (CUDA events on its stream)."""
    import torch
    q_dev = torch.from_numpy(q_res).cuda(db.device)
    n = db.n_seqs
    scores = torch.empty((len(q_off) - 1, max(n, 1)), dtype=torch.int32, device=q_dev.device)
    hits = torch.empty((len(q_off) - 1, max(top_k, 1), 2), dtype=torch.int64, device=q_dev.device)

    def call():
        binding.sw_search(db.handle, q_dev, q_off, matrix, o, e, top_k, scores, hits if top_k else None,
                          stream=stream.cuda_stream, **kw)

    call()
    times = []
    for _ in range(repeats):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def autotune(db, queries, q_offsets, matrix, gap_open: int, gap_extend: int, top_k: int = 10,
             sample_queries: int = 16, cache_path: str | None = DEFAULT_CACHE, force: bool = False,
             repeats: int = 3, plain_shapes=PLAIN_SHAPES, batch_shapes=BATCH_SHAPES, cutoffs=CUTOFFS,
             forms=("plain", "batched")) -> dict:
    """Measure (or take from the cache) this batch kind's launch tuning,
    install it on db's handle, and return the sw_search keyword arguments
    it implies ({"mode": ..., "long_cutoff": ...}).  The handle keeps the
    tuning (shape tables, cutoff, and the form SW_MODE_AUTO takes) until it
    is replaced; see sw_db_set_tuning.  last_result() returns the measured
    tables and the candidates tried."""
    import torch
    queries = np.ascontiguousarray(queries, dtype=np.uint8)
    q_offsets = np.ascontiguousarray(q_offsets, dtype=np.int64)
    info = db.info()
    stream = torch.cuda.Stream(device=db.device)
    # which arithmetic the library takes for this matrix and these penalties
    probe_res, probe_off = _probe_queries(queries, 1, rows=64)
    prec = binding.sw_search(db.handle, probe_res, probe_off, matrix, gap_open, gap_extend, 0, None, None,
                             stats=True)["precision_used"]
    key = "|".join([_device_key(db.device), _batch_key(info, np.diff(q_offsets)),
                    _search_key(matrix, gap_open, gap_extend, prec), ",".join(forms)])
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except Exception:
            cache = {}
    if not force and key in cache:
        entry = cache[key]
        binding.sw_db_set_tuning(db.handle, entry["tuning"])
        _LAST.clear()
        _LAST.update(entry, cached=True)
        return dict(entry["params"])

    t_start = time.perf_counter()
    binding.sw_db_set_tuning(db.handle, None)
    tuning = {"plain": [], "batched": [], "long_cutoff": 0, "long_rows_per_lane": 0, "mode": 0}
    rows = probe_rows(info["residues"])
    plain_shapes = [x for x in plain_shapes if rows % (x[0] * x[1]) == 0]
    batch_shapes = [x for x in batch_shapes if rows % (x[0] * x[1]) == 0]
    if prec == binding.SW_PREC_I16:
        one_res, one_off = _probe_queries(queries, 1, rows)
        for (l, r) in plain_shapes:
            try:
                g = _median_rate(db, one_res, one_off, matrix, gap_open, gap_extend, stream, repeats,
                                 mode=binding.SW_MODE_PLAIN, lanes=l, rows_per_lane=r)
            except binding.SwError:
                continue
            if g > 0:
                tuning["plain"].append((l, r, g))
        if "batched" in forms:
            two_res, two_off = _probe_queries(queries, 2, rows)
            for (l, r) in batch_shapes:
                try:
                    g = _median_rate(db, two_res, two_off, matrix, gap_open, gap_extend, stream, repeats,
                                     mode=binding.SW_MODE_BATCHED, lanes=l, rows_per_lane=r)
                except binding.SwError:
                    continue
                if g > 0:
                    tuning["batched"].append((l, r, g))
    binding.sw_db_set_tuning(db.handle, tuning)

    # the cutoff and the form, on a sample of the batch with the measured tables
    s_res, s_off = _sample(queries, q_offsets, sample_queries)
    tried = []
    mode_of = {"plain": binding.SW_MODE_PLAIN, "batched": binding.SW_MODE_BATCHED}
    for form in forms:
        if form == "batched" and prec != binding.SW_PREC_I16:
            continue
        for cut in cutoffs:
            try:
                ms = _median_search_ms(db, s_res, s_off, matrix, gap_open, gap_extend, top_k, stream, repeats,
                                       mode=mode_of[form], long_cutoff=cut)
            except binding.SwError:
                continue
            tried.append({"form": form, "long_cutoff": cut, "ms": ms})
    if not tried:
        raise RuntimeError("no candidate launch configuration ran")
    best = min(tried, key=lambda x: x["ms"])
    tuning["long_cutoff"] = best["long_cutoff"]
    tuning["mode"] = mode_of[best["form"]]
    binding.sw_db_set_tuning(db.handle, tuning)
    cells = int(np.diff(s_off).sum()) * info["residues"]
    params = {"mode": tuning["mode"], "long_cutoff": tuning["long_cutoff"]}
    entry = {"params": params, "tuning": tuning, "sample_cells": cells, "probe_rows": rows,
             "sample_gcups": cells / (best["ms"] * 1e-3) / 1e9 if best["ms"] > 0 else 0.0,
             "tried": tried, "tune_seconds": time.perf_counter() - t_start}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache[key] = entry
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    _LAST.clear()
    _LAST.update(entry, cached=False)
    return dict(params)


_LAST: dict = {}


def last_result() -> dict:
    """The measured (or cached) entry of the last autotune() call: params,
    tuning tables, sample GCUPS, the candidates tried and the time spent."""
    return dict(_LAST)
