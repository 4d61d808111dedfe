"""Autotuner for the search's launch parameters.

It picks, for one GPU, database and kind of query batch:

- the lane packing: sequence pairs in the int16x2 halves with one launch per
  query (the plain form), or query pairs with one persistent launch (the
  batched form);
- the subwarp width (lanes), which sets the sequences per 256-thread block;
- the query rows held per lane;
- the length above which database sequences go to the intra-task kernel.

Each candidate is timed on a bounded sample of the batch (queries spread
over its length range) against the whole resident database, with the
library's own CUDA-event kernel timings.  The winner is cached in a JSON file
keyed by GPU name, SM count, database size and the batch's length profile, so
the next batch of the same kind reuses it.  The launch parameters never change
the scores; only the time does.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import binding

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "swdb", "autotune.json")

CANDIDATES = (
    [{"mode": binding.SW_MODE_PLAIN, "lanes": 0, "rows_per_lane": 0}]
    + [{"mode": binding.SW_MODE_BATCHED, "lanes": l, "rows_per_lane": r} for l, r in
       [(8, 16), (8, 24), (8, 32), (16, 24), (16, 32)]]
)
CUTOFFS = (2048, 3072, 6144)


def _device_key(device: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|sm{p.multi_processor_count}"


def _batch_key(db_info: dict, lengths: np.ndarray) -> str:
    q = np.percentile(lengths, [10, 50, 90]).astype(int) if len(lengths) else [0, 0, 0]
    nq_bucket = int(2 ** np.ceil(np.log2(max(len(lengths), 1))))
    return (f"db{db_info['n_seqs']}:{db_info['residues']}:{db_info['max_length']}"
            f"|nq{nq_bucket}|len{q[0]}-{q[1]}-{q[2]}")


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


def autotune(db, queries, q_offsets, matrix, gap_open: int, gap_extend: int, top_k: int = 10,
             sample_queries: int = 16, cache_path: str | None = DEFAULT_CACHE, force: bool = False,
             candidates=CANDIDATES, cutoffs=CUTOFFS) -> dict:
    """Return the fastest launch parameters (keyword arguments of sw_search)
    for this kind of batch, measuring them if the cache has no entry."""
    queries = np.ascontiguousarray(queries, dtype=np.uint8)
    q_offsets = np.ascontiguousarray(q_offsets, dtype=np.int64)
    info = db.info()
    key = _device_key(db.device) + "|" + _batch_key(info, np.diff(q_offsets))
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except Exception:
            cache = {}
    if not force and key in cache:
        return dict(cache[key]["params"])

    s_res, s_off = _sample(queries, q_offsets, sample_queries)
    cells = int(np.diff(s_off).sum()) * info["residues"]
    results = []
    for cand in candidates:
        for cut in cutoffs:
            params = dict(cand, long_cutoff=cut)
            try:
                binding.sw_search(db.handle, s_res, s_off, matrix, gap_open, gap_extend, top_k, None, None,
                                  stats=True, **params)                 # warm-up (and plan validation)
                t0 = time.perf_counter()
                st = binding.sw_search(db.handle, s_res, s_off, matrix, gap_open, gap_extend, top_k, None, None,
                                       stats=True, **params)
                dt = time.perf_counter() - t0
            except binding.SwError:
                continue
            results.append((dt, params, st))
    if not results:
        raise RuntimeError("no candidate launch configuration ran")
    results.sort(key=lambda r: r[0])
    best_dt, best, _ = results[0]
    entry = {"params": best, "gcups": cells / best_dt / 1e9, "sample_cells": cells,
             "tried": [{"params": p, "gcups": cells / d / 1e9} for d, p, _ in results]}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache[key] = entry
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return dict(best)
