"""CPU oracle for protein database search by Smith-Waterman/Gotoh scoring.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the library.  It shares no code
with the CUDA path; the only thing both sides consume is the seeded inputs
of the ``synth`` module.

- ``score`` / ``score_pairs`` / ``all_scores``: the Gotoh recurrences of
  Section 2.2 (Smith-Waterman local alignment) with affine gaps as in the
  experiments of Section 4.1, written out in plain C (``gotoh.c``), int64.
- ``top_k``: the k best database entries of a score row, ordered by score
  descending and then database index ascending (the paper is silent on ties;
  this order is the reading this build takes).
- ``score``/``score_pairs``/``all_scores`` with ``mode`` = "global",
  "semiglobal" or "overlap": the textbook variants of the same recurrences
  (first row and column, no zero floor, where the score is read) written
  out in ``modes.c``.
- ``align`` / ``align_pairs``: one optimal local alignment per pair, read
  off the same matrices by the traceback rules stated in ``traceback.c``
  (end cell first in row-major order; diagonal before E before F; a gap
  opens as soon as it can), plain C, int64.  With ``mode`` = "global",
  "semiglobal" or "overlap": the same rules on the matrices of ``modes.c``
  with the mode's end cell and boundary (``align_modes.c``).

Parity of every function here is pinned by tests/test_oracle_pins.py,
tests/test_oracle_mode_pins.py, tests/test_oracle_align_pins.py and
tests/test_oracle_align_mode_pins.py (brute-force enumeration, textbook
reductions, hand-worked examples, invariants, rescoring of the returned
alignments).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "gotoh.c"), os.path.join(_HERE, "traceback.c"), os.path.join(_HERE, "modes.c"),
         os.path.join(_HERE, "align_modes.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgotoh.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C files with gcc into oracle/_build/libgotoh.so."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(x) for x in _SRCS)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               *_SRCS, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.swo_score.restype = i64
            lib.swo_score.argtypes = [p, i64, p, i64, p, ctypes.c_int32, i64, i64]
            lib.swo_score_pairs.restype = ctypes.c_int
            lib.swo_score_pairs.argtypes = [p, p, p, p, p, p, i64, p, ctypes.c_int32, i64, i64,
                                            ctypes.c_int, p]
            lib.swo_score_mode.restype = i64
            lib.swo_score_mode.argtypes = [p, i64, p, i64, p, ctypes.c_int32, i64, i64, ctypes.c_int32]
            lib.swo_score_pairs_mode.restype = ctypes.c_int
            lib.swo_score_pairs_mode.argtypes = [p, p, p, p, p, p, i64, p, ctypes.c_int32, i64, i64, ctypes.c_int32,
                                                 ctypes.c_int, p]
            lib.swo_align.restype = i64
            lib.swo_align.argtypes = [p, i64, p, i64, p, ctypes.c_int32, i64, i64, p, p, p]
            lib.swo_align_mode.restype = ctypes.c_int
            lib.swo_align_mode.argtypes = [p, i64, p, i64, p, ctypes.c_int32, i64, i64, ctypes.c_int32, p, p, p, p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _matrix(S) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.int32)
    assert S.ndim == 2 and S.shape[0] == S.shape[1]
    return S


MODES = {"local": 0, "global": 1, "semiglobal": 2, "overlap": 3}


def _mode(mode) -> int:
    m = MODES.get(mode, mode) if isinstance(mode, str) else int(mode)
    if m not in MODES.values():
        raise ValueError(f"unknown alignment mode {mode!r}")
    return m


def score(q, t, S, gap_open: int, gap_extend: int, mode="local") -> int:
    """Alignment score of query q against target t (uint8 codes); local
    (Smith-Waterman) unless mode says otherwise."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.uint8)
    t = np.ascontiguousarray(t, dtype=np.uint8)
    S = _matrix(S)
    A = S.shape[0]
    if len(q) and int(q.max()) >= A or len(t) and int(t.max()) >= A:
        raise ValueError("residue code outside the matrix")
    md = _mode(mode)
    qq = q if len(q) else np.zeros(1, np.uint8)
    tt = t if len(t) else np.zeros(1, np.uint8)
    if md == 0:
        r = lib.swo_score(_ptr(qq), len(q), _ptr(tt), len(t), _ptr(S), A, int(gap_open), int(gap_extend))
        if r < 0:
            raise MemoryError("oracle scratch allocation failed")
    else:
        r = lib.swo_score_mode(_ptr(qq), len(q), _ptr(tt), len(t), _ptr(S), A, int(gap_open), int(gap_extend), md)
        if r == np.iinfo(np.int64).min:
            raise MemoryError("oracle scratch allocation failed")
    return int(r)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def score_pairs(queries, db, q_idx, t_idx, S, gap_open: int, gap_extend: int,
                threads: int | None = None, mode="local") -> np.ndarray:
    """Scores of the pairs (queries.seq(q_idx[k]), db.seq(t_idx[k])) as int64."""
    lib = _load()
    S = _matrix(S)
    q_idx = np.ascontiguousarray(q_idx, dtype=np.int64)
    t_idx = np.ascontiguousarray(t_idx, dtype=np.int64)
    assert q_idx.shape == t_idx.shape
    qres = np.ascontiguousarray(queries.residues, dtype=np.uint8)
    qoff = np.ascontiguousarray(queries.offsets, dtype=np.int64)
    tres = np.ascontiguousarray(db.residues, dtype=np.uint8)
    toff = np.ascontiguousarray(db.offsets, dtype=np.int64)
    if len(q_idx) and (q_idx.min() < 0 or q_idx.max() >= len(qoff) - 1
                       or t_idx.min() < 0 or t_idx.max() >= len(toff) - 1):
        raise IndexError("pair index out of range")
    A = S.shape[0]
    if (len(qres) and int(qres.max()) >= A) or (len(tres) and int(tres.max()) >= A):
        raise ValueError("residue code outside the matrix")
    out = np.empty(len(q_idx), dtype=np.int64)
    if len(q_idx) == 0:
        return out
    if qres.size == 0:
        qres = np.zeros(1, np.uint8)
    if tres.size == 0:
        tres = np.zeros(1, np.uint8)
    md = _mode(mode)
    if md == 0:
        rc = lib.swo_score_pairs(_ptr(qres), _ptr(qoff), _ptr(q_idx), _ptr(tres), _ptr(toff),
                                 _ptr(t_idx), len(q_idx), _ptr(S), A, int(gap_open), int(gap_extend),
                                 int(threads or default_threads()), _ptr(out))
        bad = (out < 0).any()
    else:
        rc = lib.swo_score_pairs_mode(_ptr(qres), _ptr(qoff), _ptr(q_idx), _ptr(tres), _ptr(toff),
                                      _ptr(t_idx), len(q_idx), _ptr(S), A, int(gap_open), int(gap_extend), md,
                                      int(threads or default_threads()), _ptr(out))
        bad = (out == np.iinfo(np.int64).min).any()
    if rc != 0 or bad:
        raise MemoryError("oracle failed")
    return out


def all_scores(queries, db, S, gap_open: int, gap_extend: int,
               threads: int | None = None, mode="local") -> np.ndarray:
    """(n_queries, n_db) matrix of scores, database in its original order."""
    nq, nt = queries.n, db.n
    qi = np.repeat(np.arange(nq, dtype=np.int64), nt)
    ti = np.tile(np.arange(nt, dtype=np.int64), nq)
    return score_pairs(queries, db, qi, ti, S, gap_open, gap_extend, threads, mode=mode).reshape(nq, nt)


def top_k(scores_row, k: int):
    """The k best entries of one query's score row.

    Order: score descending, then database index ascending.  Returns
    (scores, indices) as int64 arrays padded with -1 when k > len(row).
    """
    row = np.asarray(scores_row, dtype=np.int64)
    order = np.lexsort((np.arange(len(row)), -row))[:k]
    s = np.full(k, -1, dtype=np.int64)
    i = np.full(k, -1, dtype=np.int64)
    s[:len(order)] = row[order]
    i[:len(order)] = order
    return s, i


def align(q, t, S, gap_open: int, gap_extend: int, mode="local") -> dict:
    """One optimal alignment of query q against target t (uint8 codes), local
    unless mode says otherwise.

    Returns {"score", "q_begin", "q_end", "t_begin", "t_end", "ops"}: the
    alignment covers q[q_begin:q_end] and t[t_begin:t_end]; ops (uint8) run
    from its start to its end, 0 = M, 1 = I (query residue opposite a gap),
    2 = D (target residue opposite a gap).
    """
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.uint8)
    t = np.ascontiguousarray(t, dtype=np.uint8)
    S = _matrix(S)
    A = S.shape[0]
    if len(q) and int(q.max()) >= A or len(t) and int(t.max()) >= A:
        raise ValueError("residue code outside the matrix")
    md = _mode(mode)
    coords = np.zeros(4, dtype=np.int64)
    ops = np.zeros(max(len(q) + len(t), 1), dtype=np.uint8)
    n_ops = np.zeros(1, dtype=np.int64)
    qq = q if len(q) else np.zeros(1, np.uint8)
    tt = t if len(t) else np.zeros(1, np.uint8)
    if md == 0:
        r = lib.swo_align(_ptr(qq), len(q), _ptr(tt), len(t), _ptr(S), A, int(gap_open), int(gap_extend),
                          _ptr(coords), _ptr(ops), _ptr(n_ops))
        if r < 0:
            raise MemoryError("oracle scratch allocation failed")
    else:
        sc = np.zeros(1, dtype=np.int64)
        rc = lib.swo_align_mode(_ptr(qq), len(q), _ptr(tt), len(t), _ptr(S), A, int(gap_open), int(gap_extend),
                                md, _ptr(sc), _ptr(coords), _ptr(ops), _ptr(n_ops))
        if rc != 0:
            raise MemoryError("oracle scratch allocation failed")
        r = sc[0]
    return {"score": int(r), "q_begin": int(coords[0]), "q_end": int(coords[1]),
            "t_begin": int(coords[2]), "t_end": int(coords[3]), "ops": ops[:int(n_ops[0])].copy()}


def align_pairs(queries, db, q_idx, t_idx, S, gap_open: int, gap_extend: int,
                threads: int | None = None, mode="local") -> list:
    """``align`` of the pairs (queries.seq(q_idx[k]), db.seq(t_idx[k])), spread
    over threads (the C call releases the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor
    q_idx = [int(x) for x in q_idx]
    t_idx = [int(x) for x in t_idx]

    def one(k):
        return align(queries.seq(q_idx[k]), db.seq(t_idx[k]), S, gap_open, gap_extend, mode=mode)

    with ThreadPoolExecutor(max_workers=threads or default_threads()) as ex:
        return list(ex.map(one, range(len(q_idx))))
