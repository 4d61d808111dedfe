"""ctypes binding of libswdb.so: argument marshalling only.

Every function here has the name of the C entry point it calls (see
include/swdb.h for argument meaning, layouts, ownership and errors).  Host
buffers are numpy arrays; device buffers are torch CUDA tensors (torch is
only the device-memory and stream provider).  No arithmetic of the search
happens in Python.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SW_OK = 0
SW_PREC_AUTO, SW_PREC_I16, SW_PREC_I32 = 0, 1, 2
SW_MODE_AUTO, SW_MODE_PLAIN, SW_MODE_BATCHED = 0, 1, 2
SW_FLAG_GRAPH = 1
SW_ALIGN_LOCAL, SW_ALIGN_GLOBAL, SW_ALIGN_SEMIGLOBAL, SW_ALIGN_OVERLAP = 0, 1, 2, 3

HIT_DTYPE = np.dtype([("score", "<i4"), ("reserved", "<i4"), ("db_index", "<i8")])
SW_OP_M, SW_OP_I, SW_OP_D = 0, 1, 2
ALIGNMENT_DTYPE = np.dtype([("score", "<i4"), ("reserved", "<i4"), ("q_begin", "<i8"), ("q_end", "<i8"),
                            ("t_begin", "<i8"), ("t_end", "<i8"), ("ops_offset", "<i8"), ("ops_len", "<i8")])

_STATUS = {0: "SW_OK", 1: "SW_ERR_INVALID_ARG", 2: "SW_ERR_OOM", 3: "SW_ERR_CUDA", 4: "SW_ERR_TIMEOUT",
           5: "SW_ERR_OVERFLOW", 6: "SW_ERR_UNSUPPORTED"}


class SwError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_STATUS.get(code, code)}: {message}")
        self.code = code


class SwSearchOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("mode", ctypes.c_int32), ("long_cutoff", ctypes.c_int64),
                ("lanes", ctypes.c_int32), ("rows_per_lane", ctypes.c_int32),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t), ("flags", ctypes.c_int32),
                ("long_rows_per_lane", ctypes.c_int32), ("alignment", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("status_out", ctypes.c_void_p)]


class SwSearchStats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("rescored", ctypes.c_int64), ("long_sequences", ctypes.c_int64),
                ("precision_used", ctypes.c_int32), ("mode_used", ctypes.c_int32),
                ("lanes_used", ctypes.c_int32), ("rows_per_lane_used", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("inter_ms", ctypes.c_float), ("rescore_ms", ctypes.c_float),
                ("intra_ms", ctypes.c_float), ("other_ms", ctypes.c_float), ("inter_launches", ctypes.c_int32),
                ("inter_cells", ctypes.c_int64), ("long_cells", ctypes.c_int64),
                ("graph_replayed", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class SwAlignStats(ctypes.Structure):
    _fields_ = [("forward_cells", ctypes.c_int64), ("traceback_cells", ctypes.c_int64),
                ("forward_ms", ctypes.c_float), ("traceback_ms", ctypes.c_float), ("launches", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SwShapeRate(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("rows_per_lane", ctypes.c_int32), ("gcups", ctypes.c_float)]


SW_TUNING_MAX_SHAPES = 16


class SwTuning(ctypes.Structure):
    _fields_ = [("n_plain", ctypes.c_int32), ("n_batched", ctypes.c_int32),
                ("plain", SwShapeRate * SW_TUNING_MAX_SHAPES), ("batched", SwShapeRate * SW_TUNING_MAX_SHAPES),
                ("long_cutoff", ctypes.c_int64), ("long_rows_per_lane", ctypes.c_int32), ("mode", ctypes.c_int32)]


class SwDbInfo(ctypes.Structure):
    _fields_ = [("n_seqs", ctypes.c_int64), ("residues", ctypes.c_int64), ("max_length", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("alphabet_size", ctypes.c_int32), ("device", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load libswdb.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.sw_db_load.argtypes = [vp, vp, i64, i32, ctypes.c_int, ctypes.POINTER(vp)]
    lib.sw_db_free.argtypes = [vp]
    lib.sw_db_get_info.argtypes = [vp, ctypes.POINTER(SwDbInfo)]
    lib.sw_search_workspace_size.argtypes = [vp, vp, i32, i32, ctypes.POINTER(SwSearchOpts), ctypes.POINTER(sz)]
    lib.sw_search.argtypes = [vp, vp, vp, i32, vp, i32, i32, i32, vp, vp, ctypes.POINTER(SwSearchOpts),
                              ctypes.POINTER(SwSearchStats), vp]
    lib.sw_top_k.argtypes = [vp, i64, i64, i32, vp, vp]
    lib.sw_probe_alu_rate.argtypes = [ctypes.c_int, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
    lib.sw_search_no_alloc.argtypes = [vp, vp, i32, vp, i32, i32, vp, vp]
    lib.sw_probe_wait_timeout.argtypes = [ctypes.c_int, i64, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
    lib.sw_align_ops_capacity.argtypes = [vp, vp, i32, vp, vp, i64, ctypes.POINTER(i64)]
    lib.sw_align.argtypes = [vp, vp, vp, i32, vp, vp, i64, vp, i32, i32, vp, vp, i64,
                             ctypes.POINTER(SwAlignStats), vp]
    lib.sw_align_mode.argtypes = [vp, vp, vp, i32, vp, vp, i64, vp, i32, i32, i32, vp, vp, i64,
                                  ctypes.POINTER(SwAlignStats), vp]
    lib.sw_align_mode.restype = ctypes.c_int
    lib.sw_db_set_tuning.argtypes = [vp, ctypes.POINTER(SwTuning)]
    lib.sw_db_get_tuning.argtypes = [vp, ctypes.POINTER(SwTuning)]
    lib.sw_shard_plan.argtypes = [vp, i64, i32, vp, vp]
    lib.sw_hits_merge.argtypes = [vp, vp, vp, i32, i32, i32, vp]
    lib.sw_scores_scatter.argtypes = [vp, vp, i64, i32, i64, vp]
    for name in ("sw_align", "sw_align_ops_capacity", "sw_probe_wait_timeout", "sw_shard_plan", "sw_hits_merge",
                 "sw_scores_scatter", "sw_db_set_tuning", "sw_db_get_tuning"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("sw_db_load", "sw_db_free", "sw_db_get_info", "sw_search_workspace_size", "sw_search",
                 "sw_top_k", "sw_probe_alu_rate", "sw_search_no_alloc"):
        getattr(lib, name).restype = ctypes.c_int
    lib.sw_last_error.restype = ctypes.c_char_p
    lib.sw_last_error.argtypes = []
    lib.sw_version.restype = ctypes.c_char_p
    lib.sw_version.argtypes = []
    _lib = lib
    return lib


def sw_last_error() -> str:
    return load_library().sw_last_error().decode()


def sw_version() -> str:
    return load_library().sw_version().decode()


def _check(rc: int):
    if rc != SW_OK:
        raise SwError(rc, sw_last_error())


def _is_tensor(x) -> bool:
    return type(x).__module__.startswith("torch") and hasattr(x, "data_ptr")


def _addr(x, dtype, name: str):
    """(address, is_cuda) of a contiguous numpy array or torch tensor."""
    if x is None:
        return None, False
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError(f"{name} must be C-contiguous")
        if dtype is not None and x.dtype != dtype:
            raise TypeError(f"{name} must have dtype {dtype}, got {x.dtype}")
        return (x.ctypes.data if x.size else None), False
    if _is_tensor(x):
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if dtype is not None:
            import torch
            want = {np.dtype(np.uint8): torch.uint8, np.dtype(np.int32): torch.int32,
                    np.dtype(np.int64): torch.int64}.get(np.dtype(dtype))
            if want is not None and x.dtype != want:
                raise TypeError(f"{name} must have dtype {want}, got {x.dtype}")
        return (x.data_ptr() if x.numel() else None), bool(x.is_cuda)
    raise TypeError(f"{name}: expected a numpy array or torch tensor, got {type(x)}")


def sw_db_load(residues: np.ndarray, offsets: np.ndarray, alphabet_size: int, device: int = 0):
    """Upload a database; returns the opaque handle (a ctypes void pointer)."""
    lib = load_library()
    residues = np.ascontiguousarray(residues, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    h = ctypes.c_void_p()
    rp = residues.ctypes.data if residues.size else None
    _check(lib.sw_db_load(rp, offsets.ctypes.data, len(offsets) - 1, alphabet_size, device, ctypes.byref(h)))
    return h


def sw_db_free(handle) -> None:
    if handle:
        _check(load_library().sw_db_free(handle))


def sw_db_get_info(handle) -> dict:
    info = SwDbInfo()
    _check(load_library().sw_db_get_info(handle, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in SwDbInfo._fields_}


def sw_db_set_tuning(handle, tuning: dict | None) -> None:
    """Install a launch tuning on a handle, or None for the library's tables.
    tuning: {"plain": [(lanes, rows, gcups), ...], "batched": [...],
    "long_cutoff": int, "long_rows_per_lane": int, "mode": int} (keys optional)."""
    if tuning is None:
        _check(load_library().sw_db_set_tuning(handle, None))
        return
    t = SwTuning()
    for key, arr, count in (("plain", t.plain, "n_plain"), ("batched", t.batched, "n_batched")):
        rows = list(tuning.get(key, []))
        if len(rows) > SW_TUNING_MAX_SHAPES:
            raise ValueError(f"at most {SW_TUNING_MAX_SHAPES} {key} shapes")
        for i, (l, r, g) in enumerate(rows):
            arr[i].lanes, arr[i].rows_per_lane, arr[i].gcups = int(l), int(r), float(g)
        setattr(t, count, len(rows))
    t.long_cutoff = int(tuning.get("long_cutoff", 0))
    t.long_rows_per_lane = int(tuning.get("long_rows_per_lane", 0))
    t.mode = int(tuning.get("mode", 0))
    _check(load_library().sw_db_set_tuning(handle, ctypes.byref(t)))


def sw_db_get_tuning(handle) -> dict:
    """The handle's active tuning (the library's tables when none is installed)."""
    t = SwTuning()
    _check(load_library().sw_db_get_tuning(handle, ctypes.byref(t)))
    return {"plain": [(t.plain[i].lanes, t.plain[i].rows_per_lane, float(t.plain[i].gcups)) for i in range(t.n_plain)],
            "batched": [(t.batched[i].lanes, t.batched[i].rows_per_lane, float(t.batched[i].gcups))
                        for i in range(t.n_batched)],
            "long_cutoff": int(t.long_cutoff), "long_rows_per_lane": int(t.long_rows_per_lane), "mode": int(t.mode)}


def _opts(precision, mode, long_cutoff, lanes, rows_per_lane, workspace, flags=0, long_rows_per_lane=0,
          alignment=SW_ALIGN_LOCAL, status_out=None):
    o = SwSearchOpts()
    if status_out is not None:
        addr, is_cuda = _addr(status_out, np.int32, "status_out")
        if not is_cuda and not (_is_tensor(status_out) and status_out.is_pinned()):
            raise ValueError("status_out must be a CUDA tensor or a pinned host tensor (int32)")
        o.status_out = addr
    o.alignment = alignment
    o.flags = flags
    o.long_rows_per_lane = long_rows_per_lane
    o.precision = precision
    o.mode = mode
    o.long_cutoff = long_cutoff
    o.lanes = lanes
    o.rows_per_lane = rows_per_lane
    if workspace is not None:
        addr, is_cuda = _addr(workspace, None, "workspace")
        if not is_cuda:
            raise ValueError("workspace must be a CUDA tensor")
        o.workspace = addr
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def sw_search_workspace_size(handle, q_offsets, top_k: int, precision=SW_PREC_AUTO, mode=SW_MODE_AUTO,
                             long_cutoff=0, lanes=0, rows_per_lane=0, long_rows_per_lane=0,
                             alignment=SW_ALIGN_LOCAL) -> int:
    q_offsets = np.ascontiguousarray(q_offsets, dtype=np.int64)
    o = _opts(precision, mode, long_cutoff, lanes, rows_per_lane, None, 0, long_rows_per_lane, alignment)
    n = ctypes.c_size_t()
    _check(load_library().sw_search_workspace_size(handle, q_offsets.ctypes.data, len(q_offsets) - 1, top_k,
                                                   ctypes.byref(o), ctypes.byref(n)))
    return int(n.value)


def sw_search(handle, queries, q_offsets, matrix, gap_open: int, gap_extend: int, top_k: int,
              scores_out=None, hits_out=None, precision=SW_PREC_AUTO, mode=SW_MODE_AUTO, long_cutoff=0,
              lanes=0, rows_per_lane=0, workspace=None, stats: bool = False, stream=None, graph: bool = False,
              long_rows_per_lane=0, alignment=SW_ALIGN_LOCAL, status_out=None):
    """Run sw_search.  Outputs are written into scores_out / hits_out (numpy =
    host, torch CUDA tensor = device).  Returns a stats dict when stats=True.
    status_out (an int32 CUDA or pinned tensor) receives the device-side status
    on the stream: 0, or SW_ERR_TIMEOUT when a bounded wait gave up."""
    lib = load_library()
    q_offsets = np.ascontiguousarray(q_offsets, dtype=np.int64)
    matrix = np.ascontiguousarray(matrix, dtype=np.int32)
    qp, q_cuda = _addr(queries, np.uint8, "queries")
    sp, s_cuda = _addr(scores_out, np.int32, "scores_out")
    if hits_out is not None and isinstance(hits_out, np.ndarray) and hits_out.dtype != HIT_DTYPE:
        raise TypeError("hits_out must have dtype HIT_DTYPE")
    hp, h_cuda = _addr(hits_out, None, "hits_out")
    o = _opts(precision, mode, long_cutoff, lanes, rows_per_lane, workspace, SW_FLAG_GRAPH if graph else 0,
              long_rows_per_lane, alignment, status_out)
    st = SwSearchStats() if stats else None
    if stream is None and (q_cuda or s_cuda or h_cuda or workspace is not None or status_out is not None):
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    rc = lib.sw_search(handle, qp, q_offsets.ctypes.data, len(q_offsets) - 1, matrix.ctypes.data,
                       int(gap_open), int(gap_extend), int(top_k), sp, hp, ctypes.byref(o),
                       ctypes.byref(st) if st is not None else None, stream)
    _check(rc)
    if st is not None:
        return {f: getattr(st, f) for f, _ in SwSearchStats._fields_}
    return None


def sw_top_k(scores, n_rows: int, n_cols: int, top_k: int, hits, stream=None) -> None:
    """Top-k of device score rows into device hits (both torch CUDA tensors)."""
    sp, s_cuda = _addr(scores, np.int32, "scores")
    hp, h_cuda = _addr(hits, None, "hits")
    if (sp is not None and not s_cuda) or not h_cuda:
        raise ValueError("sw_top_k takes device buffers")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(load_library().sw_top_k(sp, n_rows, n_cols, top_k, hp, stream))


def sw_probe_alu_rate(device: int = 0, mode: int = 0):
    """(rate per SM cycle, SM count): mode 0 = int16x2 DPX add-max ops,
    mode 1 = inter-task cell updates from registers."""
    rate = ctypes.c_double()
    sms = ctypes.c_int32()
    _check(load_library().sw_probe_alu_rate(device, mode, ctypes.byref(rate), ctypes.byref(sms)))
    return float(rate.value), int(sms.value)


def sw_probe_wait_timeout(device: int = 0, spin_iters: int = 100000):
    """Run the kernels' bounded wait on a flag nothing sets; returns
    (status recorded by the kernel, elapsed ms).  SW_ERR_TIMEOUT (4) means the
    wait gave up as designed."""
    st = ctypes.c_int32(0)
    ms = ctypes.c_double(0.0)
    _check(load_library().sw_probe_wait_timeout(int(device), int(spin_iters), ctypes.byref(st), ctypes.byref(ms)))
    return st.value, ms.value


def sw_search_no_alloc(handle, query, matrix, gap_open: int, gap_extend: int, scores, stream=None) -> None:
    """One query (torch CUDA uint8 tensor) against a loaded database into a
    device score row (torch CUDA int32 tensor of n_seqs), with no device
    allocation during the call.  For callers that cannot allocate at search
    time (inside CUDA graph capture, allocation-free serving loops, memory
    owned by another pool); scratch is a fixed library-owned device array."""
    qp, q_cuda = _addr(query, np.uint8, "query")
    sp, s_cuda = _addr(scores, np.int32, "scores")
    if (qp is not None and not q_cuda) or not s_cuda:
        raise ValueError("sw_search_no_alloc takes device buffers")
    matrix = np.ascontiguousarray(matrix, dtype=np.int32)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    m = query.numel() if query is not None else 0
    _check(load_library().sw_search_no_alloc(handle, qp, m, matrix.ctypes.data, int(gap_open), int(gap_extend),
                                             sp, stream))


def _pairs(pair_query, pair_target):
    pq = np.ascontiguousarray(pair_query, dtype=np.int32)
    pt = np.ascontiguousarray(pair_target, dtype=np.int64)
    if pq.shape != pt.shape or pq.ndim != 1:
        raise ValueError("pair_query and pair_target must be 1-D arrays of the same length")
    return pq, pt


def sw_align_ops_capacity(handle, q_offsets, pair_query, pair_target) -> int:
    q_offsets = np.ascontiguousarray(q_offsets, dtype=np.int64)
    pq, pt = _pairs(pair_query, pair_target)
    out = ctypes.c_int64(0)
    _check(load_library().sw_align_ops_capacity(handle, q_offsets.ctypes.data, len(q_offsets) - 1,
                                                pq.ctypes.data if len(pq) else None,
                                                pt.ctypes.data if len(pt) else None, len(pq), ctypes.byref(out)))
    return out.value


def sw_align(handle, queries, q_offsets, pair_query, pair_target, matrix, gap_open: int, gap_extend: int,
             stats: bool = False, stream=None, alignment=SW_ALIGN_LOCAL):
    """Alignments of the pairs (query pair_query[k], database sequence
    pair_target[k]), local unless alignment names another mode (then
    sw_align_mode).  Returns (alignments ALIGNMENT_DTYPE [n_pairs], ops uint8,
    stats dict or None); pair k's ops are ops[ops_offset : ops_offset + ops_len]."""
    q_offsets = np.ascontiguousarray(q_offsets, dtype=np.int64)
    pq, pt = _pairs(pair_query, pair_target)
    qp, _ = _addr(queries, np.uint8, "queries")
    matrix = np.ascontiguousarray(matrix, dtype=np.int32)
    cap = sw_align_ops_capacity(handle, q_offsets, pq, pt)
    aln = np.zeros(len(pq), dtype=ALIGNMENT_DTYPE)
    ops = np.zeros(max(cap, 1), dtype=np.uint8)
    st = SwAlignStats()
    _check(load_library().sw_align_mode(handle, qp, q_offsets.ctypes.data, len(q_offsets) - 1,
                                        pq.ctypes.data if len(pq) else None, pt.ctypes.data if len(pt) else None,
                                        len(pq), matrix.ctypes.data, int(gap_open), int(gap_extend), int(alignment),
                                        aln.ctypes.data if len(pq) else None, ops.ctypes.data, cap,
                                        ctypes.byref(st) if stats else None, stream))
    sd = {f: getattr(st, f) for f, _ in SwAlignStats._fields_} if stats else None
    return aln, ops[:cap], sd


def sw_shard_plan(offsets, n_shards: int):
    """Partition a database (offsets, host) into n_shards residue-balanced,
    length-stratified shards.  Returns (members int64 [n_seqs], member_offsets
    int64 [n_shards + 1]); shard s is members[member_offsets[s]:member_offsets[s+1]]
    (the caller's indices, increasing)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = len(offsets) - 1
    members = np.zeros(max(n, 1), dtype=np.int64)
    moff = np.zeros(int(n_shards) + 1 if n_shards > 0 else 1, dtype=np.int64)
    _check(load_library().sw_shard_plan(offsets.ctypes.data, n, int(n_shards), members.ctypes.data, moff.ctypes.data))
    return members[:n], moff


def sw_hits_merge(shard_hits, members, member_offsets, top_k: int) -> np.ndarray:
    """Merge shards' top-k lists (HIT_DTYPE [n_shards, n_q, top_k], shard-local
    indices) into the unsharded top-k (HIT_DTYPE [n_q, top_k], caller's indices)."""
    shard_hits = np.ascontiguousarray(shard_hits, dtype=HIT_DTYPE)
    members = np.ascontiguousarray(members, dtype=np.int64)
    moff = np.ascontiguousarray(member_offsets, dtype=np.int64)
    n_shards, n_q = shard_hits.shape[0], shard_hits.shape[1]
    if shard_hits.shape[2] != top_k or len(moff) != n_shards + 1:
        raise ValueError("shard_hits must be [n_shards, n_q, top_k] and member_offsets n_shards + 1 long")
    out = np.zeros((n_q, top_k), dtype=HIT_DTYPE)
    _check(load_library().sw_hits_merge(shard_hits.ctypes.data if shard_hits.size else None,
                                        members.ctypes.data if members.size else None, moff.ctypes.data,
                                        n_shards, n_q, int(top_k), out.ctypes.data if out.size else None))
    return out


def sw_scores_scatter(shard_scores, members, scores_out) -> None:
    """Write one shard's score rows (int32 [n_q, n_members]) into the columns
    `members` of the unsharded table scores_out (int32 [n_q, n_seqs], host)."""
    shard_scores = np.ascontiguousarray(shard_scores, dtype=np.int32)
    members = np.ascontiguousarray(members, dtype=np.int64)
    if not (isinstance(scores_out, np.ndarray) and scores_out.dtype == np.int32 and scores_out.flags.c_contiguous):
        raise TypeError("scores_out must be a C-contiguous int32 numpy array")
    n_q, n_seqs = scores_out.shape
    if shard_scores.shape != (n_q, len(members)):
        raise ValueError("shard_scores must be [n_q, len(members)]")
    _check(load_library().sw_scores_scatter(shard_scores.ctypes.data if shard_scores.size else None,
                                            members.ctypes.data if members.size else None, len(members), n_q,
                                            n_seqs, scores_out.ctypes.data if scores_out.size else None))


class ShardedDatabase:
    """A database split into residue-balanced shards (sw_shard_plan), one
    resident handle per shard; shard s lives on devices[s % len(devices)].
    search() runs the full query batch on every shard and merges: top-k by
    sw_hits_merge, score rows by sw_scores_scatter.  Results equal an
    unsharded search's, ties included."""

    def __init__(self, residues, offsets, alphabet_size: int, n_shards: int, devices=(0,)):
        residues = np.ascontiguousarray(residues, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n_seqs = len(offsets) - 1
        self.members, self.member_offsets = sw_shard_plan(offsets, n_shards)
        self.shards = []
        try:
            for s in range(n_shards):
                idx = self.members[self.member_offsets[s]:self.member_offsets[s + 1]]
                lens = offsets[idx + 1] - offsets[idx]
                off = np.zeros(len(idx) + 1, dtype=np.int64)
                np.cumsum(lens, out=off[1:])
                res = (np.concatenate([residues[offsets[i]:offsets[i + 1]] for i in idx]) if len(idx)
                       else np.zeros(0, np.uint8))
                self.shards.append(Database(res, off, alphabet_size, device=devices[s % len(devices)]))
        except Exception:
            self.close()
            raise

    def shard_members(self, s: int) -> np.ndarray:
        return self.members[self.member_offsets[s]:self.member_offsets[s + 1]]

    def search(self, queries, q_offsets, matrix, gap_open: int, gap_extend: int, top_k: int = 10,
               want_scores: bool = True, **kw):
        """Returns (scores [n_q, n_seqs] int32 or None, hits [n_q, top_k] HIT_DTYPE)."""
        nq = len(q_offsets) - 1
        scores = np.empty((nq, self.n_seqs), dtype=np.int32) if want_scores else None
        shard_hits = np.empty((len(self.shards), nq, max(top_k, 0)), dtype=HIT_DTYPE)
        for s, d in enumerate(self.shards):
            sc, h, _ = d.search(queries, q_offsets, matrix, gap_open, gap_extend, top_k=top_k,
                                want_scores=want_scores, **kw)
            if top_k > 0:
                shard_hits[s] = h
            if want_scores:
                sw_scores_scatter(sc, self.shard_members(s), scores)
        hits = sw_hits_merge(shard_hits, self.members, self.member_offsets, top_k) if top_k > 0 else None
        return scores, hits

    def close(self):
        for d in getattr(self, "shards", []):
            d.close()
        self.shards = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Database:
    """A resident database (wraps sw_db_load / sw_search / sw_db_free)."""

    def __init__(self, residues, offsets, alphabet_size: int, device: int = 0):
        self.handle = sw_db_load(residues, offsets, alphabet_size, device)
        self.n_seqs = len(offsets) - 1
        self.device = device

    def info(self) -> dict:
        return sw_db_get_info(self.handle)

    def search(self, queries, q_offsets, matrix, gap_open: int, gap_extend: int, top_k: int = 10,
               want_scores: bool = True, on_device: bool = False, **kw):
        """Returns (scores [n_q, n_seqs] int32, hits [n_q, top_k] HIT_DTYPE, stats or None).
        on_device=True returns torch CUDA tensors (hits as int64 [n_q, top_k, 2] view)."""
        nq = len(q_offsets) - 1
        if on_device:
            import torch
            dev = torch.device("cuda", self.device)
            scores = torch.empty((nq, self.n_seqs), dtype=torch.int32, device=dev) if want_scores else None
            hits = torch.empty((nq, max(top_k, 0), 2), dtype=torch.int64, device=dev) if top_k > 0 else None
        else:
            scores = np.empty((nq, self.n_seqs), dtype=np.int32) if want_scores else None
            hits = np.empty((nq, max(top_k, 0)), dtype=HIT_DTYPE) if top_k > 0 else None
        stats = sw_search(self.handle, queries, q_offsets, matrix, gap_open, gap_extend, top_k, scores, hits, **kw)
        return scores, hits, stats

    def align(self, queries, q_offsets, pair_query, pair_target, matrix, gap_open: int, gap_extend: int,
              stats: bool = False, alignment=SW_ALIGN_LOCAL):
        """Alignments of chosen (query, database sequence) pairs: see sw_align and sw_align_mode."""
        return sw_align(self.handle, queries, q_offsets, pair_query, pair_target, matrix, gap_open, gap_extend,
                        stats=stats, alignment=alignment)

    def close(self):
        if getattr(self, "handle", None):
            sw_db_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
