#!/usr/bin/env python
"""GCUPS benchmark of exhaustive Smith-Waterman/Gotoh protein database search.

One step = the whole hot path over one batch: every query of the workload
scored against every database sequence (int16x2 inter-task kernel, int32
rescore of saturated pairs, top-k), database resident in HBM.  The metric is
giga cell updates per second (Section 4.2 of the paper uses GCUPS), device
timed with CUDA events; the result is bit-exact with the CPU oracle
(checked on the sampled pairs of the cpu_baseline leg and in tests/).

Default workload (N=1): 20 queries of lengths 144..5478 (log grid) vs a
synthetic 565,000-sequence database (lognormal mean 360, 2..35,000, one of
35,000), BLOSUM62, gap 10/1, top 10: the shape of the paper's Swiss-Prot
experiment (Section 4.1) with seeded synthetic residues.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) the database is sharded: every rank loads one
residue-balanced, length-stratified shard (sw_shard_plan) on its own GPU and
scores the whole query batch against it; the one exchange step all-gathers
each shard's top-k and merges them (sw_hits_merge).  The total work is fixed
("strong" scaling); rank 0 prints one JSON line.  --multi replicas instead
gives every rank its own query batch against a full copy of the database
(independent problems, "weak" scaling).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "GCUPS (device-timed, bit-exact vs oracle)"
UNIT = "GCUPS"
# Minimum packed int16x2 DPX operations per cell update of the recurrences:
# E, F, H (2), H-o, running max per cell pair = 5.5 per 2 cells.
DPX_OPS_PER_CELL = 2.75
I32_DPX_OPS_PER_CELL = 3.0
# Non-local modes in packed int16x2: E, F, H (2) and the profile permute per
# cell pair, no running max over the matrix = 5 per 2 cells.
MODES16_OPS_PER_CELL = 2.5
# Batched form (two queries against one database sequence): the profile is a
# ready int16x2 word per row, no byte permute: 4.5 per cell pair.
BATCH_OPS_PER_CELL = 2.25
ALIGNMENTS = {"local": 0, "global": 1, "semiglobal": 2, "overlap": 3}
RESULT_TIMEOUT_S = 300.0   # a served request that takes longer than this is a failure


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="swissprot_like_20q", choices=sorted(synth.WORKLOADS))
    p.add_argument("--db-scale", type=float, default=1.0, help="fraction of the database (1.0 = full size)")
    p.add_argument("--lanes", type=int, default=0)
    p.add_argument("--rows", type=int, default=0)
    p.add_argument("--precision", type=int, default=0)
    p.add_argument("--long-rows", type=int, default=0, help="rows per lane of the intra-task kernel (8, 16 or 32)")
    p.add_argument("--long-cutoff", type=int, default=0,
                   help="database sequences longer than this go to the intra-task kernel (0 = library default)")
    p.add_argument("--mode", choices=["plain", "batched"], default="plain",
                   help="plain: one inter-task launch per query (the paper's form); "
                        "batched: all queries in one persistent launch")
    p.add_argument("--autotune", choices=["auto", "on", "off"], default="auto",
                   help="measure the launch tuning (shape rate tables, cutoff, form) on this GPU and database "
                        "before timing: auto = for the batched form and the serving loop")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--serve", action="store_true",
                   help="serving benchmark: Poisson request stream against a resident database "
                        "(continuous batching), reports p50/p99 latency and sustained GCUPS")
    p.add_argument("--serve-db-scale", type=float, default=0.1,
                   help="fraction of the 20M-sequence serving database (0.1 = 2M sequences)")
    p.add_argument("--serve-requests", type=int, default=96)
    p.add_argument("--serve-max-batch", type=int, default=32,
                   help="most requests per batch (the server's default; larger batches pair queries of closer "
                        "lengths)")
    p.add_argument("--serve-point-requests", type=int, default=0,
                   help="requests per Poisson load point (0 = half of --serve-requests)")
    p.add_argument("--serve-check", type=int, default=8,
                   help="served requests whose hits are checked against the oracle's scores and against a plain "
                        "search of the same query")
    p.add_argument("--graph", action="store_true",
                   help="capture the search into a CUDA graph on the first call and replay it")
    p.add_argument("--alignment", choices=["local", "global", "semiglobal", "overlap"], default="local",
                   help="alignment mode of the search (local = Smith-Waterman, the paper's)")
    p.add_argument("--sweep", action="store_true",
                   help="GCUPS against query length: each query of the workload searched alone, at the "
                        "workload's gap penalties and at 10/2")
    p.add_argument("--align", action="store_true",
                   help="traceback benchmark: align the top-k hits of the workload's search")
    p.add_argument("--sub-records", default="auto",
                   help="other workloads timed after the main one, each reported with its own roofline, clocks "
                        "and oracle sample: comma list of db2k_q100, long_4q_50k, batched_512q (batched and "
                        "plain forms), 'none', or 'auto' (all of them on one GPU for the default workload)")
    p.add_argument("--sub-steps", type=int, default=0, help="timed steps of every sub-record (0 = per workload)")
    p.add_argument("--sub-warmup", type=int, default=-1, help="warm-up steps of every sub-record (-1 = per workload)")
    p.add_argument("--multi", choices=["shard", "replicas"], default="shard",
                   help="with N > 1 ranks: shard the database (strong scaling, the default) or run "
                        "independent replicas with their own queries (weak scaling)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-cells", type=float, default=6e10,
                   help="cells of the oracle's bounded sample (about 10-20 s on 16 cores)")
    return p.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed helpers (torchrun); single-process runs skip them

class Dist:
    """Rank, world and device of this process.  Each local rank takes GPU
    local_rank (modulo the GPUs visible, so more ranks than GPUs share them
    round-robin); the process group is NCCL when every local rank has a GPU
    of its own, else gloo."""

    def __init__(self, backend: str | None = None, init: bool = True):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.local_world = int(os.environ.get("LOCAL_WORLD_SIZE", str(self.world)))
        self.pg = None
        self.backend = None
        self.device = self.local_rank
        try:
            import torch
            n_dev = torch.cuda.device_count() if torch.cuda.is_available() else 0
        except Exception:
            n_dev = 0
        if n_dev > 0:
            self.device = self.local_rank % n_dev
        if self.world > 1 and init:
            import torch.distributed as dist
            if backend is None:
                backend = "nccl" if n_dev >= self.local_world else "gloo"
            if backend == "nccl":
                import torch
                torch.cuda.set_device(self.device)
            dist.init_process_group(backend=backend)
            self.pg = dist
            self.backend = backend

    def _tensor(self, x):
        import torch
        dev = "cuda" if self.pg is not None and self.backend == "nccl" else "cpu"
        return torch.tensor([float(x)], dtype=torch.float64, device=dev)

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if self.pg is None:
            return float(x)
        t = self._tensor(x)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if self.pg is None:
            return float(x)
        t = self._tensor(x)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


def combine_ranks(dist: Dist, local_ms: float, local_cells: float):
    """Whole-job throughput: cells of all ranks over the slowest rank's time."""
    t = dist.max(local_ms)
    cells = dist.sum(local_cells)
    return t, cells, (cells / (t * 1e-3) / 1e9 if t > 0 else 0.0)


# ---------------------------------------------------------------------------
# clocks during the timed region

def smi_gpu_id(device: int) -> str:
    """An nvidia-smi --id that names the same GPU as CUDA device `device`.

    nvidia-smi ignores CUDA_VISIBLE_DEVICES, so a CUDA ordinal can name
    another GPU of the machine; the device UUID (or else its PCI bus id)
    names this one."""
    import torch
    p = torch.cuda.get_device_properties(device)
    uuid = getattr(p, "uuid", None)
    if uuid is not None:
        u = str(uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    dom, bus, dv = (getattr(p, k, None) for k in ("pci_domain_id", "pci_bus_id", "pci_device_id"))
    if bus is not None:
        return f"{int(dom or 0):08x}:{int(bus):02x}:{int(dv or 0):02x}.0"
    return str(device)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        try:
            self.gpu = smi_gpu_id(device)
        except Exception:
            self.gpu = str(device)
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "gpu": self.gpu}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            # timed region shorter than one sampling period: read the clocks once now
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", "--query-gpu=clocks.sm,clocks.max.sm",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=10).stdout.split(",")
                return {"sm_mhz": float(out[0]), "sm_max_mhz": float(out[1]), "reasons": sorted(reasons),
                        "samples": 0, "gpu": self.gpu, "note": "timed region shorter than the 200 ms sampling "
                                                               "period; clocks read once right after it"}
            except Exception:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "gpu": self.gpu}


# ---------------------------------------------------------------------------

def launch_key(args) -> str:
    """The launch configuration a DRAM-traffic record was measured under."""
    key = (f"{args.workload}/scale{args.db_scale:g}/{args.mode}/lanes{args.lanes}/rows{args.rows}"
           f"/prec{args.precision}/longrows{args.long_rows}/cutoff{args.long_cutoff}")
    alignment = getattr(args, "alignment", "local")
    return key if alignment == "local" else key + f"/{alignment}"


def traffic_per_launch(args):
    """Average DRAM bytes (read + written) per launch of the step's dominant
    kernel, from the committed ncu record of every launch of one step of this
    same launch configuration, if it was taken on the current source of that
    kernel (the record's source= file, k_inter16.cu when absent; else None)."""
    csrc = os.path.join(ROOT, "paper_2203_11100_gb300", "csrc")
    try:
        key = launch_key(args)
        for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
            for line in open(path):
                if not line.startswith("traffic:"):
                    continue
                rec = dict(kv.split("=", 1) for kv in line.split()[1:])
                if rec.get("launch") != key:
                    continue
                src = os.path.join(csrc, os.path.basename(rec.get("source", "k_inter16.cu")))
                if rec.get("source_sha256") == hashlib.sha256(open(src, "rb").read()).hexdigest():
                    return float(rec["dram_bytes_per_launch"])
    except Exception:
        return None
    return None


def cpu_baseline(w, gpu_scores, seed: int, target_cells: float, mode: str = "local"):
    """Time the oracle (as it stands) on a bounded sample of the workload, on
    all host cores, and check the GPU's scores for the same pairs."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    qlen = w.queries.lengths.astype(np.float64)
    mean_t = float(w.db.lengths.mean()) if w.db.n else 1.0
    per_query = max(1, int(target_cells / max(qlen.sum(), 1.0) / max(mean_t, 1.0)))
    per_query = min(per_query, w.db.n)
    t_idx = np.sort(rng.choice(w.db.n, size=per_query, replace=False)) if w.db.n else np.zeros(0, np.int64)
    qi = np.repeat(np.arange(w.queries.n, dtype=np.int64), len(t_idx))
    ti = np.tile(t_idx.astype(np.int64), w.queries.n)
    cells = float((qlen[qi] * w.db.lengths[ti]).sum())
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    got = oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend, threads=threads, mode=mode)
    dt = time.perf_counter() - t0
    exact = None
    if gpu_scores is not None:
        exact = bool(np.array_equal(got, gpu_scores[qi, ti].astype(np.int64)))
    return {"value": cells / dt / 1e9 if dt > 0 else 0.0, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"all {w.queries.n} queries x {len(t_idx)} random database sequences "
                      f"({cells:.3g} cells, {dt:.1f} s)",
            "sample_bit_exact_vs_gpu": exact}


def run_ours(args, dist: Dist):
    import torch
    import paper_2203_11100_gb300 as swdb

    dev = dist.device
    torch.cuda.set_device(dev)
    swdb.load_library()
    seed = synth.SEED + 7919 * dist.rank
    w = synth.make_workload(args.workload, seed=synth.SEED, db_scale=args.db_scale)
    if dist.rank:
        # independent query batch per rank, same shape
        alt = synth.make_workload(args.workload, seed=seed, db_scale=args.db_scale)
        w.queries = alt.queries
    nq, n = w.queries.n, w.db.n
    cells_step = float(w.cells)
    db = swdb.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET), device=dev)
    # A stream of its own, so that the CUDA events bracket the searches on the
    # stream they run on (the legacy default stream's handle is NULL, which the
    # library reads as "the handle's own stream").
    stream = torch.cuda.Stream(device=dev)
    q_dev = torch.from_numpy(w.queries.residues).to(f"cuda:{dev}")
    scores = torch.empty((nq, n), dtype=torch.int32, device=f"cuda:{dev}")
    hits = torch.empty((nq, w.top_k, 2), dtype=torch.int64, device=f"cuda:{dev}")
    kw = dict(lanes=args.lanes, rows_per_lane=args.rows, precision=args.precision, long_rows_per_lane=args.long_rows,
              long_cutoff=args.long_cutoff,
              mode=swdb.SW_MODE_BATCHED if args.mode == "batched" else swdb.SW_MODE_PLAIN,
              alignment=ALIGNMENTS[args.alignment])
    tuned = None
    if want_autotune(args, args.mode == "batched") and args.alignment == "local":
        tuned = tune(db, w, forms=(args.mode,))
        if not args.long_cutoff:
            kw["long_cutoff"] = tuned["params"]["long_cutoff"]

    def step(stats=True):
        return swdb.sw_search(db.handle, q_dev, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend, w.top_k,
                              scores, hits, stats=stats, stream=stream.cuda_stream, graph=args.graph, **kw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st_all = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    local_ms = ev0.elapsed_time(ev1)
    t_ms, cells_all, gcups = combine_ranks(dist, local_ms, cells_step * args.steps)

    inter_ms = sum(s["inter_ms"] for s in st_all)
    launches = sum(s["launches"] for s in st_all)
    if args.graph:
        # A replayed graph reports no per-launch events: count the kernels of
        # one uncaptured step of the same search (outside the timed region).
        launches = args.steps * swdb.sw_search(db.handle, q_dev, w.queries.offsets, w.matrix, w.gap_open,
                                               w.gap_extend, w.top_k, scores, hits, stats=True,
                                               stream=stream.cuda_stream, **kw)["launches"]
    rescored = sum(s["rescored"] for s in st_all)
    rescore_ms = sum(s["rescore_ms"] for s in st_all)
    long_ms = sum(s["intra_ms"] for s in st_all)
    other_ms = sum(s["other_ms"] for s in st_all)
    st0 = st_all[0]

    # end to end through the C ABI with pinned host buffers
    q_host = torch.from_numpy(w.queries.residues).pin_memory()
    s_host = torch.empty((nq, n), dtype=torch.int32).pin_memory()
    h_host = torch.empty((nq, w.top_k, 2), dtype=torch.int64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        swdb.sw_search(db.handle, q_host, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend, w.top_k,
                       s_host, h_host, **kw)
    e2e_local = (time.perf_counter() - t0) * 1e3
    e2e_ms, e2e_cells, e2e_gcups = combine_ranks(dist, e2e_local, cells_step * args.e2e_steps)

    out = None
    if dist.rank == 0:
        rate_dpx, sms = swdb.sw_probe_alu_rate(dev, 0)
        rate_cells, _ = swdb.sw_probe_alu_rate(dev, 1)
        rate_u8x4, _ = swdb.sw_probe_alu_rate(dev, 2)
        mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        local = args.alignment == "local"
        packed = local or st0["precision_used"] == swdb.SW_PREC_I16
        batched = st0["mode_used"] == swdb.SW_MODE_BATCHED
        roof = step_roofline(st_all, args.alignment, packed, batched, rate_dpx, sms, mhz,
                             cells_step * args.steps / (t_ms * 1e-3) / 1e9, args.graph)
        ceiling = rate_cells * sms * mhz * 1e6 / 1e9
        traffic = traffic_per_launch(args)
        cb = None
        if not args.no_cpu_baseline:
            cb = cpu_baseline(w, scores.cpu().numpy(), seed + 1, args.cpu_sample_cells, mode=args.alignment)
        out = {
            "metric": METRIC, "value": gcups, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i16x2" if packed else "i32", "data": "synthetic",
            "config": {"workload": args.workload, "alignment": args.alignment, "queries": nq,
                       "query_residues": int(w.queries.lengths.sum()),
                       "db_seqs": n, "db_residues": int(w.db.lengths.sum()), "cells_per_step": cells_step,
                       "matrix": "BLOSUM62", "gap_open": w.gap_open, "gap_extend": w.gap_extend,
                       "top_k": w.top_k,
                       "mode": "plain (one launch per query)" if args.mode == "plain"
                               else "batched (query pairs, one persistent launch)",
                       "launch_shape": "lanes x rows per lane chosen per query by the library's rate model"
                                       if not (args.lanes or args.rows) else f"{args.lanes}x{args.rows}",
                       "l2": "inputs larger than L2 (database layout "
                             f"{db.info()['device_bytes'] / 1e6:.0f} MB > 129 MB), no flush",
                       "parallelism": f"{dist.world} independent GPU(s)",
                       "cuda_graph": "captured once, replayed every step (roofline achieved = whole step)"
                                     if args.graph else "no",
                       "autotune": tuned if tuned else "off (the library's measured shape tables)"},
            "roofline": {**roof, "traffic": traffic,
                         "register_only_ceiling_gcups": ceiling,
                         "probe_cells_per_sm_cycle": {"int16x2_shipped_sequence": rate_cells,
                                                      "int8x4_byte_simd": rate_u8x4}},
            "cpu_baseline": cb,
            "e2e": {"value": e2e_gcups, "unit": UNIT, "h2d_bytes_per_step": int(w.queries.residues.nbytes),
                    "d2h_bytes_per_step": int(nq * n * 4 + nq * w.top_k * 16), "ms_per_step": e2e_ms / args.e2e_steps},
            "gpu_launches": launches,
            "kernel_ms": {"inter": inter_ms, "long_side_stream": long_ms, "rescore": rescore_ms,
                          "profile_topk": other_ms},
            "long_sequences": st0["long_sequences"],
            "rescored_per_step": rescored / args.steps,
            "clocks": clk,
        }
        subs = sub_record_names(args, dist)
        if subs:
            out["workloads"] = run_sub_records(args, subs, db, w, rate_dpx, sms, dev)
            if "batched_512q/batched" in out["workloads"] and "batched_512q/plain" in out["workloads"]:
                b = out["workloads"]["batched_512q/batched"]["value"]
                p_ = out["workloads"]["batched_512q/plain"]["value"]
                out["batched_vs_plain"] = {"workload": "batched_512q", "batched_gcups": b, "plain_gcups": p_,
                                           "ratio": b / p_ if p_ else None}
    db.close()
    return out


# ---------------------------------------------------------------------------
# sub-records: the other workloads, measured after the main one

SUB_DEFAULTS = {            # (warm-up, timed steps) per workload
    "db2k_q100": (5, 50),
    "long_4q_50k": (3, 5),
    "batched_512q": (1, 3),     # 38-45 s per step: one warm-up step allocates and settles
}


def want_autotune(args, default: bool) -> bool:
    return args.autotune == "on" or (args.autotune == "auto" and default)


def tune(db, w, forms=("plain", "batched"), sample_queries: int = 8, cutoffs=(0, 2048, 6144)) -> dict:
    """Run the autotuner for this database and batch (outside any timed
    region) and summarise what it chose and measured."""
    from paper_2203_11100_gb300 import autotune
    params = autotune.autotune(db, w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                               top_k=w.top_k, sample_queries=sample_queries, cutoffs=cutoffs, repeats=2,
                               forms=forms, force=True, cache_path=None)
    r = autotune.last_result()
    fmt = lambda rows: [{"lanes": l, "rows": rr, "gcups": round(g, 1)} for l, rr, g in rows]
    return {"params": params, "plain_shapes": fmt(r["tuning"]["plain"]), "batched_shapes": fmt(r["tuning"]["batched"]),
            "tried": r["tried"], "tune_seconds": r["tune_seconds"], "probe_rows": r.get("probe_rows"),
            "how": "shape rates: median CUDA-event kernel rate of a probe query cut from the batch "
                   f"(pairs of them for the batched kernel); cutoff and form: median whole-search time of "
                   f"{sample_queries} queries spread over the batch's lengths"}


def sub_record_names(args, dist) -> list:
    if args.sub_records == "none" or args.impl != "ours":
        return []
    if args.sub_records == "auto":
        default = (dist.world == 1 and args.workload == "swissprot_like_20q" and args.db_scale == 1.0
                   and args.mode == "plain" and args.alignment == "local" and not args.graph
                   and not (args.lanes or args.rows or args.precision or args.long_rows or args.long_cutoff))
        return list(SUB_DEFAULTS) if default else []
    names = [x.strip() for x in args.sub_records.split(",") if x.strip()]
    for n in names:
        if n not in SUB_DEFAULTS:
            raise SystemExit(f"unknown sub-record workload {n!r}")
    return names


def timed_steps(step, steps: int, warmup: int, stream, dev: int):
    """W untimed warm-up calls, then K calls bracketed by CUDA events on the
    launching stream, with the SM clocks sampled meanwhile."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st_all = [step() for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), st_all, clocks.stop()


def step_roofline(st_all, alignment: str, packed: bool, batched: bool, rate_dpx: float, sms: int, mhz: float,
                  step_gcups: float, graph: bool) -> dict:
    """Roofline of a step's dominant kernel: the kernel that computes most of
    the step's cells (the intra-task launch on the side stream when the long
    pairs hold most of them, else the main-stream scoring kernel), its own
    cells over its own CUDA-event time, against the DPX-issue peak for that
    kernel's ALU operations per cell.  A replayed graph has no per-kernel
    events, so there the whole step's rate stands in."""
    local = alignment == "local"
    if local:
        if batched:
            kernel, opc = "k_batch_i16x2", BATCH_OPS_PER_CELL
            note = " (query pairs: one ready int16x2 profile word per row, no permute)"
        else:
            kernel, opc, note = "k_inter_i16x2", DPX_OPS_PER_CELL, ""
    elif packed:
        kernel, opc = "k_modes_i16x2", MODES16_OPS_PER_CELL
        note = " (int16x2 pairs: E, F, H and the profile permute, no running max)"
    else:
        kernel, opc, note = "k_modes_i32", I32_DPX_OPS_PER_CELL, " (int32: E, F and H, one cell per operation)"
    inter_cells = float(sum(s["inter_cells"] for s in st_all))
    inter_ms = sum(s["inter_ms"] for s in st_all)
    long_cells = float(sum(s["long_cells"] for s in st_all))
    long_ms = sum(s["intra_ms"] for s in st_all)
    inter_rate = inter_cells / (inter_ms * 1e-3) / 1e9 if inter_ms > 0 else 0.0
    achieved, launch_ms = inter_rate, inter_ms / max(sum(s["inter_launches"] for s in st_all), 1)
    extra = {}
    if local and long_cells > inter_cells and long_ms > 0 and not graph:
        extra["inter_task"] = {"kernel": kernel, "achieved": inter_rate}
        kernel, opc = "k_intra_i16x2", DPX_OPS_PER_CELL
        note = " (intra-task kernel: long sequences, on the side stream)"
        achieved, launch_ms = long_cells / (long_ms * 1e-3) / 1e9, long_ms / max(len(st_all), 1)
    peak = rate_dpx * sms * mhz * 1e6 / opc / 1e9
    if "inter_task" in extra:
        # the two kernels share the SMs for most of the step, so each one's
        # event time includes the other's work: the whole step against the peak
        extra["both_kernels_frac_of_peak"] = step_gcups / peak
    if graph:
        achieved = step_gcups
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GCUPS",
            "frac": achieved / peak if peak else None, "kernel": kernel,
            "peak_basis": f"measured {rate_dpx:.1f} DPX ops/SM/cycle x {sms} SMs x {mhz:.0f} MHz (median under "
                          f"load) / {opc} ops per cell" + note,
            "avg_launch_ms": launch_ms, **extra}


def kernel_roofline(st_all, family: str, kernel: str, ops_per_cell: float, rate_dpx: float, sms: int,
                    mhz: float, note: str = "") -> dict:
    """Achieved cell rate of one kernel family (its own cells over its own
    CUDA-event time) against the DPX-issue roofline for ops_per_cell."""
    if family == "long":
        cells = float(sum(s["long_cells"] for s in st_all))
        ms = sum(s["intra_ms"] for s in st_all)
        launches = len(st_all)
    else:
        cells = float(sum(s["inter_cells"] for s in st_all))
        ms = sum(s["inter_ms"] for s in st_all)
        launches = sum(s["inter_launches"] for s in st_all)
    peak = rate_dpx * sms * mhz * 1e6 / ops_per_cell / 1e9
    achieved = cells / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GCUPS",
            "frac": achieved / peak if peak else None, "traffic": None, "kernel": kernel,
            "peak_basis": f"measured {rate_dpx:.1f} DPX ops/SM/cycle x {sms} SMs x {mhz:.0f} MHz (median under "
                          f"load) / {ops_per_cell} ops per cell" + note,
            "kernel_ms_per_step": ms / max(len(st_all), 1), "avg_launch_ms": ms / max(launches, 1)}


def oracle_sample(w, scores_dev, hits_dev, seed: int, max_cells: float) -> dict:
    """The GPU's scores of a bounded sample of pairs against the oracle (all
    host cores): every query's best hit, then random pairs up to max_cells
    (every pair when the whole workload fits), and the top-k of sampled rows."""
    import torch
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    nq, n = w.queries.n, w.db.n
    qlen = w.queries.lengths.astype(np.float64)
    tlen = w.db.lengths.astype(np.float64)
    hits = hits_dev.cpu().numpy()
    if float(w.cells) <= max_cells:
        qi = np.repeat(np.arange(nq, dtype=np.int64), n)
        ti = np.tile(np.arange(n, dtype=np.int64), nq)
        what = "every pair"
    else:
        qi = [np.arange(nq, dtype=np.int64)]
        ti = [hits[:, 0, 1].astype(np.int64)]
        budget = max_cells - float((qlen[qi[0]] * tlen[ti[0]]).sum())
        k = max(0, int(budget / (qlen.mean() * tlen.mean())))
        qi.append(rng.integers(0, nq, k))
        ti.append(rng.integers(0, n, k))
        qi, ti = np.concatenate(qi), np.concatenate(ti)
        what = f"each query's best hit and {k} random pairs"
    cells = float((qlen[qi] * tlen[ti]).sum())
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    want = oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend, threads=threads)
    dt = time.perf_counter() - t0
    got = scores_dev[torch.from_numpy(qi).to(scores_dev.device), torch.from_numpy(ti).to(scores_dev.device)]
    exact = bool(np.array_equal(got.cpu().numpy().astype(np.int64), want))
    # top-k of the rows checked in full (small workloads) or the best hit's score (others)
    if what == "every pair":
        for q in range(nq):
            s_, i_ = oracle.top_k(want[q * n:(q + 1) * n], w.top_k)
            exact &= bool(np.array_equal((hits[q, :, 0] & 0xffffffff).astype(np.int32).astype(np.int64), s_))
            exact &= bool(np.array_equal(hits[q, :, 1], i_))
    return {"pairs": int(len(qi)), "what": what, "cells": cells, "oracle_s": dt, "cores": threads,
            "bit_exact_vs_gpu": exact}


def run_sub_records(args, names, db_main, w_main, rate_dpx: float, sms: int, dev: int) -> dict:
    import torch
    import paper_2203_11100_gb300 as swdb
    out = {}
    stream = torch.cuda.Stream(device=dev)
    for name in names:
        warm, steps = SUB_DEFAULTS[name]
        if args.sub_warmup >= 0:
            warm = args.sub_warmup
        if args.sub_steps > 0:
            steps = args.sub_steps
        tuned = None
        if name == "batched_512q":
            w = synth.make_workload(name, seed=synth.SEED, db=w_main.db)
            db, own = db_main, False
            forms = [("batched", swdb.SW_MODE_BATCHED), ("plain", swdb.SW_MODE_PLAIN)]
            if want_autotune(args, True):
                tuned = tune(db, w)      # both forms use the measured tables and the chosen cutoff
        else:
            w = synth.make_workload(name, seed=synth.SEED)
            db, own = swdb.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET), device=dev), True
            forms = [("plain", swdb.SW_MODE_PLAIN)]
        q_dev = torch.from_numpy(w.queries.residues).to(f"cuda:{dev}")
        scores = torch.empty((w.queries.n, w.db.n), dtype=torch.int32, device=f"cuda:{dev}")
        hits = torch.empty((w.queries.n, w.top_k, 2), dtype=torch.int64, device=f"cuda:{dev}")
        for form, mode in forms:
            kw = dict(mode=mode)
            if tuned:
                kw["long_cutoff"] = tuned["params"]["long_cutoff"]

            def step():
                return swdb.sw_search(db.handle, q_dev, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                                      w.top_k, scores, hits, stats=True, stream=stream.cuda_stream, **kw)

            ms, st_all, clk = timed_steps(step, steps, warm, stream, dev)
            mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
            cells = float(w.cells)
            if name == "long_4q_50k":
                roof = kernel_roofline(st_all, "long", "k_intra_i16x2", DPX_OPS_PER_CELL, rate_dpx, sms, mhz,
                                       " (intra-task kernel: long sequences, on the side stream)")
                roof["inter_task"] = kernel_roofline(st_all, "inter", "k_inter_i16x2", DPX_OPS_PER_CELL,
                                                     rate_dpx, sms, mhz)
                # the two launches share the SMs for most of the step, so each one's
                # event time includes the other's work: the whole step against the peak
                roof["both_kernels_frac_of_peak"] = cells * steps / (ms * 1e-3) / 1e9 / roof["peak"]
            elif form == "batched":
                roof = kernel_roofline(st_all, "inter", "k_batch_i16x2", BATCH_OPS_PER_CELL, rate_dpx, sms, mhz,
                                       " (query pairs: one ready int16x2 profile word per row, no permute)")
                roof["frac_of_plain_kernel_roofline"] = roof["achieved"] / (rate_dpx * sms * mhz * 1e6 /
                                                                            DPX_OPS_PER_CELL / 1e9)
            else:
                roof = kernel_roofline(st_all, "inter", "k_inter_i16x2", DPX_OPS_PER_CELL, rate_dpx, sms, mhz)
            rec = {"workload": name, "form": form, "value": cells * steps / (ms * 1e-3) / 1e9, "unit": UNIT,
                   "steps": steps, "warmup": warm, "ms_per_step": ms / steps, "cells_per_step": cells,
                   "queries": w.queries.n, "query_residues": int(w.queries.lengths.sum()), "db_seqs": w.db.n,
                   "db_residues": int(w.db.lengths.sum()), "roofline": roof, "clocks": clk,
                   "gpu_launches": sum(s["launches"] for s in st_all),
                   "kernel_ms_per_step": {k: sum(s[k + "_ms"] for s in st_all) / steps
                                          for k in ("inter", "rescore", "intra", "other")},
                   "long_sequences": st_all[0]["long_sequences"],
                   "rescored_per_step": sum(s["rescored"] for s in st_all) / steps,
                   "launch": {k: v for k, v in kw.items() if k != "mode"} or "library choice per query",
                   "autotune": tuned if tuned else "off (the library's measured shape tables)"}
            if not args.no_cpu_baseline:
                rec["oracle_sample"] = oracle_sample(w, scores, hits, synth.SEED + 31 + len(out),
                                                     max_cells=4e10 if name == "batched_512q" else 1e10)
            out[f"{name}/{form}"] = rec
        del scores, hits, q_dev
        if own:
            db.close()
        elif tuned:
            swdb.sw_db_set_tuning(db.handle, None)
    return out


def run_sharded(args, dist: Dist):
    """The database sharded over the ranks (one shard per GPU), every query
    against every shard, then the top-k exchange: an all-gather of each
    shard's n_q x top_k hits and the merge into the unsharded top-k on rank 0.
    One step = the whole workload (all queries x the whole database): strong
    scaling.  Rank 0 checks the merged hits' best entries against the oracle."""
    import torch
    import paper_2203_11100_gb300 as swdb
    from paper_2203_11100_gb300 import multigpu

    dev = dist.device
    torch.cuda.set_device(dev)
    swdb.load_library()
    w = synth.make_workload(args.workload, seed=synth.SEED, db_scale=args.db_scale)
    members, moff = swdb.sw_shard_plan(w.db.offsets, dist.world)
    mine = members[moff[dist.rank]:moff[dist.rank + 1]]
    lens = w.db.lengths[mine]
    off = np.zeros(len(mine) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    res = np.concatenate([w.db.seq(int(i)) for i in mine]) if len(mine) else np.zeros(0, np.uint8)
    db = swdb.Database(res, off, len(synth.ALPHABET), device=dev)
    stream = torch.cuda.Stream(device=dev)
    nq = w.queries.n
    q_dev = torch.from_numpy(w.queries.residues).to(f"cuda:{dev}")
    scores = torch.empty((nq, max(len(mine), 1)), dtype=torch.int32, device=f"cuda:{dev}")
    hits = torch.empty((nq, w.top_k, 2), dtype=torch.int64, device=f"cuda:{dev}")
    kw = dict(mode=swdb.SW_MODE_BATCHED if args.mode == "batched" else swdb.SW_MODE_PLAIN)
    merged = [None]

    def step():
        with torch.cuda.stream(stream):
            st = swdb.sw_search(db.handle, q_dev, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend, w.top_k,
                                scores, hits, stats=True, stream=stream.cuda_stream, **kw)
            if dist.pg is not None:
                local = hits if dist.backend == "nccl" else hits.cpu()
                merged[0] = multigpu.exchange_hits(dist.pg, local, members, moff, w.top_k, dst=0)
            else:
                merged[0] = swdb.sw_hits_merge(multigpu.tensor_to_hits(hits)[None], members, moff, w.top_k)
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st_all = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    local_ms = ev0.elapsed_time(ev1)
    t_ms = dist.max(local_ms)
    cells_step = float(w.cells)
    gcups = cells_step * args.steps / (t_ms * 1e-3) / 1e9
    shard_cells = dist.sum(float(w.queries.lengths.sum()) * float(lens.sum()))

    # end to end: queries from pinned host memory, each shard's hits back to
    # the host, the exchange and the merge
    q_host = torch.from_numpy(w.queries.residues).pin_memory()
    h_host = torch.empty((nq, w.top_k, 2), dtype=torch.int64).pin_memory()
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        swdb.sw_search(db.handle, q_host, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend, w.top_k, None,
                       h_host, **kw)
        if dist.pg is not None:
            multigpu.exchange_hits(dist.pg, h_host.to(f"cuda:{dev}") if dist.backend == "nccl" else h_host,
                                   members, moff, w.top_k, dst=0)
        else:
            swdb.sw_hits_merge(multigpu.tensor_to_hits(h_host)[None], members, moff, w.top_k)
    torch.cuda.synchronize()
    e2e_ms = dist.max((time.perf_counter() - t0) * 1e3)
    out = None
    if dist.rank == 0:
        rate_dpx, sms = swdb.sw_probe_alu_rate(dev, 0)
        mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        roof = kernel_roofline(st_all, "inter", "k_inter_i16x2", DPX_OPS_PER_CELL, rate_dpx, sms, mhz,
                               " (rank 0's shard)")
        check = None
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            h = merged[0]
            qi = np.arange(nq, dtype=np.int64)
            ti = h[:, 0]["db_index"].astype(np.int64)
            want = oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend)
            check = {"pairs": int(nq), "what": "each query's merged best hit (caller's index)",
                     "bit_exact_vs_gpu": bool(np.array_equal(want, h[:, 0]["score"].astype(np.int64)))}
        out = {"metric": METRIC, "value": gcups, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
               "scaling": "strong", "vs_baseline": None, "dtype": "i16x2", "data": "synthetic",
               "config": {"workload": args.workload, "queries": nq, "db_seqs": w.db.n,
                          "db_residues": int(w.db.lengths.sum()), "cells_per_step": cells_step,
                          "shard_residues": [int(w.db.lengths[members[moff[r]:moff[r + 1]]].sum())
                                             for r in range(dist.world)],
                          "matrix": "BLOSUM62", "gap_open": w.gap_open, "gap_extend": w.gap_extend,
                          "top_k": w.top_k, "mode": args.mode,
                          "parallelism": f"database sharded over {dist.world} GPU(s) (residue-balanced, "
                                         "length-stratified); top-k all-gather + merge on rank 0",
                          "l2": "inputs larger than L2, no flush" if int(lens.sum()) > 129e6 else
                                "shard layout may fit L2; each launch streams it once per query"},
               "roofline": roof, "clocks": clk,
               "gpu_launches": sum(s["launches"] for s in st_all), "shard_cells_all_ranks": shard_cells,
               "merged_hits_check": check,
               "e2e": {"value": cells_step * args.e2e_steps / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
                       "h2d_bytes_per_step": int(w.queries.residues.nbytes) * dist.world,
                       "d2h_bytes_per_step": int(nq * w.top_k * 16) * dist.world,
                       "ms_per_step": e2e_ms / args.e2e_steps}}
    db.close()
    return out


def run_serving(args, dist: Dist):
    """Continuous-batching server under Poisson arrivals (config of the
    serving workload at a stated database fraction)."""
    import torch
    import paper_2203_11100_gb300 as swdb
    from paper_2203_11100_gb300.serve import SearchServer

    dev = dist.device
    torch.cuda.set_device(dev)
    swdb.load_library()
    dbs = synth.serving_database(db_scale=args.serve_db_scale)
    n_req = args.serve_requests
    reqs = synth.serving_requests(4 * n_req, seed=synth.SEED + 7919 * dist.rank)
    S = synth.blosum62()
    db = swdb.Database(dbs.residues, dbs.offsets, len(synth.ALPHABET), device=dev)
    residues = int(dbs.lengths.sum())
    clocks = ClockSampler(dev)

    launch = {}
    tuned = None
    if want_autotune(args, True):
        sample = synth.Workload("serving sample", synth.seqset_from_list([reqs.seq(i) for i in range(64)]), dbs, S,
                                10, 1, 10)
        tuned = tune(db, sample, forms=("batched",), sample_queries=4)
        launch = {"long_cutoff": tuned["params"]["long_cutoff"]}

    def new_server():
        return SearchServer(db, S, 10, 1, top_k=10, max_batch=args.serve_max_batch, streams=3, max_query_len=8000,
                            launch=launch)

    # warm-up: one batch through a server
    srv = new_server()
    for f in [srv.submit(reqs.seq(i)) for i in range(args.serve_max_batch)]:
        f.result(timeout=RESULT_TIMEOUT_S)
    srv.close()

    clocks.start()
    # saturation: every request queued at once (closed system)
    srv = new_server()
    t0 = time.perf_counter()
    futs = [srv.submit(reqs.seq(i)) for i in range(n_req)]
    served = [f.result(timeout=RESULT_TIMEOUT_S) for f in futs]
    sat_s = time.perf_counter() - t0
    sat = srv.stats()
    srv.close()
    sat_rate = n_req / sat_s
    sat_cells = float(reqs.lengths[:n_req].sum()) * residues

    points = []
    rng = np.random.default_rng(synth.SEED + 11)
    base = n_req
    for frac in (0.5, 0.8, 0.95):
        rate = frac * sat_rate
        count = args.serve_point_requests or max(16, n_req // 2)
        gaps = rng.exponential(1.0 / rate, count)
        srv = new_server()
        t_start = time.perf_counter()
        arrivals = t_start + np.cumsum(gaps)
        futs = []
        for i in range(count):
            now = time.perf_counter()
            if arrivals[i] > now:
                time.sleep(arrivals[i] - now)
            futs.append(srv.submit(reqs.seq(base + i)))
        for f in futs:
            f.result(timeout=RESULT_TIMEOUT_S)
        st = srv.stats()
        srv.close()
        base += count
        points.append({"offered_rate_per_s": rate, "load": frac, "requests": count, "p50_ms": st["p50_ms"],
                       "p99_ms": st["p99_ms"], "mean_batch": st["mean_batch"], "gcups": st["gcups"]})
    clk = clocks.stop()

    # the plain one-query-per-launch form on the same saturation requests
    q_off = reqs.offsets[:n_req + 1].copy()
    q_res = reqs.residues[:int(q_off[-1])]
    q_dev = torch.from_numpy(q_res).to(f"cuda:{dev}")
    hits = torch.empty((n_req, 10, 2), dtype=torch.int64, device=f"cuda:{dev}")
    swdb.sw_search(db.handle, q_dev, q_off, S, 10, 1, 10, None, hits, mode=swdb.SW_MODE_PLAIN)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    swdb.sw_search(db.handle, q_dev, q_off, S, 10, 1, 10, None, hits, mode=swdb.SW_MODE_PLAIN, stats=True)
    plain_s = time.perf_counter() - t0
    # served results: the same hits as the plain search of the same query, and
    # every hit's score equal to the oracle's score of that pair
    check = None
    if args.serve_check > 0:
        import oracle
        from paper_2203_11100_gb300 import multigpu
        oracle.build()
        k = min(args.serve_check, n_req)
        plain = multigpu.tensor_to_hits(hits[:k])
        same = all(np.array_equal(served[i]["score"], plain[i]["score"]) and
                   np.array_equal(served[i]["db_index"], plain[i]["db_index"]) for i in range(k))
        qi = np.repeat(np.arange(k, dtype=np.int64), 10)
        ti = np.concatenate([served[i]["db_index"] for i in range(k)]).astype(np.int64)
        qs = synth.SeqSet(reqs.residues, reqs.offsets)
        t0 = time.perf_counter()
        want = oracle.score_pairs(qs, dbs, qi, ti, S, 10, 1)
        got = np.concatenate([served[i]["score"] for i in range(k)]).astype(np.int64)
        check = {"requests": k, "hits_equal_plain_search": bool(same), "hit_scores_equal_oracle":
                 bool(np.array_equal(want, got)), "oracle_pairs": int(len(qi)), "oracle_s": time.perf_counter() - t0}
    db.close()
    value = sat_cells / sat_s / 1e9
    return {"metric": "GCUPS (served: continuous batching, database resident in HBM)", "value": value,
            "unit": UNIT, "n_gpus": dist.world, "steps": 1, "warmup": 1, "ms_per_step": sat_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i16x2",
            "data": "synthetic",
            "config": {"workload": "serving", "db_seqs": dbs.n, "db_residues": residues,
                       "db_fraction_of_20M": args.serve_db_scale, "requests_saturation": n_req,
                       "request_lengths": "lognormal mean 400, 30..8000", "matrix": "BLOSUM62",
                       "gap_open": 10, "gap_extend": 1, "top_k": 10, "max_batch": args.serve_max_batch,
                       "streams": 3, "autotune": tuned if tuned else "off"},
            "serving": {"saturation_rate_per_s": sat_rate, "saturation_p50_ms": sat["p50_ms"],
                        "saturation_p99_ms": sat["p99_ms"], "points": points,
                        "plain_one_launch_per_query_gcups": sat_cells / plain_s / 1e9,
                        "served_check": check},
            "clocks": clk}


def run_sweep(args, dist: Dist):
    """GCUPS against query length, as in the paper's query-length figure
    (Section 4.2): every query of the workload searched alone against the
    whole database (one plain search per query), K timed steps after W
    warm-up steps each, at the workload's penalties and at the paper's 10/2
    (Section 4.1)."""
    import torch
    import paper_2203_11100_gb300 as swdb

    dev = dist.device
    torch.cuda.set_device(dev)
    swdb.load_library()
    w = synth.make_workload(args.workload, seed=synth.SEED, db_scale=args.db_scale)
    db = swdb.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET), device=dev)
    residues = int(w.db.lengths.sum())
    # A stream of its own: the legacy default stream's handle is NULL, which
    # the library reads as "the handle's own stream".
    stream = torch.cuda.Stream(device=dev)
    scores = torch.empty((1, w.db.n), dtype=torch.int32, device=f"cuda:{dev}")
    hits = torch.empty((1, w.top_k, 2), dtype=torch.int64, device=f"cuda:{dev}")
    clocks = ClockSampler(dev)
    clocks.start()
    rows = []
    totals = {}
    for o, e in ((w.gap_open, w.gap_extend), (10, 2)):
        cells_sum = ms_sum = 0.0
        for qi in range(w.queries.n):
            q = w.queries.seq(qi)
            q_dev = torch.from_numpy(np.ascontiguousarray(q)).to(f"cuda:{dev}")
            q_off = np.array([0, len(q)], dtype=np.int64)

            def step():
                swdb.sw_search(db.handle, q_dev, q_off, w.matrix, o, e, w.top_k, scores, hits,
                               stream=stream.cuda_stream, mode=swdb.SW_MODE_PLAIN)

            for _ in range(args.warmup):
                step()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(args.steps):
                step()
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            cells = float(len(q)) * residues * args.steps
            rows.append({"m": len(q), "gap": f"{o}/{e}", "gcups": cells / ms / 1e6, "ms_per_search": ms / args.steps})
            cells_sum += cells
            ms_sum += ms
        totals[f"{o}/{e}"] = cells_sum / ms_sum / 1e6
    clk = clocks.stop()
    db.close()
    key = f"{w.gap_open}/{w.gap_extend}"
    return {"metric": "GCUPS by query length (device-timed, one query per search)", "value": totals[key],
            "unit": UNIT, "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "i16x2", "data": "synthetic",
            "config": {"workload": f"{args.workload}: each query alone", "db_seqs": w.db.n, "db_residues": residues,
                       "query_lengths": [int(x) for x in w.queries.lengths], "matrix": "BLOSUM62",
                       "penalties": list(totals)},
            "aggregate_gcups": totals, "sweep": rows, "clocks": clk}


def run_align(args, dist: Dist):
    """Traceback of the top-k hits: search the workload once, then align every
    (query, hit) pair with sw_align (sw_align_mode for --alignment other than
    local, the hits of that mode's search); W warm-up and K timed calls."""
    import torch
    import paper_2203_11100_gb300 as swdb

    dev = dist.device
    torch.cuda.set_device(dev)
    swdb.load_library()
    w = synth.make_workload(args.workload, seed=synth.SEED, db_scale=args.db_scale)
    db = swdb.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET), device=dev)
    mode = ALIGNMENTS[args.alignment]
    _, hits, _ = db.search(w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                           top_k=w.top_k, want_scores=False, alignment=mode)
    pq = np.repeat(np.arange(w.queries.n, dtype=np.int32), w.top_k)
    pt = hits["db_index"].reshape(-1).astype(np.int64)
    keep = pt >= 0
    pq, pt = pq[keep], pt[keep]
    for _ in range(args.warmup):
        db.align(w.queries.residues, w.queries.offsets, pq, pt, w.matrix, w.gap_open, w.gap_extend, alignment=mode)
    clocks = ClockSampler(dev)
    clocks.start()
    fwd_ms = tb_ms = 0.0
    wall = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        aln, ops, st = db.align(w.queries.residues, w.queries.offsets, pq, pt, w.matrix, w.gap_open,
                                w.gap_extend, stats=True, alignment=mode)
        wall.append(time.perf_counter() - t0)
        fwd_ms += st["forward_ms"]
        tb_ms += st["traceback_ms"]
    clk = clocks.stop()
    db.close()
    if not np.array_equal(aln["score"], hits["score"].reshape(-1)[keep]):
        raise RuntimeError("alignment scores differ from the search scores")
    n = len(pq)
    fwd_cells, tb_cells = st["forward_cells"], st["traceback_cells"]
    lens_q, lens_t = w.queries.lengths[pq], w.db.lengths[pt]
    cb = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        order = np.argsort(lens_q * lens_t, kind="stable")
        pick, cells = [], 0
        for k in order:                                # smallest pairs first, up to ~1e10 cells
            c = int(lens_q[k]) * int(lens_t[k])
            if cells + c > 1e10:
                break
            pick.append(int(k))
            cells += c
        t0 = time.perf_counter()
        want = oracle.align_pairs(w.queries, w.db, pq[pick], pt[pick], w.matrix, w.gap_open, w.gap_extend,
                                  mode=args.alignment)
        dt = time.perf_counter() - t0
        exact = True
        for k, wa in zip(pick, want):
            o0 = int(aln["ops_offset"][k])
            got = ops[o0:o0 + int(aln["ops_len"][k])]
            exact &= (int(aln["score"][k]), int(aln["q_begin"][k]), int(aln["q_end"][k]), int(aln["t_begin"][k]),
                      int(aln["t_end"][k])) == (wa["score"], wa["q_begin"], wa["q_end"], wa["t_begin"], wa["t_end"])
            exact &= bool(np.array_equal(got, wa["ops"]))
        cb = {"value": len(pick) / dt, "unit": "alignments/s", "cores": oracle.default_threads(), "kind": "oracle",
              "gcups": cells / dt / 1e9,
              "sample": f"the {len(pick)} smallest of the {n} pairs ({cells:.3g} cells, {dt:.1f} s)",
              "sample_bit_exact_vs_gpu": exact}
    dev_s = (fwd_ms + tb_ms) / 1e3
    e2e_s = float(np.sum(wall))
    return {"metric": "alignments of the top-k hits per second (device-timed, bit-exact vs oracle)",
            "value": n * args.steps / dev_s, "unit": "alignments/s", "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": (fwd_ms + tb_ms) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": {"workload": f"{args.workload} top-{w.top_k} hits", "alignment": args.alignment, "pairs": n,
                       "query_lengths": [int(lens_q.min()), int(lens_q.max())],
                       "target_lengths": [int(lens_t.min()), int(lens_t.max())],
                       "forward_cells_per_step": fwd_cells, "traceback_cells_per_step": tb_cells,
                       "matrix": "BLOSUM62", "gap_open": w.gap_open, "gap_extend": w.gap_extend},
            "kernel_ms": {"forward": fwd_ms / args.steps, "traceback": tb_ms / args.steps},
            "gcups": {"forward": fwd_cells / (fwd_ms / args.steps) / 1e6,
                      "traceback": tb_cells / (tb_ms / args.steps) / 1e6},
            "longest_pair_cells": int((lens_q * lens_t).max()),
            "e2e": {"value": n * args.steps / e2e_s, "unit": "alignments/s",
                    "h2d_bytes_per_step": int(w.queries.offsets[-1]) + n * 12,
                    "d2h_bytes_per_step": n * 40 + int(ops.nbytes), "ms_per_step": e2e_s * 1e3 / args.steps},
            "cpu_baseline": cb, "gpu_launches": 2 * args.steps, "clocks": clk}


def run_reference(args, dist: Dist):
    """The oracle timed on the host cores, one bounded sample per step."""
    if dist.rank != 0:
        return None
    import oracle
    oracle.build()
    w = synth.make_workload(args.workload, seed=synth.SEED, db_scale=args.db_scale)
    rng = np.random.default_rng(synth.SEED + 99)
    threads = oracle.default_threads()
    qlen = w.queries.lengths.astype(np.float64)
    per_query = max(1, int(args.cpu_sample_cells / 4 / qlen.sum() / w.db.lengths.mean()))
    per_query = min(per_query, w.db.n)

    def step():
        t_idx = rng.choice(w.db.n, size=per_query, replace=False)
        qi = np.repeat(np.arange(w.queries.n, dtype=np.int64), len(t_idx))
        ti = np.tile(t_idx.astype(np.int64), w.queries.n)
        cells = float((qlen[qi] * w.db.lengths[ti]).sum())
        t0 = time.perf_counter()
        oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend, threads=threads)
        return cells, time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    cells = secs = 0.0
    for _ in range(args.steps):
        c, s = step()
        cells += c
        secs += s
    v = cells / secs / 1e9
    single = single_thread_oracle()
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": args.workload, "queries": w.queries.n, "db_seqs": w.db.n,
                       "matrix": "BLOSUM62", "gap_open": w.gap_open, "gap_extend": w.gap_extend, "top_k": w.top_k},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"per step: all {w.queries.n} queries x {per_query} random database "
                                       f"sequences (~{cells / args.steps:.3g} cells)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "single_thread_oracle": single, "host": host_info()}


def host_info() -> dict:
    """Core count and CPU model of the host the oracle runs on."""
    import platform
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu part", "processor name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu": model}


def single_thread_oracle() -> dict:
    """Single-thread oracle GCUPS: the whole 1 x 100 vs 2,000 workload, and a
    fixed ~1e9-cell sample of the default workload (all 20 queries x the
    same random database sequences)."""
    import oracle
    out = {}
    w = synth.make_workload("db2k_q100", seed=synth.SEED)
    qi = np.zeros(w.db.n, dtype=np.int64)
    ti = np.arange(w.db.n, dtype=np.int64)
    t0 = time.perf_counter()
    oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend, threads=1)
    out["db2k_q100_gcups"] = float(w.cells) / (time.perf_counter() - t0) / 1e9
    w = synth.make_workload("swissprot_like_20q", seed=synth.SEED)
    rng = np.random.default_rng(synth.SEED + 5)
    per_query = int(1e9 / w.queries.lengths.sum() / w.db.lengths.mean())
    t_idx = np.sort(rng.choice(w.db.n, size=per_query, replace=False)).astype(np.int64)
    qi = np.repeat(np.arange(w.queries.n, dtype=np.int64), len(t_idx))
    ti = np.tile(t_idx, w.queries.n)
    cells = float((w.queries.lengths[qi].astype(np.float64) * w.db.lengths[ti]).sum())
    t0 = time.perf_counter()
    oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend, threads=1)
    out["swissprot_like_20q_sample_gcups"] = cells / (time.perf_counter() - t0) / 1e9
    out["swissprot_like_20q_sample_cells"] = cells
    return out


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        dist = Dist(init=False)   # rank 0 alone runs the oracle; other ranks exit without work
        out = run_reference(args, dist)
    elif args.serve:
        dist = Dist()
        out = run_serving(args, dist)
    elif args.align:
        dist = Dist()
        out = run_align(args, dist)
    elif args.sweep:
        dist = Dist()
        out = run_sweep(args, dist)
    else:
        dist = Dist()
        if dist.world > 1 and args.multi == "shard":
            out = run_sharded(args, dist)
        else:
            out = run_ours(args, dist)
    if out is not None and dist.rank == 0:
        print(json.dumps(out), flush=True)
    dist.close()


if __name__ == "__main__":
    main()
