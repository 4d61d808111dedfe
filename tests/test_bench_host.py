"""Host logic of bench.py (CPU only): the launch key and DRAM-traffic record
lookup behind ``roofline.traffic``, the choice of the step's dominant kernel
and its peak, and the reference arm's JSON line (the oracle on the host
cores)."""
import hashlib
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_launch_key_names_the_configuration():
    b = _bench()
    base = b.launch_key(b.parse_args([]))
    assert base == "swissprot_like_20q/scale1/plain/lanes0/rows0/prec0/longrows0/cutoff0"
    assert b.launch_key(b.parse_args(["--alignment", "global"])) == base + "/global"
    assert b.launch_key(b.parse_args(["--lanes", "8", "--rows", "24"])) != base
    assert b.launch_key(b.parse_args(["--db-scale", "0.5"])) != base


def test_traffic_record_needs_the_same_launch_and_kernel_source(tmp_path, monkeypatch):
    b = _bench()
    csrc = tmp_path / "paper_2203_11100_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k_inter16.cu").write_text("// inter kernel v1\n")
    (csrc / "k_modes16.cu").write_text("// modes kernel v1\n")
    sha = lambda p: hashlib.sha256(p.read_bytes()).hexdigest()
    key = b.launch_key(b.parse_args([]))
    gkey = b.launch_key(b.parse_args(["--alignment", "global"]))
    (tmp_path / "profiles" / "x.md").write_text(
        "# a capture\n\n"
        f"traffic: launch={key} dram_bytes_per_launch=1000 source_sha256={sha(csrc / 'k_inter16.cu')}\n"
        f"traffic: launch={gkey} source=k_modes16.cu dram_bytes_per_launch=2000 "
        f"source_sha256={sha(csrc / 'k_modes16.cu')}\n")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.traffic_per_launch(b.parse_args([])) == 1000.0
    assert b.traffic_per_launch(b.parse_args(["--alignment", "global"])) == 2000.0
    assert b.traffic_per_launch(b.parse_args(["--alignment", "overlap"])) is None     # no record
    assert b.traffic_per_launch(b.parse_args(["--lanes", "8", "--rows", "32"])) is None
    (csrc / "k_inter16.cu").write_text("// inter kernel v2\n")                        # kernel changed
    assert b.traffic_per_launch(b.parse_args([])) is None
    assert b.traffic_per_launch(b.parse_args(["--alignment", "global"])) == 2000.0


def test_reference_arm_prints_one_json_line():
    """--impl reference times the oracle on the host cores and prints the contract's keys."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-sample-cells", "1e8"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "GCUPS" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "swissprot_like_20q"


def test_sub_records_only_for_the_default_single_gpu_line():
    b = _bench()
    one = b.Dist(init=False)
    assert b.sub_record_names(b.parse_args([]), one) == ["db2k_q100", "long_4q_50k", "batched_512q"]
    assert b.sub_record_names(b.parse_args(["--sub-records", "none"]), one) == []
    assert b.sub_record_names(b.parse_args(["--mode", "batched"]), one) == []
    assert b.sub_record_names(b.parse_args(["--db-scale", "0.5"]), one) == []
    assert b.sub_record_names(b.parse_args(["--sub-records", "long_4q_50k"]), one) == ["long_4q_50k"]
    two = b.Dist(init=False)
    two.world = 2
    assert b.sub_record_names(b.parse_args([]), two) == []
    with pytest.raises(SystemExit):
        b.sub_record_names(b.parse_args(["--sub-records", "nope"]), one)


def test_oracle_sample_flags_a_wrong_score():
    """The sub-records' oracle check: exact scores and hits pass, one changed
    score fails (CPU tensors stand in for the device buffers)."""
    import numpy as np
    import torch

    import oracle
    import synth
    b = _bench()
    w = synth.make_workload("db2k_q100", db_scale=0.05)
    want = oracle.all_scores(w.queries, w.db, w.matrix, w.gap_open, w.gap_extend)
    hits = np.zeros((w.queries.n, w.top_k, 2), np.int64)
    for q in range(w.queries.n):
        s_, i_ = oracle.top_k(want[q], w.top_k)
        hits[q, :, 0] = s_ & 0xffffffff
        hits[q, :, 1] = i_
    scores = torch.from_numpy(want.astype(np.int32))
    rec = b.oracle_sample(w, scores, torch.from_numpy(hits), 1, max_cells=1e12)
    assert rec["bit_exact_vs_gpu"] and rec["what"] == "every pair" and rec["pairs"] == w.db.n
    scores[0, 3] += 1
    assert not b.oracle_sample(w, scores, torch.from_numpy(hits), 1, max_cells=1e12)["bit_exact_vs_gpu"]
    # a bounded sample of a larger workload: each query's best hit plus random pairs
    rec = b.oracle_sample(w, torch.from_numpy(want.astype(np.int32)), torch.from_numpy(hits), 1, max_cells=1e6)
    assert rec["bit_exact_vs_gpu"] and rec["what"].startswith("each query's best hit")


def _stats(inter_cells, inter_ms, long_cells, intra_ms, launches=20):
    return {"inter_cells": inter_cells, "inter_ms": inter_ms, "long_cells": long_cells, "intra_ms": intra_ms,
            "inter_launches": launches}


def test_step_roofline_names_the_kernel_that_computes_most_cells():
    b = _bench()
    peak_275 = 64.0 * 152 * 2070.0 * 1e6 / 2.75 / 1e9
    # plain local step: the inter-task kernel, its cells over its own event time
    r = b.step_roofline([_stats(6e12, 1000.0, 2e11, 60.0)] * 2, "local", True, False, 64.0, 152, 2070.0, 5900.0,
                        False)
    assert r["kernel"] == "k_inter_i16x2"
    assert r["achieved"] == pytest.approx(6e12 * 2 / 2.0 / 1e9)
    assert r["peak"] == pytest.approx(peak_275) and r["avg_launch_ms"] == pytest.approx(50.0)
    # long pairs hold most cells: the intra-task kernel on its own 2.75-op peak, even in the
    # batched form, with the main-stream kernel and the whole step beside it
    r = b.step_roofline([_stats(1e12, 1200.0, 4.7e12, 1000.0)], "local", True, True, 64.0, 152, 2070.0, 5700.0,
                        False)
    assert r["kernel"] == "k_intra_i16x2" and r["peak"] == pytest.approx(peak_275)
    assert r["achieved"] == pytest.approx(4.7e12 / 1.0 / 1e9)
    assert r["inter_task"]["kernel"] == "k_batch_i16x2"
    assert r["both_kernels_frac_of_peak"] == pytest.approx(5700.0 / peak_275)
    # an intra-task launch whose event time spans the step but holds few cells is not dominant
    r = b.step_roofline([_stats(2.5e14, 37000.0, 1e12, 37800.0, 1)], "local", True, True, 64.0, 152, 2070.0,
                        6900.0, False)
    assert r["kernel"] == "k_batch_i16x2"
    assert r["peak"] == pytest.approx(64.0 * 152 * 2070.0 * 1e6 / 2.25 / 1e9)
    assert "inter_task" not in r
    # alignment modes: packed and int32 peaks; a replayed graph reports the step's rate
    assert b.step_roofline([_stats(6e12, 950.0, 0.0, 0.0)], "global", True, False, 64.0, 152, 2070.0, 6300.0,
                           False)["kernel"] == "k_modes_i16x2"
    r = b.step_roofline([_stats(6e12, 3000.0, 0.0, 0.0)], "overlap", False, False, 64.0, 152, 2070.0, 1990.0,
                        False)
    assert r["kernel"] == "k_modes_i32" and r["peak"] == pytest.approx(64.0 * 152 * 2070.0 * 1e6 / 3.0 / 1e9)
    r = b.step_roofline([_stats(0.0, 0.0, 0.0, 0.0)], "local", True, False, 64.0, 152, 2070.0, 6000.0, True)
    assert r["achieved"] == 6000.0
