"""A database sharded into several resident handles on one GPU (GPU).

Each shard is loaded with sw_db_load and searched with the full query batch;
the shards' top-k lists are merged with sw_hits_merge and their score rows
scattered with sw_scores_scatter.  The result must equal the unsharded
search and the oracle bit for bit, ties included (many sequences repeat, so
equal scores fall on different shards).  The same exchange step that
bench.py runs between ranks (multigpu.exchange_hits) is checked on the GPU
search's own device output in test_shard_host.py's gloo test form.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _db_with_repeats(rng, n_base, n):
    base = [synth.random_residues(rng, int(x)) for x in
            np.concatenate([rng.integers(2, 700, n_base - 2), [3300, 4100]])]   # long pairs take part
    return synth.seqset_from_list([base[int(i)] for i in rng.integers(0, n_base, n)] + base[-2:])


@pytest.mark.parametrize("n_shards", [2, 3, 5])
def test_sharded_equals_unsharded_and_oracle(gpu, n_shards):
    rng = np.random.default_rng(90 + n_shards)
    db = _db_with_repeats(rng, 150, 900)
    qs = synth.seqset_from_lengths(rng, [40, 333, 1500])
    S = synth.blosum62()
    k = 12
    want = oracle.all_scores(qs, db, S, 10, 1)
    with gpu.Database(db.residues, db.offsets, 24) as d:
        s1, h1, _ = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=k)
    with gpu.ShardedDatabase(db.residues, db.offsets, 24, n_shards) as sd:
        for s in range(n_shards):
            assert sd.shards[s].info()["n_seqs"] == len(sd.shard_members(s))
        ss, hs = sd.search(qs.residues, qs.offsets, S, 10, 1, top_k=k)
        sb, hb = sd.search(qs.residues, qs.offsets, S, 10, 1, top_k=k, mode=gpu.SW_MODE_BATCHED)
    np.testing.assert_array_equal(ss, want)
    np.testing.assert_array_equal(sb, want)
    np.testing.assert_array_equal(ss, s1)
    ties = 0
    for q in range(qs.n):
        ws, wi = oracle.top_k(want[q], k)
        ties += int(len(np.unique(ws)) < k)
        for h in (hs, hb, h1):
            np.testing.assert_array_equal(h[q]["score"], ws)
            np.testing.assert_array_equal(h[q]["db_index"], wi)
    assert ties >= 1


def test_exchange_of_device_hits_single_rank(gpu):
    """The exchange step on a world of one (gloo, in process): the device
    output of sw_search goes through all_gather and the merge unchanged."""
    import os
    import socket

    import torch
    import torch.distributed as dist

    from paper_2203_11100_gb300 import multigpu
    rng = np.random.default_rng(97)
    db = _db_with_repeats(rng, 60, 300)
    qs = synth.seqset_from_lengths(rng, [77, 500])
    S = synth.blosum62()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        members, moff = gpu.sw_shard_plan(db.offsets, 1)
        with gpu.Database(db.residues, db.offsets, 24) as d:
            _, hits, _ = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=10, on_device=True, want_scores=False)
            torch.cuda.synchronize()
            merged = multigpu.exchange_hits(dist, hits.cpu(), members, moff, 10)
    finally:
        dist.destroy_process_group()
    want = oracle.all_scores(qs, db, S, 10, 1)
    for q in range(qs.n):
        ws, wi = oracle.top_k(want[q], 10)
        np.testing.assert_array_equal(merged[q]["score"], ws)
        np.testing.assert_array_equal(merged[q]["db_index"], wi)


def test_sharded_bench_two_ranks(gpu):
    """bench.py's sharded form under torchrun with two ranks (on one GPU the
    ranks share it and exchange over gloo; their kernels never wait on each
    other): one JSON line, strong scaling, both shards' residues, and the
    merged best hits equal to the oracle's scores."""
    import json
    import os
    import socket
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(root, "bench.py"),
           "--gpus", "2", "--steps", "2", "--warmup", "1", "--e2e-steps", "1", "--db-scale", "0.02"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["n_gpus"] == 2 and out["scaling"] == "strong" and out["value"] > 0
    assert len(out["config"]["shard_residues"]) == 2 and min(out["config"]["shard_residues"]) > 0
    assert out["merged_hits_check"]["bit_exact_vs_gpu"] is True
    assert out["e2e"]["value"] > 0
