"""Served results equal the same query searched alone (GPU).

The server batches requests as they arrive and overlaps batches on several
streams; each query's top-k hits must be identical to those of a plain
search of that query by itself (scores are integers: tolerance 0), whatever
batch it landed in and whichever queries shared it.
"""
import threading
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_served_equals_alone(gpu):
    from paper_2203_11100_gb300.serve import SearchServer
    rng = np.random.default_rng(50)
    db = synth.seqset_from_lengths(rng, synth.lognormal_lengths(rng, 3000, 360.0, 2, 4000))
    S = synth.blosum62()
    W = synth.ALPHABET.index("W")
    queries = [synth.random_residues(rng, int(n)) for n in rng.integers(30, 900, 40)]
    queries[7] = np.full(3200, W, dtype=np.uint8)          # saturating, multi-pass
    queries[11] = np.zeros(0, dtype=np.uint8)              # empty query
    with gpu.Database(db.residues, db.offsets, 24) as d:
        alone = []
        for q in queries:
            _, hits, _ = d.search(q, np.array([0, len(q)], np.int64), S, 10, 1, top_k=10,
                                  want_scores=False, mode=gpu.SW_MODE_PLAIN)
            alone.append(hits[0])
        srv = SearchServer(d, S, 10, 1, top_k=10, max_batch=8, streams=3, max_query_len=4000)
        futures = [None] * len(queries)

        def client(idx):
            for i in idx:
                time.sleep(float(rng.uniform(0, 0.003)))
                futures[i] = srv.submit(queries[i])

        threads = [threading.Thread(target=client, args=(list(range(k, len(queries), 4)),)) for k in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        served = [f.result(timeout=120) for f in futures]
        st = srv.stats()
        srv.close()
    for i, (a, b) in enumerate(zip(alone, served)):
        np.testing.assert_array_equal(a["score"], b["score"], err_msg=f"query {i}")
        np.testing.assert_array_equal(a["db_index"], b["db_index"], err_msg=f"query {i}")
    assert st["completed"] == len(queries)
    assert st["batches"] >= 2 and st["p99_ms"] >= st["p50_ms"] > 0


def test_memory_budget_limits_batches(gpu):
    from paper_2203_11100_gb300.serve import SearchServer
    rng = np.random.default_rng(51)
    db = synth.seqset_from_lengths(rng, rng.integers(10, 300, 500))
    S = synth.blosum62()
    queries = [synth.random_residues(rng, 100) for _ in range(12)]
    with gpu.Database(db.residues, db.offsets, 24) as d:
        one = 100 + 500 * 4 + 10 * 16 + (500 // 2 + 16) * 4 + 32 * 4 * 356
        srv = SearchServer(d, S, 10, 1, top_k=10, max_batch=8, streams=2, mem_budget=2 * one, max_query_len=200)
        futs = [srv.submit(q) for q in queries]
        res = [f.result(timeout=60) for f in futs]
        st = srv.stats()
        srv.close()
        assert max(srv.batch_sizes) <= 2
        for q, r in zip(queries, res):
            _, hits, _ = d.search(q, np.array([0, len(q)], np.int64), S, 10, 1, top_k=10, want_scores=False)
            np.testing.assert_array_equal(hits[0]["score"], r["score"])
            np.testing.assert_array_equal(hits[0]["db_index"], r["db_index"])
    assert st["completed"] == 12
