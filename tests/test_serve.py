"""Served results equal the same query searched alone, and the oracle (GPU).

The server batches requests as they arrive and overlaps batches on several
streams; each query's top-k hits must be identical to those of a plain
search of that query by itself and to the oracle's top-k of the query's
exact scores (scores are integers: tolerance 0), whatever batch it landed in
and whichever queries shared it.
"""
import threading
import time

import numpy as np
import pytest

import oracle
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
    qs = synth.seqset_from_list(queries)
    want = oracle.all_scores(qs, db, S, 10, 1)
    for i, (a, b) in enumerate(zip(alone, served)):
        np.testing.assert_array_equal(a["score"], b["score"], err_msg=f"query {i}")
        np.testing.assert_array_equal(a["db_index"], b["db_index"], err_msg=f"query {i}")
        ws, wi = oracle.top_k(want[i], 10)
        np.testing.assert_array_equal(b["score"], ws, err_msg=f"query {i} vs oracle")
        np.testing.assert_array_equal(b["db_index"], wi, err_msg=f"query {i} vs oracle")
    assert st["completed"] == len(queries)
    assert st["batches"] >= 2 and st["p99_ms"] >= st["p50_ms"] > 0
    assert st["peak_in_flight_bytes"] <= st["mem_budget"]


def test_memory_budget_limits_batches(gpu):
    """A budget that holds the workspace of two queries but not three: no
    batch exceeds two, the bytes in flight never exceed the budget, and every
    result equals the oracle's top-k."""
    from paper_2203_11100_gb300.serve import SearchServer
    rng = np.random.default_rng(51)
    db = synth.seqset_from_lengths(rng, rng.integers(10, 300, 500))
    S = synth.blosum62()
    queries = [synth.random_residues(rng, 100) for _ in range(12)]
    with gpu.Database(db.residues, db.offsets, 24) as d:
        ws = [gpu.sw_search_workspace_size(d.handle, np.arange(k + 1, dtype=np.int64) * 100, 10,
                                           mode=gpu.SW_MODE_BATCHED) for k in (1, 2, 3)]
        assert ws[0] < ws[1] < ws[2]
        budget = ws[1] + 256
        srv = SearchServer(d, S, 10, 1, top_k=10, max_batch=8, streams=2, mem_budget=budget, max_query_len=200)
        futs = [srv.submit(q) for q in queries]
        res = [f.result(timeout=60) for f in futs]
        st = srv.stats()
        srv.close()
        assert max(srv.batch_sizes) <= 2
        assert st["peak_in_flight_bytes"] <= budget
        # a query whose own workspace exceeds the budget fails, the server goes on
        small = SearchServer(d, S, 10, 1, top_k=10, max_batch=8, streams=2, mem_budget=ws[0] // 2,
                             max_query_len=200)
        with pytest.raises(MemoryError):
            small.submit(queries[0]).result(timeout=60)
        small.close()
    want = oracle.all_scores(synth.seqset_from_list(queries), db, S, 10, 1)
    for i, r in enumerate(res):
        s_, i_ = oracle.top_k(want[i], 10)
        np.testing.assert_array_equal(r["score"], s_)
        np.testing.assert_array_equal(r["db_index"], i_)
    assert st["completed"] == 12
