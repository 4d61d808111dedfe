"""Parity at the benchmark's full sizes, in the launch configuration it times.

The oracle cannot score whole workloads of 10^12-10^14 cells, so each
full-size search is checked (a) against the oracle one pair at a time on a
deterministic sample -- every top-k hit, the longest database sequences and
random pairs -- and (b) by properties that hold at any size: every score is
>= 0, the top-k hits are exactly the best entries of the returned score table
in (score desc, index asc) order, and the batched form returns the same full
score table as the plain form.  Scores are integers: tolerance 0.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _hits_consistent(scores_row, hits_row, k):
    s, i = oracle.top_k(scores_row, k)
    np.testing.assert_array_equal(hits_row["score"], s)
    np.testing.assert_array_equal(hits_row["db_index"], i)


def _sample_pairs(w, scores, hits, rng, n_random, n_longest):
    qi, ti = [], []
    for q in range(w.queries.n):                         # every top-k hit
        for t in hits[q]["db_index"]:
            if t >= 0:
                qi.append(q)
                ti.append(int(t))
    longest = np.argsort(w.db.lengths)[::-1][:n_longest]  # the longest database sequences
    for q in range(w.queries.n):
        for t in longest:
            qi.append(q)
            ti.append(int(t))
    qi += list(rng.integers(0, w.queries.n, n_random))   # random pairs
    ti += list(rng.integers(0, w.db.n, n_random))
    qi = np.array(qi, dtype=np.int64)
    ti = np.array(ti, dtype=np.int64)
    want = oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend)
    np.testing.assert_array_equal(scores[qi, ti].astype(np.int64), want)
    return len(qi)


def test_swissprot_like_full_size_plain_and_batched(gpu):
    w = synth.make_workload("swissprot_like_20q")       # the default benchmark workload
    rng = np.random.default_rng(70)
    with gpu.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET)) as d:
        sp, hp, st = d.search(w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                              top_k=w.top_k, stats=True)  # bench's launch configuration (plain, library shapes)
        sb, hb, _ = d.search(w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                             top_k=w.top_k, mode=gpu.SW_MODE_BATCHED)
    assert st["long_sequences"] > 0                      # the long-sequence path took part
    assert (sp >= 0).all()
    np.testing.assert_array_equal(sp, sb)
    np.testing.assert_array_equal(hp, hb)
    for q in range(w.queries.n):
        _hits_consistent(sp[q], hp[q], w.top_k)
    n = _sample_pairs(w, sp, hp, rng, n_random=600, n_longest=3)
    assert n >= 600 + 200


def test_long_queries_full_size(gpu):
    w = synth.make_workload("long_4q_50k")
    rng = np.random.default_rng(71)
    with gpu.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET)) as d:
        s, h, st = d.search(w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                            top_k=w.top_k, stats=True)
    assert st["long_sequences"] >= 4000
    assert (s >= 0).all()
    for q in range(w.queries.n):
        _hits_consistent(s[q], h[q], w.top_k)
    # long x long pairs cost up to 1.2e9 cells each: sample the hits, two long and
    # a few medium sequences, and random pairs
    qi, ti = [], []
    for q in range(w.queries.n):
        for t in h[q]["db_index"][:3]:
            qi.append(q)
            ti.append(int(t))
    order = np.argsort(w.db.lengths)
    picks = [order[-1], order[int(len(order) * 0.95)], order[len(order) // 2], order[0]]
    for q in range(w.queries.n):
        for t in picks:
            qi.append(q)
            ti.append(int(t))
    qi += list(rng.integers(0, w.queries.n, 40))
    ti += list(rng.integers(0, w.db.n, 40))
    qi = np.array(qi, np.int64)
    ti = np.array(ti, np.int64)
    want = oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend)
    np.testing.assert_array_equal(s[qi, ti].astype(np.int64), want)


def test_db2k_q100_in_full(gpu):
    """The small plain workload (1 x 100 vs 2,000 sequences) in full: every
    score and the top-10 equal the oracle's, in the bench's configuration."""
    w = synth.make_workload("db2k_q100")
    with gpu.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET)) as d:
        s, h, _ = d.search(w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                           top_k=w.top_k, stats=True)
    want = oracle.all_scores(w.queries, w.db, w.matrix, w.gap_open, w.gap_extend)
    np.testing.assert_array_equal(s.astype(np.int64), want)
    ws, wi = oracle.top_k(want[0], w.top_k)
    np.testing.assert_array_equal(h[0]["score"], ws)
    np.testing.assert_array_equal(h[0]["db_index"], wi)


def test_batched_512_queries_full_size(gpu):
    """512 queries (50..5,000) against the full 565,000-sequence database in
    the batched form, checked against the oracle on a stratified sample:
    every top-k hit, every rescored pair, 100 pairs among the 100 longest
    targets and 10,000 random pairs; the hits are the best entries of the
    returned score table."""
    w = synth.make_workload("batched_512q")
    rng = np.random.default_rng(73)
    with gpu.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET)) as d:
        s, h, st = d.search(w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                            top_k=w.top_k, mode=gpu.SW_MODE_BATCHED, stats=True)
    assert st["mode_used"] == gpu.SW_MODE_BATCHED and st["long_sequences"] > 0
    assert (s >= 0).all()
    for q in range(w.queries.n):
        _hits_consistent(s[q], h[q], w.top_k)
    qi = [np.repeat(np.arange(w.queries.n), w.top_k)]
    ti = [h["db_index"].reshape(-1)]
    sat = np.argwhere(s >= 32767 - int(w.matrix.max()))          # pairs the int32 rescore produced
    qi.append(sat[:, 0])
    ti.append(sat[:, 1])
    longest = np.argsort(w.db.lengths)[::-1][:100]
    qi.append(rng.integers(0, w.queries.n, 100))
    ti.append(longest)
    qi.append(rng.integers(0, w.queries.n, 10_000))
    ti.append(rng.integers(0, w.db.n, 10_000))
    qi = np.concatenate(qi).astype(np.int64)
    ti = np.concatenate(ti).astype(np.int64)
    assert st["rescored"] == len(sat)
    want = oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend)
    np.testing.assert_array_equal(s[qi, ti].astype(np.int64), want)


def test_batched_512_queries_sampled(gpu):
    w = synth.make_workload("batched_512q", db_scale=0.1)
    rng = np.random.default_rng(72)
    with gpu.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET)) as d:
        s, h, st = d.search(w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                            top_k=w.top_k, mode=gpu.SW_MODE_BATCHED, stats=True)
    assert st["mode_used"] == gpu.SW_MODE_BATCHED
    assert (s >= 0).all()
    for q in range(0, w.queries.n, 7):
        _hits_consistent(s[q], h[q], w.top_k)
    qi = rng.integers(0, w.queries.n, 800).astype(np.int64)
    ti = rng.integers(0, w.db.n, 800).astype(np.int64)
    want = oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend)
    np.testing.assert_array_equal(s[qi, ti].astype(np.int64), want)


def test_traceback_of_the_default_workloads_hits(gpu):
    """sw_align on the 200 top-10 hits of the default workload, in the
    configuration bench.py --align times: every alignment equals the oracle's."""
    w = synth.make_workload("swissprot_like_20q")
    with gpu.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET)) as d:
        _, hits, _ = d.search(w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                              top_k=w.top_k, want_scores=False)
        pq = np.repeat(np.arange(w.queries.n, dtype=np.int32), w.top_k)
        pt = hits["db_index"].reshape(-1).astype(np.int64)
        aln, ops, _ = d.align(w.queries.residues, w.queries.offsets, pq, pt, w.matrix, w.gap_open, w.gap_extend)
    np.testing.assert_array_equal(aln["score"], hits["score"].reshape(-1))
    for k, wa in enumerate(oracle.align_pairs(w.queries, w.db, pq, pt, w.matrix, w.gap_open, w.gap_extend)):
        assert (int(aln["q_begin"][k]), int(aln["q_end"][k]), int(aln["t_begin"][k]), int(aln["t_end"][k])) == \
            (wa["q_begin"], wa["q_end"], wa["t_begin"], wa["t_end"]), k
        o0 = int(aln["ops_offset"][k])
        np.testing.assert_array_equal(ops[o0:o0 + int(aln["ops_len"][k])], wa["ops"])


@pytest.mark.parametrize("mode,code", [("global", 1), ("semiglobal", 2), ("overlap", 3)])
def test_alignment_modes_full_size_sampled(gpu, mode, code):
    """The default workload in each non-local mode (the configuration
    bench.py --alignment times), checked on every top-k hit, the longest
    sequences and random pairs; the hits are the best entries of the table."""
    w = synth.make_workload("swissprot_like_20q")
    rng = np.random.default_rng(80 + code)
    with gpu.Database(w.db.residues, w.db.offsets, len(synth.ALPHABET)) as d:
        s, h, _ = d.search(w.queries.residues, w.queries.offsets, w.matrix, w.gap_open, w.gap_extend,
                           top_k=w.top_k, stats=True, alignment=code)
    for q in range(w.queries.n):
        _hits_consistent(s[q], h[q], w.top_k)
    qi, ti = [], []
    for q in range(w.queries.n):
        for t in h[q]["db_index"]:
            qi.append(q)
            ti.append(int(t))
    longest = np.argsort(w.db.lengths)[::-1][:2]
    for q in range(w.queries.n):
        for t in longest:
            qi.append(q)
            ti.append(int(t))
    qi += list(rng.integers(0, w.queries.n, 400))
    ti += list(rng.integers(0, w.db.n, 400))
    qi = np.array(qi, np.int64)
    ti = np.array(ti, np.int64)
    want = oracle.score_pairs(w.queries, w.db, qi, ti, w.matrix, w.gap_open, w.gap_extend, mode=mode)
    np.testing.assert_array_equal(s[qi, ti].astype(np.int64), want)
