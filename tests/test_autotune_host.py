"""Host-side pieces of the autotuner (no GPU): sampling and cache keys."""
import numpy as np

from paper_2203_11100_gb300 import autotune


def test_sample_spreads_over_lengths():
    lens = np.array([5, 100, 7, 3000, 40, 900, 60, 1500])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    res = np.arange(off[-1], dtype=np.int64).astype(np.uint8)
    s_res, s_off = autotune._sample(res, off, 3)
    got = sorted(np.diff(s_off).tolist())
    assert got == [5, 100, 3000] or got[0] == 5 and got[-1] == 3000
    assert len(s_res) == s_off[-1]


def test_batch_key_depends_on_shape():
    info = {"n_seqs": 10, "residues": 1000, "max_length": 300}
    k1 = autotune._batch_key(info, np.array([100, 200, 300]))
    k2 = autotune._batch_key(info, np.array([1000, 2000, 3000]))
    k3 = autotune._batch_key(info, np.array([100, 200, 300]))
    assert k1 != k2 and k1 == k3


def test_search_key_separates_matrix_penalties_and_precision(monkeypatch):
    from paper_2203_11100_gb300 import binding
    monkeypatch.setattr(binding, "sw_version", lambda: "v")
    S = np.eye(4, dtype=np.int32)
    T = S.copy()
    T[0, 1] = 2
    k = autotune._search_key(S, 10, 1, 1)
    assert k == autotune._search_key(S.copy(), 10, 1, 1)
    assert k != autotune._search_key(T, 10, 1, 1)
    assert k != autotune._search_key(S, 10, 2, 1)
    assert k != autotune._search_key(S, 11, 1, 1)
    assert k != autotune._search_key(S, 10, 1, 2)


def test_probe_queries_are_whole_strips_of_the_batch():
    res = np.arange(100, dtype=np.uint8) % 20
    q, off = autotune._probe_queries(res, 2)
    assert off.tolist() == [0, autotune.RATE_ROWS, 2 * autotune.RATE_ROWS]
    assert len(q) == 2 * autotune.RATE_ROWS and np.array_equal(q[:100], res)
    for lanes, rows in autotune.PLAIN_SHAPES + autotune.BATCH_SHAPES:
        assert autotune.RATE_ROWS % (lanes * rows) == 0


def test_probe_rows_shrink_for_huge_databases():
    assert autotune.probe_rows(200_000_000) == 3072          # the default workload's database
    assert autotune.probe_rows(1_000_000_000) == 1536
    assert autotune.probe_rows(7_200_000_000) == 768          # the 20M-sequence serving database
    assert autotune.probe_rows(10**12) == 768
