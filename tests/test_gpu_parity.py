"""GPU search vs the CPU oracle, bit-exact, through the C ABI.

Scores are integers, so the tolerance is zero: every (query, sequence) score
and every top-k hit must equal the oracle's (Section 2.2 recurrences with
the affine gaps of Section 4.1; top-k ordered by score, then index).
Sizes span several bundles, several query passes and ragged tails.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

I16_SHAPES = [(4, 16), (4, 24), (4, 32), (8, 16), (16, 16), (32, 8), (32, 16), (8, 24), (8, 32), (16, 32), (32, 32)]
I32_SHAPES = [(8, 16), (16, 16), (32, 16), (32, 32)]


def _db(rng, n, lo, hi, A=20):
    if A == 20:
        return synth.seqset_from_lengths(rng, rng.integers(lo, hi + 1, n))
    return synth.random_seqset(rng, n, lo, hi, A)


def _check(gpu, qs, db, S, o, e, k=10, **kw):
    A = S.shape[0]
    want = oracle.all_scores(qs, db, S, o, e)
    with gpu.Database(db.residues, db.offsets, A) as d:
        scores, hits, stats = d.search(qs.residues, qs.offsets, S, o, e, top_k=k, stats=True, **kw)
    np.testing.assert_array_equal(scores, want)
    for i in range(qs.n):
        ws, wi = oracle.top_k(want[i], k)
        np.testing.assert_array_equal(hits[i]["score"], ws)
        np.testing.assert_array_equal(hits[i]["db_index"], wi)
    return stats


@pytest.mark.parametrize("lanes,rows", I16_SHAPES)
def test_int16x2_blosum62_shapes(gpu, lanes, rows):
    rng = np.random.default_rng(lanes * 100 + rows)
    db = _db(rng, 293, 1, 400)
    qs = synth.seqset_from_lengths(rng, [1, 37, 128, 129, 700])
    st = _check(gpu, qs, db, synth.blosum62(), 10, 1, precision=gpu.SW_PREC_I16, lanes=lanes,
                rows_per_lane=rows)
    assert st["precision_used"] == gpu.SW_PREC_I16
    assert st["lanes_used"] == lanes and st["rows_per_lane_used"] == rows
    assert st["cells"] == int(qs.lengths.sum()) * int(db.lengths.sum())


@pytest.mark.parametrize("lanes,rows", [(4, 16), (4, 32), (8, 16), (8, 24), (32, 32)])
def test_int16x2_persistent_slots_reused(gpu, lanes, rows):
    """Far more sequence chunks than resident blocks: each block slot takes many
    chunks in turn and reuses its strip-boundary scratch for every pass of every
    chunk (multi-pass queries, ragged last chunk, short and empty sequences)."""
    rng = np.random.default_rng(900 + lanes * 100 + rows)
    db = _db(rng, 120001, 0, 30)
    qs = synth.seqset_from_lengths(rng, [129, 300, 1100])
    _check(gpu, qs, db, synth.blosum62(), 10, 1, precision=gpu.SW_PREC_I16, mode=gpu.SW_MODE_PLAIN,
           lanes=lanes, rows_per_lane=rows)


@pytest.mark.parametrize("lanes,rows", I32_SHAPES)
def test_int32_blosum62_shapes(gpu, lanes, rows):
    rng = np.random.default_rng(7 + lanes * 100 + rows)
    db = _db(rng, 181, 1, 300)
    qs = synth.seqset_from_lengths(rng, [3, 200, 555])
    st = _check(gpu, qs, db, synth.blosum62(), 10, 2, precision=gpu.SW_PREC_I32, lanes=lanes,
                rows_per_lane=rows)
    assert st["precision_used"] == gpu.SW_PREC_I32


@pytest.mark.parametrize("seed", range(6))
def test_random_matrices_and_penalties(gpu, seed):
    rng = np.random.default_rng(300 + seed)
    A = int(rng.integers(2, 25))
    S = synth.random_matrix(rng, A, -8, 12, symmetric=bool(seed % 2))
    o = int(rng.integers(0, 15))
    e = int(rng.integers(0, 6))
    db = _db(rng, 150, 0, 250, A=A)
    qs = synth.random_seqset(rng, 3, 0, 300, A)
    _check(gpu, qs, db, S, o, e, k=7)


def test_open_less_than_extend(gpu):
    rng = np.random.default_rng(11)
    db = _db(rng, 100, 1, 200)
    qs = synth.seqset_from_lengths(rng, [90, 260])
    _check(gpu, qs, db, synth.blosum62(), 1, 4)


def test_paper_penalties_10_2(gpu):
    rng = np.random.default_rng(12)
    db = _db(rng, 400, 2, 600)
    qs = synth.seqset_from_lengths(rng, [144, 500])
    _check(gpu, qs, db, synth.blosum62(), 10, 2)


def test_large_penalties_use_int32(gpu):
    rng = np.random.default_rng(13)
    db = _db(rng, 80, 1, 200)
    qs = synth.seqset_from_lengths(rng, [150])
    st = _check(gpu, qs, db, synth.blosum62() * 20, 200, 30)
    assert st["precision_used"] == gpu.SW_PREC_I32


def test_saturation_rescored_exactly(gpu):
    """Self-hits of long sequences exceed the int16 range and must be rescored."""
    rng = np.random.default_rng(14)
    W = synth.ALPHABET.index("W")
    long_w = np.full(3100, W, dtype=np.uint8)              # 3100 * 11 = 34100 > 32767
    mixed = synth.random_residues(rng, 2500)
    seqs = [synth.random_residues(rng, int(n)) for n in rng.integers(1, 300, 60)]
    seqs[5] = long_w
    seqs[17] = mixed
    seqs[40] = np.concatenate([mixed[:1200], long_w[:3000]])  # W run alone scores 33000
    db = synth.seqset_from_list(seqs)
    qs = synth.seqset_from_list([long_w, mixed, synth.random_residues(rng, 50)])
    st = _check(gpu, qs, db, synth.blosum62(), 10, 1, precision=gpu.SW_PREC_I16)
    assert st["rescored"] >= 2


def test_saturation_inflated_matrix(gpu):
    rng = np.random.default_rng(15)
    A = 4
    S = np.full((A, A), -3, dtype=np.int32)
    np.fill_diagonal(S, 110)                               # 110 + o <= 127 keeps the int8 profile
    base = rng.integers(0, A, 400).astype(np.uint8)        # self score 44000
    seqs = [rng.integers(0, A, int(n)).astype(np.uint8) for n in rng.integers(1, 200, 40)]
    seqs[3] = base
    db = synth.seqset_from_list(seqs)
    qs = synth.seqset_from_list([base, base[:100]])
    st = _check(gpu, qs, db, S, 12, 2, precision=gpu.SW_PREC_I16)
    assert st["rescored"] >= 1


@pytest.mark.parametrize("cutoff", [-1, 0, 64, 300])
def test_long_sequence_split(gpu, cutoff):
    """Sequences longer than the cutoff run in a concurrent launch; scores
    must not depend on where the split falls."""
    rng = np.random.default_rng(22)
    lens = np.concatenate([rng.integers(1, 200, 100), rng.integers(400, 1500, 21), [3500, 3100]])
    rng.shuffle(lens)
    db = synth.seqset_from_lengths(rng, lens)
    qs = synth.seqset_from_lengths(rng, [90, 700])
    st = _check(gpu, qs, db, synth.blosum62(), 10, 1, long_cutoff=cutoff)
    if cutoff > 0:
        assert st["long_sequences"] >= (lens > cutoff).sum()
        assert st["long_cells"] + st["inter_cells"] == st["cells"]
    if cutoff < 0:
        assert st["long_sequences"] == 0


@pytest.mark.parametrize("qlens", [[1, 100, 256], [256, 0, 37], [257, 40]])
def test_long_pairs_of_short_queries(gpu, qlens):
    """Few (long pair, query) tasks with every query within 256 rows: the long pairs run
    in the inter-task kernel at 32 lanes x 8 rows on the side stream (a 257-row query
    falls back to the intra-task kernel).  Within 256 rows an int8 profile cannot
    saturate int16 (at most 117 x 256), so the second matrix only widens the scores."""
    rng = np.random.default_rng(24)
    lens = np.concatenate([rng.integers(1, 300, 150), rng.integers(600, 5000, 12), [9000]])
    rng.shuffle(lens)
    db = synth.seqset_from_lengths(rng, lens)
    qs = synth.seqset_from_lengths(rng, qlens)
    st = _check(gpu, qs, db, synth.blosum62(), 10, 1, long_cutoff=500, precision=gpu.SW_PREC_I16,
                mode=gpu.SW_MODE_PLAIN)
    assert st["long_sequences"] >= (lens > 500).sum()
    S = synth.random_matrix(rng, 24, -20, 110, symmetric=True)
    _check(gpu, qs, db, S, 10, 1, long_cutoff=500, precision=gpu.SW_PREC_I16, mode=gpu.SW_MODE_PLAIN)


@pytest.mark.parametrize("long_rows", [8, 16, 32])
def test_intra_task_multi_superpass(gpu, long_rows):
    """Queries longer than one super-pass of the intra-task kernel (1,024 rows at 8
    rows per lane, 2,048 at 16 and 32), against long sequences of ragged lengths."""
    rng = np.random.default_rng(23)
    lens = np.concatenate([rng.integers(65, 900, 40), rng.integers(1, 64, 30), [1, 2, 3, 4, 5]])
    db = synth.seqset_from_lengths(rng, lens)
    qs = synth.seqset_from_lengths(rng, [2047, 2048, 2049, 4200, 33])
    st = _check(gpu, qs, db, synth.blosum62(), 10, 1, long_cutoff=64, long_rows_per_lane=long_rows)
    assert st["long_sequences"] >= 40


def test_edge_cases(gpu):
    rng = np.random.default_rng(16)
    S = synth.blosum62()
    # zero-length sequences, lengths not multiple of 4, count not multiple of 16
    db = synth.seqset_from_lengths(rng, [0, 1, 2, 3, 5, 0, 7, 33, 0])
    qs = synth.seqset_from_lengths(rng, [0, 1, 4, 31])
    _check(gpu, qs, db, S, 10, 1, k=20)                    # top_k > n_seqs pads with -1
    _check(gpu, qs, db, S, 10, 1, k=1)


def test_empty_database_and_no_queries(gpu):
    S = synth.blosum62()
    empty = synth.SeqSet(np.zeros(0, np.uint8), np.zeros(1, np.int64))
    rng = np.random.default_rng(17)
    qs = synth.seqset_from_lengths(rng, [10, 0])
    with gpu.Database(empty.residues, empty.offsets, 24) as d:
        scores, hits, _ = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=3)
        assert scores.shape == (2, 0)
        assert (hits["score"] == -1).all() and (hits["db_index"] == -1).all()
    db = synth.seqset_from_lengths(rng, [5, 6])
    with gpu.Database(db.residues, db.offsets, 24) as d:
        scores, hits, _ = d.search(np.zeros(0, np.uint8), np.zeros(1, np.int64), S, 10, 1, top_k=3)
        assert scores.shape == (0, 2)


def test_alphabet_of_one(gpu):
    S = np.array([[3]], dtype=np.int32)
    db = synth.SeqSet(np.zeros(10, np.uint8), np.array([0, 4, 10], np.int64))
    qs = synth.SeqSet(np.zeros(6, np.uint8), np.array([0, 6], np.int64))
    _check(gpu, qs, db, S, 2, 1, k=2)


def test_device_buffers_match_host(gpu):
    import torch
    rng = np.random.default_rng(18)
    db = _db(rng, 120, 1, 300)
    qs = synth.seqset_from_lengths(rng, [100, 260])
    S = synth.blosum62()
    with gpu.Database(db.residues, db.offsets, 24) as d:
        hs, hh, _ = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=5)
        q_dev = torch.from_numpy(qs.residues).cuda()
        ds, dh, _ = d.search(q_dev, qs.offsets, S, 10, 1, top_k=5, on_device=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ds.cpu().numpy(), hs)
        dh = dh.cpu().numpy()
        np.testing.assert_array_equal((dh[..., 0] & 0xffffffff).astype(np.int64), hh["score"])
        np.testing.assert_array_equal(dh[..., 1], hh["db_index"])


def test_caller_workspace(gpu):
    import torch
    rng = np.random.default_rng(19)
    db = _db(rng, 64, 1, 200)
    qs = synth.seqset_from_lengths(rng, [300])
    S = synth.blosum62()
    want = oracle.all_scores(qs, db, S, 10, 1)
    with gpu.Database(db.residues, db.offsets, 24) as d:
        n = gpu.sw_search_workspace_size(d.handle, qs.offsets, 10)
        ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        scores = np.empty((1, db.n), np.int32)
        gpu.sw_search(d.handle, qs.residues, qs.offsets, S, 10, 1, 0, scores_out=scores, workspace=ws)
        np.testing.assert_array_equal(scores, want)
        small = torch.empty(16, dtype=torch.uint8, device="cuda")
        with pytest.raises(gpu.SwError):
            gpu.sw_search(d.handle, qs.residues, qs.offsets, S, 10, 1, 0, scores_out=scores, workspace=small)


def test_top_k_entry_point_ties(gpu):
    import torch
    rng = np.random.default_rng(20)
    for n, k in [(0, 3), (5, 10), (1000, 10), (70000, 64), (3000, 4096)]:
        rows = rng.integers(0, 6, size=(3, n)).astype(np.int32)  # heavy ties
        s = torch.from_numpy(rows).cuda()
        hits = torch.empty((3, k, 2), dtype=torch.int64, device="cuda")
        gpu.sw_top_k(s, 3, n, k, hits)
        torch.cuda.synchronize()
        h = hits.cpu().numpy()
        for r in range(3):
            ws, wi = oracle.top_k(rows[r], k)
            np.testing.assert_array_equal((h[r, :, 0] & 0xffffffff).astype(np.int32).astype(np.int64), ws)
            np.testing.assert_array_equal(h[r, :, 1], wi)


def test_invalid_arguments_reported(gpu):
    rng = np.random.default_rng(21)
    db = _db(rng, 10, 1, 20)
    S = synth.blosum62()
    with gpu.Database(db.residues, db.offsets, 24) as d:
        with pytest.raises(gpu.SwError) as e:
            d.search(np.array([30], np.uint8), np.array([0, 1]), S, 10, 1)
        assert e.value.code == 1
        with pytest.raises(gpu.SwError) as e:
            d.search(np.array([3], np.uint8), np.array([0, 1]), S, -1, 1)
        assert e.value.code == 1
        with pytest.raises(gpu.SwError) as e:
            d.search(np.array([3], np.uint8), np.array([0, 1]), S * 40, 10, 1, precision=gpu.SW_PREC_I16)
        assert e.value.code == 6
        with pytest.raises(gpu.SwError) as e:
            d.search(np.array([3], np.uint8), np.array([0, 1]), S, 10, 1, lanes=5)
        assert e.value.code == 6


# --- batched persistent form (query pairs in the int16x2 halves) ------------

BATCH_SHAPES = [(8, 16), (8, 32), (16, 16), (16, 32)]


@pytest.mark.parametrize("lanes,rows", BATCH_SHAPES)
def test_batched_matches_oracle(gpu, lanes, rows):
    rng = np.random.default_rng(40 + lanes + rows)
    db = _db(rng, 333, 1, 500)
    qs = synth.seqset_from_lengths(rng, [0, 1, 17, 130, 131, 256, 257, 700, 64])   # odd count, one empty
    st = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode=gpu.SW_MODE_BATCHED, lanes=lanes,
                rows_per_lane=rows)
    assert st["mode_used"] == gpu.SW_MODE_BATCHED
    assert st["inter_launches"] == 1


def test_batched_long_split_and_saturation(gpu):
    rng = np.random.default_rng(41)
    W = synth.ALPHABET.index("W")
    seqs = [synth.random_residues(rng, int(n)) for n in rng.integers(1, 900, 120)]
    seqs[3] = np.full(3100, W, dtype=np.uint8)                      # long and saturating
    seqs[50] = np.concatenate([synth.random_residues(rng, 300), np.full(3000, W, np.uint8)])
    seqs[51] = np.full(2990, W, dtype=np.uint8)                     # saturates, not long at cutoff 3072
    db = synth.seqset_from_list(seqs)
    qs = synth.seqset_from_list([np.full(3050, W, np.uint8), synth.random_residues(rng, 2200),
                                 synth.random_residues(rng, 40)])
    for cutoff in (0, 200):
        st = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode=gpu.SW_MODE_BATCHED, long_cutoff=cutoff)
        assert st["rescored"] >= 3


def test_batched_equals_plain(gpu):
    rng = np.random.default_rng(42)
    db = _db(rng, 2000, 2, 1200)
    qs = synth.seqset_from_lengths(rng, rng.integers(1, 1500, 11))
    S = synth.blosum62()
    with gpu.Database(db.residues, db.offsets, 24) as d:
        sp, hp, _ = d.search(qs.residues, qs.offsets, S, 11, 1, top_k=25, mode=gpu.SW_MODE_PLAIN)
        sb, hb, _ = d.search(qs.residues, qs.offsets, S, 11, 1, top_k=25, mode=gpu.SW_MODE_BATCHED)
    np.testing.assert_array_equal(sp, sb)
    np.testing.assert_array_equal(hp, hb)


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_graph_capture_and_replay(gpu, mode):
    """The captured work replays exactly, and reads new query contents."""
    import torch
    m = gpu.SW_MODE_PLAIN if mode == "plain" else gpu.SW_MODE_BATCHED
    rng = np.random.default_rng(60)
    lens = np.concatenate([rng.integers(1, 700, 200), [3300, 3500]])   # includes long sequences
    db = synth.seqset_from_lengths(rng, lens)
    S = synth.blosum62()
    qlens = [90, 300, 1200]
    with gpu.Database(db.residues, db.offsets, 24) as d:
        q_off = np.concatenate([[0], np.cumsum(qlens)]).astype(np.int64)
        q_dev = torch.empty(int(q_off[-1]), dtype=torch.uint8, device="cuda")
        scores = torch.empty((len(qlens), db.n), dtype=torch.int32, device="cuda")
        hits = torch.empty((len(qlens), 5, 2), dtype=torch.int64, device="cuda")
        for rep in range(3):
            qs = synth.seqset_from_lengths(rng, qlens)       # new contents, same lengths
            q_dev.copy_(torch.from_numpy(qs.residues))
            st = gpu.sw_search(d.handle, q_dev, q_off, S, 10, 1, 5, scores, hits, mode=m, graph=True, stats=True)
            assert st["graph_replayed"] == (1 if rep > 0 else 0)
            torch.cuda.synchronize()
            want = oracle.all_scores(qs, db, S, 10, 1)
            np.testing.assert_array_equal(scores.cpu().numpy(), want)
            h = hits.cpu().numpy()
            for i in range(len(qlens)):
                ws, wi = oracle.top_k(want[i], 5)
                np.testing.assert_array_equal((h[i, :, 0] & 0xffffffff).astype(np.int64), ws)
                np.testing.assert_array_equal(h[i, :, 1], wi)
        # a different signature (other penalties) captures again
        st = gpu.sw_search(d.handle, q_dev, q_off, S, 11, 2, 5, scores, hits, mode=m, graph=True, stats=True)
        assert st["graph_replayed"] == 0


def test_autotune_picks_and_caches(gpu, tmp_path):
    """The autotuner measures the shape tables, cutoff and form, installs them
    on the handle, caches them, and the tuned searches (explicit parameters
    and SW_MODE_AUTO) still equal the oracle."""
    from paper_2203_11100_gb300 import autotune
    rng = np.random.default_rng(61)
    db = synth.seqset_from_lengths(rng, synth.lognormal_lengths(rng, 3000, 360.0, 2, 5000))
    qs = synth.seqset_from_lengths(rng, rng.integers(50, 1500, 12))
    S = synth.blosum62()
    cache = tmp_path / "tune.json"
    with gpu.Database(db.residues, db.offsets, 24) as d:
        params = autotune.autotune(d, qs.residues, qs.offsets, S, 10, 1, sample_queries=4, cache_path=str(cache),
                                   cutoffs=(0, 1024), repeats=2)
        first = autotune.last_result()
        assert cache.exists() and not first["cached"]
        assert set(params) == {"mode", "long_cutoff"} and params["long_cutoff"] in (0, 1024)
        tuned = gpu.sw_db_get_tuning(d.handle)
        assert len(tuned["plain"]) == len(autotune.PLAIN_SHAPES)
        assert len(tuned["batched"]) == len(autotune.BATCH_SHAPES)
        assert all(g > 0 for _, _, g in tuned["plain"] + tuned["batched"])
        assert tuned["mode"] == params["mode"] and tuned["long_cutoff"] == params["long_cutoff"]
        gpu.sw_db_set_tuning(d.handle, None)
        assert gpu.sw_db_get_tuning(d.handle)["long_cutoff"] == 0
        again = autotune.autotune(d, qs.residues, qs.offsets, S, 10, 1, cache_path=str(cache))
        assert again == params and autotune.last_result()["cached"]
        assert gpu.sw_db_get_tuning(d.handle) == tuned                 # reinstalled from the cache
        scores, _, _ = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=0, **params)
        auto, _, st = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=0, stats=True)   # SW_MODE_AUTO
        assert st["mode_used"] == params["mode"]
    want = oracle.all_scores(qs, db, S, 10, 1)
    np.testing.assert_array_equal(scores, want)
    np.testing.assert_array_equal(auto, want)


def test_tuned_tables_drive_the_shape_choice(gpu):
    """A table with one plain shape makes every query of a search use it; a
    shape the kernel does not support is rejected; scores stay exact."""
    rng = np.random.default_rng(62)
    db = _db(rng, 500, 1, 700)
    qs = synth.seqset_from_lengths(rng, [90, 700, 2000])
    S = synth.blosum62()
    with gpu.Database(db.residues, db.offsets, 24) as d:
        gpu.sw_db_set_tuning(d.handle, {"plain": [(16, 32, 1000.0)], "batched": [(8, 24, 1000.0)]})
        scores, _, st = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=0, stats=True, mode=gpu.SW_MODE_PLAIN)
        assert (st["lanes_used"], st["rows_per_lane_used"]) == (16, 32)
        sb, _, stb = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=0, stats=True, mode=gpu.SW_MODE_BATCHED)
        assert (stb["lanes_used"], stb["rows_per_lane_used"]) == (8, 24)
        with pytest.raises(gpu.SwError):
            gpu.sw_db_set_tuning(d.handle, {"plain": [(8, 40, 1000.0)]})
        with pytest.raises(gpu.SwError):
            gpu.sw_db_set_tuning(d.handle, {"plain": [(8, 16, -1.0)]})
    want = oracle.all_scores(qs, db, S, 10, 1)
    np.testing.assert_array_equal(scores, want)
    np.testing.assert_array_equal(sb, want)


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_workspace_bound_covers_mixed_batches(gpu, mode):
    """A workspace sized for n queries of the maximum length fits every batch
    of at most n queries no longer than that (how the server sizes its own)."""
    import torch
    m = gpu.SW_MODE_PLAIN if mode == "plain" else gpu.SW_MODE_BATCHED
    rng = np.random.default_rng(80)
    db = synth.seqset_from_lengths(rng, np.concatenate([rng.integers(1, 900, 400), [3500, 4100]]))
    S = synth.blosum62()
    n, maxlen = 8, 3000
    with gpu.Database(db.residues, db.offsets, 24) as d:
        bound = gpu.sw_search_workspace_size(d.handle, np.arange(n + 1, dtype=np.int64) * maxlen, 10, mode=m)
        ws = torch.empty(bound, dtype=torch.uint8, device="cuda")
        for lens in ([3000, 40, 100, 129, 250, 700, 2999, 1], [5, 6], [3000] * 8, [64] * 7):
            qs = synth.seqset_from_lengths(rng, lens)
            scores = np.empty((qs.n, db.n), np.int32)
            gpu.sw_search(d.handle, qs.residues, qs.offsets, S, 10, 1, 0, scores_out=scores, workspace=ws, mode=m)
            np.testing.assert_array_equal(scores, oracle.all_scores(qs, db, S, 10, 1))


def test_batched_single_query_runs_plain(gpu):
    """A batched search with one non-empty query (nothing to pair it with) runs
    in the plain form, exactly, and a workspace sized for the batched form of
    that many queries still fits it."""
    import torch
    rng = np.random.default_rng(64)
    db = _db(rng, 300, 1, 900)
    S = synth.blosum62()
    for lens in ([700], [0, 333, 0]):
        qs = synth.seqset_from_lengths(rng, lens)
        st = _check(gpu, qs, db, S, 10, 1, mode=gpu.SW_MODE_BATCHED)
        assert st["mode_used"] == gpu.SW_MODE_PLAIN
    with gpu.Database(db.residues, db.offsets, 24) as d:
        off = np.array([0, 700], np.int64)
        ws = torch.empty(gpu.sw_search_workspace_size(d.handle, off, 10, mode=gpu.SW_MODE_BATCHED),
                         dtype=torch.uint8, device="cuda")
        q = synth.seqset_from_lengths(rng, [700])
        scores = np.empty((1, db.n), np.int32)
        gpu.sw_search(d.handle, q.residues, q.offsets, S, 10, 1, 0, scores_out=scores, workspace=ws,
                      mode=gpu.SW_MODE_BATCHED)
    np.testing.assert_array_equal(scores, oracle.all_scores(q, db, S, 10, 1))


@pytest.mark.parametrize("lanes,rows", [(8, 32), (8, 24), (8, 16), (32, 32), (4, 32)])
def test_last_strip_heights(gpu, lanes, rows):
    """The last strip of a query takes the fewest rows per lane (a multiple of
    8) that cover its remaining rows: remainders at and around every such
    boundary, after one and after several full strips, equal the oracle."""
    rng = np.random.default_rng(66 + lanes + rows)
    db = _db(rng, 120, 1, 500)
    tr = lanes * rows
    rems = sorted({r for b in range(8, rows + 1, 8) for r in (lanes * b - 1, lanes * b, lanes * b + 1)
                   if 1 <= r <= tr} | {1, tr})
    qlens = [r for r in rems] + [2 * tr + r for r in rems[::3]]
    qs = synth.seqset_from_lengths(rng, qlens)
    _check(gpu, qs, db, synth.blosum62(), 10, 1, lanes=lanes, rows_per_lane=rows)


@pytest.mark.parametrize("lanes,rows", [(8, 32), (8, 24), (8, 16), (16, 32)])
def test_batched_last_strip_heights(gpu, lanes, rows):
    """The batched kernel sizes a pair's last strip by its longer query, the
    fewest rows per lane (a multiple of 8) that cover the rest: pairs whose
    remainders sit at and around every such boundary equal the oracle."""
    rng = np.random.default_rng(77 + lanes + rows)
    db = _db(rng, 120, 1, 500)
    tr = lanes * rows
    rems = sorted({r for b in range(8, rows + 1, 8) for r in (lanes * b - 1, lanes * b, lanes * b + 1)
                   if 1 <= r <= tr} | {1, tr})
    qlens = rems + [2 * tr + r for r in rems[::2]] + [5]
    qs = synth.seqset_from_lengths(rng, qlens)
    st = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode=gpu.SW_MODE_BATCHED, lanes=lanes,
                rows_per_lane=rows)
    assert st["mode_used"] == gpu.SW_MODE_BATCHED
