"""Global, semi-global and overlap scores on the GPU vs the CPU oracle
(oracle/modes.c), through the C ABI.  Integer scores, tolerance 0; sizes
span several 256-row strips and ragged tails; scores go negative, so the
top-k order of signed scores is checked too."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

MODES = {"global": 1, "semiglobal": 2, "overlap": 3}


def _check(gpu, qs, db, S, o, e, mode, k=10, **kw):
    want = oracle.all_scores(qs, db, S, o, e, mode=mode)
    with gpu.Database(db.residues, db.offsets, S.shape[0]) as d:
        scores, hits, st = d.search(qs.residues, qs.offsets, S, o, e, top_k=k, stats=True,
                                    alignment=MODES[mode], **kw)
    np.testing.assert_array_equal(scores, want)
    for i in range(qs.n):
        ws, wi = oracle.top_k(want[i], k)
        kk = min(k, db.n)
        np.testing.assert_array_equal(hits[i]["score"][:kk], ws[:kk])
        np.testing.assert_array_equal(hits[i]["db_index"], wi)
    return scores, st


@pytest.mark.parametrize("mode", sorted(MODES))
def test_blosum62_strips_and_tails(gpu, mode):
    rng = np.random.default_rng(100 + MODES[mode])
    db = synth.seqset_from_lengths(rng, np.concatenate([rng.integers(1, 600, 150), [0, 1, 255, 256, 257]]))
    qs = synth.seqset_from_lengths(rng, [1, 31, 256, 257, 700])
    scores, st = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode)
    if mode == "global":
        assert (scores < 0).any()
    assert st["precision_used"] == gpu.SW_PREC_I16
    assert st["long_cells"] == 0                      # every pair fits the packed kernel
    _, st32 = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode, precision=gpu.SW_PREC_I32)
    assert st32["precision_used"] == gpu.SW_PREC_I32


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("seed", range(3))
def test_random_matrices_and_penalties(gpu, mode, seed):
    rng = np.random.default_rng(200 + 10 * seed + MODES[mode])
    A = int(rng.integers(2, 25))
    S = synth.random_matrix(rng, A, -8, 12, symmetric=bool(seed % 2))
    o, e = [(10, 1), (2, 5), (0, 3)][seed]                 # includes open < extend and free opening
    db = synth.random_seqset(rng, 80, 0, 400, A)
    qs = synth.random_seqset(rng, 3, 0, 600, A)
    _check(gpu, qs, db, S, o, e, mode)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_empty_sequences(gpu, mode):
    rng = np.random.default_rng(300 + MODES[mode])
    db = synth.seqset_from_lengths(rng, [0, 3, 0, 40])
    qs = synth.seqset_from_lengths(rng, [0, 5, 300])
    _check(gpu, qs, db, synth.blosum62(), 11, 2, mode, k=6)


def test_modes_ordered_like_the_oracle(gpu):
    """global <= semi-global <= overlap <= local on the same search."""
    rng = np.random.default_rng(400)
    db = synth.seqset_from_lengths(rng, rng.integers(1, 500, 120))
    qs = synth.seqset_from_lengths(rng, [90, 400])
    S = synth.blosum62()
    with gpu.Database(db.residues, db.offsets, 24) as d:
        out = {m: d.search(qs.residues, qs.offsets, S, 10, 1, top_k=0, alignment=a)[0]
               for m, a in [("local", 0)] + sorted(MODES.items())}
    assert (out["global"] <= out["semiglobal"]).all()
    assert (out["semiglobal"] <= out["overlap"]).all()
    assert (out["overlap"] <= out["local"]).all()


def test_signed_top_k_entry_point(gpu):
    import torch
    rng = np.random.default_rng(401)
    rows = rng.integers(-50, 50, size=(3, 1000)).astype(np.int32)
    rows[1, :] = -7                                          # all tied, all negative
    sc = torch.from_numpy(rows).cuda()
    hits = torch.empty((3, 12, 2), dtype=torch.int64, device="cuda")
    gpu.sw_top_k(sc, 3, 1000, 12, hits)
    h = hits.cpu().numpy()
    for i in range(3):
        ws, wi = oracle.top_k(rows[i], 12)
        np.testing.assert_array_equal((h[i, :, 0] & 0xffffffff).astype(np.int64).astype(np.int32), ws)
        np.testing.assert_array_equal(h[i, :, 1], wi)


def test_overflow_rejected(gpu):
    rng = np.random.default_rng(402)
    db = synth.seqset_from_lengths(rng, [100, 200])
    qs = synth.seqset_from_lengths(rng, [50])
    with gpu.Database(db.residues, db.offsets, 24) as d:
        with pytest.raises(gpu.SwError, match="SW_ERR_OVERFLOW"):
            d.search(qs.residues, qs.offsets, synth.blosum62(), 1 << 20, 1 << 20, top_k=1, alignment=1)
        with pytest.raises(gpu.SwError, match="SW_ERR_INVALID_ARG"):
            d.search(qs.residues, qs.offsets, synth.blosum62(), 10, 1, top_k=1, alignment=7)


def test_workspace_and_graph(gpu):
    """A caller workspace sized by sw_search_workspace_size, and graph replay."""
    import torch
    rng = np.random.default_rng(403)
    db = synth.seqset_from_lengths(rng, rng.integers(1, 700, 60))
    qs = synth.seqset_from_lengths(rng, [120, 640])
    S = synth.blosum62()
    want = oracle.all_scores(qs, db, S, 10, 1, mode="semiglobal")
    with gpu.Database(db.residues, db.offsets, 24) as d:
        n = gpu.sw_search_workspace_size(d.handle, qs.offsets, 5, alignment=2)
        ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        q_dev = torch.from_numpy(qs.residues).cuda()
        sc = torch.empty((qs.n, db.n), dtype=torch.int32, device="cuda")
        hits = torch.empty((qs.n, 5, 2), dtype=torch.int64, device="cuda")
        for rep in range(3):
            st = gpu.sw_search(d.handle, q_dev, qs.offsets, S, 10, 1, 5, sc, hits, workspace=ws, graph=True,
                               alignment=2, stats=True)
            assert st["graph_replayed"] == (1 if rep > 0 else 0)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(sc.cpu().numpy(), want)
            h = hits.cpu().numpy()
            for i in range(qs.n):
                ws_, wi = oracle.top_k(want[i], 5)
                np.testing.assert_array_equal((h[i, :, 0] & 0xffffffff).astype(np.int64).astype(np.int32), ws_)
                np.testing.assert_array_equal(h[i, :, 1], wi)


# ---- packed int16x2 kernel (k_modes16.cu) ----------------------------------

@pytest.mark.parametrize("rows", [16, 24, 32])
@pytest.mark.parametrize("mode", sorted(MODES))
def test_packed_shapes_and_virtual_rows(gpu, mode, rows):
    """Each shape, with queries that fill whole strips (no virtual rows) and
    queries padded at the top (1 .. 8*rows - 1 virtual rows), one and several
    strips, against pairs of unequal and empty sequences."""
    rng = np.random.default_rng(500 + rows + MODES[mode])
    tr = 8 * rows
    db = synth.seqset_from_lengths(rng, np.concatenate([rng.integers(1, 500, 120), [0, 1, 2, 3, 4, 5, 257, 600]]))
    qs = synth.seqset_from_lengths(rng, [1, tr - 1, tr, tr + 1, 2 * tr, 3 * tr - 5])
    _, st = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode, lanes=8, rows_per_lane=rows)
    assert st["precision_used"] == gpu.SW_PREC_I16
    assert st["rows_per_lane_used"] == rows
    assert st["long_cells"] == 0


@pytest.mark.parametrize("rows", [16, 24, 32])
@pytest.mark.parametrize("mode", sorted(MODES))
def test_packed_last_strip_heights(gpu, mode, rows):
    """The last strip takes the fewest rows per lane (8, 16, 24 or all) that
    cover the rest, with the virtual rows on top making up the difference:
    remainders at and around every 8-row boundary, in one strip and after
    one and two full strips, equal the oracle."""
    rng = np.random.default_rng(520 + rows + MODES[mode])
    tr = 8 * rows
    db = synth.seqset_from_lengths(rng, np.concatenate([rng.integers(1, 400, 90), [0, 1, 5, 300]]))
    rems = sorted({r for b in range(8, rows + 1, 8) for r in (8 * b - 1, 8 * b, 8 * b + 1) if 1 <= r <= tr} | {1})
    qs = synth.seqset_from_lengths(rng, rems + [tr + r for r in rems[::2]] + [2 * tr + r for r in rems[1::3]])
    _, st = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode, lanes=8, rows_per_lane=rows)
    assert st["precision_used"] == gpu.SW_PREC_I16
    assert st["long_cells"] == 0


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("o,e", [(10, 1), (3, 7), (0, 2), (5, 5)])
def test_packed_equals_int32_and_oracle(gpu, mode, o, e):
    """Random non-symmetric matrices; open above, below and equal to extend, and free opening
    (the global virtual rows then score S = -min(o, e) with H(v, 0) = -(o - min(o, e)) = 0 or not)."""
    rng = np.random.default_rng(600 + 7 * o + e + MODES[mode])
    S = synth.random_matrix(rng, 20, -6, 9, symmetric=False)
    db = synth.random_seqset(rng, 90, 0, 700, 20)
    qs = synth.random_seqset(rng, 4, 1, 900, 20)
    packed, st = _check(gpu, qs, db, S, o, e, mode)
    assert st["precision_used"] == gpu.SW_PREC_I16
    i32, _ = _check(gpu, qs, db, S, o, e, mode, precision=gpu.SW_PREC_I32)
    np.testing.assert_array_equal(packed, i32)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_packed_lower_bound_edge(gpu, mode):
    """o = 10, e = 1: g(k) = k + 9.  A pair of Lp columns (the longer length rounded up to
    4) runs packed when g(m) (0 for overlap) + g(Lp) + o + 128 <= 32768.  The pair at the
    largest such Lp runs packed, with global scores near -32,500; the pair above it, int32."""
    rng = np.random.default_rng(700 + MODES[mode])
    m = 100
    gm = 0 if mode == "overlap" else m + 9
    lp = 32768 - 10 - 128 - 9 - gm
    lp -= lp % 4
    db = synth.seqset_from_lengths(rng, [lp + 1, lp + 1, lp, lp - 3, 2000, 10])
    qs = synth.seqset_from_lengths(rng, [m])
    scores, st = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode, k=6)
    assert st["long_cells"] == m * 2 * (lp + 1)        # only the first pair went to int32
    if mode == "global":
        assert scores[0, 2] < -32000


@pytest.mark.parametrize("mode", sorted(MODES))
def test_packed_upper_bound_edge(gpu, mode):
    """BLOSUM62 max(S) = 11 (W/W).  A pair runs packed when 11 * (min(m, Lp) + 1) <= 32767,
    i.e. min(m, Lp) <= 2977: an all-W query of 2977 against an all-W target of 2977 scores
    11 * 2977 = 32,747 in the packed kernel; a query of 2978 sends that pair to int32."""
    w = synth.ALPHABET.index("W")
    rng = np.random.default_rng(800 + MODES[mode])
    other = synth.seqset_from_lengths(rng, [500])
    db = synth.seqset_from_list([np.full(2977, w), np.full(2977, w), other.residues, np.full(3, w)])
    qs = synth.seqset_from_list([np.full(2977, w), np.full(2978, w)])
    scores, st = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode, k=4)
    assert scores[0, 0] == 11 * 2977
    assert st["long_cells"] == 2978 * 2 * 2977         # query 2's first pair only


@pytest.mark.parametrize("mode", sorted(MODES))
def test_packed_column_cap_of_taller_queries(gpu, mode):
    """A query taller than one strip keeps strip-boundary rows for at most 4096 columns:
    a pair of 4100 columns goes to int32, one of exactly 4096 runs packed."""
    rng = np.random.default_rng(900 + MODES[mode])
    db = synth.seqset_from_lengths(rng, [4097, 4096, 4093, 100, 64])
    qs = synth.seqset_from_lengths(rng, [300, 90])
    _, st = _check(gpu, qs, db, synth.blosum62(), 10, 1, mode, k=5)
    assert st["long_cells"] == 300 * (4097 + 4096)     # the 90-row query fits one strip: no cap
