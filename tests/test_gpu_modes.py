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
    assert st["precision_used"] == gpu.SW_PREC_I32


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
