"""GPU traceback (sw_align) vs the CPU oracle's traceback, through the C ABI.

Alignments are integer data: score, the four coordinates and every op must
equal the oracle's (oracle/traceback.c: end cell first in row-major order,
diagonal before E before F, gaps open as soon as they can, stop at the
first H = 0).  Sizes span several 256-row strips with ragged tails, small
alphabets with free gap opening (many equal-score alternatives), and the
edge cases (empty sequences, zero scores, one residue, repeated pairs).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _check_pairs(gpu, qs, db, S, o, e, pq, pt, A=None, mode="local"):
    A = A or S.shape[0]
    with gpu.Database(db.residues, db.offsets, A) as d:
        aln, ops, st = d.align(qs.residues, qs.offsets, pq, pt, S, o, e, stats=True,
                               alignment=oracle.MODES[mode])
    want = oracle.align_pairs(qs, db, pq, pt, S, o, e, mode=mode)
    for k, w in enumerate(want):
        a = aln[k]
        got = {"score": int(a["score"]), "q_begin": int(a["q_begin"]), "q_end": int(a["q_end"]),
               "t_begin": int(a["t_begin"]), "t_end": int(a["t_end"])}
        exp = {x: w[x] for x in got}
        assert got == exp, (k, int(pq[k]), int(pt[k]), got, exp)
        g_ops = ops[int(a["ops_offset"]):int(a["ops_offset"]) + int(a["ops_len"])]
        np.testing.assert_array_equal(g_ops, w["ops"], err_msg=f"pair {k}")
    return aln, ops, st


def _all_pairs(nq, nt):
    pq = np.repeat(np.arange(nq, dtype=np.int32), nt)
    pt = np.tile(np.arange(nt, dtype=np.int64), nq)
    return pq, pt


def test_blosum62_several_strips(gpu):
    rng = np.random.default_rng(1)
    db = synth.seqset_from_lengths(rng, [1, 2, 255, 256, 257, 600, 1100, 31, 0, 90])
    qs = synth.seqset_from_lengths(rng, [1, 100, 256, 257, 513, 800])
    pq, pt = _all_pairs(qs.n, db.n)
    _, _, st = _check_pairs(gpu, qs, db, synth.blosum62(), 10, 1, pq, pt)
    assert st["forward_cells"] == int(sum(qs.lengths[pq] * db.lengths[pt]))


def test_related_sequences_with_gaps(gpu):
    """Targets derived from the queries by substitutions, insertions and
    deletions: long alignments with many gaps crossing strip boundaries."""
    rng = np.random.default_rng(2)
    qlist, tlist = [], []
    for L in (300, 700, 1000):
        q = rng.integers(0, 20, L).astype(np.uint8)
        t = []
        for x in q:
            u = rng.random()
            if u < 0.05:
                continue                                       # deletion
            if u < 0.10:
                t.extend(rng.integers(0, 20, int(rng.integers(1, 6))))   # insertion run
            t.append(int(rng.integers(0, 20)) if rng.random() < 0.2 else int(x))
        qlist.append(q)
        tlist.append(np.array(t, np.uint8))
    qs = synth.seqset_from_list(qlist)
    db = synth.seqset_from_list(tlist)
    pq, pt = _all_pairs(qs.n, db.n)
    for o, e in ((10, 1), (11, 2), (5, 5), (2, 4)):
        aln, _, _ = _check_pairs(gpu, qs, db, synth.blosum62(), o, e, pq, pt)
        assert (aln["score"][pq == pt] > 500).all()


@pytest.mark.parametrize("seed", range(4))
def test_small_alphabets_many_ties(gpu, seed):
    rng = np.random.default_rng(10 + seed)
    A = int(rng.integers(2, 4))
    S = rng.integers(-3, 5, size=(A, A)).astype(np.int32)
    o = [0, 0, 1, 3][seed]
    e = int(rng.integers(0, 3))
    db = synth.random_seqset(rng, 12, 0, 400, A)
    qs = synth.random_seqset(rng, 4, 1, 600, A)
    pq, pt = _all_pairs(qs.n, db.n)
    _check_pairs(gpu, qs, db, S, o, e, pq, pt)


@pytest.mark.parametrize("seed", range(3))
def test_random_matrices(gpu, seed):
    rng = np.random.default_rng(30 + seed)
    A = int(rng.integers(2, 25))
    S = synth.random_matrix(rng, A, -8, 12, symmetric=bool(seed % 2))
    o, e = int(rng.integers(0, 15)), int(rng.integers(0, 6))
    db = synth.random_seqset(rng, 20, 0, 700, A)
    qs = synth.random_seqset(rng, 3, 0, 700, A)
    pq, pt = _all_pairs(qs.n, db.n)
    _check_pairs(gpu, qs, db, S, o, e, pq, pt)


def test_edge_cases(gpu):
    rng = np.random.default_rng(40)
    S = synth.blosum62()
    db = synth.seqset_from_lengths(rng, [0, 1, 5, 300])
    qs = synth.seqset_from_lengths(rng, [0, 1, 257])
    pq = np.array([0, 0, 1, 1, 2, 2, 2, 2, 2, 1], np.int32)        # repeated pairs included
    pt = np.array([0, 3, 0, 1, 0, 1, 2, 3, 3, 1], np.int64)
    aln, _, _ = _check_pairs(gpu, qs, db, S, 10, 1, pq, pt)
    assert aln["score"][0] == 0 and aln["ops_len"][0] == 0
    neg = -np.abs(S) - 1                                             # every H is 0
    aln, _, _ = _check_pairs(gpu, qs, db, neg.astype(np.int32), 3, 1, pq, pt)
    assert (aln["score"] == 0).all() and (aln["ops_len"] == 0).all()
    with gpu.Database(db.residues, db.offsets, 24) as d:
        a, ops, _ = d.align(qs.residues, qs.offsets, np.zeros(0, np.int32), np.zeros(0, np.int64), S, 10, 1)
        assert len(a) == 0


def test_hits_of_a_search_and_scores_agree(gpu):
    """Align the top-k hits of a search: the alignment score equals the search
    score, and the alignments equal the oracle's."""
    rng = np.random.default_rng(50)
    db = synth.seqset_from_lengths(rng, synth.lognormal_lengths(rng, 3000, 360.0, 2, 4000))
    qs = synth.seqset_from_lengths(rng, [144, 466, 1500])
    S = synth.blosum62()
    with gpu.Database(db.residues, db.offsets, 24) as d:
        scores, hits, _ = d.search(qs.residues, qs.offsets, S, 10, 1, top_k=10)
        pq = np.repeat(np.arange(qs.n, dtype=np.int32), 10)
        pt = hits["db_index"].reshape(-1).astype(np.int64)
        aln, ops, _ = d.align(qs.residues, qs.offsets, pq, pt, S, 10, 1)
    np.testing.assert_array_equal(aln["score"], hits["score"].reshape(-1))
    want = oracle.align_pairs(qs, db, pq, pt, S, 10, 1)
    for k, w in enumerate(want):
        assert (int(aln["q_begin"][k]), int(aln["q_end"][k]), int(aln["t_begin"][k]), int(aln["t_end"][k])) == \
            (w["q_begin"], w["q_end"], w["t_begin"], w["t_end"])
        o0 = int(aln["ops_offset"][k])
        np.testing.assert_array_equal(ops[o0:o0 + int(aln["ops_len"][k])], w["ops"])


def test_pairs_beyond_one_chunk(gpu):
    """More scratch than one chunk (1 GiB): 100 pairs of 2,000 x 35,000."""
    rng = np.random.default_rng(60)
    db = synth.seqset_from_lengths(rng, [35000] * 100)
    qs = synth.seqset_from_lengths(rng, [2000] * 4)
    pq = (np.arange(100) % 4).astype(np.int32)
    pt = np.arange(100, dtype=np.int64)
    _check_pairs(gpu, qs, db, synth.blosum62(), 10, 1, pq, pt)


def test_more_strips_than_warps(gpu):
    """Queries of 9 and 12 strips: warps of the forward pass take a second
    strip each (the wavefront wraps around the CTA's 8 warps)."""
    rng = np.random.default_rng(70)
    db = synth.seqset_from_lengths(rng, [1, 700, 2500, 4100])
    qs = synth.seqset_from_lengths(rng, [2049, 3000])
    pq, pt = _all_pairs(qs.n, db.n)
    for o, e in ((10, 1), (3, 5), (0, 2)):
        _check_pairs(gpu, qs, db, synth.blosum62(), o, e, pq, pt)


# ---- non-local modes (sw_align_mode; oracle/align_modes.c) -------------------

MODE_NAMES = ["global", "semiglobal", "overlap"]


@pytest.mark.parametrize("mode", MODE_NAMES)
def test_modes_several_strips(gpu, mode):
    """Every pair of queries spanning 1-4 strips (ragged tails) and targets from 1 to
    1,100 residues, including empty ones: score, coordinates and every op."""
    rng = np.random.default_rng(300 + MODE_NAMES.index(mode))
    db = synth.seqset_from_lengths(rng, [1, 2, 255, 256, 257, 600, 1100, 31, 0, 90])
    qs = synth.seqset_from_lengths(rng, [1, 100, 256, 257, 513, 800, 0])
    pq, pt = _all_pairs(qs.n, db.n)
    aln, _, _ = _check_pairs(gpu, qs, db, synth.blosum62(), 10, 1, pq, pt, mode=mode)
    if mode == "global":
        assert (aln["score"] < 0).any()


@pytest.mark.parametrize("mode", MODE_NAMES)
@pytest.mark.parametrize("o,e", [(0, 2), (3, 7), (5, 5)])
def test_modes_ties_and_penalties(gpu, mode, o, e):
    """A 3-letter alphabet with free or cheap gap opening: many equal-score paths, so the
    end cell and every step follow the tie rules; open below, above and equal to extend."""
    rng = np.random.default_rng(400 + 10 * o + e + MODE_NAMES.index(mode))
    S = rng.integers(-2, 3, size=(3, 3)).astype(np.int32)
    db = synth.random_seqset(rng, 40, 0, 300, 3)
    qs = synth.random_seqset(rng, 3, 0, 400, 3)
    pq, pt = _all_pairs(qs.n, db.n)
    _check_pairs(gpu, qs, db, S, o, e, pq, pt, mode=mode)


@pytest.mark.parametrize("mode", MODE_NAMES)
def test_mode_alignment_scores_equal_search_scores(gpu, mode):
    """The alignment's score is the mode's search score of the same pair."""
    rng = np.random.default_rng(500 + MODE_NAMES.index(mode))
    db = synth.seqset_from_lengths(rng, rng.integers(0, 700, 60))
    qs = synth.seqset_from_lengths(rng, [50, 333])
    S = synth.blosum62()
    with gpu.Database(db.residues, db.offsets, 24) as d:
        scores, _, _ = d.search(qs.residues, qs.offsets, S, 11, 1, top_k=0, alignment=oracle.MODES[mode])
        pq, pt = _all_pairs(qs.n, db.n)
        aln, _, _ = d.align(qs.residues, qs.offsets, pq, pt, S, 11, 1, alignment=oracle.MODES[mode])
    np.testing.assert_array_equal(aln["score"].reshape(qs.n, db.n), scores)


def test_mode_alignment_rejects_unknown_mode_and_overflow(gpu):
    rng = np.random.default_rng(600)
    db = synth.seqset_from_lengths(rng, [100, 200])
    qs = synth.seqset_from_lengths(rng, [50])
    with gpu.Database(db.residues, db.offsets, 24) as d:
        with pytest.raises(gpu.SwError, match="SW_ERR_INVALID_ARG"):
            d.align(qs.residues, qs.offsets, [0], [0], synth.blosum62(), 10, 1, alignment=5)
        with pytest.raises(gpu.SwError, match="SW_ERR_OVERFLOW"):
            d.align(qs.residues, qs.offsets, [0], [0], synth.blosum62(), 1 << 20, 1 << 20, alignment=1)
