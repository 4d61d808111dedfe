"""Pins of the CPU oracle to results fixed by the mathematics (no GPU).

The oracle writes out the Smith-Waterman/Gotoh recurrences (Section 2.2,
with the affine gap penalties of Section 4.1).  These tests check it against
explicit enumeration, textbook special cases, hand-worked values and
invariants, so that a dropped term, a wrong sign or index, or a transposed
operand in it fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BIG = 10 ** 6


def _rng(seed):
    return np.random.default_rng(1000 + seed)


# --- brute-force enumeration of all local alignments -----------------------

@pytest.mark.parametrize("seed", range(60))
def test_brute_force_open_ge_extend(seed):
    rng = _rng(seed)
    A = int(rng.integers(2, 5))
    S = synth.random_matrix(rng, A, -5, 5, symmetric=bool(seed % 3 == 0))
    m = int(rng.integers(0, 6))
    n = int(rng.integers(0, 6))
    q = rng.integers(0, A, m).astype(np.uint8)
    t = rng.integers(0, A, n).astype(np.uint8)
    e = int(rng.integers(0, 4))
    o = e + int(rng.integers(0, 5))
    want = pins.brute_force_local(q, t, S, o, e)
    assert oracle.score(q, t, S, o, e) == want


@pytest.mark.parametrize("seed", range(20))
def test_brute_force_open_lt_extend(seed):
    rng = _rng(500 + seed)
    A = int(rng.integers(2, 4))
    S = synth.random_matrix(rng, A, -3, 6)
    q = rng.integers(0, A, int(rng.integers(1, 6))).astype(np.uint8)
    t = rng.integers(0, A, int(rng.integers(1, 6))).astype(np.uint8)
    o = int(rng.integers(0, 3))
    e = o + int(rng.integers(1, 4))
    want = pins.brute_force_local(q, t, S, o, e, reopen=True)
    assert oracle.score(q, t, S, o, e) == want


def test_brute_force_six_by_six_asymmetric():
    rng = _rng(77)
    S = synth.random_matrix(rng, 3, -4, 6)
    assert not np.array_equal(S, S.T)
    for _ in range(3):
        q = rng.integers(0, 3, 6).astype(np.uint8)
        t = rng.integers(0, 3, 6).astype(np.uint8)
        assert oracle.score(q, t, S, 3, 1) == pins.brute_force_local(q, t, S, 3, 1)


# --- textbook reductions ----------------------------------------------------

@pytest.mark.parametrize("seed", range(15))
def test_identity_free_gaps_is_lcs(seed):
    rng = _rng(100 + seed)
    A = int(rng.integers(2, 6))
    S = np.eye(A, dtype=np.int32)
    q = rng.integers(0, A, int(rng.integers(0, 40))).astype(np.uint8)
    t = rng.integers(0, A, int(rng.integers(0, 40))).astype(np.uint8)
    assert oracle.score(q, t, S, 0, 0) == pins.lcs_length(q, t)


@pytest.mark.parametrize("seed", range(15))
def test_no_mismatch_no_gap_is_longest_common_substring(seed):
    rng = _rng(200 + seed)
    A = int(rng.integers(2, 4))
    S = np.where(np.eye(A, dtype=bool), 1, -BIG).astype(np.int32)
    q = rng.integers(0, A, int(rng.integers(0, 30))).astype(np.uint8)
    t = rng.integers(0, A, int(rng.integers(0, 30))).astype(np.uint8)
    assert oracle.score(q, t, S, BIG, BIG) == pins.longest_common_substring(q, t)


@pytest.mark.parametrize("seed", range(15))
def test_no_gap_is_kadane_on_diagonals(seed):
    rng = _rng(300 + seed)
    A = int(rng.integers(2, 8))
    S = synth.random_matrix(rng, A, -6, 5)
    q = rng.integers(0, A, int(rng.integers(0, 25))).astype(np.uint8)
    t = rng.integers(0, A, int(rng.integers(0, 25))).astype(np.uint8)
    assert oracle.score(q, t, S, BIG, BIG) == pins.best_diagonal_kadane(q, t, S)


# --- hand-worked examples ---------------------------------------------------

def _hand_examples():
    rows = []
    with open(os.path.join(GOLDEN, "hand_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            mat, q, t, o, e, want = line.split()
            rows.append((mat, q, t, int(o), int(e), int(want)))
    return rows


@pytest.mark.parametrize("mat,q,t,o,e,want", _hand_examples())
def test_hand_examples(mat, q, t, o, e, want):
    if mat == "AC2":
        S = np.array([[5, -4], [-4, 5]], dtype=np.int32)
        enc = lambda s: np.array(["AC".index(c) for c in s], dtype=np.uint8)
    else:
        S = synth.blosum62()
        enc = synth.encode
    assert oracle.score(enc(q), enc(t), S, o, e) == want


# --- invariants -------------------------------------------------------------

def _protein(rng, lo, hi):
    return synth.random_residues(rng, int(rng.integers(lo, hi + 1)))


@pytest.mark.parametrize("seed", range(10))
def test_bounds(seed):
    rng = _rng(400 + seed)
    S = synth.blosum62()
    q, t = _protein(rng, 1, 200), _protein(rng, 1, 200)
    s = oracle.score(q, t, S, 10, 1)
    assert s >= 0
    assert s >= int(S[np.ix_(q, t)].max())
    assert s <= min(len(q), len(t)) * int(S.max())


@pytest.mark.parametrize("seed", range(10))
def test_swap_symmetry(seed):
    rng = _rng(450 + seed)
    q, t = _protein(rng, 1, 150), _protein(rng, 1, 150)
    S = synth.blosum62()
    assert oracle.score(q, t, S, 10, 1) == oracle.score(t, q, S, 10, 1)
    # with an asymmetric matrix, swapping the sequences transposes the matrix
    Sa = synth.random_matrix(rng, 20, -4, 6)
    assert not np.array_equal(Sa, Sa.T)
    assert oracle.score(q, t, Sa, 5, 2) == oracle.score(t, q, np.ascontiguousarray(Sa.T), 5, 2)


@pytest.mark.parametrize("seed", range(6))
def test_monotone_under_append(seed):
    rng = _rng(470 + seed)
    S = synth.blosum62()
    q, t = _protein(rng, 1, 80), _protein(rng, 1, 80)
    s = oracle.score(q, t, S, 10, 1)
    q2 = np.concatenate([q, _protein(rng, 1, 20)])
    t2 = np.concatenate([_protein(rng, 1, 20), t])
    assert oracle.score(q2, t, S, 10, 1) >= s
    assert oracle.score(q, t2, S, 10, 1) >= s


@pytest.mark.parametrize("seed", range(6))
def test_non_increasing_in_penalties(seed):
    rng = _rng(490 + seed)
    S = synth.blosum62()
    q, t = _protein(rng, 20, 120), _protein(rng, 20, 120)
    prev = None
    for o in range(0, 16, 3):
        s = oracle.score(q, t, S, o, 1)
        assert prev is None or s <= prev
        prev = s
    prev = None
    for e in range(0, 8):
        s = oracle.score(q, t, S, 10, e)
        assert prev is None or s <= prev
        prev = s


def test_blosum62_table():
    S = synth.blosum62()
    assert S.shape == (24, 24)
    assert np.array_equal(S, S.T)
    W, C = synth.ALPHABET.index("W"), synth.ALPHABET.index("C")
    assert S.max() == 11 and S[W, W] == 11
    assert S.min() == -4
    assert S[C, C] == 9
    std = S[:20, :20]
    d = np.diag(std)
    assert (d > 0).all()
    # S(a,b) <= (S(a,a) + S(b,b)) / 2 on the standard residues: the condition
    # under which a sequence's best local alignment with itself is the diagonal
    assert (2 * std <= d[:, None] + d[None, :]).all()


@pytest.mark.parametrize("seed", range(6))
def test_self_score_is_diagonal_sum(seed):
    rng = _rng(520 + seed)
    S = synth.blosum62()
    q = _protein(rng, 1, 400)
    assert oracle.score(q, q, S, 10, 1) == int(S[q, q].sum())


def test_empty_sequences():
    S = synth.blosum62()
    e = np.zeros(0, dtype=np.uint8)
    x = synth.encode("ACDEFG")
    assert oracle.score(e, x, S, 10, 1) == 0
    assert oracle.score(x, e, S, 10, 1) == 0
    assert oracle.score(e, e, S, 10, 1) == 0


def test_score_pairs_matches_score():
    rng = _rng(600)
    S = synth.blosum62()
    qs = synth.seqset_from_lengths(rng, [0, 5, 60])
    db = synth.seqset_from_lengths(rng, [0, 1, 17, 90, 33])
    got = oracle.all_scores(qs, db, S, 10, 1, threads=3)
    for i in range(qs.n):
        for j in range(db.n):
            assert got[i, j] == oracle.score(qs.seq(i), db.seq(j), S, 10, 1)


# --- top-k ordering ---------------------------------------------------------

@pytest.mark.parametrize("seed", range(10))
def test_top_k_order(seed):
    rng = _rng(700 + seed)
    n = int(rng.integers(0, 60))
    row = rng.integers(0, 8, n)  # many ties
    k = int(rng.integers(1, 80))
    s, i = oracle.top_k(row, k)
    want = sorted(range(n), key=lambda j: (-int(row[j]), j))[:k]
    assert list(i[:len(want)]) == want
    assert list(s[:len(want)]) == [int(row[j]) for j in want]
    assert (i[len(want):] == -1).all() and (s[len(want):] == -1).all()
