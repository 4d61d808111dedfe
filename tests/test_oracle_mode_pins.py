"""Pins for the oracle's non-local alignment modes (``oracle.score`` with
mode "global", "semiglobal", "overlap"; oracle/modes.c).

- Brute force: explicit enumeration of end-to-end alignments of the right
  substrings (tests/pins.py), tiny inputs, random asymmetric matrices.
- Textbook reduction: with 0 on the diagonal, -1 off it and unit gaps the
  global score is minus the Levenshtein distance.
- No gaps: with prohibitive gap costs, global over equal lengths is the
  diagonal sum and semi-global the best window sum.
- Order and symmetry: global <= semi-global <= overlap <= local for any
  input; global and overlap are symmetric for a symmetric matrix.
- Hand-worked values (tests/golden/mode_examples.txt).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "mode_examples.txt")
MODES = ("global", "semiglobal", "overlap")


def _golden():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [x.strip() for x in line.split("|")]
        S = np.array([[int(v) for v in r.split()] for r in f[1].split(";")])
        o, e = (int(v) for v in f[2].split())
        out.append((f[0], S, o, e, [int(v) for v in f[3].split()], [int(v) for v in f[4].split()],
                    [int(v) for v in f[5].split()]))
    return out


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c[0])
def test_hand_examples(case):
    name, S, o, e, q, t, want = case
    assert [oracle.score(q, t, S, o, e, mode=m) for m in MODES] == want


@pytest.mark.parametrize("seed", range(30))
def test_brute_force(seed):
    rng = np.random.default_rng(7000 + seed)
    for _ in range(6):
        A = int(rng.integers(1, 4))
        S = rng.integers(-4, 5, size=(A, A))
        o, e = int(rng.integers(0, 5)), int(rng.integers(0, 4))
        m = int(rng.integers(0, 5))
        n = int(rng.integers(0, 6 - max(m, 1)))
        q, t = rng.integers(0, A, m), rng.integers(0, A, n)
        for md in MODES:
            assert oracle.score(q, t, S, o, e, mode=md) == pins.brute_force_mode(q, t, S, o, e, md), (md, q, t)


@pytest.mark.parametrize("seed", range(8))
def test_levenshtein(seed):
    rng = np.random.default_rng(7100 + seed)
    A = int(rng.integers(2, 6))
    S = -(1 - np.eye(A, dtype=np.int64))
    for _ in range(10):
        q = rng.integers(0, A, int(rng.integers(0, 60)))
        t = rng.integers(0, A, int(rng.integers(0, 60)))
        assert oracle.score(q, t, S, 1, 1, mode="global") == -pins.levenshtein(q, t)


def test_without_gaps():
    rng = np.random.default_rng(72)
    S = synth.blosum62()
    big = 10 ** 6
    for _ in range(10):
        L = int(rng.integers(1, 40))
        q, t = rng.integers(0, 20, L), rng.integers(0, 20, L)
        assert oracle.score(q, t, S, big, big, mode="global") == int(sum(S[a][b] for a, b in zip(q, t)))
        t2 = rng.integers(0, 20, L + int(rng.integers(0, 20)))
        best = max(int(sum(S[a][b] for a, b in zip(q, t2[d:d + L]))) for d in range(len(t2) - L + 1))
        assert oracle.score(q, t2, S, big, big, mode="semiglobal") == best


@pytest.mark.parametrize("seed", range(6))
def test_order_and_symmetry(seed):
    rng = np.random.default_rng(7200 + seed)
    A = int(rng.integers(2, 25))
    for sym in (True, False):
        S = synth.random_matrix(rng, A, -6, 9, symmetric=sym)
        for _ in range(8):
            o, e = int(rng.integers(0, 12)), int(rng.integers(0, 4))
            q = rng.integers(0, A, int(rng.integers(0, 80)))
            t = rng.integers(0, A, int(rng.integers(0, 80)))
            g, s_, ov = (oracle.score(q, t, S, o, e, mode=m) for m in MODES)
            loc = oracle.score(q, t, S, o, e)
            assert g <= s_ <= ov <= loc
            assert ov >= 0
            if sym:
                assert g == oracle.score(t, q, S, o, e, mode="global")
                assert ov == oracle.score(t, q, S, o, e, mode="overlap")


def test_empty_sequences():
    S = synth.blosum62()
    q = [0, 1, 2, 3, 4]
    assert oracle.score(q, [], S, 10, 2, mode="global") == -(10 + 4 * 2)
    assert oracle.score([], q, S, 10, 2, mode="global") == -(10 + 4 * 2)
    assert oracle.score([], [], S, 10, 2, mode="global") == 0
    assert oracle.score(q, [], S, 10, 2, mode="semiglobal") == -(10 + 4 * 2)
    assert oracle.score([], q, S, 10, 2, mode="semiglobal") == 0
    assert oracle.score(q, [], S, 10, 2, mode="overlap") == 0
