"""Pins for the oracle's traceback (``oracle.align``), none of which reads the
oracle's matrices.

- Rescoring: walking the returned ops over the returned coordinates and
  pricing each column (S for M; a gap run of k columns priced open +
  (k-1)*min(open, extend), the price the recurrences give) reproduces the
  score, which equals ``oracle.score`` (gotoh.c).
- Brute force on tiny inputs: every local alignment is enumerated as an
  explicit list of columns; the end cell is the first cell in row-major
  order where some optimal alignment ends, and the traceback's tie rules,
  restated as a greedy choice over the set of optimal alignments walked
  backwards from that cell, pick exactly the returned alignment.
- Hand-worked examples (tests/golden/align_examples.txt).
- Properties: a non-empty alignment starts and ends with M, and every prefix
  ending with an M scores > 0 (the path stops at the first H = 0).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests.pins import alignment_end, enumerate_alignments

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "align_examples.txt")
OPS = {"M": 0, "I": 1, "D": 2}


def rescore(q, t, S, o, e, aln):
    """Score of the alignment described by aln (ops from its start)."""
    i, j = aln["q_begin"], aln["t_begin"]
    cont = min(o, e)
    total, prev = 0, None
    prefix_after_m = []
    for op in aln["ops"]:
        if op == 0:
            total += int(S[q[i]][t[j]])
            i += 1
            j += 1
            prefix_after_m.append(total)
        else:
            total -= cont if prev == op else o
            if op == 1:
                i += 1
            else:
                j += 1
        prev = op
    return total, (i, j), prefix_after_m


def rule_choice(q, t, S, o, e):
    """The alignment the traceback rules select, found over the enumerated set
    of optimal alignments (no dynamic programming)."""
    alns = enumerate_alignments(q, t, S, o, e)
    best = max((a[3] for a in alns), default=0)
    if best <= 0:
        return {"score": 0, "q_begin": 0, "q_end": 0, "t_begin": 0, "t_end": 0, "ops": []}
    ends = sorted({alignment_end(a[0], a[1], a[2]) for a in alns if a[3] == best})
    end = ends[0]                                   # first in row-major order
    C = [a for a in alns if a[3] == best and alignment_end(a[0], a[1], a[2]) == end]
    pos, state = 0, "H"
    while True:
        if state == "H":
            stop = [a for a in C if len(a[2]) == pos]
            if stop:                                # the path stops at H = 0
                C = stop
                break
            for op in "MDI":                        # diagonal, then E, then F
                nxt = [a for a in C if a[2][len(a[2]) - 1 - pos][0] == op]
                if nxt:
                    C = nxt
                    break
            if op == "M":
                pos += 1
            else:
                state = op
        else:                                       # inside a gap: opening wins
            opens = [a for a in C if a[2][len(a[2]) - 1 - pos][1]]
            if opens:
                C = opens
                state = "H"
            pos += 1
    i0, j0, cols, score = C[0]
    return {"score": score, "q_begin": i0, "q_end": end[0], "t_begin": j0, "t_end": end[1],
            "ops": [OPS[c[0]] for c in cols]}


def _same(a, b):
    assert a["score"] == b["score"]
    for k in ("q_begin", "q_end", "t_begin", "t_end"):
        assert a[k] == b[k], k
    assert list(a["ops"]) == list(b["ops"])


@pytest.mark.parametrize("seed", range(40))
def test_tie_rules_match_brute_force(seed):
    rng = np.random.default_rng(5000 + seed)
    for k in range(16):
        A = int(rng.integers(1, 4))
        S = rng.integers(-3, 5, size=(A, A))
        o = 0 if k % 2 else int(rng.integers(0, 4))      # free gap opening makes ties common
        e = int(rng.integers(0, 4))
        m = int(rng.integers(0, 5))
        n = int(rng.integers(0, 7 - max(m, 1)))
        q = rng.integers(0, A, m)
        t = rng.integers(0, A, n)
        _same(oracle.align(q, t, S, o, e), rule_choice(q, t, S, o, e))


def _golden():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [x.strip() for x in line.split("|")]
        S = np.array([[int(v) for v in row.split()] for row in f[1].split(";")])
        o, e = (int(v) for v in f[2].split())
        q = [int(v) for v in f[3].split()]
        t = [int(v) for v in f[4].split()]
        c = [int(v) for v in f[6].split()]
        out.append((f[0], S, o, e, q, t, int(f[5]), c, [OPS[ch] for ch in f[7]]))
    return out


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c[0])
def test_hand_examples(case):
    name, S, o, e, q, t, score, c, ops = case
    a = oracle.align(q, t, S, o, e)
    _same(a, {"score": score, "q_begin": c[0], "q_end": c[1], "t_begin": c[2], "t_end": c[3], "ops": ops})
    _same(a, rule_choice(q, t, S, o, e))


@pytest.mark.parametrize("seed", range(12))
def test_rescoring_and_properties(seed):
    rng = np.random.default_rng(6000 + seed)
    for _ in range(15):
        if seed % 3 == 0:
            S, A = synth.blosum62(), 20
        else:
            A = int(rng.integers(2, 25))
            S = synth.random_matrix(rng, A, -6, 9, symmetric=bool(seed % 2))
        o = int(rng.integers(0, 13))
        e = int(rng.integers(0, 5))
        q = rng.integers(0, A, int(rng.integers(0, 90)))
        t = rng.integers(0, A, int(rng.integers(0, 90)))
        a = oracle.align(q, t, S, o, e)
        assert a["score"] == oracle.score(q, t, S, o, e)
        total, end, prefixes = rescore(q, t, S, o, e, a)
        assert total == a["score"]
        assert end == (a["q_end"], a["t_end"])
        ops = list(a["ops"])
        n_m, n_i, n_d = ops.count(0), ops.count(1), ops.count(2)
        assert n_m + n_i == a["q_end"] - a["q_begin"]
        assert n_m + n_d == a["t_end"] - a["t_begin"]
        assert 0 <= a["q_begin"] <= a["q_end"] <= len(q)
        assert 0 <= a["t_begin"] <= a["t_end"] <= len(t)
        if a["score"] > 0:
            assert ops[0] == 0 and ops[-1] == 0
            assert min(prefixes) > 0
        else:
            assert ops == [] and (a["q_begin"], a["q_end"], a["t_begin"], a["t_end"]) == (0, 0, 0, 0)


def test_self_alignment_is_the_diagonal():
    """BLOSUM62 satisfies S(a,b) <= (S(a,a)+S(b,b))/2, so a sequence's best
    local alignment with itself is the whole diagonal (no gaps)."""
    rng = np.random.default_rng(61)
    S = synth.blosum62()
    for L in (1, 7, 150):
        q = rng.integers(0, 20, L)
        a = oracle.align(q, q, S, 10, 1)
        assert a["score"] == int(sum(S[x][x] for x in q))
        assert (a["q_begin"], a["q_end"], a["t_begin"], a["t_end"]) == (0, L, 0, L)
        assert list(a["ops"]) == [0] * L
