"""Pins for the oracle's traceback in the non-local modes
(``oracle.align(..., mode=...)``, oracle/align_modes.c), none of which reads
the oracle's matrices.

- Brute force on tiny inputs: every alignment the mode allows is enumerated
  as an explicit list of columns; the end cell is the first candidate cell of
  the mode (last row, and last column for overlap; (m, n) for global) in
  row-major order where an optimal alignment ends, and the tie rules, restated
  as a greedy choice over the optimal alignments walked backwards from it,
  pick exactly the returned alignment.
- Rescoring: walking the returned ops over the returned coordinates and
  pricing each column (S for M; a gap run of k columns priced open +
  (k-1)*min(open, extend)) reproduces the score, which equals the mode's
  score of ``oracle.score`` (modes.c, itself pinned by brute force).
- The coordinates the mode fixes: global covers both sequences, semi-global
  the whole query, overlap starts on the first row or column and ends on the
  last row or column.
- Hand-worked examples (tests/golden/align_mode_examples.txt).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests.pins import alignment_end, enumerate_mode_alignments

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "align_mode_examples.txt")
OPS = {"M": 0, "I": 1, "D": 2}
MODES = ["global", "semiglobal", "overlap"]


def rescore_mode(q, t, S, o, e, aln):
    """Score of the alignment described by aln (ops from its start)."""
    i, j = aln["q_begin"], aln["t_begin"]
    cont = min(o, e)
    total, prev = 0, None
    for op in aln["ops"]:
        if op == 0:
            total += int(S[q[i]][t[j]])
            i += 1
            j += 1
        else:
            total -= cont if prev == op else o
            if op == 1:
                i += 1
            else:
                j += 1
        prev = op
    return total, (i, j)


def _candidates(m, n, mode):
    """The mode's end cells in row-major order."""
    if mode == "global":
        return [(m, n)]
    if mode == "semiglobal":
        return [(m, j) for j in range(n + 1)]
    return [(i, n) for i in range(m)] + [(m, j) for j in range(n + 1)]


def rule_choice_mode(q, t, S, o, e, mode):
    """The alignment the traceback rules select, found over the enumerated set
    of optimal alignments of the mode (no dynamic programming)."""
    alns = enumerate_mode_alignments(q, t, S, o, e, mode)
    best = max(a[3] for a in alns)
    ends = {alignment_end(a[0], a[1], a[2]) for a in alns if a[3] == best}
    end = next(c for c in _candidates(len(q), len(t), mode) if c in ends)
    C = [a for a in alns if a[3] == best and alignment_end(a[0], a[1], a[2]) == end]
    pos, state = 0, "H"
    while True:
        if state == "H":
            stop = [a for a in C if len(a[2]) == pos]
            if stop:                                # the path starts here
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
    assert [int(x) for x in a["ops"]] == [int(x) for x in b["ops"]]


def _golden():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [x.strip() for x in line.split("|")]
        S = np.array([[int(v) for v in row.split()] for row in f[2].split(";")])
        o, e = (int(v) for v in f[3].split())
        q = [int(v) for v in f[4].split()]
        t = [int(v) for v in f[5].split()]
        c = [int(v) for v in f[7].split()]
        ops = [OPS[ch] for ch in f[8]] if len(f) > 8 else []
        out.append((f[0], f[1], S, o, e, q, t, int(f[6]), c, ops))
    return out


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c[0])
def test_hand_examples(case):
    name, mode, S, o, e, q, t, score, c, ops = case
    a = oracle.align(q, t, S, o, e, mode=mode)
    _same(a, {"score": score, "q_begin": c[0], "q_end": c[1], "t_begin": c[2], "t_end": c[3], "ops": ops})
    _same(a, rule_choice_mode(q, t, S, o, e, mode))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", range(12))
def test_tie_rules_match_brute_force(mode, seed):
    rng = np.random.default_rng(7000 + 10 * seed + MODES.index(mode))
    for k in range(12):
        A = int(rng.integers(1, 4))
        S = rng.integers(-3, 5, size=(A, A))
        o = 0 if k % 2 else int(rng.integers(0, 4))      # free gap opening makes ties common
        e = int(rng.integers(0, 4))
        m = int(rng.integers(0, 5))
        n = int(rng.integers(0, 7 - max(m, 1)))
        q = rng.integers(0, A, m)
        t = rng.integers(0, A, n)
        _same(oracle.align(q, t, S, o, e, mode=mode), rule_choice_mode(q, t, S, o, e, mode))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", range(6))
def test_rescoring_and_mode_coordinates(mode, seed):
    rng = np.random.default_rng(8000 + 10 * seed + MODES.index(mode))
    for _ in range(12):
        if seed % 3 == 0:
            S, A = synth.blosum62(), 20
        else:
            A = int(rng.integers(2, 25))
            S = synth.random_matrix(rng, A, -6, 9, symmetric=bool(seed % 2))
        o = int(rng.integers(0, 13))
        e = int(rng.integers(0, 5))
        q = rng.integers(0, A, int(rng.integers(0, 80)))
        t = rng.integers(0, A, int(rng.integers(0, 80)))
        m, n = len(q), len(t)
        a = oracle.align(q, t, S, o, e, mode=mode)
        assert a["score"] == oracle.score(q, t, S, o, e, mode=mode)
        total, end = rescore_mode(q, t, S, o, e, a)
        assert total == a["score"]
        assert end == (a["q_end"], a["t_end"])
        ops = [int(x) for x in a["ops"]]
        assert ops.count(0) + ops.count(1) == a["q_end"] - a["q_begin"]
        assert ops.count(0) + ops.count(2) == a["t_end"] - a["t_begin"]
        if mode == "global":
            assert (a["q_begin"], a["q_end"], a["t_begin"], a["t_end"]) == (0, m, 0, n)
        elif mode == "semiglobal":
            assert (a["q_begin"], a["q_end"]) == (0, m)
        else:
            assert a["q_begin"] == 0 or a["t_begin"] == 0
            assert a["q_end"] == m or a["t_end"] == n


def test_global_of_a_sequence_with_itself_is_the_diagonal():
    """BLOSUM62 satisfies S(a,b) <= (S(a,a)+S(b,b))/2 and every gap costs, so the
    global alignment of a sequence with itself is the whole diagonal."""
    rng = np.random.default_rng(71)
    S = synth.blosum62()
    for L in (1, 9, 120):
        q = rng.integers(0, 20, L)
        a = oracle.align(q, q, S, 10, 1, mode="global")
        assert a["score"] == int(sum(S[x][x] for x in q))
        assert [int(x) for x in a["ops"]] == [0] * L


def test_empty_sequences():
    """One side empty: global is the other side's leading gap, semi-global the
    query's (an empty query aligns to nothing), overlap the empty alignment."""
    S = synth.blosum62()
    q = np.array([3, 1, 4], np.uint8)
    g3 = 10 + 2 * 1
    a = oracle.align(q, [], S, 10, 1, mode="global")
    assert (a["score"], [int(x) for x in a["ops"]]) == (-g3, [1, 1, 1])
    a = oracle.align([], q, S, 10, 1, mode="global")
    assert (a["score"], [int(x) for x in a["ops"]]) == (-g3, [2, 2, 2])
    a = oracle.align(q, [], S, 10, 1, mode="semiglobal")
    assert (a["score"], [int(x) for x in a["ops"]]) == (-g3, [1, 1, 1])
    a = oracle.align([], q, S, 10, 1, mode="semiglobal")
    assert (a["score"], len(a["ops"])) == (0, 0)
    for qq, tt in ((q, []), ([], q)):
        a = oracle.align(qq, tt, S, 10, 1, mode="overlap")
        assert (a["score"], len(a["ops"]), a["q_begin"], a["t_begin"]) == (0, 0, 0, 0)
