"""Independent checks the oracle is pinned to (no dynamic programming on H/E/F).

Each function computes, by a different route, a quantity that the
Smith-Waterman/Gotoh score (Section 2.2; affine gaps as in Section 4.1)
must equal in a special case:

- ``brute_force_local``: explicit enumeration of every local alignment of
  every pair of substrings, each gap run priced open + (k-1)*extend.
- ``lcs_length``: the textbook longest-common-subsequence DP (the score when
  S is the identity and gaps are free).
- ``longest_common_substring``: by direct comparison of all substring pairs
  (the score when mismatches and gaps are prohibitively expensive).
- ``best_diagonal_kadane``: Kadane's maximum subarray along every diagonal
  (the score when gaps are prohibitively expensive).
- ``enumerate_alignments``: every local alignment as an explicit list of
  columns, each gap column marked as opening its gap or extending it (the
  raw material of the traceback pins).
- ``brute_force_global`` and the mode scores built on it: global,
  semi-global and overlap scores as maxima over explicitly enumerated
  end-to-end alignments of the right substrings.
- ``levenshtein``: the classic edit distance (global score with unit costs).
"""
from __future__ import annotations

import sys

import numpy as np


def brute_force_local(q, t, S, gap_open: int, gap_extend: int, reopen: bool = False) -> int:
    """Maximum over all local alignments, enumerated one by one.

    An alignment is a path of columns: M (q_i over t_j, scores S[q_i][t_j]),
    X (q_i over a gap) and Y (a gap over t_j).  A maximal run of X (or Y)
    columns of length k costs open + (k-1)*extend.  With ``reopen`` a run may
    also be priced as several adjacent gaps (each continuing column costs
    min(open, extend)), which is what the recurrences give when open < extend.
    The empty alignment scores 0.
    """
    q = [int(x) for x in q]
    t = [int(x) for x in t]
    m, n = len(q), len(t)
    best = 0
    cont = min(gap_open, gap_extend) if reopen else gap_extend
    sys.setrecursionlimit(max(1000, 10 * (m + n) + 100))

    def dfs(i, j, last, score):
        nonlocal best
        if last is not None and score > best:
            best = score
        if i < m and j < n:
            dfs(i + 1, j + 1, "M", score + int(S[q[i]][t[j]]))
        if i < m:
            dfs(i + 1, j, "X", score - (cont if last == "X" else gap_open))
        if j < n:
            dfs(i, j + 1, "Y", score - (cont if last == "Y" else gap_open))

    for i0 in range(m + 1):
        for j0 in range(n + 1):
            dfs(i0, j0, None, 0)
    return best


def lcs_length(a, b) -> int:
    """Classic LCS DP: L[i][j] = L[i-1][j-1] + 1 on a match, else the max of L[i-1][j], L[i][j-1]."""
    a = list(a)
    b = list(b)
    L = [[0] * (len(b) + 1) for _ in range(len(a) + 1)]
    for i in range(1, len(a) + 1):
        for j in range(1, len(b) + 1):
            if a[i - 1] == b[j - 1]:
                L[i][j] = L[i - 1][j - 1] + 1
            else:
                L[i][j] = max(L[i - 1][j], L[i][j - 1])
    return L[len(a)][len(b)]


def longest_common_substring(a, b) -> int:
    a = bytes(bytearray(int(x) for x in a))
    b = bytes(bytearray(int(x) for x in b))
    best = 0
    for i in range(len(a)):
        for k in range(best + 1, len(a) - i + 1):
            if a[i:i + k] in b:
                best = k
            else:
                break
    return best


def best_diagonal_kadane(q, t, S) -> int:
    """max(0, max over diagonals of the maximum-sum contiguous run of S(q_i, t_{i+d}))."""
    q = np.asarray(q, dtype=np.int64)
    t = np.asarray(t, dtype=np.int64)
    m, n = len(q), len(t)
    best = 0
    for d in range(-(m - 1), n):
        run = 0
        for i in range(m):
            j = i + d
            if 0 <= j < n:
                run = max(0, run + int(S[q[i]][t[j]]))
                best = max(best, run)
    return best


def enumerate_alignments(q, t, S, gap_open: int, gap_extend: int):
    """Every non-empty local alignment of every pair of substrings.

    Yields (i0, j0, cols, score): the alignment starts after q[:i0] and
    t[:j0]; cols is a tuple of (op, opens) with op "M", "I" (q residue
    opposite a gap) or "D" (t residue opposite a gap), and opens True when a
    gap column starts a new gap (priced open) rather than extending the gap
    of the previous column (priced extend; only possible right after a gap
    column of the same kind).  Both pricings of a continuing column are
    enumerated, so the maximum over alignments is the recurrences' score
    whether open >= extend or not.
    """
    q = [int(x) for x in q]
    t = [int(x) for x in t]
    m, n = len(q), len(t)
    out = []

    def dfs(i0, j0, i, j, cols, score):
        if cols:
            out.append((i0, j0, tuple(cols), score))
        last = cols[-1][0] if cols else None
        if i < m and j < n:
            cols.append(("M", False))
            dfs(i0, j0, i + 1, j + 1, cols, score + int(S[q[i]][t[j]]))
            cols.pop()
        for op, di, dj in (("I", 1, 0), ("D", 0, 1)):
            if i + di > m or j + dj > n:
                continue
            cols.append((op, True))
            dfs(i0, j0, i + di, j + dj, cols, score - gap_open)
            cols.pop()
            if last == op:
                cols.append((op, False))
                dfs(i0, j0, i + di, j + dj, cols, score - gap_extend)
                cols.pop()

    for i0 in range(m + 1):
        for j0 in range(n + 1):
            dfs(i0, j0, i0, j0, [], 0)
    return out


def alignment_end(i0, j0, cols):
    """(i, j) after the last column of an alignment starting at (i0, j0)."""
    i, j = i0, j0
    for op, _ in cols:
        if op in "MI":
            i += 1
        if op in "MD":
            j += 1
    return i, j


def enumerate_mode_alignments(q, t, S, gap_open: int, gap_extend: int, mode: str):
    """Every alignment a non-local mode allows, as explicit column lists.

    Yields (i0, j0, cols, score) as enumerate_alignments does (gap columns
    priced open, or extend right after a gap column of the same kind, both
    pricings listed), restricted to the mode's start and end:
    global starts at (0, 0) and ends at (m, n); semi-global starts at (0, j0)
    and ends at (m, j1); overlap starts with i0 = 0 or j0 = 0 and ends with
    i1 = m or j1 = n.  Empty alignments are included where start = end is
    allowed.
    """
    q = [int(x) for x in q]
    t = [int(x) for x in t]
    m, n = len(q), len(t)
    out = []

    def ends_ok(i, j):
        if mode == "global":
            return i == m and j == n
        if mode == "semiglobal":
            return i == m
        return i == m or j == n

    def dfs(i0, j0, i, j, cols, score):
        if ends_ok(i, j):
            out.append((i0, j0, tuple(cols), score))
        last = cols[-1][0] if cols else None
        if i < m and j < n:
            cols.append(("M", False))
            dfs(i0, j0, i + 1, j + 1, cols, score + int(S[q[i]][t[j]]))
            cols.pop()
        for op, di, dj in (("I", 1, 0), ("D", 0, 1)):
            if i + di > m or j + dj > n:
                continue
            cols.append((op, True))
            dfs(i0, j0, i + di, j + dj, cols, score - gap_open)
            cols.pop()
            if last == op:
                cols.append((op, False))
                dfs(i0, j0, i + di, j + dj, cols, score - gap_extend)
                cols.pop()

    if mode == "global":
        starts = [(0, 0)]
    elif mode == "semiglobal":
        starts = [(0, j0) for j0 in range(n + 1)]
    elif mode == "overlap":
        starts = [(i0, 0) for i0 in range(m + 1)] + [(0, j0) for j0 in range(1, n + 1)]
    else:
        raise ValueError(mode)
    for i0, j0 in starts:
        dfs(i0, j0, i0, j0, [], 0)
    return out


def brute_force_global(q, t, S, gap_open: int, gap_extend: int) -> int:
    """Maximum over every end-to-end alignment of q against t, enumerated one
    by one (columns M, I, D; a run of k gap columns of one kind costs open +
    (k-1)*extend, and may be split into adjacent gaps priced open each, which
    is what the recurrences give when open < extend)."""
    q = [int(x) for x in q]
    t = [int(x) for x in t]
    m, n = len(q), len(t)
    cont = min(gap_open, gap_extend)
    best = None
    sys.setrecursionlimit(max(1000, 10 * (m + n) + 100))

    def dfs(i, j, last, score):
        nonlocal best
        if i == m and j == n:
            best = score if best is None else max(best, score)
            return
        if i < m and j < n:
            dfs(i + 1, j + 1, "M", score + int(S[q[i]][t[j]]))
        if i < m:
            dfs(i + 1, j, "I", score - (cont if last == "I" else gap_open))
        if j < n:
            dfs(i, j + 1, "D", score - (cont if last == "D" else gap_open))

    dfs(0, 0, None, 0)
    return best


def brute_force_mode(q, t, S, gap_open: int, gap_extend: int, mode: str) -> int:
    """Global: q against t end to end.  Semi-global: q end to end against any
    substring t[j0:j1].  Overlap: q[i0:i1] against t[j0:j1] where the
    alignment starts on the first row or column (i0 = 0 or j0 = 0) and ends
    on the last row or column (i1 = m or j1 = n)."""
    m, n = len(q), len(t)
    if mode == "global":
        return brute_force_global(q, t, S, gap_open, gap_extend)
    if mode == "semiglobal":
        return max(brute_force_global(q, t[j0:j1], S, gap_open, gap_extend)
                   for j0 in range(n + 1) for j1 in range(j0, n + 1))
    if mode == "overlap":
        best = None
        for i0 in range(m + 1):
            for j0 in range(n + 1):
                if i0 and j0:
                    continue
                for i1 in range(i0, m + 1):
                    for j1 in range(j0, n + 1):
                        if i1 != m and j1 != n:
                            continue
                        v = brute_force_global(q[i0:i1], t[j0:j1], S, gap_open, gap_extend)
                        best = v if best is None else max(best, v)
        return best
    raise ValueError(mode)


def levenshtein(a, b) -> int:
    """Classic edit distance: D[i][j] = min(D[i-1][j] + 1, D[i][j-1] + 1,
    D[i-1][j-1] + (a_i != b_j))."""
    a = list(a)
    b = list(b)
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[-1]
