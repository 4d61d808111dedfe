"""The facts the packed alignment-mode kernel (k_modes16.cu) rests on, checked
on the recurrences themselves with a plain dynamic program written here (CPU
only; no GPU, no oracle code).

1. Bounds.  In every mode, every cell satisfies
       H(i, j) >= H(i, 0) - g(j)             (the E chain along row i alone)
       H(i, j) <= max(S, 0) * min(i, j)       (each diagonal step adds at most
                                                max(S); boundary values <= 0)
   with g(k) = o + (k-1) min(o, e).  The host sends a pair to int16 only when
   these bounds, widened by the largest addend, fit; the kernel checks nothing.
2. Virtual rows.  Padding the query at the top with P rows whose profile is
   S = 0 (semi-global, overlap) or S = -min(o, e) (global), with H(v, 0) = 0
   (semi-global, overlap) or -(o - min(o, e)) and 0 on the last virtual row
   (global), and E(i, 0) = H(i, 0) - o, gives the real rows exactly the H, E
   and F of the unpadded matrix.
"""
import numpy as np
import pytest

NEG = -(1 << 40)
MODES = ["global", "semiglobal", "overlap"]


def lead(k, o, e):
    return 0 if k <= 0 else o + (k - 1) * min(o, e)


def dp(prof_rows, t, col0, row0, o, e, e_col0):
    """H, E, F of the recurrences without a floor.  prof_rows[i-1][c] is the
    score of row i against code c; col0[i] = H(i, 0); row0[j] = H(0, j);
    e_col0[i] = E(i, 0)."""
    m, n = len(prof_rows), len(t)
    H = np.zeros((m + 1, n + 1), np.int64)
    E = np.full((m + 1, n + 1), NEG, np.int64)
    F = np.full((m + 1, n + 1), NEG, np.int64)
    H[0, :] = row0
    H[:, 0] = col0
    E[:, 0] = e_col0
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            E[i, j] = max(E[i, j - 1] - e, H[i, j - 1] - o)
            F[i, j] = max(F[i - 1, j] - e, H[i - 1, j] - o)
            H[i, j] = max(H[i - 1, j - 1] + prof_rows[i - 1][t[j - 1]], E[i, j], F[i, j])
    return H, E, F


def mode_matrix(q, t, S, o, e, mode):
    m, n = len(q), len(t)
    col0 = [0 if mode == "overlap" else -lead(i, o, e) for i in range(m + 1)]
    row0 = [-lead(j, o, e) if mode == "global" else 0 for j in range(n + 1)]
    return dp([S[x] for x in q], t, col0, row0, o, e, [NEG] * (m + 1))


def _cases(seed, count):
    rng = np.random.default_rng(seed)
    for k in range(count):
        A = int(rng.integers(1, 6))
        lo = int(rng.integers(-6, 1))
        S = rng.integers(lo, lo + int(rng.integers(1, 12)), size=(A, A))    # max(S) may be negative
        o = int(rng.integers(0, 8))
        e = int(rng.integers(0, 8))                                         # o < e, o = e and o > e
        q = rng.integers(0, A, int(rng.integers(0, 14)))
        t = rng.integers(0, A, int(rng.integers(0, 14)))
        yield S, o, e, q, t


@pytest.mark.parametrize("mode", MODES)
def test_bounds_hold_on_every_cell(mode):
    for S, o, e, q, t in _cases(11 + MODES.index(mode), 150):
        H, E, F = mode_matrix(q, t, S, o, e, mode)
        smax = max(int(S.max()), 0)
        m, n = len(q), len(t)
        for i in range(m + 1):
            for j in range(n + 1):
                assert H[i, j] >= H[i, 0] - lead(j, o, e)
                assert H[i, j] <= smax * min(i, j)
                if i and j:                                 # the intermediates the kernel forms
                    assert E[i, j] >= H[i, j - 1] - o and F[i, j] >= H[i - 1, j] - o


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("P", [0, 1, 2, 5])
def test_virtual_rows_reproduce_the_first_row(mode, P):
    for S, o, e, q, t in _cases(100 + 10 * P + MODES.index(mode), 60):
        m, n = len(q), len(t)
        gmin = min(o, e)
        H, E, F = mode_matrix(q, t, S, o, e, mode)
        # padded: rows 1..P virtual, rows P+1..P+m the query
        sv = -gmin if mode == "global" else 0
        prof = [np.full(S.shape[0], sv, np.int64)] * P + [S[x] for x in q]
        col0 = [0] * (P + m + 1)
        for i in range(1, P + m + 1):
            ir = i - P
            if ir >= 1:
                col0[i] = 0 if mode == "overlap" else -lead(ir, o, e)
            elif ir < 0:
                col0[i] = -(o - gmin) if mode == "global" else 0
        if mode == "global" and P > 0:
            col0[0] = -(o - gmin)                          # row 0 above the first virtual row
        row0 = [-((o - gmin) + j * gmin) if mode == "global" else 0 for j in range(n + 1)]
        row0[0] = col0[0]
        e_col0 = [c - o for c in col0]                      # E(i, 0) = H(i, 0) - o
        Hp, Ep, Fp = dp(prof, t, col0, row0, o, e, e_col0)
        np.testing.assert_array_equal(Hp[P:, :], H)
        np.testing.assert_array_equal(Ep[P + 1:, 1:], E[1:, 1:])
        np.testing.assert_array_equal(Fp[P + 1:, 1:], F[1:, 1:])
