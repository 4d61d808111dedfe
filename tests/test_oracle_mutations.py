"""The pins catch plausible mistakes in the oracle (CPU only).

Each case below plants one mistake in a temporary copy of oracle/gotoh.c
(a dropped term, a wrong penalty, a transposed matrix operand, an index
slip, a wrong initial value), compiles it, and checks that the pins of
test_oracle_pins (brute-force enumeration, textbook reductions, the
hand-worked values, invariants) reject the mutant.  The real oracle passes
the same battery.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import synth
from tests import pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "gotoh.c")

MUTATIONS = {
    "extend_uses_open": ("E = max2(E - e, Hleft - o);", "E = max2(E - o, Hleft - o);"),
    "vertical_open_uses_extend": ("F = max2(Frow[j] - e, Hup - o);", "F = max2(Frow[j] - e, Hup - e);"),
    "matrix_transposed": ("int64_t H = Hdiag + (int64_t)Srow[t[j - 1]];",
                          "int64_t H = Hdiag + (int64_t)S[(size_t)t[j - 1] * (size_t)A + q[i - 1]];"),
    "no_zero_floor": ("H = max2(H, 0);", ""),
    "dropped_vertical_gap": ("H = max2(H, F);", ""),
    "dropped_horizontal_gap": ("H = max2(H, E);", ""),
    "diag_from_left": ("Hdiag = Hup;", "Hdiag = Hleft;"),
    "target_index_slip": ("Srow[t[j - 1]]", "Srow[t[j < n ? j : j - 1]]"),
    # (E or F starting at 0 instead of -inf is NOT a mistake: boundary gap
    # values stay below 0 <= H and never win a max, so that variant is exact.)
    "boundary_h_one": ("Hrow[j] = 0; Frow[j] = NEG_INF;", "Hrow[j] = 1; Frow[j] = NEG_INF;"),
    "best_not_tracked_last_row": ("if (H > best) best = H;", "if (H > best && i < m) best = H;"),
}


def _build(tmp_path, name, src_text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", str(c), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    lib.swo_score.restype = ctypes.c_int64
    lib.swo_score.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                              ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64]

    def score(q, t, S, o, e):
        q = np.ascontiguousarray(q, np.uint8)
        t = np.ascontiguousarray(t, np.uint8)
        S = np.ascontiguousarray(S, np.int32)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        return int(lib.swo_score(vp(q), len(q), vp(t), len(t), vp(S), S.shape[0], o, e))
    return score


def _battery(score):
    """Return the list of failed pin checks for a scoring function."""
    fails = []
    rng = np.random.default_rng(4242)
    for k in range(40):
        A = int(rng.integers(2, 5))
        S = synth.random_matrix(rng, A, -5, 5)
        q = rng.integers(0, A, int(rng.integers(1, 6))).astype(np.uint8)
        t = rng.integers(0, A, int(rng.integers(1, 6))).astype(np.uint8)
        e = int(rng.integers(0, 3))
        o = e + int(rng.integers(1, 4))
        if score(q, t, S, o, e) != pins.brute_force_local(q, t, S, o, e):
            fails.append(f"brute_force[{k}]")
    from tests.test_oracle_pins import _hand_examples
    ac2 = np.array([[5, -4], [-4, 5]], dtype=np.int32)
    for mat, qs, ts, o, e, want in _hand_examples():
        if mat == "AC2":
            enc = lambda s: np.array(["AC".index(c) for c in s], dtype=np.uint8)
            M = ac2
        else:
            enc, M = synth.encode, synth.blosum62()
        if score(enc(qs), enc(ts), M, o, e) != want:
            fails.append(f"hand[{qs}/{ts}/{o}/{e}]")
    S = synth.blosum62()
    for k in range(4):
        q = synth.random_residues(rng, 60)
        if score(q, q, S, 10, 1) != int(S[q, q].sum()):
            fails.append(f"self_score[{k}]")
    for k in range(4):
        A = 3
        Sid = np.eye(A, dtype=np.int32)
        q = rng.integers(0, A, 20).astype(np.uint8)
        t = rng.integers(0, A, 25).astype(np.uint8)
        if score(q, t, Sid, 0, 0) != pins.lcs_length(q, t):
            fails.append(f"lcs[{k}]")
    return fails


def test_real_oracle_passes_battery(tmp_path):
    score = _build(tmp_path, "real", open(SRC).read())
    assert _battery(score) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    score = _build(tmp_path, name, src.replace(old, new))
    assert _battery(score), f"mutation {name} was not caught by any pin"
