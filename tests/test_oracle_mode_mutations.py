"""The mode pins catch plausible mistakes in oracle/modes.c (CPU only).

Each case plants one mistake in a temporary copy (a wrong first row or
column, a zero floor left in, the score read from the wrong place, a gap
priced o + k*e), compiles it, and checks that the pins of
test_oracle_mode_pins reject it.  The real file passes the same battery.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import synth
from tests import pins
from tests.test_oracle_mode_pins import MODES, _golden

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "modes.c")

MUTATIONS = {
    "semiglobal_row0_gapped": ("Hrow[j] = (mode == 1) ? -gap_cost(j, o, e) : 0;",
                               "Hrow[j] = (mode != 3) ? -gap_cost(j, o, e) : 0;"),
    "overlap_col0_gapped": ("const int64_t Hcol0 = (mode == 3) ? 0 : -gap_cost(i, o, e);",
                            "const int64_t Hcol0 = -gap_cost(i, o, e);"),
    "zero_floor_kept": ("            H = max2(H, F);\n            Hdiag = Hup;",
                        "            H = max2(H, F);\n            H = max2(H, 0);\n            Hdiag = Hup;"),
    "gap_cost_o_plus_ke": ("return k <= 0 ? 0 : o + (k - 1) * (e < o ? e : o);", "return k <= 0 ? 0 : o + k * (e < o ? e : o);"),
    "gap_cost_no_reopen": ("return k <= 0 ? 0 : o + (k - 1) * (e < o ? e : o);", "return k <= 0 ? 0 : o + (k - 1) * e;"),
    "global_reads_last_row_max": ("        score = Hrow[n];                             /* H(m, n) */",
                                  "        score = Hrow[0]; for (int64_t j = 1; j <= n; ++j) score = max2(score, Hrow[j]);"),
    "overlap_forgets_last_column": ("score = (mode == 2) ? last : max2(last, best_row);", "score = last;"),
    # (Leaving H(m,0) out of the semi-global maximum is NOT a mistake: down
    # every column j >= 1, F(i,j) >= H(i,0) by induction from H(0,j) = 0, so
    # H(m,0) never exceeds the rest of the last row.)
    "diag_from_col0_zero": ("int64_t Hdiag = Hrow[0];      /* H(i-1, 0) */", "int64_t Hdiag = 0;            /* H(i-1, 0) */"),
}


def _build(tmp_path, name, src_text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-pthread", str(c), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    lib.swo_score_mode.restype = ctypes.c_int64
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.swo_score_mode.argtypes = [vp, i64, vp, i64, vp, ctypes.c_int32, i64, i64, ctypes.c_int32]

    def score(q, t, S, o, e, mode):
        q = np.ascontiguousarray(q, np.uint8)
        t = np.ascontiguousarray(t, np.uint8)
        S = np.ascontiguousarray(S, np.int32)
        qq = q if len(q) else np.zeros(1, np.uint8)
        tt = t if len(t) else np.zeros(1, np.uint8)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        return int(lib.swo_score_mode(p(qq), len(q), p(tt), len(t), p(S), S.shape[0], o, e, MODES.index(mode) + 1))
    return score


def _battery(score):
    fails = []
    for name, S, o, e, q, t, want in _golden():
        if [score(q, t, S, o, e, m) for m in MODES] != want:
            fails.append(f"golden:{name}")
    rng = np.random.default_rng(73)
    for k in range(60):
        A = int(rng.integers(1, 4))
        S = rng.integers(-4, 5, size=(A, A))
        o, e = int(rng.integers(0, 5)), int(rng.integers(0, 4))
        m = int(rng.integers(0, 5))
        n = int(rng.integers(0, 6 - max(m, 1)))
        q, t = rng.integers(0, A, m), rng.integers(0, A, n)
        for md in MODES:
            if score(q, t, S, o, e, md) != pins.brute_force_mode(q, t, S, o, e, md):
                fails.append(f"brute:{md}[{k}]")
    Sl = -(1 - np.eye(4, dtype=np.int64))
    for k in range(10):
        q, t = rng.integers(0, 4, 30), rng.integers(0, 4, 25)
        if score(q, t, Sl, 1, 1, "global") != -pins.levenshtein(q, t):
            fails.append(f"levenshtein[{k}]")
    return fails


def test_real_modes_pass_battery(tmp_path):
    assert _battery(_build(tmp_path, "real", open(SRC).read())) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mode_mutant_is_caught(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    assert _battery(_build(tmp_path, name, src.replace(old, new))), f"mutation {name} was not caught by any pin"
