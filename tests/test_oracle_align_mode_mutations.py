"""The mode-traceback pins catch plausible mistakes in the oracle's traceback
of the non-local modes (CPU only).

Each case plants one mistake in a temporary copy of oracle/align_modes.c (the
last maximum instead of the first, a missed candidate, a dropped or extra
boundary gap, a zero floor, a swapped priority, a wrong flag, a wrong
first-column price, unreversed output, an index slip), compiles it, and
checks that the pins of test_oracle_align_mode_pins (brute-force tie rules,
hand-worked examples, rescoring, the mode's coordinates) reject it.  The real
file passes the same battery.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import synth
from tests.pins import brute_force_mode
from tests.test_oracle_align_mode_pins import MODES, _golden, rescore_mode, rule_choice_mode

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "align_modes.c")
MODE_CODE = {"global": 1, "semiglobal": 2, "overlap": 3}

MUTATIONS = {
    "last_maximum_of_row": ("if (Hrow[j] > best) { best = Hrow[j]; bi = m; bj = j; }",
                            "if (Hrow[j] >= best) { best = Hrow[j]; bi = m; bj = j; }"),
    "overlap_ignores_last_column": ("        if (mode == 3)\n            for (int64_t i = 0; i < m; ++i)",
                                    "        if (0)\n            for (int64_t i = 0; i < m; ++i)"),
    "semi_ends_at_last_column_only": ("    if (mode == 1) {\n        best = Hrow[n];",
                                      "    if (mode != 3) {\n        best = Hrow[n];"),
    "global_first_row_gap_dropped": ("if (mode == 1) while (j > 0) { rev[k++] = 2; --j; }", ""),
    "semi_stops_at_first_column": ("if (mode != 3) while (i > 0) { rev[k++] = 1; --i; }",
                                   "if (mode == 1) while (i > 0) { rev[k++] = 1; --i; }"),
    "overlap_pays_first_column": ("if (mode != 3) while (i > 0) { rev[k++] = 1; --i; }",
                                  "while (i > 0) { rev[k++] = 1; --i; }"),
    "horizontal_before_diagonal": ("if (r & R_DIAG) { rev[k++] = 0; --i; --j; }\n            else if (r & R_HE) state = 1;",
                                   "if (r & R_HE) state = 1;\n            else if (r & R_DIAG) { rev[k++] = 0; --i; --j; }"),
    "zero_floor": ("const int64_t H = amax2(D, amax2(E, F));", "const int64_t H = amax2(amax2(D, amax2(E, F)), 0);"),
    "semi_first_column_free": ("const int64_t Hcol0 = (mode == 3) ? 0 : -lead(i, o, e);",
                               "const int64_t Hcol0 = (mode >= 2) ? 0 : -lead(i, o, e);"),
    "leading_gap_extends_at_e": ("return k <= 0 ? 0 : o + (k - 1) * (e < o ? e : o);",
                                 "return k <= 0 ? 0 : o + (k - 1) * e;"),
    "e_open_reads_f_flag": ("if (r & R_EOPEN) state = 0;", "if (r & R_FOPEN) state = 0;"),
    "ops_not_reversed": ("ops[x] = rev[k - 1 - x];", "ops[x] = rev[x];"),
    "target_begin_off_by_one": ("coords[2] = j;", "coords[2] = j + 1;"),
}


def _build(tmp_path, name, src_text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", str(c), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    vp_t, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.swo_align_mode.restype = ctypes.c_int
    lib.swo_align_mode.argtypes = [vp_t, i64, vp_t, i64, vp_t, ctypes.c_int32, i64, i64, ctypes.c_int32,
                                   vp_t, vp_t, vp_t, vp_t]

    def align(q, t, S, o, e, mode):
        q = np.ascontiguousarray(q, np.uint8)
        t = np.ascontiguousarray(t, np.uint8)
        S = np.ascontiguousarray(S, np.int32)
        sc = np.zeros(1, np.int64)
        coords = np.zeros(4, np.int64)
        ops = np.zeros(len(q) + len(t) + 1, np.uint8)
        n_ops = np.zeros(1, np.int64)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        qq = q if len(q) else np.zeros(1, np.uint8)
        tt = t if len(t) else np.zeros(1, np.uint8)
        lib.swo_align_mode(vp(qq), len(q), vp(tt), len(t), vp(S), S.shape[0], o, e, MODE_CODE[mode],
                           vp(sc), vp(coords), vp(ops), vp(n_ops))
        return {"score": int(sc[0]), "q_begin": int(coords[0]), "q_end": int(coords[1]), "t_begin": int(coords[2]),
                "t_end": int(coords[3]), "ops": [int(x) for x in ops[:int(n_ops[0])]]}
    return align


def _key(a):
    return (a["score"], a["q_begin"], a["q_end"], a["t_begin"], a["t_end"], tuple(int(x) for x in a["ops"]))


def _battery(align):
    """Return the list of failed pin checks for a mode-alignment function."""
    fails = []
    for name, mode, S, o, e, q, t, score, c, ops in _golden():
        if _key(align(q, t, S, o, e, mode)) != (score, c[0], c[1], c[2], c[3], tuple(ops)):
            fails.append(f"golden:{name}")
    rng = np.random.default_rng(79)
    for k in range(240):
        mode = MODES[k % 3]
        A = int(rng.integers(1, 4))
        S = rng.integers(-3, 5, size=(A, A))
        o = 0 if k % 2 else int(rng.integers(0, 4))
        e = int(rng.integers(0, 4))
        m = int(rng.integers(0, 5))
        n = int(rng.integers(0, 7 - max(m, 1)))
        q, t = rng.integers(0, A, m), rng.integers(0, A, n)
        if _key(align(q, t, S, o, e, mode)) != _key(rule_choice_mode(q, t, S, o, e, mode)):
            fails.append(f"brute[{k}]")
        elif align(q, t, S, o, e, mode)["score"] != brute_force_mode(q, t, S, o, e, mode):
            fails.append(f"score[{k}]")
    for k in range(30):
        mode = MODES[k % 3]
        S = synth.blosum62()
        q, t = rng.integers(0, 20, 50), rng.integers(0, 20, 60)
        a = align(q, t, S, 10, 1, mode)
        try:
            total, end = rescore_mode(q, t, S, 10, 1, a)
        except IndexError:
            fails.append(f"rescore_index[{k}]")
            continue
        if total != a["score"] or end != (a["q_end"], a["t_end"]):
            fails.append(f"rescore[{k}]")
    return fails


def test_real_mode_traceback_passes_battery(tmp_path):
    assert _battery(_build(tmp_path, "real", open(SRC).read())) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mode_traceback_mutant_is_caught(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    assert _battery(_build(tmp_path, name, src.replace(old, new))), f"mutation {name} was not caught by any pin"
