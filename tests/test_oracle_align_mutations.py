"""The traceback pins catch plausible mistakes in the oracle's traceback (CPU only).

Each case plants one mistake in a temporary copy of oracle/traceback.c (the
last maximum instead of the first, a swapped priority, a flag read from the
wrong neighbour, a missing stop, an index slip, unreversed output), compiles
it, and checks that the pins of test_oracle_align_pins (brute-force tie
rules, hand-worked examples, rescoring and path properties) reject it.  The
real traceback passes the same battery.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import synth
from tests.test_oracle_align_pins import _golden, rescore, rule_choice

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "traceback.c")

MUTATIONS = {
    "last_maximum": ("if (H > best) { best = H; bi = i; bj = j; }",
                     "if (H >= best && H > 0) { best = H; bi = i; bj = j; }"),
    "horizontal_before_diagonal": ("if (r & R_DIAG) { rev[k++] = 0; --i; --j; }\n                else if (r & R_HE) state = 1;",
                            "if (r & R_HE) state = 1;\n                else if (r & R_DIAG) { rev[k++] = 0; --i; --j; }"),
    "horizontal_gap_dropped": ("else if (r & R_HE) state = 1;", "else if (0) state = 1;"),
    "vertical_before_horizontal": ("else if (r & R_HE) state = 1;\n                else if (r & R_HF) state = 2;",
                                   "else if (r & R_HF) state = 2;\n                else if (r & R_HE) state = 1;"),
    "e_open_reads_f_flag": ("if (r & R_EOPEN) state = 0;", "if (r & R_FOPEN) state = 0;"),
    "f_open_from_left": ("if (F == Hup - o) r |= R_FOPEN;", "if (F == Hleft - o) r |= R_FOPEN;"),
    "no_stop_at_zero": ("if (r & R_ZERO) break;", ""),
    "zero_flag_from_diagonal": ("if (H == 0) r |= R_ZERO;", "if (D == 0) r |= R_ZERO;"),
    "query_begin_off_by_one": ("coords[0] = i;", "coords[0] = i + 1;"),
    "ops_not_reversed": ("ops[x] = rev[k - 1 - x];", "ops[x] = rev[x];"),
    "vertical_gap_emits_d": ("rev[k++] = 1;", "rev[k++] = 2;"),
}


def _build(tmp_path, name, src_text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", str(c), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    lib.swo_align.restype = ctypes.c_int64
    vp_t, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.swo_align.argtypes = [vp_t, i64, vp_t, i64, vp_t, ctypes.c_int32, i64, i64, vp_t, vp_t, vp_t]

    def align(q, t, S, o, e):
        q = np.ascontiguousarray(q, np.uint8)
        t = np.ascontiguousarray(t, np.uint8)
        S = np.ascontiguousarray(S, np.int32)
        coords = np.zeros(4, np.int64)
        ops = np.zeros(max(len(q) + len(t), 1), np.uint8)
        n_ops = np.zeros(1, np.int64)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        qq = q if len(q) else np.zeros(1, np.uint8)
        tt = t if len(t) else np.zeros(1, np.uint8)
        r = lib.swo_align(vp(qq), len(q), vp(tt), len(t), vp(S), S.shape[0], o, e, vp(coords), vp(ops), vp(n_ops))
        return {"score": int(r), "q_begin": int(coords[0]), "q_end": int(coords[1]), "t_begin": int(coords[2]),
                "t_end": int(coords[3]), "ops": [int(x) for x in ops[:int(n_ops[0])]]}
    return align


def _key(a):
    return (a["score"], a["q_begin"], a["q_end"], a["t_begin"], a["t_end"], tuple(int(x) for x in a["ops"]))


def _battery(align):
    """Return the list of failed pin checks for an alignment function."""
    fails = []
    for name, S, o, e, q, t, score, c, ops in _golden():
        if _key(align(q, t, S, o, e)) != (score, c[0], c[1], c[2], c[3], tuple(ops)):
            fails.append(f"golden:{name}")
    rng = np.random.default_rng(77)
    for k in range(400):
        A = int(rng.integers(1, 4))
        S = rng.integers(-3, 5, size=(A, A))
        o = 0 if k % 2 else int(rng.integers(0, 4))      # free gap opening makes ties common
        e = int(rng.integers(0, 4))
        m = int(rng.integers(0, 5))
        n = int(rng.integers(0, 7 - max(m, 1)))
        q, t = rng.integers(0, A, m), rng.integers(0, A, n)
        if _key(align(q, t, S, o, e)) != _key(rule_choice(q, t, S, o, e)):
            fails.append(f"brute[{k}]")
    for k in range(40):
        S = synth.blosum62()
        q, t = rng.integers(0, 20, 60), rng.integers(0, 20, 70)
        a = align(q, t, S, 10, 1)
        try:
            total, end, prefixes = rescore(q, t, S, 10, 1, a)
        except IndexError:
            fails.append(f"rescore_index[{k}]")
            continue
        if total != a["score"] or end != (a["q_end"], a["t_end"]) or (prefixes and min(prefixes) <= 0):
            fails.append(f"rescore[{k}]")
    return fails


def test_real_traceback_passes_battery(tmp_path):
    assert _battery(_build(tmp_path, "real", open(SRC).read())) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_traceback_mutant_is_caught(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    assert _battery(_build(tmp_path, name, src.replace(old, new))), f"mutation {name} was not caught by any pin"
