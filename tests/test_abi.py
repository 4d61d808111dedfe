"""The C ABI library loads and exports what include/swdb.h declares (no GPU).

Also checks the argument validation that happens on the host before any
CUDA call, so it runs without a device.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sw_\w+)\s*\(", text, flags=re.M):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11100_gb300 import build, binding
    build.build()
    return binding.load_library()


def test_header_declares_entry_points():
    names = _declared_functions()
    for n in ("sw_db_load", "sw_db_free", "sw_search", "sw_top_k", "sw_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_version(lib):
    assert lib.sw_version().decode().startswith("swdb")


def test_load_rejects_bad_arguments_on_host(lib):
    from paper_2203_11100_gb300 import binding
    res = np.array([0, 1, 2], dtype=np.uint8)
    off = np.array([0, 3], dtype=np.int64)
    h = ctypes.c_void_p()
    # alphabet too large
    rc = lib.sw_db_load(res.ctypes.data, off.ctypes.data, 1, 40, 0, ctypes.byref(h))
    assert rc == 1 and "alphabet" in binding.sw_last_error()
    # code out of range
    rc = lib.sw_db_load(res.ctypes.data, off.ctypes.data, 1, 2, 0, ctypes.byref(h))
    assert rc == 1 and "code" in binding.sw_last_error()
    # decreasing offsets
    bad = np.array([0, 3, 1], dtype=np.int64)
    rc = lib.sw_db_load(res.ctypes.data, bad.ctypes.data, 2, 4, 0, ctypes.byref(h))
    assert rc == 1
    # NULL out
    rc = lib.sw_db_load(res.ctypes.data, off.ctypes.data, 1, 4, 0, None)
    assert rc == 1
    assert not h.value


def test_search_rejects_null_db(lib):
    from paper_2203_11100_gb300 import binding
    with pytest.raises(binding.SwError) as e:
        binding.sw_search(None, np.zeros(3, np.uint8), np.array([0, 3]), np.eye(4, dtype=np.int32), 1, 1, 1)
    assert e.value.code == 1


def test_top_k_rejects_bad_sizes(lib):
    assert lib.sw_top_k(None, 1, 10, 5000, None, None) == 1
    assert lib.sw_top_k(None, -1, 10, 5, None, None) == 1
    assert lib.sw_top_k(None, 0, 10, 5, None, None) == 0


def test_align_rejects_bad_arguments_on_host(lib):
    from paper_2203_11100_gb300 import binding
    pq = np.zeros(1, np.int32)
    pt = np.zeros(1, np.int64)
    off = np.array([0, 3], dtype=np.int64)
    out = ctypes.c_int64(0)
    rc = lib.sw_align_ops_capacity(None, off.ctypes.data, 1, pq.ctypes.data, pt.ctypes.data, 1, ctypes.byref(out))
    assert rc == 1 and "db is NULL" in binding.sw_last_error()
    rc = lib.sw_align_ops_capacity(None, off.ctypes.data, 1, pq.ctypes.data, pt.ctypes.data, 1, None)
    assert rc == 1 and "bytes is NULL" in binding.sw_last_error()
    rc = lib.sw_align(None, None, off.ctypes.data, 1, pq.ctypes.data, pt.ctypes.data, 1, None, 10, 1,
                      None, None, 0, None, None)
    assert rc == 1 and "db is NULL" in binding.sw_last_error()
    rc = lib.sw_align_mode(None, None, off.ctypes.data, 1, pq.ctypes.data, pt.ctypes.data, 1, None, 10, 1, 7,
                           None, None, 0, None, None)
    assert rc == 1 and "unknown alignment mode" in binding.sw_last_error()
    rc = lib.sw_align_mode(None, None, off.ctypes.data, 1, pq.ctypes.data, pt.ctypes.data, 1, None, 10, 1, 1,
                           None, None, 0, None, None)
    assert rc == 1 and "db is NULL" in binding.sw_last_error()


def test_alignment_struct_sizes():
    from paper_2203_11100_gb300 import binding
    assert binding.ALIGNMENT_DTYPE.itemsize == 56
    assert ctypes.sizeof(binding.SwAlignStats) == 32


def test_struct_sizes_match_the_header(tmp_path):
    """The binding's structs have the sizes the C compiler gives the header's."""
    import subprocess
    from paper_2203_11100_gb300 import binding
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "swdb.h"\nint main(void) {\n'
                   '  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(sw_search_opts), sizeof(sw_search_stats),\n'
                   '         sizeof(sw_alignment), sizeof(sw_align_stats), sizeof(sw_hit), sizeof(sw_db_info));\n'
                   '  return 0;\n}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(binding.SwSearchOpts), ctypes.sizeof(binding.SwSearchStats),
            binding.ALIGNMENT_DTYPE.itemsize, ctypes.sizeof(binding.SwAlignStats), binding.HIT_DTYPE.itemsize,
            ctypes.sizeof(binding.SwDbInfo)]
    assert got == want


def test_wait_probe_rejects_bad_arguments_on_host(lib):
    from paper_2203_11100_gb300 import binding
    st = ctypes.c_int32(0)
    ms = ctypes.c_double(0.0)
    assert lib.sw_probe_wait_timeout(0, 0, ctypes.byref(st), ctypes.byref(ms)) == 1
    assert "spin_iters" in binding.sw_last_error()
    assert lib.sw_probe_wait_timeout(0, 1 << 26, ctypes.byref(st), ctypes.byref(ms)) == 1
    assert lib.sw_probe_wait_timeout(0, 1000, None, ctypes.byref(ms)) == 1


def test_tuning_struct_size_matches_the_header(tmp_path):
    import subprocess
    from paper_2203_11100_gb300 import binding
    src = tmp_path / "tsize.c"
    src.write_text('#include <stdio.h>\n#include "swdb.h"\nint main(void) {\n'
                   '  printf("%zu %zu\\n", sizeof(sw_tuning), sizeof(sw_shape_rate));\n  return 0;\n}\n')
    exe = tmp_path / "tsize"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(binding.SwTuning), ctypes.sizeof(binding.SwShapeRate)] == [408, 12]


def test_tuning_rejects_bad_tables_on_host(lib):
    from paper_2203_11100_gb300 import binding
    assert lib.sw_db_set_tuning(None, None) == 1
    assert "db is NULL" in binding.sw_last_error()
