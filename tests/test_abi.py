"""The C ABI library without a GPU: it loads, exports every function that
include/ldd.h declares, and rejects bad arguments before touching a device."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ldd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ldd_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ldd_create_graph", "ldd_decompose", "ldd_cut_edges", "ldd_set_stream",
                     "ldd_destroy_graph", "ldd_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(ldd):
    lib = ctypes.CDLL(ldd.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(ldd):
    for code in range(0, -7, -1):
        s = ldd.ldd_status_string(code)
        assert s.startswith("LDD_")
    assert "unknown" in ldd.ldd_status_string(42)


def test_argument_errors_need_no_device(ldd):
    lib = ctypes.CDLL(ldd.library_path())
    lib.ldd_decompose.argtypes = [ctypes.c_void_p, ctypes.c_double] + [ctypes.c_void_p] * 3
    lib.ldd_cut_edges.argtypes = [ctypes.c_void_p] * 3
    lib.ldd_set_stream.argtypes = [ctypes.c_void_p] * 2
    lib.ldd_create_graph.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.c_void_p]
    assert lib.ldd_decompose(None, 0.1, None, None, None) == ldd.LDD_ERR_ARG
    assert lib.ldd_cut_edges(None, None, None) == ldd.LDD_ERR_ARG
    lib.ldd_decompose_batch.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 5
    assert lib.ldd_decompose_batch(None, 1, None, None, None, None, None) == ldd.LDD_ERR_ARG
    assert lib.ldd_set_stream(None, None) == ldd.LDD_ERR_ARG
    lib.ldd_block_decompose.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 7
    blocks = ctypes.c_int32(-1)
    assert lib.ldd_block_decompose(None, 1, None, None, None, None, None, None,
                                   ctypes.byref(blocks)) == ldd.LDD_ERR_ARG
    assert blocks.value == 0
    lib.ldd_set_wait_limits.argtypes = [ctypes.c_void_p] * 2
    assert lib.ldd_set_wait_limits(None, None) == ldd.LDD_ERR_ARG
    lib.ldd_create_union.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.ldd_union_size.argtypes = [ctypes.c_void_p] * 3
    lib.ldd_union_decompose.argtypes = [ctypes.c_void_p] * 6
    u = ctypes.c_void_p()
    assert lib.ldd_create_union(0, None, ctypes.byref(u)) == ldd.LDD_ERR_ARG
    nulls = (ctypes.c_void_p * 2)(None, None)
    assert lib.ldd_create_union(2, nulls, ctypes.byref(u)) == ldd.LDD_ERR_ARG
    assert lib.ldd_create_union(1, nulls, None) == ldd.LDD_ERR_ARG
    assert lib.ldd_union_size(None, None, None) == ldd.LDD_ERR_ARG
    assert lib.ldd_union_decompose(None, None, None, None, None, None) == ldd.LDD_ERR_ARG
    lib.ldd_server_create.argtypes = [ctypes.c_void_p] * 2
    lib.ldd_server_submit.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double] + [ctypes.c_void_p] * 5
    lib.ldd_server_wait.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.ldd_server_destroy.argtypes = [ctypes.c_void_p]
    srv = ctypes.c_void_p()
    assert lib.ldd_server_create(None, ctypes.byref(srv)) == ldd.LDD_ERR_ARG
    bad = ldd.ServerConfig(1 << 30, 0, 1, 0, 0, 0, 0)  # max_batch 0
    assert lib.ldd_server_create(ctypes.byref(bad), ctypes.byref(srv)) == ldd.LDD_ERR_ARG
    bad = ldd.ServerConfig(0, 4, 1, 0, 0, 0, 0)  # no budget
    assert lib.ldd_server_create(ctypes.byref(bad), ctypes.byref(srv)) == ldd.LDD_ERR_ARG
    t = ctypes.c_int64()
    assert lib.ldd_server_submit(None, None, 0.1, None, None, None, None, ctypes.byref(t)) == ldd.LDD_ERR_ARG
    assert lib.ldd_server_wait(None, 0, None) == ldd.LDD_ERR_ARG
    assert lib.ldd_server_destroy(None) == ldd.LDD_OK
    lib.ldd_decompose_retry.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32] + [ctypes.c_void_p] * 5
    acc = ctypes.c_int32(5)
    assert lib.ldd_decompose_retry(None, 0.1, 1, None, 0, 0, None, None, None, None,
                                   ctypes.byref(acc)) == ldd.LDD_ERR_ARG
    assert acc.value == -1
    lib.ldd_decompose_ranked.argtypes = [ctypes.c_void_p] * 5
    assert lib.ldd_decompose_ranked(None, None, None, None, None) == ldd.LDD_ERR_ARG
    lib.ldd_get_tuning.argtypes = [ctypes.c_void_p] * 2
    lib.ldd_set_tuning.argtypes = [ctypes.c_void_p] * 2
    lib.ldd_autotune.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    tun = ldd.Tuning()
    assert lib.ldd_get_tuning(None, ctypes.byref(tun)) == ldd.LDD_ERR_ARG
    assert lib.ldd_set_tuning(None, ctypes.byref(tun)) == ldd.LDD_ERR_ARG
    assert lib.ldd_autotune(None, None, 1, ctypes.byref(tun)) == ldd.LDD_ERR_ARG
    lib.ldd_set_graph_replay.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.ldd_set_graph_replay(None, 1) == ldd.LDD_ERR_ARG
    out = ctypes.c_void_p()
    rp = np.zeros(4, dtype=np.int32)
    assert lib.ldd_create_graph(3, 0, rp.ctypes.data, None, 1, None) == ldd.LDD_ERR_ARG
    assert lib.ldd_create_graph(-1, 0, rp.ctypes.data, None, 1, ctypes.byref(out)) == ldd.LDD_ERR_ARG
    assert lib.ldd_create_graph(1 << 30, 0, rp.ctypes.data, None, 1, ctypes.byref(out)) == ldd.LDD_ERR_RANGE
    assert lib.ldd_create_graph(3, 1 << 31, rp.ctypes.data, None, 1, ctypes.byref(out)) == ldd.LDD_ERR_RANGE
    assert lib.ldd_create_graph(3, 2, None, None, 1, ctypes.byref(out)) == ldd.LDD_ERR_ARG
    lib.ldd_destroy_graph(None)  # no-op
    assert "NULL" in ldd.ldd_last_error() or ldd.ldd_last_error() == ""


def test_binding_checks_dtypes(ldd):
    with pytest.raises(TypeError):
        ldd._addr(np.zeros(4, dtype=np.int64), "i32", 4, "row_ptr")
    with pytest.raises(ValueError):
        ldd._addr(np.zeros(2, dtype=np.int32), "i32", 4, "row_ptr")
    assert ldd._addr(np.zeros(4, dtype=np.int32), "i32", 4, "row_ptr") != 0


def test_stats_layout_matches_header(ldd, tmp_path):
    """The binding's ldd_stats mirror has the C struct's size and offsets."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in ldd._Stats._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "ldd.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(ldd_stats));\n' +
                   "".join(f'  printf("%zu\\n", offsetof(ldd_stats, {f}));\n' for f in fields) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(ldd._Stats)
    assert got[1:] == [getattr(ldd._Stats, f).offset for f in fields]
