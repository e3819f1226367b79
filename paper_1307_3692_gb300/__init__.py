"""GB300 (sm_103a) exponential-shift low-diameter decomposition.

Python binding of the C ABI in ``include/ldd.h`` (libldd.so): the same entry
points under the same names, argument marshalling only.  Every step of a
decomposition runs in the library's CUDA kernels; there is no CPU path.  The
library must have been built (``__graft_entry__.build()`` or
``python -m paper_1307_3692_gb300._build``); importing without it raises.

Method: Miller, Peng, Xu, "Parallel Graph Decompositions Using Random Shifts"
(2013) -- each vertex u carries a shift delta_u ~ Exp(beta) and every vertex v
joins the u minimising dist(u, v) - delta_u (Algorithm 2), computed as the
delayed-start BFS of Section 4.

Buffers may be torch tensors (CPU or CUDA), numpy arrays, or raw integer
addresses; dtypes are int32 for the CSR and outputs, float64 for shifts.
"""
from __future__ import annotations

import ctypes
import os

from ._build import LIB as _LIB_PATH

__all__ = [
    "LddError", "LddGraph", "ldd_create_graph", "ldd_decompose", "ldd_cut_edges",
    "ldd_set_stream", "ldd_destroy_graph", "ldd_status_string", "ldd_last_error",
    "ldd_get_stats", "ldd_set_timing", "ldd_cut_edges_noalloc", "ldd_get_round_profile",
    "ldd_decompose_batch", "ldd_set_graph_replay", "ldd_create_union", "ldd_union_size", "ldd_union_decompose", "LddUnion",
    "library_path", "LDD_OK", "LDD_ERR_ARG",
    "LDD_ERR_GRAPH", "LDD_ERR_RANGE", "LDD_ERR_OOM", "LDD_ERR_CUDA", "LDD_ERR_TIMEOUT",
]

LDD_OK, LDD_ERR_ARG, LDD_ERR_GRAPH, LDD_ERR_RANGE = 0, -1, -2, -3
LDD_ERR_OOM, LDD_ERR_CUDA, LDD_ERR_TIMEOUT = -4, -5, -6

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"{_LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(_LIB_PATH)


class _Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "n", "nnz", "n_active", "small_components", "max_floor_shift", "rounds", "last_level", "items", "edges", "pull_rounds", "push_arcs", "pull_arcs",
        "pull_vertices",
        "launches", "cut_launches", "exact_rank")] + [("bfs_grid", ctypes.c_int32), ("bfs_block", ctypes.c_int32)] + [
        (name, ctypes.c_float) for name in (
            "ms_h2d", "ms_rank", "ms_bfs", "ms_finalize", "ms_d2h", "ms_total", "ms_cut",
            "ms_replay")] + [("replayed", ctypes.c_int32)]


_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_lib.ldd_create_graph.argtypes = [_i32, _i64, _vp, _vp, ctypes.c_int, ctypes.POINTER(_vp)]
_lib.ldd_create_graph.restype = ctypes.c_int
_lib.ldd_decompose.argtypes = [_vp, ctypes.c_double, _vp, _vp, _vp]
_lib.ldd_decompose.restype = ctypes.c_int
_lib.ldd_decompose_batch.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
_lib.ldd_decompose_batch.restype = ctypes.c_int
_lib.ldd_create_union.argtypes = [ctypes.c_int, _vp, ctypes.POINTER(_vp)]
_lib.ldd_create_union.restype = ctypes.c_int
_lib.ldd_union_size.argtypes = [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]
_lib.ldd_union_size.restype = ctypes.c_int
_lib.ldd_union_decompose.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
_lib.ldd_union_decompose.restype = ctypes.c_int
_lib.ldd_cut_edges.argtypes = [_vp, _vp, ctypes.POINTER(_i64)]
_lib.ldd_cut_edges.restype = ctypes.c_int
_lib.ldd_cut_edges_noalloc.argtypes = [_i32, _i64, _vp, _vp, _vp, _vp, _vp]
_lib.ldd_cut_edges_noalloc.restype = ctypes.c_int
_lib.ldd_set_stream.argtypes = [_vp, _vp]
_lib.ldd_set_stream.restype = ctypes.c_int
_lib.ldd_destroy_graph.argtypes = [_vp]
_lib.ldd_destroy_graph.restype = None
_lib.ldd_status_string.argtypes = [ctypes.c_int]
_lib.ldd_status_string.restype = ctypes.c_char_p
_lib.ldd_last_error.argtypes = []
_lib.ldd_last_error.restype = ctypes.c_char_p
_lib.ldd_get_stats.argtypes = [_vp, ctypes.POINTER(_Stats)]
_lib.ldd_get_stats.restype = ctypes.c_int
_lib.ldd_get_round_profile.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
_lib.ldd_get_round_profile.restype = ctypes.c_int
_lib.ldd_set_timing.argtypes = [_vp, ctypes.c_int]
_lib.ldd_set_timing.restype = ctypes.c_int
_lib.ldd_set_graph_replay.argtypes = [_vp, ctypes.c_int]
_lib.ldd_set_graph_replay.restype = ctypes.c_int


def library_path() -> str:
    return _LIB_PATH


class LddError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.ldd_last_error().decode() or ""
        super().__init__(f"{where}: {ldd_status_string(status)}" + (f" ({msg})" if msg else ""))


def _check(status: int, where: str) -> None:
    if status != LDD_OK:
        raise LddError(status, where)


def _addr(buf, dtype_name: str, count: int | None, what: str) -> int:
    """Address of a torch tensor / numpy array / raw int, with dtype and size checks."""
    if buf is None:
        return 0
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):  # torch.Tensor
        if not buf.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        if str(buf.dtype).split(".")[-1] != {"i32": "int32", "f64": "float64"}[dtype_name]:
            raise TypeError(f"{what}: dtype {buf.dtype}, expected {dtype_name}")
        if count is not None and buf.numel() < count:
            raise ValueError(f"{what}: {buf.numel()} elements, need {count}")
        return int(buf.data_ptr())
    if hasattr(buf, "__array_interface__"):  # numpy
        want = {"i32": "<i4", "f64": "<f8"}[dtype_name]
        if buf.dtype.str != want or not buf.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{what}: need a C-contiguous {dtype_name} array, got {buf.dtype}")
        if count is not None and buf.size < count:
            raise ValueError(f"{what}: {buf.size} elements, need {count}")
        return int(buf.__array_interface__["data"][0])
    raise TypeError(f"{what}: unsupported buffer type {type(buf)}")


def ldd_status_string(status: int) -> str:
    return _lib.ldd_status_string(status).decode()


def ldd_last_error() -> str:
    return _lib.ldd_last_error().decode()


def ldd_create_graph(n: int, nnz: int, row_ptr, col_idx, validate: int = 1) -> int:
    """Handle of a library-owned device copy of the CSR (see include/ldd.h)."""
    out = _vp()
    _check(_lib.ldd_create_graph(n, nnz, _addr(row_ptr, "i32", n + 1, "row_ptr"),
                                 _addr(col_idx, "i32", nnz, "col_idx"), int(validate),
                                 ctypes.byref(out)), "ldd_create_graph")
    return int(out.value)


def ldd_decompose(g: int, beta: float, shifts, out_center, out_dist, n: int | None = None) -> None:
    _check(_lib.ldd_decompose(g, float(beta), _addr(shifts, "f64", n, "shifts"),
                              _addr(out_center, "i32", n, "out_center"),
                              _addr(out_dist, "i32", n, "out_dist")), "ldd_decompose")


def ldd_decompose_batch(g: int, betas, shifts, out_center, out_dist, n: int | None = None,
                        want_cut: bool = True):
    """k pipelined decompositions (include/ldd.h); returns the k cut counts
    (or None without want_cut).  shifts, out_center, out_dist: sequences of k
    buffers each."""
    k = len(betas)
    if not (len(shifts) == len(out_center) == len(out_dist) == k):
        raise ValueError("betas, shifts, out_center and out_dist need the same length")
    b = (ctypes.c_double * max(k, 1))(*[float(x) for x in betas])
    sp = (_vp * max(k, 1))(*[_addr(x, "f64", n, "shifts") for x in shifts])
    cp = (_vp * max(k, 1))(*[_addr(x, "i32", n, "out_center") for x in out_center])
    dp = (_vp * max(k, 1))(*[_addr(x, "i32", n, "out_dist") for x in out_dist])
    cuts = (_i64 * max(k, 1))()
    _check(_lib.ldd_decompose_batch(g, k, b, sp, cp, dp, cuts if want_cut else None),
           "ldd_decompose_batch")
    return [int(cuts[i]) for i in range(k)] if want_cut else None


def ldd_create_union(members) -> int:
    """Handle of the disjoint union of the member graphs (handles or LddGraph)."""
    hs = [getattr(m, "handle", m) for m in members]
    arr = (_vp * max(len(hs), 1))(*hs)
    out = _vp()
    _check(_lib.ldd_create_union(len(hs), arr, ctypes.byref(out)), "ldd_create_union")
    return int(out.value)


def ldd_union_size(u: int) -> tuple[int, int]:
    """(k, total) of a union."""
    k, total = _i32(0), _i64(0)
    _check(_lib.ldd_union_size(u, ctypes.byref(k), ctypes.byref(total)), "ldd_union_size")
    return int(k.value), int(total.value)


def ldd_union_decompose(u: int, betas, shifts, out_center, out_dist, want_cut: bool = True):
    """Every member of a union in one pass (include/ldd.h); returns the k cut
    counts (or None without want_cut)."""
    k, total = ldd_union_size(u)
    if len(betas) != k:
        raise ValueError(f"{len(betas)} betas for {k} members")
    b = (ctypes.c_double * k)(*[float(x) for x in betas])
    cuts = (_i64 * k)()
    _check(_lib.ldd_union_decompose(u, b, _addr(shifts, "f64", total, "shifts"),
                                    _addr(out_center, "i32", total, "out_center"),
                                    _addr(out_dist, "i32", total, "out_dist"),
                                    cuts if want_cut else None), "ldd_union_decompose")
    return [int(cuts[i]) for i in range(k)] if want_cut else None


def ldd_cut_edges(g: int, center, n: int | None = None) -> int:
    out = _i64(0)
    _check(_lib.ldd_cut_edges(g, _addr(center, "i32", n, "center"), ctypes.byref(out)),
           "ldd_cut_edges")
    return int(out.value)


def ldd_cut_edges_noalloc(n: int, nnz: int, row_ptr, col_idx, center, stream=None) -> int:
    """Cut count from device-resident CSR and labels, with no device allocation
    (see include/ldd.h for who needs this and its limits)."""
    out = _i64(0)
    handle = getattr(stream, "cuda_stream", stream)
    _check(_lib.ldd_cut_edges_noalloc(n, nnz, _addr(row_ptr, "i32", n + 1, "row_ptr"),
                                      _addr(col_idx, "i32", nnz, "col_idx"),
                                      _addr(center, "i32", n, "center"), ctypes.byref(out),
                                      handle or 0), "ldd_cut_edges_noalloc")
    return int(out.value)


def ldd_set_stream(g: int, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t address, or None."""
    handle = getattr(stream, "cuda_stream", stream)
    _check(_lib.ldd_set_stream(g, handle or 0), "ldd_set_stream")


def ldd_destroy_graph(g: int) -> None:
    _lib.ldd_destroy_graph(g)


def ldd_set_timing(g: int, enable: bool) -> None:
    _check(_lib.ldd_set_timing(g, int(bool(enable))), "ldd_set_timing")


def ldd_set_graph_replay(g: int, enable: bool) -> None:
    _check(_lib.ldd_set_graph_replay(g, int(bool(enable))), "ldd_set_graph_replay")


def ldd_get_round_profile(g: int, cap: int = 256):
    """(clocks, kinds) of the last BFS's rounds (see include/ldd.h)."""
    import numpy as np

    clocks = np.zeros((cap, 3), dtype=np.int64)
    kinds = np.zeros(cap, dtype=np.int32)
    cnt = ctypes.c_int(0)
    _check(_lib.ldd_get_round_profile(g, clocks.ctypes.data, kinds.ctypes.data, cap,
                                      ctypes.byref(cnt)), "ldd_get_round_profile")
    return clocks[:cnt.value], kinds[:cnt.value]


def ldd_get_stats(g: int) -> dict:
    st = _Stats()
    _check(_lib.ldd_get_stats(g, ctypes.byref(st)), "ldd_get_stats")
    return {name: getattr(st, name) for name, _ in _Stats._fields_}


class LddGraph:
    """Owns one ldd_graph handle; sizes checked on every call."""

    def __init__(self, row_ptr, col_idx, validate: bool = True):
        self.n = int(row_ptr.shape[0]) - 1
        self.nnz = int(col_idx.shape[0])
        self.handle = ldd_create_graph(self.n, self.nnz, row_ptr, col_idx, validate)

    def decompose(self, beta: float, shifts, out_center, out_dist) -> None:
        ldd_decompose(self.handle, beta, shifts, out_center, out_dist, self.n)

    def decompose_batch(self, betas, shifts, out_center, out_dist, want_cut: bool = True):
        return ldd_decompose_batch(self.handle, betas, shifts, out_center, out_dist, self.n,
                                   want_cut)

    def cut_edges(self, center) -> int:
        return ldd_cut_edges(self.handle, center, self.n)

    def set_stream(self, stream) -> None:
        ldd_set_stream(self.handle, stream)

    def set_timing(self, enable: bool) -> None:
        ldd_set_timing(self.handle, enable)

    def set_graph_replay(self, enable: bool) -> None:
        ldd_set_graph_replay(self.handle, enable)

    def stats(self) -> dict:
        return ldd_get_stats(self.handle)

    def round_profile(self):
        return ldd_get_round_profile(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", 0):
            ldd_destroy_graph(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LddUnion(LddGraph):
    """Owns a union handle (ldd_create_union): k member graphs decomposed in
    one pass.  ``offsets[s]`` is member s's first entry in the caller layout."""

    def __init__(self, members):
        self.handle = ldd_create_union(members)
        self.k, self.total = ldd_union_size(self.handle)
        ns = [int(getattr(m, "n")) for m in members] if all(hasattr(m, "n") for m in members) \
            else None
        self.offsets = None if ns is None else [sum(ns[:i]) for i in range(len(ns) + 1)]
        self.n = self.total

    def decompose(self, betas, shifts, out_center, out_dist, want_cut: bool = True):
        return ldd_union_decompose(self.handle, betas, shifts, out_center, out_dist, want_cut)

    def decompose_batch(self, *a, **kw):
        raise TypeError("a union is decomposed with decompose()")

    def cut_edges(self, center) -> int:
        raise TypeError("a union's cut counts come from decompose()")
