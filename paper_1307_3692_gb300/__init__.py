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
    "ldd_decompose_batch", "ldd_decompose_ranked", "ldd_autotune", "ldd_get_tuning",
    "ldd_set_tuning", "ldd_decompose_retry", "default_bounds", "ldd_set_graph_replay", "ldd_create_union", "LddServer", "ldd_union_size", "ldd_union_decompose", "LddUnion",
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
            "ms_replay")] + [("replayed", ctypes.c_int32)] + [
        (name, ctypes.c_float) for name in ("ms_create_upload", "ms_create_components",
                                            "ms_create_total", "ms_block_total",
                                            "ms_block_residual")] + [
        (name, ctypes.c_int64) for name in ("block_arcs_scanned", "block_arcs_kept",
                                            "bfs_windows", "bfs_overflow")]


_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_lib.ldd_create_graph.argtypes = [_i32, _i64, _vp, _vp, ctypes.c_int, ctypes.POINTER(_vp)]
_lib.ldd_create_graph.restype = ctypes.c_int
_lib.ldd_decompose.argtypes = [_vp, ctypes.c_double, _vp, _vp, _vp]
_lib.ldd_decompose.restype = ctypes.c_int
_lib.ldd_decompose_retry.argtypes = [_vp, ctypes.c_double, ctypes.c_int, _vp, _i64, _i32, _vp,
                                     _vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32),
                                     ctypes.POINTER(_i32)]
_lib.ldd_decompose_retry.restype = ctypes.c_int
_lib.ldd_decompose_ranked.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.ldd_decompose_ranked.restype = ctypes.c_int
_lib.ldd_decompose_batch.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
_lib.ldd_decompose_batch.restype = ctypes.c_int
_lib.ldd_block_decompose.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp,
                                     ctypes.POINTER(_i32)]
_lib.ldd_block_decompose.restype = ctypes.c_int
_lib.ldd_create_union.argtypes = [ctypes.c_int, _vp, ctypes.POINTER(_vp)]
_lib.ldd_create_union.restype = ctypes.c_int
_lib.ldd_union_size.argtypes = [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]
_lib.ldd_union_size.restype = ctypes.c_int
_lib.ldd_union_decompose.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
_lib.ldd_union_decompose.restype = ctypes.c_int
class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("one_at_a_time", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("max_vertices", ctypes.c_int64),
                ("max_arcs", ctypes.c_int64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("batch_id", ctypes.c_int64), ("submit_us", ctypes.c_double),
                ("start_us", ctypes.c_double), ("end_us", ctypes.c_double),
                ("batch_fill_us", ctypes.c_double), ("batch_run_us", ctypes.c_double)]


_lib.ldd_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]
_lib.ldd_server_create.restype = ctypes.c_int
_lib.ldd_server_submit.argtypes = [_vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp,
                                   ctypes.POINTER(_i64)]
_lib.ldd_server_submit.restype = ctypes.c_int
_lib.ldd_server_wait.argtypes = [_vp, _i64, ctypes.POINTER(RequestInfo)]
_lib.ldd_server_wait.restype = ctypes.c_int
_lib.ldd_server_footprint.argtypes = [_vp, _vp, ctypes.POINTER(_i64)]
_lib.ldd_server_footprint.restype = ctypes.c_int
_lib.ldd_server_destroy.argtypes = [_vp]
_lib.ldd_server_destroy.restype = ctypes.c_int
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
class Tuning(ctypes.Structure):
    _fields_ = [("bfs_blocks_per_sm", ctypes.c_int32), ("pull_alpha", ctypes.c_int32),
                ("pull_beta", ctypes.c_int32), ("pull_gamma", ctypes.c_int32),
                ("probe_min_arcs", ctypes.c_int32), ("low_degree_rounds", ctypes.c_int32),
                ("window_levels", ctypes.c_int32), ("window_max_frontier", ctypes.c_int32),
                ("window_queue", ctypes.c_int32), ("bfs_span", ctypes.c_int32),
                ("ms", ctypes.c_float)]


_lib.ldd_get_tuning.argtypes = [_vp, ctypes.POINTER(Tuning)]
_lib.ldd_get_tuning.restype = ctypes.c_int
_lib.ldd_set_tuning.argtypes = [_vp, ctypes.POINTER(Tuning)]
_lib.ldd_set_tuning.restype = ctypes.c_int
_lib.ldd_autotune.argtypes = [_vp, _vp, ctypes.c_int, ctypes.POINTER(Tuning)]
_lib.ldd_autotune.restype = ctypes.c_int
_lib.ldd_set_graph_replay.argtypes = [_vp, ctypes.c_int]
_lib.ldd_set_graph_replay.restype = ctypes.c_int


class WaitLimits(ctypes.Structure):
    _fields_ = [("barrier_polls", ctypes.c_uint32), ("lookback_polls", ctypes.c_uint32),
                ("stall_barrier", ctypes.c_uint32), ("stall_lookback", ctypes.c_uint32)]


_lib.ldd_set_wait_limits.argtypes = [_vp, ctypes.POINTER(WaitLimits)]
_lib.ldd_set_wait_limits.restype = ctypes.c_int
_lib.ldd_get_wait_limits.argtypes = [_vp, ctypes.POINTER(WaitLimits)]
_lib.ldd_get_wait_limits.restype = ctypes.c_int


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


def ldd_decompose_retry(g: int, beta: float, shifts, max_cut: int, max_radius: int, out_center,
                        out_dist, n: int | None = None):
    """Las Vegas loop of Theorem 1.2's proof (include/ldd.h): returns
    (accepted index or -1, cut, radius)."""
    k = len(shifts)
    sp = (_vp * max(k, 1))(*[_addr(x, "f64", n, "shifts") for x in shifts])
    cut, rad, acc = _i64(0), _i32(0), _i32(-1)
    _check(_lib.ldd_decompose_retry(g, float(beta), k, sp, int(max_cut), int(max_radius),
                                    _addr(out_center, "i32", n, "out_center"),
                                    _addr(out_dist, "i32", n, "out_dist"), ctypes.byref(cut),
                                    ctypes.byref(rad), ctypes.byref(acc)), "ldd_decompose_retry")
    return int(acc.value), int(cut.value), int(rad.value)


def default_bounds(n: int, m: int, beta: float, c: float = 2.0):
    """(max_cut, max_radius) of a (beta, c ln(n) / beta) decomposition: at most
    beta m cut edges (Definition 1.1) and radius at most c ln(n) / beta
    (Lemma 3.2: delta_max exceeds it with probability about n^(1 - c))."""
    import math
    return int(math.floor(beta * m)), int(math.ceil(c * math.log(max(n, 2)) / beta))


def ldd_decompose_ranked(g: int, levels, perm, out_center, out_dist, n: int | None = None) -> None:
    """The permutation variant (include/ldd.h): integer levels and a tie-break
    permutation in place of FP64 shifts."""
    _check(_lib.ldd_decompose_ranked(g, _addr(levels, "i32", n, "levels"),
                                     _addr(perm, "i32", n, "perm"),
                                     _addr(out_center, "i32", n, "out_center"),
                                     _addr(out_dist, "i32", n, "out_dist")), "ldd_decompose_ranked")


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


def ldd_block_decompose(g: int, betas, shifts, out_center=None, out_dist=None,
                        out_arc_block=None, n: int | None = None, nnz: int | None = None):
    """Blocks by repeated decomposition (include/ldd.h).  shifts: k buffers;
    out_center / out_dist: None or k buffers; out_arc_block: None or an int32
    buffer of nnz.  Returns (blocks, remaining) with remaining[i] the edges of
    G_i for i = 0 .. blocks."""
    k = len(betas)
    if len(shifts) != k:
        raise ValueError("betas and shifts need the same length")
    for name, arr in (("out_center", out_center), ("out_dist", out_dist)):
        if arr is not None and len(arr) != k:
            raise ValueError(f"{name} needs {k} buffers")
    b = (ctypes.c_double * max(k, 1))(*[float(x) for x in betas])
    sp = (_vp * max(k, 1))(*[_addr(x, "f64", n, "shifts") for x in shifts])
    cp = None if out_center is None else (_vp * max(k, 1))(
        *[_addr(x, "i32", n, "out_center") for x in out_center])
    dp = None if out_dist is None else (_vp * max(k, 1))(
        *[_addr(x, "i32", n, "out_dist") for x in out_dist])
    rem = (_i64 * (k + 1))()
    blocks = _i32(0)
    _check(_lib.ldd_block_decompose(g, k, b, sp, cp, dp,
                                    _addr(out_arc_block, "i32", nnz, "out_arc_block"), rem,
                                    ctypes.byref(blocks)), "ldd_block_decompose")
    nb = int(blocks.value)
    return nb, [int(rem[i]) for i in range(nb + 1)]


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


def _tuning_dict(t: Tuning) -> dict:
    return {name: getattr(t, name) for name, _ in Tuning._fields_}


def ldd_get_tuning(g: int) -> dict:
    t = Tuning()
    _check(_lib.ldd_get_tuning(g, ctypes.byref(t)), "ldd_get_tuning")
    return _tuning_dict(t)


def ldd_set_tuning(g: int, **fields) -> None:
    t = Tuning()
    _check(_lib.ldd_get_tuning(g, ctypes.byref(t)), "ldd_get_tuning")
    for k, v in fields.items():
        setattr(t, k, v)
    _check(_lib.ldd_set_tuning(g, ctypes.byref(t)), "ldd_set_tuning")


def ldd_autotune(g: int, shifts, reps: int = 2, n: int | None = None) -> dict:
    """Times decompositions of this shift vector while varying the launch
    parameters (include/ldd.h); keeps and returns the best."""
    t = Tuning()
    _check(_lib.ldd_autotune(g, _addr(shifts, "f64", n, "shifts"), int(reps), ctypes.byref(t)),
           "ldd_autotune")
    return _tuning_dict(t)


def ldd_set_graph_replay(g: int, enable: bool) -> None:
    _check(_lib.ldd_set_graph_replay(g, int(bool(enable))), "ldd_set_graph_replay")


def ldd_get_wait_limits(g: int) -> dict:
    w = WaitLimits()
    _check(_lib.ldd_get_wait_limits(g, ctypes.byref(w)), "ldd_get_wait_limits")
    return {name: getattr(w, name) for name, _ in WaitLimits._fields_}


def ldd_set_wait_limits(g: int, barrier_polls: int = 0, lookback_polls: int = 0,
                        stall_barrier: int = 0, stall_lookback: int = 0) -> None:
    """Poll limits of the device-side waits (0: default) and the stall
    switches that tests of the timeout path use (include/ldd.h)."""
    w = WaitLimits(barrier_polls, lookback_polls, stall_barrier, stall_lookback)
    _check(_lib.ldd_set_wait_limits(g, ctypes.byref(w)), "ldd_set_wait_limits")


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

    def decompose_ranked(self, levels, perm, out_center, out_dist) -> None:
        ldd_decompose_ranked(self.handle, levels, perm, out_center, out_dist, self.n)

    def decompose_retry(self, beta: float, shifts, max_cut: int, max_radius: int, out_center,
                        out_dist):
        return ldd_decompose_retry(self.handle, beta, shifts, max_cut, max_radius, out_center,
                                   out_dist, self.n)

    def cut_edges(self, center) -> int:
        return ldd_cut_edges(self.handle, center, self.n)

    def block_decompose(self, betas, shifts, out_center=None, out_dist=None,
                        out_arc_block=None):
        return ldd_block_decompose(self.handle, betas, shifts, out_center, out_dist,
                                   out_arc_block, self.n, self.nnz)

    def set_stream(self, stream) -> None:
        ldd_set_stream(self.handle, stream)

    def set_timing(self, enable: bool) -> None:
        ldd_set_timing(self.handle, enable)

    def set_graph_replay(self, enable: bool) -> None:
        ldd_set_graph_replay(self.handle, enable)

    def tuning(self) -> dict:
        return ldd_get_tuning(self.handle)

    def set_tuning(self, **fields) -> None:
        ldd_set_tuning(self.handle, **fields)

    def autotune(self, shifts, reps: int = 2) -> dict:
        return ldd_autotune(self.handle, shifts, reps, self.n)

    def wait_limits(self) -> dict:
        return ldd_get_wait_limits(self.handle)

    def set_wait_limits(self, **fields) -> None:
        ldd_set_wait_limits(self.handle, **fields)

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


def _cut_addr(out_cut):
    """Address of a one-element int64 holder: a ctypes.c_int64 or a numpy array."""
    if out_cut is None:
        return None
    if isinstance(out_cut, ctypes.c_int64):
        return ctypes.addressof(out_cut)
    if hasattr(out_cut, "__array_interface__") and out_cut.dtype.str == "<i8" and out_cut.size >= 1:
        return int(out_cut.__array_interface__["data"][0])
    raise TypeError("out_cut: need a ctypes.c_int64 or an int64 numpy array")


class LddServer:
    """A request server (ldd_server_* in include/ldd.h): continuous batching of
    decompositions of resident graphs.  submit() takes host buffers and
    returns a ticket; wait() blocks for it and returns its ldd_request_info as
    a dict (times in microseconds on the server's clock)."""

    def __init__(self, hbm_budget_bytes: int, max_batch: int = 64, slots: int = 2,
                 one_at_a_time: bool = False, max_vertices: int = 0, max_arcs: int = 0):
        cfg = ServerConfig(int(hbm_budget_bytes), int(max_batch), int(slots), int(one_at_a_time),
                           0, int(max_vertices), int(max_arcs))
        out = _vp()
        _check(_lib.ldd_server_create(ctypes.byref(cfg), ctypes.byref(out)), "ldd_server_create")
        self.handle = int(out.value)
        self._keep = {}

    def submit(self, graph, beta: float, shifts, out_center, out_dist, out_cut=None) -> int:
        n = graph.n
        t = _i64(-1)
        _check(_lib.ldd_server_submit(self.handle, graph.handle, float(beta),
                                      _addr(shifts, "f64", n, "shifts"),
                                      _addr(out_center, "i32", n, "out_center"),
                                      _addr(out_dist, "i32", n, "out_dist"),
                                      _cut_addr(out_cut),
                                      ctypes.byref(t)), "ldd_server_submit")
        self._keep[int(t.value)] = (shifts, out_center, out_dist, out_cut)
        return int(t.value)

    def wait(self, ticket: int) -> dict:
        info = RequestInfo()
        status = _lib.ldd_server_wait(self.handle, int(ticket), ctypes.byref(info))
        self._keep.pop(int(ticket), None)
        _check(status, "ldd_server_wait")
        return {name: getattr(info, name) for name, _ in RequestInfo._fields_}

    def footprint(self, graph) -> int:
        out = _i64(0)
        _check(_lib.ldd_server_footprint(self.handle, graph.handle, ctypes.byref(out)),
               "ldd_server_footprint")
        return int(out.value)

    def close(self) -> None:
        if getattr(self, "handle", 0):
            _lib.ldd_server_destroy(self.handle)
            self.handle = 0
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
