"""ORACLE -- test infrastructure only.

Plain, slow, obviously-correct CPU implementations of the exponential-shift
low-diameter decomposition (Miller, Peng, Xu 2013).  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import this package; the CUDA library never does, and the two share no
code.  The only common dependency is ``ldd_gen`` (seeded inputs).

* ``oracle_ldd``       -- multi-source Dijkstra over exact labels (C, ldd_oracle.c):
                          Algorithm 2 via the super-source reduction of Section 4.
* ``oracle_ldd_ranked`` -- the permutation variant of Section 4 (integer
                          levels + a tie-break permutation), through
                          ``oracle_ldd`` on shifts that order the same way.
* ``oracle_cut_edges`` -- Definition 1.1's count of edges between pieces.
* ``oracle_block_decompose`` -- blocks by repeated decomposition (Section 1,
                          related work): decompose, keep the cut edges,
                          decompose them again, until no edge is left.
* ``oracle_certify``   -- O(m) optimality certificate (Lemma 3.1 predecessor +
                          non-improvability), usable at any size.
* ``brute.brute_ldd``  -- Algorithm 2 written out literally: all-pairs BFS and
                          an exact-rational argmin (tiny graphs only).

Every function here is pinned in ``tests/test_oracle.py`` against values and
properties fixed by the paper and by mathematics, not against itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CERT_CODES = {
    0: "ok",
    1: "center out of range or negative distance",
    2: "center is not its own center at distance 0",
    3: "no predecessor in the same piece at distance - 1 (Lemma 3.1)",
    4: "improvable by the vertex's own start label -delta_v",
    5: "improvable by a neighbour's label + 1",
}


def build(force: bool = False) -> str:
    """Compile ldd_oracle.c (gcc, single-threaded, -O2).  Returns the path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.oracle_ldd.argtypes = [i64, vp, vp, vp, vp, vp]
            lib.oracle_ldd.restype = ctypes.c_int
            lib.oracle_cut_edges.argtypes = [i64, vp, vp, vp]
            lib.oracle_cut_edges.restype = i64
            lib.oracle_certify.argtypes = [i64, vp, vp, vp, vp, vp, ctypes.POINTER(i64)]
            lib.oracle_certify.restype = ctypes.c_int
            _lib = lib
        return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def oracle_ldd(row_ptr, col, delta):
    """(center, dist) int32 arrays: argmin_u dist(u,v) - delta_u, ties to smaller u."""
    rp, prp = _c(row_ptr, np.int32)
    cl, pcl = _c(col, np.int32)
    dl, pdl = _c(delta, np.float64)
    n = rp.shape[0] - 1
    center = np.empty(n, dtype=np.int32)
    dist = np.empty(n, dtype=np.int32)
    rc = _load().oracle_ldd(n, prp, pcl, pdl, center.ctypes.data, dist.ctypes.data)
    if rc == -1:
        raise ValueError("shifts must be finite and >= 0")
    if rc != 0:
        raise MemoryError("oracle_ldd allocation failed")
    return center, dist


def oracle_ldd_ranked(row_ptr, col, levels, perm):
    """(center, dist) of the permutation variant: v joins the u minimising
    (dist(u, v) - levels[u], perm[u]).  Section 4 notes the fractional part of
    a shift only orders vertices inside an integer level, so the shifts
    levels[u] + (n - perm[u]) / (n + 1) -- whose fractional parts fall in
    perm order -- give the same assignment; the call checks that FP64 kept
    that order (floor and strict order inside every level) before using them."""
    lv = np.ascontiguousarray(levels, dtype=np.int64)
    pm = np.ascontiguousarray(perm, dtype=np.int64)
    n = lv.shape[0]
    if n and (lv.min() < 0 or not np.array_equal(np.sort(pm), np.arange(n))):
        raise ValueError("levels must be >= 0 and perm a permutation of 0 .. n-1")
    delta = lv.astype(np.float64) + (n - pm).astype(np.float64) / (n + 1)
    if n:
        by = np.lexsort((pm, lv))  # level ascending, position ascending
        same = lv[by][1:] == lv[by][:-1]
        if (not np.array_equal(np.floor(delta), lv.astype(np.float64))
                or not np.all(delta[by][1:][same] < delta[by][:-1][same])):
            raise ValueError("levels too large for an exact FP64 stand-in")
    return oracle_ldd(row_ptr, col, delta)


def oracle_cut_edges(row_ptr, col, center) -> int:
    rp, prp = _c(row_ptr, np.int32)
    cl, pcl = _c(col, np.int32)
    ce, pce = _c(center, np.int32)
    return int(_load().oracle_cut_edges(rp.shape[0] - 1, prp, pcl, pce))


def oracle_certify(row_ptr, col, delta, center, dist):
    """(code, bad_vertex); code 0 means (center, dist) is the exact optimum."""
    rp, prp = _c(row_ptr, np.int32)
    cl, pcl = _c(col, np.int32)
    dl, pdl = _c(delta, np.float64)
    ce, pce = _c(center, np.int32)
    di, pdi = _c(dist, np.int32)
    bad = ctypes.c_int64(-1)
    code = _load().oracle_certify(rp.shape[0] - 1, prp, pcl, pdl, pce, pdi, ctypes.byref(bad))
    return int(code), int(bad.value)


def oracle_block_decompose(row_ptr, col, shifts_list):
    """Block decomposition by repeated low-diameter decomposition.

    Section 1 (related work) observes that Linial and Saks' block
    decomposition -- O(log n) blocks whose connected pieces have diameter
    O(log n) -- follows from running a (1/2, O(log n)) decomposition again and
    again on the edges that are not yet in a block, since each run leaves at
    most half of them (in expectation; Corollary 3.5 gives 1 - e^-beta).

    The steps, in that order: G_0 = G.  While G_i has an arc and a shift
    vector is left: decompose G_i = (V, E_i) with shifts_list[i]
    (``oracle_ldd``); the arcs of E_i whose two ends share a piece form block
    i; the others, in their original order, are E_{i+1}.

    Returns (centers, dists, arc_block, remaining):
      centers[i], dists[i]  int32[n]: iteration i's decomposition of G_i;
      arc_block             int32[nnz]: the block of every arc of the input
                            CSR, -1 for arcs still cut after the last
                            iteration;
      remaining             list of ints: remaining[i] = the undirected edges
                            of G_i ({v, w} with v < w; the input's self-loops
                            are not counted and join block 0), for i = 0 ..
                            blocks, where blocks = len(centers).
    """
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int64)
    n = rp.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    alive = np.arange(cl.shape[0], dtype=np.int64)  # input arc ids of E_i
    arc_block = np.full(cl.shape[0], -1, dtype=np.int32)
    cur_rp, cur_col = rp, cl
    remaining = [int((src < cl).sum())]
    centers, dists = [], []
    for i, sh in enumerate(shifts_list):
        if alive.shape[0] == 0:
            break
        c, d = oracle_ldd(cur_rp, cur_col, sh)
        inside = c[src[alive]] == c[cl[alive]]
        arc_block[alive[inside]] = i
        alive = alive[~inside]
        counts = np.bincount(src[alive], minlength=n)
        cur_rp = np.concatenate(([0], np.cumsum(counts)))
        cur_col = cl[alive]
        remaining.append(int((src[alive] < cl[alive]).sum()))
        centers.append(c)
        dists.append(d)
    return centers, dists, arc_block, remaining
