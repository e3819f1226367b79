"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds none of the decomposition's arithmetic.  It makes the two
inputs of the method (Miller, Peng, Xu 2013): a symmetric int32 CSR graph
(Definition 1.1: undirected, unweighted) and the shifts delta_u ~ Exp(beta)
of Algorithm 2 step 1, drawn in FP64 from Philox4x32-10 (the counter layout
is documented in ``gen.c``).  Everything is compiled C (``gen.c``), loaded
with ctypes; the shared object is built on first use with gcc.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libldd_gen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libldd_gen.so (gcc, OpenMP).  Returns the path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, u64, u32, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
        vp = ctypes.c_void_p
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.ldd_philox4x32_10.argtypes = [vp, vp, vp]
        lib.ldd_philox_stream.argtypes = [u64, u64, i64, u32, u32, vp]
        lib.ldd_gen_uniforms.argtypes = [i64, u64, vp]
        lib.ldd_gen_shifts.argtypes = [i64, dbl, u64, vp]
        lib.ldd_grid2d_nnz.argtypes = [i64, i64]
        lib.ldd_grid2d_nnz.restype = i64
        lib.ldd_gen_grid2d.argtypes = [i64, i64, vp, vp]
        lib.ldd_grid3d_nnz.argtypes = [i64, i64, i64]
        lib.ldd_grid3d_nnz.restype = i64
        lib.ldd_gen_grid3d.argtypes = [i64, i64, i64, vp, vp]
        lib.ldd_gen_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64, pp, pp]
        lib.ldd_gen_rmat.restype = i64
        lib.ldd_gen_rgg.argtypes = [i64, dbl, u64, pp, pp]
        lib.ldd_gen_rgg.restype = i64
        lib.ldd_gen_free.argtypes = [vp]
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------- random numbers
def philox4x32_10(counter, key) -> np.ndarray:
    """One Philox4x32-10 block: 4 uint32 words for a 4-word counter, 2-word key."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().ldd_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_stream(seed: int, first: int, count: int, w2: int = 0, w3: int = 0) -> np.ndarray:
    """Words for counters (i_lo, i_hi, w2, w3), i = first..first+count-1; shape (count, 4)."""
    out = np.zeros((count, 4), dtype=np.uint32)
    _load().ldd_philox_stream(seed, first, count, w2, w3, _ptr(out))
    return out


def uniforms(n: int, seed: int) -> np.ndarray:
    """U_u in (0, 1], 53-bit, from the shift counter layout."""
    out = np.empty(n, dtype=np.float64)
    _load().ldd_gen_uniforms(n, seed, _ptr(out))
    return out


def shifts(n: int, beta: float, seed: int) -> np.ndarray:
    """delta_u = -ln(U_u) / beta, FP64 (Algorithm 2 step 1; Section 2 CDF)."""
    out = np.empty(n, dtype=np.float64)
    _load().ldd_gen_shifts(n, float(beta), seed, _ptr(out))
    return out


def permutation(n: int, seed: int) -> np.ndarray:
    """A uniform random permutation of 0 .. n-1 as positions: perm[u] = the
    position of u after sorting the vertices by a 64-bit Philox4x32-10 word
    (key seed, counter (u, 0, 5, 0); ties by u)."""
    w = philox_stream(seed, 0, n, 5, 0).astype(np.uint64)
    key = (w[:, 0] << np.uint64(32)) | w[:, 1]
    order = np.lexsort((np.arange(n), key))
    perm = np.empty(n, dtype=np.int32)
    perm[order] = np.arange(n, dtype=np.int32)
    return perm


def ranked_inputs(n: int, beta: float, seed: int):
    """Inputs of the permutation variant: levels = floor of the Exp(beta)
    shifts of ``shifts(n, beta, seed)`` and an independent random permutation
    (seed + 1) as the tie-break."""
    levels = np.floor(shifts(n, beta, seed)).astype(np.int32)
    return levels, permutation(n, seed + 1)


# ---------------------------------------------------------------- graphs
@dataclass
class CSR:
    """Symmetric int32 CSR.  ``m`` counts undirected edges (nnz // 2)."""
    name: str
    row_ptr: np.ndarray
    col: np.ndarray

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def m(self) -> int:
        return self.nnz // 2


def grid2d(nx: int, ny: int) -> CSR:
    lib = _load()
    nnz = lib.ldd_grid2d_nnz(nx, ny) if nx * ny > 0 else 0
    rp = np.zeros(nx * ny + 1, dtype=np.int32)
    col = np.zeros(max(nnz, 0), dtype=np.int32)
    if nx * ny > 0:
        lib.ldd_gen_grid2d(nx, ny, _ptr(rp), _ptr(col))
    return CSR(f"grid2d_{nx}x{ny}", rp, col)


def grid3d(nx: int, ny: int, nz: int) -> CSR:
    lib = _load()
    nnz = lib.ldd_grid3d_nnz(nx, ny, nz) if nx * ny * nz > 0 else 0
    rp = np.zeros(nx * ny * nz + 1, dtype=np.int32)
    col = np.zeros(max(nnz, 0), dtype=np.int32)
    if nx * ny * nz > 0:
        lib.ldd_gen_grid3d(nx, ny, nz, _ptr(rp), _ptr(col))
    return CSR(f"grid3d_{nx}x{ny}x{nz}", rp, col)


def _take(n: int, nnz: int, rp_p, col_p, name: str) -> CSR:
    lib = _load()
    if nnz < 0:
        raise MemoryError(f"{name}: generator failed")
    rp = np.ctypeslib.as_array(ctypes.cast(rp_p, ctypes.POINTER(ctypes.c_int32)), shape=(n + 1,)).copy()
    col = (np.ctypeslib.as_array(ctypes.cast(col_p, ctypes.POINTER(ctypes.c_int32)), shape=(nnz,)).copy()
           if nnz > 0 else np.zeros(0, dtype=np.int32))
    lib.ldd_gen_free(rp_p)
    lib.ldd_gen_free(col_p)
    return CSR(name, rp, col)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 7) -> CSR:
    """R-MAT, symmetrised, self-loops and duplicate arcs removed, rows ascending."""
    rp_p, col_p = ctypes.c_void_p(), ctypes.c_void_p()
    nnz = _load().ldd_gen_rmat(scale, edge_factor, a, b, c, seed, ctypes.byref(rp_p), ctypes.byref(col_p))
    return _take(1 << scale, nnz, rp_p, col_p, f"rmat{scale}_ef{edge_factor}_s{seed}")


def rgg(n: int, seed: int, mean_degree: float = 8.0) -> CSR:
    """Random geometric graph in [0,1)^2 with radius sqrt(mean_degree / (pi n))."""
    radius = math.sqrt(mean_degree / (math.pi * n))
    rp_p, col_p = ctypes.c_void_p(), ctypes.c_void_p()
    nnz = _load().ldd_gen_rgg(n, radius, seed, ctypes.byref(rp_p), ctypes.byref(col_p))
    return _take(n, nnz, rp_p, col_p, f"rgg{n}_s{seed}")


def from_edges(n: int, edges, name: str = "edges") -> CSR:
    """Symmetric CSR from an undirected edge list (self-loops and repeats dropped)."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    rp = np.zeros(n + 1, dtype=np.int32)
    cols = []
    for v in range(n):
        nb = sorted(adj[v])
        cols.extend(nb)
        rp[v + 1] = rp[v] + len(nb)
    return CSR(name, rp, np.asarray(cols, dtype=np.int32))


def random_graph(n: int, p: float, seed: int) -> CSR:
    """Erdos-Renyi G(n, p) from numpy's PCG64 (small test graphs only)."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    return from_edges(n, list(zip(iu[keep].tolist(), ju[keep].tolist())), f"gnp{n}_{p}_{seed}")


# ---------------------------------------------------------------- named workloads
WORKLOADS = {
    # 2D 4-neighbour grid 256x256, beta 0.1, shift seed 1
    "grid2d_256": dict(graph=("grid2d", 256, 256), betas=(0.1,), shift_seed=1),
    # R-MAT scale 22, ef 16, (.57,.19,.19,.05), graph seed 7; beta in {0.02, 0.1, 0.5}
    "rmat22": dict(graph=("rmat", 22, 16, 0.57, 0.19, 0.19, 7), betas=(0.02, 0.1, 0.5), shift_seed=1),
    # 3D 6-neighbour grid 256^3, beta 0.01
    "grid3d_256": dict(graph=("grid3d", 256, 256, 256), betas=(0.01,), shift_seed=1),
    # R-MAT scale 20 with the scale-22 parameters: a quarter-size case whose
    # arrays still exceed the L2 cache, for detailed kernel profiles
    "rmat20": dict(graph=("rmat", 20, 16, 0.57, 0.19, 0.19, 7), betas=(0.02, 0.1, 0.5), shift_seed=1),
}

# Batched workloads (one union decomposition per step):
#  rgg_batch_1024: 1,024 random geometric graphs in the unit square, n uniform
#    on [1,000, 200,000], mean degree 8, beta uniform on [0.02, 0.5), graph and
#    shift seed 11 + i (batch_members).
#  rmat20_seeds_64: 64 shift vectors (seeds 1 .. 64) of one R-MAT scale-20
#    graph (the scale-22 parameters, seed 7) at beta 0.1.
# Serving workload: a Poisson stream (mean 2,000 requests/s for 2 s) over
# resident R-MAT graphs of scales 14..22 (the scale-22 parameters, seed 7) and
# 2D grids 64^2 .. 2048^2; beta from {0.02, 0.05, 0.1, 0.2, 0.5}; each request
# takes one of two pre-drawn shift vectors per (graph, beta), shift seed
# 1000 + 100 graph + 10 beta + seed index; a 120 GB HBM budget.
# Block decomposition by repeated decomposition (Section 1's remark on Linial
# and Saks' blocks): one R-MAT scale-20 graph (scale-22 parameters, seed 7),
# beta 1/2, shift vectors of seeds first_seed .. first_seed + vectors - 1
# (far more than the O(log n) iterations the loop needs).
BLOCK_WORKLOADS = {
    "rmat20_blocks": dict(graph=("rmat", 20, 16, 0.57, 0.19, 0.19, 7), beta=0.5, vectors=48,
                          first_seed=1),
}

SERVE_WORKLOADS = {
    "serve_mix": dict(rmat_scales=tuple(range(14, 23)), grids=(64, 128, 256, 512, 1024, 2048),
                      betas=(0.02, 0.05, 0.1, 0.2, 0.5), seeds=2, rate=2000.0, seconds=2.0,
                      master_seed=21, hbm_budget=120 << 30),
}

BATCH_WORKLOADS = {
    "rgg_batch_1024": dict(kind="rgg", count=1024, n_lo=1000, n_hi=200000, beta_lo=0.02,
                           beta_hi=0.5, master_seed=11),
    "rmat20_seeds_64": dict(kind="seeds", graph=("rmat", 20, 16, 0.57, 0.19, 0.19, 7),
                            copies=64, beta=0.1, first_seed=1),
    # the first 128 graphs of rgg_batch_1024: a profiling case a few GB in size
    "rgg_batch_128": dict(kind="rgg", count=128, n_lo=1000, n_hi=200000, beta_lo=0.02,
                          beta_hi=0.5, master_seed=11),
}


def batch_members(count: int, n_lo: int, n_hi: int, beta_lo: float, beta_hi: float,
                  master_seed: int):
    """Per-member (n, beta, graph_seed, shift_seed) of a batch of random graphs:
    n uniform on [n_lo, n_hi] and beta uniform on [beta_lo, beta_hi), both
    from Philox4x32-10 with key master_seed and counter (i, 0, 3, 0) (words 0-1
    give n, words 2-3 beta, each as a 53-bit uniform); graph seed and shift
    seed are master_seed + i."""
    w = philox_stream(master_seed, 0, count, 3, 0).astype(np.uint64)
    u1 = ((w[:, 0] << np.uint64(32)) | w[:, 1]) >> np.uint64(11)
    u2 = ((w[:, 2] << np.uint64(32)) | w[:, 3]) >> np.uint64(11)
    u1 = u1.astype(np.float64) * 2.0 ** -53
    u2 = u2.astype(np.float64) * 2.0 ** -53
    span = n_hi - n_lo + 1
    out = []
    for i in range(count):
        n = n_lo + min(int(u1[i] * span), span - 1)
        beta = beta_lo + (beta_hi - beta_lo) * float(u2[i])
        out.append((n, beta, master_seed + i, master_seed + i))
    return out


def rgg_batch(count: int = 1024, n_lo: int = 1000, n_hi: int = 200000, beta_lo: float = 0.02,
              beta_hi: float = 0.5, master_seed: int = 11, mean_degree: float = 8.0):
    """A batch of random geometric graphs with their own beta and shifts:
    list of (CSR, beta, shifts)."""
    out = []
    for n, beta, gseed, sseed in batch_members(count, n_lo, n_hi, beta_lo, beta_hi, master_seed):
        G = rgg(n, gseed, mean_degree)
        out.append((G, beta, shifts(n, beta, sseed)))
    return out


def serve_requests(n_graphs: int, n_betas: int, n_seeds: int, rate: float, seconds: float,
                   master_seed: int):
    """A Poisson stream of requests: (arrival_s, graph index, beta index, seed
    index) in arrival order.  Request i draws Philox4x32-10 with key
    master_seed and counter (i, 0, 4, 0): words 0-1 give the exponential
    inter-arrival gap -ln(U)/rate (U a 53-bit uniform on (0, 1]), words 2 and 3
    the graph and the (beta, seed) pair by modulo."""
    out = []
    t = 0.0
    i = 0
    chunk = 4096
    while True:
        w = philox_stream(master_seed, i, chunk, 4, 0).astype(np.uint64)
        u = (((w[:, 0] << np.uint64(32)) | w[:, 1]) >> np.uint64(11)).astype(np.float64)
        u = (u + 1.0) * 2.0 ** -53
        for j in range(chunk):
            t += -math.log(u[j]) / rate
            if t >= seconds:
                return out
            gi = int(w[j, 2] % np.uint64(n_graphs))
            pair = int(w[j, 3] % np.uint64(n_betas * n_seeds))
            out.append((t, gi, pair // n_seeds, pair % n_seeds))
        i += chunk


def make_graph(spec) -> CSR:
    kind = spec[0]
    if kind == "grid2d":
        return grid2d(*spec[1:])
    if kind == "grid3d":
        return grid3d(*spec[1:])
    if kind == "rmat":
        return rmat(*spec[1:])
    if kind == "rgg":
        return rgg(*spec[1:])
    raise ValueError(kind)
