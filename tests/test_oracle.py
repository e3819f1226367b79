"""Pins of the CPU oracle to facts outside itself (CPU only).

* hand-derived worked examples of Eq. (1) / Algorithm 2 (tests/golden);
* the definition written out literally (all-pairs BFS + exact rational argmin),
  exhaustively on every graph with up to 5 vertices and on random graphs;
* the O(m) optimality certificate (Lemma 3.1 predecessor + non-improvability)
  on mid-size graphs, and its rejection of perturbed answers;
* limits: delta_max < 1 gives singletons; one dominant shift per component
  gives scipy's BFS distances; equal shifts give singletons;
* Lemma 3.2 (E[delta_max] = H_n / beta, radius <= floor(delta_max)),
  Lemma 3.4 / Corollary 3.5 (mean cut fraction <= 1 - exp(-beta)) and the
  trend of Figure 1, averaged over seeds;
* mutants of the oracle (a flipped tie-break, a dropped fraction, a wrong
  edge length, ...) must each fail at least one of these pins.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import ldd_gen as gen
import oracle
from oracle.brute import brute_cut_edges, brute_ldd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.txt")


def load_golden():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "case":
            cur = {"name": rest}
            cases.append(cur)
        elif key == "n":
            cur["n"] = int(rest)
        elif key == "edges":
            cur["edges"] = [] if rest == "-" else [tuple(map(int, e.split("-"))) for e in rest.split()]
        elif key == "shifts":
            cur["shifts"] = np.array([float(x) for x in rest.split()])
        elif key in ("center", "dist"):
            cur[key] = [int(x) for x in rest.split()]
        elif key == "cut":
            cur["cut"] = int(rest)
    return cases


GOLDEN_CASES = load_golden()


def _graph(case):
    return gen.from_edges(case["n"], case["edges"], case["name"])


@pytest.mark.parametrize("case", GOLDEN_CASES, ids=[c["name"] for c in GOLDEN_CASES])
def test_golden_worked_examples(case):
    G = _graph(case)
    c, d = oracle.oracle_ldd(G.row_ptr, G.col, case["shifts"])
    assert list(c) == case["center"] and list(d) == case["dist"]
    assert oracle.oracle_cut_edges(G.row_ptr, G.col, c) == case["cut"]
    # the literal definition agrees as well
    bc, bd = brute_ldd(G.row_ptr, G.col, case["shifts"])
    assert bc == case["center"] and bd == case["dist"]
    assert brute_cut_edges(G.row_ptr, G.col, bc) == case["cut"]


def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield [p for i, p in enumerate(pairs) if mask >> i & 1]


def test_exhaustive_small_graphs_vs_definition():
    rng = np.random.default_rng(2024)
    checked = 0
    for n in range(1, 6):
        for edges in _all_graphs(n):
            G = gen.from_edges(n, edges)
            for kind in range(3):
                beta = float(rng.choice([0.2, 0.7, 2.0]))
                d = rng.exponential(1.0 / beta, n)
                if kind == 1:
                    d = np.floor(d)               # fractions all 0: ties by id
                elif kind == 2:
                    d = np.round(d * 2) / 2       # many exact ties in value
                c, di = oracle.oracle_ldd(G.row_ptr, G.col, d)
                bc, bd = brute_ldd(G.row_ptr, G.col, d)
                assert list(c) == bc and list(di) == bd, (n, edges, d)
                checked += 1
    assert checked > 3000


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_vs_definition(seed):
    rng = np.random.default_rng(seed)
    for _ in range(25):
        n = int(rng.integers(2, 13))
        G = gen.random_graph(n, float(rng.uniform(0.05, 0.6)), int(rng.integers(1 << 30)))
        beta = float(rng.choice([0.05, 0.3, 1.0, 4.0]))
        d = gen.shifts(n, beta, int(rng.integers(1 << 30)))
        c, di = oracle.oracle_ldd(G.row_ptr, G.col, d)
        bc, bd = brute_ldd(G.row_ptr, G.col, d)
        assert list(c) == bc and list(di) == bd
        assert oracle.oracle_cut_edges(G.row_ptr, G.col, c) == brute_cut_edges(G.row_ptr, G.col, bc)


@pytest.mark.parametrize("G,beta", [(gen.grid2d(64, 64), 0.1), (gen.grid3d(12, 12, 12), 0.05),
                                    (gen.rmat(12), 0.1), (gen.rgg(3000, 3), 0.2)],
                         ids=["grid2d", "grid3d", "rmat12", "rgg"])
def test_certificate_holds_and_rejects_perturbations(G, beta):
    d = gen.shifts(G.n, beta, 17)
    c, di = oracle.oracle_ldd(G.row_ptr, G.col, d)
    assert oracle.oracle_certify(G.row_ptr, G.col, d, c, di) == (0, -1)
    src = np.repeat(np.arange(G.n), np.diff(G.row_ptr))
    boundary = np.flatnonzero(c[src] != c[G.col])  # arcs between two pieces
    for e in np.random.default_rng(5).choice(boundary, min(40, boundary.size), replace=False):
        v, w = int(src[e]), int(G.col[e])
        c2, d2 = c.copy(), di.copy()
        c2[v], d2[v] = c[w], di[w] + 1             # move v into w's piece
        assert oracle.oracle_certify(G.row_ptr, G.col, d, c2, d2)[0] != 0
    d3 = di.copy()
    d3[int(np.argmax(di))] += 1                    # a distance one too large
    assert oracle.oracle_certify(G.row_ptr, G.col, d, c, d3)[0] != 0
    c4 = c.copy()
    c4[int(np.argmax(di))] = int(np.argmax(di))    # a non-center claiming itself
    assert oracle.oracle_certify(G.row_ptr, G.col, d, c4, di)[0] != 0


def test_large_beta_gives_singletons():
    G = gen.rmat(12)
    d = gen.shifts(G.n, 1e4, 3)
    assert d.max() < 1.0
    c, di = oracle.oracle_ldd(G.row_ptr, G.col, d)
    assert np.array_equal(c, np.arange(G.n)) and not di.any()
    assert oracle.oracle_cut_edges(G.row_ptr, G.col, c) == G.m


def test_equal_shifts_give_singletons():
    G = gen.grid2d(20, 30)
    c, di = oracle.oracle_ldd(G.row_ptr, G.col, np.full(G.n, 3.5))
    assert np.array_equal(c, np.arange(G.n))


def test_dominant_shift_gives_bfs_distances():
    """beta -> 0 limit: a shift larger than every distance makes its vertex the
    center of its whole component at textbook BFS distance (scipy csgraph)."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg

    G = gen.rmat(11)
    A = sp.csr_matrix((np.ones(G.nnz), G.col, G.row_ptr), shape=(G.n, G.n))
    ncomp, lab = cg.connected_components(A, directed=False)
    d = gen.shifts(G.n, 1.0, 9)
    roots = {}
    for v in range(G.n):
        roots.setdefault(lab[v], v)
    for r in roots.values():
        d[r] = 1e6
    c, di = oracle.oracle_ldd(G.row_ptr, G.col, d)
    src = np.array(sorted(roots.values()))
    bfs = cg.shortest_path(A, unweighted=True, directed=False, indices=src)
    for i, r in enumerate(src):
        members = lab == lab[r]
        assert (c[members] == r).all()
        assert np.array_equal(di[members], bfs[i][members].astype(np.int32))


def test_radius_bound_lemma_3_2():
    """dist(center, v) <= delta_center - delta_v <= delta_max (proof of Theorem 1.2)."""
    from fractions import Fraction

    for G, beta, seed in [(gen.grid2d(80, 80), 0.05, 1), (gen.rmat(12), 0.2, 2)]:
        d = gen.shifts(G.n, beta, seed)
        c, di = oracle.oracle_ldd(G.row_ptr, G.col, d)
        assert di.max() <= math.floor(d.max())
        for v in np.random.default_rng(seed).choice(G.n, 500, replace=False):
            assert Fraction(int(di[v])) <= Fraction(float(d[c[v]])) - Fraction(float(d[v]))


def test_expected_max_shift_lemma_3_2():
    """E[max_u delta_u] = H_n / beta (Lemma 3.2), for the shift generator."""
    n, beta, seeds = 1000, 0.1, 3000
    m = np.array([gen.shifts(n, beta, s).max() for s in range(seeds)])
    Hn = sum(1.0 / i for i in range(1, n + 1))
    se = m.std(ddof=1) / math.sqrt(seeds)
    assert abs(m.mean() - Hn / beta) < 5 * se, (m.mean(), Hn / beta, se)


@pytest.mark.parametrize("beta", [0.02, 0.1, 0.5])
def test_cut_fraction_bound_lemma_3_4(beta):
    """P[edge cut] <= 1 - exp(-beta) for every edge (Lemma 3.4 with c = 1,
    Corollary 3.5); the mean over seeds must respect it up to sampling error."""
    G = gen.grid2d(64, 64)
    fr = []
    for s in range(150):
        d = gen.shifts(G.n, beta, 1000 + s)
        c, _ = oracle.oracle_ldd(G.row_ptr, G.col, d)
        fr.append(oracle.oracle_cut_edges(G.row_ptr, G.col, c) / G.m)
    fr = np.array(fr)
    bound = 1.0 - math.exp(-beta)
    assert fr.mean() <= bound + 4 * fr.std(ddof=1) / math.sqrt(len(fr)), (fr.mean(), bound)
    assert fr.mean() > 0.0


def test_figure1_trend():
    """Figure 1: lower beta gives fewer, larger pieces and fewer cut edges."""
    G = gen.grid2d(100, 100)
    rows = []
    for beta in [0.5, 0.2, 0.1, 0.05, 0.02]:
        pieces, cut, rad = [], [], []
        for s in range(12):
            d = gen.shifts(G.n, beta, 77 + s)
            c, di = oracle.oracle_ldd(G.row_ptr, G.col, d)
            pieces.append(len(np.unique(c)))
            cut.append(oracle.oracle_cut_edges(G.row_ptr, G.col, c))
            rad.append(di.max())
        rows.append((np.mean(pieces), np.mean(cut), np.mean(rad)))
    for a, b in zip(rows, rows[1:]):
        assert b[0] < a[0] and b[1] < a[1] and b[2] > a[2], rows


# ----------------------------------------------------------------- mutation tests
MUTANTS = {
    "tie_break_reversed": ("return C1 < C2;", "return C1 > C2;"),
    "fraction_reversed": ("if (F1 != F2) return F1 > F2;", "if (F1 != F2) return F1 < F2;"),
    "fraction_dropped": ("if (F1 != F2) return F1 > F2;", ""),
    "edge_length_two": ("const int64_t I1 = s.I[v] + 1;", "const int64_t I1 = s.I[v] + 2;"),
    "dist_not_counted": ("s.D[w] = s.D[v] + 1;", "s.D[w] = s.D[v];"),
    "shift_sign_flipped": ("s.I[u] = -fl[u];", "s.I[u] = fl[u];"),
    "fraction_is_whole_shift": ("fr[u] = delta[u] - a;", "fr[u] = delta[u];"),
    "heap_wrong_child": ("if (l + 1 < s->size && vless(s, s->heap[l + 1], s->heap[l])) b = l + 1;",
                         "if (l + 1 < s->size && vless(s, s->heap[l], s->heap[l + 1])) b = l + 1;"),
}


def _build_mutant(tmp, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ldd_oracle.c")).read()
    assert old in src, f"mutant {name}: pattern not found"
    path = os.path.join(tmp, f"{name}.c")
    open(path, "w").write(src.replace(old, new))
    so = os.path.join(tmp, f"{name}.so")
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-std=c11", path, "-o", so, "-lm"])
    lib = ctypes.CDLL(so)
    lib.oracle_ldd.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5
    return lib


def _mutant_ldd(lib, G, d):
    n = G.n
    c = np.empty(n, np.int32)
    di = np.empty(n, np.int32)
    rp, col, dd = (np.ascontiguousarray(G.row_ptr), np.ascontiguousarray(G.col),
                   np.ascontiguousarray(d, dtype=np.float64))
    lib.oracle_ldd(n, rp.ctypes.data, col.ctypes.data, dd.ctypes.data, c.ctypes.data, di.ctypes.data)
    return [int(x) for x in c], [int(x) for x in di]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc needed to build mutants")
def test_mutants_are_caught():
    tmp = tempfile.mkdtemp()
    rng = np.random.default_rng(99)
    pool = [(_graph(c), c["shifts"]) for c in GOLDEN_CASES]
    for _ in range(60):
        n = int(rng.integers(3, 11))
        G = gen.random_graph(n, float(rng.uniform(0.2, 0.6)), int(rng.integers(1 << 30)))
        d = rng.exponential(2.0, n)
        pool.append((G, d))
        pool.append((G, np.floor(d)))
    try:
        for name, (old, new) in MUTANTS.items():
            lib = _build_mutant(tmp, name, old, new)
            caught = any(_mutant_ldd(lib, G, d) != brute_ldd(G.row_ptr, G.col, d) for G, d in pool)
            assert caught, f"mutant {name} passed every pin"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
