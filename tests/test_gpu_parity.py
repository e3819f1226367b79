"""Bit-exact parity of the CUDA path (through the C ABI) against the CPU oracle.

The tolerance is zero: the decomposition is integer and exact (center id and
hop distance per vertex), and the cut count is an integer.  Sizes span
several BFS spans (4096 arcs), several sort tiles (4096 keys) and ragged
tails; edge cases cover empty graphs, isolated vertices, hubs wider than one
CTA span, exact ties and the limits beta -> 0 and beta -> infinity.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import ldd_gen as gen
import oracle
from tests.gpu_util import assert_parity, run_gpu

pytestmark = pytest.mark.gpu


def _cases():
    yield "grid2d_37x53", gen.grid2d(37, 53), 0.1, 1
    yield "grid2d_1x1000_path", gen.grid2d(1, 1000), 0.05, 2
    yield "grid2d_64x64_b002", gen.grid2d(64, 64), 0.02, 3
    yield "grid3d_9x11x13", gen.grid3d(9, 11, 13), 0.2, 4
    yield "rmat10", gen.rmat(10), 0.1, 5
    yield "rmat12_b05", gen.rmat(12), 0.5, 6
    yield "rmat14_b002", gen.rmat(14), 0.02, 7
    yield "rmat17_b01", gen.rmat(17), 0.1, 13  # more vertices than the cut's hot table
    yield "rgg5000", gen.rgg(5000, 11), 0.1, 8
    yield "gnp300_dense", gen.random_graph(300, 0.3, 9), 0.3, 9
    yield "gnp2000_sparse", gen.random_graph(2000, 0.001, 10), 0.1, 10
    hub = [(0, i) for i in range(1, 12001)] + [(i, i + 1) for i in range(1, 12000, 2)]
    yield "star12000", gen.from_edges(12001, hub, "star12000"), 0.2, 11
    yield "complete60", gen.from_edges(60, [(i, j) for i in range(60) for j in range(i)], "k60"), 1.0, 12


@pytest.mark.parametrize("name,G,beta,seed", list(_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_parity_small(ldd, cuda, name, G, beta, seed):
    shifts = gen.shifts(G.n, beta, seed)
    assert_parity(ldd, G, shifts, beta)


@pytest.mark.parametrize("host", [False, True], ids=["device_buffers", "host_buffers"])
def test_host_and_device_buffers(ldd, cuda, host):
    G = gen.rmat(11)
    shifts = gen.shifts(G.n, 0.1, 21)
    assert_parity(ldd, G, shifts, 0.1, host=host)


def test_integer_shifts_ties(ldd, cuda):
    """floor() of the shifts: every fraction is 0, so all same-level ties go to the smaller id."""
    G = gen.grid2d(50, 41)
    shifts = np.floor(gen.shifts(G.n, 0.05, 31))
    assert_parity(ldd, G, shifts, 0.05)


def test_all_equal_shifts_are_singletons(ldd, cuda):
    """dist(v,v) - d = -d beats 1 - d: every vertex is its own piece (Eq. (1))."""
    G = gen.grid2d(30, 30)
    shifts = np.full(G.n, 7.25)
    center, dist, cut, _ = assert_parity(ldd, G, shifts, 0.1)
    assert np.array_equal(center, np.arange(G.n)) and not dist.any() and cut == G.m


def test_large_beta_singletons(ldd, cuda):
    """delta_max < 1: no shift can pay for one hop, every vertex is a singleton."""
    G = gen.rmat(12)
    shifts = gen.shifts(G.n, 1e4, 41)
    assert shifts.max() < 1.0
    center, dist, cut, _ = assert_parity(ldd, G, shifts, 1e4)
    assert np.array_equal(center, np.arange(G.n)) and cut == G.m


def test_small_beta_one_piece_per_component(ldd, cuda):
    """One shift far above every distance: its vertex takes its whole component
    and dist is the BFS distance (the beta -> 0 limit)."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg

    G = gen.rmat(11)
    shifts = gen.shifts(G.n, 1.0, 51)
    ncomp, labels = cg.connected_components(sp.csr_matrix(
        (np.ones(G.nnz), G.col, G.row_ptr), shape=(G.n, G.n)), directed=False)
    big = {}
    for v in range(G.n):
        big.setdefault(labels[v], v)
    for lab, v in big.items():
        shifts[v] = 1e6
    center, dist, _, _ = assert_parity(ldd, G, shifts, 1e-5)
    for lab, v in big.items():
        assert (center[labels == lab] == v).all()


def test_bucket_table_regrowth(ldd, cuda):
    """A tiny graph with a tiny beta has floor(delta_max) > n: the start-bucket
    table is regrown and the BFS rerun."""
    G = gen.grid2d(3, 4)
    shifts = gen.shifts(G.n, 0.001, 61)
    assert math.floor(shifts.max()) + 2 > G.n + 2
    assert_parity(ldd, G, shifts, 0.001)


def test_no_edges_and_single_vertex(ldd, cuda):
    G = gen.from_edges(100, [], "empty100")
    center, dist, cut, _ = assert_parity(ldd, G, gen.shifts(100, 0.1, 71), 0.1)
    assert np.array_equal(center, np.arange(100)) and cut == 0
    G1 = gen.from_edges(1, [], "single")
    assert_parity(ldd, G1, gen.shifts(1, 0.1, 72), 0.1)


def test_zero_vertices(ldd, cuda):
    g = ldd.LddGraph(np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32))
    g.decompose(0.1, np.zeros(0), np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.int32))
    assert g.cut_edges(np.zeros(0, dtype=np.int32)) == 0
    g.close()


def test_determinism(ldd, cuda):
    G = gen.rmat(13)
    shifts = gen.shifts(G.n, 0.1, 81)
    runs = [run_gpu(ldd, G, shifts)[:3] for _ in range(4)]
    for c, d, k in runs[1:]:
        assert np.array_equal(c, runs[0][0]) and np.array_equal(d, runs[0][1]) and k == runs[0][2]


def test_repeated_calls_one_graph(ldd, cuda):
    """One graph object, many decompositions with different betas and seeds."""
    import torch

    G = gen.rmat(12)
    g = ldd.LddGraph(G.row_ptr, G.col)
    c = torch.empty(G.n, dtype=torch.int32, device=cuda)
    d = torch.empty(G.n, dtype=torch.int32, device=cuda)
    for i, beta in enumerate([0.02, 0.5, 0.1, 0.002, 3.0]):
        shifts = gen.shifts(G.n, beta, 90 + i)
        g.decompose(beta, torch.from_numpy(shifts).to(cuda), c, d)
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts)
        assert np.array_equal(c.cpu().numpy(), oc) and np.array_equal(d.cpu().numpy(), od)
        assert g.cut_edges(c) == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    g.close()


@pytest.mark.parametrize("bad,status", [(float("nan"), -1), (-1.0, -1), (2.0 ** 31, -3),
                                        (float("inf"), -3)])
def test_bad_shift_rejected(ldd, cuda, bad, status):
    G = gen.grid2d(20, 20)
    shifts = gen.shifts(G.n, 0.1, 5)
    shifts[137] = bad
    g = ldd.LddGraph(G.row_ptr, G.col)
    with pytest.raises(ldd.LddError) as e:
        g.decompose(0.1, shifts, np.empty(G.n, np.int32), np.empty(G.n, np.int32))
    assert e.value.status == status
    # the graph stays usable
    good = gen.shifts(G.n, 0.1, 6)
    c, d = np.empty(G.n, np.int32), np.empty(G.n, np.int32)
    g.decompose(0.1, good, c, d)
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, good)
    assert np.array_equal(c, oc) and np.array_equal(d, od)
    g.close()


@pytest.mark.parametrize("beta", [0.0, -0.5, float("nan"), float("inf")])
def test_bad_beta_rejected(ldd, cuda, beta):
    G = gen.grid2d(5, 5)
    g = ldd.LddGraph(G.row_ptr, G.col)
    with pytest.raises(ldd.LddError) as e:
        g.decompose(beta, gen.shifts(G.n, 0.1, 1), np.empty(G.n, np.int32), np.empty(G.n, np.int32))
    assert e.value.status == ldd.LDD_ERR_ARG
    g.close()


def test_invalid_graphs_rejected(ldd, cuda):
    rp = np.array([0, 1, 1], dtype=np.int32)  # arc 0->1 without 1->0
    col = np.array([1], dtype=np.int32)
    with pytest.raises(ldd.LddError) as e:
        ldd.LddGraph(rp, col, validate=True)
    assert e.value.status == ldd.LDD_ERR_GRAPH
    rp = np.array([0, 1, 2], dtype=np.int32)
    col = np.array([1, 5], dtype=np.int32)  # out of range
    with pytest.raises(ldd.LddError) as e:
        ldd.LddGraph(rp, col, validate=True)
    assert e.value.status == ldd.LDD_ERR_GRAPH
    with pytest.raises(ldd.LddError) as e:
        ldd.ldd_create_graph(2, 2, np.array([0, 2, 1], dtype=np.int32), np.array([1, 0], dtype=np.int32), 1)
    assert e.value.status == ldd.LDD_ERR_GRAPH


def test_stream_and_timing(ldd, cuda):
    import torch

    G = gen.rmat(12)
    shifts = gen.shifts(G.n, 0.1, 3)
    g = ldd.LddGraph(G.row_ptr, G.col)
    s = torch.cuda.Stream()
    g.set_stream(s)
    g.set_timing(True)
    c = torch.empty(G.n, dtype=torch.int32, device=cuda)
    d = torch.empty(G.n, dtype=torch.int32, device=cuda)
    with torch.cuda.stream(s):
        sh = torch.from_numpy(shifts).to(cuda)
    s.synchronize()
    g.decompose(0.1, sh, c, d)
    st = g.stats()
    assert st["ms_bfs"] >= 0 and st["ms_total"] >= st["ms_bfs"] and st["launches"] > 0
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts)
    assert np.array_equal(c.cpu().numpy(), oc)
    g.close()


def _disjoint_union(parts, name):
    edges, off = [], 0
    for n_i, e_i in parts:
        edges += [(u + off, v + off) for u, v in e_i]
        off += n_i
    return gen.from_edges(off, edges, name)


def test_component_size_boundaries(ldd, cuda):
    """Components of 2..32 vertices go to the warp solver, larger ones to the
    BFS rounds: paths, cliques and stars on both sides of the 32 boundary."""
    def path(k):
        return k, [(i, i + 1) for i in range(k - 1)]

    def clique(k):
        return k, [(i, j) for i in range(k) for j in range(i)]

    def star(k):
        return k, [(0, i) for i in range(1, k)]

    parts = [path(1), path(2), path(3), path(31), path(32), path(33), clique(32), clique(33),
             star(32), star(33), path(200), (7, [])]
    G = _disjoint_union(parts * 3, "mixed_components")
    for seed, beta in [(1, 0.05), (2, 0.3), (3, 2.0)]:
        shifts = gen.shifts(G.n, beta, seed)
        _, _, _, st = assert_parity(ldd, G, shifts, beta)
    # small: 2, 3, 31, 32 (path), 32 (clique), 32 (star) per copy
    assert st["small_components"] == 3 * 6
    assert st["n_active"] == 3 * (33 + 33 + 33 + 200)
    shifts = np.floor(gen.shifts(G.n, 0.2, 4))  # exact ties inside the small components
    assert_parity(ldd, G, shifts, 0.2)


def test_many_small_components_and_a_giant(ldd, cuda):
    """R-MAT plus thousands of tiny components: the structure that makes the
    delayed-start rounds run to floor(delta_max) without the component split."""
    rng = np.random.default_rng(5)
    base = gen.rmat(13)
    parts = [(base.n, [(v, int(w)) for v in range(base.n)
                       for w in base.col[base.row_ptr[v]:base.row_ptr[v + 1]] if v < w])]
    for _ in range(3000):
        k = int(rng.integers(2, 9))
        parts.append((k, [(i, int(rng.integers(0, i))) for i in range(1, k)]))
    G = _disjoint_union(parts, "rmat13_plus_trees")
    for beta in (0.02, 0.5):
        _, _, _, st = assert_parity(ldd, G, gen.shifts(G.n, beta, 77), beta)
        assert st["small_components"] >= 3000


def test_component_labels_deep_trees(ldd, cuda):
    """Long paths and a broom give deep union-find trees; the component split
    must match scipy's labelling (reported counts) and the oracle."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg

    k = 60000
    edges = [(i, i + 1) for i in range(k - 1)]                     # a long path
    edges += [(k + i, k + i + 1) for i in range(40)]               # a 41-vertex path
    edges += [(k + 41 + i, k + 41 + i + 1) for i in range(20)]     # a 21-vertex path
    edges += [(k + 62, k + 63 + i) for i in range(500)]            # a star (broom head)
    G = gen.from_edges(k + 563 + 5, edges, "paths_and_broom")
    A = sp.csr_matrix((np.ones(G.nnz), G.col, G.row_ptr), shape=(G.n, G.n))
    _, lab = cg.connected_components(A, directed=False)
    sz = np.bincount(lab)
    for beta, seed in [(0.05, 1), (0.01, 2)]:
        _, _, _, st = assert_parity(ldd, G, gen.shifts(G.n, beta, seed), beta)
        assert st["small_components"] == int(((sz >= 2) & (sz <= 32)).sum())
        assert st["n_active"] == int(sz[lab][sz[lab] > 32].size)


@pytest.mark.parametrize("seed", [1, 2])
def test_component_labels_no_giant(ldd, cuda, seed):
    """Many mid-size components and no giant one (random trees of 20..80
    vertices, each in a random vertex order, plus isolated vertices): the
    sampled common root is an ordinary component, and every other one must
    still be joined arc by arc.  Counts match scipy's labelling, labels the
    oracle."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg

    rng = np.random.default_rng(seed)
    n = 30000
    perm = rng.permutation(n)
    edges, at = [], 0
    while at < n - 100:
        size = int(rng.integers(20, 81))
        ids = perm[at:at + size]
        for i in range(1, size):  # a random tree: vertex i hangs off an earlier one
            edges.append((int(ids[i]), int(ids[int(rng.integers(0, i))])))
        at += size
    G = gen.from_edges(n, edges, f"forest{seed}")
    A = sp.csr_matrix((np.ones(G.nnz), G.col, G.row_ptr), shape=(G.n, G.n))
    _, lab = cg.connected_components(A, directed=False)
    sz = np.bincount(lab)
    _, _, _, st = assert_parity(ldd, G, gen.shifts(G.n, 0.1, seed), 0.1)
    assert st["small_components"] == int(((sz >= 2) & (sz <= 32)).sum())
    assert st["n_active"] == int(sz[lab][sz[lab] > 32].size)


@pytest.mark.parametrize("kind,exact", [("equal_codes_unequal_fractions", 1), ("tiny_shifts", 1),
                                        ("half_ties", 1), ("short_equal_runs", 0)])
def test_fraction_rank_exact_fallback(ldd, cuda, kind, exact):
    """Fractions crowded into one bucket (equal in their top 32 bits but not
    below, all below 2^-32, or only two distinct values) fill one bucket beyond its
    cap and force the exact 64-bit rank path; short runs of exactly equal
    fractions stay on the bucket path, their ties resolved by id."""
    rng = np.random.default_rng(3)
    G = gen.grid2d(40, 30)
    if kind == "equal_codes_unequal_fractions":
        shifts = rng.integers(0, 40, G.n) + 0.5 + rng.integers(0, 1 << 12, G.n) * 2.0 ** -45
    elif kind == "tiny_shifts":
        shifts = rng.random(G.n) * 2.0 ** -33 + rng.integers(0, 3, G.n)
    elif kind == "half_ties":
        shifts = rng.integers(0, 60, G.n) * 0.5
    else:  # 400 distinct fractions, three vertices each
        fr = rng.random(400)
        shifts = rng.integers(0, 30, G.n) + fr[rng.permutation(G.n) % 400]
    _, _, _, st = assert_parity(ldd, G, shifts, 0.1)
    assert st["exact_rank"] == exact


def test_special_shift_values(ldd, cuda):
    """The split of a shift into floor and fraction works on the bits of the
    double: subnormals, -0, values one ulp either side of an integer, and
    large values with few fraction bits must split exactly as floor() does."""
    rng = np.random.default_rng(17)
    G = gen.rmat(12)
    special = np.array([0.0, -0.0, 5e-324, 2.2250738585072014e-308, 1e-300, 2.0 ** -40,
                        np.nextafter(1.0, 0.0), 1.0, np.nextafter(1.0, 2.0), np.nextafter(2.0, 0.0),
                        2.0, 0.5, 3.0000000000000004, 1048575.9999999999, 1048576.0,
                        np.nextafter(1048576.0, 2e6), 524288.5, 7.25])
    shifts = np.where(rng.random(G.n) < 0.5, special[rng.integers(0, special.size, G.n)],
                      gen.shifts(G.n, 0.1, 17))
    _, _, _, st = assert_parity(ldd, G, shifts, 0.1)
    assert st["max_floor_shift"] == int(np.floor(shifts.max()))


@pytest.mark.parametrize("beta", [0.02, 0.5, 1.0])
def test_fraction_rank_bucket_path_taken(ldd, cuda, beta):
    """Exponential shifts with beta <= 1 are ranked on the bucket path (the
    exact path is only for crowded fractions)."""
    G = gen.rmat(14)
    _, _, _, st = assert_parity(ldd, G, gen.shifts(G.n, beta, 41), beta)
    assert st["exact_rank"] == 0


def test_self_loops_and_repeated_arcs(ldd, cuda):
    """Self-loops and repeated arcs change no distance; a vertex whose only
    arcs are self-loops is a component of its own (its own center).  The cut
    counts repeated edges with their multiplicity."""
    base = gen.rmat(11)
    rng = np.random.default_rng(21)
    adj = [list(base.col[base.row_ptr[v]:base.row_ptr[v + 1]]) for v in range(base.n)]
    for v in rng.choice(base.n, 300, replace=False):
        adj[v].append(int(v))
    for v in rng.choice(base.n, 200, replace=False):
        w = next((int(x) for x in adj[v] if x != v), None)
        if w is not None:
            adj[v].append(w)
            adj[w].append(int(v))
    rp = np.zeros(base.n + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(a) for a in adj])
    col = np.asarray([x for a in adj for x in sorted(a)], dtype=np.int32)
    G = gen.CSR("rmat11_loops_multi", rp, col)
    assert any(len(a) > 0 and all(x == v for x in a) for v, a in enumerate(adj))
    for beta in (0.05, 0.5):
        assert_parity(ldd, G, gen.shifts(G.n, beta, 31), beta)


@pytest.mark.parametrize("low_degree", ["1", "0"])
def test_bottom_up_after_an_empty_round(ldd, cuda, low_degree, monkeypatch):
    """A round with an empty frontier jumps to the next start bucket and
    leaves no unsettled list, so a bottom-up round after it must start from
    every vertex the loop owns.  Two 30 x 30 grids: the first starts within
    levels 0 .. 10 and is settled long before the second starts, from level
    195 on; every round with enough frontier arcs is forced bottom-up."""
    monkeypatch.setenv("LDD_PULL_ALPHA", "1000000000")
    monkeypatch.setenv("LDD_PULL_BETA", "1000000000")
    monkeypatch.setenv("LDD_WINDOW_LEVELS", "1")
    monkeypatch.setenv("LDD_LOW_DEGREE_ROUNDS", low_degree)
    g1 = gen.grid2d(30, 30)
    src = np.repeat(np.arange(g1.n), np.diff(g1.row_ptr))
    edges = [(int(u), int(v)) for u, v in zip(src, g1.col) if u < v]
    edges += [(u + g1.n, v + g1.n) for u, v in edges]
    G = gen.from_edges(2 * g1.n, edges, "two_grids")
    rng = np.random.default_rng(3)
    shifts = np.concatenate([190.0 + 10.0 * rng.random(g1.n), 5.0 * rng.random(g1.n)])
    _, _, _, st = assert_parity(ldd, G, shifts, 0.1)
    assert st["pull_rounds"] > 0


@pytest.mark.parametrize("mode", ["always_pull", "alternate", "default"])
def test_bottom_up_rounds(ldd, cuda, mode, monkeypatch):
    """Bottom-up (pull) rounds with the exact min-rank early exit give the same
    keys as top-down rounds: forced every round, alternated, and by heuristic.
    Low-degree graphs run level by level here (a window of levels is always
    top-down)."""
    env = {"always_pull": ("1000000000", "1000000000"), "alternate": ("1000000000", "1"),
           "default": ("14", "24")}[mode]
    monkeypatch.setenv("LDD_PULL_ALPHA", env[0])
    monkeypatch.setenv("LDD_PULL_BETA", env[1])
    monkeypatch.setenv("LDD_WINDOW_LEVELS", "1")
    cases = [(gen.rmat(13), 0.1, 1), (gen.rmat(14), 0.02, 2), (gen.grid2d(60, 70), 0.05, 3),
             (gen.grid3d(14, 15, 16), 0.2, 4), (gen.rgg(4000, 5), 0.3, 5)]
    for G, beta, seed in cases:
        for floor_shifts in (False, True):
            shifts = gen.shifts(G.n, beta, seed)
            if floor_shifts:
                shifts = np.floor(shifts)  # fraction ties: the id breaks them
            _, _, _, st = assert_parity(ldd, G, shifts, beta)
            if mode != "default":
                assert st["pull_rounds"] > 0
