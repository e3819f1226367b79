"""Pins of the permutation variant's oracle (Section 4: a random permutation
of the vertices stands in for the fractional parts of the shifts), CPU only:

* the variant's definition written out (all-pairs BFS, argmin over the
  integer pair (dist(u, v) - level_u, perm_u)), exhaustively on every graph
  with up to 5 vertices and on random graphs;
* limits: equal levels give singletons; one dominant level per component
  gives BFS distances from that vertex;
* the input recipe: perm is a permutation, levels are the floors of the
  exponential shifts;
* the oracle rejects bad input.
"""
from __future__ import annotations

import itertools

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import ldd_gen as gen
import oracle
from oracle.brute import brute_ldd_ranked


def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield [p for i, p in enumerate(pairs) if mask >> i & 1]


def test_exhaustive_small_graphs_vs_definition():
    rng = np.random.default_rng(7)
    checked = 0
    for n in range(1, 6):
        for edges in _all_graphs(n):
            G = gen.from_edges(n, edges)
            for _ in range(2):
                levels = rng.integers(0, 3, n).astype(np.int32)
                perm = rng.permutation(n).astype(np.int32)
                c, d = oracle.oracle_ldd_ranked(G.row_ptr, G.col, levels, perm)
                bc, bd = brute_ldd_ranked(G.row_ptr, G.col, levels, perm)
                assert list(c) == bc and list(d) == bd, (n, edges, levels, perm)
                checked += 1
    assert checked > 2000


@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_vs_definition(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(20):
        n = int(rng.integers(2, 13))
        G = gen.random_graph(n, float(rng.uniform(0.05, 0.6)), int(rng.integers(1 << 30)))
        levels, perm = gen.ranked_inputs(n, float(rng.choice([0.1, 0.5, 2.0])),
                                         int(rng.integers(1 << 30)))
        c, d = oracle.oracle_ldd_ranked(G.row_ptr, G.col, levels, perm)
        bc, bd = brute_ldd_ranked(G.row_ptr, G.col, levels, perm)
        assert list(c) == bc and list(d) == bd


def test_equal_levels_give_singletons():
    G = gen.grid2d(20, 15)
    perm = gen.permutation(G.n, 3)
    c, d = oracle.oracle_ldd_ranked(G.row_ptr, G.col, np.full(G.n, 4, np.int32), perm)
    assert np.array_equal(c, np.arange(G.n)) and not d.any()


def test_dominant_level_gives_bfs_distances():
    G = gen.rgg(800, 4)
    levels = np.zeros(G.n, np.int32)
    A = sp.csr_matrix((np.ones(G.nnz), G.col, G.row_ptr), shape=(G.n, G.n))
    ncomp, lab = csg.connected_components(A, directed=False)
    heads = [int(np.flatnonzero(lab == k)[0]) for k in range(ncomp)]
    levels[heads] = G.n  # farther than any path: every vertex joins its component's head
    c, d = oracle.oracle_ldd_ranked(G.row_ptr, G.col, levels, gen.permutation(G.n, 5))
    for h in heads:
        ref = csg.shortest_path(A, unweighted=True, indices=h)
        members = lab == lab[h]
        assert np.all(c[members] == h)
        assert np.array_equal(d[members], ref[members].astype(np.int32))


def test_ranked_inputs_recipe():
    levels, perm = gen.ranked_inputs(5000, 0.1, 9)
    assert np.array_equal(np.sort(perm), np.arange(5000))
    assert np.array_equal(levels, np.floor(gen.shifts(5000, 0.1, 9)).astype(np.int32))
    assert not np.array_equal(perm, gen.permutation(5000, 11))  # seeded
    # positions are uniform: mean position ~ (n - 1) / 2 over the first half of ids
    assert abs(perm[:2500].mean() - 2499.5) < 0.05 * 5000


def test_bad_input_rejected():
    G = gen.grid2d(3, 3)
    with pytest.raises(ValueError):
        oracle.oracle_ldd_ranked(G.row_ptr, G.col, np.full(9, -1, np.int32), np.arange(9))
    with pytest.raises(ValueError):
        oracle.oracle_ldd_ranked(G.row_ptr, G.col, np.zeros(9, np.int32), np.zeros(9, np.int32))
