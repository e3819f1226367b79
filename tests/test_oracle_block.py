"""Pins of the block-decomposition oracle (blocks by repeated decomposition,
Section 1's remark on Linial and Saks' block decompositions), CPU only:

* hand-derived worked examples (tests/golden/block_examples.txt);
* the loop written out literally over brute-force decompositions
  (``oracle.brute.brute_block_decompose``), exhaustively on small graphs and on
  random graphs, with tie-heavy and Exp(1/2) shifts;
* invariants on mid-size graphs: every edge lands in exactly one block, both
  arcs of an edge in the same one; block i's edges lie inside pieces of
  iteration i and the edges left are exactly the ones it cut (Definition 1.1's
  count on G_i); the loop stops when nothing is left;
* the paper's reason the loop is short: each (1/2, .) decomposition keeps at
  most a 1 - e^{-1/2} < 1/2 fraction of the edges in expectation
  (Corollary 3.5), so O(log m) blocks suffice.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import pytest

import ldd_gen as gen
import oracle
from oracle.brute import brute_block_decompose

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "block_examples.txt")


def load_cases():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "case":
            cur = {"name": rest, "shifts": {}, "center": {}, "dist": {}}
            cases.append(cur)
        elif key == "n":
            cur["n"] = int(rest)
        elif key == "edges":
            cur["edges"] = [tuple(map(int, e.split("-"))) for e in rest.split()]
        elif key.startswith("shifts"):
            cur["shifts"][int(key[6:])] = np.array([float(x) for x in rest.split()])
        elif key.startswith("center"):
            cur["center"][int(key[6:])] = [int(x) for x in rest.split()]
        elif key.startswith("dist"):
            cur["dist"][int(key[4:])] = [int(x) for x in rest.split()]
        elif key in ("edge_block", "remaining"):
            cur[key] = [int(x) for x in rest.split()]
        elif key == "blocks":
            cur["blocks"] = int(rest)
    return cases


CASES = load_cases()


def arc_of(G, u, v):
    row = G.col[G.row_ptr[u]:G.row_ptr[u + 1]]
    return int(G.row_ptr[u] + int(np.flatnonzero(row == v)[0]))


def edge_blocks(G, edges, arc_block):
    out = []
    for u, v in edges:
        a, b = arc_block[arc_of(G, u, v)], arc_block[arc_of(G, v, u)]
        assert a == b, f"edge {u}-{v}: its two arcs are in blocks {a} and {b}"
        out.append(int(a))
    return out


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_golden_block_examples(case):
    G = gen.from_edges(case["n"], case["edges"], case["name"])
    shifts = [case["shifts"][i] for i in sorted(case["shifts"])]
    for fn in (oracle.oracle_block_decompose, brute_block_decompose):
        cs, ds, ab, rem = fn(G.row_ptr, G.col, shifts)
        assert len(cs) == case["blocks"]
        assert list(rem) == case["remaining"]
        assert edge_blocks(G, case["edges"], ab) == case["edge_block"]
        for i in case["center"]:
            assert list(cs[i]) == case["center"][i], (fn.__name__, i)
            assert list(ds[i]) == case["dist"][i], (fn.__name__, i)


def _tie_shifts(n, rng, k):
    """Half-integers and small integers: many exact ties of Eq. (1)."""
    return [rng.integers(0, 4, n) / 2.0 for _ in range(k)]


def _exp_shifts(n, seed, k, beta=0.5):
    return [gen.shifts(n, beta, seed * 100 + i) for i in range(k)]


def _same(G, shifts):
    cs, ds, ab, rem = oracle.oracle_block_decompose(G.row_ptr, G.col, shifts)
    bc, bd, bb, br = brute_block_decompose(G.row_ptr, G.col, shifts)
    assert len(cs) == len(bc) and list(rem) == list(br)
    assert list(ab) == list(bb)
    for i in range(len(cs)):
        assert list(cs[i]) == list(bc[i]) and list(ds[i]) == list(bd[i])


def test_exhaustive_small_graphs_vs_literal_loop():
    rng = np.random.default_rng(5)
    for n in range(1, 6):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            edges = [p for i, p in enumerate(pairs) if mask >> i & 1]
            G = gen.from_edges(n, edges)
            _same(G, _tie_shifts(n, rng, 6))
            _same(G, _exp_shifts(n, mask + 17 * n, 6))


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_vs_literal_loop(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(6, 13))
    G = gen.random_graph(n, float(rng.uniform(0.15, 0.6)), seed)
    _same(G, _exp_shifts(n, seed, 10))
    _same(G, _tie_shifts(n, rng, 10))


@pytest.mark.parametrize("G", [gen.rmat(11), gen.grid2d(40, 37), gen.rgg(3000, 9)],
                         ids=["rmat11", "grid40x37", "rgg3000"])
def test_block_invariants(G):
    k = 40
    shifts = _exp_shifts(G.n, 7, k)
    cs, ds, ab, rem = oracle.oracle_block_decompose(G.row_ptr, G.col, shifts)
    src = np.repeat(np.arange(G.n), np.diff(G.row_ptr))
    dst = G.col.astype(np.int64)
    rev = np.empty_like(ab)  # the reverse arc of every arc
    order = np.lexsort((dst, src))
    rorder = np.lexsort((src, dst))
    rev[order] = ab[rorder]
    assert np.array_equal(ab, rev), "the two arcs of an edge sit in different blocks"
    blocks = len(cs)
    assert rem[-1] == 0 and (ab >= 0).all(), "edges left after the loop ended"
    assert rem[0] == G.m
    for i in range(blocks):
        alive = ab >= i  # E_i
        inside = cs[i][src] == cs[i][dst]
        assert np.array_equal(ab[alive] == i, inside[alive])
        # E_{i+1} is exactly what iteration i cut (Definition 1.1 on G_i)
        rp_i = np.concatenate(([0], np.cumsum(np.bincount(src[alive], minlength=G.n))))
        cut = oracle.oracle_cut_edges(rp_i, dst[alive], cs[i])
        assert cut == rem[i + 1]
        # Lemma 3.2 per iteration: radius <= floor(delta_max)
        assert ds[i].max() <= math.floor(shifts[i].max())


def test_halving_and_block_count():
    """Corollary 3.5 at beta = 1/2: an edge of G_i stays cut with probability
    at most 1 - e^{-1/2} ~ 0.39, so |E_{i+1}| / |E_i| averages below that and
    the loop ends after O(log m) blocks."""
    bound = 1 - math.exp(-0.5)
    G = gen.grid2d(30, 30)
    ratios, counts = [], []
    for seed in range(30):
        _, _, _, rem = oracle.oracle_block_decompose(G.row_ptr, G.col, _exp_shifts(G.n, seed, 60))
        assert rem[-1] == 0
        ratios.append(rem[1] / rem[0])
        counts.append(len(rem) - 1)
    assert np.mean(ratios) <= bound + 0.03
    assert max(counts) <= 3 * math.log2(G.m)


def test_degenerate_inputs():
    # no edges: no block
    G = gen.from_edges(4, [])
    cs, ds, ab, rem = oracle.oracle_block_decompose(G.row_ptr, G.col, _exp_shifts(4, 1, 3))
    assert cs == [] and list(rem) == [0] and ab.shape == (0,)
    # one dominant shift per component: one block holds every edge
    G = gen.from_edges(7, [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6)])
    sh = np.zeros(7)
    sh[1], sh[5] = 100.0, 100.0
    cs, ds, ab, rem = oracle.oracle_block_decompose(G.row_ptr, G.col, [sh, sh])
    assert len(cs) == 1 and list(rem) == [5, 0] and (ab == 0).all()
    # shift vectors run out first: the edges left have block -1
    G = gen.grid2d(6, 6)
    same = [np.full(G.n, 0.5)] * 2  # equal shifts: singletons, nothing ever joins a block
    cs, ds, ab, rem = oracle.oracle_block_decompose(G.row_ptr, G.col, same)
    assert len(cs) == 2 and list(rem) == [G.m] * 3 and (ab == -1).all()


MUTANTS = {
    "keeps the uncut edges": ("alive = alive[~inside]", "alive = alive[inside]"),
    "numbers blocks from 1": ("arc_block[alive[inside]] = i", "arc_block[alive[inside]] = i + 1"),
    "never shrinks the graph": ("cur_col = cl[alive]", "cur_col = cur_col"),
    "counts arcs, not edges": ("remaining.append(int((src[alive] < cl[alive]).sum()))",
                               "remaining.append(int(alive.shape[0]))"),
    "reuses the first shifts": ("c, d = oracle_ldd(cur_rp, cur_col, sh)",
                                "c, d = oracle_ldd(cur_rp, cur_col, shifts_list[0])"),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistakes_are_caught(name):
    """A copy of the oracle with one plausible mistake fails a golden case."""
    import inspect

    src = inspect.getsource(oracle.oracle_block_decompose)
    old, new = MUTANTS[name]
    assert old in src
    ns = dict(oracle.__dict__)
    exec(src.replace(old, new), ns)
    fn = ns["oracle_block_decompose"]
    for case in CASES:
        G = gen.from_edges(case["n"], case["edges"], case["name"])
        shifts = [case["shifts"][i] for i in sorted(case["shifts"])]
        try:
            cs, ds, ab, rem = fn(G.row_ptr, G.col, shifts)
            if (len(cs) != case["blocks"] or list(rem) != case["remaining"]
                    or edge_blocks(G, case["edges"], ab) != case["edge_block"]
                    or any(list(cs[i]) != case["center"][i] or list(ds[i]) != case["dist"][i]
                           for i in case["center"])):
                return
        except (AssertionError, IndexError, ValueError):
            return
    pytest.fail(f"mutant '{name}' passes every golden case")
