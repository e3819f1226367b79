"""GPU parity of the block decomposition by repeated decomposition
(ldd_block_decompose; Section 1's remark on Linial and Saks' blocks): every
iteration's centers and distances, every arc's block and the edges left before
each iteration equal the oracle's loop (oracle.oracle_block_decompose), element
by element."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle
from tests.test_oracle_block import CASES, edge_blocks

pytestmark = pytest.mark.gpu


def _run(ldd, G, shifts, cuda, host=False, want_paths=True):
    k = len(shifts)
    if host:
        g = ldd.LddGraph(G.row_ptr, G.col)
        sh = [np.ascontiguousarray(s) for s in shifts]
        cs = [np.full(G.n, -9, np.int32) for _ in range(k)]
        ds = [np.full(G.n, -9, np.int32) for _ in range(k)]
        ab = np.full(G.nnz, -9, np.int32)
    else:
        g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda))
        sh = [torch.from_numpy(s).to(cuda) for s in shifts]
        cs = [torch.full((G.n,), -9, dtype=torch.int32, device=cuda) for _ in range(k)]
        ds = [torch.full((G.n,), -9, dtype=torch.int32, device=cuda) for _ in range(k)]
        ab = torch.full((G.nnz,), -9, dtype=torch.int32, device=cuda)
    nb, rem = g.block_decompose([0.5] * k, sh, cs if want_paths else None,
                                ds if want_paths else None, ab)
    tonp = (lambda x: x) if host else (lambda x: x.cpu().numpy())
    out = (nb, rem, [tonp(c) for c in cs], [tonp(d) for d in ds], tonp(ab))
    return g, out


def _check(G, shifts, got):
    nb, rem, cs, ds, ab = got
    oc, od, oab, orem = oracle.oracle_block_decompose(G.row_ptr, G.col, shifts)
    assert nb == len(oc) and rem == list(orem)
    bad = np.flatnonzero(ab != oab)
    assert bad.size == 0, f"{G.name}: {bad.size} arcs in another block, first {bad[:5]}"
    for i in range(nb):
        assert np.array_equal(cs[i], oc[i]), f"{G.name}: centers differ in iteration {i}"
        assert np.array_equal(ds[i], od[i]), f"{G.name}: distances differ in iteration {i}"


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_golden_block_examples_on_gpu(ldd, cuda, case):
    G = gen.from_edges(case["n"], case["edges"], case["name"])
    shifts = [case["shifts"][i] for i in sorted(case["shifts"])]
    g, (nb, rem, cs, ds, ab) = _run(ldd, G, shifts, cuda)
    assert nb == case["blocks"] and rem == case["remaining"]
    assert edge_blocks(G, case["edges"], ab) == case["edge_block"]
    for i in case["center"]:
        assert list(cs[i]) == case["center"][i] and list(ds[i]) == case["dist"][i]
    g.close()


GRAPHS = {
    "rmat14": lambda: gen.rmat(14),
    "rmat17": lambda: gen.rmat(17),  # hub rows of thousands of arcs
    "grid2d_96x75": lambda: gen.grid2d(96, 75),
    "grid3d_20": lambda: gen.grid3d(20, 20, 20),
    "rgg_20000": lambda: gen.rgg(20000, 4),
    "star_6000": lambda: gen.from_edges(6001, [(0, i) for i in range(1, 6001)], "star6000"),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_blocks_match_oracle(ldd, cuda, name):
    G = GRAPHS[name]()
    shifts = [gen.shifts(G.n, 0.5, 300 + i) for i in range(60)]
    g, got = _run(ldd, G, shifts, cuda)
    assert got[1][-1] == 0, "60 iterations should leave no edge"
    _check(G, shifts, got)
    # a second call on the same graph object (buffers reused) with other shifts
    shifts2 = [gen.shifts(G.n, 0.5, 900 + i) for i in range(60)]
    nb, rem, cs, ds, ab = [None] * 5
    c2 = [torch.empty(G.n, dtype=torch.int32, device=cuda) for _ in shifts2]
    d2 = [torch.empty(G.n, dtype=torch.int32, device=cuda) for _ in shifts2]
    ab2 = torch.empty(G.nnz, dtype=torch.int32, device=cuda)
    nb, rem = g.block_decompose([0.5] * 60, [torch.from_numpy(s).to(cuda) for s in shifts2],
                                c2, d2, ab2)
    _check(G, shifts2, (nb, rem, [c.cpu().numpy() for c in c2], [d.cpu().numpy() for d in d2],
                        ab2.cpu().numpy()))
    g.close()


def test_blocks_host_buffers_and_no_paths(ldd, cuda):
    G = gen.rmat(12)
    shifts = [gen.shifts(G.n, 0.5, 40 + i) for i in range(50)]
    g, got = _run(ldd, G, shifts, cuda, host=True)
    _check(G, shifts, got)
    g.close()
    # without per-iteration outputs: blocks and counts only
    g, (nb, rem, _, _, ab) = _run(ldd, G, shifts, cuda, want_paths=False)
    _, _, oab, orem = oracle.oracle_block_decompose(G.row_ptr, G.col, shifts)
    assert rem == list(orem) and np.array_equal(ab, oab)
    g.close()


def test_blocks_edge_cases(ldd, cuda):
    # shift vectors run out: equal shifts make singletons, nothing joins a block
    G = gen.grid2d(7, 6)
    same = [np.full(G.n, 0.5)] * 3
    g, (nb, rem, cs, ds, ab) = _run(ldd, G, same, cuda)
    assert nb == 3 and rem == [G.m] * 4 and (ab == -1).all()
    # k = 0, and a graph without arcs
    assert g.block_decompose([], []) == (0, [G.m])
    g.close()
    E = gen.from_edges(5, [])
    g = ldd.LddGraph(E.row_ptr, E.col)
    assert g.block_decompose([0.5], [np.zeros(5)]) == (0, [0])
    g.close()
    # a bad shift in iteration 1: iteration 0's outputs are complete
    G = gen.rmat(10)
    shifts = [gen.shifts(G.n, 0.5, 1), np.full(G.n, -1.0)]
    g = ldd.LddGraph(G.row_ptr, G.col)
    c = [np.empty(G.n, np.int32) for _ in shifts]
    d = [np.empty(G.n, np.int32) for _ in shifts]
    with pytest.raises(ldd.LddError) as e:
        g.block_decompose([0.5, 0.5], shifts, c, d)
    assert e.value.status == ldd.LDD_ERR_ARG
    oc, od, _, _ = oracle.oracle_block_decompose(G.row_ptr, G.col, shifts[:1])
    assert np.array_equal(c[0], oc[0]) and np.array_equal(d[0], od[0])
    # still usable afterwards
    ok = [gen.shifts(G.n, 0.5, 7 + i) for i in range(40)]
    _, got = _run(ldd, G, ok, cuda)
    _check(G, ok, got)
    g.close()
