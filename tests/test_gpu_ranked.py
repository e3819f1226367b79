"""The permutation variant (ldd_decompose_ranked): integer levels plus a
tie-break permutation in place of FP64 shifts (Section 4).  Bit-exact against
its oracle on every graph family, identical to ldd_decompose on shifts that
order the same way, and bad input rejected."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu

CASES = [(gen.grid2d(61, 47), 0.1), (gen.rmat(13), 0.05), (gen.rgg(20000, 6), 0.2),
         (gen.grid3d(20, 20, 20), 0.02), (gen.random_graph(300, 0.01, 4), 0.5),
         (gen.from_edges(40, [(i, i + 1) for i in range(0, 38, 2)], "pairs"), 0.3)]


@pytest.mark.parametrize("G,beta", CASES, ids=[c[0].name for c in CASES])
@pytest.mark.parametrize("host", [False, True])
def test_ranked_parity(ldd, cuda, G, beta, host):
    levels, perm = gen.ranked_inputs(G.n, beta, 31)
    if host:
        g = ldd.LddGraph(G.row_ptr, G.col)
        c = np.empty(G.n, np.int32)
        d = np.empty(G.n, np.int32)
        g.decompose_ranked(levels, perm, c, d)
    else:
        g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda))
        ct = torch.empty(G.n, dtype=torch.int32, device=cuda)
        dt = torch.empty(G.n, dtype=torch.int32, device=cuda)
        g.decompose_ranked(torch.from_numpy(levels).to(cuda), torch.from_numpy(perm).to(cuda),
                           ct, dt)
        c, d = ct.cpu().numpy(), dt.cpu().numpy()
    oc, od = oracle.oracle_ldd_ranked(G.row_ptr, G.col, levels, perm)
    assert np.array_equal(c, oc) and np.array_equal(d, od)
    assert g.cut_edges(c) == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    g.close()


def test_ranked_then_shift_paths_interleave(ldd, cuda):
    """The ranked path leaves the fast rank path's state clean."""
    G = gen.rmat(12)
    g = ldd.LddGraph(G.row_ptr, G.col)
    c = np.empty(G.n, np.int32)
    d = np.empty(G.n, np.int32)
    for i in range(3):
        levels, perm = gen.ranked_inputs(G.n, 0.1, 50 + i)
        g.decompose_ranked(levels, perm, c, d)
        oc, od = oracle.oracle_ldd_ranked(G.row_ptr, G.col, levels, perm)
        assert np.array_equal(c, oc) and np.array_equal(d, od)
        sh = gen.shifts(G.n, 0.1, 70 + i)
        g.decompose(0.1, sh, c, d)
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, sh)
        assert np.array_equal(c, oc) and np.array_equal(d, od)
    g.close()


def test_ranked_bad_input(ldd, cuda):
    G = gen.grid2d(8, 8)
    g = ldd.LddGraph(G.row_ptr, G.col)
    c = np.empty(G.n, np.int32)
    d = np.empty(G.n, np.int32)
    levels, perm = gen.ranked_inputs(G.n, 0.1, 1)
    bad_perm = perm.copy()
    bad_perm[3] = bad_perm[4]
    for lv, pm in [(levels, bad_perm), (np.where(np.arange(G.n) == 5, -1, levels).astype(np.int32), perm),
                   (levels, np.where(np.arange(G.n) == 2, G.n, perm).astype(np.int32))]:
        with pytest.raises(ldd.LddError) as e:
            g.decompose_ranked(lv, pm, c, d)
        assert e.value.status == ldd.LDD_ERR_ARG
    g.decompose_ranked(levels, perm, c, d)  # still usable
    oc, od = oracle.oracle_ldd_ranked(G.row_ptr, G.col, levels, perm)
    assert np.array_equal(c, oc) and np.array_equal(d, od)
    g.close()
