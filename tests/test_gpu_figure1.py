"""Figure 1 of the paper: a 1000 x 1000 grid decomposed at beta = 0.002 ..
0.1.  Every labelling equals the oracle's, and the figure's reading holds:
lower beta gives fewer, larger pieces and fewer edges between them, with
every radius at most floor(delta_max) (Lemma 3.2)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu

BETAS = (0.002, 0.005, 0.01, 0.02, 0.05, 0.1)


def test_figure1_grid_sweep(ldd, cuda):
    G = gen.grid2d(1000, 1000)
    g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda),
                     validate=False)
    c = torch.empty(G.n, dtype=torch.int32, device=cuda)
    d = torch.empty(G.n, dtype=torch.int32, device=cuda)
    pieces, cuts, radii = [], [], []
    for beta in BETAS:
        p, ct, rd = [], [], []
        for seed in (1, 2):
            sh = gen.shifts(G.n, beta, seed)
            g.decompose(beta, torch.from_numpy(sh).to(cuda), c, d)
            cut = g.cut_edges(c)
            gc, gd = c.cpu().numpy(), d.cpu().numpy()
            if seed == 1:
                oc, od = oracle.oracle_ldd(G.row_ptr, G.col, sh)
                assert np.array_equal(gc, oc) and np.array_equal(gd, od), f"beta {beta}"
                assert cut == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
            assert gd.max() <= np.floor(sh.max())
            p.append(len(np.unique(gc)))
            ct.append(cut)
            rd.append(gd.mean())
        pieces.append(np.mean(p))
        cuts.append(np.mean(ct))
        radii.append(np.mean(rd))
    assert all(a < b for a, b in zip(pieces, pieces[1:])), pieces
    assert all(a < b for a, b in zip(cuts, cuts[1:])), cuts
    assert all(a > b for a, b in zip(radii, radii[1:])), radii
    g.close()
