"""Full-size workloads, in the configuration bench.py times: every vertex of
every decomposition compared with the oracle (zero tolerance), plus the O(m)
optimality certificate on the GPU output itself and the cut count."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["grid2d_256", "rmat22", "grid3d_256"])
def test_fullsize_workload(ldd, cuda, name):
    spec = gen.WORKLOADS[name]
    G = gen.make_graph(spec["graph"])
    g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda),
                     validate=False)
    c = torch.empty(G.n, dtype=torch.int32, device=cuda)
    d = torch.empty(G.n, dtype=torch.int32, device=cuda)
    for beta in spec["betas"]:
        shifts = gen.shifts(G.n, beta, spec["shift_seed"])
        g.decompose(beta, torch.from_numpy(shifts).to(cuda), c, d)
        cut = g.cut_edges(c)
        gc, gd = c.cpu().numpy(), d.cpu().numpy()
        code, bad = oracle.oracle_certify(G.row_ptr, G.col, shifts, gc, gd)
        assert code == 0, f"{name} beta={beta}: certificate fails ({oracle.CERT_CODES[code]}) at {bad}"
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts)
        nbad = int((gc != oc).sum() + (gd != od).sum())
        assert nbad == 0, f"{name} beta={beta}: {nbad} mismatches"
        assert cut == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
        assert gd.max() <= np.floor(shifts.max())  # radius <= floor(delta_max), Lemma 3.2
        if G.nnz <= 1 << 27:  # the allocation-free count, near its span-table limit
            rp = torch.from_numpy(G.row_ptr).to(cuda)
            col = torch.from_numpy(G.col).to(cuda)
            assert ldd.ldd_cut_edges_noalloc(G.n, G.nnz, rp, col, c) == cut
            del rp, col
    g.close()
