"""Launch parameters (ldd_set_tuning / ldd_autotune): the round loop's
push/pull thresholds, key-probe threshold and CTAs per SM change speed only --
every setting gives the oracle's labels bit for bit -- and the autotuner keeps
a setting from its candidates."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu

SETTINGS = [dict(pull_alpha=0), dict(pull_alpha=1000, pull_gamma=0), dict(pull_beta=1),
            dict(probe_min_arcs=0), dict(probe_min_arcs=1 << 30), dict(bfs_blocks_per_sm=1)]


@pytest.mark.parametrize("G,beta", [(gen.rmat(14), 0.1), (gen.grid2d(90, 70), 0.05)],
                         ids=["rmat14", "grid2d"])
def test_every_setting_is_exact(ldd, cuda, G, beta):
    g = ldd.LddGraph(G.row_ptr, G.col)
    sh = gen.shifts(G.n, beta, 5)
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, sh)
    base = g.tuning()
    for st in SETTINGS:
        g.set_tuning(**(base | st))
        assert g.tuning()["pull_alpha"] == (base | st)["pull_alpha"]
        c = np.empty(G.n, np.int32)
        d = np.empty(G.n, np.int32)
        g.decompose(beta, sh, c, d)
        assert np.array_equal(c, oc) and np.array_equal(d, od), st
    with pytest.raises(ldd.LddError):
        g.set_tuning(bfs_blocks_per_sm=0)
    with pytest.raises(ldd.LddError):
        g.set_tuning(pull_beta=0)
    g.close()


def test_autotune_plain_and_union(ldd, cuda):
    G = gen.rmat(15)
    g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda))
    sh = gen.shifts(G.n, 0.1, 2)
    t = g.autotune(sh, reps=1)
    assert t["ms"] > 0 and t["pull_alpha"] in (4, 8, 14, 24, 48)
    assert t["bfs_blocks_per_sm"] in (1, 2) and g.tuning()["pull_beta"] == t["pull_beta"]
    c = np.empty(G.n, np.int32)
    d = np.empty(G.n, np.int32)
    g.decompose(0.1, sh, c, d)
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, sh)
    assert np.array_equal(c, oc) and np.array_equal(d, od)
    u = ldd.LddUnion([g] * 4)
    shs = [gen.shifts(G.n, 0.1, 10 + i) for i in range(4)]
    t = u.autotune(np.concatenate(shs), reps=1)
    assert t["ms"] > 0
    cu = np.empty(u.total, np.int32)
    du = np.empty(u.total, np.int32)
    u.decompose([0.1] * 4, np.concatenate(shs), cu, du)
    for i in range(4):
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shs[i])
        assert np.array_equal(cu[i * G.n:(i + 1) * G.n], oc)
        assert np.array_equal(du[i * G.n:(i + 1) * G.n], od)
    u.close()
    g.close()
