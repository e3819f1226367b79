"""Launch parameters (ldd_set_tuning / ldd_autotune): the round loop's
push/pull thresholds, key-probe threshold, CTAs per SM, round mode, windows
and arcs per CTA step change speed only --
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
            dict(probe_min_arcs=0), dict(probe_min_arcs=1 << 30), dict(bfs_blocks_per_sm=1),
            dict(low_degree_rounds=0), dict(low_degree_rounds=1, probe_min_arcs=0),
            dict(low_degree_rounds=1, pull_alpha=1000, pull_gamma=0, pull_beta=1000),
            dict(bfs_span=256), dict(bfs_span=1024, low_degree_rounds=0, probe_min_arcs=0)]


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
    for bad in (0, 255, 300, 4352):  # spans: multiples of 256 from 256 to 4096
        with pytest.raises(ldd.LddError):
            g.set_tuning(**(base | dict(bfs_span=bad)))
    g.close()


def test_autotune_plain_and_union(ldd, cuda):
    G = gen.rmat(15)
    g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda))
    sh = gen.shifts(G.n, 0.1, 2)
    t = g.autotune(sh, reps=1)
    assert t["ms"] > 0 and t["pull_alpha"] in (4, 8, 14, 24, 48)
    assert t["bfs_blocks_per_sm"] in (1, 2) and g.tuning()["pull_beta"] == t["pull_beta"]
    assert t["bfs_span"] in (1024, 2048, 4096)
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


@pytest.mark.parametrize("name", ["grid3d_40", "grid2d_300x200_small_beta", "rgg_30000",
                                  "gnp_600", "path_5000"])
def test_low_degree_rounds_both_ways(ldd, cuda, name):
    """Graphs whose vertices have at most 32 arcs run the low-degree rounds by
    default, with windows of eight levels; level by level and the
    edge-balanced rounds give the same labels (all = oracle), with and without
    bottom-up rounds and key probes, on a plain graph and in a union."""
    G, beta = {"grid3d_40": (gen.grid3d(40, 40, 40), 0.05),
               "grid2d_300x200_small_beta": (gen.grid2d(300, 200), 0.01),
               "rgg_30000": (gen.rgg(30000, 3), 0.2),
               "gnp_600": (gen.random_graph(600, 0.02, 4), 0.1),
               "path_5000": (gen.grid2d(5000, 1), 0.02)}[name]
    assert int(np.diff(G.row_ptr).max()) <= 32
    sh = gen.shifts(G.n, beta, 8)
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, sh)
    g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda))
    assert g.tuning()["low_degree_rounds"] == 1
    base = g.tuning()
    assert base["window_levels"] == 8  # windows of levels by default
    for st in (dict(), dict(low_degree_rounds=1, window_levels=1), dict(low_degree_rounds=0),
               dict(low_degree_rounds=1, window_levels=1, pull_alpha=1000, pull_gamma=0),
               dict(low_degree_rounds=1, window_levels=1, probe_min_arcs=0, bfs_blocks_per_sm=2)):
        g.set_tuning(**(base | st))
        c = torch.empty(G.n, dtype=torch.int32, device=cuda)
        d = torch.empty(G.n, dtype=torch.int32, device=cuda)
        g.decompose(beta, torch.from_numpy(sh).to(cuda), c, d)
        assert np.array_equal(c.cpu().numpy(), oc) and np.array_equal(d.cpu().numpy(), od), st
        st_ = g.stats()
        if st.get("low_degree_rounds") == 1 and st_["pull_rounds"] == 0:
            assert st_["push_arcs"] <= G.nnz  # level by level: every arc offered at most once
    u = ldd.LddUnion([g, g, g])
    assert u.tuning()["window_levels"] == 1  # unions: level by level by default
    shs = [gen.shifts(G.n, beta, 20 + i) for i in range(3)]
    for ldr, wl in ((1, 8), (1, 1), (0, 8)):
        u.set_tuning(**(u.tuning() | dict(low_degree_rounds=ldr, window_levels=wl)))
        cu = torch.empty(u.total, dtype=torch.int32, device=cuda)
        du = torch.empty(u.total, dtype=torch.int32, device=cuda)
        u.decompose([beta] * 3, torch.from_numpy(np.concatenate(shs)).to(cuda), cu, du)
        for i in range(3):
            oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shs[i])
            assert np.array_equal(cu[i * G.n:(i + 1) * G.n].cpu().numpy(), oc)
            assert np.array_equal(du[i * G.n:(i + 1) * G.n].cpu().numpy(), od)
    u.close()
    g.close()


@pytest.mark.parametrize("name", ["grid3d_48", "grid2d_400x300", "rgg_big_frontiers", "path_3000"])
def test_windows_of_levels_are_exact(ldd, cuda, name):
    """Low-degree rounds with windows of 2 .. 64 levels between grid barriers:
    label-correcting inside a window, so a vertex may be expanded twice, but
    the labels equal the oracle's.  Local queues limited to one or a few
    dozen entries per CTA overflow, and the overflow list carries vertices into
    the next round; the random geometric graph at beta 0.5 starts many centers
    at once."""
    G, beta = {"grid3d_48": (gen.grid3d(48, 48, 48), 0.03),
               "grid2d_400x300": (gen.grid2d(400, 300), 0.02),
               "rgg_big_frontiers": (gen.rgg(1_500_000, 6), 0.5),
               "path_3000": (gen.grid2d(3000, 1), 0.01)}[name]
    sh = gen.shifts(G.n, beta, 13)
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, sh)
    g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda))
    base = g.tuning()
    c = torch.empty(G.n, dtype=torch.int32, device=cuda)
    d = torch.empty(G.n, dtype=torch.int32, device=cuda)
    runs = []
    for wl, wmax, wq in ((2, 1 << 18, 0), (4, 1 << 18, 0), (8, 1 << 18, 0), (64, 1 << 18, 0),
                         (8, 1 << 30, 0), (8, 0, 0), (3, 1 << 30, 0), (8, 1 << 30, 64),
                         (5, 1 << 30, 1)):
        g.set_tuning(**(base | dict(window_levels=wl, window_max_frontier=wmax, window_queue=wq)))
        g.decompose(beta, torch.from_numpy(sh).to(cuda), c, d)
        st = g.stats()
        assert np.array_equal(c.cpu().numpy(), oc) and np.array_equal(d.cpu().numpy(), od), \
            (wl, wmax, wq)
        runs.append((wl, wmax, wq, st["bfs_windows"], st["bfs_overflow"], st["items"]))
        assert st["items"] >= st["n_active"]  # every BFS vertex expanded at least once
        if wmax == 0:
            assert st["bfs_windows"] == 0 and st["bfs_overflow"] == 0
        if wq == 1 and name != "path_3000":  # one local entry per CTA and level: full queues
            assert st["bfs_overflow"] > 0, runs
    assert any(r[3] > 0 for r in runs), runs
    # a union of three copies, windows on
    u = ldd.LddUnion([g, g, g])
    u.set_tuning(**(u.tuning() | dict(window_levels=8, window_max_frontier=1 << 30,
                                      window_queue=16)))
    shs = [gen.shifts(G.n, beta, 40 + i) for i in range(3)]
    cu = torch.empty(u.total, dtype=torch.int32, device=cuda)
    du = torch.empty(u.total, dtype=torch.int32, device=cuda)
    u.decompose([beta] * 3, torch.from_numpy(np.concatenate(shs)).to(cuda), cu, du)
    assert u.stats()["bfs_windows"] > 0
    for i in range(3):
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shs[i])
        assert np.array_equal(cu[i * G.n:(i + 1) * G.n].cpu().numpy(), oc)
        assert np.array_equal(du[i * G.n:(i + 1) * G.n].cpu().numpy(), od)
    u.close()
    g.close()
