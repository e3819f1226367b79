"""CUDA-graph replay (ldd_set_graph_replay): the captured fast path must give
exactly the oracle's answer on every call, fall back to the regular path for
the inputs that need it, and pick the replay up again afterwards."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu


def _check(G, shifts, c, d):
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts)
    assert np.array_equal(np.asarray(c), oc) and np.array_equal(np.asarray(d), od)
    return oc


def test_replay_plain_graph(ldd, cuda):
    G = gen.rmat(13)
    g = ldd.LddGraph(G.row_ptr, G.col)
    g.set_graph_replay(True)
    kinds = []
    for i in range(5):
        sh = gen.shifts(G.n, 0.1, 200 + i)
        if i % 2:  # device buffers
            c = torch.empty(G.n, dtype=torch.int32, device=cuda)
            d = torch.empty(G.n, dtype=torch.int32, device=cuda)
            g.decompose(0.1, torch.from_numpy(sh).to(cuda), c, d)
            c, d = c.cpu().numpy(), d.cpu().numpy()
        else:
            c = np.empty(G.n, np.int32)
            d = np.empty(G.n, np.int32)
            g.decompose(0.1, sh, c, d)
        oc = _check(G, sh, c, d)
        kinds.append(g.stats()["replayed"])
        assert g.cut_edges(c) == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    assert kinds[0] == 0 and all(k == 1 for k in kinds[1:]), kinds
    g.set_graph_replay(False)
    sh = gen.shifts(G.n, 0.1, 300)
    c = np.empty(G.n, np.int32)
    d = np.empty(G.n, np.int32)
    g.decompose(0.1, sh, c, d)
    _check(G, sh, c, d)
    assert g.stats()["replayed"] == 0
    g.close()


def test_replay_falls_back_and_resumes(ldd, cuda):
    """Shifts that need the exact rank path, then a start-bucket table
    regrowth, in the middle of a replayed sequence."""
    G = gen.grid2d(40, 30)
    rng = np.random.default_rng(9)
    crowded = rng.random(G.n) * 2.0 ** -33 + rng.integers(0, 3, G.n)
    huge = gen.shifts(G.n, 0.1, 3)
    huge[7] = 5000.5
    seq = [gen.shifts(G.n, 0.1, 4), gen.shifts(G.n, 0.2, 5), crowded, gen.shifts(G.n, 0.1, 6),
           huge, gen.shifts(G.n, 0.1, 7), gen.shifts(G.n, 0.3, 8)]
    g = ldd.LddGraph(G.row_ptr, G.col)
    g.set_graph_replay(True)
    kinds = []
    for sh in seq:
        c = np.empty(G.n, np.int32)
        d = np.empty(G.n, np.int32)
        g.decompose(0.1, sh, c, d)
        _check(G, sh, c, d)
        kinds.append((g.stats()["replayed"], g.stats()["exact_rank"]))
    assert kinds[2] == (0, 1)          # exact path, not replayed
    assert kinds[4][0] == 0            # table regrowth, not replayed
    assert kinds[3][0] == 1 and kinds[5][0] == 1 and kinds[6][0] == 1, kinds
    g.close()


def test_replay_union(ldd, cuda):
    Gs = [gen.rgg(2000 + 97 * i, 30 + i) for i in range(6)] + [gen.rmat(11)]
    betas = [0.05, 0.1, 0.2, 0.3, 0.4, 0.5, 0.1]
    mem = [ldd.LddGraph(G.row_ptr, G.col) for G in Gs]
    u = ldd.LddUnion(mem)
    u.set_graph_replay(True)
    for it in range(4):
        shifts = [gen.shifts(G.n, b, 500 + 10 * it + i) for i, (G, b) in enumerate(zip(Gs, betas))]
        cat = np.concatenate(shifts)
        want_cut = it != 2
        if it % 2:
            c = torch.empty(u.total, dtype=torch.int32, device=cuda)
            d = torch.empty(u.total, dtype=torch.int32, device=cuda)
            cuts = u.decompose(betas, torch.from_numpy(cat).to(cuda), c, d, want_cut=want_cut)
            c, d = c.cpu().numpy(), d.cpu().numpy()
        else:
            c = np.empty(u.total, np.int32)
            d = np.empty(u.total, np.int32)
            cuts = u.decompose(betas, cat, c, d, want_cut=want_cut)
        assert u.stats()["replayed"] == (1 if it > 0 else 0)
        for s, G in enumerate(Gs):
            lo, hi = u.offsets[s], u.offsets[s + 1]
            oc = _check(G, shifts[s], c[lo:hi], d[lo:hi])
            if want_cut:
                assert cuts[s] == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    u.close()
    for m in mem:
        m.close()
