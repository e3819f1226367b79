"""Batches as disjoint unions (ldd_create_union / ldd_union_decompose): every
member of a union decomposition must equal the oracle on that member alone
(center, dist and cut count, zero tolerance), whatever the mix of member
sizes, shapes, betas and buffer placements, and equal k separate calls."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu


def _members():
    """Member graphs of different shapes, sizes (not multiples of 32, one
    empty, one without arcs) and component structure."""
    star = gen.from_edges(40, [(0, i) for i in range(1, 40)], "star40")
    pairs = gen.from_edges(70, [(2 * i, 2 * i + 1) for i in range(20)], "pairs")  # + isolated
    return [gen.grid2d(37, 29), gen.rmat(12), star, gen.rgg(3001, 5), pairs,
            gen.from_edges(0, [], "empty"), gen.random_graph(45, 0.05, 3), gen.rgg(999, 8),
            gen.from_edges(33, [], "isolated33")]


def _check_members(Gs, shifts, cen, dis, cuts, offsets):
    for s, G in enumerate(Gs):
        lo, hi = offsets[s], offsets[s + 1]
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts[s])
        assert np.array_equal(cen[lo:hi], oc), f"member {s} ({G.name}): center"
        assert np.array_equal(dis[lo:hi], od), f"member {s} ({G.name}): dist"
        assert cuts[s] == oracle.oracle_cut_edges(G.row_ptr, G.col, oc), f"member {s}: cut"


@pytest.mark.parametrize("placement", ["device", "host"])
def test_union_of_mixed_members(ldd, cuda, placement):
    Gs = _members()
    betas = [0.02, 0.1, 0.5, 0.05, 0.3, 0.2, 1.0, 0.07, 0.1]
    shifts = [gen.shifts(G.n, b, 40 + i) for i, (G, b) in enumerate(zip(Gs, betas))]
    mem = [ldd.LddGraph(G.row_ptr, G.col) for G in Gs]
    u = ldd.LddUnion(mem)
    for m in mem:  # the union holds its own copies
        m.close()
    assert u.k == len(Gs) and u.total == sum(G.n for G in Gs)
    cat = np.concatenate(shifts)
    if placement == "device":
        c = torch.empty(u.total, dtype=torch.int32, device=cuda)
        d = torch.empty(u.total, dtype=torch.int32, device=cuda)
        cuts = u.decompose(betas, torch.from_numpy(cat).to(cuda), c, d)
        cen, dis = c.cpu().numpy(), d.cpu().numpy()
    else:
        cen = np.empty(u.total, np.int32)
        dis = np.empty(u.total, np.int32)
        cuts = u.decompose(betas, cat, cen, dis)
    _check_members(Gs, shifts, cen, dis, cuts, u.offsets)
    # a second call with other shifts on the same union
    shifts2 = [gen.shifts(G.n, b, 90 + i) for i, (G, b) in enumerate(zip(Gs, betas))]
    cuts2 = u.decompose(betas, np.concatenate(shifts2), cen, dis)
    _check_members(Gs, shifts2, cen, dis, cuts2, u.offsets)
    u.close()


def test_union_of_one_graph_many_seeds(ldd, cuda):
    """k shift vectors of one graph (the tree-embedding use): the same member
    handle k times."""
    G = gen.rmat(14)
    g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda))
    k = 12
    u = ldd.LddUnion([g] * k)
    shifts = [gen.shifts(G.n, 0.1, 1 + i) for i in range(k)]
    c = torch.empty(u.total, dtype=torch.int32, device=cuda)
    d = torch.empty(u.total, dtype=torch.int32, device=cuda)
    cuts = u.decompose([0.1] * k, torch.from_numpy(np.concatenate(shifts)).to(cuda), c, d)
    _check_members([G] * k, shifts, c.cpu().numpy(), d.cpu().numpy(), cuts, u.offsets)
    # identical to separate calls on the member graph
    c1 = torch.empty(G.n, dtype=torch.int32, device=cuda)
    d1 = torch.empty(G.n, dtype=torch.int32, device=cuda)
    for i in (0, k - 1):
        g.decompose(0.1, torch.from_numpy(shifts[i]).to(cuda), c1, d1)
        assert torch.equal(c1, c[i * G.n:(i + 1) * G.n]) and torch.equal(d1, d[i * G.n:(i + 1) * G.n])
        assert g.cut_edges(c1) == cuts[i]
    u.close()
    g.close()


def test_union_of_random_geometric_graphs(ldd, cuda):
    """A reduced copy of the 1,024-graph batch: 48 random geometric graphs,
    n uniform on [1,000, 20,000], beta uniform on [0.02, 0.5)."""
    batch = gen.rgg_batch(48, 1000, 20000, master_seed=5)
    Gs = [b[0] for b in batch]
    mem = [ldd.LddGraph(G.row_ptr, G.col, validate=False) for G in Gs]
    u = ldd.LddUnion(mem)
    cen = np.empty(u.total, np.int32)
    dis = np.empty(u.total, np.int32)
    cuts = u.decompose([b[1] for b in batch], np.concatenate([b[2] for b in batch]), cen, dis)
    _check_members(Gs, [b[2] for b in batch], cen, dis, cuts, u.offsets)
    st = u.stats()
    assert st["launches"] > 0 and st["rounds"] > 0
    u.close()
    for m in mem:
        m.close()


def test_union_errors(ldd, cuda):
    G = gen.grid2d(10, 10)
    g = ldd.LddGraph(G.row_ptr, G.col)
    u = ldd.LddUnion([g, g])
    good = gen.shifts(G.n, 0.2, 1)
    bad = good.copy()
    bad[3] = -1.0
    cen = np.empty(2 * G.n, np.int32)
    dis = np.empty(2 * G.n, np.int32)
    with pytest.raises(ldd.LddError) as e:
        u.decompose([0.2, 0.2], np.concatenate([good, bad]), cen, dis)
    assert e.value.status == ldd.LDD_ERR_ARG
    with pytest.raises(ldd.LddError):
        u.decompose([0.2, float("nan")], np.concatenate([good, good]), cen, dis)
    with pytest.raises(ValueError):
        u.decompose([0.2], np.concatenate([good, good]), cen, dis)
    # a union is not a plain graph, nor a member
    with pytest.raises(ldd.LddError) as e:
        ldd.ldd_decompose(u.handle, 0.2, np.concatenate([good, good]), cen, dis, 2 * G.n)
    assert e.value.status == ldd.LDD_ERR_ARG
    with pytest.raises(ldd.LddError):
        ldd.LddUnion([u])
    # still usable after the failures
    cuts = u.decompose([0.2, 0.2], np.concatenate([good, good]), cen, dis)
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, good)
    assert np.array_equal(cen[:G.n], oc) and np.array_equal(cen[G.n:], oc)
    assert cuts[0] == cuts[1] == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    u.close()
    g.close()


def test_union_of_many_members(ldd, cuda):
    """More members than the round loop keeps per-member floors for in shared
    memory (4,096): the global per-member table path.  Every member is a
    connected 6x7 grid (42 vertices, so the round loop handles it), plus one
    larger R-MAT member; betas and seeds vary per member."""
    small = gen.grid2d(6, 7)
    big = gen.rmat(12)
    gs = ldd.LddGraph(small.row_ptr, small.col)
    gb = ldd.LddGraph(big.row_ptr, big.col)
    k = 4300
    members = [gs] * k + [gb]
    Gs = [small] * k + [big]
    rng = np.random.default_rng(8)
    betas = [float(x) for x in rng.uniform(0.05, 1.0, k + 1)]
    shifts = [gen.shifts(G.n, b, 7000 + i) for i, (G, b) in enumerate(zip(Gs, betas))]
    u = ldd.LddUnion(members)
    cen = torch.empty(u.total, dtype=torch.int32, device=cuda)
    dis = torch.empty(u.total, dtype=torch.int32, device=cuda)
    cuts = u.decompose(betas, torch.from_numpy(np.concatenate(shifts)).to(cuda), cen, dis)
    _check_members(Gs, shifts, cen.cpu().numpy(), dis.cpu().numpy(), cuts, u.offsets)
    assert u.stats()["rounds"] > 0
    u.close()
    gs.close()
    gb.close()
