"""ldd_decompose_batch: k pipelined decompositions must give exactly what k
separate ldd_decompose + ldd_cut_edges calls give, whatever mix of host and
device buffers, and stop cleanly at a failing item."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu


def _pinned(a: np.ndarray) -> torch.Tensor:
    t = torch.empty(a.shape, dtype=torch.from_numpy(a).dtype, pin_memory=True)
    t.copy_(torch.from_numpy(a))
    return t


def test_batch_matches_single_calls_and_oracle(ldd, cuda):
    G = gen.rmat(13)
    betas = [0.02, 0.1, 0.5, 0.1, 1.0]
    shifts = [gen.shifts(G.n, b, 100 + i) for i, b in enumerate(betas)]
    # mixed placement: pinned host, device, pageable host
    sh = [_pinned(shifts[0]), torch.from_numpy(shifts[1]).to(cuda), shifts[2],
          _pinned(shifts[3]), torch.from_numpy(shifts[4]).to(cuda)]
    cen = [torch.empty(G.n, dtype=torch.int32, pin_memory=True),
           torch.empty(G.n, dtype=torch.int32, device=cuda),
           np.empty(G.n, dtype=np.int32),
           torch.empty(G.n, dtype=torch.int32, device=cuda),
           torch.empty(G.n, dtype=torch.int32, pin_memory=True)]
    dis = [torch.empty(G.n, dtype=torch.int32, pin_memory=True),
           np.empty(G.n, dtype=np.int32),
           torch.empty(G.n, dtype=torch.int32, device=cuda),
           torch.empty(G.n, dtype=torch.int32, device=cuda),
           torch.empty(G.n, dtype=torch.int32, pin_memory=True)]
    g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda))
    cuts = g.decompose_batch(betas, sh, cen, dis)
    as_np = lambda x: x.cpu().numpy() if hasattr(x, "cpu") else x
    for i, b in enumerate(betas):
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts[i])
        assert np.array_equal(as_np(cen[i]), oc), f"item {i}: center"
        assert np.array_equal(as_np(dis[i]), od), f"item {i}: dist"
        assert cuts[i] == oracle.oracle_cut_edges(G.row_ptr, G.col, oc), f"item {i}: cut"
    # the batch leaves the graph usable for single calls, and a second batch agrees
    c1 = np.empty(G.n, dtype=np.int32)
    d1 = np.empty(G.n, dtype=np.int32)
    g.decompose(betas[0], shifts[0], c1, d1)
    assert np.array_equal(c1, as_np(cen[0]))
    again = g.decompose_batch(betas[:2], [shifts[0], shifts[1]],
                              [np.empty(G.n, np.int32) for _ in range(2)],
                              [np.empty(G.n, np.int32) for _ in range(2)])
    assert again == cuts[:2]
    g.close()


@pytest.mark.parametrize("where", ["host", "device"])
def test_batch_with_fallback_items(ldd, cuda, where):
    """Items that need the exact rank path or a larger start-bucket table
    inside a pipelined batch: they are redone alone after the others, and the
    items queued behind them (which start from the floor counts the failed
    item left) are still exact."""
    G = gen.grid2d(40, 30)
    rng = np.random.default_rng(9)
    crowded = rng.random(G.n) * 2.0 ** -33 + rng.integers(0, 3, G.n)  # exact path
    huge = gen.shifts(G.n, 0.1, 3)
    huge[7] = 5000.5                                                    # A + 2 > n + 2
    normal = gen.shifts(G.n, 0.1, 4)
    other = gen.shifts(G.n, 0.3, 5)
    items = [normal, crowded, other, crowded, huge, normal, other]
    betas = [0.1, 0.1, 0.3, 0.1, 0.1, 0.1, 0.3]
    g = ldd.LddGraph(G.row_ptr, G.col)
    if where == "host":
        sh = items
        cen = [np.empty(G.n, np.int32) for _ in items]
        dis = [np.empty(G.n, np.int32) for _ in items]
    else:
        sh = [torch.from_numpy(x).to(cuda) for x in items]
        cen = [torch.empty(G.n, dtype=torch.int32, device=cuda) for _ in items]
        dis = [torch.empty(G.n, dtype=torch.int32, device=cuda) for _ in items]
    cuts = g.decompose_batch(betas, sh, cen, dis)
    for i, shifts in enumerate(items):
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts)
        c = cen[i] if where == "host" else cen[i].cpu().numpy()
        d = dis[i] if where == "host" else dis[i].cpu().numpy()
        assert np.array_equal(c, oc) and np.array_equal(d, od), f"item {i}"
        assert cuts[i] == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    g.close()


def test_batch_stops_at_a_bad_item(ldd, cuda):
    G = gen.grid2d(20, 20)
    good = gen.shifts(G.n, 0.2, 1)
    bad = good.copy()
    bad[5] = -1.0
    cen = [np.full(G.n, -7, np.int32) for _ in range(3)]
    dis = [np.full(G.n, -7, np.int32) for _ in range(3)]
    g = ldd.LddGraph(G.row_ptr, G.col)
    with pytest.raises(ldd.LddError) as e:
        g.decompose_batch([0.2] * 3, [good, bad, good], cen, dis)
    assert e.value.status == ldd.LDD_ERR_ARG
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, good)
    assert np.array_equal(cen[0], oc) and np.array_equal(dis[0], od)  # before the failure
    with pytest.raises(ldd.LddError):
        g.decompose_batch([0.2, float("nan")], [good, good], cen[:2], dis[:2])
    assert g.decompose_batch([], [], [], []) == []
    # still usable
    assert g.decompose_batch([0.2], [good], cen[:1], dis[:1]) == [
        oracle.oracle_cut_edges(G.row_ptr, G.col, oc)]
    g.close()


def test_batch_first_vector_uploaded_in_pieces(ldd, cuda):
    """A host shift vector of at least 2^20 entries at the head of a batch goes up
    in pieces, each ranked as it lands; every item must still equal the oracle."""
    G = gen.grid2d(1024, 1024)
    betas = [0.1, 0.3, 0.05]
    items = [gen.shifts(G.n, b, 40 + i) for i, b in enumerate(betas)]
    sh = [_pinned(x) for x in items]
    cen = [_pinned(np.zeros(G.n, np.int32)) for _ in items]
    dis = [_pinned(np.zeros(G.n, np.int32)) for _ in items]
    g = ldd.LddGraph(G.row_ptr, G.col)
    cuts = g.decompose_batch(betas, sh, cen, dis)
    for i, shifts in enumerate(items):
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts)
        assert np.array_equal(cen[i].numpy(), oc) and np.array_equal(dis[i].numpy(), od), f"item {i}"
        assert cuts[i] == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    g.close()


def test_batch_first_vector_in_pieces_needs_the_exact_rank(ldd, cuda):
    """The first host vector goes up in pieces; when its fractions are crowded
    (exact rank path) it is redone alone after the others, from the host copy."""
    G = gen.grid2d(1024, 1024)
    rng = np.random.default_rng(12)
    crowded = rng.random(G.n) * 2.0 ** -33 + rng.integers(0, 4, G.n)
    items = [crowded, gen.shifts(G.n, 0.2, 13)]
    sh = [_pinned(x) for x in items]
    cen = [_pinned(np.zeros(G.n, np.int32)) for _ in items]
    dis = [_pinned(np.zeros(G.n, np.int32)) for _ in items]
    g = ldd.LddGraph(G.row_ptr, G.col)
    cuts = g.decompose_batch([0.1, 0.2], sh, cen, dis)
    for i, shifts in enumerate(items):
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts)
        assert np.array_equal(cen[i].numpy(), oc) and np.array_equal(dis[i].numpy(), od), f"item {i}"
        assert cuts[i] == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    g.close()


@pytest.mark.parametrize("where", ["device", "host"])
def test_batch_cut_counts_in_waves(ldd, cuda, where):
    """With device outputs the cut counts of a batch are counted a wave of up to
    four labelings at a time (k = 5: a wave of four, then one of one); with host
    outputs one at a time.  Every count must equal the oracle's, with a hot
    table larger than the part a CTA keeps in shared memory (R-MAT 15: 32,768
    hot slots)."""
    G = gen.rmat(15)
    betas = [0.02, 0.1, 0.5, 0.2, 0.05]
    items = [gen.shifts(G.n, b, 70 + i) for i, b in enumerate(betas)]
    if where == "device":
        sh = [torch.from_numpy(x).to(cuda) for x in items]
        cen = [torch.empty(G.n, dtype=torch.int32, device=cuda) for _ in items]
        dis = [torch.empty(G.n, dtype=torch.int32, device=cuda) for _ in items]
    else:
        sh = items
        cen = [np.empty(G.n, np.int32) for _ in items]
        dis = [np.empty(G.n, np.int32) for _ in items]
    g = ldd.LddGraph(G.row_ptr, G.col)
    for k in (5, 4, 3, 2):
        cuts = g.decompose_batch(betas[:k], sh[:k], cen[:k], dis[:k])
        for i in range(k):
            oc, od = oracle.oracle_ldd(G.row_ptr, G.col, items[i])
            c = cen[i].cpu().numpy() if where == "device" else cen[i]
            assert np.array_equal(c, oc), f"k {k} item {i}: center"
            assert cuts[i] == oracle.oracle_cut_edges(G.row_ptr, G.col, oc), f"k {k} item {i}: cut"
    g.close()
