"""The timeout path of the bounded device-side waits.

The round loop ends every round at a grid-wide barrier and the fraction rank's
scans wait on their predecessor tiles.  Each wait gives up after a set number
of polls, records the failure, and the call returns LDD_ERR_TIMEOUT.  These
tests make the waits run out on purpose, without faulting or hanging
anything: the stall switches make a wait depend on a CTA or a tile that does
not exist, so it can only end by running out of its (small) poll budget.  The
same graph object must then decompose exactly as the oracle does once the
limits are back to normal.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu


def _graph(ldd, G, cuda):
    return ldd.LddGraph(torch.from_numpy(G.row_ptr).to(cuda), torch.from_numpy(G.col).to(cuda))


def _exact(ldd, g, G, shifts, cuda):
    c = torch.empty(G.n, dtype=torch.int32, device=cuda)
    d = torch.empty(G.n, dtype=torch.int32, device=cuda)
    g.decompose(0.1, torch.from_numpy(shifts).to(cuda), c, d)
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts)
    assert np.array_equal(c.cpu().numpy(), oc) and np.array_equal(d.cpu().numpy(), od)
    assert g.cut_edges(c) == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)


@pytest.mark.parametrize("which", ["barrier", "lookback"])
def test_wait_runs_out_then_graph_is_exact(ldd, cuda, which):
    G = gen.rmat(14)
    shifts = gen.shifts(G.n, 0.1, 3)
    g = _graph(ldd, G, cuda)
    c = torch.full((G.n,), -7, dtype=torch.int32, device=cuda)
    d = torch.empty(G.n, dtype=torch.int32, device=cuda)
    if which == "barrier":
        g.set_wait_limits(barrier_polls=2000, stall_barrier=1)
    else:
        g.set_wait_limits(lookback_polls=2000, stall_lookback=1)
    for _ in range(2):  # twice in a row: the failure leaves nothing behind
        with pytest.raises(ldd.LddError) as e:
            g.decompose(0.1, torch.from_numpy(shifts).to(cuda), c, d)
        assert e.value.status == ldd.LDD_ERR_TIMEOUT
    torch.cuda.synchronize()  # the context is still usable
    g.set_wait_limits()
    lim = g.wait_limits()
    assert lim["stall_barrier"] == 0 and lim["stall_lookback"] == 0
    assert lim["barrier_polls"] > 2000 and lim["lookback_polls"] > 2000
    _exact(ldd, g, G, shifts, cuda)
    g.close()


def test_batch_and_union_wait_runs_out(ldd, cuda):
    """The pipelined batch and a union's round loop give up the same way."""
    G = gen.rmat(13)
    sh = [gen.shifts(G.n, 0.1, s) for s in (1, 2)]
    g = _graph(ldd, G, cuda)
    g.set_wait_limits(barrier_polls=2000, stall_barrier=1)
    cs = [torch.empty(G.n, dtype=torch.int32, device=cuda) for _ in sh]
    ds = [torch.empty(G.n, dtype=torch.int32, device=cuda) for _ in sh]
    dsh = [torch.from_numpy(s).to(cuda) for s in sh]
    with pytest.raises(ldd.LddError) as e:
        g.decompose_batch([0.1, 0.1], dsh, cs, ds)
    assert e.value.status == ldd.LDD_ERR_TIMEOUT
    g.set_wait_limits()
    cuts = g.decompose_batch([0.1, 0.1], dsh, cs, ds)
    for s, c, d, cut in zip(sh, cs, ds, cuts):
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, s)
        assert np.array_equal(c.cpu().numpy(), oc) and np.array_equal(d.cpu().numpy(), od)
        assert cut == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    u = ldd.LddUnion([g, g])
    u.set_wait_limits(barrier_polls=2000, stall_barrier=1)
    cat = torch.cat(dsh)
    c2 = torch.empty(2 * G.n, dtype=torch.int32, device=cuda)
    d2 = torch.empty(2 * G.n, dtype=torch.int32, device=cuda)
    with pytest.raises(ldd.LddError) as e:
        u.decompose([0.1, 0.1], cat, c2, d2)
    assert e.value.status == ldd.LDD_ERR_TIMEOUT
    u.set_wait_limits()
    u.decompose([0.1, 0.1], cat, c2, d2)
    assert torch.equal(c2[:G.n], cs[0]) and torch.equal(c2[G.n:], cs[1])
    assert torch.equal(d2[:G.n], ds[0]) and torch.equal(d2[G.n:], ds[1])
    u.close()
    g.close()


def test_wait_limits_arguments(ldd, cuda):
    G = gen.grid2d(8, 8)
    g = _graph(ldd, G, cuda)
    with pytest.raises(ldd.LddError) as e:
        g.set_wait_limits(stall_barrier=2)
    assert e.value.status == ldd.LDD_ERR_ARG
    g.set_wait_limits(barrier_polls=123, lookback_polls=456)
    assert g.wait_limits() == {"barrier_polls": 123, "lookback_polls": 456, "stall_barrier": 0,
                               "stall_lookback": 0}
    g.close()
