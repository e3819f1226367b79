"""The Las Vegas loop of Theorem 1.2's proof (ldd_decompose_retry): the first
shift vector whose decomposition meets both bounds is accepted, and the
returned labels, cut count and radius are that decomposition's, exactly."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu


def _truth(G, shifts):
    out = []
    for sh in shifts:
        c, d = oracle.oracle_ldd(G.row_ptr, G.col, sh)
        out.append((c, d, oracle.oracle_cut_edges(G.row_ptr, G.col, c), int(d.max())))
    return out


@pytest.mark.parametrize("device", [False, True])
def test_retry_accepts_first_meeting_bounds(ldd, cuda, device):
    G = gen.grid2d(48, 40)
    shifts = [gen.shifts(G.n, 0.1, 300 + i) for i in range(6)]
    truth = _truth(G, shifts)
    cuts = [t[2] for t in truth]
    rads = [t[3] for t in truth]
    # bounds that the first tries miss: the smallest radius, and any cut
    max_radius = min(rads)
    max_cut = max(cuts)
    want = next(i for i in range(6) if cuts[i] <= max_cut and rads[i] <= max_radius)
    g = ldd.LddGraph(G.row_ptr, G.col)
    if device:
        sh = [torch.from_numpy(x).to(cuda) for x in shifts]
        c = torch.empty(G.n, dtype=torch.int32, device=cuda)
        d = torch.empty(G.n, dtype=torch.int32, device=cuda)
    else:
        sh = shifts
        c = np.empty(G.n, np.int32)
        d = np.empty(G.n, np.int32)
    acc, cut, rad = g.decompose_retry(0.1, sh, max_cut, max_radius, c, d)
    c = c.cpu().numpy() if device else c
    d = d.cpu().numpy() if device else d
    assert acc == want and cut == cuts[want] and rad == rads[want]
    assert np.array_equal(c, truth[want][0]) and np.array_equal(d, truth[want][1])
    # nothing meets a cut bound of -1: the last try is returned
    acc, cut, rad = g.decompose_retry(0.1, shifts, -1, 10 ** 6, np.empty(G.n, np.int32),
                                      np.empty(G.n, np.int32))
    assert acc == -1 and cut == cuts[-1] and rad == rads[-1]
    g.close()


def test_retry_default_bounds(ldd, cuda):
    """With Definition 1.1's cut bound (beta m) and radius 2 ln(n) / beta, the
    first draw is accepted on a grid (Lemma 3.2, Corollary 3.5)."""
    G = gen.grid2d(200, 150)
    beta = 0.05
    max_cut, max_radius = ldd.default_bounds(G.n, G.m, beta)
    shifts = [gen.shifts(G.n, beta, 9 + i) for i in range(3)]
    g = ldd.LddGraph(G.row_ptr, G.col)
    c = np.empty(G.n, np.int32)
    d = np.empty(G.n, np.int32)
    acc, cut, rad = g.decompose_retry(beta, shifts, max_cut, max_radius, c, d)
    assert acc == 0 and cut <= max_cut and rad <= max_radius
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts[0])
    assert np.array_equal(c, oc) and np.array_equal(d, od)
    g.close()
