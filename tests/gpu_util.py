"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs, and compare element by element."""
from __future__ import annotations

import numpy as np
import torch

import oracle


def run_gpu(ldd, G, shifts, beta=0.1, host=False, dev=None):
    """(center, dist, cut, stats) from libldd; host=True passes host buffers."""
    dev = dev or torch.device("cuda:0")
    if host:
        g = ldd.LddGraph(G.row_ptr, G.col, validate=True)
        center = np.empty(G.n, dtype=np.int32)
        dist = np.empty(G.n, dtype=np.int32)
        g.decompose(beta, np.ascontiguousarray(shifts), center, dist)
        cut = g.cut_edges(center)
    else:
        g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(dev), torch.from_numpy(G.col).to(dev),
                         validate=True)
        c_t = torch.empty(G.n, dtype=torch.int32, device=dev)
        d_t = torch.empty(G.n, dtype=torch.int32, device=dev)
        g.decompose(beta, torch.from_numpy(np.ascontiguousarray(shifts)).to(dev), c_t, d_t)
        cut = g.cut_edges(c_t)
        center, dist = c_t.cpu().numpy(), d_t.cpu().numpy()
    st = g.stats()
    g.close()
    return center, dist, cut, st


def assert_parity(ldd, G, shifts, beta=0.1, host=False):
    center, dist, cut, st = run_gpu(ldd, G, shifts, beta, host)
    oc, od = oracle.oracle_ldd(G.row_ptr, G.col, shifts)
    bad_c = np.flatnonzero(center != oc)
    bad_d = np.flatnonzero(dist != od)
    assert bad_c.size == 0, (f"{G.name}: center differs at {bad_c.size} vertices, first {bad_c[:5]}: "
                             f"gpu {center[bad_c[:5]]} oracle {oc[bad_c[:5]]}")
    assert bad_d.size == 0, (f"{G.name}: dist differs at {bad_d.size} vertices, first {bad_d[:5]}: "
                             f"gpu {dist[bad_d[:5]]} oracle {od[bad_d[:5]]}")
    ocut = oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
    assert cut == ocut, f"{G.name}: cut {cut} != oracle {ocut}"
    return center, dist, cut, st
