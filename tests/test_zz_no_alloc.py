"""ldd_cut_edges_noalloc: the cut count for callers that cannot allocate device
memory when they need it (a process whose framework allocator owns the whole
memory pool, or a latency-critical loop that cannot pay for cudaMalloc's
device-wide synchronisation).  It must give exactly what ldd_cut_edges gives,
call after call, although every call reuses the same fixed scratch array.

This file is named to run last; it also passes when run on its own.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu


def _labels(ldd, G, beta, seed, dev):
    g = ldd.LddGraph(torch.from_numpy(G.row_ptr).to(dev), torch.from_numpy(G.col).to(dev))
    c = torch.empty(G.n, dtype=torch.int32, device=dev)
    d = torch.empty(G.n, dtype=torch.int32, device=dev)
    g.decompose(beta, torch.from_numpy(gen.shifts(G.n, beta, seed)).to(dev), c, d)
    return g, c


@pytest.mark.parametrize("G,beta", [(gen.grid2d(96, 75), 0.1), (gen.rmat(13), 0.3),
                                    (gen.from_edges(5000, [(0, i) for i in range(1, 4999)], "star"), 0.2)],
                         ids=["grid2d", "rmat13", "star_with_isolated"])
def test_noalloc_matches_cut_edges_twice(ldd, cuda, G, beta):
    g, center = _labels(ldd, G, beta, 7, cuda)
    expected = oracle.oracle_cut_edges(G.row_ptr, G.col, center.cpu().numpy())
    assert g.cut_edges(center) == expected
    rp = torch.from_numpy(G.row_ptr).to(cuda)
    col = torch.from_numpy(G.col).to(cuda)
    first = ldd.ldd_cut_edges_noalloc(G.n, G.nnz, rp, col, center)
    second = ldd.ldd_cut_edges_noalloc(G.n, G.nnz, rp, col, center)  # scratch reused
    assert first == expected and second == expected
    # device-side output and an explicit stream give the same count
    out = torch.full((1,), -1, dtype=torch.int64, device=cuda)
    s = torch.cuda.Stream()
    lib = ctypes.CDLL(ldd.library_path())
    lib.ldd_cut_edges_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int64] + [ctypes.c_void_p] * 5
    rc = lib.ldd_cut_edges_noalloc(G.n, G.nnz, rp.data_ptr(), col.data_ptr(), center.data_ptr(),
                                   out.data_ptr(), s.cuda_stream)
    assert rc == ldd.LDD_OK and int(out.item()) == expected
    # a different labelling right after: nothing left over from the last call
    other = torch.arange(G.n, dtype=torch.int32, device=cuda)
    assert ldd.ldd_cut_edges_noalloc(G.n, G.nnz, rp, col, other) == G.m
    assert oracle.oracle_cut_edges(G.row_ptr, G.col, other.cpu().numpy()) == G.m
    g.close()


def test_noalloc_rejects_what_it_cannot_do(ldd, cuda):
    G = gen.grid2d(10, 10)
    rp = torch.from_numpy(G.row_ptr).to(cuda)
    col = torch.from_numpy(G.col).to(cuda)
    c = torch.zeros(G.n, dtype=torch.int32, device=cuda)
    with pytest.raises(ldd.LddError) as e:  # beyond the 2^27-arc scratch limit
        ldd.ldd_cut_edges_noalloc(G.n, (1 << 27) + 1, rp.data_ptr(), col.data_ptr(), c)
    assert e.value.status == ldd.LDD_ERR_RANGE
    with pytest.raises(ldd.LddError) as e:  # host inputs would need a device copy
        ldd.ldd_cut_edges_noalloc(G.n, G.nnz, G.row_ptr, G.col, c)
    assert e.value.status == ldd.LDD_ERR_ARG
    assert ldd.ldd_cut_edges_noalloc(G.n, 0, rp, col[:0], c) == 0


def test_noalloc_rejects_memory_of_another_gpu(ldd, cuda):
    """Inputs on a second GPU are refused before any launch (only where the
    machine has one: nothing runs on the second device)."""
    if torch.cuda.device_count() < 2:
        pytest.skip("one CUDA device")
    G = gen.grid2d(10, 10)
    other = torch.device("cuda", 1)
    rp = torch.from_numpy(G.row_ptr).to(other)
    col = torch.from_numpy(G.col).to(other)
    c = torch.zeros(G.n, dtype=torch.int32, device=other)
    with torch.cuda.device(0):
        with pytest.raises(ldd.LddError) as e:
            ldd.ldd_cut_edges_noalloc(G.n, G.nnz, rp, col, c)
    assert e.value.status == ldd.LDD_ERR_ARG
