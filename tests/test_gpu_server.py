"""The request server (ldd_server_*): continuous batching must return, for
every request, exactly what the request gives alone -- the oracle's answer and
ldd_decompose's output on the same graph, bit for bit -- whatever else shares
its batch; admission must respect the workspace capacities; a bad request
fails alone."""
from __future__ import annotations

import threading

import numpy as np
import pytest
import torch

import ldd_gen as gen
import oracle

pytestmark = pytest.mark.gpu


def _graphs():
    return [gen.grid2d(64, 48), gen.rmat(12), gen.rgg(5000, 3), gen.rmat(10),
            gen.from_edges(50, [(0, 1), (2, 3), (3, 4)], "sparse50"), gen.grid2d(17, 5),
            gen.grid2d(700, 700)]


def _alone(ldd, G, beta, shifts):
    g = ldd.LddGraph(G.row_ptr, G.col)
    c = np.empty(G.n, np.int32)
    d = np.empty(G.n, np.int32)
    g.decompose(beta, shifts, c, d)
    cut = g.cut_edges(c)
    g.close()
    return c, d, cut


def _submit_all(srv, gs, Gs, reqs):
    """Inputs first, then every submit in a tight loop (so that requests queue
    while earlier ones run)."""
    prepared = []
    for gi, beta, seed in reqs:
        G = Gs[gi]
        sh = torch.from_numpy(gen.shifts(G.n, beta, seed)).pin_memory()
        prepared.append((gi, beta, seed, sh, np.full(G.n, -1, np.int32),
                         np.full(G.n, -1, np.int32), np.zeros(1, np.int64)))
    out = []
    for gi, beta, seed, sh, c, d, cut in prepared:
        t = srv.submit(gs[gi], beta, sh, c, d, cut)
        out.append((t, gi, beta, seed, sh, c, d, cut))
    return out


def test_server_mix_equals_alone(ldd, cuda):
    Gs = _graphs()
    gs = [ldd.LddGraph(G.row_ptr, G.col) for G in Gs]
    rng = np.random.default_rng(4)
    betas = [0.02, 0.05, 0.1, 0.2, 0.5]
    # a long request first (hundreds of rounds), so that the rest queue behind it
    reqs = [(len(Gs) - 1, 0.005, 999)] + [
        (int(rng.integers(len(Gs) - 1)), betas[int(rng.integers(5))], 1000 + i) for i in range(47)]
    srv = ldd.LddServer(2 << 30, max_batch=16, slots=1)
    subs = _submit_all(srv, gs, Gs, reqs)
    sizes = []
    for t, gi, beta, seed, sh, c, d, cut in subs:
        info = srv.wait(t)
        assert info["status"] == 0
        assert info["submit_us"] <= info["start_us"] <= info["end_us"]
        sizes.append(info["batch_size"])
        G = Gs[gi]
        oc, od = oracle.oracle_ldd(G.row_ptr, G.col, sh.numpy())
        assert np.array_equal(c, oc) and np.array_equal(d, od), f"request {t} on {G.name}"
        assert cut[0] == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
        ac, ad, acut = _alone(ldd, G, beta, sh.numpy())
        assert np.array_equal(c, ac) and np.array_equal(d, ad) and cut[0] == acut
    assert max(sizes) > 1  # requests were batched
    srv.close()
    for g in gs:
        g.close()


def test_server_admission_caps_and_bad_request(ldd, cuda):
    Gs = [gen.grid2d(32, 32), gen.grid2d(64, 64)]
    gs = [ldd.LddGraph(G.row_ptr, G.col) for G in Gs]
    # a workspace of 2,048 vertices: the 64x64 grid never fits, two 32x32 do
    srv = ldd.LddServer(1 << 30, max_batch=8, slots=1, max_vertices=2048, max_arcs=1 << 20)
    sh_big = gen.shifts(Gs[1].n, 0.1, 1)
    with pytest.raises(ldd.LddError) as e:
        srv.submit(gs[1], 0.1, sh_big, np.empty(Gs[1].n, np.int32), np.empty(Gs[1].n, np.int32))
    assert e.value.status == ldd.LDD_ERR_RANGE
    assert srv.footprint(gs[1]) > srv.footprint(gs[0]) > 0
    good = [gen.shifts(Gs[0].n, 0.1, 10 + i) for i in range(5)]
    bad = good[2].copy()
    bad[7] = float("nan")
    shifts = [good[0], good[1], bad, good[3], good[4]]
    outs = [(np.empty(Gs[0].n, np.int32), np.empty(Gs[0].n, np.int32)) for _ in shifts]
    ts = [srv.submit(gs[0], 0.1, sh, c, d) for sh, (c, d) in zip(shifts, outs)]
    infos = []
    for i, t in enumerate(ts):
        if i == 2:
            with pytest.raises(ldd.LddError) as e:
                srv.wait(t)
            assert e.value.status == ldd.LDD_ERR_ARG
            continue
        infos.append(srv.wait(t))
        oc, od = oracle.oracle_ldd(Gs[0].row_ptr, Gs[0].col, shifts[i])
        assert np.array_equal(outs[i][0], oc) and np.array_equal(outs[i][1], od)
    assert all(inf["batch_size"] <= 2 for inf in infos)  # 2 x 1,024 vertices per batch
    srv.close()
    for g in gs:
        g.close()


def test_server_one_at_a_time_and_threads(ldd, cuda):
    Gs = _graphs()[:4]
    gs = [ldd.LddGraph(G.row_ptr, G.col) for G in Gs]
    reqs = [(i % len(Gs), 0.1, 77 + i) for i in range(12)]
    for one in (True, False):
        srv = ldd.LddServer(1 << 30, max_batch=8, slots=2, one_at_a_time=one)
        results = {}

        def client(part):
            subs = _submit_all(srv, gs, Gs, part)
            for t, gi, beta, seed, sh, c, d, cut in subs:
                info = srv.wait(t)
                results[(gi, seed)] = (sh.numpy(), c, d, cut[0], info)

        th = [threading.Thread(target=client, args=(reqs[j::3],)) for j in range(3)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        assert len(results) == len(reqs)
        for (gi, seed), (sh, c, d, cut, info) in results.items():
            G = Gs[gi]
            oc, od = oracle.oracle_ldd(G.row_ptr, G.col, sh)
            assert np.array_equal(c, oc) and np.array_equal(d, od)
            assert cut == oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
            if one:
                assert info["batch_size"] == 1
        srv.close()
    for g in gs:
        g.close()


def test_server_slots_overlap_exact(ldd, cuda):
    """Three workers: their batches run side by side on the device, round
    loops ordered by the gate; every request still equals its result alone."""
    Gs = _graphs()
    gs = [ldd.LddGraph(G.row_ptr, G.col) for G in Gs]
    rng = np.random.default_rng(9)
    betas = [0.02, 0.1, 0.5]
    big = len(Gs) - 1
    reqs = [(big, 0.005, 500)] + [
        (int(rng.integers(len(Gs))), betas[int(rng.integers(3))], 600 + i) for i in range(35)]
    srv = ldd.LddServer(2 << 30, max_batch=4, slots=3)
    subs = _submit_all(srv, gs, Gs, reqs)
    infos = []
    for t, gi, beta, seed, sh, c, d, cut in subs:
        info = srv.wait(t)
        infos.append(info)
        G = Gs[gi]
        if gi == big:
            oc, od, ocut = _alone(ldd, G, beta, sh.numpy())
        else:
            oc, od = oracle.oracle_ldd(G.row_ptr, G.col, sh.numpy())
            ocut = oracle.oracle_cut_edges(G.row_ptr, G.col, oc)
        assert np.array_equal(c, oc) and np.array_equal(d, od), (gi, beta, seed)
        assert cut[0] == ocut
    # batches of different workers were in flight at the same time
    spans = {}
    for inf in infos:
        spans[inf["batch_id"]] = (inf["start_us"], inf["end_us"])
    iv = sorted(spans.values())
    assert any(iv[i + 1][0] < iv[i][1] for i in range(len(iv) - 1)), iv[:8]
    srv.close()
    for g in gs:
        g.close()
