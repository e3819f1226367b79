"""Seeded input generators (CPU only): graph shapes of the named workloads,
CSR invariants, determinism, and the distribution of the shifts."""
from __future__ import annotations

import math

import numpy as np
import pytest

import ldd_gen as gen


def _check_csr(G):
    rp, col = G.row_ptr, G.col
    assert rp[0] == 0 and rp[-1] == G.nnz and (np.diff(rp) >= 0).all()
    assert ((col >= 0) & (col < G.n)).all()
    src = np.repeat(np.arange(G.n), np.diff(rp))
    assert not (src == col).any(), "self-loop"
    fwd = set(zip(src.tolist(), col.tolist()))
    assert len(fwd) == G.nnz, "repeated arc"
    assert all((w, v) in fwd for v, w in fwd), "asymmetric"
    for v in range(G.n):
        row = col[rp[v]:rp[v + 1]]
        assert (np.diff(row) > 0).all(), "row not ascending"


def test_grid2d_256_matches_workload_sizes():
    G = gen.grid2d(256, 256)
    assert (G.n, G.m, G.nnz) == (65536, 130560, 261120)
    deg = np.diff(G.row_ptr)
    assert deg.min() == 2 and deg.max() == 4


def test_grid3d_256_size_formula():
    lib = gen._load()
    assert lib.ldd_grid3d_nnz(256, 256, 256) // 2 == 50135040


@pytest.mark.parametrize("G", [gen.grid2d(7, 5), gen.grid3d(4, 3, 5), gen.rmat(9), gen.rgg(800, 2)],
                         ids=["grid2d", "grid3d", "rmat9", "rgg"])
def test_csr_invariants(G):
    _check_csr(G)


def test_grid_neighbours():
    G = gen.grid2d(5, 4)
    v = 1 * 5 + 2  # (x=2, y=1)
    assert list(G.col[G.row_ptr[v]:G.row_ptr[v + 1]]) == [2, 6, 8, 12]
    G3 = gen.grid3d(3, 3, 3)
    assert list(G3.col[G3.row_ptr[13]:G3.row_ptr[14]]) == [4, 10, 12, 14, 16, 22]


def test_rmat_deterministic_and_seeded():
    a, b, c = gen.rmat(12, seed=7), gen.rmat(12, seed=7), gen.rmat(12, seed=8)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert not np.array_equal(a.col[:1000], c.col[:1000])


def test_rmat_skew():
    """R-MAT with a = 0.57 concentrates edges on low ids: vertex 0 is the hub."""
    G = gen.rmat(14)
    deg = np.diff(G.row_ptr)
    assert deg[0] == deg.max() and deg[0] > 50 * deg.mean()
    assert (deg == 0).sum() > 0.2 * G.n  # many isolated vertices, as expected of R-MAT


def test_rgg_mean_degree():
    G = gen.rgg(20000, 5)
    # boundary effects lower the mean slightly below the target 8
    assert 7.0 < G.nnz / G.n < 8.2


@pytest.mark.parametrize("ctr,key,expected", [
    ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
    ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
    ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
     [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
], ids=["zeros", "ones", "pi"])
def test_philox_known_answers(ctr, key, expected):
    """Philox4x32-10 against the known-answer vectors published with the
    Random123 library (Salmon et al., SC'11): counter, key -> four words.  The
    third case takes its counter and key from the hexadecimal digits of pi."""
    got = [int(x) for x in gen.philox4x32_10(ctr, key)]
    assert got == expected, [hex(x) for x in got]


def test_philox_counter_and_key_sensitivity():
    base = gen.philox4x32_10([0, 0, 0, 0], [1, 0])
    assert not np.array_equal(base, gen.philox4x32_10([1, 0, 0, 0], [1, 0]))
    assert not np.array_equal(base, gen.philox4x32_10([0, 0, 0, 0], [2, 0]))
    assert not np.array_equal(base, gen.philox4x32_10([0, 0, 0, 1], [1, 0]))
    words = gen.philox_stream(1, 0, 4)
    assert np.array_equal(words[0], base)


def test_philox_uniform_bytes():
    """Chi-square of the byte histogram of 2^20 words (4 MiB)."""
    from scipy import stats

    w = gen.philox_stream(12345, 0, 1 << 18).reshape(-1)
    counts = np.bincount(w.view(np.uint8), minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4
    bits = np.unpackbits(w.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 1e-3


def test_uniforms_open_closed_interval():
    u = gen.uniforms(1 << 20, 3)
    assert (u > 0).all() and (u <= 1).all()
    assert abs(u.mean() - 0.5) < 2e-3


@pytest.mark.parametrize("beta", [0.02, 0.1, 0.5, 3.0])
def test_shifts_are_exponential(beta):
    """delta = -ln(U)/beta has CDF 1 - exp(-beta x) (Section 2)."""
    from scipy import stats

    d = gen.shifts(200000, beta, 11)
    assert (d >= 0).all() and not np.signbit(d).any()
    assert stats.kstest(d, "expon", args=(0, 1.0 / beta)).pvalue > 1e-3
    assert abs(d.mean() * beta - 1.0) < 0.01


def test_shift_counter_layout():
    """delta_u depends on (seed, u) only: a prefix of a longer draw is the shorter draw."""
    a = gen.shifts(1000, 0.1, 5)
    b = gen.shifts(5000, 0.1, 5)
    assert np.array_equal(a, b[:1000])
    w = gen.philox_stream(5, 0, 1000)
    u = ((w[:, 0].astype(np.uint64) << np.uint64(32)) | w[:, 1]) >> np.uint64(11)
    U = (u.astype(np.float64) + 1.0) * 2.0 ** -53
    assert np.array_equal(gen.uniforms(1000, 5), U)
    assert np.allclose(a, -np.log(U) / 0.1, rtol=1e-15, atol=0)


def test_order_statistics_fact_2_1():
    """Fact 2.1: the gap X_(n) - X_(n-1) of n i.i.d. Exp(beta) is Exp(beta)."""
    from scipy import stats

    n, beta = 200, 0.5
    gaps = []
    for s in range(3000):
        d = np.sort(gen.shifts(n, beta, 50000 + s))
        gaps.append(d[-1] - d[-2])
    assert stats.kstest(gaps, "expon", args=(0, 1.0 / beta)).pvalue > 1e-3
    assert math.isclose(np.mean(gaps) * beta, 1.0, rel_tol=0.08)


def test_batch_members_recipe():
    """The batched workload's per-member sizes and betas: deterministic, inside
    their ranges, roughly uniform, and seeds master + i."""
    m = gen.batch_members(1024, 1000, 200000, 0.02, 0.5, 11)
    assert m == gen.batch_members(1024, 1000, 200000, 0.02, 0.5, 11)
    ns = np.array([x[0] for x in m])
    bs = np.array([x[1] for x in m])
    assert ns.min() >= 1000 and ns.max() <= 200000
    assert bs.min() >= 0.02 and bs.max() < 0.5
    assert abs(ns.mean() - 100500) < 0.05 * 100500  # uniform mean, 1024 draws
    assert abs(bs.mean() - 0.26) < 0.02
    assert [x[2] for x in m[:3]] == [11, 12, 13] and [x[3] for x in m[:3]] == [11, 12, 13]
    assert gen.batch_members(4, 5, 5, 0.1, 0.1, 3)[0][:2] == (5, 0.1)
