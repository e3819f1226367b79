"""ORACLE -- test infrastructure only.

Algorithm 2 of Miller, Peng, Xu (2013) written out literally, for tiny graphs:

    for every vertex v, S_u gets v for the u minimising
        dist_{-delta}(u, v) = dist(u, v) - delta_u            (Eq. (1))
    breaking ties lexicographically (smaller vertex id first).

``dist`` is computed by a plain BFS from every vertex (all pairs), and the
shifted distance is evaluated in exact rational arithmetic
(``fractions.Fraction`` represents each FP64 shift exactly), so this shares no
reasoning with the integer/fraction label split used elsewhere.  Vertices in
other connected components are at infinite distance and never compete.
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction


def bfs_distances(n, row_ptr, col, src):
    dist = [None] * n
    dist[src] = 0
    q = deque([src])
    while q:
        v = q.popleft()
        for e in range(int(row_ptr[v]), int(row_ptr[v + 1])):
            w = int(col[e])
            if dist[w] is None:
                dist[w] = dist[v] + 1
                q.append(w)
    return dist


def brute_ldd(row_ptr, col, delta):
    """(center, dist) lists by all-pairs BFS + exact argmin over (shifted distance, id)."""
    n = len(row_ptr) - 1
    apsp = [bfs_distances(n, row_ptr, col, u) for u in range(n)]
    shift = [Fraction(float(d)) for d in delta]
    center, dist = [], []
    for v in range(n):
        best = None
        for u in range(n):
            d = apsp[u][v]
            if d is None:
                continue
            cand = (Fraction(d) - shift[u], u)
            if best is None or cand < best:
                best = cand
        center.append(best[1])
        dist.append(apsp[best[1]][v])
    return center, dist


def brute_ldd_ranked(row_ptr, col, levels, perm):
    """The permutation variant (Section 4: a random permutation stands in for
    the fractional parts) written out: v joins the u minimising
    (dist(u, v) - levels[u], perm[u]), all integers."""
    n = len(row_ptr) - 1
    apsp = [bfs_distances(n, row_ptr, col, u) for u in range(n)]
    center, dist = [], []
    for v in range(n):
        best = None
        for u in range(n):
            d = apsp[u][v]
            if d is None:
                continue
            cand = (d - int(levels[u]), int(perm[u]))
            if best is None or cand < best:
                best = (cand[0], cand[1], u)
        center.append(best[2])
        dist.append(apsp[best[2]][v])
    return center, dist


def brute_cut_edges(row_ptr, col, center):
    """Edges {v, w} (each counted once, v < w) with endpoints in different pieces."""
    n = len(row_ptr) - 1
    cut = 0
    for v in range(n):
        for e in range(int(row_ptr[v]), int(row_ptr[v + 1])):
            w = int(col[e])
            if v < w and center[v] != center[w]:
                cut += 1
    return cut


def brute_block_decompose(row_ptr, col, shifts_list):
    """Blocks by repeated decomposition, literally: keep a list of the edges
    not yet in a block (as input arc ids), rebuild the graph of those edges,
    decompose it by ``brute_ldd``, move the edges inside a piece to the
    current block, repeat while edges are left.  Same outputs as
    ``oracle.oracle_block_decompose`` (lists instead of arrays)."""
    n = len(row_ptr) - 1
    arcs = []  # (v, w, input arc id)
    for v in range(n):
        for e in range(int(row_ptr[v]), int(row_ptr[v + 1])):
            arcs.append((v, int(col[e]), e))
    block = [-1] * len(arcs)
    left = list(arcs)
    remaining = [sum(1 for v, w, _ in left if v < w)]
    centers, dists = [], []
    for i, sh in enumerate(shifts_list):
        if not left:
            break
        rows = [[] for _ in range(n)]
        for v, w, _ in left:
            rows[v].append(w)
        rp, cl = [0], []
        for v in range(n):
            cl.extend(rows[v])
            rp.append(len(cl))
        c, d = brute_ldd(rp, cl, sh)
        nxt = []
        for v, w, e in left:
            if c[v] == c[w]:
                block[e] = i
            else:
                nxt.append((v, w, e))
        left = nxt
        remaining.append(sum(1 for v, w, _ in left if v < w))
        centers.append(c)
        dists.append(d)
    return centers, dists, block, remaining
