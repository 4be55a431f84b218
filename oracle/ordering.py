"""Oracle for the clique-peeling vertex ordering -- TEST INFRASTRUCTURE ONLY.

Plain Python, for small and medium graphs.  Section 6.2 of the paper orders
the vertices for compression by repeatedly finding a large clique with its
heuristic, removing it and starting again; the vertices then follow the
cliques in the order found, each clique's members by degree.  Taken one
clique at a time that is millions of steps on a large graph, so the ordering
here takes cliques in rounds (the reading the CUDA path implements):

  round: every alive vertex v grows Algorithm 1's greedy clique C(v) among
         the alive vertices: C = {v}, then each alive neighbour u of v in
         decreasing core number (ties: larger degree, then smaller id) joins
         if it is adjacent to every member so far;
         key(v) = (|C(v)|, -rank(v)), rank a permutation of the vertices
         (the identity unless one is given: ties to the smaller id);
         C(v) is accepted iff, for every member u, no clique C(w)
         containing u has a larger key;
         accepted cliques are disjoint (two cliques sharing a vertex cannot
         both hold the larger key there) and the one of largest key is always
         accepted, so every round removes at least one clique;
         they are appended to the order by increasing start vertex v, each
         clique's members by decreasing degree (ties: smaller id); their
         vertices die.
  until no vertex is alive.

Degrees and core numbers are those of the whole graph.  The first clique
accepted in round one is the largest greedy clique over all start vertices
(ties to the smaller rank): with the identity rank, the deterministic form
of Algorithm 1.  Rounds run until no vertex is alive; with ranks that follow
the graph's structure (a path numbered end to end) that can take a round per
clique, which a random rank avoids.
"""
from __future__ import annotations

import numpy as np


def _greedy(rows, nbs, core, deg, v, alive):
    """Algorithm 1's greedy clique from v over the alive vertices: scan v's
    alive neighbours by decreasing core number (ties: larger degree, then
    smaller id) and add each one adjacent to every member so far."""
    cand = [u for u in rows[v].tolist() if alive[u]]
    cand.sort(key=lambda u: (-int(core[u]), -int(deg[u]), u))
    c = [v]
    for u in cand:
        if all(u in nbs[x] for x in c):
            c.append(u)
    return c


def greedy_clique(g, core, v, alive):
    """The greedy clique grown from v in one round, `alive` the boolean mask
    of the vertices not yet placed (for checking single cliques of a large
    order one by one: rows are read only where the scan needs them)."""

    class Rows(dict):
        def __missing__(self, x):
            r = g.col_idx[g.row_ptr[x]:g.row_ptr[x + 1]]
            self[x] = r
            return r

    class Sets(dict):
        def __missing__(self, x):
            r = set(g.col_idx[g.row_ptr[x]:g.row_ptr[x + 1]].tolist())
            self[x] = r
            return r

    return _greedy(Rows(), Sets(), core, np.diff(g.row_ptr), int(v), alive)


def relabel(g, order):
    """The CSR of the graph with vertex order[i] renamed i, every row sorted
    ascending: (row_ptr, col_idx)."""
    n = g.n
    order = np.asarray(order, np.int64)
    assert sorted(order.tolist()) == list(range(n)), "order must be a permutation"
    pos = np.empty(n, np.int64)
    pos[order] = np.arange(n)
    rp = np.zeros(n + 1, np.int64)
    rows = []
    for i in range(n):
        v = order[i]
        rows.append(np.sort(pos[g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]]))
        rp[i + 1] = rp[i] + rows[-1].size
    ci = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    return rp, ci


def clique_order(g, core, rank=None):
    """Returns (order, group_starts, group_round): order is a permutation of
    the vertices (order[i] = the vertex placed at position i); the cliques
    occupy order[group_starts[j]:group_starts[j+1]], accepted in round
    group_round[j] (from 0)."""
    n = g.n
    rank = np.arange(n) if rank is None else np.asarray(rank)
    assert sorted(rank.tolist()) == list(range(n)), "rank must be a permutation"
    deg = np.diff(g.row_ptr)
    rows = [g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]] for v in range(n)]
    nbs = [set(r.tolist()) for r in rows]
    alive = np.ones(n, bool)
    order, starts, rounds = [], [], []
    r = 0
    while alive.any():
        cl = {}
        for v in np.nonzero(alive)[0].tolist():
            cl[v] = _greedy(rows, nbs, core, deg, v, alive)
        best = {}
        for v, c in cl.items():
            k = (len(c), -int(rank[v]))
            for u in c:
                if u not in best or k > best[u]:
                    best[u] = k
        for v in sorted(cl):
            c = cl[v]
            k = (len(c), -int(rank[v]))
            if all(best[u] == k for u in c):
                starts.append(len(order))
                rounds.append(r)
                order.extend(sorted(c, key=lambda u: (-int(deg[u]), u)))
                alive[c] = False
        r += 1
        assert r <= n, "a round accepted no clique"
    starts.append(n)
    return np.array(order, np.int32), np.array(starts, np.int64), np.array(rounds, np.int32)


def gap_bits(g, order):
    """Mean bits per adjacency entry of gap coding under a vertex order:
    with pi(v) the position of v, each row's neighbours sorted by position
    are coded as the gap from pi(v) to the first and between consecutive
    ones, log2(1 + gap) bits each -- the locality that gap-based graph
    compression (bvgraph and its kind) exploits.  Lower is better."""
    pos = np.empty(g.n, np.int64)
    pos[np.asarray(order)] = np.arange(g.n)
    tot = 0.0
    for v in range(g.n):
        r = np.sort(pos[g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]])
        if r.size == 0:
            continue
        gaps = np.empty(r.size, np.int64)
        gaps[0] = abs(r[0] - pos[v])
        gaps[1:] = np.diff(r)
        tot += float(np.log2(1.0 + gaps).sum())
    return tot / max(int(g.row_ptr[-1]), 1)
