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
            cand = [u for u in rows[v].tolist() if alive[u]]
            cand.sort(key=lambda u: (-int(core[u]), -int(deg[u]), u))
            c = [v]
            for u in cand:
                if all(u in nbs[x] for x in c):
                    c.append(u)
            cl[v] = c
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
