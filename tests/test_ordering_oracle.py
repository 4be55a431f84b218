"""Pins of the clique-peeling ordering oracle (oracle/ordering.py): graphs
worked by hand, the link to the deterministic Algorithm 1, and the
properties that hold for any graph."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import ordering as OO


def _order(g, rank=None):
    return OO.clique_order(g, oracle.core_numbers(g), rank)[:2]


def test_path_worked_by_hand():
    """P4 = 0-1-2-3, every core number 1.  Round 1: C(0) = {0,1}; from 1 the
    candidates are 2 (degree 2) then 0, so C(1) = {1,2}; C(2) = {2,1};
    C(3) = {3,2}.  Keys (2,0) > (2,-1) > (2,-2) > (2,-3): vertex 1's best is
    C(0)'s, so only C(0) is accepted.  Round 2: {2,3} from 2.  Members by
    degree: [1, 0], [2, 3]."""
    order, starts = _order(gg.path(4))
    assert order.tolist() == [1, 0, 2, 3] and starts.tolist() == [0, 2, 4]


def test_path_with_reversed_rank_worked_by_hand():
    """P4 with rank(v) = 3 - v.  Round 0: C(3) = {3,2} has the best key
    (2, 0) and holds vertices 2 and 3; C(0) = {0,1} (2,-3) loses vertex 1 to
    C(1) = {1,2} (2,-2), which loses vertex 2 to C(3).  Round 1: C(1) =
    {1,0} (2,-2) beats C(0) = {0,1} (2,-3).  Members by degree."""
    order, starts, rounds = OO.clique_order(gg.path(4), oracle.core_numbers(gg.path(4)), np.array([3, 2, 1, 0]))
    assert order.tolist() == [2, 3, 1, 0] and starts.tolist() == [0, 2, 4] and rounds.tolist() == [0, 1]


def test_path_numbered_end_to_end_takes_a_round_per_clique():
    """With identity ranks each round of a path accepts only its lowest
    clique {2i, 2i+1}: vertex 2i+1's other clique C(2i+2) = {2i+2, 2i+1}
    (ties by id) has a smaller key, and so on down the path."""
    g = gg.path(12)
    order, starts, rounds = OO.clique_order(g, oracle.core_numbers(g))
    assert rounds.tolist() == list(range(6))
    assert [sorted(order[starts[j]:starts[j + 1]].tolist()) for j in range(6)] == [[2 * j, 2 * j + 1] for j in range(6)]


def test_core_number_before_degree_worked_by_hand():
    """Edges 0-2 0-5 0-6 1-3 2-3 2-4 5-6: triangle {0,5,6} (core 2) and a
    tree through 2 (core 1; degrees 0:3 1:1 2:3 3:2 4:1 5:2 6:2).  From 0 the
    candidates by core number are 5, 6, then 2 (degree 3 but core 1), so
    C(0) = {0,5,6} (3, 0) and holds 0, 5, 6; C(1) = {1,3} wins vertex 3
    over C(3) = {3,2}; C(2) = {2,0} loses 0, C(4) = {4,2} loses 2 to C(2).
    Round 0: [0,5,6], [3,1] (by degree); round 1: C(2) = {2,4} -> [2,4]."""
    g = gg.from_edges(7, [0, 0, 0, 1, 2, 2, 5], [2, 5, 6, 3, 3, 4, 6])
    order, starts, rounds = OO.clique_order(g, oracle.core_numbers(g))
    assert order.tolist() == [0, 5, 6, 3, 1, 2, 4]
    assert starts.tolist() == [0, 3, 5, 7] and rounds.tolist() == [0, 0, 1]


def test_star_worked_by_hand():
    """star(5): C(0) = {0, 1} (the leaves are not adjacent), C(i) = {i, 0};
    C(0) holds the largest key.  Round 2: leaves 2, 3, 4 alone."""
    order, starts = _order(gg.star(5))
    assert order.tolist() == [0, 1, 2, 3, 4] and starts.tolist() == [0, 2, 3, 4, 5]


def test_disjoint_cliques_one_round():
    g = gg.disjoint_cliques([4, 7, 3])
    order, starts = _order(g)
    # one round: every clique accepted, placed by start vertex (its smallest id)
    assert starts.tolist() == [0, 4, 11, 14]
    assert order.tolist() == list(range(14))


def test_first_clique_is_the_deterministic_heuristic():
    for g in [gg.rmat(11, 8, planted=12, seed=3), gg.chung_lu(2000, 2.5, 8.0, 200.0, planted=9, seed=7),
              gg.erdos_renyi(300, 0.1, planted=10, seed=5)]:
        K = oracle.core_numbers(g)
        order, starts, rnd = OO.clique_order(g, K)
        H = set(oracle.heuristic_clique(g, K, mode=1).tolist())
        groups = [set(order[starts[j]:starts[j + 1]].tolist()) for j in range(len(starts) - 1)]
        # C(v*) of the largest key over all start vertices is accepted in round 0
        assert H in groups and rnd[groups.index(H)] == 0
        assert len(H) == max(len(c) for c, r in zip(groups, rnd) if r == 0)


@pytest.mark.parametrize("seed", range(4))
def test_properties_on_random_graphs(seed):
    """A permutation; every group a clique, maximal among the vertices not
    placed before its round; members by decreasing degree."""
    g = gg.random_small(40 + 10 * seed, 0.2, 900 + seed)
    rank = np.random.default_rng(seed).permutation(g.n) if seed % 2 else None
    order, starts, rnd = OO.clique_order(g, oracle.core_numbers(g), rank)
    assert sorted(order.tolist()) == list(range(g.n))
    assert np.all(np.diff(rnd) >= 0)
    deg = np.diff(g.row_ptr)
    nb = [set(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    for j in range(len(starts) - 1):
        c = order[starts[j]:starts[j + 1]]
        assert oracle.is_clique(g, c)
        # maximal among the vertices still alive in its round
        alive = set(order[starts[np.searchsorted(rnd, rnd[j])]:].tolist())
        ext = set.intersection(*[nb[x] for x in c.tolist()]) & alive
        assert not ext
        d = deg[c]
        assert all(d[i] > d[i + 1] or (d[i] == d[i + 1] and c[i] < c[i + 1]) for i in range(len(c) - 1))


def test_gap_bits_closed_forms():
    # a path in its natural order: the two end rows code one gap of 1 (1 bit);
    # every inner row codes |v-1 - v| = 1 then 2 -> 1 + log2 3 bits
    g = gg.path(10)
    want = (2 * 1 + 8 * (1 + np.log2(3))) / 18
    assert OO.gap_bits(g, np.arange(10)) == pytest.approx(want)
    # K4 in natural order, gaps per row: (1,1,1), (1,2,1), (2,1,2), (3,1,1)
    g = gg.complete(4)
    want = (3 + (2 + np.log2(3)) + (1 + 2 * np.log2(3)) + (2 + 2)) / 12
    assert OO.gap_bits(g, np.arange(4)) == pytest.approx(want)
    # reversing the order of a path changes nothing (gaps are symmetric)
    g = gg.path(10)
    assert OO.gap_bits(g, np.arange(10)[::-1]) == pytest.approx(OO.gap_bits(g, np.arange(10)))


def test_greedy_clique_alone_matches_the_rounds():
    """Each clique of the order is the greedy clique of one of its members
    over the vertices not placed before its round."""
    g = gg.rmat(9, 8, planted=8, seed=4)
    K = oracle.core_numbers(g)
    order, starts, rnd = OO.clique_order(g, K)
    for j in range(0, len(rnd), 7):
        first = starts[np.searchsorted(rnd, rnd[j])]
        alive = np.zeros(g.n, bool)
        alive[order[first:]] = True
        grp = sorted(order[starts[j]:starts[j + 1]].tolist())
        assert any(sorted(OO.greedy_clique(g, K, v, alive)) == grp for v in grp)


def test_relabel_definition():
    g = gg.rmat(8, 6, seed=2)
    # identity: the graph itself
    rp, ci = OO.relabel(g, np.arange(g.n))
    assert np.array_equal(rp, g.row_ptr) and np.array_equal(ci, g.col_idx)
    perm = np.random.default_rng(3).permutation(g.n)
    rp, ci = OO.relabel(g, perm)
    # degrees follow the vertices; every edge maps to an edge; rows sorted
    assert np.array_equal(np.diff(rp), np.diff(g.row_ptr)[perm])
    pos = np.empty(g.n, np.int64)
    pos[perm] = np.arange(g.n)
    for v in range(g.n):
        row = ci[rp[pos[v]]:rp[pos[v] + 1]]
        assert np.all(np.diff(row) > 0)
        assert set(row.tolist()) == set(pos[g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]]].tolist())
    # the inverse permutation gives the original back
    h = gg.Graph(rp, ci, "relabelled")
    rp2, ci2 = OO.relabel(h, pos)
    assert np.array_equal(rp2, g.row_ptr) and np.array_equal(ci2, g.col_idx)
    # gap cost is the same whether computed on the relabelled CSR with the
    # identity or on the original with the order
    assert OO.gap_bits(g, perm) == pytest.approx(OO.gap_bits(h, np.arange(g.n)))
