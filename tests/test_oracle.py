"""Pins of the CPU oracle against what the paper and the mathematics fix.

Core numbers (Section 3): brute-force k-core definition, closed forms,
networkx's independent routine, and the peeling certificate.
omega (Section 1 definition; Algorithm 2): brute-force subset enumeration on
n <= 18, closed forms, networkx's independent exact routine, planted cliques in
sparse graphs, Fact 1's bound chain, relabelling invariance.
Algorithm 1: returns a clique no larger than omega and no larger than K+1,
exact on disjoint unions of cliques.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle


def adj_sets(g):
    return [set(g.col_idx[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]


def brute_cores(g):
    """K(v) = largest k such that v survives in the k-core, where the k-core is
    what remains after repeatedly deleting vertices of degree < k."""
    adj = adj_sets(g)
    core = [0] * g.n
    k = 0
    while True:
        alive = set(range(g.n))
        changed = True
        while changed:
            changed = False
            for v in list(alive):
                if len(adj[v] & alive) < k:
                    alive.discard(v)
                    changed = True
        if not alive:
            break
        for v in alive:
            core[v] = k
        k += 1
    return np.array(core, np.int32)


def brute_omega(g):
    """Largest subset S with every pair adjacent, by enumerating all 2^n subsets."""
    n = g.n
    if n == 0:
        return 0
    assert n <= 18
    masks = np.zeros(n, np.int64)
    for v, nb in enumerate(adj_sets(g)):
        for u in nb:
            masks[v] |= 1 << u
    S = np.arange(1 << n, dtype=np.int64)
    ok = np.ones(S.shape, bool)
    for v in range(n):
        inS = (S >> v) & 1 == 1
        allowed = masks[v] | (1 << v)
        ok &= ~inS | ((S & ~allowed) == 0)
    pop = np.zeros(S.shape, np.int64)
    for v in range(n):
        pop += (S >> v) & 1
    return int(pop[ok].max())


def small_random_graphs():
    out = []
    for seed in range(40):
        n = 3 + seed % 16
        p = [0.1, 0.3, 0.5, 0.7, 0.9][seed % 5]
        out.append(gg.random_small(n, p, seed + 100))
    return out


# ------------------------------------------------------------ core numbers --

@pytest.mark.parametrize("g", small_random_graphs(), ids=lambda g: g.name)
def test_cores_match_bruteforce_definition(g):
    assert np.array_equal(oracle.core_numbers(g), brute_cores(g))


def test_cores_closed_forms():
    assert np.all(oracle.core_numbers(gg.complete(9)) == 8)
    assert np.all(oracle.core_numbers(gg.cycle(11)) == 2)
    assert np.all(oracle.core_numbers(gg.path(7)) == 1)
    assert np.all(oracle.core_numbers(gg.star(12)) == 1)
    assert np.all(oracle.core_numbers(gg.empty(5)) == 0)
    assert np.all(oracle.core_numbers(gg.petersen()) == 3)  # 3-regular, connected
    assert np.all(oracle.core_numbers(gg.complete_bipartite(4, 7)) == 4)
    c = oracle.core_numbers(gg.disjoint_cliques([3, 5, 2]))
    assert c.tolist() == [2] * 3 + [4] * 5 + [1] * 2


def test_cores_match_networkx_on_generated_graphs():
    nx = pytest.importorskip("networkx")
    for g in [gg.chung_lu(3000, 2.5, 8.0, 300.0, planted=9, seed=7),
              gg.rmat(11, 8, planted=12, seed=3),
              gg.erdos_renyi(500, 0.05, planted=10, seed=5)]:
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        src = np.repeat(np.arange(g.n), g.degrees())
        G.add_edges_from(zip(src.tolist(), g.col_idx.tolist()))
        ref = nx.core_number(G)
        assert np.array_equal(oracle.core_numbers(g), np.array([ref[v] for v in range(g.n)]))


def test_core_peeling_certificate():
    """K(v) = k iff v has >= k neighbours of core >= k and fewer than k+1
    neighbours of core >= k+1 (both follow from the k-core definition)."""
    g = gg.rmat(12, 16, planted=20, seed=9)
    K = oracle.core_numbers(g)
    src = np.repeat(np.arange(g.n), g.degrees())
    kn = K[g.col_idx]
    ge = np.bincount(src[kn >= K[src]], minlength=g.n)
    gt = np.bincount(src[kn >= K[src] + 1], minlength=g.n)
    assert np.all(ge >= K)
    assert np.all(gt < K + 1)


def test_core_order_is_degeneracy_order():
    """In the returned visiting order every vertex has at most K(v) later neighbours."""
    g = gg.chung_lu(4000, 2.2, 10.0, 500.0, planted=12, seed=4)
    K, order = oracle.core_numbers(g, with_order=True)
    pos = np.empty(g.n, np.int64)
    pos[order] = np.arange(g.n)
    src = np.repeat(np.arange(g.n), g.degrees())
    later = np.bincount(src[pos[g.col_idx] > pos[src]], minlength=g.n)
    assert np.all(later <= K)
    assert np.all(np.diff(K[order]) >= 0)


# ------------------------------------------------------------------ omega --

@pytest.mark.parametrize("g", small_random_graphs(), ids=lambda g: g.name)
def test_omega_matches_bruteforce(g):
    om, wit, _ = oracle.max_clique(g)
    assert om == brute_omega(g)
    assert len(wit) == om and oracle.is_clique(g, wit)


def test_omega_closed_forms():
    cases = [
        (gg.empty(0), 0), (gg.empty(1), 1), (gg.empty(6), 1),
        (gg.complete(2), 2), (gg.complete(17), 17),
        (gg.cycle(3), 3), (gg.cycle(4), 2), (gg.cycle(9), 2),
        (gg.path(10), 2), (gg.star(20), 2), (gg.petersen(), 2),
        (gg.complete_bipartite(6, 9), 2),
        (gg.turan(20, 4), 4), (gg.turan(31, 7), 7),
        (gg.disjoint_cliques([4, 9, 3, 9, 2]), 9),
        (gg.mycielski(4), 2), (gg.mycielski(6), 2),
    ]
    for g, want in cases:
        om, wit, _ = oracle.max_clique(g)
        assert om == want, g.name
        assert len(wit) == om and oracle.is_clique(g, wit)
    om, wit, _ = oracle.max_clique(gg.empty(6))
    assert wit.tolist() == [0] or len(wit) == 1


def test_omega_matches_networkx_exact():
    nx = pytest.importorskip("networkx")
    for seed in range(6):
        g = gg.erdos_renyi(60 + 10 * seed, [0.3, 0.5, 0.7][seed % 3], planted=0, seed=200 + seed)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        src = np.repeat(np.arange(g.n), g.degrees())
        G.add_edges_from(zip(src.tolist(), g.col_idx.tolist()))
        _, w = nx.max_weight_clique(G, weight=None)
        om, wit, _ = oracle.max_clique(g)
        assert om == w
        assert oracle.is_clique(g, wit)


@pytest.mark.parametrize("seed", range(6))
def test_planted_clique_in_sparse_graph(seed):
    """Sparse G(n, p) with p*n << n has natural omega <= 4 w.h.p.; a planted
    k >= 8 clique is then exactly omega and the planted set is the witness."""
    k = 8 + 3 * seed
    g = gg.erdos_renyi(2000, 4.0 / 1999, planted=k, seed=300 + seed)
    om, wit, _ = oracle.max_clique(g)
    assert om == k
    assert np.array_equal(np.sort(wit), np.sort(g.planted))


def test_fact1_bound_chain_and_witness():
    """omega <= L(G) <= K(G)+1 <= Delta(G)+1 with L the greedy colouring in
    degeneracy order (decreasing core number)."""
    for g in [gg.chung_lu(5000, 2.5, 8.0, 400.0, planted=11, seed=1),
              gg.rmat(12, 16, planted=14, seed=2), gg.turan(40, 6), gg.mycielski(5)]:
        K, order = oracle.core_numbers(g, with_order=True)
        L = oracle.greedy_colors(g, order[::-1].copy())
        om, wit, st = oracle.max_clique(g)
        H = oracle.heuristic_clique(g, K)
        assert len(H) <= om <= L <= K.max() + 1 <= g.degrees().max() + 1
        assert oracle.is_clique(g, wit) and oracle.is_clique(g, H)
        assert st["max_core"] == K.max() and st["heuristic"] == len(H)


def test_relabel_invariance():
    g = gg.chung_lu(3000, 2.3, 12.0, 300.0, planted=10, seed=11)
    h = gg.relabel(g, 5)
    assert oracle.max_clique(g)[0] == oracle.max_clique(h)[0]
    assert np.array_equal(np.sort(oracle.core_numbers(g)), np.sort(oracle.core_numbers(h)))


# -------------------------------------------------------------- heuristic --

def test_heuristic_disjoint_cliques_exact():
    g = gg.disjoint_cliques([5, 12, 7, 12, 3])
    for mode in (0, 1):
        H = oracle.heuristic_clique(g, mode=mode)
        assert len(H) == 12 and oracle.is_clique(g, H)
    # mode 1 breaks ties by the smallest start vertex: the first 12-clique
    assert oracle.heuristic_clique(g, mode=1).tolist() == list(range(5, 17))


@pytest.mark.parametrize("g", small_random_graphs()[::3], ids=lambda g: g.name)
def test_heuristic_valid_and_bounded(g):
    K = oracle.core_numbers(g)
    om = brute_omega(g)
    for mode in (0, 1):
        H = oracle.heuristic_clique(g, K, mode)
        assert oracle.is_clique(g, H)
        assert len(H) <= om
        assert len(H) <= (K.max() + 1 if g.n else 0)
        if g.n:
            assert len(H) >= 1


def test_heuristic_mode1_is_max_over_start_vertices():
    """Mode 1 is the largest greedy clique over all start vertices: it is at
    least the greedy clique grown from any single vertex, here checked through
    the planted clique (every planted vertex's greedy run stays inside it when
    the planted vertices dominate the core order)."""
    g = gg.erdos_renyi(400, 0.02, planted=15, seed=42)
    H = oracle.heuristic_clique(g, mode=1)
    assert len(H) == 15
    assert np.array_equal(H, np.sort(g.planted))


# ------------------------------------------ tight cases and tie-breaks --

def test_greedy_colouring_closed_forms():
    """Greedy colouring (Section 3): a complete graph needs n colours in any
    order; an edgeless graph one; disjoint cliques the largest clique; a
    cycle visited along the cycle 2 (even) or 3 (odd); a complete bipartite
    graph visited one side first 2."""
    rng = np.random.default_rng(0)
    assert oracle.greedy_colors(gg.complete(7), rng.permutation(7)) == 7
    assert oracle.greedy_colors(gg.empty(5), np.arange(5)) == 1
    g = gg.disjoint_cliques([3, 6, 2])
    assert oracle.greedy_colors(g, rng.permutation(g.n)) == 6
    assert oracle.greedy_colors(gg.cycle(10), np.arange(10)) == 2
    assert oracle.greedy_colors(gg.cycle(11), np.arange(11)) == 3
    assert oracle.greedy_colors(gg.complete_bipartite(4, 6), np.arange(10)) == 2
    assert oracle.greedy_colors(gg.star(8), np.arange(8)) == 2


def test_is_clique_definition_cases():
    """A clique is a set of distinct vertices, every pair adjacent."""
    k5, p = gg.complete(5), gg.path(4)
    assert oracle.is_clique(k5, [0, 1, 2, 3, 4]) and oracle.is_clique(k5, [3])
    assert oracle.is_clique(p, [1, 2])
    assert not oracle.is_clique(p, [0, 1, 2])       # 0 and 2 are not adjacent
    assert not oracle.is_clique(p, [0, 1, 3])       # only the last pair fails
    assert not oracle.is_clique(k5, [1, 2, 2])      # a repeated vertex
    assert not oracle.is_clique(k5, [2, 1, 2])
    assert not oracle.is_clique(k5, [0, 5])         # out of range
    assert not oracle.is_clique(gg.empty(3), [0, 1])


def tight_instance(k):
    """A k-clique Q whose members have core number exactly k-1, each also
    joined to one vertex of a triangle-free (k-1)-regular graph that has a
    smaller id, the same core number and the same degree, so Algorithm 1's
    greedy step from any member of Q takes that vertex first and stops at
    two; for k >= 4 a separate (k-1)-clique.  Algorithm 1 then ends one short
    of omega = k, and every member of the maximum clique sits exactly on the
    pruning bound K(v) >= |H|."""
    if k == 3:
        base_n, edges, attach = 9, [(i, (i + 1) % 9) for i in range(9)], [0, 3, 6]
    elif k == 5:
        # K_{4,4}: triangle-free and 4-regular
        base_n, edges, attach = 8, [(a, b) for a in range(4) for b in range(4, 8)], [0, 1, 2, 4, 5]
    else:
        pg = gg.petersen()
        src = np.repeat(np.arange(pg.n), pg.degrees())
        keep = src < pg.col_idx
        base_n, edges, attach = pg.n, list(zip(src[keep].tolist(), pg.col_idx[keep].tolist())), [0, 2, 4, 6]
    Q = list(range(base_n, base_n + k))
    edges += [(a, b) for i, a in enumerate(Q) for b in Q[i + 1:]] + list(zip(Q, attach))
    n = base_n + k
    if k >= 4:
        R = list(range(n, n + k - 1))
        edges += [(a, b) for i, a in enumerate(R) for b in R[i + 1:]]
        n += k - 1
    s, d = zip(*edges)
    return gg.from_edges(n, s, d), Q


@pytest.mark.parametrize("k", [3, 4, 5])
def test_tight_instances_where_the_heuristic_is_one_short(k):
    """Every bound of Algorithm 2 is met with equality here (the pruning
    test K(v) >= |H|, the neighbourhood core and colour tests of
    InitialBranch, the colour test of Branch), so an off-by-one in any of
    them loses the maximum clique."""
    g, Q = tight_instance(k)
    K = oracle.core_numbers(g)
    assert K[Q].tolist() == [k - 1] * k
    for mode in (0, 1):
        H = oracle.heuristic_clique(g, K, mode)
        assert len(H) == k - 1 and oracle.is_clique(g, H)
    om, wit, st = oracle.max_clique(g)
    assert om == k == brute_omega(g)
    assert wit.tolist() == Q
    assert st["heuristic"] == k - 1


def test_heuristic_tie_breaks():
    """Ties in Algorithm 1's core order (the reading: larger degree first,
    then smaller id), worked by hand.  Triangles {0,1,2} and {0,3,4}, and a
    pendant on each of 3 and 4: vertices 0-4 have core number 2, vertex 0
    degree 4, vertices 3 and 4 degree 3, vertices 1 and 2 degree 2.  From 0
    the candidates are taken as 3, 4, 1, 2, giving {0,3,4}; vertex 0 comes
    first in the visiting order, and no later start beats size 3."""
    g = gg.from_edges(7, [0, 0, 1, 0, 0, 3, 3, 4], [1, 2, 2, 3, 4, 4, 5, 6])
    assert oracle.core_numbers(g)[:5].tolist() == [2] * 5
    for mode in (0, 1):
        assert oracle.heuristic_clique(g, mode=mode).tolist() == [0, 3, 4]


def test_heuristic_running_maximum():
    """Algorithm 1 with its running maximum: in K(3,3) plus a separate
    triangle the bipartite vertices (core 3) come first and give max = 2;
    the triangle's vertices (core 2, not below max) are still started, and
    their candidates with core >= max give the triangle."""
    src = [0, 0, 0, 1, 1, 1, 2, 2, 2, 6, 6, 7]
    dst = [3, 4, 5, 3, 4, 5, 3, 4, 5, 7, 8, 8]
    g = gg.from_edges(9, src, dst)
    assert oracle.heuristic_clique(g, mode=0).tolist() == [6, 7, 8]


# ------------------------------------------------- threaded exact search --
# The threaded search (Section 4.5: workers sharing the incumbent) must give
# the same omega as the definition for every interleaving, so each pin runs
# it with 1, 2 and 4 workers.

THREADS = (1, 2, 4)


@pytest.mark.parametrize("g", small_random_graphs(), ids=lambda g: g.name)
def test_threaded_omega_matches_bruteforce(g):
    om = brute_omega(g)
    for t in THREADS:
        o, wit, st = oracle.max_clique_threads(g, t)
        assert o == om, t
        assert len(wit) == o and oracle.is_clique(g, wit)
        assert st["heuristic"] <= om


def test_threaded_omega_closed_forms():
    cases = [
        (gg.empty(0), 0), (gg.empty(1), 1), (gg.empty(6), 1),
        (gg.complete(2), 2), (gg.complete(17), 17),
        (gg.cycle(3), 3), (gg.cycle(4), 2), (gg.cycle(9), 2),
        (gg.path(10), 2), (gg.star(20), 2), (gg.petersen(), 2),
        (gg.complete_bipartite(6, 9), 2),
        (gg.turan(20, 4), 4), (gg.turan(31, 7), 7), (gg.turan(60, 11), 11),
        (gg.disjoint_cliques([4, 9, 3, 9, 2]), 9),
        (gg.mycielski(4), 2), (gg.mycielski(6), 2),
    ]
    for g, want in cases:
        for t in THREADS:
            om, wit, _ = oracle.max_clique_threads(g, t)
            assert om == want, (g.name, t)
            assert len(wit) == om and oracle.is_clique(g, wit)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_threaded_tight_instances(k):
    """Every bound of the threaded search (the pruning K >= |H|, the root's
    |P| + 1 test, the neighbourhood-core filter, both colour tests) is met
    with equality by the maximum clique Q, so an off-by-one in any of them
    loses it; the maximum clique is unique, so the witness is Q."""
    g, Q = tight_instance(k)
    for t in THREADS:
        om, wit, st = oracle.max_clique_threads(g, t)
        assert om == k and wit.tolist() == Q, t
        assert st["heuristic"] == k - 1
    h = gg.relabel(g, 3)
    for t in THREADS:
        om, wit, _ = oracle.max_clique_threads(h, t)
        assert om == k and oracle.is_clique(h, wit)


def test_threaded_heuristic_is_the_printed_algorithm():
    """The threaded search's Algorithm 1 (start vertices shared by the
    workers in decreasing core order, running maximum shared): exact on
    disjoint cliques, and the running-maximum graph of
    test_heuristic_running_maximum still gives the triangle."""
    g = gg.disjoint_cliques([5, 12, 7, 12, 3])
    src = [0, 0, 0, 1, 1, 1, 2, 2, 2, 6, 6, 7]
    dst = [3, 4, 5, 3, 4, 5, 3, 4, 5, 7, 8, 8]
    r = gg.from_edges(9, src, dst)
    for t in THREADS:
        assert oracle.max_clique_threads(g, t)[2]["heuristic"] == 12
        assert oracle.max_clique_threads(r, t)[2]["heuristic"] == 3


def test_threaded_matches_single_thread_on_generated_graphs():
    for g in [gg.chung_lu(3000, 2.5, 8.0, 300.0, planted=9, seed=7),
              gg.rmat(11, 8, planted=12, seed=3),
              gg.erdos_renyi(500, 0.05, planted=10, seed=5),
              gg.rmat(12, 16, planted=14, seed=2)]:
        om, _, st1 = oracle.max_clique(g)
        for t in THREADS:
            o, wit, st = oracle.max_clique_threads(g, t)
            assert o == om and oracle.is_clique(g, wit) and len(wit) == o
            assert st["max_core"] == st1["max_core"]
            assert st["heuristic"] <= om


# ----------------------------------------------- partitioned search (4.5) --
# The roots split over `parts` ranks by their position in one shared
# degeneracy order: every clique has exactly one lowest-ranked member, so
# the largest clique found by any part is omega.

def _other_degeneracy_order(g):
    """A degeneracy order by a different rule than Batagelj-Zaversnik's:
    repeatedly remove a vertex of minimum remaining degree, ties to the
    LARGEST id (a plain restatement of the definition)."""
    adj = adj_sets(g)
    deg = {v: len(adj[v]) for v in range(g.n)}
    alive = set(range(g.n))
    out = []
    while alive:
        v = max(alive, key=lambda x: (-deg[x], x))
        out.append(v)
        alive.discard(v)
        for u in adj[v]:
            if u in alive:
                deg[u] -= 1
    return np.array(out, np.int32)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_partition_covers_every_clique(k):
    graphs = [tight_instance(k)[0], gg.relabel(tight_instance(k)[0], 5)] + small_random_graphs()[::4]
    for g in graphs:
        om = brute_omega(g) if g.n <= 18 else oracle.max_clique(g)[0]
        for parts in (1, 2, 3, 5):
            for order in (None, _other_degeneracy_order(g)):
                res = [oracle.max_clique_part(g, r, parts, order) for r in range(parts)]
                assert max(o for o, _, _ in res) == om, (g.name, parts)
                for o, wit, _ in res:
                    assert len(wit) == o and oracle.is_clique(g, wit)


def test_partition_on_generated_graphs():
    for g in [gg.rmat(12, 16, planted=14, seed=2), gg.chung_lu(3000, 2.5, 8.0, 300.0, planted=9, seed=7)]:
        om = oracle.max_clique(g)[0]
        K, order = oracle.core_numbers(g, with_order=True)
        for parts in (2, 4):
            res = [oracle.max_clique_part(g, r, parts, order, threads=2) for r in range(parts)]
            assert max(o for o, _, _ in res) == om
            # the parts share the work: with one worker each (same heuristic,
            # same pruning) their roots are disjoint and make up all roots
            one = [oracle.max_clique_part(g, r, parts, order, threads=1)[2]["initial_branch"] for r in range(parts)]
            assert sum(one) == oracle.max_clique_part(g, 0, 1, order, threads=1)[2]["initial_branch"]


def test_partition_refuses_an_order_that_is_not_a_degeneracy_order():
    g = gg.star(10)  # the centre first has 9 later neighbours but core number 1
    with pytest.raises(RuntimeError):
        oracle.max_clique_part(g, 0, 2, np.arange(10, dtype=np.int32))
    with pytest.raises(RuntimeError):
        oracle.max_clique_part(g, 0, 2, np.zeros(10, dtype=np.int32))  # not a permutation


def test_turan_with_planted_clique_closed_form():
    """Turan T(220, 20) (parts of 11) with a clique planted on 5 vertices of
    each of parts 0..4: outside the planted set a clique holds one vertex per
    part, so omega = 25 + (20 - 5) = 40 -- the small analogue of the GPU test
    of roots beyond 4,096 candidates."""
    n, r, per, parts = 220, 20, 5, 5
    size = n // r
    part = np.arange(n) // size
    src, dst = [], []
    for v in range(n):
        for u in range(v + 1, n):
            if part[u] != part[v]:
                src.append(v)
                dst.append(u)
    S = [p * size + i for p in range(parts) for i in range(per)]
    for a in range(len(S)):
        for b in range(a + 1, len(S)):
            if part[S[a]] == part[S[b]]:
                src.append(S[a])
                dst.append(S[b])
    g = gg.from_edges(n, np.array(src), np.array(dst))
    om, wit, _ = oracle.max_clique(g)
    assert om == per * parts + (r - parts) and oracle.is_clique(g, wit)
    assert oracle.max_clique_threads(g, 3)[0] == om


def test_threaded_search_effort_close_to_single_thread():
    """The threaded search recolours Branch's candidates in vertex-id order,
    as the single-thread search does; coloured in ascending peel rank (the
    order that colours worst) it visited 71,333 Branch nodes on this graph
    against the single-thread search's 145.  The node counts may differ by
    the root order, not by orders of magnitude."""
    g = gg.rmat(13, 16, 0.57, 0.19, 0.19, planted=40, seed=2)
    om, _, st1 = oracle.max_clique(g)
    o, _, st = oracle.max_clique_threads(g, 1)
    assert o == om == 40
    assert st["nodes"] <= 4 * st1["nodes"] + 1000
