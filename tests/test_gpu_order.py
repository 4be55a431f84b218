"""Parity of the clique-peeling vertex order, the relabelling and the gap
cost (CUDA path through the C ABI) with oracle/ordering.py.

The order is integer work with one defined answer (tie ranks make every key
distinct), so order, clique boundaries and rounds must match bit for bit;
the relabelled CSR too.  The gap cost is a sum of positive terms that the
kernel takes in single precision (1 + gap rounded once, relative error
2^-24; log2f within 1 ulp, 2^-23 relative; together below 2^-22 = 2.4e-7 of
each term, and so of the sum) and adds in double: the relative difference
from the oracle's float64 must stay below 2.4e-7 plus the double sums' own
rounding, so the tests allow 3e-7.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import ordering as OO

pytestmark = pytest.mark.gpu
GAP_RTOL = 3e-7

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1302_6256_gb300 as m
    m.load_library()
    return m


def load(mc, g):
    return mc.mc_load_csr(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda(), mc.MC_VALIDATE)


def order_graphs():
    """Several warps' and blocks' worth of vertices with ragged tails, hubs
    whose greedy filters take the merge path, degenerate cases."""
    return [
        gg.empty(1), gg.empty(9), gg.complete(2), gg.complete(40), gg.path(2), gg.path(37), gg.cycle(11),
        gg.star(70), gg.petersen(), gg.turan(60, 5), gg.disjoint_cliques([3, 9, 1, 6]),
        gg.random_small(45, 0.3, 1), gg.random_small(80, 0.15, 2),
        gg.erdos_renyi(600, 0.05, planted=9, seed=3),
        gg.rmat(11, 8, planted=14, seed=5),
        gg.chung_lu(5000, 2.2, 10.0, 400.0, planted=12, seed=6),
        gg.relabel(gg.rmat(10, 12, planted=10, seed=7), 8),
    ]


@pytest.mark.parametrize("g", order_graphs(), ids=lambda g: g.name)
def test_clique_order_bit_exact(mc, g):
    K = oracle.core_numbers(g)
    want = OO.clique_order(g, K)
    h = load(mc, g)
    order, starts, rounds, st = mc.mc_clique_order(h)
    assert np.array_equal(order, want[0])
    assert np.array_equal(starts, want[1])
    assert np.array_equal(rounds, want[2])
    assert st["rounds"] == (int(want[2][-1]) + 1 if g.n else 0)
    h.close()


def _hub_graph(n=5200, seed=11):
    """A hub adjacent to every other vertex (degree n - 1 > 4,096, so its
    clique is grown by the block grower) over a sparse random graph with a
    planted clique of 12."""
    rng = np.random.default_rng(seed)
    src = [np.zeros(n - 1, np.int64)]
    dst = [np.arange(1, n)]
    m = 3 * n
    a, b = rng.integers(1, n, m), rng.integers(1, n, m)
    keep = a != b
    src.append(a[keep])
    dst.append(b[keep])
    S = rng.choice(np.arange(1, n), 12, replace=False)
    for i in range(12):
        for j in range(i + 1, 12):
            src.append(np.array([S[i]]))
            dst.append(np.array([S[j]]))
    return gg.from_edges(n, np.concatenate(src), np.concatenate(dst), name="hub%d" % n)


def test_clique_order_hub_beyond_4096_bit_exact(mc):
    g = _hub_graph()
    assert int(np.diff(g.row_ptr).max()) > 4096
    want = OO.clique_order(g, oracle.core_numbers(g))
    h = load(mc, g)
    order, starts, rounds, _ = mc.mc_clique_order(h)
    assert np.array_equal(order, want[0]) and np.array_equal(starts, want[1]) and np.array_equal(rounds, want[2])
    h.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_clique_order_with_rank_bit_exact(mc, seed):
    g = [gg.path(64), gg.rmat(10, 8, planted=10, seed=9), gg.chung_lu(3000, 2.4, 8.0, 200.0, planted=9, seed=4)][seed]
    rank = np.random.default_rng(100 + seed).permutation(g.n).astype(np.int32)
    want = OO.clique_order(g, oracle.core_numbers(g), rank)
    h = load(mc, g)
    for r in (rank, torch.from_numpy(rank).cuda()):
        order, starts, rounds, _ = mc.mc_clique_order(h, r)
        assert np.array_equal(order, want[0]) and np.array_equal(starts, want[1])
        assert np.array_equal(rounds, want[2])
    h.close()


def test_clique_order_refusals_and_empty(mc):
    g = gg.path(10)
    h = load(mc, g)
    for bad in (np.zeros(10, np.int32), np.arange(1, 11, dtype=np.int32), -np.arange(10, dtype=np.int32)):
        with pytest.raises(mc.MCError) as e:
            mc.mc_clique_order(h, bad)
        assert e.value.code == mc.MC_ERR_ARG
    # the handle still works after a refusal
    assert np.array_equal(mc.mc_clique_order(h)[0], OO.clique_order(g, oracle.core_numbers(g))[0])
    h.close()
    h = load(mc, gg.empty(0))
    order, starts, rounds, st = mc.mc_clique_order(h)
    assert order.size == 0 and starts.tolist() == [0] and rounds.size == 0 and st["rounds"] == 0
    assert mc.mc_gap_bits(h) == 0.0
    h.close()
    bt = gg.Batch([gg.complete(3), gg.path(4)])
    b = mc.mc_load_batch(bt.voff, bt.row_ptr, bt.col_idx)
    with pytest.raises(mc.MCError):
        mc.mc_clique_order(b)
    b.close()


def relabel_graphs():
    # rows in every sorter tier: <= 32 (registers), <= 1,024 (warp, shared
    # memory), <= 16,384 (block, shared memory), above (block, global scratch)
    return [gg.path(5), gg.rmat(11, 8, seed=3), gg.star(900), gg.star(5000), gg.star(40000),
            gg.chung_lu(20000, 2.1, 12.0, 3000.0, seed=8)]


@pytest.mark.parametrize("g", relabel_graphs(), ids=lambda g: g.name)
def test_relabel_and_gap_bits(mc, g):
    h = load(mc, g)
    rng = np.random.default_rng(g.n)
    for order in (np.arange(g.n, dtype=np.int32), rng.permutation(g.n).astype(np.int32),
                  mc.mc_clique_order(h)[0]):
        rp, ci = mc.mc_relabel(h, order)
        wrp, wci = OO.relabel(g, order)
        assert np.array_equal(rp, wrp) and np.array_equal(ci, wci)
        got, want = mc.mc_gap_bits(h, order), OO.gap_bits(g, order)
        assert abs(got - want) <= GAP_RTOL * want
    ident = OO.gap_bits(g, np.arange(g.n))
    assert abs(mc.mc_gap_bits(h) - ident) <= GAP_RTOL * ident
    for bad in (np.zeros(g.n, np.int32), np.full(g.n, g.n, np.int32)):
        with pytest.raises(mc.MCError) as e:
            mc.mc_relabel(h, bad)
        assert e.value.code == mc.MC_ERR_ARG
    h.close()


def test_clique_order_rmat_s22_properties(mc):
    """R-MAT scale 22 (the solve's workload, 4.2M vertices): a permutation;
    sampled cliques are cliques, ordered by degree, and each is the greedy
    clique of one of its members over the vertices not placed before its
    round (oracle, one clique at a time); rounds never decrease; round 0
    holds the largest greedy clique, the deterministic heuristic's size."""
    from graphgen import workloads as W
    g = W.rmat_s22()
    h = load(mc, g)
    order, starts, rounds, st = mc.mc_clique_order(h)
    n = g.n
    assert np.array_equal(np.sort(order), np.arange(n, dtype=np.int32))
    assert starts[0] == 0 and starts[-1] == n and np.all(np.diff(starts) > 0)
    assert np.all(np.diff(rounds) >= 0) and st["rounds"] == rounds[-1] + 1
    sizes = np.diff(starts)
    assert sizes[rounds == 0].max() == len(mc.mc_heuristic_clique(h, mode=1))
    deg = np.diff(g.row_ptr)
    K = mc.mc_core_numbers(h)[0]
    rng = np.random.default_rng(22)
    first_of_round = {}
    for r in np.unique(rounds):
        first_of_round[int(r)] = starts[np.searchsorted(rounds, r)]
    sample = np.unique(np.r_[0, 1, len(sizes) - 1, np.argsort(-sizes)[:20], rng.integers(0, len(sizes), 150)])
    for j in sample.tolist():
        grp = order[starts[j]:starts[j + 1]]
        assert oracle.is_clique(g, grp)
        d = deg[grp]
        assert all(d[i] > d[i + 1] or (d[i] == d[i + 1] and grp[i] < grp[i + 1]) for i in range(len(grp) - 1))
        alive = np.zeros(n, bool)
        alive[order[first_of_round[int(rounds[j])]:]] = True
        want = sorted(grp.tolist())
        assert any(sorted(OO.greedy_clique(g, K, v, alive)) == want for v in want), j
    # the clique order is more local than the vertex ids of R-MAT
    assert mc.mc_gap_bits(h, order) < mc.mc_gap_bits(h)
    h.close()
