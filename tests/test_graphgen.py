"""The shared input generators: every graph is a simple symmetric CSR, the
same seed gives the same graph, and each family follows its recipe (the
Chung-Lu weights' mean, cap and Pareto tail; the Erdos-Renyi edge count;
R-MAT's vertex count and sampled edges; planted cliques; the parameter
ranges of the Erdos-Renyi batch).  The random numbers are SplitMix64 outputs
and the logarithm and exponential are series evaluations; both are pinned
to independent references."""
import math

import numpy as np
import pytest

import graphgen as gg


def assert_simple_symmetric(g):
    rp, ci, n = g.row_ptr, g.col_idx, g.n
    assert rp.dtype == np.int64 and ci.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == ci.shape[0] and np.all(np.diff(rp) >= 0)
    assert ci.size == 0 or (ci.min() >= 0 and ci.max() < n)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    assert not np.any(src == ci), "self-loop"
    # strictly increasing inside every row
    same_row = src[1:] == src[:-1]
    assert np.all(ci[1:][same_row] > ci[:-1][same_row]), "unsorted or duplicate"
    # every arc has its reverse: the sorted (src, dst) and (dst, src) lists agree
    fwd = src * n + ci
    rev = np.sort(ci.astype(np.int64) * n + src)
    assert np.array_equal(fwd, rev), "not symmetric"


def assert_planted(g):
    members = g.planted
    if members is None or len(members) == 0:
        return
    assert len(np.unique(members)) == len(members)
    for i, a in enumerate(members):
        row = set(g.col_idx[g.row_ptr[a]:g.row_ptr[a + 1]].tolist())
        assert all(int(b) in row for b in members[i + 1:])


@pytest.mark.parametrize("make", [
    lambda: gg.rmat(12, 16, planted=20, seed=3),
    lambda: gg.chung_lu(5000, 2.3, 10.0, 500.0, planted=12, seed=4),
    lambda: gg.erdos_renyi(700, 0.03, planted=9, seed=5),
    lambda: gg.erdos_renyi(64, 1.0, planted=10, seed=6),
    lambda: gg.relabel(gg.chung_lu(3000, 2.5, 8.0, 300.0, planted=10, seed=7), 2),
    lambda: gg.complete(9), lambda: gg.cycle(7), lambda: gg.star(6), lambda: gg.empty(4),
    lambda: gg.turan(12, 5), lambda: gg.mycielski(5), lambda: gg.petersen(),
], ids=["rmat", "chung-lu", "er", "er-complete", "relabel", "K9", "C7", "star", "empty", "turan", "mycielski",
        "petersen"])
def test_every_generator_gives_a_simple_symmetric_csr(make):
    g = make()
    assert_simple_symmetric(g)
    assert_planted(g)


def test_batch_is_block_diagonal():
    b = gg.er_batch(12, seed=9)
    whole = gg.Graph(b.row_ptr, b.col_idx, "batch")
    assert_simple_symmetric(whole)
    src = np.repeat(np.arange(b.n), np.diff(b.row_ptr))
    gid = np.searchsorted(b.voff, src, side="right") - 1
    assert np.all(b.voff[gid] <= b.col_idx) and np.all(b.col_idx < b.voff[gid + 1])
    for i, g in enumerate(b.graphs):
        v0 = b.voff[i]
        assert np.array_equal(b.row_ptr[v0:v0 + g.n + 1] - b.row_ptr[v0], g.row_ptr)


def test_same_seed_same_graph():
    a, b = gg.rmat(11, 8, planted=10, seed=5), gg.rmat(11, 8, planted=10, seed=5)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    c = gg.rmat(11, 8, planted=10, seed=6)
    assert not (np.array_equal(a.row_ptr, c.row_ptr) and np.array_equal(a.col_idx, c.col_idx))


def test_splitmix64_reference_outputs():
    """gg_rand(key, i) is the (i+1)-th output of SplitMix64 whose state starts
    at key; from state 0 the published generator's first outputs are these."""
    assert [gg.rand_u64(0, i) for i in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_series_log_and_exp_against_the_library():
    for x in [1e-300, 1e-9, 0.001, 0.3, 0.5, 0.999, 1.0, 1.5, 2.0, 10.0, 1234.5, 1e12]:
        assert gg.det_log(x) == pytest.approx(math.log(x), rel=1e-14, abs=1e-15)
    # exp reduces x by k ln 2 with ln 2 rounded to a double (error ~2.3e-17),
    # so its relative error grows by that much per unit of |k| = |x| / ln 2
    for x in [-700.0, -30.0, -1.0, -1e-9, 0.0, 1e-9, 0.5, 1.0, 7.25, 300.0]:
        assert gg.det_exp(x) == pytest.approx(math.exp(x), rel=4e-16 + 5e-17 * abs(x) / math.log(2))


def test_chung_lu_weights_recipe():
    """Pareto(gamma) weights: capped at cap, their mean exactly the stated
    mean (the scale is solved for it), and below the cap the tail falls as
    x^-(gamma-1)."""
    n, gamma, mean, cap = 200_000, 2.5, 8.0, 1000.0
    w = np.empty(n, np.float64)
    assert gg._L().gg_chung_lu_weights(n, gamma, mean, cap, 1, w.ctypes.data) == 0
    assert w.mean() == pytest.approx(mean, rel=1e-9)
    assert w.max() <= cap and w.min() > 0
    xmin = w.min()
    tail = lambda t: np.mean(w > t * xmin)
    for t in (2.0, 4.0):
        assert tail(4 * t) / tail(t) == pytest.approx(4.0 ** -(gamma - 1), rel=0.08)


def test_erdos_renyi_edge_count():
    """G(n, p): the edge count is Binomial(n(n-1)/2, p); within five standard
    deviations of its mean."""
    n, p = 2000, 0.01
    g = gg.erdos_renyi(n, p, planted=0, seed=12)
    N = n * (n - 1) / 2
    assert abs(g.m - N * p) < 5 * math.sqrt(N * p * (1 - p))


def test_rmat_shape():
    """2^scale vertices; at most edge_factor * 2^scale distinct edges after
    deduplication (plus the planted clique's), and a heavy-tailed degree
    distribution (the largest degree far above the mean)."""
    g = gg.rmat(14, 16, planted=0, seed=8)
    assert g.n == 1 << 14
    assert 0.5 * 16 * g.n < g.m <= 16 * g.n
    d = g.degrees()
    assert d.max() > 20 * d.mean()


def test_er_batch_parameter_ranges():
    for i in range(200):
        n, p, k, s = gg.er_batch_params(i, seed=3)
        assert 64 <= n <= 4096 and 8 <= k <= 24
        d = p * (n - 1)
        assert p == 1.0 or 8.0 <= d <= 64.0 + 1e-9
        assert s == (3 << 32) + i
