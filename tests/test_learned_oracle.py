"""Pins of the learned-ordering oracle (features, network, loss, gradient)
against definitions, closed forms and finite differences."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import learned as OL


def random_params(seed, scale=0.3):
    r = np.random.default_rng(seed)
    return (r.standard_normal(OL.NPARAMS) * scale).astype(np.float32)


def test_bf16_rounding_closed_forms():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 65504.0], np.float32)
    r = OL.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # exact tie rounds to the even mantissa
    assert r[2] == np.float32(1.0 + 2 ** -7)
    assert r[3] == -2.5 and r[4] == 0.0
    assert r[5] == 65536.0


def test_gradient_matches_central_differences():
    r = np.random.default_rng(3)
    x = r.random((40, OL.F))
    y = (r.random(40) < 0.3).astype(np.float64)
    p = random_params(5).astype(np.float64)
    g = OL.gradient(p, x, y, 4.0, bf16=False)
    eps = 1e-6
    idx = list(range(0, OL.NPARAMS, 97)) + [OL.OFF_B3, OL.OFF_W3 + 5, OL.OFF_B1 + 7, OL.OFF_W1 + 11]
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (OL.loss(pp.astype(np.float64), x, y, 4.0, bf16=False) -
              OL.loss(pm.astype(np.float64), x, y, 4.0, bf16=False)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])), i


def test_zero_network_closed_form():
    p = np.zeros(OL.NPARAMS, np.float32)
    p[OL.OFF_B3] = 0.7
    x = np.random.default_rng(1).random((10, OL.F))
    y = np.array([1, 0, 0, 1, 0, 0, 0, 1, 0, 0], np.float64)
    s = OL.forward(p, x)
    assert np.allclose(s, 0.7)
    w = np.where(y > 0.5, 3.0, 1.0)
    sig = 1 / (1 + np.exp(-0.7))
    assert OL.loss(p, x, y, 3.0) == pytest.approx(np.mean(w * (np.log1p(np.exp(0.7)) - y * 0.7)))
    g = OL.gradient(p, x, y, 3.0)
    assert g[OL.OFF_B3] == pytest.approx(np.mean(w * (sig - y)))
    assert np.all(g[:OL.OFF_B3] == 0.0)


def test_gradient_uses_bf16_weights():
    r = np.random.default_rng(7)
    x = r.random((20, OL.F))
    y = (r.random(20) < 0.5).astype(np.float64)
    p = random_params(9)
    q = p.copy()
    for a, b in [(OL.OFF_W1, OL.OFF_B1), (OL.OFF_W2, OL.OFF_B2), (OL.OFF_W3, OL.OFF_B3)]:
        q[a:b] = OL.bf16_round(p[a:b])
    assert np.allclose(OL.gradient(p, x, y, 2.0, bf16=True), OL.gradient(q, x, y, 2.0, bf16=False))


def _f(d, dmax, k, kmax, t, chi, c):
    """The feature row for the given quantities (the definitions)."""
    T = OL.T
    return [np.log1p(d) / np.log1p(dmax), k / kmax, t / (T * (T - 1) / 2), (chi + 1) / (T + 1), c / max(d, 1),
            np.log1p(c) / np.log1p(dmax)]


def test_features_closed_forms():
    # star: centre 0 with n-1 leaves, every core number 1; the leaves are
    # pairwise non-adjacent, so no triangle and one colour
    n = 9
    g = gg.star(n)
    f = OL.features(g, oracle.core_numbers(g))
    assert np.allclose(f[0], _f(8, 8, 1, 1, 0, 1, 8))
    assert np.allclose(f[1:], _f(1, 8, 1, 1, 0, 1, 1))
    # K_n: Q is the first min(T, n-1) other vertices, all adjacent
    for n in (5, 17, 20):
        g = gg.complete(n)
        f = OL.features(g, oracle.core_numbers(g))
        q = min(OL.T, n - 1)
        assert np.allclose(f, _f(n - 1, n - 1, n - 1, n - 1, q * (q - 1) // 2, q, n - 1))
    # cycles: the two neighbours are adjacent only in C_3
    g = gg.cycle(3)
    assert np.allclose(OL.features(g, oracle.core_numbers(g)), _f(2, 2, 2, 2, 1, 2, 2))
    g = gg.cycle(8)
    assert np.allclose(OL.features(g, oracle.core_numbers(g)), _f(2, 2, 2, 2, 0, 1, 2))
    # disjoint K4 and K2: Kmax = 3, Dmax = 3
    g = gg.disjoint_cliques([4, 2])
    f = OL.features(g, oracle.core_numbers(g))
    assert np.allclose(f[0], _f(3, 3, 3, 3, 3, 3, 3))
    assert np.allclose(f[4], _f(1, 3, 1, 3, 0, 1, 1))
    # isolated vertices: no neighbour, chi = 0
    f = OL.features(gg.empty(3), np.zeros(3, np.int32))
    assert np.allclose(f, [[0.0, 0.0, 0.0, 1 / (OL.T + 1), 0.0, 0.0]] * 3)


def test_features_turan_worked_by_hand():
    """Turan T(32, 4), parts = id mod 4, 24-regular (every core number 24).
    Vertex 0's first 8 neighbours are 1 2 3 5 6 7 9 10: parts 1, 2, 3 with
    3, 3 and 2 members.  Edges among them join different parts:
    C(8,2) - 2 C(3,2) - C(2,2) = 28 - 6 - 1 = 21.  The greedy colouring of a
    complete multipartite graph gives each part one colour: 3 colours."""
    assert OL.T == 8
    g = gg.turan(32, 4)
    f = OL.features(g, oracle.core_numbers(g))
    assert np.allclose(f[0], _f(24, 24, 24, 24, 21, 3, 24))
    # vertex 5 (part 1): first neighbours 0 2 3 4 6 7 8 10, parts 0, 2, 3
    # with 3, 3, 2 members again
    assert np.allclose(f[5], _f(24, 24, 24, 24, 21, 3, 24))
    # vertex 31 (part 3): first neighbours 0 1 2 4 5 6 8 9, parts 0, 1, 2
    # with 3, 3, 2 members
    assert np.allclose(f[31], _f(24, 24, 24, 24, 21, 3, 24))


def test_features_first_T_in_id_order():
    """Q(v) is the FIRST T qualifying neighbours in id order.  Vertex 0 is
    joined to 1..20; 1..16 are pairwise adjacent; each of 17..20 is joined to
    all of 1..16 and to nothing else.  Degrees: 20 (0 and 1..16), 17
    (17..20); the whole graph is a 17-core and no 18-core exists, so every
    core number is 17.  With T = 8, Q(0) = 1..8, a clique: 28 edges, 8
    colours.  (The last 8 neighbours, 13..20, would give C(4,2) + 4 * 4 = 22
    edges and 5 colours.)  Q(17) = 0..7 and Q(1) = 0, 2..8: cliques too."""
    assert OL.T == 8
    src, dst = [], []
    for u in range(1, 21):
        src.append(0)
        dst.append(u)
    for a in range(1, 17):
        for b in range(a + 1, 17):
            src.append(a)
            dst.append(b)
        for b in range(17, 21):
            src.append(a)
            dst.append(b)
    g = gg.from_edges(21, src, dst)
    K = oracle.core_numbers(g)
    assert np.all(K == 17)
    f = OL.features(g, K)
    assert np.allclose(f[0], _f(20, 20, 17, 17, 28, 8, 20))
    assert np.allclose(f[17], _f(17, 20, 17, 17, 28, 8, 17))
    assert np.allclose(f[1], _f(20, 20, 17, 17, 28, 8, 20))


def test_features_mixed_neighbour_cores():
    """K4 on {0,1,2,3} with the path 0-4-5 attached: vertex 0 (K = 3) keeps
    its three K4 neighbours (a triangle, three colours) and not vertex 4
    (K = 1); vertex 4 keeps both neighbours 0 and 5, which are not adjacent
    (Kmax = 3, Dmax = 4)."""
    g = gg.from_edges(6, [0, 0, 0, 1, 1, 2, 0, 4], [1, 2, 3, 2, 3, 3, 4, 5])
    K = oracle.core_numbers(g)
    assert K.tolist() == [3, 3, 3, 3, 1, 1]
    f = OL.features(g, K)
    assert np.allclose(f[0], _f(4, 4, 3, 3, 3, 3, 3))
    assert np.allclose(f[1], _f(3, 4, 3, 3, 3, 3, 3))
    assert np.allclose(f[4], _f(2, 4, 1, 3, 0, 1, 2))
    assert np.allclose(f[5], _f(1, 4, 1, 3, 0, 1, 1))


def test_features_core_filter_before_truncation():
    """Q(v) takes the first T neighbours among those with K(u) >= K(v), not
    the first T neighbours: vertex 0 is joined to T leaves (ids 1..T) and is
    in a (T+1)-clique with ids T+1..2T.  The leaves come first in id order
    but have core number 1 < K(0) = T, so Q(0) is the T clique members (all
    adjacent, T colours)."""
    T = OL.T
    # vertices 1..T: independent, each joined to 0; vertices T+1..2T: K_T with 0
    src, dst = [], []
    for u in range(1, T + 1):
        src.append(0)
        dst.append(u)
    clique = [0] + list(range(T + 1, 2 * T + 1))
    for a in range(len(clique)):
        for b in range(a + 1, len(clique)):
            src.append(clique[a])
            dst.append(clique[b])
    g = gg.from_edges(2 * T + 1, src, dst)
    K = oracle.core_numbers(g)
    assert K[0] == T and K[1] == 1 and K[T + 1] == T
    f = OL.features(g, K)
    # vertex 0: degree 2T, c = T (the clique members), Q = the clique members
    assert np.allclose(f[0], _f(2 * T, 2 * T, T, T, T * (T - 1) // 2, T, T))
    # a leaf (K = 1): its one neighbour 0 has K >= 1
    assert np.allclose(f[1], _f(1, 2 * T, 1, T, 0, 1, 1))


def test_adam_closed_forms():
    """Adam's bias correction makes a constant gradient g move every
    parameter by lr * g / (|g| + eps) at every step, the first included; a
    zero gradient never moves it; the moments follow their geometric sums."""
    r = np.random.default_rng(4)
    p0 = r.standard_normal(50)
    g = r.standard_normal(50) * 10.0 ** r.integers(-6, 2, 50)
    g[:3] = 0.0
    lr = 1e-3
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 6):
        q, m, v = OL.adam_step(p, m, v, g, t, lr)
        assert np.allclose(p - q, lr * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)
        p = q
    assert np.all(p[:3] == p0[:3])
    assert np.allclose(m, (1 - 0.9 ** 5) * g) and np.allclose(v, (1 - 0.999 ** 5) * g * g)
    # two steps with different gradients, worked out by hand for one parameter
    q, m1, v1 = OL.adam_step([1.0], [0.0], [0.0], [2.0], 1, 0.1)
    q, m2, v2 = OL.adam_step(q, m1, v1, [-1.0], 2, 0.1)
    mh = (0.9 * 0.2 - 0.1) / (1 - 0.81)
    vh = (0.999 * 0.004 + 0.001) / (1 - 0.999 ** 2)
    assert q[0] == pytest.approx(1.0 - 0.1 * 2.0 / (2.0 + 1e-8) - 0.1 * mh / (np.sqrt(vh) + 1e-8), rel=1e-12)
