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


def test_features_closed_forms():
    # star: centre 0 with n-1 leaves; every core number is 1
    n = 9
    g = gg.star(n)
    K = oracle.core_numbers(g)
    f = OL.features(g, K)
    assert np.allclose(f[0], [1.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    leaf = [np.log1p(1) / np.log1p(n - 1), 1.0, np.log1p(1) / np.log1p(n - 1), 1.0, 1.0, 1.0]
    assert np.allclose(f[1:], leaf)
    # disjoint K4 and K2: Kmax = 3, Dmax = 3
    g = gg.disjoint_cliques([4, 2])
    f = OL.features(g, oracle.core_numbers(g))
    assert np.allclose(f[0], [1.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    assert np.allclose(f[4], [np.log1p(1) / np.log1p(3), 1 / 3, np.log1p(1) / np.log1p(3), 1 / 3, 1 / 3, 1.0])
    # isolated vertex
    f = OL.features(gg.empty(3), np.zeros(3, np.int32))
    assert np.allclose(f, 0.0)


def test_features_mixed_neighbour_cores():
    """K4 on {0,1,2,3} with the path 0-4-5 attached: vertex 0 sees core
    numbers 3, 3, 3, 1, so the maximum, the mean and the count of
    neighbours at its own core number all differ (Kmax = 3, Dmax = 4)."""
    g = gg.from_edges(6, [0, 0, 0, 1, 1, 2, 0, 4], [1, 2, 3, 2, 3, 3, 4, 5])
    K = oracle.core_numbers(g)
    assert K.tolist() == [3, 3, 3, 3, 1, 1]
    f = OL.features(g, K)
    L4 = np.log1p(4)
    assert np.allclose(f[0], [1.0, 1.0, np.log1p(3) / L4, 1.0, 2.5 / 3, 3 / 4])
    assert np.allclose(f[4], [np.log1p(2) / L4, 1 / 3, np.log1p(2) / L4, 1.0, 2 / 3, 1.0])
    assert np.allclose(f[5], [np.log1p(1) / L4, 1 / 3, np.log1p(1) / L4, 1 / 3, 1 / 3, 1.0])


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
