"""CUDA kernels of the learned ordering against the numpy oracle, and the
learned ordering keeping omega exact whatever the scores are."""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import learned as OL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1302_6256_gb300 as m
    m.load_library()
    return m


def test_features_match_oracle(mc):
    for g in [gg.chung_lu(3000, 2.4, 10.0, 300.0, planted=12, seed=3), gg.rmat(12, 16, planted=20, seed=4),
              gg.star(40), gg.empty(5)]:
        h = mc.mc_load_csr(g.row_ptr, g.col_idx)
        f = mc.mc_features(h)
        ref = OL.features(g, oracle.core_numbers(g))
        assert f.shape == ref.shape
        assert np.allclose(f, ref, rtol=2e-6, atol=2e-6)


def test_forward_and_gradient_match_oracle(mc):
    r = np.random.default_rng(11)
    x = r.random((1000, OL.F)).astype(np.float32)
    y = (r.random(1000) < 0.1).astype(np.float32)
    m = mc.MLP(seed=5)
    p = m.get_params()
    s = m.forward(x)
    ref = OL.forward(p, x)
    # fp32 accumulation of bf16 weights against the float64 evaluation
    assert np.allclose(s, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
    g, loss = m.gradient(x, y, pos_weight=9.0)
    gref = OL.gradient(p, x, y, 9.0)
    assert loss == pytest.approx(OL.loss(p, x, y, 9.0), rel=1e-4)
    assert np.allclose(g, gref, rtol=1e-3, atol=1e-4 * np.abs(gref).max())


def test_training_reduces_loss(mc):
    r = np.random.default_rng(2)
    x = r.random((4000, OL.F)).astype(np.float32)
    y = ((x[:, 1] + 0.5 * x[:, 3]) > 1.0).astype(np.float32)
    m = mc.MLP(seed=1)
    first = m.train_step(x, y, pos_weight=1.0, lr=3e-3)
    for _ in range(300):
        last = m.train_step(x, y, pos_weight=1.0, lr=3e-3)
    assert last < 0.5 * first
    # the trained parameters reproduce the oracle's loss
    assert m.gradient(x, y, 1.0)[1] == pytest.approx(OL.loss(m.get_params(), x, y, 1.0), rel=1e-4)


@pytest.mark.parametrize("kind", ["random", "reverse-core", "core"])
def test_learned_ordering_keeps_omega_exact(mc, kind):
    for g in [gg.chung_lu(20000, 2.3, 12.0, 800.0, planted=18, seed=15), gg.rmat(14, 16, planted=30, seed=16),
              gg.erdos_renyi(400, 0.5, planted=0, seed=19)]:
        K = oracle.core_numbers(g)
        if kind == "random":
            s = np.random.default_rng(0).random(g.n).astype(np.float32)
        elif kind == "reverse-core":
            s = -K.astype(np.float32)
        else:
            s = K.astype(np.float32)
        h = mc.mc_load_csr(g.row_ptr, g.col_idx)
        om, wit, st = mc.mc_max_clique(h, ordering=1, scores=s, seeds=16)
        assert om == oracle.max_clique(g)[0]
        assert oracle.is_clique(g, wit)
