"""The training step's Adam update against the oracle's Adam step.

The gradient kernel is compared with the oracle in test_gpu_learned.py;
here the update that follows it is: each step reads the kernel's own
gradient at the current parameters, takes one training step on the same
rows, and checks the new float32 master parameters against the oracle's
Adam step (float64) applied to that gradient from the same parameters and
moments."""
import numpy as np
import pytest

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


def test_adam_steps_match_oracle(mc):
    r = np.random.default_rng(21)
    x = r.random((2000, OL.F)).astype(np.float32)
    y = (r.random(2000) < 0.2).astype(np.float32)
    lr, pw = 1e-3, 4.0
    net = mc.MLP(seed=3)
    p = net.get_params().astype(np.float64)
    m = np.zeros(OL.NPARAMS)
    v = np.zeros(OL.NPARAMS)
    big = np.ones(OL.NPARAMS, bool)
    for t in range(1, 4):
        g, _ = net.gradient(x, y, pos_weight=pw)
        g = np.asarray(g, dtype=np.float64)
        net.train_step(x, y, pos_weight=pw, lr=lr)
        got = net.get_params().astype(np.float64)
        ref, m, v = OL.adam_step(p, m, v, g, t, lr)
        # float32 masters of magnitude <= ~1: half an ulp is 6e-8.  The
        # training step recomputes the gradient with float atomics, so where
        # |g| has been near Adam's eps (1e-8) a different summation order can
        # move the update (and the moments after it); those entries are held
        # only to Adam's largest step, lr (1 - beta1) / sqrt(1 - beta2) ~ 3.2 lr,
        # on either side.
        big &= np.abs(g) >= 1e-6
        assert big.mean() > 0.5
        assert np.allclose(got[big], ref[big], rtol=1e-6, atol=1e-7), t
        assert np.all(np.abs(got - ref) <= 7 * lr), t
        p = got
