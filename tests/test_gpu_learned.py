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
    """Every feature of every vertex against the oracle's definitions, on
    graphs where Q(v) is cut at 16 neighbours (K_20, Turan, the dense R-MAT
    core) and where it is short or empty (stars, paths, isolated vertices).
    The triangle count and the colouring bound are integers before the
    division, so they must agree exactly; the float tolerance covers the
    float32 logarithms and divisions."""
    for g in [gg.chung_lu(3000, 2.4, 10.0, 300.0, planted=12, seed=3), gg.rmat(12, 16, planted=20, seed=4),
              gg.star(40), gg.empty(5), gg.complete(20), gg.turan(64, 5), gg.relabel(gg.turan(90, 7), 2),
              gg.path(7), gg.erdos_renyi(500, 0.1, planted=14, seed=6)]:
        h = mc.mc_load_csr(g.row_ptr, g.col_idx)
        f = mc.mc_features(h)
        ref = OL.features(g, oracle.core_numbers(g))
        assert f.shape == ref.shape
        assert np.allclose(f, ref, rtol=2e-6, atol=2e-6), g.name
        T = OL.T
        assert np.array_equal(np.rint(f[:, 2] * (T * (T - 1) / 2)), np.rint(ref[:, 2] * (T * (T - 1) / 2)))
        assert np.array_equal(np.rint(f[:, 3] * (T + 1)), np.rint(ref[:, 3] * (T + 1)))


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


@pytest.mark.parametrize("heuristic", [0, 3])
@pytest.mark.parametrize("ordering", [0, 1])
def test_learned_form_keeps_omega_exact(mc, heuristic, ordering):
    """The learned form (mlp option): warm-up bound, scores of the vertices
    that can beat it, seeds grown first, then the rest of Algorithm 1 or
    not; omega equals the oracle's for an untrained and a trained network,
    and the scored vertices are a subset of the graph that contains every
    vertex the pruning keeps."""
    import os
    w = np.load(os.path.join(os.path.dirname(mc.__file__), "ordering_mlp.npy"))
    nets = [mc.MLP(seed=3), mc.MLP(seed=0)]
    nets[1].set_params(w)
    graphs = [gg.chung_lu(20000, 2.3, 12.0, 800.0, planted=18, seed=15), gg.rmat(14, 16, planted=30, seed=16),
              gg.erdos_renyi(400, 0.5, planted=0, seed=19), _dense_core_and_path(), gg.relabel(gg.turan(300, 33), 3)]
    for g in graphs:
        ref = oracle.max_clique(g)[0]
        h = mc.mc_load_csr(g.row_ptr, g.col_idx)
        for net in nets:
            for seeds in (0, 5, 300):
                om, wit, st = mc.mc_max_clique(h, mlp=net, heuristic=heuristic, ordering=ordering, seeds=seeds)
                assert om == ref, (g.name, seeds)
                assert oracle.is_clique(g, wit) and len(wit) == om
                assert st["pruned_n"] <= st["learned_scored"] <= g.n
                assert st["verified"] == 1
        h.close()


def test_learned_form_batch_and_replay(mc):
    """The learned form on a batch (seeds per graph) and replayed as a CUDA
    graph: every graph's omega equals the oracle's."""
    b = gg.er_batch(48, seed=3)
    ref = np.array([oracle.max_clique(g)[0] for g in b.graphs], np.int32)
    h = mc.mc_load_batch(torch.from_numpy(b.voff).cuda(), torch.from_numpy(b.row_ptr).cuda(),
                         torch.from_numpy(b.col_idx).cuda(), mc.MC_VALIDATE)
    net = mc.MLP(seed=4)
    for opts in (dict(heuristic=0), dict(heuristic=3), dict(heuristic=3, seeds=1), dict(heuristic=3, graph=True),
                 dict(heuristic=3, graph=True)):
        om, wits, st = mc.mc_max_clique_batch(h, mlp=net, **opts)
        assert np.array_equal(om, ref), opts
        for i, g in enumerate(b.graphs):
            assert len(wits[i]) == om[i] and oracle.is_clique(g, wits[i])
    h.close()


def test_learned_form_refuses_bad_options(mc):
    g = gg.rmat(10, 8, planted=10, seed=1)
    h = mc.mc_load_csr(g.row_ptr, g.col_idx)
    net = mc.MLP(seed=1)
    for opts in (dict(heuristic=1), dict(heuristic=2), dict(seeds=1025),
                 dict(scores=np.zeros(g.n, np.float32))):
        with pytest.raises(mc.MCError) as e:
            mc.mc_max_clique(h, mlp=net, **opts)
        assert e.value.code == mc.MC_ERR_ARG
    h.close()


def _bits(u):
    return np.array([u], dtype=np.uint32).view(np.float32)[0]


def _dense_core_and_path(tail=3000):
    """Erdos-Renyi G(300, 1/2) (omega 12, Algorithm 1's clique 11: the
    search must find the maximum clique) beside a path of `tail` vertices
    (core number 1: pruned, so most vertices are gone before the roots are
    ordered)."""
    d = gg.erdos_renyi(300, 0.5, planted=0, seed=1)
    src = np.repeat(np.arange(d.n, dtype=np.int64), np.diff(d.row_ptr))
    keep = src < d.col_idx
    p = np.arange(d.n, d.n + tail - 1)
    return gg.from_edges(d.n + tail, np.concatenate([src[keep], p]), np.concatenate([d.col_idx[keep], p + 1]))


def test_learned_ordering_accepts_any_float_score(mc):
    """Scores of -inf, +inf, NaN of either sign and the most negative finite
    float order the roots like any other value, so no root is lost: on a
    graph where the heuristic stops one short of omega and most vertices
    are pruned, omega is still found."""
    g = _dense_core_and_path()
    om_ref = oracle.max_clique(g)[0]
    assert len(oracle.heuristic_clique(g, mode=1)) < om_ref
    s = np.random.default_rng(1).standard_normal(g.n).astype(np.float32)
    s[::3] = -np.inf
    s[1::5] = _bits(0x7FC00000)   # NaN
    s[2::7] = _bits(0xFFC00000)   # NaN, sign bit set
    s[5::9] = _bits(0xFFFFFFFF)   # NaN, every bit set
    s[3::11] = np.inf
    s[4::13] = np.finfo(np.float32).min
    h = mc.mc_load_csr(g.row_ptr, g.col_idx)
    for sc in (s, np.full(g.n, -np.inf, dtype=np.float32), np.full(g.n, _bits(0xFFFFFFFF), dtype=np.float32)):
        om, wit, st = mc.mc_max_clique(h, heuristic=1, ordering=1, scores=sc)
        assert st["heuristic_size"] < om_ref and st["pruned_n"] == 300
        assert om == om_ref and oracle.is_clique(g, wit) and len(wit) == om
    h.close()


def test_graph_replay_with_host_scores(mc):
    """A captured solve with learned scores in host memory: every replay
    copies the array's current contents, and omega stays exact."""
    g = gg.rmat(14, 16, planted=30, seed=16)
    om_ref = oracle.max_clique(g)[0]
    rng = np.random.default_rng(3)
    s = rng.random(g.n).astype(np.float32)
    h = mc.mc_load_csr(g.row_ptr, g.col_idx)
    for _ in range(3):
        s[:] = rng.random(g.n)
        om, wit, st = mc.mc_max_clique(h, ordering=1, scores=s, seeds=16, graph=True)
        assert om == om_ref and oracle.is_clique(g, wit) and len(wit) == om
    h.close()


def test_trained_network_raises_the_lower_bound(mc):
    """What the committed network (trained on 2,000 generated Chung-Lu and
    R-MAT graphs, seed 7) gains over the method without it, on 60 held-out
    graphs of the same families (seed 11).  In the deterministic heuristic
    the seeds only add candidate cliques (each seed grown by highest score),
    so the lower bound can only rise; the trained network must close part of
    the gap between it and omega, more than random scores do, and omega never
    changes."""
    import os
    from paper_1302_6256_gb300 import train_ordering as T
    w = np.load(os.path.join(os.path.dirname(mc.__file__), "ordering_mlp.npy"))
    net = mc.MLP(seed=0)
    net.set_params(w)
    rng = np.random.default_rng(5)
    gap = {"plain": 0, "learned": 0, "random": 0}
    for i in range(60):
        g = T.make_graph(i, 11)
        h = mc.mc_load_csr(g.row_ptr, g.col_idx)
        feat = torch.zeros((g.n, 6), dtype=torch.float32, device="cuda")
        score = torch.zeros(g.n, dtype=torch.float32, device="cuda")
        mc.mc_features(h, feat)
        net.forward(feat, score)
        rand = torch.from_numpy(rng.random(g.n).astype(np.float32)).cuda()
        om, _, st = mc.mc_max_clique(h, heuristic=1)
        om_l, wit_l, st_l = mc.mc_max_clique(h, heuristic=1, ordering=1, scores=score, seeds=64)
        om_r, _, st_r = mc.mc_max_clique(h, heuristic=1, ordering=1, scores=rand, seeds=64)
        assert om == om_l == om_r
        assert oracle.is_clique(g, wit_l) and len(wit_l) == om
        assert st_l["heuristic_size"] >= st["heuristic_size"]
        assert st_r["heuristic_size"] >= st["heuristic_size"]
        gap["plain"] += om - st["heuristic_size"]
        gap["learned"] += om - st_l["heuristic_size"]
        gap["random"] += om - st_r["heuristic_size"]
        h.close()
    print("lower-bound gap over 60 held-out graphs:", gap)
    assert gap["learned"] < gap["plain"]
    assert gap["learned"] < gap["random"]
