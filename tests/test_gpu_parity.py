"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Core numbers and omega are unique, so they must match bit for bit; every
witness must be a clique of size omega (several maximum cliques may exist, so
witnesses are checked for validity, not compared).  The deterministic
heuristic must return exactly the oracle's clique.
"""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from test_oracle import tight_instance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1302_6256_gb300 as m
    m.load_library()
    return m


_REF = {}


def ref_omega(g):
    """Oracle omega, computed once per graph."""
    if g.name not in _REF:
        _REF[g.name] = oracle.max_clique(g)[0]
    return _REF[g.name]


def load(mc, g, device=True, flags=None):
    if flags is None:
        flags = mc.MC_VALIDATE
    if device:
        return mc.mc_load_csr(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col_idx).cuda(), flags)
    return mc.mc_load_csr(g.row_ptr, g.col_idx, flags)


def small_graphs():
    out = [gg.empty(0), gg.empty(1), gg.empty(7), gg.complete(2), gg.complete(33), gg.cycle(3), gg.cycle(10),
           gg.path(9), gg.star(50), gg.petersen(), gg.complete_bipartite(5, 8), gg.turan(40, 6), gg.turan(130, 9),
           gg.disjoint_cliques([4, 17, 9, 17]), gg.mycielski(5), gg.mycielski(7)]
    for s in range(12):
        out.append(gg.random_small(5 + s, 0.2 + 0.06 * s, 500 + s))
    # every bound of Algorithm 2 met with equality by the maximum clique, the
    # heuristic one short (test_oracle.tight_instance); relabelled copies too
    for k in (3, 4, 5):
        g = tight_instance(k)[0]
        g.name = "tight%d" % k
        out.append(g)
        out.append(gg.relabel(g, 7))
    return out


def medium_graphs():
    """Sizes that span warp-class (|N+| <= 128) and block-class roots, ragged
    bit words, and several tiles."""
    return [
        gg.erdos_renyi(200, 0.5, planted=0, seed=11),
        gg.erdos_renyi(400, 0.3, planted=20, seed=12),
        gg.erdos_renyi(300, 0.6, planted=0, seed=13),
        gg.erdos_renyi(400, 0.5, planted=0, seed=19),
        gg.erdos_renyi(3000, 0.01, planted=25, seed=14),
        gg.chung_lu(20000, 2.3, 12.0, 800.0, planted=18, seed=15),
        gg.rmat(14, 16, planted=30, seed=16),
        gg.rmat(16, 16, planted=35, seed=17),
        gg.relabel(gg.turan(300, 33), 3),
    ]


@pytest.mark.parametrize("g", small_graphs() + medium_graphs(), ids=lambda g: g.name)
def test_core_numbers_bit_exact(mc, g):
    h = load(mc, g)
    core, kmax = mc.mc_core_numbers(h)
    ref = oracle.core_numbers(g)
    assert np.array_equal(core, ref)
    assert kmax == (int(ref.max()) if g.n else 0)


def _is_degeneracy_order(g, order, core):
    """Every vertex has at most K(v) neighbours after it in the order."""
    pos = np.empty(g.n, np.int64)
    pos[order] = np.arange(g.n)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    later = np.bincount(src[pos[g.col_idx] > pos[src]], minlength=g.n)
    return np.array_equal(np.sort(order), np.arange(g.n)) and bool(np.all(later <= core))


def test_peel_block_lists_overflow_and_long_cascades(mc):
    """Shapes that push the peel past its per-block lists, with core numbers
    fixed by closed forms: a perfect matching of 2^21 vertices (level 1 is
    every vertex at once, 13,800 rows per block against lists of 4,096: the
    rest becomes work items while the scan still claims), a path of 200,000
    vertices (one cascade 100,000 steps long, past a block's edge budget, so
    its list spills into the next sub-round) and K(40, 400000) (at level 40
    the 400,000 rows of 40 edges overflow the 2,048 chunk entries of every
    block).  The peel order must stay a degeneracy order."""
    n = 1 << 21
    ev = np.arange(0, n, 2)
    cases = [(gg.from_edges(n, ev, ev + 1, "matching"), 1), (gg.path(200000), 1),
             (gg.complete_bipartite(40, 400000), 40)]
    for g, k in cases:
        h = load(mc, g, flags=0)
        core, kmax = mc.mc_core_numbers(h)
        assert kmax == k and np.all(core == k), g.name
        order = mc.mc_peel_order(h).copy()
        assert _is_degeneracy_order(g, order, core), g.name
        om, wit, st = mc.mc_max_clique(h)
        assert om == 2 and oracle.is_clique(g, wit), g.name
        h.close()


@pytest.mark.parametrize("g", small_graphs() + medium_graphs(), ids=lambda g: g.name)
def test_max_clique_matches_oracle(mc, g):
    h = load(mc, g)
    om, wit, st = mc.mc_max_clique(h)
    assert om == ref_omega(g)
    assert len(wit) == om and oracle.is_clique(g, wit)
    assert list(wit) == sorted(wit)
    assert st["verified"] == 1


@pytest.mark.parametrize("g", medium_graphs(), ids=lambda g: g.name)
def test_heuristic_deterministic_bit_exact(mc, g):
    h = load(mc, g)
    H = mc.mc_heuristic_clique(h, mode=1)
    ref = oracle.heuristic_clique(g, mode=1)
    assert np.array_equal(H, ref)


@pytest.mark.parametrize("g", medium_graphs()[:6], ids=lambda g: g.name)
def test_heuristic_racy_is_valid(mc, g):
    h = load(mc, g)
    om = ref_omega(g)
    H = mc.mc_heuristic_clique(h, mode=0)
    assert 1 <= len(H) <= om and oracle.is_clique(g, H)


@pytest.mark.parametrize("opts", [dict(ordering=2), dict(no_neigh_cores=True), dict(heuristic=1),
                                  dict(heuristic=2), dict(heuristic=3), dict(warp_max=16), dict(warp_max=1),
                                  dict(no_split=True), dict(heuristic=2, warp_max=16), dict(layout=1),
                                  dict(no_bitmap=True), dict(layout=1, no_bitmap=True, heuristic=2)],
                         ids=lambda o: ",".join("%s=%s" % kv for kv in o.items()))
def test_options_keep_omega(mc, opts):
    for g in medium_graphs()[:6]:
        h = load(mc, g)
        om, wit, _ = mc.mc_max_clique(h, **opts)
        assert om == ref_omega(g), g.name
        assert oracle.is_clique(g, wit)


def test_split_tasks_keep_omega(mc):
    """Workers past their Branch-node budget spill the rest of their trees
    to the task queue.  Small budgets force spills on every tree, from warp
    and block workers and from tasks themselves; the result must equal the
    unsplit search and the oracle."""
    seen = 0
    graphs = medium_graphs()[:4] + [gg.relabel(gg.turan(300, 33), 3), gg.rmat(14, 16, planted=30, seed=16)]
    for g in graphs:
        h = load(mc, g)
        om2, wit2, st2 = mc.mc_max_clique(h, heuristic=2, warp_max=16, no_split=True)
        assert om2 == ref_omega(g), g.name
        assert st2["tasks"] == 0
        for budget in (1, 7, 64):
            for wm in (16, 0):
                om, wit, st = mc.mc_max_clique(h, heuristic=2, warp_max=wm, split_nodes=budget)
                assert om == om2, (g.name, budget, wm)
                assert oracle.is_clique(g, wit)
                seen += st["tasks"]
    assert seen > 0


def test_host_pointers_and_repeat_calls(mc):
    g = gg.chung_lu(5000, 2.4, 10.0, 500.0, planted=14, seed=21)
    h = load(mc, g, device=False)
    ref = oracle.max_clique(g)[0]
    for _ in range(3):
        om, wit, _ = mc.mc_max_clique(h)
        assert om == ref and oracle.is_clique(g, wit)


def test_device_witness_buffer(mc):
    g = gg.erdos_renyi(500, 0.2, planted=16, seed=22)
    h = load(mc, g)
    out = torch.zeros(600, dtype=torch.int32, device="cuda")
    om, wit, _ = mc.mc_max_clique(h, witness_out=out)
    assert om == oracle.max_clique(g)[0]
    assert oracle.is_clique(g, wit.cpu().numpy())


def test_batch_matches_oracle(mc):
    b = gg.er_batch(48, seed=3)
    h = mc.mc_load_batch(torch.from_numpy(b.voff).cuda(), torch.from_numpy(b.row_ptr).cuda(),
                         torch.from_numpy(b.col_idx).cuda(), mc.MC_VALIDATE)
    om, wits, st = mc.mc_max_clique_batch(h)
    for i, g in enumerate(b.graphs):
        ref = oracle.max_clique(g)[0]
        assert om[i] == ref, (i, g.name)
        assert len(wits[i]) == om[i] and oracle.is_clique(g, wits[i])
    core, _ = mc.mc_core_numbers(h)
    ref_core = np.concatenate([oracle.core_numbers(g) for g in b.graphs])
    assert np.array_equal(core, ref_core)


def test_batch_equals_single_calls(mc):
    b = gg.er_batch(16, seed=9)
    h = mc.mc_load_batch(b.voff, b.row_ptr, b.col_idx)
    om, _, _ = mc.mc_max_clique_batch(h)
    for i, g in enumerate(b.graphs):
        assert om[i] == mc.mc_max_clique(load(mc, g))[0]


def test_invalid_graph_rejected(mc):
    # asymmetric: 0->1 without 1->0
    rp = np.array([0, 1, 1], np.int64)
    ci = np.array([1], np.int32)
    with pytest.raises(mc.MCError) as e:
        mc.mc_load_csr(rp, ci, mc.MC_VALIDATE)
    assert e.value.code == mc.MC_ERR_INVALID_GRAPH
    # self loop
    rp = np.array([0, 2, 3], np.int64)
    ci = np.array([0, 1, 0], np.int32)
    with pytest.raises(mc.MCError):
        mc.mc_load_csr(rp, ci, mc.MC_VALIDATE)
    # a duplicate entry, an unsorted row, a column equal to n, a decreasing
    # row_ptr, row_ptr[0] != 0 (each array holds row_ptr[n] entries, so the
    # check reads only inside them)
    bad = [([0, 2, 3], [1, 1, 0]),
           ([0, 2, 3, 4], [2, 1, 0, 0]),
           ([0, 1, 2], [2, 0]),
           ([0, 2, 1, 4], [1, 2, 0, 0]),
           ([1, 2, 3], [1, 0, 0])]
    for rp, ci in bad:
        with pytest.raises(mc.MCError) as e:
            mc.mc_load_csr(np.array(rp, np.int64), np.array(ci, np.int32), mc.MC_VALIDATE)
        assert e.value.code == mc.MC_ERR_INVALID_GRAPH, (rp, ci)
    # a valid graph still loads after the refusals
    h = mc.mc_load_csr(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32), mc.MC_VALIDATE)
    assert mc.mc_max_clique(h)[0] == 2


def test_buffer_too_small_reports_size(mc):
    g = gg.complete(20)
    h = load(mc, g)
    with pytest.raises(mc.MCError) as e:
        mc.mc_max_clique(h, witness_out=np.zeros(5, np.int32))
    assert e.value.code == mc.MC_ERR_BUFFER


def test_spin_limit_timeout_is_reported_and_context_survives(mc):
    """A device wait that runs out returns MC_ERR_TIMEOUT (no fault), and the
    next call on the same context works."""
    g = gg.rmat(14, 16, planted=20, seed=5)
    h = load(mc, g)
    with pytest.raises(mc.MCError) as e:
        mc.mc_max_clique(h, spin_limit=1)
    assert e.value.code == mc.MC_ERR_TIMEOUT
    h2 = load(mc, g)
    om, wit, _ = mc.mc_max_clique(h2)
    assert om == oracle.max_clique(g)[0]


def test_chung_lu_20k_golden(mc):
    from graphgen import workloads as W
    gold = json.load(open(os.path.join(HERE, "golden", "chung-lu-20k.json")))
    g = W.chung_lu_20k()
    assert g.n == gold["n"] and g.m == gold["m"]
    h = load(mc, g)
    core, kmax = mc.mc_core_numbers(h)
    import hashlib
    assert hashlib.sha256(core.astype("<i4").tobytes()).hexdigest() == gold["core_sha256"]
    om, wit, _ = mc.mc_max_clique(h)
    assert om == gold["omega"]
    assert oracle.is_clique(g, wit)


def test_rmat_s22_golden(mc):
    """The benchmark's workload at full size, in the benchmark's launch
    configuration: omega and the core-number hash against the stored oracle run."""
    path = os.path.join(HERE, "golden", "rmat-s22.json")
    if not os.path.exists(path):
        pytest.skip("oracle golden file for rmat-s22 not generated")
    from graphgen import workloads as W
    import hashlib
    gold = json.load(open(path))
    g = W.rmat_s22()
    assert g.n == gold["n"] and g.m == gold["m"]
    h = load(mc, g, flags=0)
    core, kmax = mc.mc_core_numbers(h)
    assert hashlib.sha256(core.astype("<i4").tobytes()).hexdigest() == gold["core_sha256"]
    om, wit, st = mc.mc_max_clique(h)
    assert om == gold["omega"]
    assert oracle.is_clique(g, wit)


def check_omega_properties(g, om, wit, st, kmax, planted):
    """What fixes omega where the oracle's exact search is out of reach: the
    witness is a clique of size omega in g, the planted clique bounds omega
    from below, and omega <= K(G) + 1 (Fact 1) and >= the heuristic's clique."""
    assert len(wit) == om and oracle.is_clique(g, wit)
    assert planted <= om <= kmax + 1
    assert st["heuristic_size"] <= om and st["verified"] == 1


def test_rmat_s24_cores_golden(mc):
    """R-MAT scale 24 (16.8 M vertices, 260 M edges) at full size: the core
    numbers against the stored oracle run (hash and K(G)); omega against the
    oracle's threaded search once the file holds it, and always through the
    properties that fix it."""
    path = os.path.join(HERE, "golden", "rmat-s24.json")
    if not os.path.exists(path):
        pytest.skip("oracle golden file for rmat-s24 not generated")
    from graphgen import workloads as W
    import hashlib
    gold = json.load(open(path))
    g = W.rmat_s24()
    assert g.n == gold["n"] and g.m == gold["m"]
    h = load(mc, g, flags=0)
    core, kmax = mc.mc_core_numbers(h)
    assert kmax == gold["max_core"]
    assert hashlib.sha256(core.astype("<i4").tobytes()).hexdigest() == gold["core_sha256"]
    om, wit, st = mc.mc_max_clique(h)
    if gold.get("omega") is not None:
        assert om == gold["omega"]
    check_omega_properties(g, om, wit, st, kmax, 60)
    h.close()


def test_er_batch_4096_golden(mc):
    """The 4,096-graph Erdos-Renyi batch at full size (8.5 M vertices, 154 M
    edges), loaded and solved as the benchmark does (device arrays, one
    batched solve, then the same solve replayed as a CUDA graph): every
    graph's omega against the stored oracle run, every witness a clique of
    that size in its own graph."""
    path = os.path.join(HERE, "golden", "er-batch-4096.json")
    if not os.path.exists(path):
        pytest.skip("oracle golden file for the 4,096-graph batch not generated")
    from graphgen import workloads as W
    gold = json.load(open(path))
    b = W.er_batch_4096()
    assert b.count == gold["graphs"] == 4096 and b.n == gold["n"] and b.m == gold["m"]
    ref = np.array(gold["omegas"], np.int32)
    h = mc.mc_load_batch(torch.from_numpy(b.voff).cuda(), torch.from_numpy(b.row_ptr).cuda(),
                         torch.from_numpy(b.col_idx).cuda(), 0)
    for replay in (False, True, True):
        om, wits, _ = mc.mc_max_clique_batch(h, graph=replay)
        assert np.array_equal(om, ref)
    for i in range(0, b.count, 97):
        assert len(wits[i]) == ref[i] and oracle.is_clique(b.graphs[i], wits[i])
    h.close()


@pytest.mark.slow
def test_chung_lu_100m_golden(mc):
    """The social-network-scale workload (Chung-Lu, 10^8 vertices, about 1.8
    billion edges) at full size: core-number hash and K(G) against the stored
    oracle run; omega against it where the oracle reached it, else through
    the properties that fix it.  Generating the graph takes about two minutes
    on a 16-core host; MC_SKIP_FULL_SIZE=1 skips it."""
    if os.environ.get("MC_SKIP_FULL_SIZE") == "1":
        pytest.skip("MC_SKIP_FULL_SIZE=1")
    path = os.path.join(HERE, "golden", "chung-lu-100m.json")
    if not os.path.exists(path):
        pytest.skip("oracle golden file for chung-lu-100m not generated")
    from graphgen import workloads as W
    import hashlib
    gold = json.load(open(path))
    g = W.chung_lu_100m()
    assert g.n == gold["n"] and g.m == gold["m"]
    h = load(mc, g, flags=0)
    core, kmax = mc.mc_core_numbers(h)
    assert kmax == gold["max_core"]
    assert hashlib.sha256(core.astype("<i4").tobytes()).hexdigest() == gold["core_sha256"]
    om, wit, st = mc.mc_max_clique(h)
    if gold["omega"] is not None:
        assert om == gold["omega"]
    check_omega_properties(g, om, wit, st, kmax, 80)
    h.close()


def test_graph_replay_single_and_batch(mc):
    """opt graph=1: the first call solves and captures, later calls replay the
    captured CUDA graph; every replay must give the oracle's omega."""
    g = gg.rmat(14, 16, planted=30, seed=16)
    h = load(mc, g)
    for _ in range(3):
        om, wit, st = mc.mc_max_clique(h, graph=True)
        assert om == ref_omega(g) and oracle.is_clique(g, wit)
    b = gg.er_batch(32, seed=3)
    hb = mc.mc_load_batch(b.voff, b.row_ptr, b.col_idx)
    direct, _, _ = mc.mc_max_clique_batch(hb)
    for _ in range(3):
        om, wits, _ = mc.mc_max_clique_batch(hb, graph=True)
        assert np.array_equal(om, direct)
        for i, gi in enumerate(b.graphs):
            assert len(wits[i]) == om[i] and oracle.is_clique(gi, wits[i])
    for i, gi in enumerate(b.graphs[:8]):
        assert om[i] == ref_omega(gi)


def test_big_neighbourhoods_turan(mc):
    """Roots with more than 1024 later neighbours use the big-class worker
    (adjacency matrix in global memory).  Turan T(1200, 300): every vertex
    has degree 1196, omega = 300 (closed form)."""
    g = gg.relabel(gg.turan(1200, 300), 5)
    h = load(mc, g)
    core, kmax = mc.mc_core_numbers(h)
    assert kmax == 1196 and np.array_equal(core, oracle.core_numbers(g))
    om, wit, st = mc.mc_max_clique(h)
    assert om == 300
    assert oracle.is_clique(g, wit)
    om2, wit2, _ = mc.mc_max_clique(h, heuristic=2)  # no heuristic: the search finds it alone
    assert om2 == 300 and oracle.is_clique(g, wit2)


def _turan_with_planted(n, r, per_part, parts):
    """Turan T(n, r) (parts of n/r consecutive vertices) with a clique planted
    on the first `per_part` vertices of each of the first `parts` parts."""
    size = n // r
    part = np.arange(n) // size
    src, dst = [], []
    for v in range(n):
        u = np.arange(v + 1, n)
        u = u[part[u] != part[v]]
        src.append(np.full(u.size, v))
        dst.append(u)
    S = np.array([p * size + i for p in range(parts) for i in range(per_part)])
    for a in range(len(S)):
        for b in range(a + 1, len(S)):
            if part[S[a]] == part[S[b]]:
                src.append(np.array([S[a]]))
                dst.append(np.array([S[b]]))
    return gg.from_edges(n, np.concatenate(src), np.concatenate(dst), name="turan%d_%d_planted" % (n, r))


def test_neighbourhoods_beyond_4096_candidates(mc):
    """Roots with more than 4,096 candidates are solved as the graphs their
    candidates induce.  Turan T(4400, 20) (degree 4180, K(G) > 4096) with a
    clique planted on 5 vertices of each of parts 0..4: a clique holds at
    most one vertex of a part outside the planted set, so omega = 25 + 15 =
    40 by construction.  Without the heuristic the first large root's
    subgraph finds it; with it, the large roots are solved from the bound."""
    g = gg.relabel(_turan_with_planted(4400, 20, 5, 5), 13)
    h = load(mc, g, flags=0)
    core, kmax = mc.mc_core_numbers(h)
    assert kmax > 4096
    for opts in (dict(), dict(heuristic=2), dict(heuristic=2, no_split=True)):
        om, wit, st = mc.mc_max_clique(h, **opts)
        assert om == 40 and len(wit) == 40 and oracle.is_clique(g, wit), opts
        assert st["verified"] == 1 and st["huge_roots"] > 0, opts
    # a batch holding such a graph is refused before any search launch
    b = gg.Batch([g, gg.complete(3)])
    hb = mc.mc_load_batch(torch.from_numpy(b.voff).cuda(), torch.from_numpy(b.row_ptr).cuda(),
                          torch.from_numpy(b.col_idx).cuda())
    with pytest.raises(mc.MCError) as e:
        mc.mc_max_clique_batch(hb)
    assert e.value.code == mc.MC_ERR_UNSUPPORTED
    hb.close()
    h.close()


def test_autotune_returns_a_working_setting(mc):
    g = gg.rmat(14, 16, planted=30, seed=16)
    h = load(mc, g)
    opts, ms = mc.mc_autotune(h, repeats=1)
    assert opts["warp_max"] in (32, 64, 128) and ms > 0
    assert opts["layout"] in (0, 1) and opts["no_bitmap"] in (False, True)
    om, wit, _ = mc.mc_max_clique(h, **opts)
    assert om == ref_omega(g) and oracle.is_clique(g, wit)


def test_partitioned_search_matches_oracle(mc):
    """The root partition (Section 4.5) on one GPU, its parts solved one after
    the other with one shared peel order: the largest part is the oracle's
    omega and every part's witness is a clique of its size; each part
    examines only its own roots.  (No part waits on another.)"""
    from paper_1302_6256_gb300.partition import library_steps, partitioned_max_clique
    graphs = [gg.relabel(tight_instance(5)[0], 3), gg.rmat(14, 16, planted=30, seed=16),
              gg.chung_lu(20000, 2.3, 12.0, 800.0, planted=18, seed=15), gg.erdos_renyi(400, 0.5, planted=0, seed=19)]
    for g in graphs:
        ref = ref_omega(g)
        h = load(mc, g)
        mc.mc_core_numbers(h)
        order = mc.mc_peel_order(h).copy()
        whole = mc.mc_max_clique(h, order=order)[2]["roots"]
        for parts in (2, 3):
            res = [mc.mc_max_clique(h, order=order, part_rank=r, part_count=parts) for r in range(parts)]
            assert max(om for om, _, _ in res) == ref, (g.name, parts)
            for om, wit, st in res:
                assert len(wit) == om and oracle.is_clique(g, wit)
            # with the same heuristic bound the parts' roots make up all roots
            if len({st["heuristic_size"] for _, _, st in res}) == 1:
                assert sum(st["roots"] for _, _, st in res) == whole
        peel, solve = library_steps(h)
        om, wit, owner, sizes = partitioned_max_clique(peel, solve, 0, 1, g.n)
        assert om == ref and oracle.is_clique(g, wit)
        h.close()


def test_order_option_refuses_what_is_not_a_degeneracy_order(mc):
    g = gg.star(30)  # the centre first: 29 later neighbours, core number 1
    h = load(mc, g)
    for bad in (np.arange(30, dtype=np.int32), np.zeros(30, dtype=np.int32),
                np.r_[np.arange(1, 30), 30].astype(np.int32)):
        with pytest.raises(mc.MCError) as e:
            mc.mc_max_clique(h, order=bad)
        assert e.value.code == mc.MC_ERR_ARG
    for opts in (dict(part_rank=2, part_count=2), dict(part_rank=1, part_count=0),
                 dict(order=np.r_[np.arange(1, 30), 0].astype(np.int32), graph=True)):
        with pytest.raises(mc.MCError):
            mc.mc_max_clique(h, **opts)
    # a valid order (the leaves first) and a plain solve still work afterwards
    om, wit, _ = mc.mc_max_clique(h, order=np.r_[np.arange(1, 30), 0].astype(np.int32))
    assert om == 2 and oracle.is_clique(g, wit)
    assert mc.mc_max_clique(h)[0] == 2
    h.close()


@pytest.mark.parametrize("opts", [dict(repeel=4), dict(repeel=3, heuristic=2), dict(repeel=7, heuristic=2, warp_max=16),
                                  dict(repeel=2, heuristic=3, no_split=True)],
                         ids=lambda o: ",".join("%s=%s" % kv for kv in o.items()))
def test_repeel_keeps_omega(mc, opts):
    """Work-triggered re-pruning: the roots searched in ranges of peel
    positions, the pruned graph rebuilt whenever omega rose in between; omega
    equals the oracle's on graphs where the heuristic falls short."""
    graphs = medium_graphs()[:7] + [gg.relabel(tight_instance(5)[0], 9)]
    for g in graphs:
        h = load(mc, g)
        om, wit, st = mc.mc_max_clique(h, **opts)
        assert om == ref_omega(g), (g.name, opts)
        assert len(wit) == om and oracle.is_clique(g, wit) and st["verified"] == 1
        h.close()


def test_repeel_rebuilds_when_omega_rises(mc):
    """With no heuristic the first range (the densest roots) finds omega, so
    the pruned graph is rebuilt with it before the next range; the later
    ranges then examine fewer roots than one pass without the heuristic."""
    g = gg.rmat(14, 16, planted=30, seed=16)
    h = load(mc, g)
    om1, _, st1 = mc.mc_max_clique(h, heuristic=2)
    om, wit, st = mc.mc_max_clique(h, heuristic=2, repeel=4)
    assert om == om1 == ref_omega(g) and oracle.is_clique(g, wit)
    assert st["rebuilds"] >= 1 and st["roots"] < st1["roots"]
    for bad in (dict(repeel=3, graph=True), dict(repeel=3, ordering=2), dict(repeel=-1)):
        with pytest.raises(mc.MCError) as e:
            mc.mc_max_clique(h, **bad)
        assert e.value.code == mc.MC_ERR_ARG
    h.close()
