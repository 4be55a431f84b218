"""The multi-rank root partition (Section 4.5) on CPU: two or three gloo
ranks run the exchange of paper_1302_6256_gb300.partition -- rank 0's peel
order broadcast, every rank searching its part of the roots, the sizes
gathered, the owner's witness broadcast -- with the oracle's partitioned
search as each rank's local solve; every rank must end with the oracle's
omega and a witness that is a clique of that size."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _graphs():
    import graphgen as gg
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from test_oracle import tight_instance
    return [gg.relabel(tight_instance(5)[0], 3), gg.rmat(12, 16, planted=14, seed=2),
            gg.chung_lu(3000, 2.5, 8.0, 300.0, planted=9, seed=7), gg.erdos_renyi(300, 0.5, planted=0, seed=1)]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import oracle
    from paper_1302_6256_gb300.partition import partitioned_max_clique
    out = []
    for g in _graphs():
        calls = []

        def peel_order():
            calls.append(rank)
            return oracle.core_numbers(g, with_order=True)[1]

        def solve_part(order, r, w):
            om, wit, _ = oracle.max_clique_part(g, r, w, order)
            return om, wit

        om, wit, owner, sizes = partitioned_max_clique(peel_order, solve_part, rank, world, g.n)
        out.append((om, bool(oracle.is_clique(g, wit)) and len(wit) == om, owner, sizes, calls))
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_search_gloo(world):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [oracle.max_clique(g)[0] for g in _graphs()]
    for r in range(world):
        for (om, ok, owner, sizes, calls), w in zip(res[r], want):
            assert om == w and ok
            assert max(sizes) == w and sizes[owner] == w
            assert calls == ([0] if r == 0 else [])  # only rank 0 computes the shared order
    # all ranks agree on the sizes and the owner
    for gi in range(len(want)):
        assert len({tuple(res[r][gi][3]) for r in range(world)}) == 1
        assert len({res[r][gi][2] for r in range(world)}) == 1


def test_single_rank_needs_no_process_group():
    import graphgen as gg
    import oracle
    from paper_1302_6256_gb300.partition import partitioned_max_clique
    g = gg.rmat(11, 8, planted=12, seed=3)
    om, wit, owner, sizes = partitioned_max_clique(
        lambda: oracle.core_numbers(g, with_order=True)[1],
        lambda order, r, w: oracle.max_clique_part(g, r, w, order)[:2], 0, 1, g.n)
    assert om == oracle.max_clique(g)[0] and owner == 0 and sizes == [om]
    assert oracle.is_clique(g, wit) and len(wit) == om
