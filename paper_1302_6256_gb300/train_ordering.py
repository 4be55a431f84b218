"""Train the vertex-scoring network of the learned ordering.

Training data: generated graphs (a mix of Chung-Lu graphs with hub cores
from sparse to dense and R-MAT graphs, n from 10k to 200k, a planted clique
of 10 to 50 vertices), each solved exactly by this
library; a vertex is labelled 1 if it is in the maximum clique the exact solve
returns.  Rows: every positive vertex, plus negatives drawn half from all
vertices and half from the hard ones (core number >= omega - 1), up to
`neg_ratio` per positive.  The network (6 -> 64 -> 64 -> 1, BF16 weights,
FP32 accumulation) is trained by the library's own forward, backward and
Adam kernels; the scores never change omega, only the search order.

    python -m paper_1302_6256_gb300.train_ordering --graphs 2000 --out ordering_mlp.npy
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import graphgen as gg  # noqa: E402
import paper_1302_6256_gb300 as mc  # noqa: E402

DEFAULT_OUT = os.path.join(HERE, "ordering_mlp.npy")


def graph_params(i: int, seed: int):
    """Family and sizes of training graph i (counter-based, reproducible).
    Chung-Lu graphs take their weight cap from the hub-to-hub edge
    probability cap^2 / (n mean), drawn in [0.01, 0.25]: from hub cores that
    hold small cliques only (the planted clique has a low core number, as in
    a social network of 10^8 vertices) to dense hub cores."""
    k = gg.key(seed, 5000 + i)
    u = [(gg.rand_u64(k, j) >> 11) / 9007199254740992.0 for j in range(6)]
    planted = 10 + int(u[1] * 41)
    if u[0] < 0.5:
        n = 10_000 + int(u[2] * 190_001)
        gamma = 2.1 + 0.7 * u[3]
        mean = 6.0 + 34.0 * u[4]
        cap = (0.1 + 0.4 * u[5]) * (n * mean) ** 0.5
        return ("chung-lu", dict(n=n, gamma=gamma, mean=mean, cap=max(50.0, cap), planted=planted,
                                 seed=(seed << 20) + i))
    scale = 14 + int(u[2] * 4)  # 16k .. 131k vertices
    return ("rmat", dict(scale=scale, edge_factor=8 + int(u[3] * 9), planted=planted, seed=(seed << 20) + i))


def make_graph(i: int, seed: int):
    fam, p = graph_params(i, seed)
    if fam == "chung-lu":
        return gg.chung_lu(p["n"], p["gamma"], p["mean"], p["cap"], planted=p["planted"], seed=p["seed"])
    return gg.rmat(p["scale"], p["edge_factor"], planted=p["planted"], seed=p["seed"])


def sample_rows(g, feat, core, witness, omega, rng, neg_ratio):
    pos = np.zeros(g.n, bool)
    pos[witness] = True
    pidx = np.nonzero(pos)[0]
    hard = np.nonzero((core >= max(omega - 1, 0)) & ~pos)[0]
    anyneg = np.nonzero(~pos)[0]
    want = neg_ratio * max(len(pidx), 1)
    h = rng.choice(hard, size=min(len(hard), want // 2), replace=False) if len(hard) else np.zeros(0, int)
    a = rng.choice(anyneg, size=min(len(anyneg), want - len(h)), replace=False) if len(anyneg) else np.zeros(0, int)
    idx = np.concatenate([pidx, h, a])
    return feat[idx], pos[idx].astype(np.float32)


def _log(*a):
    print(*a, flush=True)


def build_dataset(graphs: int, seed: int, neg_ratio: int, workers: int, log=_log, budget_s: float = 0.0):
    rng = np.random.default_rng(seed)
    X, Y, info = [], [], []
    t0 = time.time()
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(make_graph, i, seed) for i in range(min(graphs, workers * 2))]
        nxt = len(futs)
        for i in range(graphs):
            g = futs[i].result()
            if nxt < graphs:
                futs.append(ex.submit(make_graph, nxt, seed))
                nxt += 1
            h = mc.mc_load_csr(g.row_ptr, g.col_idx)
            om, wit, st = mc.mc_max_clique(h)
            core, _ = mc.mc_core_numbers(h)
            feat = mc.mc_features(h)
            h.close()
            x, y = sample_rows(g, feat, np.asarray(core), np.asarray(wit), om, rng, neg_ratio)
            X.append(x)
            Y.append(y)
            info.append((g.n, g.m, om, st["heuristic_size"]))
            futs[i] = None
            if (i + 1) % max(1, graphs // 20) == 0:
                log("  %d/%d graphs, %.0f s" % (i + 1, graphs, time.time() - t0))
            if budget_s > 0 and time.time() - t0 > budget_s:
                log("  time budget reached after %d graphs" % (i + 1))
                break
        for f in futs:
            if f is not None:
                f.cancel()
    return np.concatenate(X), np.concatenate(Y), info


def train(X, Y, epochs: int, batch: int, lr: float, seed: int, log=_log):
    m = mc.MLP(seed=seed)
    npos = float(Y.sum())
    pos_weight = (len(Y) - npos) / max(npos, 1.0)
    rng = np.random.default_rng(seed)
    import torch
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    losses = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(len(Y))).cuda()
        tot, nb = 0.0, 0
        for b in range(0, len(Y), batch):
            idx = perm[b:b + batch]
            xb = Xd[idx].contiguous()
            yb = Yd[idx].contiguous()
            tot += m.train_step(xb, yb, pos_weight=pos_weight, lr=lr)
            nb += 1
        losses.append(tot / max(nb, 1))
        log("  epoch %d loss %.4f" % (ep + 1, losses[-1]))
    return m, pos_weight, losses


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--neg-ratio", type=int, default=40)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--budget-s", type=float, default=0.0, help="stop adding graphs after this many seconds")
    a = ap.parse_args(argv)
    t = time.time()
    X, Y, info = build_dataset(a.graphs, a.seed, a.neg_ratio, a.workers, budget_s=a.budget_s)
    print("dataset: %d rows, %d positive, %.0f s" % (len(Y), int(Y.sum()), time.time() - t), flush=True)
    m, pw, losses = train(X, Y, a.epochs, a.batch, a.lr, a.seed)
    p = m.get_params()
    np.save(a.out, p)
    meta = {"graphs": len(info), "graphs_requested": a.graphs, "seed": a.seed, "rows": int(len(Y)), "positives": int(Y.sum()), "pos_weight": pw,
            "epochs": a.epochs, "lr": a.lr, "batch": a.batch, "losses": losses,
            "omega_gap_mean": float(np.mean([o - hs for (_, _, o, hs) in info])), "seconds": time.time() - t}
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    main()
