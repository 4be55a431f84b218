"""Seeded synthetic graph generators (shared input module).

This package is the only code that both the CPU oracle side and the CUDA side
use.  It draws random graphs and builds simple, symmetric, sorted CSR arrays
(``row_ptr`` int64[n+1], ``col_idx`` int32[2m]); it holds none of the clique
method's arithmetic.  The C core (``graphgen.c``) is compiled on first use with
``-ffp-contract=off`` so that x86-64 and AArch64 hosts generate bit-identical
graphs.

Workload shapes follow the paper's social and information networks (Table 1:
heavy-tailed degrees, a dense core, a large clique): Chung-Lu power-law graphs,
R-MAT graphs and batches of small Erdos-Renyi graphs, each optionally with a
planted clique of k uniformly chosen vertices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgraphgen.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``graphgen.c`` into ``_build/libgraphgen.so`` (idempotent)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
            vp = ctypes.c_void_p
            lib.gg_key.argtypes = [u64, u64]; lib.gg_key.restype = u64
            lib.gg_rand.argtypes = [u64, u64]; lib.gg_rand.restype = u64
            lib.gg_log.argtypes = [dbl]; lib.gg_log.restype = dbl
            lib.gg_exp.argtypes = [dbl]; lib.gg_exp.restype = dbl
            lib.gg_rmat_edges.argtypes = [i32, i64, dbl, dbl, dbl, u64, i32, vp, vp]
            lib.gg_rmat_edges.restype = i32
            lib.gg_chung_lu_weights.argtypes = [i64, dbl, dbl, dbl, u64, vp]
            lib.gg_chung_lu_weights.restype = i32
            lib.gg_chung_lu_edges.argtypes = [i64, vp, i64, u64, i32, vp, vp]
            lib.gg_chung_lu_edges.restype = i32
            lib.gg_er_edges.argtypes = [i64, dbl, u64, vp, vp, i64]
            lib.gg_er_edges.restype = i64
            lib.gg_planted.argtypes = [i64, i64, u64, vp, vp, vp]
            lib.gg_planted.restype = i32
            lib.gg_csr_from_edges.argtypes = [i64, i64, vp, vp, i32, vp, vp]
            lib.gg_csr_from_edges.restype = i64
            lib.gg_permutation.argtypes = [i64, u64, vp]
            lib.gg_permutation.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


class Graph:
    """A simple undirected graph in CSR form plus how it was made."""

    def __init__(self, row_ptr: np.ndarray, col_idx: np.ndarray, name: str = "",
                 planted: np.ndarray | None = None):
        self.row_ptr = row_ptr
        self.col_idx = col_idx
        self.name = name
        self.planted = planted if planted is not None else np.zeros(0, np.int32)

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        """Undirected edge count."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def __repr__(self) -> str:
        return "Graph(%s, n=%d, m=%d)" % (self.name, self.n, self.m)


def key(seed: int, stream: int) -> int:
    return int(_L().gg_key(seed & (2**64 - 1), stream & (2**64 - 1)))


def rand_u64(k: int, ctr: int) -> int:
    return int(_L().gg_rand(k, ctr))


def det_log(x: float) -> float:
    return float(_L().gg_log(x))


def det_exp(x: float) -> float:
    return float(_L().gg_exp(x))


def from_edges(n: int, src, dst, name: str = "", planted=None) -> Graph:
    """Simple symmetric CSR (sorted rows, no loops, no duplicates) from pairs."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    row_ptr = np.zeros(n + 1, np.int64)
    col = np.empty(max(1, 2 * m), np.int32)
    nnz = _L().gg_csr_from_edges(n, m, _ptr(src), _ptr(dst), _threads(), _ptr(row_ptr), _ptr(col))
    if nnz < 0:
        raise MemoryError("graphgen: CSR build failed (%d)" % nnz)
    return Graph(row_ptr, col[:nnz].copy(), name, planted)


def _planted_edges(n: int, k: int, seed: int):
    members = np.zeros(max(k, 1), np.int32)
    kk = k * (k - 1) // 2
    s = np.zeros(max(kk, 1), np.int32)
    d = np.zeros(max(kk, 1), np.int32)
    if k > 0:
        rc = _L().gg_planted(n, k, seed, _ptr(members), _ptr(s), _ptr(d))
        if rc != 0:
            raise ValueError("graphgen: planted clique of %d in n=%d" % (k, n))
    return members[:k].copy(), s[:kk], d[:kk]


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         planted: int = 0, seed: int = 1) -> Graph:
    """R-MAT graph on 2**scale vertices from edge_factor * 2**scale sampled
    edges (no noise, vertex ids randomly relabelled), symmetrised and
    deduplicated, plus an optional planted clique."""
    n = 1 << scale
    ne = edge_factor * n
    members, ps, pd = _planted_edges(n, planted, seed)
    src = np.empty(ne + ps.shape[0], np.int32)
    dst = np.empty(ne + ps.shape[0], np.int32)
    rc = _L().gg_rmat_edges(scale, ne, a, b, c, seed, _threads(), _ptr(src), _ptr(dst))
    if rc != 0:
        raise ValueError("graphgen: rmat failed (%d)" % rc)
    src[ne:] = ps
    dst[ne:] = pd
    name = "rmat scale=%d ef=%d abc=(%g,%g,%g) planted=%d seed=%d" % (scale, edge_factor, a, b, c, planted, seed)
    return from_edges(n, src, dst, name, members)


def chung_lu(n: int, gamma: float, mean: float, cap: float, planted: int = 0, seed: int = 1) -> Graph:
    """Chung-Lu graph: i.i.d. Pareto(gamma) expected degrees with the given mean
    (after capping at cap, the weights' mean), round(n * mean / 2) endpoint
    pairs drawn proportional to w, then symmetrised and deduplicated, plus an
    optional planted clique."""
    w = np.empty(n, np.float64)
    rc = _L().gg_chung_lu_weights(n, gamma, mean, cap, seed, _ptr(w))
    if rc != 0:
        raise ValueError("graphgen: chung-lu weights failed (%d)" % rc)
    ne = int(round(n * mean / 2.0))
    members, ps, pd = _planted_edges(n, planted, seed)
    src = np.empty(ne + ps.shape[0], np.int32)
    dst = np.empty(ne + ps.shape[0], np.int32)
    rc = _L().gg_chung_lu_edges(n, _ptr(w), ne, seed, _threads(), _ptr(src), _ptr(dst))
    if rc != 0:
        raise MemoryError("graphgen: chung-lu edges failed (%d)" % rc)
    src[ne:] = ps
    dst[ne:] = pd
    name = "chung-lu n=%d gamma=%g mean=%g cap=%g planted=%d seed=%d" % (n, gamma, mean, cap, planted, seed)
    return from_edges(n, src, dst, name, members)


def erdos_renyi(n: int, p: float, planted: int = 0, seed: int = 1) -> Graph:
    """G(n, p) plus an optional planted clique."""
    exp_m = p * n * (n - 1) / 2.0
    cap = int(min(n * (n - 1) // 2, exp_m + 10 * (exp_m ** 0.5) + 64))
    src = np.empty(cap + planted * planted, np.int32)
    dst = np.empty(cap + planted * planted, np.int32)
    m = _L().gg_er_edges(n, p, seed, _ptr(src), _ptr(dst), cap)
    if m < 0:
        raise RuntimeError("graphgen: er edge buffer too small")
    members, ps, pd = _planted_edges(n, planted, seed)
    src[m:m + ps.shape[0]] = ps
    dst[m:m + ps.shape[0]] = pd
    tot = m + ps.shape[0]
    return from_edges(n, src[:tot], dst[:tot], "er n=%d p=%.6g planted=%d seed=%d" % (n, p, planted, seed), members)


# ------------------------------------------------------------ batches ---

class Batch:
    """Many independent graphs stored as one block-diagonal CSR.

    ``voff[g]:voff[g+1]`` is the vertex range of graph g; column indices are
    global (vertex ids of the union)."""

    def __init__(self, graphs: list[Graph], name: str = ""):
        self.graphs = graphs
        self.name = name
        ns = np.array([g.n for g in graphs], np.int64)
        self.voff = np.zeros(len(graphs) + 1, np.int64)
        np.cumsum(ns, out=self.voff[1:])
        nnzs = np.array([g.nnz for g in graphs], np.int64)
        eoff = np.zeros(len(graphs) + 1, np.int64)
        np.cumsum(nnzs, out=eoff[1:])
        n = int(self.voff[-1])
        self.row_ptr = np.zeros(n + 1, np.int64)
        self.col_idx = np.empty(int(eoff[-1]), np.int32)
        for i, g in enumerate(graphs):
            v0 = int(self.voff[i])
            self.row_ptr[v0 + 1:v0 + g.n + 1] = g.row_ptr[1:] + eoff[i]
            self.col_idx[eoff[i]:eoff[i + 1]] = g.col_idx + v0

    @property
    def count(self) -> int:
        return len(self.graphs)

    @property
    def n(self) -> int:
        return int(self.voff[-1])

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1]) // 2


def er_batch_params(i: int, seed: int = 3):
    """Parameters of graph i of the Erdos-Renyi batch: n ~ U[64, 4096],
    mean degree ~ U[8, 64], planted clique size ~ U[8, 24], p = min(1, d/(n-1))."""
    k = key(seed, 1000 + i)
    n = 64 + int(rand_u64(k, 0) % 4033)
    u = (rand_u64(k, 1) >> 11) * (1.0 / 9007199254740992.0)
    d = 8.0 + 56.0 * u
    planted = 8 + int(rand_u64(k, 2) % 17)
    p = min(1.0, d / (n - 1))
    return n, p, planted, (seed << 32) + i


def er_batch(count: int, seed: int = 3) -> Batch:
    gs = []
    for i in range(count):
        n, p, k, s = er_batch_params(i, seed)
        gs.append(erdos_renyi(n, p, k, s))
    return Batch(gs, "er-batch count=%d n~U[64,4096] d~U[8,64] planted~U[8,24] seed=%d" % (count, seed))


# ------------------------------------------------- small fixed families ---

def complete(n: int) -> Graph:
    s, d = np.triu_indices(n, 1)
    return from_edges(n, s, d, "K%d" % n)


def empty(n: int) -> Graph:
    return from_edges(n, np.zeros(0, np.int32), np.zeros(0, np.int32), "empty%d" % n)


def cycle(n: int) -> Graph:
    v = np.arange(n)
    return from_edges(n, v, (v + 1) % n, "C%d" % n)


def path(n: int) -> Graph:
    v = np.arange(n - 1)
    return from_edges(n, v, v + 1, "P%d" % n)


def star(n: int) -> Graph:
    v = np.arange(1, n)
    return from_edges(n, np.zeros(n - 1, np.int32), v, "star%d" % n)


def complete_bipartite(a: int, b: int) -> Graph:
    s, d = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return from_edges(a + b, s.ravel(), d.ravel(), "K%d,%d" % (a, b))


def turan(n: int, r: int) -> Graph:
    """Complete r-partite graph with parts as equal as possible (round robin)."""
    part = np.arange(n) % r
    s, d = np.triu_indices(n, 1)
    keep = part[s] != part[d]
    return from_edges(n, s[keep], d[keep], "T(%d,%d)" % (n, r))


def disjoint_cliques(sizes) -> Graph:
    src, dst, off = [], [], 0
    for k in sizes:
        s, d = np.triu_indices(k, 1)
        src.append(s + off)
        dst.append(d + off)
        off += k
    return from_edges(off, np.concatenate(src) if src else [], np.concatenate(dst) if dst else [],
                      "cliques%s" % (tuple(sizes),))


def mycielski(k: int) -> Graph:
    """Mycielski graph M_k: triangle-free with chromatic number k (M_2 = K_2)."""
    edges = [(0, 1)]
    n = 2
    for _ in range(k - 2):
        new = list(edges)
        for (u, v) in edges:
            new.append((u, n + v))
            new.append((v, n + u))
        for i in range(n):
            new.append((n + i, 2 * n))
        edges = new
        n = 2 * n + 1
    e = np.array(edges, np.int32)
    return from_edges(n, e[:, 0], e[:, 1], "mycielski%d" % k)


def petersen() -> Graph:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    e = np.array(outer + spokes + inner, np.int32)
    return from_edges(10, e[:, 0], e[:, 1], "petersen")


def random_small(n: int, p: float, seed: int) -> Graph:
    return erdos_renyi(n, p, 0, seed)


def relabel(g: Graph, seed: int) -> Graph:
    """The same graph under a seeded random vertex permutation."""
    perm = np.empty(g.n, np.int32)
    _L().gg_permutation(g.n, key(seed, 77), _ptr(perm))
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.int32), deg)
    return from_edges(g.n, perm[src], perm[g.col_idx], g.name + "/relabel%d" % seed,
                      np.sort(perm[g.planted]) if g.planted.size else None)
