"""GB300 exact maximum clique (Rossi, Gleich, Gebremedhin, Patwary).

A thin ctypes binding over the C ABI of ``include/mc.h`` (the CUDA library
``_build/libmc.so``).  The functions have the C names and do argument
marshalling only: every step of the method runs in the library's CUDA kernels.
Arrays may be torch tensors (CPU or CUDA) or numpy arrays; CUDA tensors are
passed to the library as device pointers, the rest as host pointers.  There is
no CPU fallback: if the library is missing the import of a function fails
loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

MC_OK = 0
MC_ERR_ARG = -1
MC_ERR_INVALID_GRAPH = -2
MC_ERR_OOM = -3
MC_ERR_BUFFER = -4
MC_ERR_TIMEOUT = -5
MC_ERR_CUDA = -6
MC_ERR_DEVICE_CHECK = -7
MC_ERR_UNSUPPORTED = -8
MC_ERR_TOO_LARGE = -9

MC_VALIDATE = 1
MC_BORROW = 2

_lib = None
_lock = threading.Lock()


class MCError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, strerror(code), code))


class Options(ctypes.Structure):
    _fields_ = [("ordering", ctypes.c_int32), ("no_neigh_cores", ctypes.c_int32),
                ("heuristic", ctypes.c_int32), ("warp_max", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("scores", ctypes.c_void_p),
                ("seeds", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("no_split", ctypes.c_int32), ("split_nodes", ctypes.c_int32),
                ("mlp", ctypes.c_void_p), ("order", ctypes.c_void_p), ("part_rank", ctypes.c_int32),
                ("part_count", ctypes.c_int32), ("layout", ctypes.c_int32), ("no_bitmap", ctypes.c_int32),
                ("repeel", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_cores", ctypes.c_double),
                ("ms_heuristic", ctypes.c_double), ("ms_prune", ctypes.c_double),
                ("ms_search", ctypes.c_double), ("ms_verify", ctypes.c_double),
                ("ms_search_block", ctypes.c_double), ("ms_search_big", ctypes.c_double),
                ("ms_search_warp", ctypes.c_double), ("ms_search_tasks", ctypes.c_double),
                ("n", ctypes.c_int64), ("edges", ctypes.c_int64), ("pruned_n", ctypes.c_int64),
                ("pruned_arcs", ctypes.c_int64), ("roots", ctypes.c_int64),
                ("roots_colored", ctypes.c_int64), ("roots_branched", ctypes.c_int64),
                ("nodes", ctypes.c_int64), ("donations", ctypes.c_int64),
                ("neighbourhood_entries", ctypes.c_int64), ("neighbourhood_entries_block", ctypes.c_int64),
                ("tasks", ctypes.c_int64), ("heuristic_grows", ctypes.c_int64),
                ("heuristic_tests", ctypes.c_int64), ("heuristic_row_entries", ctypes.c_int64),
                ("max_core", ctypes.c_int32), ("heuristic_size", ctypes.c_int32),
                ("omega", ctypes.c_int32), ("verified", ctypes.c_int32),
                ("prune_row_entries", ctypes.c_int64), ("ms_learned", ctypes.c_double),
                ("learned_scored", ctypes.c_int64), ("rebuilds", ctypes.c_int64),
                ("huge_roots", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load ``libmc.so`` (building it with nvcc first if allowed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError("CUDA library %s is missing; run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        i64, i32, u32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p
        L.mc_load_csr.argtypes = [i64, vp, vp, u32, vp, ctypes.POINTER(vp)]
        L.mc_load_batch.argtypes = [i32, vp, vp, vp, u32, vp, ctypes.POINTER(vp)]
        L.mc_free.argtypes = [vp]
        L.mc_free.restype = None
        L.mc_graph_info.argtypes = [vp, vp, vp, vp]
        L.mc_core_numbers.argtypes = [vp, vp, vp]
        L.mc_heuristic_clique.argtypes = [vp, vp, i32, vp, i32, vp]
        L.mc_max_clique.argtypes = [vp, vp, vp, vp, i32, vp]
        L.mc_max_clique_batch.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        L.mc_verify_clique.argtypes = [vp, vp, i32, vp]
        L.mc_peel_order.argtypes = [vp, vp]
        L.mc_peel_order.restype = ctypes.c_int
        L.mc_strerror.argtypes = [ctypes.c_int]
        L.mc_strerror.restype = ctypes.c_char_p
        L.mc_version.restype = ctypes.c_int
        L.mc_launch_count.restype = i64
        for name in ("mc_load_csr", "mc_load_batch", "mc_graph_info", "mc_core_numbers", "mc_heuristic_clique",
                     "mc_max_clique", "mc_max_clique_batch", "mc_verify_clique"):
            getattr(L, name).restype = ctypes.c_int
        _extend(L)
        _lib = L
        return L


def _extend(L):
    """Declare the learned-ordering entry points."""
    vp, i64, i32, f32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_uint64
    L.mc_features.argtypes = [vp, vp]
    L.mc_mlp_create.argtypes = [u64, vp, ctypes.POINTER(vp)]
    L.mc_mlp_free.argtypes = [vp]
    L.mc_mlp_free.restype = None
    L.mc_mlp_num_params.restype = ctypes.c_int
    L.mc_mlp_get_params.argtypes = [vp, vp]
    L.mc_mlp_set_params.argtypes = [vp, vp]
    L.mc_mlp_forward.argtypes = [vp, vp, i64, vp]
    L.mc_mlp_gradient.argtypes = [vp, vp, vp, i64, f32, vp, ctypes.POINTER(f32)]
    L.mc_mlp_train_step.argtypes = [vp, vp, vp, i64, f32, f32, ctypes.POINTER(f32)]
    L.mc_autotune.argtypes = [vp, vp, i32, vp, ctypes.POINTER(ctypes.c_double)]
    L.mc_autotune.restype = ctypes.c_int
    L.mc_clique_order.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(i64), vp]
    L.mc_relabel.argtypes = [vp, vp, vp, vp]
    L.mc_gap_bits.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
    for name in ("mc_clique_order", "mc_relabel", "mc_gap_bits"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("mc_features", "mc_mlp_create", "mc_mlp_get_params", "mc_mlp_set_params", "mc_mlp_forward",
                 "mc_mlp_gradient", "mc_mlp_train_step"):
        getattr(L, name).restype = ctypes.c_int


def strerror(code: int) -> str:
    try:
        return load_library(False).mc_strerror(code).decode()
    except Exception:
        return "error %d" % code


def _check(rc: int, where: str):
    if rc != MC_OK:
        raise MCError(rc, where)


def _ptr(a):
    """(address, keepalive) of a contiguous torch tensor or numpy array."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            a = a.contiguous()
        return a.data_ptr(), a
    a = np.ascontiguousarray(a)
    return a.ctypes.data, a


def _in(a, dtype, what):
    """An input array as a contiguous array of `dtype`, the C type the
    library reads: numpy input (or a sequence) is converted, a torch tensor
    of another dtype is converted on its own device (and kept alive by the
    caller of _ptr).  Integer conversions must keep every value."""
    dtype = np.dtype(dtype)
    if hasattr(a, "data_ptr"):
        import torch
        want = getattr(torch, dtype.name)
        if a.dtype != want:
            if dtype.kind == "i":
                if a.dtype.is_floating_point or a.dtype == torch.bool:
                    raise TypeError("%s must hold integers, got %s" % (what, a.dtype))
                info = np.iinfo(dtype)
                if a.numel() and (int(a.max()) > info.max or int(a.min()) < info.min):
                    raise ValueError("%s has values outside %s" % (what, dtype.name))
            a = a.to(want)
        return a.contiguous()
    arr = np.asarray(a)
    if arr.dtype != dtype:
        if dtype.kind == "i":
            if arr.dtype.kind not in "iu":
                raise TypeError("%s must hold integers, got %s" % (what, arr.dtype))
            info = np.iinfo(dtype)
            if arr.size and (int(arr.max()) > info.max or int(arr.min()) < info.min):
                raise ValueError("%s has values outside %s" % (what, dtype.name))
        arr = arr.astype(dtype)
    return np.ascontiguousarray(arr)


def _out(a, dtype, min_len, what):
    """An output buffer the library writes in place: it must already have
    the C type, be contiguous and writable, and hold at least min_len
    values (the library cannot see its size)."""
    dtype = np.dtype(dtype)
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != getattr(torch, dtype.name):
            raise TypeError("%s must be %s, got %s" % (what, dtype.name, a.dtype))
        if not a.is_contiguous():
            raise ValueError("%s must be contiguous" % what)
        size = a.numel()
    else:
        if not isinstance(a, np.ndarray) or a.dtype != dtype:
            raise TypeError("%s must be a %s array" % (what, dtype.name))
        if not a.flags.c_contiguous or not a.flags.writeable:
            raise ValueError("%s must be contiguous and writable" % what)
        size = a.size
    if size < min_len:
        raise ValueError("%s holds %d values, needs %d" % (what, size, min_len))
    return a


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Graph:
    """Owning handle of a loaded graph (``mc_graph*``)."""

    def __init__(self, handle, n: int, count: int, keep=None):
        self._h = handle
        self.n = n
        self.count = count
        self._keep = keep

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load_library().mc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mc_load_csr(row_ptr, col_idx, flags: int = 0, stream=None) -> Graph:
    L = load_library()
    row_ptr = _in(row_ptr, np.int64, "row_ptr")
    col_idx = _in(col_idx, np.int32, "col_idx")
    rp, krp = _ptr(row_ptr)
    ci, kci = _ptr(col_idx)
    n = int(row_ptr.shape[0]) - 1
    h = ctypes.c_void_p()
    _check(L.mc_load_csr(n, rp, ci, flags, _stream_handle(stream), ctypes.byref(h)), "mc_load_csr")
    return Graph(h, n, 1, (krp, kci) if flags & MC_BORROW else None)


def mc_load_batch(voff, row_ptr, col_idx, flags: int = 0, stream=None) -> Graph:
    L = load_library()
    voff = _in(voff, np.int64, "voff")
    row_ptr = _in(row_ptr, np.int64, "row_ptr")
    col_idx = _in(col_idx, np.int32, "col_idx")
    vo, kvo = _ptr(voff)
    rp, krp = _ptr(row_ptr)
    ci, kci = _ptr(col_idx)
    count = int(voff.shape[0]) - 1
    h = ctypes.c_void_p()
    _check(L.mc_load_batch(count, vo, rp, ci, flags, _stream_handle(stream), ctypes.byref(h)), "mc_load_batch")
    return Graph(h, int(row_ptr.shape[0]) - 1, count, (krp, kci) if flags & MC_BORROW else None)


def mc_free(g: Graph):
    g.close()


def mc_core_numbers(g: Graph, core_out=None):
    """Core numbers into core_out (n int32, host or device) and K(G)."""
    L = load_library()
    if core_out is None:
        core_out = np.zeros(max(g.n, 1), np.int32)
    p, keep = _ptr(_out(core_out, np.int32, g.n, "core_out"))
    mk = ctypes.c_int32(0)
    _check(L.mc_core_numbers(g.handle, p, ctypes.byref(mk)), "mc_core_numbers")
    return core_out[:g.n], mk.value


def mc_heuristic_clique(g: Graph, mode: int = 0, core=None):
    L = load_library()
    cap = g.n + 1
    out = np.zeros(cap, np.int32)
    size = ctypes.c_int32(0)
    cp, kc = _ptr(None if core is None else _in(core, np.int32, "core"))
    _check(L.mc_heuristic_clique(g.handle, cp, mode, out.ctypes.data, cap, ctypes.byref(size)),
           "mc_heuristic_clique")
    return out[:size.value].copy()


def _scores_arg(scores, n):
    """Learned scores as one float32 per vertex: numpy input is converted,
    a torch tensor must already be float32; the length must be n."""
    if scores is None:
        return None
    if hasattr(scores, "data_ptr"):
        if str(scores.dtype) != "torch.float32":
            raise TypeError("scores must be a float32 tensor, got %s" % scores.dtype)
    else:
        scores = np.ascontiguousarray(scores, dtype=np.float32)
    if scores.ndim != 1 or int(scores.shape[0]) != n:
        raise ValueError("scores must hold one value per vertex (%d), got shape %s" % (n, tuple(scores.shape)))
    return scores


def _options(n, ordering=0, no_neigh_cores=False, heuristic=0, warp_max=0, spin_limit=0, scores=None, seeds=0,
             graph=False, no_split=False, split_nodes=0, mlp=None, order=None, part_rank=0, part_count=0, layout=0,
             no_bitmap=False, repeel=0):
    scores = _scores_arg(scores, n)
    o = Options()
    if order is not None:
        order = _in(order, np.int32, "order")
        if order.ndim != 1 or int(order.shape[0]) != n:
            raise ValueError("order must hold one vertex per position (%d), got shape %s" % (n, tuple(order.shape)))
        op, okeep = _ptr(order)
        o.order = op
        o._order_ref = okeep
    o.part_rank = part_rank
    o.part_count = part_count
    o.layout = layout
    o.no_bitmap = 1 if no_bitmap else 0
    o.repeel = repeel
    if mlp is not None:
        if not isinstance(mlp, MLP):
            raise TypeError("mlp must be an MLP handle")
        o.mlp = mlp._h.value
    o.split_nodes = split_nodes
    o.graph = 1 if graph else 0
    o.no_split = 1 if no_split else 0
    o.ordering = ordering
    o.no_neigh_cores = 1 if no_neigh_cores else 0
    o.heuristic = heuristic
    o.warp_max = warp_max
    o.spin_limit = spin_limit
    sp, keep = _ptr(scores)
    o.scores = sp
    o.seeds = seeds
    o._mlp_ref = mlp  # keeps the network alive as long as the options
    return o, keep


def mc_max_clique(g: Graph, witness_out=None, **opts):
    """Returns (omega, witness, stats dict).  witness_out: optional int32
    buffer (host or device) of at least omega entries."""
    L = load_library()
    o, keep = _options(g.n, **opts)
    st = Stats()
    om = ctypes.c_int32(0)
    if witness_out is None:
        witness_out = np.zeros(g.n + 1, np.int32)
    wp, kw = _ptr(_out(witness_out, np.int32, 0, "witness_out"))
    cap = int(witness_out.numel() if hasattr(witness_out, "numel") else witness_out.size)
    _check(L.mc_max_clique(g.handle, ctypes.byref(o), ctypes.byref(om), wp, cap, ctypes.byref(st)), "mc_max_clique")
    return om.value, witness_out[:om.value], st.as_dict()


def mc_max_clique_batch(g: Graph, **opts):
    """Returns (omegas[count], list of witnesses, stats dict)."""
    L = load_library()
    o, keep = _options(g.n, **opts)
    st = Stats()
    om = np.zeros(g.count, np.int32)
    offs = np.zeros(g.count + 1, np.int64)
    wit = np.zeros(g.n + 1, np.int32)
    _check(L.mc_max_clique_batch(g.handle, ctypes.byref(o), om.ctypes.data, wit.ctypes.data, int(wit.shape[0]),
                                 offs.ctypes.data, ctypes.byref(st)), "mc_max_clique_batch")
    wits = [wit[offs[i]:offs[i + 1]].copy() for i in range(g.count)]
    return om, wits, st.as_dict()


def mc_peel_order(g: Graph, out=None):
    """The degeneracy order of the last core-number computation (n int32,
    host or device output)."""
    L = load_library()
    if out is None:
        out = np.zeros(max(g.n, 1), np.int32)
    p, keep = _ptr(_out(out, np.int32, g.n, "out"))
    _check(L.mc_peel_order(g.handle, p), "mc_peel_order")
    return out[:g.n]


class OrderStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("pad_", ctypes.c_int32), ("grows", ctypes.c_int64),
                ("tests", ctypes.c_int64), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


def mc_clique_order(g: Graph, rank=None):
    """Clique-peeling vertex order (Section 6.2, taken in rounds).  Returns
    (order, group_starts, group_round, stats): numpy arrays on the host;
    clique j occupies order[group_starts[j]:group_starts[j+1]]."""
    L = load_library()
    n = g.n
    order = np.zeros(max(n, 1), np.int32)
    starts = np.zeros(n + 1, np.int64)
    rounds = np.zeros(max(n, 1), np.int32)
    rk = _in(rank, np.int32, "rank") if rank is not None else None
    rp, keep = _ptr(rk)
    groups = ctypes.c_int64(0)
    st = OrderStats()
    _check(L.mc_clique_order(g.handle, rp, order.ctypes.data, starts.ctypes.data, rounds.ctypes.data,
                             ctypes.byref(groups), ctypes.byref(st)), "mc_clique_order")
    k = groups.value
    return order[:n], starts[:k + 1], rounds[:k], st.as_dict()


def mc_relabel(g: Graph, order):
    """The CSR relabelled by `order` (new vertex i = order[i]), rows sorted:
    (row_ptr int64, col_idx int32) numpy arrays."""
    L = load_library()
    order = _in(order, np.int32, "order")
    op, keep = _ptr(order)
    n, edges = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(L.mc_graph_info(g.handle, ctypes.byref(n), ctypes.byref(edges), None), "mc_graph_info")
    nnz = 2 * edges.value
    rp = np.zeros(g.n + 1, np.int64)
    ci = np.zeros(max(nnz, 1), np.int32)
    _check(L.mc_relabel(g.handle, op, rp.ctypes.data, ci.ctypes.data), "mc_relabel")
    return rp, ci[:nnz]


def mc_gap_bits(g: Graph, order=None) -> float:
    """Mean log2(1 + gap) per adjacency entry of the graph relabelled by
    `order` (None: as loaded)."""
    L = load_library()
    o = _in(order, np.int32, "order") if order is not None else None
    op, keep = _ptr(o)
    out = ctypes.c_double(0.0)
    _check(L.mc_gap_bits(g.handle, op, ctypes.byref(out)), "mc_gap_bits")
    return out.value


def mc_verify_clique(g: Graph, vertices) -> bool:
    L = load_library()
    vertices = _in(vertices, np.int32, "vertices")
    vp, keep = _ptr(vertices)
    out = ctypes.c_int32(0)
    k = int(vertices.shape[0])
    _check(L.mc_verify_clique(g.handle, vp, k, ctypes.byref(out)), "mc_verify_clique")
    return bool(out.value)


def mc_launch_count() -> int:
    return int(load_library().mc_launch_count())


def mc_version() -> int:
    return int(load_library().mc_version())


# --------------------------------------------------- learned ordering ---

def mc_features(g: Graph, feat_out=None):
    """Per-vertex features (n x 6 float32), host or device output."""
    L = load_library()
    if feat_out is None:
        feat_out = np.zeros((max(g.n, 1), 6), np.float32)
    p, keep = _ptr(_out(feat_out, np.float32, 6 * g.n, "feat_out"))
    _check(L.mc_features(g.handle, p), "mc_features")
    return feat_out[:g.n]


class MLP:
    """Handle of the scoring network (mc_mlp*)."""

    def __init__(self, seed: int = 0, stream=None):
        L = load_library()
        h = ctypes.c_void_p()
        _check(L.mc_mlp_create(seed, _stream_handle(stream), ctypes.byref(h)), "mc_mlp_create")
        self._h = h
        self.nparams = int(L.mc_mlp_num_params())

    def close(self):
        if self._h:
            load_library().mc_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.zeros(self.nparams, np.float32)
        _check(load_library().mc_mlp_get_params(self._h, out.ctypes.data), "mc_mlp_get_params")
        return out

    def set_params(self, p):
        p = _in(p, np.float32, "params")
        if int(p.shape[0]) != self.nparams or p.ndim != 1:
            raise ValueError("params must hold %d values, got shape %s" % (self.nparams, tuple(p.shape)))
        pp, kp = _ptr(p)
        _check(load_library().mc_mlp_set_params(self._h, pp), "mc_mlp_set_params")

    @staticmethod
    def _rows(feat, label=None):
        """Features as float32 (n, 6) rows and labels as float32 n values."""
        feat = _in(feat, np.float32, "feat")
        if feat.ndim != 2 or int(feat.shape[1]) != 6:
            raise ValueError("feat must have shape (n, 6), got %s" % (tuple(feat.shape),))
        n = int(feat.shape[0])
        if label is not None:
            label = _in(label, np.float32, "label")
            if label.ndim != 1 or int(label.shape[0]) != n:
                raise ValueError("label must have shape (%d,), got %s" % (n, tuple(label.shape)))
        return feat, label, n

    def forward(self, feat, out=None):
        feat, _, n = self._rows(feat)
        if out is None:
            out = np.zeros(max(n, 1), np.float32)
        fp, kf = _ptr(feat)
        op, ko = _ptr(_out(out, np.float32, n, "out"))
        _check(load_library().mc_mlp_forward(self._h, fp, n, op), "mc_mlp_forward")
        return out[:n]

    def gradient(self, feat, label, pos_weight=1.0):
        feat, label, n = self._rows(feat, label)
        g = np.zeros(self.nparams, np.float32)
        loss = ctypes.c_float(0)
        fp, kf = _ptr(feat)
        lp, kl = _ptr(label)
        _check(load_library().mc_mlp_gradient(self._h, fp, lp, n, pos_weight, g.ctypes.data, ctypes.byref(loss)),
               "mc_mlp_gradient")
        return g, loss.value

    def train_step(self, feat, label, pos_weight=1.0, lr=1e-3):
        feat, label, n = self._rows(feat, label)
        loss = ctypes.c_float(0)
        fp, kf = _ptr(feat)
        lp, kl = _ptr(label)
        _check(load_library().mc_mlp_train_step(self._h, fp, lp, n, pos_weight, lr, ctypes.byref(loss)),
               "mc_mlp_train_step")
        return loss.value


def mc_autotune(g: Graph, repeats: int = 2, **opts):
    """Fastest (warp_max, no_split, split_nodes, heuristic, graph) setting
    for this graph; returns (options dict, ms)."""
    L = load_library()
    base, keep = _options(g.n, **opts)
    best = Options()
    ms = ctypes.c_double(0)
    _check(L.mc_autotune(g.handle, ctypes.byref(base), repeats, ctypes.byref(best), ctypes.byref(ms)), "mc_autotune")
    return {"warp_max": best.warp_max, "no_split": bool(best.no_split), "split_nodes": best.split_nodes,
            "layout": best.layout, "no_bitmap": bool(best.no_bitmap), "heuristic": best.heuristic,
            "graph": bool(best.graph)}, ms.value
