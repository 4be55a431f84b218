"""CPU oracle for exact maximum clique -- TEST INFRASTRUCTURE ONLY.

Python access to ``oracle.c`` (plain C written from the paper's definitions
and algorithms; single-threaded except for ``max_clique_threads``).  Only ``tests/``, the smoke check and the
benchmark's CPU-baseline leg may import this package; the CUDA library never
does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c")]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``_build/liboracle.so``."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    srcs = list(_SRCS)
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread"] + srcs
                   + ["-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Stats(ctypes.Structure):
    _fields_ = [("pruned_n", ctypes.c_int64), ("initial_branch", ctypes.c_int64),
                ("full_branch", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("heuristic", ctypes.c_int32), ("max_core", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def configure(lib):
    """Declare the C signatures on a loaded oracle library (also used by the
    tests that load a copy of the oracle with a planted mistake)."""
    i64, i32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    lib.orc_core_numbers.argtypes = [i64, vp, vp, vp, vp]
    lib.orc_core_numbers.restype = ctypes.c_int
    lib.orc_greedy_colors.argtypes = [i64, vp, vp, vp, vp]
    lib.orc_greedy_colors.restype = i32
    lib.orc_heuristic_clique.argtypes = [i64, vp, vp, vp, ctypes.c_int, vp, i32, vp]
    lib.orc_heuristic_clique.restype = ctypes.c_int
    lib.orc_max_clique.argtypes = [i64, vp, vp, vp, vp, i32, vp]
    lib.orc_max_clique.restype = ctypes.c_int
    lib.orc_is_clique.argtypes = [i64, vp, vp, vp, i32]
    lib.orc_is_clique.restype = ctypes.c_int
    lib.orc_max_clique_threads.argtypes = [i64, vp, vp, i32, vp, vp, i32, vp]
    lib.orc_max_clique_threads.restype = ctypes.c_int
    lib.orc_max_clique_part.argtypes = [i64, vp, vp, vp, i32, i32, i32, vp, vp, i32, vp]
    lib.orc_max_clique_part.restype = ctypes.c_int
    return lib


def _L():
    global _lib
    with _lock:
        if _lib is None:
            _lib = configure(ctypes.CDLL(build()))
    return _lib


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, np.int32)
    return rp, ci, int(rp.shape[0] - 1)


def core_numbers(g, with_order: bool = False):
    """K(v) for every vertex (Batagelj-Zaversnik)."""
    rp, ci, n = _csr(g)
    core = np.zeros(max(n, 1), np.int32)
    order = np.zeros(max(n, 1), np.int32)
    rc = _L().orc_core_numbers(n, rp.ctypes.data, ci.ctypes.data, core.ctypes.data, order.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle core numbers failed: %d" % rc)
    return (core[:n], order[:n]) if with_order else core[:n]


def greedy_colors(g, order) -> int:
    """Number of colours of the greedy colouring in the given order."""
    rp, ci, n = _csr(g)
    order = np.ascontiguousarray(order, dtype=np.int32)
    return int(_L().orc_greedy_colors(n, rp.ctypes.data, ci.ctypes.data, order.ctypes.data, None))


def heuristic_clique(g, core=None, mode: int = 0):
    """Algorithm 1.  mode 0 as printed; mode 1 the deterministic
    all-start-vertices form.  Returns the clique (sorted)."""
    rp, ci, n = _csr(g)
    if core is None:
        core = core_numbers(g)
    core = np.ascontiguousarray(core, dtype=np.int32)
    if core.size == 0:
        core = np.zeros(1, np.int32)
    cap = int(core.max()) + 2 if n else 1
    H = np.zeros(cap, np.int32)
    size = ctypes.c_int32(0)
    rc = _L().orc_heuristic_clique(n, rp.ctypes.data, ci.ctypes.data, core.ctypes.data, mode,
                                   H.ctypes.data, cap, ctypes.addressof(size))
    if rc != 0:
        raise RuntimeError("oracle heuristic failed: %d" % rc)
    return H[:size.value].copy()


def max_clique(g):
    """Algorithm 2.  Returns (omega, witness sorted ascending, stats dict)."""
    rp, ci, n = _csr(g)
    cap = n + 1
    W = np.zeros(max(cap, 1), np.int32)
    om = ctypes.c_int32(0)
    st = Stats()
    rc = _L().orc_max_clique(n, rp.ctypes.data, ci.ctypes.data, ctypes.addressof(om), W.ctypes.data, cap,
                             ctypes.addressof(st))
    if rc != 0:
        raise RuntimeError("oracle max clique failed: %d" % rc)
    return om.value, W[:om.value].copy(), st.as_dict()


def max_clique_threads(g, threads: int):
    """The exact search by `threads` workers sharing the incumbent (Section
    4.5), roots in a static degeneracy order.  omega is the same as
    max_clique's; the witness may be another maximum clique.  Returns
    (omega, witness sorted ascending, stats dict)."""
    rp, ci, n = _csr(g)
    cap = n + 1
    W = np.zeros(max(cap, 1), np.int32)
    om = ctypes.c_int32(0)
    st = Stats()
    rc = _L().orc_max_clique_threads(n, rp.ctypes.data, ci.ctypes.data, int(threads), ctypes.addressof(om),
                                     W.ctypes.data, cap, ctypes.addressof(st))
    if rc != 0:
        raise RuntimeError("oracle threaded max clique failed: %d" % rc)
    return om.value, W[:om.value].copy(), st.as_dict()


def max_clique_part(g, part_rank: int, part_count: int, order=None, threads: int = 1):
    """The threaded search restricted to the roots at positions part_rank,
    part_rank + part_count, ... of `order` (a degeneracy order; None = the
    oracle's own).  Returns (the largest clique size this part found, its
    witness, stats); the maximum over the parts is omega."""
    rp, ci, n = _csr(g)
    cap = n + 1
    W = np.zeros(max(cap, 1), np.int32)
    om = ctypes.c_int32(0)
    st = Stats()
    op = None
    if order is not None:
        order = np.ascontiguousarray(order, dtype=np.int32)
        op = order.ctypes.data
    rc = _L().orc_max_clique_part(n, rp.ctypes.data, ci.ctypes.data, op, int(part_rank), int(part_count),
                                  int(threads), ctypes.addressof(om), W.ctypes.data, cap, ctypes.addressof(st))
    if rc != 0:
        raise RuntimeError("oracle partitioned max clique failed: %d" % rc)
    return om.value, W[:om.value].copy(), st.as_dict()


def is_clique(g, vs) -> bool:
    rp, ci, n = _csr(g)
    vs = np.ascontiguousarray(vs, dtype=np.int32)
    if vs.size == 0:
        return True
    return bool(_L().orc_is_clique(n, rp.ctypes.data, ci.ctypes.data, vs.ctypes.data, int(vs.size)))
