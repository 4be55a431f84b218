"""The C ABI library builds for sm_103a, loads, and exports every function
that include/mc.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mc_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_method_calls():
    names = declared_functions()
    for want in ("mc_load_csr", "mc_core_numbers", "mc_heuristic_clique", "mc_max_clique", "mc_free",
                 "mc_strerror", "mc_max_clique_batch", "mc_load_batch"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1302_6256_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version_without_gpu():
    import paper_1302_6256_gb300 as mc
    L = mc.load_library()
    assert L.mc_strerror(mc.MC_ERR_BUFFER).decode() == "output buffer too small"
    assert L.mc_version() >= 100


def test_no_cpu_fallback_in_product_package():
    """The package never imports the oracle or the generators."""
    pkg = os.path.join(ROOT, "paper_1302_6256_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "orc_" not in src, f


def test_options_marshal_learned_scores():
    """Learned scores reach the library as one float32 per vertex: numpy
    input of another dtype is converted, a wrong length is refused before
    any call (the C side cannot see the array's length)."""
    import numpy as np
    import paper_1302_6256_gb300 as mc
    o, keep = mc._options(4, ordering=1, scores=np.arange(4, dtype=np.float64), seeds=2, graph=True)
    assert keep.dtype == np.float32 and o.scores == keep.ctypes.data
    assert o.ordering == 1 and o.seeds == 2 and o.graph == 1
    f32 = np.zeros(4, np.float32)
    o, keep = mc._options(4, ordering=1, scores=f32)
    assert o.scores == f32.ctypes.data  # no copy: graph replay sees later writes
    with pytest.raises(ValueError):
        mc._options(5, ordering=1, scores=f32)
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        mc._options(4, ordering=1, scores=torch.zeros(4, dtype=torch.float64))
    o, keep = mc._options(4, ordering=1, scores=torch.zeros(4, dtype=torch.float32))
    assert o.scores == keep.data_ptr()


def test_binding_converts_inputs_and_checks_outputs():
    """Inputs reach the library in its C types (converted when they are not,
    refused when a value would not survive the conversion); output buffers,
    which the library writes in place without knowing their size, must have
    the right type, layout and size already."""
    import numpy as np
    import paper_1302_6256_gb300 as mc
    rp = mc._in(np.array([0, 1, 2], np.int32), np.int64, "row_ptr")
    assert rp.dtype == np.int64 and rp.tolist() == [0, 1, 2]
    ci = mc._in([1, 0], np.int32, "col_idx")
    assert ci.dtype == np.int32 and ci.flags.c_contiguous
    assert mc._in(np.arange(10, dtype=np.int32)[::2], np.int32, "x").flags.c_contiguous
    with pytest.raises(ValueError):
        mc._in(np.array([2 ** 31], np.int64), np.int32, "col_idx")
    with pytest.raises(TypeError):
        mc._in(np.array([0.5]), np.int32, "col_idx")
    assert mc._in(np.zeros(3), np.float32, "feat").dtype == np.float32
    core = np.zeros(4, np.int32)
    assert mc._out(core, np.int32, 4, "core_out") is core
    with pytest.raises(ValueError):
        mc._out(core, np.int32, 5, "core_out")
    with pytest.raises(TypeError):
        mc._out(np.zeros(4, np.int64), np.int32, 4, "core_out")
    with pytest.raises(ValueError):
        mc._out(np.zeros(8, np.int32)[::2], np.int32, 4, "core_out")
    feat, label, n = mc.MLP._rows(np.zeros((5, 6)), [0, 1, 0, 0, 1])
    assert n == 5 and feat.dtype == np.float32 and label.dtype == np.float32
    with pytest.raises(ValueError):
        mc.MLP._rows(np.zeros((5, 4)))
    with pytest.raises(ValueError):
        mc.MLP._rows(np.zeros((5, 6)), np.zeros(4))
    torch = pytest.importorskip("torch")
    t = mc._in(torch.tensor([0, 3], dtype=torch.int32), np.int64, "row_ptr")
    assert t.dtype == torch.int64 and t.tolist() == [0, 3]
    with pytest.raises(TypeError):
        mc._out(torch.zeros(4, dtype=torch.int64), np.int32, 4, "witness_out")
    with pytest.raises(ValueError):
        mc._in(torch.tensor([-1], dtype=torch.int64) * 2 ** 40, np.int32, "col_idx")


def test_argument_errors_before_any_cuda_call():
    """The C entry points refuse bad arguments with MC_ERR_ARG (or, for the
    fixed-scratch core numbers, MC_ERR_TOO_LARGE) before they touch the GPU,
    so these calls run on a machine without one."""
    import paper_1302_6256_gb300 as mc
    L = mc.load_library()
    vp = ctypes.c_void_p
    h = vp()
    assert L.mc_load_csr(-1, None, None, 0, None, ctypes.byref(h)) == mc.MC_ERR_ARG
    assert L.mc_load_csr(3 * 10 ** 9, None, None, 0, None, ctypes.byref(h)) == mc.MC_ERR_ARG
    assert L.mc_load_csr(0, None, None, 0, None, None) == mc.MC_ERR_ARG
    assert L.mc_load_csr(5, None, None, 0, None, ctypes.byref(h)) == mc.MC_ERR_ARG  # rows missing
    assert L.mc_load_batch(0, None, None, None, 0, None, ctypes.byref(h)) == mc.MC_ERR_ARG
    om = ctypes.c_int32(7)
    assert L.mc_max_clique(None, None, ctypes.byref(om), None, 0, None) == mc.MC_ERR_ARG
    assert L.mc_max_clique_batch(None, None, None, None, 0, None, None) == mc.MC_ERR_ARG
    assert L.mc_core_numbers(None, None, None) == mc.MC_ERR_ARG
    size = ctypes.c_int32(0)
    assert L.mc_heuristic_clique(None, None, 0, None, 0, ctypes.byref(size)) == mc.MC_ERR_ARG
    assert L.mc_graph_info(None, None, None, None) == mc.MC_ERR_ARG
    ok = ctypes.c_int32(0)
    assert L.mc_verify_clique(None, None, 0, ctypes.byref(ok)) == mc.MC_ERR_ARG
    assert L.mc_mlp_create(1, None, None) == mc.MC_ERR_ARG
    L.mc_free(None)
    L.mc_mlp_free(None)
    L.mc_core_numbers_noalloc.argtypes = [ctypes.c_int64, vp, vp, vp, ctypes.POINTER(ctypes.c_int32), vp]
    L.mc_core_numbers_noalloc.restype = ctypes.c_int
    assert L.mc_core_numbers_noalloc(-1, None, None, None, None, None) == mc.MC_ERR_ARG
    dummy = ctypes.c_int64(0)
    p = ctypes.addressof(dummy)
    assert L.mc_core_numbers_noalloc((1 << 20) + 1, p, p, p, None, None) == mc.MC_ERR_TOO_LARGE
    assert L.mc_strerror(mc.MC_ERR_UNSUPPORTED).decode().startswith("a batch graph with core number above 4096")
    # the clique-peeling order, relabelling and gap cost refuse a null handle
    groups = ctypes.c_int64(5)
    assert L.mc_clique_order(None, None, None, None, None, ctypes.byref(groups), None) == mc.MC_ERR_ARG
    assert L.mc_relabel(None, None, None, None) == mc.MC_ERR_ARG
    bits = ctypes.c_double(1.0)
    assert L.mc_gap_bits(None, None, ctypes.byref(bits)) == mc.MC_ERR_ARG
