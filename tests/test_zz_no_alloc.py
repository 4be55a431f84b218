"""mc_core_numbers_noalloc: core numbers for callers that cannot allocate
device memory (allocator hooks, hosts that own the whole device budget).  It
must give exactly the oracle's core numbers (Batagelj-Zaversnik), and what
mc_core_numbers gives, call after call, although every call reuses the same
fixed device array; and it must refuse inputs it cannot hold or whose row
offsets and column entries are out of bounds before its peel runs.  This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_1302_6256_gb300 as mc
    L = mc.load_library()
    L.mc_core_numbers_noalloc.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]
    L.mc_core_numbers_noalloc.restype = ctypes.c_int
    return mc, L


def library_cores(mc, g):
    h = mc.mc_load_csr(g.row_ptr, g.col_idx, 0)
    core, kmax = mc.mc_core_numbers(h)
    h.close()
    return np.array(core), kmax


@pytest.mark.parametrize("g", [gg.rmat(14, 16, planted=20, seed=5),
                               gg.chung_lu(20000, 2.5, 8.0, 1000.0, planted=15, seed=1),
                               gg.erdos_renyi(700, 0.2, planted=12, seed=8)], ids=lambda g: g.name)
def test_noalloc_matches_oracle_and_mc_core_numbers_twice(lib, g):
    mc, L = lib
    ref = oracle.core_numbers(g)
    kref = int(ref.max())
    lib_core, lib_k = library_cores(mc, g)
    assert np.array_equal(lib_core, ref) and lib_k == kref
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(2):  # the second call sees the first call's leftovers
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        mk = ctypes.c_int32(-1)
        rc = L.mc_core_numbers_noalloc(g.n, rp.data_ptr(), ci.data_ptr(), out.data_ptr(), ctypes.byref(mk),
                                       stream.cuda_stream)
        assert rc == 0, mc.strerror(rc)
        assert np.array_equal(out.cpu().numpy(), ref)
        assert mk.value == kref


def test_noalloc_rejects_inputs_beyond_its_scratch(lib):
    mc, L = lib
    g = gg.path(4)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    mk = ctypes.c_int32(0)
    rc = L.mc_core_numbers_noalloc((1 << 20) + 1, rp.data_ptr(), ci.data_ptr(), out.data_ptr(), ctypes.byref(mk),
                                   None)
    assert rc == mc.MC_ERR_TOO_LARGE


def _call(L, n, rp, ci, out):
    mk = ctypes.c_int32(0)
    return L.mc_core_numbers_noalloc(n, rp.data_ptr(), ci.data_ptr(), out.data_ptr(), ctypes.byref(mk), None)


def test_noalloc_rejects_more_entries_than_its_scratch(lib):
    """row_ptr[n] = 2^26 + 1 entries: refused after reading that one value,
    before any kernel runs (nothing reads col_idx)."""
    mc, L = lib
    rp = torch.tensor([0, (1 << 26) + 1], dtype=torch.int64, device="cuda")
    ci = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _call(L, 1, rp, ci, out) == mc.MC_ERR_TOO_LARGE


def test_noalloc_rejects_out_of_bounds_offsets_and_columns(lib):
    """The bounds pass reads only row_ptr[0..n] and col_idx[0..row_ptr[n])
    and refuses a column entry outside [0, n), a decreasing row_ptr and a
    row_ptr[0] other than 0 before the peel runs; a valid call still works
    afterwards."""
    mc, L = lib
    g = gg.path(4)  # row_ptr [0, 1, 3, 5, 6], col_idx [1, 0, 2, 1, 3, 2]
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    rp = torch.from_numpy(g.row_ptr).cuda()
    for bad_ci in ([1, 0, 2, 1, 4, 2], [1, 0, 2, -1, 3, 2]):
        ci = torch.tensor(bad_ci, dtype=torch.int32, device="cuda")
        assert _call(L, 4, rp, ci, out) == mc.MC_ERR_INVALID_GRAPH
    ci = torch.from_numpy(g.col_idx).cuda()
    for bad_rp in ([0, 3, 1, 5, 6], [1, 1, 3, 5, 6]):
        assert _call(L, 4, torch.tensor(bad_rp, dtype=torch.int64, device="cuda"), ci, out) == \
            mc.MC_ERR_INVALID_GRAPH
    assert _call(L, 4, rp, ci, out) == 0
    assert out.cpu().numpy().tolist() == oracle.core_numbers(g).tolist()
