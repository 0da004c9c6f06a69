"""fsa_csr_noalloc: the allocation-free entry point, for callers that cannot
allocate device memory (their device memory belongs to their own pool or
capped allocator, or they run where cudaMalloc must not be called).

The test allocates the input and output buffers itself (the entry point
does not) and checks, on two calls in a row with different inputs, that the
pattern equals the one of the existing fsa_build + fsa_get_csr path, bit for
bit (it is integer index work).  This file is collected last so that a run
that stops at the first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

import fsa_inputs as fi

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2405_14492_gb300 import _native as N
    lib = N.lib()
    f = lib.fsa_csr_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    return lib, N


def _noalloc_csr(locs, gamma):
    import torch
    lib, N = _lib()
    n = locs.shape[0]
    d_locs = torch.tensor(locs, dtype=torch.float64, device="cuda")
    d_rowptr = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    nnz = ctypes.c_int64(-1)
    # size query (no column buffer), then the real call
    st = lib.fsa_csr_noalloc(d_locs.data_ptr(), n, gamma, d_rowptr.data_ptr(), None, 0, ctypes.byref(nnz), None)
    assert st == 0, lib.fsa_last_error()
    rowptr_query = d_rowptr.cpu().numpy().copy()   # the size query writes every row pointer
    d_col = torch.full((max(nnz.value, 1),), -7, dtype=torch.int32, device="cuda")
    st = lib.fsa_csr_noalloc(d_locs.data_ptr(), n, gamma, d_rowptr.data_ptr(), d_col.data_ptr(), nnz.value,
                             ctypes.byref(nnz), None)
    assert st == 0, lib.fsa_last_error()
    torch.cuda.synchronize()
    rowptr = d_rowptr.cpu().numpy()
    assert np.array_equal(rowptr_query, rowptr)
    return rowptr, d_col[:nnz.value].cpu().numpy()


def _existing_csr(locs, gamma):
    import paper_2405_14492_gb300 as F
    with F.FSAHandle(locs, locs[:1], gamma) as h:
        return h.csr()


def test_noalloc_csr_matches_existing_entry_point_twice():
    cases = [(fi.uniform_locations(20011, 31), 0.012),     # several thousand cells, ragged size
             (fi.uniform_locations(5003, 32) * 0.3, 0.02)]  # second call: other size, grid and extent
    for locs, gamma in cases:
        rp, col = _noalloc_csr(locs, gamma)
        rp0, col0 = _existing_csr(locs, gamma)
        assert np.array_equal(rp, rp0)
        assert np.array_equal(col, col0)


def test_noalloc_rejects_too_large_and_small_capacity():
    import torch
    lib, N = _lib()
    n = 65537
    d_locs = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    d_rowptr = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    nnz = ctypes.c_int64(0)
    st = lib.fsa_csr_noalloc(d_locs.data_ptr(), n, 0.1, d_rowptr.data_ptr(), None, 0, ctypes.byref(nnz), None)
    assert st == 1   # FSA_ERR_ARG: beyond the fixed scratch size
    assert b"65536" in lib.fsa_last_error()
    locs = fi.uniform_locations(1000, 33)
    d_locs = torch.tensor(locs, dtype=torch.float64, device="cuda")
    d_rowptr = torch.zeros(1001, dtype=torch.int64, device="cuda")
    d_col = torch.zeros(10, dtype=torch.int32, device="cuda")
    st = lib.fsa_csr_noalloc(d_locs.data_ptr(), 1000, 0.05, d_rowptr.data_ptr(), d_col.data_ptr(), 10,
                             ctypes.byref(nnz), None)
    assert st == 1 and nnz.value > 10


def test_noalloc_long_rows_stay_bounded():
    """A taper range wider than the points' extent puts every point in one
    cell and every row at n neighbours; rows and cells are heap-sorted, so
    the call ends quickly and gives the dense pattern."""
    locs = fi.uniform_locations(3001, 34) * 0.01
    rp, col = _noalloc_csr(locs, 0.5)
    n = locs.shape[0]
    assert np.array_equal(rp, np.arange(n + 1, dtype=np.int64) * n)
    assert np.array_equal(col, np.tile(np.arange(n, dtype=np.int32), n))
