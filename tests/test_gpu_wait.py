"""Failure detection without a GPU fault: a device wait that nothing completes
runs out after its bounded number of polls, reports FSA_ERR_TIMEOUT through the
error word, and leaves the context usable."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_bounded_device_wait_times_out_and_context_stays_usable():
    from paper_2405_14492_gb300 import _native as N
    f = N.lib().fsa_selftest_wait_timeout
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    fin, usable = ctypes.c_int(0), ctypes.c_int(0)
    st = f(2000, ctypes.byref(fin), ctypes.byref(usable))
    assert st == 6, N.lib().fsa_last_error()      # FSA_ERR_TIMEOUT
    assert fin.value == 1 and usable.value == 1
    # and again: nothing was left behind by the first run
    st = f(100, ctypes.byref(fin), ctypes.byref(usable))
    assert st == 6 and fin.value == 1 and usable.value == 1
