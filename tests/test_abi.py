"""CPU checks of the C-ABI boundary: the library builds, loads and exports
every entry point that include/fsa.h declares (no compute call needs a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fsa_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2405_14492_gb300 import build as B
    return B.build()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for want in ("fsa_build", "fsa_loglik_grad", "fsa_predict", "fsa_free", "fsa_get_csr", "fsa_matvec"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in sorted(_declared_symbols()) if not hasattr(lib, s)]
    assert not missing, f"not exported: {missing}"


def test_checked_build_compiles_and_exports_every_declared_symbol():
    """The checked variant (-DFSA_CHECKED: device index checks that report
    FSA_ERR_BOUNDS instead of a memory fault) builds from the same sources
    into its own library, with the same boundary, and names the new status."""
    from paper_2405_14492_gb300 import build as B
    path = B.build(checked=True)
    assert os.path.basename(path) == "libfsa_checked.so"
    lib = ctypes.CDLL(path)
    missing = [s for s in sorted(_declared_symbols()) if not hasattr(lib, s)]
    assert not missing, f"not exported: {missing}"
    lib.fsa_status_string.restype = ctypes.c_char_p
    assert lib.fsa_status_string(10) == b"FSA_ERR_BOUNDS"


def test_host_only_entry_points(libpath):
    from paper_2405_14492_gb300 import _native as N
    o = N.default_opts()
    assert o.num_probes == 50 and abs(o.cg_tol - 1e-3) < 1e-15 and o.want_grad == 1
    assert N.lib().fsa_status_string(3) == b"FSA_ERR_NOT_PD"
    b64 = N.lib().fsa_footprint_bytes(10 ** 6, 1000, 2 * 10 ** 7, 64, 0)
    b16 = N.lib().fsa_footprint_bytes(10 ** 6, 1000, 2 * 10 ** 7, 64, 1)
    assert b64 > b16 > 10 ** 9


def test_argument_errors_need_no_gpu(libpath):
    """Invalid arguments are rejected on the host before any device call."""
    import numpy as np
    from paper_2405_14492_gb300 import _native as N
    h = ctypes.c_void_p()
    locs = np.zeros((1, 2))
    st = N.lib().fsa_build(N.ptr(locs), 1, N.ptr(locs), 1, 0.1, 0, None, ctypes.byref(h))
    assert st == 1 and h.value is None
    locs = np.random.default_rng(0).random((10, 2))
    st = N.lib().fsa_build(N.ptr(locs), 10, N.ptr(locs), 11, 0.1, 0, None, ctypes.byref(h))
    assert st == 1
    st = N.lib().fsa_build(N.ptr(locs), 10, N.ptr(locs), 3, -1.0, 0, None, ctypes.byref(h))
    assert st == 1
    bad = locs.copy()
    bad[0, 0] = np.nan
    st = N.lib().fsa_build(N.ptr(locs), 10, N.ptr(bad), 3, 0.1, 0, None, ctypes.byref(h))
    assert st == 5
    assert b"inducing" in N.lib().fsa_last_error()
    out = np.zeros(11, dtype=np.int64)
    assert N.lib().fsa_kmeanspp(N.ptr(locs), 10, 11, 1, N.ptr(out), None) == 1   # m > n
    assert N.lib().fsa_kmeanspp(N.ptr(locs), 10, 0, 1, N.ptr(out), None) == 1    # m < 1
    assert b"kmeanspp" in N.lib().fsa_last_error()


def test_struct_layouts_match_the_header(tmp_path, libpath):
    """The ctypes mirrors of the ABI structs have the C sizes and offsets
    (a C program built from include/fsa.h prints them)."""
    import shutil
    import subprocess
    from paper_2405_14492_gb300 import _native as N
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fsa_theta": N.FsaTheta, "fsa_opts": N.FsaOpts, "fsa_info": N.FsaInfo,
               "fsa_server_cfg": N.FsaServerCfg, "fsa_request": N.FsaRequest, "fsa_result": N.FsaResult,
               "fsa_server_stats": N.FsaServerStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fsa.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        py = structs[cname]
        got = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert got == int(val), (cname, field, got, val)


def test_serving_without_a_gpu_fails_cleanly(libpath):
    """Server creation reports a CUDA error status (no crash) where no GPU is present."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2405_14492_gb300 import _native as N
    s = ctypes.c_void_p()
    cfg = N.FsaServerCfg()
    N.lib().fsa_default_server_cfg(ctypes.byref(cfg))
    assert cfg.max_slots == 4 and cfg.hbm_budget_bytes == 0
    cfg.max_slots = 0
    assert N.lib().fsa_server_create(ctypes.byref(cfg), ctypes.byref(s)) == 1
    cfg.max_slots = 2
    assert N.lib().fsa_server_create(ctypes.byref(cfg), ctypes.byref(s)) == 8
    assert s.value is None
