"""The C-ABI library builds, loads without a GPU and exports every symbol include/hyb.h declares."""
import ctypes
import os
import re

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "hyb.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_api():
    names = declared_symbols()
    for n in ["hyb_setup", "hyb_assemble_reduced", "hyb_solve_reduced", "hyb_recover",
              "staticcond_assemble", "staticcond_recover", "hyb_destroy", "hyb_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_08914_gb300 import hyb
    lib = ctypes.CDLL(hyb.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    # host-only calls that need no GPU
    lib.hyb_status_string.restype = ctypes.c_char_p
    assert lib.hyb_status_string(-4) == b"HYB_ERR_NOT_SPD"
    assert lib.hyb_status_string(0) == b"HYB_OK"
    lib.hyb_destroy(None)


def test_binding_refuses_cpu_tensors():
    import pytest
    import torch
    from paper_1801_08914_gb300 import hyb
    with pytest.raises(TypeError):
        hyb._ptr(torch.zeros(3, dtype=torch.float64), "x")


def test_noalloc_binding_checks_sizes_before_the_call():
    """The allocation-free solve trusts the sizes it gets; the binding refuses inconsistent
    ones before any pointer reaches the library (checked here on host tensors: the size
    checks come first, the device check after them)."""
    import pytest
    import torch
    from paper_1801_08914_gb300 import hyb
    f64, i64, i32 = torch.float64, torch.int64, torch.int32
    n = 4
    rp = torch.arange(n + 1, dtype=i64)
    col = torch.arange(n, dtype=i32)
    val = torch.ones(n, dtype=f64)
    b = torch.ones(n, dtype=f64)
    with pytest.raises(ValueError, match="x has"):
        hyb.hyb_pcg_solve_noalloc(rp, col, val, b, torch.zeros(n - 1, dtype=f64), 1, 1e-12, 10)
    with pytest.raises(ValueError, match="row_ptr has"):
        hyb.hyb_pcg_solve_noalloc(rp[:-1], col, val, b, torch.zeros(n, dtype=f64), 1, 1e-12, 10)
    with pytest.raises(ValueError, match="differ in length"):
        hyb.hyb_pcg_solve_noalloc(rp, col[:-1], val, b, torch.zeros(n, dtype=f64), 1, 1e-12, 10)
    bad = rp.clone()
    bad[n] = n + 1
    with pytest.raises(ValueError, match="exceeds"):
        hyb.hyb_pcg_solve_noalloc(bad, col, val, b, torch.zeros(n, dtype=f64), 1, 1e-12, 10)
    with pytest.raises(TypeError):                       # consistent sizes, but host memory
        hyb.hyb_pcg_solve_noalloc(rp, col, val, b, torch.zeros(n, dtype=f64), 1, 1e-12, 10)
