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
