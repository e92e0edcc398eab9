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


def test_context_bindings_check_sizes_before_the_call():
    """Every binding that hands the library device buffers checks their lengths against the
    mesh (hyb_setup) or the context's sizes first: a short buffer would be read or written
    past its end. Checked on host tensors with a stand-in context (the size checks raise
    before any pointer or handle reaches the library)."""
    import pytest
    import torch
    from paper_1801_08914_gb300 import hyb
    f64 = torch.float64

    class Sized:
        handle = 1                                       # never reaches the library here

        def sizes(self):
            return dict(n_elem=8, n_loc=6, n_lambda=12, nnz=0)

    ctx = Sized()
    lam, u, load = torch.zeros(12, dtype=f64), torch.zeros(8, 6, dtype=f64), torch.zeros(48, dtype=f64)
    short_lam, short_u = torch.zeros(11, dtype=f64), torch.zeros(47, dtype=f64)
    with pytest.raises(ValueError, match="vertices has"):
        hyb.hyb_setup(torch.zeros(3 * 27 - 3, dtype=f64), 2, 2, 2, 0, torch.ones(8, dtype=f64),
                      torch.ones(8, dtype=f64))
    with pytest.raises(ValueError, match="beta has"):
        hyb.hyb_setup(torch.zeros(3 * 27, dtype=f64), 2, 2, 2, 0, torch.ones(8, dtype=f64),
                      torch.ones(7, dtype=f64))
    with pytest.raises(TypeError):                       # nx = 0: no size check, the library decides
        hyb.hyb_setup(torch.zeros(3 * 27, dtype=f64), 0, 2, 2, 0, torch.ones(8, dtype=f64),
                      torch.ones(8, dtype=f64))
    calls = [
        lambda: hyb.hyb_assemble_reduced(ctx, short_u),
        lambda: hyb.hyb_assemble_reduced(ctx, load, short_u),
        lambda: hyb.staticcond_assemble(ctx, short_u),
        lambda: hyb.hyb_solve_reduced(ctx, 1e-12, 10, short_lam),
        lambda: hyb.hyb_recover(ctx, short_lam, u),
        lambda: hyb.hyb_recover(ctx, lam, short_u),
        lambda: hyb.staticcond_recover(ctx, short_lam, u),
        lambda: hyb.hyb_refine(ctx, 1, 1e-6, 10, lam, short_u),
        lambda: hyb.hyb_amg_apply(ctx, lam, short_lam),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="entries, expected"):
            call()
    with pytest.raises(TypeError):                       # right sizes, host memory
        hyb.hyb_recover(ctx, lam, u)
