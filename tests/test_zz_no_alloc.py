"""The allocation-free PCG entry point (hyb_pcg_solve_noalloc) against hyb_solve_reduced.

Callers that cannot allocate device memory (all of it reserved by another allocator, or
unable to afford a call that blocks the device) solve through this entry point, whose
scratch is a fixed device array inside the library. It is checked through the C ABI on
two calls in a row (the array keeps the previous call's contents) against the solution of
the context's own solver, within the 1e-12 relative tolerance of the parity tests, and the
device's free memory is checked to stay put across the calls after the first. This
file is collected last so that a stop-at-first-failure run has already run the rest.
"""
import numpy as np
import pytest

from gpu_helpers import dev, rel
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["rt0_manufactured", "rt1_contrast"])
def test_noalloc_pcg_matches_context_solver(case):
    import torch
    from paper_1801_08914_gb300 import hyb
    if case == "rt0_manufactured":
        p = inputs.make_config("1j")
    else:
        p = inputs.random_problem(6, 1, 0.2, 77, 1e-2, 1e4, name="noalloc")
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta))
    hyb.hyb_assemble_reduced(ctx, dev(p.load), None if p.ess is None else dev(p.ess))
    red = hyb.hyb_export_reduced(ctx)
    n = red["rhs"].numel()
    ref = torch.zeros(n, dtype=torch.float64, device="cuda")
    it_ref, rr_ref, _ = hyb.hyb_solve_reduced(ctx, 1e-12, 10000, ref)
    nfn = (p.order + 1) ** 2
    # every output buffer exists before the first call, so nothing below needs the caching
    # allocator; after the first call (which may load the module and look up the scratch
    # array's address) the device's free memory must not move
    xs = [torch.full((n,), float("nan") if call else 0.0, dtype=torch.float64, device="cuda") for call in range(3)]
    torch.cuda.synchronize()
    free_after_first = None
    for call, x in enumerate(xs):
        it, rr, st = hyb.hyb_pcg_solve_noalloc(red["row_ptr"], red["col"], red["val"], red["rhs"], x,
                                               nfn, 1e-12, 10000)
        torch.cuda.synchronize()
        if call == 0:
            free_after_first = torch.cuda.mem_get_info()[0]
        else:
            assert torch.cuda.mem_get_info()[0] == free_after_first, "the entry point allocated device memory"
        assert st == hyb.HYB_OK and it == it_ref
        assert rr <= 1e-12
        assert rel(x.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
    # a general CSR matrix (one row per "face") gives the same solution
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    it, rr, st = hyb.hyb_pcg_solve_noalloc(red["row_ptr"], red["col"], red["val"], red["rhs"], x, 1, 1e-12, 10000)
    assert st == hyb.HYB_OK and rel(x.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
    ctx.close()


def test_noalloc_rejects_oversized_systems():
    import torch
    from paper_1801_08914_gb300 import hyb
    rp = torch.zeros(2, dtype=torch.int64, device="cuda")
    cl = torch.zeros(1, dtype=torch.int32, device="cuda")
    v = torch.ones(1, dtype=torch.float64, device="cuda")
    b = torch.ones(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = hyb.lib()
    import ctypes
    st = lib.hyb_pcg_solve_noalloc(ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(cl.data_ptr()),
                                   ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                   ctypes.c_void_p(x.data_ptr()), (1 << 19) + 1, 1, 1e-12, 10,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), None, None)
    assert st == hyb.HYB_ERR_INVALID_ARG
    # and a valid one-row system still solves: x = 1
    it, rr, st = hyb.hyb_pcg_solve_noalloc(rp.index_fill_(0, torch.tensor([1], device="cuda"), 1), cl, v, b, x,
                                           1, 1e-12, 10)
    assert st == hyb.HYB_OK and abs(x.item() - 1.0) < 1e-15
