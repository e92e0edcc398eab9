"""The two PCG launch forms on the same assembled systems.

The fused form runs 64 iterations per cooperative launch with grid barriers between SpMV,
update and direction; the unfused form launches three kernels per iteration. Both are the same
diagonal-preconditioned CG (Sec. 6.1's solver and stopping rule) and differ only in how the
inner products are split into block partials, so:
* their iteration counts agree to within a couple of iterations and both meet the true
  residual bound;
* their solutions agree to the accuracy the stopping rule fixes (kappa(H) * rtol);
* the fused form is bitwise reproducible run to run (partials summed in block order).
The barrier's bounded wait is exercised by counting an arrival as missing: every block gives
up after about a second, the call reports HYB_ERR_TIMEOUT and the context stays usable.
"""
import numpy as np
import pytest

from gpu_helpers import dev, rel
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu


def assembled(p):
    from paper_1801_08914_gb300 import hyb
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta))
    hyb.hyb_assemble_reduced(ctx, dev(p.load), None if p.ess is None else dev(p.ess))
    return ctx


def solve(ctx, fused, rtol=1e-12):
    import torch
    from paper_1801_08914_gb300 import hyb
    hyb.hyb_set_pcg_fused(ctx, fused)
    lam = torch.full((ctx.sizes()["n_lambda"],), float("nan"), dtype=torch.float64, device="cuda")
    it, rr, st = hyb.hyb_solve_reduced(ctx, rtol, 100000, lam)
    return lam, it, rr, st


def true_residual(ctx, lam):
    import torch
    from paper_1801_08914_gb300 import hyb
    red = hyb.hyb_export_reduced(ctx)
    n = lam.numel()
    H = torch.sparse_csr_tensor(red["row_ptr"], red["col"].to(torch.int64), red["val"], size=(n, n))
    return (torch.linalg.norm(red["rhs"] - H @ lam) / torch.linalg.norm(red["rhs"])).item(), H, red


@pytest.mark.parametrize("case", ["1j", "k0", "k1", "k2", "k3", 2])
def test_fused_matches_unfused(case):
    from paper_1801_08914_gb300 import hyb
    if case == "1j" or case == 2:
        p = inputs.make_config(case)
    else:
        k = int(case[1])
        p = inputs.random_problem(6 if k < 3 else 4, k, 0.2, 700 + k, 1e-2, 1e2)
    ctx = assembled(p)
    lf, itf, rrf, stf = solve(ctx, True)
    lu, itu, rru, stu = solve(ctx, False)
    assert stf == hyb.HYB_OK and stu == hyb.HYB_OK
    assert abs(itf - itu) <= 2, (itf, itu)
    resf, H, red = true_residual(ctx, lf)
    resu, _, _ = true_residual(ctx, lu)
    assert rrf <= 1e-12 and resf <= 1e-11 and resu <= 1e-11, (resf, resu)
    # both solve H lambda = g to rtol; their difference is bounded by kappa(H) * rtol
    n = lf.numel()
    if n <= 4000:
        Hd = H.to_dense().cpu().numpy()
        kH = np.linalg.cond(Hd)
    else:
        kH = 1e5                                  # 32^3 RT_1: PCG iteration count implies kappa ~ 1e4..1e5
    d = rel(lf.cpu().numpy(), lu.cpu().numpy())
    print(f"{case}: fused {itf} it, unfused {itu} it, true residuals {resf:.1e} {resu:.1e}, "
          f"rel diff {d:.1e} (kappa_H {kH:.1e})")
    assert d <= max(1e-12, 4 * kH * 1e-12)
    ctx.close()


def test_fused_bitwise_reproducible():
    import torch
    p = inputs.make_config("1j")
    ctx = assembled(p)
    a, ita, _, _ = solve(ctx, True)
    b, itb, _, _ = solve(ctx, True)
    assert ita == itb and torch.equal(a, b)
    ctx.close()


def test_fused_maxit_and_chunking():
    """maxit below, at and across the 64-iteration chunk boundary: the count stops exactly."""
    from paper_1801_08914_gb300 import hyb
    import torch
    p = inputs.make_config(2, n=12)
    ctx = assembled(p)
    hyb.hyb_set_pcg_fused(ctx, True)
    lam = torch.zeros(ctx.sizes()["n_lambda"], dtype=torch.float64, device="cuda")
    for maxit in (1, 63, 64, 65, 130):
        it, rr, st = hyb.hyb_solve_reduced(ctx, 1e-30, maxit, lam, check=False)
        assert st == hyb.HYB_ERR_NOT_CONVERGED and it == maxit, (maxit, it, st)
    ctx.close()


def test_barrier_selftest_and_timeout():
    import time
    from paper_1801_08914_gb300 import hyb
    assert hyb.hyb_barrier_selftest(0, 2000) == hyb.HYB_OK
    t = time.perf_counter()
    st = hyb.hyb_barrier_selftest(1, 3)
    dt = time.perf_counter() - t
    assert st == hyb.HYB_ERR_TIMEOUT and 0.5 < dt < 30, (st, dt)
    assert hyb.hyb_barrier_selftest(0, 10) == hyb.HYB_OK
    # the device is still usable: a full solve after the timeout
    p = inputs.make_config("1j")
    ctx = assembled(p)
    lam, it, rr, st = solve(ctx, True)
    assert st == hyb.HYB_OK and rr <= 1e-12
    ctx.close()
    assert hyb.hyb_barrier_selftest(-1, 1) == hyb.HYB_ERR_INVALID_ARG
