"""FP64 refinement of the hybridized solve (hyb_refine).

* Pin of eq. 2.4 on the GPU path: for u = A^-1 (f - C^T lambda) the normal jump C u equals the
  reduced residual g - H lambda. After a loose PCG solve (rtol 1e-8) the jump the library
  measures matches the true residual that an independent sparse product of the exported H gives.
* Mixed precision: H assembled from FP32 element eliminations puts an error of order
  kappa(H) * 1e-7 into lambda and u; refinement steps against the FP64 jump remove it, down to
  the accuracy of the FP64-refined element solves. Measured errors against the FP64 oracle are
  printed before and after.
"""
import numpy as np
import pytest

from gpu_helpers import EPS, dev, element_kappa, rel, rel_groups, rel_inf
from oracle.hybrid import Discretization, solve_dense
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu


def run(p, precision=0, threshold=0.0, rtol=1e-14, steps=0, inner=1e-10):
    import torch
    from paper_1801_08914_gb300 import hyb
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta),
                        precision=precision, contrast_threshold=threshold)
    hyb.hyb_assemble_reduced(ctx, dev(p.load), None if p.ess is None else dev(p.ess))
    sz = ctx.sizes()
    lam = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    it, rr, st = hyb.hyb_solve_reduced(ctx, rtol, 100000, lam)
    u = torch.zeros(sz["n_elem"], sz["n_loc"], dtype=torch.float64, device="cuda")
    hyb.hyb_recover(ctx, lam, u)
    out = dict(lam0=lam.cpu().numpy().copy(), u0=u.cpu().numpy().copy(), it=it, rr=rr)
    jump, st = hyb.hyb_refine(ctx, steps, inner, 100000, lam, u)
    out.update(jump=jump, lam=lam.cpu().numpy(), u=u.cpu().numpy(), status=st, ctx=ctx)
    return out


@pytest.mark.parametrize("k,n", [(0, 5), (1, 4), (2, 3), (3, 2)])
def test_jump_equals_reduced_residual(k, n):
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.random_problem(n, k, 0.2, 800 + k, 1e-2, 1e3)
    r = run(p, rtol=1e-8)
    ctx = r["ctx"]
    red = hyb.hyb_export_reduced(ctx)
    N = red["rhs"].numel()
    H = torch.sparse_csr_tensor(red["row_ptr"], red["col"].to(torch.int64), red["val"], size=(N, N))
    lam = torch.tensor(r["lam0"], device="cuda")
    res = (torch.linalg.norm(red["rhs"] - H @ lam) / torch.linalg.norm(red["rhs"])).item()
    j0 = r["jump"][0]
    print(f"k={k}: PCG residual {r['rr']:.3e}, |g - H lambda|/|g| {res:.6e}, |C u|/|g| {j0:.6e}")
    assert res > 1e-10                                   # a loose solve: the residual dominates roundoff
    assert abs(j0 - res) <= 1e-3 * res + 100 * element_kappa(Discretization.from_problem(p)) * EPS
    ctx.close()


@pytest.mark.parametrize("k,n,hi", [(1, 4, 1e4), (2, 3, 1e4), (3, 3, 1e4), (1, 4, 1e6)])
def test_mixed_refinement_reaches_fp64_accuracy(k, n, hi):
    p = inputs.random_problem(n, k, 0.2, 410 + k if hi == 1e4 else 420, 1e-2, hi)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_dense(H, g)
    u = D.recover(lam)
    r = run(p, precision=1, threshold=1e4, steps=3)
    ev = np.linalg.eigvalsh(H.toarray())
    kH = ev[-1] / ev[0]
    kT = element_kappa(D)
    e0 = rel_inf(r["lam0"], lam), rel_groups(r["u0"], u, D.n)
    e1 = rel_inf(r["lam"], lam), rel_groups(r["u"], u, D.n)
    print(f"mixed k={k} contrast<={hi:.0e}: kappa_H {kH:.1e} kappa_T {kT:.1e}; lambda {e0[0]:.1e} -> {e1[0]:.1e}, "
          f"u {e0[1]:.1e} -> {e1[1]:.1e}; jumps " + " ".join(f"{j:.1e}" for j in r["jump"]))
    assert r["jump"][-1] < r["jump"][0]
    bound = max(1e-11, 10 * max(kH, kT) * kH * EPS)
    assert e1[0] <= bound and e1[1] <= bound, bound
    r["ctx"].close()


def test_refine_rejects_static_condensation():
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.random_problem(3, 1, 0.2, 830, 1e-2, 1e2)
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta))
    hyb.staticcond_assemble(ctx, dev(p.load), None)
    sz = ctx.sizes()
    lam = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    u = torch.zeros(sz["n_elem"], sz["n_loc"], dtype=torch.float64, device="cuda")
    _, st = hyb.hyb_refine(ctx, 1, 1e-10, 100, lam, u, check=False)
    assert st == hyb.HYB_ERR_INVALID_ARG
    ctx.close()
