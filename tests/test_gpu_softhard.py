"""The soft-hard materials test of Sec. 6.1 on the CUDA path: natural boundary faces (no
essential data, boundary-face dofs stay unknowns), mass coefficient 10^p on two cubes.

Tolerances as in the parity suite: both sides evaluate the same quadrature and algebra in a
different order, so they differ by rounding amplified by the conditioning, bounded by
max(1e-12, kappa eps) with kappa the worst element condition number (S, g) and additionally
kappa(H) (lambda, u). The soft inclusion (p = -8) raises kappa(A_T) to about 1e11..1e13; the
bounds follow. Closed form at p = 0: u = g = (1, 1, 1) exactly, lambda = 0.
The mixed path: elements with beta / alpha above the autotuned threshold (1e6) stay FP64, so
at p = -8 the soft inclusion is eliminated in FP64 and the rest in FP32; the FP64 refinement
then brings u to the FP64 solution.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from gpu_helpers import EPS, dev, element_kappa, gpu_run, rel, rel_groups, rel_inf, rel_rows
from oracle.hybrid import Discretization, solve_sparse_direct
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu


def kappa_sparse(H):
    hi = spla.eigsh(H, k=1, which="LA", return_eigenvectors=False)[0]
    lo = spla.eigsh(H.tocsc(), k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    return hi / lo


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_constant_field_closed_form(k):
    p = inputs.soft_hard_problem(k, 0.0, nz=4)
    r = gpu_run(p, rtol=1e-14, maxit=20000)
    eu = np.abs(r["u"] - p.load).max() / np.abs(p.load).max()
    print(f"soft-hard p=0 k={k}: |u - g| {eu:.1e}, |lambda| {np.abs(r['lam']).max():.1e}, PCG {r['it']} it")
    assert eu < 1e-10 and np.abs(r["lam"]).max() < 1e-12


@pytest.mark.parametrize("k,pexp", [(0, -8.0), (0, 8.0), (1, -8.0), (1, 8.0), (2, -8.0), (2, 8.0)])
def test_parity_fp64(k, pexp):
    p = inputs.soft_hard_problem(k, pexp, nz=4)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_sparse_direct(H, g)
    u = D.recover(lam)
    r = gpu_run(p, rtol=1e-15, maxit=50000)
    red = r["red"]
    assert np.array_equal(red["row_ptr"], H.indptr.astype(np.int64))
    assert np.array_equal(red["col"], H.indices.astype(np.int32))
    kT, kH = element_kappa(D), kappa_sparse(H)
    tol_S, tol_u = max(1e-12, kT * EPS), max(1e-12, max(kT, kH) * EPS)
    eS, eg = rel_rows(red["val"], H.data, H.indptr), rel_inf(red["rhs"], g)
    el, eu = rel_inf(r["lam"], lam), rel_groups(r["u"], u, D.n)
    print(f"soft-hard k={k} p={pexp:+.0f}: kT {kT:.1e} kH {kH:.1e} entry-wise S/row {eS:.1e} g {eg:.1e} "
          f"lam {el:.1e} u/element {eu:.1e} (tol {tol_S:.1e}/{tol_u:.1e}); norm-wise u {rel(r['u'], u):.1e}; "
          f"PCG {r['it']} it")
    assert eS <= tol_S and eg <= tol_S
    assert el <= tol_u and eu <= tol_u
    assert r["status"] == 0


def test_natural_flag_rules():
    """Static condensation refuses natural boundary faces; the setter validates its argument
    and switching the reading drops the assembled state."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.soft_hard_problem(1, 0.0, nz=4)
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta))
    assert hyb.lib().hyb_set_natural_bc(ctx.handle, 2) == hyb.HYB_ERR_INVALID_ARG
    hyb.hyb_set_natural_bc(ctx, True)
    assert hyb.staticcond_assemble(ctx, dev(p.load), check=False) == hyb.HYB_ERR_INVALID_ARG
    hyb.hyb_assemble_reduced(ctx, dev(p.load))
    sz = ctx.sizes()
    lam = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    assert hyb.hyb_solve_reduced(ctx, 1e-12, 20000, lam, check=False)[2] == hyb.HYB_OK
    hyb.hyb_set_natural_bc(ctx, False)
    assert hyb.hyb_solve_reduced(ctx, 1e-12, 20000, lam, check=False)[2] == hyb.HYB_ERR_INVALID_ARG
    ctx.close()


@pytest.mark.parametrize("k,pexp", [(2, -8.0), (2, 8.0), (3, -8.0), (3, 8.0), (3, 0.0)])
def test_mixed_threshold_and_refinement(k, pexp):
    """Autotuned mixed path + two FP64 refinement steps against the FP64 GPU path."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.soft_hard_problem(k, pexp, nz=4)
    r64 = gpu_run(p, rtol=1e-15, maxit=50000)
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta),
                        precision=hyb.HYB_MIXED, contrast_threshold=0.0)
    hyb.hyb_set_natural_bc(ctx, True)
    n64, n32, theta = ctx.precision_split()
    soft = int(np.sum(p.beta / p.alpha > theta))
    assert n64 == soft and n32 == p.n_elem - soft
    hyb.hyb_assemble_reduced(ctx, dev(p.load))
    sz = ctx.sizes()
    lam = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    # the mixed context's PCG applies H from its FP32 copy: its first solve goes to 1e-10, the
    # FP64 refinement steps take the jump the rest of the way
    it, rr, st = hyb.hyb_solve_reduced(ctx, 1e-10, 50000, lam, check=False)
    assert st == hyb.HYB_OK
    u = torch.zeros(sz["n_elem"], sz["n_loc"], dtype=torch.float64, device="cuda")
    hyb.hyb_recover(ctx, lam, u)
    u0 = u.cpu().numpy().copy()
    jumps, _ = hyb.hyb_refine(ctx, 2, 1e-6, 50000, lam, u)
    torch.cuda.synchronize()
    uu, ll = u.cpu().numpy(), lam.cpu().numpy()
    ctx.close()
    # the element condition numbers, from one element of each coefficient (all cells are equal boxes)
    D = Discretization.from_problem(p)
    ins = int(np.argmax(p.alpha != 1.0)) if pexp != 0.0 else 0
    kT = element_kappa(D, [0, ins])
    tol = max(1e-9, kT * EPS)
    e0, eu = rel(u0, r64["u"]), rel(uu, r64["u"])
    print(f"soft-hard mixed k={k} p={pexp:+.0f}: theta {theta:g}, {n64} FP64 + {n32} FP32 elements, "
          f"u before {e0:.1e} after {eu:.1e} (tol {tol:.1e}), jumps {['%.1e' % j for j in jumps]}")
    if pexp == 0.0:
        assert np.abs(uu - p.load).max() < 1e-10 * np.abs(p.load).max()
    else:
        assert eu <= tol and jumps[-1] <= 1e-9
