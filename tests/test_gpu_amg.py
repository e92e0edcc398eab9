"""GPU aggregation multigrid (HYB_PC_AMG) against the oracle's (oracle/amg.py) on the same seeded
problems, through the C ABI: the level sizes, the power estimates of lmax(D^{-1} A), one V-cycle
applied to a seeded vector entry by entry, and CG preconditioned by it (the direct solution,
iteration counts against the oracle's and against diagonal PCG). Sec. 4 (H is H^1-like) and
Sec. 6.1 (AMG-preconditioned CG on H)."""
import numpy as np
import pytest

from gpu_helpers import dev, rel, rel_inf
from oracle import amg
from oracle.hybrid import Discretization, pcg_diag, solve_sparse_direct
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu


def setup_ctx(p, degree, coarsest, precision=0, threshold=0.0):
    from paper_1801_08914_gb300 import hyb
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta),
                        precision=precision, contrast_threshold=threshold)
    hyb.hyb_set_preconditioner(ctx, hyb.HYB_PC_AMG, degree, coarsest)
    hyb.hyb_assemble_reduced(ctx, dev(p.load), None if p.ess is None else dev(p.ess))
    return ctx


@pytest.mark.parametrize("cfg,n,degree,coarsest", [(2, 8, 2, 8), (3, 6, 2, 8), (3, 6, 3, 1), (5, 4, 2, 8),
                                                   (1, 4, 1, 512), (2, 5, 2, 8)])
def test_vcycle_matches_oracle(cfg, n, degree, coarsest):
    """Levels, lmax estimates and z = M^{-1} r entry-wise; odd mesh (5^3: partial blocks) and a
    single-level case (4^3 RT_0, 144 unknowns <= 512: the dense inverse). The recipe's mesh and
    load with beta / alpha = 10^U(-1, 1): at the recipe's contrast (up to 10^6) the two sides' H
    differ by kappa(A_T) eps ~ 1e-10 entry-wise (both eliminate A_T = alpha M + beta K in FP64),
    which the V-cycle carries into z; here H agrees to ~1e-14 and z must too (to 1e-11)."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.make_config(cfg, n=n)
    if cfg != 1:
        p.beta = p.alpha * 10.0 ** np.random.default_rng(11).uniform(-1.0, 1.0, p.alpha.size)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    nfn = (p.order + 1) ** 2
    M = amg.AggregationAMG(H, n, n, n, nfn, degree=degree, coarsest=coarsest)
    ctx = setup_ctx(p, degree, coarsest)
    try:
        levels, sizes, lmax = hyb.hyb_amg_info(ctx)
        assert levels == len(M.A) and sizes == [A.shape[0] for A in M.A], (sizes, [A.shape[0] for A in M.A])
        for l, lo in enumerate(M.lmax):
            assert abs(1.1 * lmax[l] - lo) <= 1e-9 * lo, (l, 1.1 * lmax[l], lo)
        r = np.random.default_rng(7).standard_normal(H.shape[0])
        z = torch.zeros(H.shape[0], dtype=torch.float64, device="cuda")
        hyb.hyb_amg_apply(ctx, dev(r), z)
        zo = M.vcycle(r)
        e_inf, e2 = rel_inf(z.cpu().numpy(), zo), rel(z.cpu().numpy(), zo)
        print(f"\nAMG cfg {cfg} n {n} deg {degree}: levels {sizes}, V-cycle rel inf {e_inf:.2e}, norm {e2:.2e}")
        assert e_inf <= 1e-11
    finally:
        ctx.close()


@pytest.mark.parametrize("cfg,n", [(2, 8), (3, 6), (5, 4)])
def test_amg_pcg_iterations(cfg, n):
    """AMG-PCG to rtol 1e-12 takes the oracle's AMG-PCG iteration count (within 2) and fewer than a
    third of diagonal PCG's, on the recipe's problems (contrast up to 10^6)."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.make_config(cfg, n=n)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    nfn = (p.order + 1) ** 2
    M = amg.AggregationAMG(H, n, n, n, nfn, degree=2, coarsest=8)
    _, it_o, _ = M.pcg(g, rtol=1e-12, maxit=2000)
    _, it_d, _ = pcg_diag(H, g, rtol=1e-12)
    ctx = setup_ctx(p, 2, 8)
    try:
        lam = torch.zeros(H.shape[0], dtype=torch.float64, device="cuda")
        it, rr, st = hyb.hyb_solve_reduced(ctx, 1e-12, 2000, lam, check=False)
        print(f"\nAMG-PCG cfg {cfg} n {n}: {it} its (oracle AMG {it_o}, diagonal {it_d})")
        assert st == hyb.HYB_OK and rr <= 1e-12
        assert abs(it - it_o) <= 2 and 3 * it < it_d
    finally:
        ctx.close()


@pytest.mark.parametrize("cfg,n", [(2, 5), (3, 4), (5, 3)])
def test_amg_pcg_solution(cfg, n):
    """lambda from AMG-PCG (rtol 1e-15) against the oracle's dense solve entry-wise, within the
    parity tests' bound max(1e-12, max(kappa(A_T), kappa(H)) eps): the two sides eliminate A_T in
    FP64 in different orders, so their H differ by about kappa(A_T) eps."""
    import torch
    from paper_1801_08914_gb300 import hyb
    from gpu_helpers import EPS, element_kappa
    from oracle.hybrid import solve_dense
    p = inputs.make_config(cfg, n=n)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    ref = solve_dense(H, g)
    ev = np.linalg.eigvalsh(H.toarray())
    tol = max(1e-12, max(element_kappa(D), ev[-1] / ev[0]) * EPS)
    ctx = setup_ctx(p, 2, 8)
    try:
        lam = torch.zeros(H.shape[0], dtype=torch.float64, device="cuda")
        it, rr, st = hyb.hyb_solve_reduced(ctx, 1e-15, 2000, lam, check=False)
        e = rel_inf(lam.cpu().numpy(), ref)
        print(f"\nAMG-PCG cfg {cfg} n {n}: {it} its to {rr:.1e}, lambda rel inf {e:.2e} (bound {tol:.1e})")
        assert st in (hyb.HYB_OK, hyb.HYB_ERR_NOT_CONVERGED) and rr <= 1e-13
        assert e <= tol
    finally:
        ctx.close()


def test_amg_pcg_full_size_rt1():
    """32^3 RT_1 (the RT_1 bench recipe, 95k faces x 4 nodes): AMG-PCG converges to rtol 1e-12 in
    far fewer iterations than diagonal PCG, to the same lambda (within the two solves' tolerance)."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.make_config(2)
    ctx = setup_ctx(p, 2, 512)
    try:
        n = ctx.sizes()["n_lambda"]
        lam = torch.zeros(n, dtype=torch.float64, device="cuda")
        it, rr, st = hyb.hyb_solve_reduced(ctx, 1e-12, 5000, lam, check=False)
        assert st == hyb.HYB_OK
        hyb.hyb_set_preconditioner(ctx, hyb.HYB_PC_JACOBI, 2, 512)
        lam_d = torch.zeros(n, dtype=torch.float64, device="cuda")
        it_d, rr_d, st_d = hyb.hyb_solve_reduced(ctx, 1e-12, 100000, lam_d, check=False)
        assert st_d == hyb.HYB_OK
        e = rel(lam.cpu().numpy(), lam_d.cpu().numpy())
        print(f"\nAMG-PCG 32^3 RT_1: {it} its vs diagonal {it_d}; lambda difference {e:.2e}")
        assert 5 * it < it_d and e <= 1e-9
    finally:
        ctx.close()


def test_amg_mixed_refinement_accuracy():
    """Mixed context (every element FP32 up to beta/alpha 1e6) with AMG-preconditioned solves and
    the FP64 refinement: u within 1e-9 of the mixed-form oracle per element (as with diagonal PCG)."""
    import torch
    from paper_1801_08914_gb300 import hyb
    from gpu_helpers import rel_groups
    p = inputs.make_config(3, n=4)
    D = Discretization.from_problem(p)
    Hm, gm = D.hybridize_mixed()
    lam_o = solve_sparse_direct(Hm, gm)
    u_o = D.recover_mixed(lam_o)
    ctx = setup_ctx(p, 2, 8, precision=hyb.HYB_MIXED, threshold=1e6)
    try:
        sz = ctx.sizes()
        lam = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
        u = torch.zeros(sz["n_elem"], sz["n_loc"], dtype=torch.float64, device="cuda")
        hyb.hyb_solve_reduced(ctx, 1e-10, 5000, lam)
        hyb.hyb_recover(ctx, lam, u)
        jump = hyb.hyb_refine(ctx, 3, 1e-6, 5000, lam, u)
        eu = rel_groups(u.cpu().numpy(), u_o, sz["n_loc"])
        print(f"\nAMG mixed RT_2 4^3: jump {jump}, u rel per element {eu:.2e}")
        assert eu <= 1e-9
    finally:
        ctx.close()


def test_amg_fp32_level0_in_mixed_contexts():
    """A mixed context whose elements all took the FP32 path applies level 0 of the multigrid (its
    smoothing products and the PCG's product) from the FP32 copy of H: one V-cycle within 1e-5 of
    the same multigrid on the FP64 values (hyb_set_mixed_operator(ctx, 0)), FP32 rounding of the
    scaled operator being the only difference, and AMG-PCG iteration counts within 3 of each other."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.make_config(3, n=6)
    ctx = setup_ctx(p, 2, 8, precision=hyb.HYB_MIXED, threshold=1e6)
    try:
        n64, n32, _ = ctx.precision_split()
        assert n64 == 0 and n32 == p.alpha.size
        n = ctx.sizes()["n_lambda"]
        r = dev(np.random.default_rng(5).standard_normal(n))
        z32 = torch.zeros(n, dtype=torch.float64, device="cuda")
        z64 = torch.zeros(n, dtype=torch.float64, device="cuda")
        hyb.hyb_amg_apply(ctx, r, z32)
        lam32 = torch.zeros(n, dtype=torch.float64, device="cuda")
        it32, rr32, st32 = hyb.hyb_solve_reduced(ctx, 1e-10, 2000, lam32, check=False)
        hyb.hyb_set_mixed_operator(ctx, 0)
        hyb.hyb_amg_apply(ctx, r, z64)
        lam64 = torch.zeros(n, dtype=torch.float64, device="cuda")
        it64, rr64, st64 = hyb.hyb_solve_reduced(ctx, 1e-10, 2000, lam64, check=False)
        e = rel(z32.cpu().numpy(), z64.cpu().numpy())
        el = rel(lam32.cpu().numpy(), lam64.cpu().numpy())
        print(f"\nAMG FP32 level 0: V-cycle vs FP64 {e:.2e}; PCG {it32} vs {it64} its, lambda {el:.2e}")
        assert st32 == hyb.HYB_OK and st64 == hyb.HYB_OK
        assert e <= 1e-5 and abs(it32 - it64) <= 3 and el <= 1e-5
    finally:
        ctx.close()
