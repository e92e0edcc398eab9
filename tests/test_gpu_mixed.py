"""Mixed precision (HYB_MIXED) against the FP64 oracle and the FP64 GPU path.

Elements with contrast beta/alpha up to the threshold are eliminated in FP32 through the
hybridized mixed form (Sec. 3.2, H = H~): every factored matrix there (the alpha mass M,
Z = G^{-1} + D^T M^{-1} D) is well conditioned, so S_T carries an error of order
kappa(M, Z) u_32 ~ 1e-6 whatever the contrast below the threshold; elements above it stay
FP64. The load term g_T comes from the same FP32 solve and carries the same kind of error
(the global FP64 refinement, hyb_refine, removes both); the recovery's element solve is refined
in the mixed variables against FP64 residuals. The bounds asserted, entry by entry (S per CSR
row against the row's largest entry, u per element against the element's largest dof, lambda
and g against their largest entry): S and g <= 100 u_32 kappa_w with kappa_w the largest
kappa(M) or kappa(Z) over the elements; lambda and u <= kappa(H) times that bound. Norm-wise
numbers are printed beside them.
"""
import numpy as np
import pytest

from gpu_helpers import EPS, csr, element_kappa, gpu_run, kappa_w, rel, rel_groups, rel_inf, rel_rows
from oracle.hybrid import Discretization, solve_dense
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu
U32 = np.finfo(np.float32).eps / 2


def test_threshold_below_every_contrast_is_the_fp64_path():
    p = inputs.random_problem(4, 1, 0.2, 401, 1e-2, 1e4, name="mixed64")
    a = gpu_run(p, rtol=1e-13, maxit=20000)
    b = gpu_run(p, rtol=1e-13, maxit=20000, precision=1, threshold=1e-300)
    assert b["split"][1] == 0
    for key in ("val", "rhs"):
        assert np.array_equal(a["red"][key], b["red"][key])
    assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["u"], b["u"])


@pytest.mark.parametrize("k,n", [(0, 5), (1, 4), (2, 3), (3, 3)])
def test_mixed_fp32_path_against_oracle(k, n):
    """All elements on the FP32 path (contrast <= 1e4 = threshold)."""
    p = inputs.random_problem(n, k, 0.2, 410 + k, 1e-2, 1e4, name="mixed32")
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_dense(H, g)
    u = D.recover(lam)
    r = gpu_run(p, rtol=1e-14, maxit=20000, precision=1, threshold=1e4)
    assert r["split"] == (0, p.n_elem, 1e4)
    kw = kappa_w(D)
    ev = np.linalg.eigvalsh(H.toarray())
    kH = ev[-1] / ev[0]
    tol_S = 100 * U32 * kw
    eS, eg = rel_rows(r["red"]["val"], H.data, H.indptr), rel_inf(r["red"]["rhs"], g)
    el, eu = rel_inf(r["lam"], lam), rel_groups(r["u"], u, D.n)
    print(f"mixed k={k}: kappa_w={kw:.1e} kappa_H={kH:.1e} entry-wise S {eS:.1e} g {eg:.1e} lam {el:.1e} u {eu:.1e} "
          f"(tol S {tol_S:.1e}, lam/u {kH * tol_S:.1e}); norm-wise S {rel(r['red']['val'], H.data):.1e} "
          f"u {rel(r['u'], u):.1e}")
    assert eS <= tol_S and eg <= tol_S
    assert el <= kH * tol_S and eu <= kH * tol_S
    Hg = csr(r["red"])
    assert abs(Hg - Hg.T).max() == 0.0


def test_mixed_split_paths():
    """Contrast up to 1e6 with threshold 1e4: both paths in one assembly and one recovery."""
    p = inputs.random_problem(4, 1, 0.2, 420, 1e-2, 1e6, name="mixedsplit")
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_dense(H, g)
    u = D.recover(lam)
    r = gpu_run(p, rtol=1e-14, maxit=50000, precision=1, threshold=1e4)
    n64, n32, _ = r["split"]
    assert n64 > 0 and n32 > 0 and n64 + n32 == p.n_elem
    eS, el, eu = rel_rows(r["red"]["val"], H.data, H.indptr), rel_inf(r["lam"], lam), rel_groups(r["u"], u, D.n)
    print(f"mixed split: {n64} FP64 + {n32} FP32 elements: entry-wise S {eS:.1e} lam {el:.1e} u {eu:.1e}")
    kw = kappa_w(D)
    ev = np.linalg.eigvalsh(H.toarray())
    assert eS <= 100 * U32 * kw and eu <= (ev[-1] / ev[0]) * 100 * U32 * kw


@pytest.mark.parametrize("k,n", [(1, 4), (2, 3), (3, 3)])
def test_mixed_fp32_path_at_contrast_1e6(k, n):
    """Every element on the FP32 path at contrast up to 1e6: the bound on S is the same
    kappa(M, Z) u_32 bound as at low contrast (the mixed form does not see beta / alpha)."""
    p = inputs.random_problem(n, k, 0.2, 430 + k, 1e-2, 1e6, name="mixed32hc")
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_dense(H, g)
    u = D.recover(lam)
    r = gpu_run(p, rtol=1e-14, maxit=50000, precision=1, threshold=1e300)
    assert r["split"][1] == p.n_elem
    kw = kappa_w(D)
    ev = np.linalg.eigvalsh(H.toarray())
    kH = ev[-1] / ev[0]
    eS, el, eu = rel_rows(r["red"]["val"], H.data, H.indptr), rel_inf(r["lam"], lam), rel_groups(r["u"], u, D.n)
    print(f"mixed FP32 k={k} contrast<=1e6: kappa_w={kw:.1e} kappa_H={kH:.1e} entry-wise S {eS:.1e} lam {el:.1e} "
          f"u {eu:.1e}")
    assert eS <= 100 * U32 * kw
    assert el <= kH * 100 * U32 * kw and eu <= kH * 100 * U32 * kw


def test_threshold_autotune():
    """threshold 0 picks the faster element path for the order (all FP32 or all FP64) and
    reports it; a second set-up of the same order reuses the measurement."""
    import time
    from paper_1801_08914_gb300 import hyb
    from gpu_helpers import dev
    for k in (1, 2, 3):
        p = inputs.random_problem(3, k, 0.2, 440 + k, 1e-2, 1e6)
        ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta),
                            precision=hyb.HYB_MIXED, contrast_threshold=0.0)
        n64, n32, theta = ctx.precision_split()
        ctx.close()
        assert theta in (0.0, 1e6) and n64 + n32 == p.n_elem
        assert (n32 == int(np.sum(p.beta / p.alpha <= 1e6))) if theta == 1e6 else (n64 == p.n_elem)
        t = time.perf_counter()
        ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta),
                            precision=hyb.HYB_MIXED, contrast_threshold=0.0)
        again = ctx.precision_split()[2]
        ctx.close()
        print(f"k={k}: autotuned threshold {theta:g} ({n32} FP32, {n64} FP64), cached set-up "
              f"{1e3 * (time.perf_counter() - t):.1f} ms")
        assert again == theta
