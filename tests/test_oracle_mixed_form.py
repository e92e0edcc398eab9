"""The oracle's second route through the hybridized mixed form (Sec. 3.2, eq. 3.3-3.6).

The paper shows that the mixed-form construction gives the same multiplier system as the
primal one (H~ = H). In exact arithmetic the two routes agree; in FP64 they do not at high
contrast, because the primal route forms A_T = alpha M + beta K, whose divergence-free
structure is rounded away when its entries are added up (kappa(A_T) ~ (beta/alpha) h^-2).

Pins:
* low contrast: both routes give the same H, g, lambda and u to rounding (H~ = H, Thm 2.1);
* contrast ~1e6: an extended-precision evaluation of the primal definition (80-bit or wider
  long double, its own Cholesky, from the same FP64 inputs) is the brute-force truth. The
  mixed-form route in FP64 meets it to 1e-9 for S_T and for the element solve of the back
  substitution; the primal route in FP64 does not, which is why the mixed-form route is the
  accuracy reference of the mixed-precision GPU path at contrast 1e6.
"""
import numpy as np
import pytest

from oracle.hybrid import Discretization, solve_dense
from paper_1801_08914_gb300 import inputs

LD = np.longdouble


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("k,n", [(0, 4), (1, 3), (2, 2)])
def test_mixed_route_equals_primal_at_low_contrast(k, n):
    p = inputs.random_problem(n, k, 0.2, 700 + k, 1e-2, 1e2)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_dense(H, g)
    u = D.recover(lam)
    Hm, gm = D.hybridize_mixed()
    lam_m = solve_dense(Hm, gm)
    u_m = D.recover_mixed(lam_m)
    assert np.array_equal(H.indptr, Hm.indptr) and np.array_equal(H.indices, Hm.indices)
    for a, b in ((Hm.data, H.data), (gm, g), (lam_m, lam), (u_m, u)):
        assert rel(a, b) < 1e-11
    # the mixed recovery of the primal lambda is the primal recovery (same element solve)
    assert rel(D.recover_mixed(lam), u) < 1e-11


def _chol_solve_ld(A, B):
    """Cholesky solve in long double (plain column algorithm)."""
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        L[j, j] = np.sqrt(A[j, j] - np.dot(L[j, :j], L[j, :j]))
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    Y = B.copy()
    for j in range(n):
        Y[j] = (Y[j] - L[j, :j] @ Y[:j]) / L[j, j]
    for j in reversed(range(n)):
        Y[j] = (Y[j] - L[j + 1:, j] @ Y[j + 1:]) / L[j, j]
    return Y


def _element_matrix_ld(D, e):
    """A_T of the primal definition (Piola map, same quadrature) evaluated in long double."""
    I = D.integ
    X8 = D.mesh.element_vertices(e).astype(LD)
    J = np.einsum("ci,qcd->qid", X8, I.dN.astype(LD))
    det = (J[:, 0, 0] * (J[:, 1, 1] * J[:, 2, 2] - J[:, 1, 2] * J[:, 2, 1])
           - J[:, 0, 1] * (J[:, 1, 0] * J[:, 2, 2] - J[:, 1, 2] * J[:, 2, 0])
           + J[:, 0, 2] * (J[:, 1, 0] * J[:, 2, 1] - J[:, 1, 1] * J[:, 2, 0]))
    u = np.einsum("qnd,qid->qni", I.val.astype(LD), J) / det[:, None, None]
    dv = I.div.astype(LD) / det[:, None]
    dx = I.wts.astype(LD) * det
    M = np.einsum("q,qni,qmi->nm", dx, u, u)
    return LD(D.alpha[e]) * M + LD(D.beta[e]) * np.einsum("q,qn,qm->nm", dx, dv, dv)


@pytest.mark.skipif(np.finfo(LD).eps > 1e-18, reason="long double is not wider than double here")
@pytest.mark.parametrize("k", [1, 2])
def test_mixed_route_meets_extended_precision_at_contrast_1e6(k):
    p = inputs.random_problem(3, k, 0.2, 460 + k, 1e-2, 1e6)
    D = Discretization.from_problem(p)
    e = int(np.argmax(p.beta / p.alpha))
    contrast = p.beta[e] / p.alpha[e]
    assert contrast > 2e5
    d = D.element_reduced(e)
    dm = D.element_reduced_mixed(e)
    free = d["free"]
    A = _element_matrix_ld(D, e)[np.ix_(free, free)]
    C = d["C"].astype(LD)
    S_ref = (C @ _chol_solve_ld(A, C.T.copy())).astype(np.float64)
    err = lambda S: np.abs(S - S_ref).max() / np.abs(S_ref).max()
    e_primal, e_mixed = err(d["S"]), err(dm["S"])
    # the element solve of the back substitution with a seeded multiplier vector
    lam = np.random.default_rng(5).standard_normal(D.n_lambda)
    r = d["f"] - d["C"].T @ lam[d["lam"]]
    x_ref = _chol_solve_ld(A, r.astype(LD)[:, None])[:, 0].astype(np.float64)
    D.hybridize(elements=[e])
    x_primal = D.recover(lam)[e, free]
    x_mixed = D.recover_mixed(lam)[e, free]
    ex = lambda x: np.abs(x - x_ref).max() / np.abs(x_ref).max()
    print(f"k={k} contrast {contrast:.1e}: S_T primal {e_primal:.1e} mixed {e_mixed:.1e}; "
          f"x_T primal {ex(x_primal):.1e} mixed {ex(x_mixed):.1e}")
    assert e_mixed <= 1e-9 and ex(x_mixed) <= 1e-9
    assert e_mixed < e_primal                  # the primal FP64 route is the less accurate one here
