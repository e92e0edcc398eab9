"""CUDA path against the CPU FP64 oracle, element by element and entry by entry.

Tolerances. The FP64 GPU path must match the oracle to 1e-12 relative. Both sides
evaluate the same quadrature and the same algebra in a different order, so their
difference is rounding amplified by the conditioning: for S (the CSR values) by the
element condition number kappa(A_T), for lambda and u additionally by kappa(H). The
bound is max(1e-12, kappa eps_64), kappa the larger of the worst kappa(A_T) and kappa(H)
(dense spectra on the oracle side). On the manufactured RT_0 cases (kappa < 1e3) this is
the flat 1e-12 and it is asserted as such.

The bound is asserted entry by entry, so that one wrong small entry cannot hide under the
norm of the large ones: S row by row (max over a CSR row of |S_gpu - S_oracle| against the
largest entry of that row), u element by element (against the element's largest dof),
lambda and g entry-wise against their largest entry. Norm-wise differences are printed
beside them. Index arrays (row pointers, columns) are compared bit-exactly.
"""
import numpy as np
import pytest

from gpu_helpers import EPS, csr, element_kappa, gpu_run, rel, rel_groups, rel_inf, rel_rows
from oracle.hybrid import Discretization, solve_dense
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu


def oracle_run(p, mode="hyb"):
    D = Discretization.from_problem(p)
    if mode == "hyb":
        M, g = D.hybridize()
        lam = solve_dense(M, g)
        u = D.recover(lam)
    else:
        M, g = D.static_condense()
        lam = solve_dense(M, g)
        u = D.sc_recover(lam)
    return D, M, g, lam, u


def kappa_dense(M):
    ev = np.linalg.eigvalsh(M.toarray())
    return ev[-1] / ev[0]


def check_parity(p, mode="hyb", flat=False):
    D, M, g, lam, u = oracle_run(p, mode)
    r = gpu_run(p, mode, rtol=1e-15, maxit=20000)
    red = r["red"]
    assert np.array_equal(red["row_ptr"], M.indptr.astype(np.int64))
    assert np.array_equal(red["col"], M.indices.astype(np.int32))
    kT = element_kappa(D)
    kH = kappa_dense(M)
    tol = 1e-12 if flat else max(1e-12, max(kT, kH) * EPS)
    eS, eg, el, eu = (rel(red["val"], M.data), rel(red["rhs"], g), rel(r["lam"], lam), rel(r["u"], u))
    xS = rel_rows(red["val"], M.data, M.indptr)
    xg, xl = rel_inf(red["rhs"], g), rel_inf(r["lam"], lam)
    xu = rel_groups(r["u"], u, D.n)
    print(f"{p.name} k={p.order} {mode}: kT={kT:.1e} kH={kH:.1e} tol {tol:.1e}; entry-wise S/row {xS:.1e} "
          f"g {xg:.1e} lam {xl:.1e} u/element {xu:.1e}; norm-wise S {eS:.1e} g {eg:.1e} lam {el:.1e} u {eu:.1e}; "
          f"PCG {r['it']} it")
    assert xS <= tol and xg <= tol
    assert xl <= tol and xu <= tol
    return r


def test_config1_closed_form():
    """4^3 unjittered RT_0, u_exact in the space: lambda = -2 everywhere, u = interpolant (1e-12)."""
    p = inputs.make_config(1)
    r = check_parity(p, flat=True)
    assert np.abs(r["lam"] + 2.0).max() < 1e-12
    assert np.abs(r["u"] - p.load).max() < 1e-12 * np.abs(p.load).max()


def test_config1_jittered():
    check_parity(inputs.make_config("1j"), flat=True)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_unit_coefficients_all_orders(k):
    """Jittered 3^3 mesh, alpha = beta = 1, N(0,1) loads, zero essential BC."""
    p = inputs.random_problem(3, k, 0.2, 100 + k, 1.0, 1.0, lognormal_alpha=False, name="unit")
    check_parity(p)


@pytest.mark.parametrize("k,n", [(0, 6), (1, 5), (2, 4), (3, 3)])
def test_contrast_all_orders(k, n):
    """lognormal alpha, beta/alpha in [1e-2, 1e4], several elements of each colour and a ragged count."""
    p = inputs.random_problem(n, k, 0.2, 200 + k, 1e-2, 1e4, name="contrast")
    check_parity(p)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_static_condensation(k):
    p = inputs.random_problem(3, k, 0.2, 300 + k, 1e-2, 1e4, name="sc")
    rs = check_parity(p, mode="sc")
    # same solution as hybridization (Sec. 3.1)
    rh = gpu_run(p, "hyb", rtol=1e-15, maxit=20000)
    D = Discretization.from_problem(p)
    tol = max(1e-12, element_kappa(D) * EPS)
    assert rel_groups(rs["u"], rh["u"], D.n) <= tol


def test_reduced_system_properties_config1_jittered():
    """H symmetric to roundoff (the GPU forms S_T = D Y^T Y D, exactly symmetric per element)."""
    r = gpu_run(inputs.make_config("1j"), solve=False)
    H = csr(r["red"])
    assert abs(H - H.T).max() == 0.0
    np.linalg.cholesky(H.toarray())
