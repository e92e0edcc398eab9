"""Pins for the oracle's hybridization, static condensation and reduced solves (CPU only).

Each check is fixed by the paper or by mathematics, not by the oracle itself:
closed forms (lambda = -beta div u from the local Neumann reading of Sec. 2.3,
exact reproduction of fields in the discrete space), Theorem 2.1 (hybridized
solution = conforming solution, H SPD), the saddle-point system solved directly
(eq. 2.3), static condensation (Sec. 3.1), the near-nullspace of H (Sec. 4) and
the dof counts the paper prints.
"""
import os

import numpy as np
import pytest

from oracle.hybrid import Discretization, NotSPDError, pcg_diag, solve_dense
from paper_1801_08914_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def test_config1_closed_form_lambda_and_interpolant():
    """u_exact = (1+2x, 3-y, 0.5+z) is in RT_0 on the unjittered 4^3 mesh; div u = 2, beta = 1,
    so the multipliers are -beta div u = -2 everywhere and x_hat is the RT_0 interpolant."""
    p = inputs.make_config(1)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    assert H.shape == (144, 144) and H.nnz == 1200
    lam = solve_dense(H, g)
    assert np.abs(lam + 2.0).max() < 1e-12
    u = D.recover(lam)
    assert np.abs(u - p.load).max() < 1e-12 * np.abs(p.load).max()


def sheared_problem(n, beta, a=(0.4, -1.1, 2.0), bcoef=0.7):
    """Parallelepiped mesh x = S xi_grid; u = a + b x is in RT_0 there (Piola of an affine map).
    Dofs of the interpolant are the face flux densities (J[:,t1] x J[:,t2]) . u at the face nodes,
    computed here from cross products, independently of the oracle's Piola code."""
    S = np.array([[1.0, 0.3, -0.2], [0.1, 0.8, 0.25], [-0.15, 0.05, 1.2]])
    g = np.arange(n + 1) / n
    L, J, I = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([I.ravel(), J.ravel(), L.ravel()], 1) @ S.T
    Jm = S / n
    E = n**3
    load = np.zeros((E, 6))
    a = np.array(a)
    for e in range(E):
        i, j, l = e % n, (e // n) % n, e // (n * n)
        for f in range(6):
            ax, side = f // 2, f % 2
            t = [d for d in range(3) if d != ax]
            ref = np.array([i + 0.5, j + 0.5, l + 0.5])
            ref[ax] = [i, j, l][ax] + side
            x = S @ (ref / n)
            u = a + bcoef * x
            cof = np.cross(Jm[:, t[0]], Jm[:, t[1]])
            if ax == 1:
                cof = -cof               # cyclic order (z, x) for the y row of det(J) J^{-1}
            load[e, f] = cof @ u
    return Discretization(n, n, n, 0, verts, np.ones(E), np.full(E, beta), load, load.copy()), load


@pytest.mark.parametrize("beta", [1.0, 25.0])
def test_sheared_mesh_reproduces_linear_field(beta):
    D, interp = sheared_problem(3, beta)
    H, g = D.hybridize()
    lam = solve_dense(H, g)
    div_u = 3 * 0.7
    assert np.abs(lam + beta * div_u).max() < 1e-11 * beta * div_u
    u = D.recover(lam)
    assert np.abs(u - interp).max() < 1e-12 * np.abs(interp).max()


@pytest.mark.parametrize("k", range(4))
def test_theorem_2_1_hybridized_equals_conforming(k):
    """x_hat = P x (Thm 2.1) on a jittered mesh, unit coefficients: 1e-12 relative."""
    p = inputs.random_problem(3, k, 0.2, 11 + k, 1.0, 1.0, lognormal_alpha=False)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_dense(H, g)
    u = D.recover(lam)
    uc = D.conforming_solve()
    assert rel(u, uc) < 1e-12
    # normal continuity: second block row C x_hat = 0
    assert np.abs(D.constraint_residual(u)).max() < 1e-13 * np.abs(u).max()


def test_theorem_2_1_with_contrast():
    """Same identity with lognormal alpha and contrast up to 1e4: agreement of two FP64 routes is
    bounded by the conditioning, ||du||/||u|| <~ kappa * eps_64 with kappa the larger of
    kappa(H) and the worst element kappa(A_T) (both from dense spectra)."""
    p = inputs.random_problem(3, 1, 0.2, 5, 1e-2, 1e4)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    ev = np.linalg.eigvalsh(H.toarray())
    kappa = max(ev[-1] / ev[0], max(np.linalg.cond(D.element(e)["A"]) for e in range(D.mesh.n_elem)))
    lam = solve_dense(H, g)
    u = D.recover(lam)
    uc = D.conforming_solve()
    assert rel(u, uc) < max(1e-12, kappa * 2.2e-16)


def test_jittered_config1_all_routes_agree():
    p = inputs.make_config("1j")
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_dense(H, g)
    u = D.recover(lam)
    assert rel(u, D.conforming_solve()) < 1e-12
    S, r = D.static_condense()
    assert rel(D.sc_recover(solve_dense(S, r)), u) < 1e-12
    # essential dofs are re-inserted unchanged on boundary faces (x0 face of element 0 is one)
    assert u[0, 0] == p.ess[0, 0]
    lam_p, it, rr = pcg_diag(H, g, rtol=1e-14)
    assert rr <= 1e-14 and rel(lam_p, lam) < 1e-12


@pytest.mark.parametrize("k", [0, 1, 2])
def test_saddle_point_lu_matches(k):
    """Direct LU of [A_hat C^T; C 0] (eq. 2.3) gives the same x_hat and lambda."""
    p = inputs.random_problem(2, k, 0.2, 21 + k, 1.0, 1.0, lognormal_alpha=False)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_dense(H, g)
    u = D.recover(lam)
    us, ls = D.saddle_solve()
    assert rel(ls, lam) < 1e-12 and rel(us, u) < 1e-12


@pytest.mark.parametrize("k", range(4))
def test_static_condensation_same_solution(k):
    """S (Sec. 3.1) and H give the same solution; S shares H's sparsity pattern."""
    p = inputs.random_problem(3, k, 0.2, 31 + k, 1.0, 1.0, lognormal_alpha=False)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    u = D.recover(solve_dense(H, g))
    S, r = D.static_condense()
    usc = D.sc_recover(solve_dense(S, r))
    assert rel(usc, u) < 1e-12
    assert np.array_equal(S.indptr, H.indptr) and np.array_equal(S.indices, H.indices)


@pytest.mark.parametrize("k", range(4))
def test_local_schur_is_spd_and_symmetric(k):
    """S_T = C_T A_T^{-1} C_T^T is formed by a general product, so symmetry is a real check;
    it equals C_b S_hat_b^{-1} C_b^T with S_hat_b the interior Schur complement (Sec. 5)."""
    p = inputs.random_problem(2, k, 0.2, 41 + k, 1e-2, 1e4)
    D = Discretization.from_problem(p)
    b = D.basis
    for e in range(D.mesh.n_elem):
        d = D.element_reduced(e)
        S = d["S"]
        tol = max(1e-14, np.linalg.cond(d["A"]) * 2.2e-16) * np.abs(S).max()
        assert np.abs(S - S.T).max() <= tol
        assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0
        free = d["free"]
        ii = np.nonzero(free < b.n_interior)[0]
        bb = np.nonzero(free >= b.n_interior)[0]
        A = d["A"]
        Sh = A[np.ix_(bb, bb)]
        if ii.size:
            Sh = Sh - A[np.ix_(bb, ii)] @ np.linalg.solve(A[np.ix_(ii, ii)], A[np.ix_(ii, bb)])
        Cb = d["C"][:, bb]
        S2 = Cb @ np.linalg.solve(Sh, Cb.T)
        assert np.abs(S2 - S).max() < tol


def nnz_formula(n, k):
    """nnz(H) on an n^3 mesh counted by hand: row (f, m) couples f with the interior faces of its
    two neighbours; per axis sum over faces of 1 + [i>=2] + [i<=n-2] + 2([j>=1]+[j<=n-2]+[l>=1]+[l<=n-2])."""
    nf = (k + 1) ** 2
    per_axis = n * n * (3 * n - 5) + 8 * n * (n - 1) ** 2
    return 3 * per_axis * nf * nf


@pytest.mark.parametrize("n,k", [(2, 0), (3, 1), (4, 0), (3, 2)])
def test_reduced_size_and_nnz(n, k):
    p = inputs.random_problem(n, k, 0.1, 3, 1.0, 1.0, lognormal_alpha=False)
    D = Discretization.from_problem(p)
    H, _ = D.hybridize()
    assert H.shape[0] == 3 * n * n * (n - 1) * (k + 1) ** 2
    assert H.nnz == nnz_formula(n, k)
    assert np.abs((H - H.T).toarray()).max() < 1e-14 * abs(H).max()
    np.linalg.cholesky(H.toarray())              # SPD (Thm 2.1 proof)


def test_nnz_formula_at_benchmark_sizes():
    assert nnz_formula(4, 0) == 1200
    assert nnz_formula(32, 1) == 16_281_600
    assert nnz_formula(96, 2) == 2_318_056_704
    assert nnz_formula(64, 3) == 2_148_925_440


def test_paper_sizes_golden():
    """Global RT_k dof counts the paper prints (Tables 6.2-6.4, 6.8) from the oracle's mesh topology."""
    from oracle.basis import RTBasis
    from oracle.mesh import StructuredHexMesh
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_sizes.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) >= 5
    for r in rows:
        nx, ny, nz, k, size = map(int, r[:5])
        m = StructuredHexMesh.__new__(StructuredHexMesh)
        m.dims = (nx, ny, nz)
        nfa = []
        for d in range(3):
            across = [m.dims[a] for a in range(3) if a != d]
            nfa.append((m.dims[d] + 1) * across[0] * across[1])
        b = RTBasis(k)
        assert sum(nfa) * b.n_face_nodes + nx * ny * nz * b.n_interior == size


def test_near_nullspace_is_constant():
    """Sec. 4: for div-dominated problems the constant multiplier is H's near-nullspace."""
    p = inputs.random_problem(4, 0, 0.15, 9, 1e6, 1e6, lognormal_alpha=False)
    D = Discretization.from_problem(p)
    H, _ = D.hybridize()
    one = np.ones(H.shape[0])
    rq = lambda v: v @ (H @ v) / (v @ v)
    rng = np.random.default_rng(0)
    r = np.median([rq(rng.standard_normal(H.shape[0])) for _ in range(5)])
    assert rq(one) < 1e-3 * r


def test_not_spd_detected():
    p = inputs.random_problem(2, 0, 0.1, 3, 1.0, 1.0, lognormal_alpha=False)
    p.alpha[1] = -1.0
    p.beta[1] = 0.0
    D = Discretization.from_problem(p)
    with pytest.raises(NotSPDError):
        D.hybridize()


@pytest.mark.parametrize("k", range(4))
def test_mixed_form_gives_the_same_H(k):
    """Sec. 3.2: H~ from the hybridized mixed form equals H (A = M + B^T W^{-1} B exactly);
    also checks that identity on the element matrix itself."""
    p = inputs.random_problem(2, k, 0.2, 61 + k, 1e-2, 1e2)
    D = Discretization.from_problem(p)
    for e in range(D.mesh.n_elem):
        M, B, W, d = D.mixed_form_blocks(e)
        A2 = M + B.T @ np.linalg.solve(W, B)
        assert np.abs(A2 - d["A"]).max() < 1e-12 * np.abs(d["A"]).max()
        tol = max(1e-12, np.linalg.cond(d["A"]) * 2.2e-16)
        S1 = D.element_reduced(e)
        S2 = D.element_reduced_mixed(e)
        assert rel(S2["S"], S1["S"]) < tol and rel(S2["g"], S1["g"]) < tol
