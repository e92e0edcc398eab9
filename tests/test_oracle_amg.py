"""Pins for the oracle's aggregation multigrid preconditioner of H (CPU only).

What fixes each check, independently of the multigrid code: the mesh topology (every interior
face lies on the boundary of cells in blocks at most one apart; the face count of a block),
the Galerkin identity u^T (P^T A P) v = (P u)^T A (P v) against dense products with a
prolongation built from the face list by explicit loops, the closed form of the Chebyshev
smoother's error propagation (the scaled Chebyshev polynomial T_d((theta - t) / delta) /
T_d(theta / delta) of the eigenvalues of D^{-1/2} A D^{-1/2}), the symmetry and definiteness
of a V-cycle with equal pre- and post-smoothing, an exact coarse solve when a single level is
left, and the solution of H lambda = g by a sparse direct solve.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import amg
from oracle.hybrid import Discretization, pcg_diag, solve_sparse_direct
from oracle.mesh import StructuredHexMesh
from paper_1801_08914_gb300 import inputs


def reduced(cfg, n, order=None):
    p = inputs.make_config(cfg, n=n)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    return p, H, g


def test_face_positions_follow_the_multiplier_order():
    """face_positions lists the interior faces in the order of StructuredHexMesh.interior_face_index."""
    nx, ny, nz = 3, 4, 2
    m = StructuredHexMesh(nx, ny, nz, np.zeros(((nx + 1) * (ny + 1) * (nz + 1), 3)))
    pos = amg.face_positions(nx, ny, nz)
    assert len(pos) == m.n_interior_faces
    for idx, (d, i, j, l) in enumerate(pos):
        assert m.interior_face_index(d, [i, j, l]) == idx


def test_aggregates_are_cell_blocks():
    """On a 4^3 mesh the 2x2x2 blocks hold 12 faces at the origin block, 24 in the opposite one
    (every face of a full block whose planes lie inside the mesh), and the faces of one cell
    never span blocks more than one apart."""
    n = 4
    agg, B = amg.face_aggregates(n, n, n)
    assert B == (2, 2, 2)
    counts = np.bincount(agg, minlength=8)
    # block (0,0,0): x-faces at plane 1 only (plane 0 is the boundary), two cells across each way
    assert counts[0] == 3 * (1 * 2 * 2)
    # block (1,1,1): planes 2 and 3 along every axis
    assert counts[7] == 3 * (2 * 2 * 2)
    assert counts.sum() == 3 * (n - 1) * n * n
    m = StructuredHexMesh(n, n, n, np.zeros(((n + 1) ** 3, 3)))
    bxyz = np.stack([agg % 2, (agg // 2) % 2, agg // 4], axis=1)
    for e in range(m.n_elem):
        faces = [fi for _, fi in m.element_faces(e) if fi >= 0]
        b = bxyz[faces]
        assert (b.max(axis=0) - b.min(axis=0)).max() <= 1


def test_galerkin_operator_against_dense_products():
    """u^T A_1 v = (P u)^T H (P v) for random u, v, with P written out face by face."""
    p, H, g = reduced(2, 4)
    nfn = 4
    M = amg.AggregationAMG(H, 4, 4, 4, nfn, coarsest=1)
    Hd = H.toarray()
    nf = H.shape[0] // nfn
    B = (2, 2, 2)
    P = np.zeros((H.shape[0], 8))
    for f, (_, i, j, l) in enumerate(amg.face_positions(4, 4, 4)):
        P[f * nfn:(f + 1) * nfn, (i // 2) + 2 * ((j // 2) + 2 * (l // 2))] = 1.0
    assert f == nf - 1
    rng = np.random.default_rng(0)
    for _ in range(3):
        u, v = rng.standard_normal(8), rng.standard_normal(8)
        lhs = u @ (M.A[1] @ v)
        rhs = (P @ u) @ Hd @ (P @ v)
        assert abs(lhs - rhs) <= 1e-12 * abs(Hd).sum()
    assert len(M.A) == 3 and M.A[2].shape == (1, 1)


def test_chebyshev_smoother_is_the_scaled_chebyshev_polynomial():
    """Error propagation of one smoothing pass on A x = 0: e -> p(D^{-1} A) e with
    p(t) = T_d((theta - t) / delta) / T_d(theta / delta), checked on the eigenpairs of
    D^{-1/2} A D^{-1/2}; degrees 1 to 3."""
    p, H, g = reduced(2, 3)
    n = H.shape[0]
    Hd = H.toarray()
    d = np.diag(Hd)
    S = Hd / np.sqrt(np.outer(d, d))
    w, V = np.linalg.eigh(S)
    for degree in (1, 2, 3):
        M = amg.AggregationAMG(H, 3, 3, 3, 4, degree=degree, coarsest=1)
        theta, delta, _ = amg.chebyshev_coefficients(M.lmax[0], M.ratio, degree)
        # T_d by its defining recurrence
        def T(x):
            t0, t1 = np.ones_like(x), x
            if degree == 0:
                return t0
            for _ in range(1, degree):
                t0, t1 = t1, 2 * x * t1 - t0
            return t1
        pw = T((theta - w) / delta) / T(np.array(theta / delta))
        E = np.zeros((n, n))
        for c in range(n):
            x, _ = M.smooth(0, np.zeros(n), np.eye(n)[:, c])
            E[:, c] = x
        # in the scaled basis y = D^{1/2} e the propagation is V diag(pw) V^T
        Es = np.sqrt(d)[:, None] * E / np.sqrt(d)[None, :]
        assert np.abs(Es - (V * pw) @ V.T).max() < 1e-10


def test_power_estimate_brackets_the_largest_eigenvalue():
    """lmax(D^{-1} A) from 12 power steps lies within [0.8, 1] of the true value (the stored lmax
    adds the 10% margin)."""
    p, H, g = reduced(2, 4)
    Hd = H.toarray()
    d = np.diag(Hd)
    true = sla.eigh(Hd, np.diag(d), eigvals_only=True)[-1]
    M = amg.AggregationAMG(H, 4, 4, 4, 4, coarsest=1)
    est = M.lmax[0] / 1.1
    assert 0.8 * true <= est <= true * (1 + 1e-12)


def test_vcycle_symmetric_positive_definite():
    """z^T M y = y^T M z and y^T M y > 0 for the V-cycle M (degree 2, three levels)."""
    p, H, g = reduced(2, 4)
    M = amg.AggregationAMG(H, 4, 4, 4, 4, coarsest=1)
    assert len(M.A) == 3
    rng = np.random.default_rng(1)
    y, z = rng.standard_normal(H.shape[0]), rng.standard_normal(H.shape[0])
    a, b = z @ M.vcycle(y), y @ M.vcycle(z)
    assert abs(a - b) <= 1e-11 * (abs(a) + abs(b))
    assert y @ M.vcycle(y) > 0 and z @ M.vcycle(z) > 0


def test_single_level_is_the_exact_solve():
    """With every unknown on the coarsest level the V-cycle is H^{-1}."""
    p, H, g = reduced(2, 3)
    M = amg.AggregationAMG(H, 3, 3, 3, 4, coarsest=10 ** 6)
    assert len(M.A) == 1
    x = M.vcycle(g)
    ref = solve_sparse_direct(H, g)
    assert np.linalg.norm(x - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("cfg,n", [(2, 8), (3, 6)])
def test_amg_pcg_solves_and_beats_diagonal_pcg(cfg, n):
    """AMG-preconditioned CG reaches the direct solution (rtol 1e-12) in fewer than a third of the
    iterations diagonal PCG needs (RT_1 8^3, RT_2 6^3, contrast up to 10^6)."""
    p, H, g = reduced(cfg, n)
    ref = solve_sparse_direct(H, g)
    nfn = (p.order + 1) ** 2
    M = amg.AggregationAMG(H, n, n, n, nfn, coarsest=8)
    x, it, rr = M.pcg(g, rtol=1e-12, maxit=2000)
    xd, itd, _ = pcg_diag(H, g, rtol=1e-12)
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
    assert it * 3 < itd, (it, itd)
