"""Pins for the natural-boundary (soft-hard, Sec. 6.1) reading of the oracle (CPU only).

The soft-hard test poses eq. 5.1 over all of H(div): no boundary face carries essential data.
What fixes the answer independently of the oracle's hybridization code:
  * p = 0 (alpha = beta = 1) and g = (1, 1, 1): u = g solves alpha u - grad(beta div u) = g with
    div u = 0, so the natural condition beta div u = 0 holds; a constant field lies in RT_k on
    box cells, so the discrete solution is its interpolant exactly, and the multipliers
    (-beta div u on the faces) vanish;
  * Theorem 2.1: the hybridized solution equals the conforming one (P^T A_hat P assembled with
    +1 copies, boundary-face dofs unknown), and the saddle system of eq. 2.3 solved by LU;
  * the mixed form of Sec. 3.2 gives the same H;
  * the element-local dof order of the input contract is the oracle basis's.
"""
import numpy as np
import pytest

from oracle.basis import RTBasis
from oracle.hybrid import Discretization, solve_sparse_direct
from paper_1801_08914_gb300 import inputs


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_dof_component_contract(k):
    b = RTBasis(k)
    assert np.array_equal(np.array([c for c, _ in b.dofs]), inputs.dof_component(k))


def test_inclusion_layout():
    p = inputs.soft_hard_problem(0, 4.0, nz=8)
    assert (p.nx, p.ny, p.nz) == (16, 16, 8) and p.natural and p.ess is None
    a = p.alpha.reshape(8, 16, 16)                      # [l][j][i]
    ref = np.ones((8, 16, 16))
    ref[2:4, 4:8, 4:8] = 1e4                              # [1/4, 1/2]^3
    ref[4:6, 8:12, 8:12] = 1e4                            # [1/2, 3/4]^3
    assert np.array_equal(a, ref) and np.all(p.beta == 1.0)
    with pytest.raises(ValueError):
        inputs.soft_hard_problem(1, 0.0, nz=6)


@pytest.mark.parametrize("k", [0, 1])
def test_constant_field_reproduced(k):
    p = inputs.soft_hard_problem(k, 0.0, nz=4)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_sparse_direct(H, g)
    assert np.abs(lam).max() < 1e-12
    u = D.recover(lam)
    assert np.abs(u - p.load).max() < 1e-12 * np.abs(p.load).max()
    assert np.abs(D.constraint_residual(u)).max() < 1e-14


@pytest.mark.parametrize("k,pexp", [(0, 8.0), (0, -8.0), (1, 4.0), (1, -4.0)])
def test_hybridized_equals_conforming(k, pexp):
    p = inputs.soft_hard_problem(k, pexp, nz=4)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_sparse_direct(H, g)
    u = D.recover(lam)
    uc = D.conforming_solve()
    # alpha = 10^p < 1 makes the inclusion's divergence-free modes 10^-p times softer than the
    # rest: two different direct solves then agree to about that factor times round-off
    tol = 1e-9 * max(1.0, 10.0 ** (-pexp) / 1e2)
    assert rel(u, uc) < tol
    assert np.abs(D.constraint_residual(u)).max() < tol * np.abs(u).max()
    # the boundary-face dofs are unknowns: not all zero, unlike an essential zero trace
    b = D.basis
    bnd = [(e, a) for e in range(p.n_elem) for a, (_, fi) in enumerate(D.mesh.element_faces(e)) if fi < 0]
    vals = np.array([u[e, b.n_interior + a * D.nfn: b.n_interior + (a + 1) * D.nfn] for e, a in bnd])
    assert np.abs(vals).max() > 1e-3 * np.abs(u).max()


def test_saddle_lu_matches_natural():
    p = inputs.soft_hard_problem(0, -4.0, nz=4)
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam = solve_sparse_direct(H, g)
    u = D.recover(lam)
    us, lams = D.saddle_solve()
    assert rel(u, us) < 1e-10 and rel(lam, lams) < 1e-9


def test_mixed_form_same_H_natural():
    p = inputs.soft_hard_problem(1, -4.0, nz=4)
    D = Discretization.from_problem(p)
    for e in (0, 37, 200):
        a, m = D.element_reduced(e), D.element_reduced_mixed(e)
        assert rel(m["S"], a["S"]) < 1e-10 and rel(m["g"], a["g"]) < 1e-10


def test_static_condensation_needs_essential_faces():
    p = inputs.soft_hard_problem(0, 0.0, nz=4)
    with pytest.raises(NotImplementedError):
        Discretization.from_problem(p).static_condense()


def test_default_meshes_are_the_papers():
    """The generator's default mesh per order is the paper's initial mesh (Sec. 6.1), whose
    global RT_k dof count is the size its tables print (tests/golden/paper_sizes.txt)."""
    import os
    golden = os.path.join(os.path.dirname(__file__), "golden", "paper_sizes.txt")
    rows = [l.split() for l in open(golden) if l.strip() and l[0] != "#"]
    sh = {int(r[3]): tuple(map(int, r[:3])) + (int(r[4]),) for r in rows if "6.1" in " ".join(r[5:])}
    assert set(sh) == {0, 1, 3}
    for k, (nx, ny, nz, size) in sh.items():
        p = inputs.soft_hard_problem(k, 0.0)
        assert (p.nx, p.ny, p.nz) == (nx, ny, nz)
        b = RTBasis(k)
        faces = (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1)
        assert faces * b.n_face_nodes + p.n_elem * b.n_interior == size
