"""Pins for the oracle's master / slave hybridization and its subdomain forms (CPU only).

What fixes each check, independently of the code under test: the constraint algebra of
Example 2.1 (C P = 0, ker C = range P); a global field of RT_k on a mesh of boxes is in the
broken space on both sides of every face, so its nodal interpolant satisfies every master /
slave relation exactly; the physical normal component u.n of any conforming field (u = P x) is
the same from both sides at any point of a non-conforming face, evaluated through each side's
own trilinear map and Piola transform; Thm 2.1's equivalence (the hybridized solution is the
conforming one); the existing structured-mesh oracle (natural boundary) on the same cells when
the interface is conforming; and the subdomain eliminations (Sec. 1), which must give the same
solution with fewer multipliers / global unknowns.
"""
import numpy as np
import pytest

from oracle.element import trilinear_jacobian, trilinear_map
from oracle.hybrid import Discretization
from oracle.nonconforming import TwoLevelDiscretization
from paper_1801_08914_gb300 import inputs


def two_level(k, refine=True, gamma=0.2, lines=0.2, seed=11, nx=2, ny=2, nzc=1, nzf=2):
    p = inputs.two_level_problem(nx, ny, nzc, nzf, k, seed, refine=refine, lines=lines, gamma=gamma)
    return p, TwoLevelDiscretization(p)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_constraint_algebra(k):
    """C P = 0 and dim ker C = rank P (= the number of i and m dofs): range P = ker C."""
    _, D = two_level(k)
    assert abs(D.C @ D.P).max() <= 1e-15
    C = D.C.toarray()
    sv = np.linalg.svd(C, compute_uv=False)
    rank_C = int((sv > 1e-10 * sv[0]).sum())
    assert rank_C == D.n_lambda                         # one independent row per slave
    assert D.N - rank_C == D.P.shape[1]
    sp_ = np.linalg.svd(D.P.toarray(), compute_uv=False)
    assert int((sp_ > 1e-10 * sp_[0]).sum()) == D.P.shape[1]


def interpolate(D, field):
    """Broken nodal interpolant: dof i of element e = reference component c_i of det J J^{-1} u(x)
    at the dof's node (the inverse Piola map)."""
    b = D.basis
    u = np.zeros(D.N)
    for e in range(D.E):
        X8 = D.X8[e]
        for i in range(b.n):
            c, _ = b.dofs[i]
            xi = b.node(i)
            J = trilinear_jacobian(X8, xi)
            uh = np.linalg.det(J) * np.linalg.solve(J, field(trilinear_map(X8, xi)))
            u[e * b.n + i] = uh[c]
    return u


def rt_field(k, seed):
    """u = sum of separable terms with component c of degree <= k+1 along axis c and <= k across:
    a global field of RT_k on any mesh of axis-aligned boxes."""
    rng = np.random.default_rng(seed)
    terms = []
    for c in range(3):
        for _ in range(3):
            degs = [k + 1 if d == c else k for d in range(3)]
            coefs = [rng.standard_normal(deg + 1) for deg in degs]
            terms.append((c, coefs))

    def field(x):
        v = np.zeros(3)
        for c, coefs in terms:
            v[c] += np.prod([np.polyval(coefs[d], x[d]) for d in range(3)])
        return v
    return field


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_rt_field_interpolant_satisfies_the_relations(k):
    """On boxes (grid lines moved, no vertex jitter) the interpolant of a global RT_k field has
    C u = 0 to rounding: every conforming and every 1:4 master / slave relation holds."""
    _, D = two_level(k, gamma=0.0, lines=0.25, nzf=1)
    u = interpolate(D, rt_field(k, 5 + k))
    res = D.C @ u
    assert np.abs(res).max() <= 1e-11 * np.abs(u).max(), np.abs(res).max()


@pytest.mark.parametrize("k", [0, 1, 2])
def test_normal_component_continuous_across_nonconforming_faces(k):
    """u = P x for random x on the jittered two-level mesh: at random points of every fine
    bottom face on the interface, u.n from the fine cell equals u.n from the coarse cell below
    (each side through its own trilinear map, Piola map u = J u_hat / det J and basis)."""
    p, D = two_level(k)
    rng = np.random.default_rng(3)
    u = D.P @ rng.standard_normal(D.P.shape[1])
    b = D.basis
    worst, scale = 0.0, 0.0
    for j in range(p.my):
        for i in range(p.mx):
            ef = D.elem_index(1, i, j, 0)
            ec = D.elem_index(0, i // 2, j // 2, p.nzc - 1)
            for s, t in rng.random((3, 2)):
                xf = np.array([s, t, 0.0])
                xc = np.array([((i % 2) + s) / 2.0, ((j % 2) + t) / 2.0, 1.0])
                pf, pc = trilinear_map(D.X8[ef], xf), trilinear_map(D.X8[ec], xc)
                assert np.abs(pf - pc).max() <= 1e-14        # the same physical point
                vals = []
                for e, xr in ((ef, xf), (ec, xc)):
                    J = trilinear_jacobian(D.X8[e], xr)
                    val, _ = b.eval(xr[None, :])
                    uh = val[0].T @ u[e * b.n:(e + 1) * b.n]
                    vals.append(J @ uh / np.linalg.det(J))
                Jf = trilinear_jacobian(D.X8[ef], xf)
                nrm = np.cross(Jf[:, 0], Jf[:, 1])
                nrm /= np.linalg.norm(nrm)
                worst = max(worst, abs(vals[0] @ nrm - vals[1] @ nrm))
                scale = max(scale, abs(vals[1] @ nrm))
    assert worst <= 1e-11 * scale, (worst, scale)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_hybridized_equals_conforming(k):
    """Thm 2.1 with Example 2.1's P and C: x_hat = A_hat^{-1}(f_hat - C^T lam) equals P x."""
    _, D = two_level(k)
    u_c = D.conforming_solve()
    u_h, lam, H = D.hybridized_solve()
    assert np.linalg.norm(u_h - u_c) <= 1e-10 * np.linalg.norm(u_c)
    assert np.abs(D.C @ u_h).max() <= 1e-10 * np.abs(u_h).max()
    w = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert w[0] > 0 and np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


@pytest.mark.parametrize("k", [0, 1])
def test_conforming_interface_matches_the_structured_oracle(k):
    """With refine=False the two blocks are one structured grid; the master / slave route must
    give the solution of oracle.hybrid (natural boundary) on the same cells and load."""
    p, D = two_level(k, refine=False, lines=0.0, gamma=0.0, nx=2, ny=3, nzc=2, nzf=1)
    nz = p.nzc + p.nzf
    verts = np.concatenate([p.coarse_vertices, p.fine_vertices[(p.nx + 1) * (p.ny + 1):]])
    S = Discretization(p.nx, p.ny, nz, k, verts, p.alpha, p.beta, p.load, natural=True)
    H, g = S.hybridize()
    lam = np.linalg.solve(H.toarray(), g)
    u_s = S.recover(lam).ravel()
    u_h, _, _ = D.hybridized_solve()
    assert np.linalg.norm(u_h - u_s) <= 1e-10 * np.linalg.norm(u_s)


def block_partition(D, p):
    """Subdomains: the coarse block, and the fine block cut into 2 x 2 columns of cells."""
    part = np.zeros(D.E, dtype=np.int64)
    for e in range(D.Ec, D.E):
        _, i, j, _ = D.cell[e]
        part[e] = 1 + (i * 2 // p.mx) + 2 * (j * 2 // p.my)
    return part


@pytest.mark.parametrize("k", [0, 1, 2])
def test_subdomain_hybridization_and_condensation(k):
    """Hybridization and static condensation over subdomains (Sec. 1) reproduce the conforming
    solution, with fewer multipliers than element-level hybridization and fewer global unknowns
    than the conforming system."""
    p, D = two_level(k, nx=2, ny=2, nzc=2, nzf=2)
    part = block_partition(D, p)
    u_c = D.conforming_solve()
    u_s, lam_s, H_s = D.subdomain_hybridized_solve(part)
    assert np.linalg.norm(u_s - u_c) <= 1e-10 * np.linalg.norm(u_c)
    assert 0 < lam_s.size < D.n_lambda
    u_sc, S = D.subdomain_condensed_solve(part)
    assert np.linalg.norm(u_sc - u_c) <= 1e-10 * np.linalg.norm(u_c)
    assert 0 < S.shape[0] < D.P.shape[1]
    # one subdomain per element is element-level hybridization
    u_e, lam_e, _ = D.subdomain_hybridized_solve(np.arange(D.E))
    assert lam_e.size == D.n_lambda
    assert np.linalg.norm(u_e - u_c) <= 1e-10 * np.linalg.norm(u_c)
