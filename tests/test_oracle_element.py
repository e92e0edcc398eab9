"""Pins for the oracle's element matrices (CPU only)."""
import numpy as np
import pytest

from oracle.element import ElementIntegrator, MeshError, trilinear_jacobian, trilinear_map


def cube(h, origin=(0.0, 0.0, 0.0)):
    o = np.array(origin)
    return np.array([o + h * np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], float) for c in range(8)])


@pytest.mark.parametrize("h,alpha,beta", [(1.0, 1.0, 1.0), (0.25, 2.0, 0.5), (0.1, 3.7, 1e3)])
def test_rt0_cube_closed_form(h, alpha, beta):
    """Axis-aligned cube of side h, RT_0 (x0,x1,y0,y1,z0,z1):
    A = (alpha/h) blockdiag_3([[1/3,1/6],[1/6,1/3]]) + (beta/h^3) d d^T, d = (-1,1,-1,1,-1,1)."""
    A, M = ElementIntegrator(0).matrices(cube(h, (0.3, 0.1, 0.2)), alpha, beta)
    blk = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    Mref = np.kron(np.eye(3), blk) / h
    d = np.array([-1.0, 1, -1, 1, -1, 1])
    Aref = alpha * Mref + beta / h**3 * np.outer(d, d)
    assert np.allclose(A, Aref, rtol=1e-14, atol=1e-14 * np.abs(Aref).max())
    assert np.allclose(M, Mref, rtol=1e-14, atol=1e-14 * np.abs(Mref).max())


def test_jacobian_matches_finite_difference():
    rng = np.random.default_rng(1)
    X8 = cube(1.0) + 0.15 * rng.standard_normal((8, 3))
    xi = np.array([0.3, 0.6, 0.2])
    J = trilinear_jacobian(X8, xi)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (trilinear_map(X8, xi + e) - trilinear_map(X8, xi - e)) / (2 * h)
        assert np.allclose(J[:, d], fd, atol=1e-9)
    integ = ElementIntegrator(1)
    Jq = np.einsum("ci,qcd->qid", X8, integ.dN)
    for q in (0, 5, 26):
        assert np.allclose(Jq[q], trilinear_jacobian(X8, integ.pts[q]), atol=1e-15)


@pytest.mark.parametrize("k", range(4))
def test_affine_element_rule_is_exact(k):
    """On a parallelepiped det J is constant and the integrands are polynomials of degree <= 2k+2
    per direction, so the (k+2)-point rule already equals a (k+5)-point rule."""
    S = np.array([[1.0, 0.3, -0.2], [0.1, 0.8, 0.25], [-0.15, 0.05, 1.2]])
    X8 = np.array([S @ np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], float) for c in range(8)]) * 0.5
    A1, M1 = ElementIntegrator(k).matrices(X8, 1.3, 0.7)
    A2, M2 = ElementIntegrator(k, nq1d=k + 5).matrices(X8, 1.3, 0.7)
    assert np.allclose(A1, A2, rtol=0, atol=1e-13 * np.abs(A2).max())


@pytest.mark.parametrize("k", range(4))
def test_element_matrix_spd_and_split(k):
    rng = np.random.default_rng(k)
    X8 = cube(0.2) + 0.2 * 0.2 * (rng.random((8, 3)) - 0.5)
    integ = ElementIntegrator(k)
    A, M = integ.matrices(X8, 2.0, 5.0)
    A_mass, _ = integ.matrices(X8, 1.0, 0.0)
    A_div, _ = integ.matrices(X8, 0.0, 1.0)
    assert np.allclose(A, 2.0 * A_mass + 5.0 * A_div, atol=1e-13 * np.abs(A).max())
    assert np.allclose(A_mass, M, atol=1e-15 * np.abs(M).max())
    assert np.allclose(A, A.T, atol=1e-15 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    # the divergence part has rank = dim Q_k = (k+1)^3 (div maps RT_k onto Q_k)
    assert np.linalg.matrix_rank(A_div, tol=1e-9 * np.abs(A_div).max()) == (k + 1) ** 3


def test_inverted_element_rejected():
    X8 = cube(1.0)
    X8[[0, 1]] = X8[[1, 0]]                        # swap two corners: det J < 0 somewhere
    with pytest.raises(MeshError):
        ElementIntegrator(0).matrices(X8, 1.0, 1.0)


@pytest.mark.parametrize("k", [0, 1])
def test_corner_inverted_element_rejected(k):
    """Corner (1,1,1) pulled to 0.6 (1,1,1): det J is still positive at every Gauss point
    (the rule never sees the fold) but negative at that corner, where the three edge vectors
    (-0.4, -0.4, 0.6) and permutations span a negatively oriented frame: det = -0.2. The cell
    is not a valid (orientation-preserving) image of the reference cube, so it is refused,
    as the GPU set-up refuses it."""
    integ = ElementIntegrator(k)
    X8 = cube(1.0)
    X8[7] = 0.6
    J = np.einsum("ci,qcd->qid", X8, integ.dN)
    assert np.linalg.det(J).min() > 0.0                 # invisible to the quadrature rule
    assert integ.corner_detJ(X8)[7] == pytest.approx(-0.2)
    with pytest.raises(MeshError):
        integ.matrices(X8, 1.0, 1.0)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_energy_identity_on_parallelepiped(k):
    """For linear fields u = a + B x in RT_k on a parallelepiped x = x0 + S xi (any B for k >= 1;
    B = S D S^{-1} with D diagonal for k = 0), with c the nodal
    interpolant built here from cofactors, c^T M c' = int u.u' dx and c^T K c' = |T| div u div u'.
    The integrals are evaluated directly in physical space, independently of the oracle's Piola code."""
    from oracle.basis import RTBasis
    from oracle.quadrature import gauss_legendre
    S = np.array([[1.0, 0.3, -0.2], [0.1, 0.8, 0.25], [-0.15, 0.05, 1.2]]) * 0.4
    x0 = np.array([0.2, -0.1, 0.3])
    X8 = np.array([x0 + S @ np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], float) for c in range(8)])
    detS = np.linalg.det(S)
    cof = np.array([np.cross(S[:, 1], S[:, 2]), np.cross(S[:, 2], S[:, 0]), np.cross(S[:, 0], S[:, 1])])
    b = RTBasis(k)
    rng = np.random.default_rng(7)
    if k == 0:
        fields = [(rng.standard_normal(3), S @ np.diag(rng.standard_normal(3)) @ np.linalg.inv(S)) for _ in range(3)]
    else:
        fields = [(rng.standard_normal(3), rng.standard_normal((3, 3))) for _ in range(3)]

    def interp(a, B):
        return np.array([cof[comp] @ (a + B @ (x0 + S @ b.node(i))) for i, (comp, _) in enumerate(b.dofs)])

    xg, wg = gauss_legendre(4)
    def integral(f):
        tot = 0.0
        for i in range(4):
            for j in range(4):
                for l in range(4):
                    x = x0 + S @ np.array([xg[i], xg[j], xg[l]])
                    tot += wg[i] * wg[j] * wg[l] * f(x)
        return tot * detS

    A_div, M = ElementIntegrator(k).matrices(X8, 0.0, 1.0)
    for a1, B1 in fields:
        for a2, B2 in fields:
            c1, c2 = interp(a1, B1), interp(a2, B2)
            ref = integral(lambda x: (a1 + B1 @ x) @ (a2 + B2 @ x))
            assert abs(c1 @ M @ c2 - ref) < 1e-12 * max(1.0, abs(ref))
            refd = detS * np.trace(B1) * np.trace(B2)
            assert abs(c1 @ A_div @ c2 - refd) < 1e-12 * max(1.0, abs(refd))
