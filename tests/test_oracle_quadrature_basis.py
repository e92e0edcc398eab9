"""Pins for the oracle's quadrature rules and reference RT_k basis (CPU only)."""
import numpy as np
import pytest

from oracle.basis import RTBasis, lagrange
from oracle.quadrature import gauss_legendre, gauss_lobatto


@pytest.mark.parametrize("q", range(1, 8))
def test_gauss_legendre_exact_degree(q):
    x, w = gauss_legendre(q)
    for p in range(2 * q):                       # exact up to degree 2q-1
        assert abs(w @ x**p - 1.0 / (p + 1)) < 1e-15
    assert abs(w @ x ** (2 * q) - 1.0 / (2 * q + 1)) > 1e-12     # and not beyond
    # library routine on [-1, 1]
    xl, wl = np.polynomial.legendre.leggauss(q)
    assert np.allclose(x, 0.5 * (xl + 1), atol=1e-15, rtol=0)
    assert np.allclose(w, 0.5 * wl, atol=1e-15, rtol=0)


@pytest.mark.parametrize("q", range(2, 8))
def test_gauss_lobatto_exact_degree(q):
    x, w = gauss_lobatto(q)
    assert x[0] == 0.0 and x[-1] == 1.0
    for p in range(2 * q - 2):                   # exact up to degree 2q-3
        assert abs(w @ x**p - 1.0 / (p + 1)) < 1e-15
    assert abs(w @ x ** (2 * q - 2) - 1.0 / (2 * q - 1)) > 1e-12


def test_gauss_lobatto_known_nodes():
    # 3-point Lobatto on [-1,1] is {-1, 0, 1} with weights {1/3, 4/3, 1/3}; 4-point interior +-1/sqrt(5)
    x, w = gauss_lobatto(3)
    assert np.allclose(x, [0, 0.5, 1], atol=1e-16) and np.allclose(w, [1 / 6, 2 / 3, 1 / 6], atol=1e-16)
    x, _ = gauss_lobatto(4)
    assert np.allclose(2 * x - 1, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1], atol=1e-15)


def test_lagrange_kronecker_and_derivative():
    nodes, _ = gauss_lobatto(5)
    V, dV = lagrange(nodes, nodes)
    assert np.allclose(V, np.eye(5), atol=1e-14)
    x = np.linspace(0.03, 0.97, 11)
    V, dV = lagrange(nodes, x)
    assert np.allclose(V.sum(1), 1.0, atol=1e-14)            # partition of unity
    assert np.allclose(dV.sum(1), 0.0, atol=1e-12)
    # reproduces x^3 and its derivative
    assert np.allclose(V @ nodes**3, x**3, atol=1e-14)
    assert np.allclose(dV @ nodes**3, 3 * x**2, atol=1e-12)
    h = 1e-6
    Vp, _ = lagrange(nodes, x + h)
    Vm, _ = lagrange(nodes, x - h)
    assert np.allclose((Vp - Vm) / (2 * h), dV, atol=1e-7)


@pytest.mark.parametrize("k,n,nb,ni", [(0, 6, 6, 0), (1, 36, 24, 12), (2, 108, 54, 54), (3, 240, 96, 144)])
def test_rt_counts(k, n, nb, ni):
    b = RTBasis(k)
    assert b.n == n and 6 * b.n_face_nodes == nb and b.n_interior == ni


@pytest.mark.parametrize("k", range(4))
def test_rt_basis_dual_to_dofs(k):
    """dof_i(phi_j) = delta_ij: value of dof i's component at dof i's node."""
    b = RTBasis(k)
    nodes = np.array([b.node(i) for i in range(b.n)])
    val, _ = b.eval(nodes)
    comp = np.array([c for c, _ in b.dofs])
    D = val[np.arange(b.n), :, comp]             # D[i, j] = component comp_i of phi_j at node i
    assert np.allclose(D, np.eye(b.n), atol=1e-13)


@pytest.mark.parametrize("k", range(4))
def test_rt_basis_div_and_faces(k):
    b = RTBasis(k)
    rng = np.random.default_rng(0)
    pts = rng.random((7, 3))
    val, div = b.eval(pts)
    h = 1e-6
    fd = np.zeros_like(div)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        vp, _ = b.eval(pts + e)
        vm, _ = b.eval(pts - e)
        fd += (vp[:, :, d] - vm[:, :, d]) / (2 * h)
    assert np.allclose(fd, div, atol=1e-6 * max(1, np.abs(div).max()))
    # normal trace on face (axis, side) vanishes unless the dof belongs to that face
    for f in range(6):
        axis, side = f // 2, f % 2
        p = rng.random((5, 3))
        p[:, axis] = side
        v, _ = b.eval(p)
        on = b.face_of_dof == f
        assert np.abs(v[:, ~on, axis]).max() < 1e-13
        assert np.abs(v[:, on, axis]).max() > 0.1
    # flux identity: int over face of the normal component = face GL weight of the dof's node
    _, w = gauss_legendre(k + 1)
    wf = np.array([w[a] * w[c] for c in range(k + 1) for a in range(k + 1)])
    xg, wg = gauss_legendre(k + 3)
    for f in range(6):
        axis, side = f // 2, f % 2
        t = [d for d in range(3) if d != axis]
        P, W = [], []
        for c in range(k + 3):
            for a in range(k + 3):
                pt = np.zeros(3)
                pt[axis] = side
                pt[t[0]] = xg[a]
                pt[t[1]] = xg[c]
                P.append(pt)
                W.append(wg[a] * wg[c])
        v, _ = b.eval(np.array(P))
        flux = np.array(W) @ v[:, :, axis]
        sl = slice(b.n_interior + f * b.n_face_nodes, b.n_interior + (f + 1) * b.n_face_nodes)
        assert np.allclose(flux[sl], wf, atol=1e-14)


@pytest.mark.parametrize("k", range(4))
def test_rt_divergence_lies_in_qk_with_tensor_sparsity(k):
    """The reference divergence of every RT_k function lies in Q_k (Sec. 3.2 writes the
    divergence coupling through Q_k): its values at the (k+1)^3 Gauss-Legendre nodes reproduce
    it at random points through the Lagrange basis on those nodes. The open 1-D basis is that
    Lagrange basis, so the x-component function with nodes (i0, i1, i2) has divergence
    dL^c_{i0}(x) L^o_{i1}(y) L^o_{i2}(z), which vanishes at every node (a0, a1, a2) with
    (a1, a2) != (i1, i2): at most k + 1 nonzeros per function, dL^c_{i0}(g_{a0}) there (and
    cyclically for y and z)."""
    b = RTBasis(k)
    m = k + 1
    g, _ = gauss_legendre(m)                           # the Q_k nodes of the mixed form
    A = np.array([(a0, a1, a2) for a2 in range(m) for a1 in range(m) for a0 in range(m)])
    _, Dv = b.eval(g[A])                               # Dv[r, i] = div phi_i at node A[r]
    rng = np.random.default_rng(3)
    pts = rng.random((9, 3))
    _, div = b.eval(pts)
    L = np.ones((pts.shape[0], m ** 3))
    for d in range(3):
        L *= lagrange(g, pts[:, d])[0][:, A[:, d]]
    assert np.abs(L @ Dv - div).max() <= 1e-12 * max(1.0, np.abs(div).max())
    _, dVc = lagrange(b.closed, g)                     # dVc[p, a] = dL^c_a(g_p)
    for i, (c, idx) in enumerate(b.dofs):
        expect = np.zeros(m ** 3)
        for r, a in enumerate(A):
            if all(a[d] == idx[d] for d in range(3) if d != c):
                expect[r] = dVc[a[c], idx[c]]
        assert np.count_nonzero(expect) <= m
        assert np.abs(Dv[:, i] - expect).max() <= 1e-13 * max(1.0, np.abs(expect).max()), (k, i)
