"""Element matrices through the Piola map (oracle; test infrastructure only).

Local forms (Sec. 2.1): a_T(u, v) = (alpha u, v)_T + (beta div u, div v)_T with
alpha the mass and beta the divergence coefficient (the paper's eq. 3.3 writes
the same form with the two names swapped; this code names the mass coefficient
alpha). Functions live on the physical cell x = X(xi), X trilinear in the 8
corner vertices, and come from reference RT_k functions by the contravariant
Piola map u = J u_hat / det J, for which div u = div_hat u_hat / det J.
Integrals use dx = det J d(xi) and the (k+2)^3-point tensor Gauss-Legendre rule.
"""
from __future__ import annotations

import numpy as np

from .basis import RTBasis
from .quadrature import gauss_legendre


class MeshError(ValueError):
    pass


def trilinear_jacobian(X8, xi):
    """J[:, d] = dX/dxi_d of the trilinear map with corners X8 (corner s + 2t + 4u), at xi."""
    J = np.zeros((3, 3))
    for c in range(8):
        s = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
        for d in range(3):
            g = 1.0
            for a in range(3):
                if a == d:
                    g *= 1.0 if s[a] else -1.0
                else:
                    g *= xi[a] if s[a] else 1.0 - xi[a]
            J[:, d] += X8[c] * g
    return J


def trilinear_map(X8, xi):
    x = np.zeros(3)
    for c in range(8):
        s = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
        N = 1.0
        for a in range(3):
            N *= xi[a] if s[a] else 1.0 - xi[a]
        x += X8[c] * N
    return x


class ElementIntegrator:
    """Quadrature points and basis tables for one order k."""

    def __init__(self, k: int, nq1d: int | None = None):
        self.k = k
        self.basis = RTBasis(k)
        q = k + 2 if nq1d is None else nq1d
        x, w = gauss_legendre(q)
        pts, wts = [], []
        for c in range(q):
            for b in range(q):
                for a in range(q):
                    pts.append((x[a], x[b], x[c]))
                    wts.append(w[a] * w[b] * w[c])
        self.pts = np.array(pts)
        self.wts = np.array(wts)
        self.val, self.div = self.basis.eval(self.pts)     # (nq, n, 3), (nq, n)
        # gradients of the 8 trilinear shape functions at the points: dN[q, corner, d]
        self.dN = np.zeros((self.pts.shape[0], 8, 3))
        for c in range(8):
            s = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
            for d in range(3):
                g = np.ones(self.pts.shape[0])
                for a in range(3):
                    if a == d:
                        g = g * (1.0 if s[a] else -1.0)
                    else:
                        g = g * (self.pts[:, a] if s[a] else 1.0 - self.pts[:, a])
                self.dN[:, c, d] = g

    def matrices(self, X8, alpha, beta):
        """A_T = (alpha u_i, u_j)_T + (beta div u_i, div u_j)_T and the unit mass M_T = (u_i, u_j)_T."""
        J = np.einsum("ci,qcd->qid", X8, self.dN)            # J[q][:, d] = dX/dxi_d at point q
        detJ = np.linalg.det(J)
        if not np.all(detJ > 0.0):
            raise MeshError(f"det J = {detJ.min()} <= 0")
        # the map must be orientation-preserving on the whole cell, not only at the points of
        # the rule: det J of a trilinear map can change sign between the quadrature points and
        # the corners (a corner folded inwards), so the 8 corners are checked as well
        dc = self.corner_detJ(X8)
        if not np.all(dc > 0.0):
            raise MeshError(f"det J = {dc.min()} <= 0 at a corner")
        u = np.einsum("qnd,qid->qni", self.val, J) / detJ[:, None, None]   # Piola: J u_hat / det J
        dv = self.div / detJ[:, None]                                        # div_hat u_hat / det J
        dx = self.wts * detJ
        M = np.einsum("q,qni,qmi->nm", dx, u, u)
        A = alpha * M + beta * np.einsum("q,qn,qm->nm", dx, dv, dv)
        return A, M

    def corner_detJ(self, X8):
        return np.array([np.linalg.det(trilinear_jacobian(X8, np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], float)))
                         for c in range(8)])
