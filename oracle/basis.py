"""Reference RT_k basis on the unit cube (oracle; test infrastructure only).

The paper fixes the space (broken Raviart-Thomas RT_k on hexahedra, Sec. 6,
Fig. 5.1) but not its basis. Reading: a nodal tensor-product basis.
The x-component functions are L^c_a(x) L^o_b(y) L^o_c(z), with L^c the
Lagrange polynomials on the k+2 Gauss-Lobatto nodes (degree k+1; the end nodes
0 and 1 sit on the faces) and L^o those on the k+1 Gauss-Legendre nodes
(degree k); y and z components are the cyclic analogues. The dof of a function
is the value of its one non-zero reference component at its node, so the basis
is dual to its dofs.

Local dof order (interior dofs first, the 2x2 block form of Sec. 5):
  interior : x-comp (a=1..k, b, c) a fastest, then y-comp (a, b=1..k, c), then z-comp (a, b, c=1..k)
  faces    : x=0, x=1, y=0, y=1, z=0, z=1; within a face the two tangential node
             indices are lexicographic, the lower axis fastest.
"""
from __future__ import annotations

import numpy as np

from .quadrature import gauss_legendre, gauss_lobatto


def lagrange(nodes, x):
    """Values V[p, a] = L_a(x_p) and derivatives dV of the Lagrange polynomials on `nodes`."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    m = nodes.size
    V = np.ones((x.size, m))
    dV = np.zeros((x.size, m))
    for a in range(m):
        for b in range(m):
            if b == a:
                continue
            V[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
        # product rule: sum over the dropped factor
        for d in range(m):
            if d == a:
                continue
            t = np.full(x.size, 1.0 / (nodes[a] - nodes[d]))
            for b in range(m):
                if b == a or b == d:
                    continue
                t *= (x - nodes[b]) / (nodes[a] - nodes[b])
            dV[:, a] += t
    return V, dV


class RTBasis:
    """Nodal RT_k basis on [0,1]^3 with the dof order of the module docstring."""

    def __init__(self, k: int):
        if k < 0:
            raise ValueError("order k >= 0")
        self.k = k
        self.closed, _ = gauss_lobatto(k + 2)
        self.open, _ = gauss_legendre(k + 1)
        self.n_interior = 3 * k * (k + 1) ** 2
        self.n_face_nodes = (k + 1) ** 2
        self.n = self.n_interior + 6 * self.n_face_nodes
        dofs = []                                          # (component, (a, b, c)) node indices
        for comp in range(3):
            rng = [range(k + 1)] * 3
            rng = list(rng)
            rng[comp] = range(1, k + 1)
            for c in rng[2]:
                for b in rng[1]:
                    for a in rng[0]:
                        dofs.append((comp, (a, b, c)))
        for face in range(6):
            comp, side = face // 2, face % 2
            t = [d for d in range(3) if d != comp]        # tangential axes, lower first
            for s1 in range(k + 1):
                for s0 in range(k + 1):
                    idx = [0, 0, 0]
                    idx[comp] = 0 if side == 0 else k + 1
                    idx[t[0]] = s0
                    idx[t[1]] = s1
                    dofs.append((comp, tuple(idx)))
        assert len(dofs) == self.n
        self.dofs = dofs
        self.face_of_dof = np.full(self.n, -1)
        self.face_node_of_dof = np.full(self.n, -1)
        for f in range(6):
            for m in range(self.n_face_nodes):
                i = self.n_interior + f * self.n_face_nodes + m
                self.face_of_dof[i] = f
                self.face_node_of_dof[i] = m

    def node(self, i):
        """Reference position of dof i."""
        comp, idx = self.dofs[i]
        return np.array([self.closed[idx[d]] if d == comp else self.open[idx[d]] for d in range(3)])

    def eval(self, pts):
        """Values (P, n, 3) and reference divergences (P, n) at points pts (P, 3)."""
        pts = np.atleast_2d(np.asarray(pts, dtype=np.float64))
        Vc, dVc, Vo = [], [], []
        for d in range(3):
            v, dv = lagrange(self.closed, pts[:, d])
            Vc.append(v)
            dVc.append(dv)
            Vo.append(lagrange(self.open, pts[:, d])[0])
        P = pts.shape[0]
        val = np.zeros((P, self.n, 3))
        div = np.zeros((P, self.n))
        for i, (comp, idx) in enumerate(self.dofs):
            f = np.ones(P)
            g = np.ones(P)
            for d in range(3):
                if d == comp:
                    f = f * Vc[d][:, idx[d]]
                    g = g * dVc[d][:, idx[d]]
                else:
                    f = f * Vo[d][:, idx[d]]
                    g = g * Vo[d][:, idx[d]]
            val[:, i, comp] = f
            div[:, i] = g
        return val, div
