"""Hybridization with master / slave interface dofs and at subdomain level (oracle; test
infrastructure only: nothing on the product path imports it).

Definitions followed (arXiv:1801.08914):
  * Example 2.1: the broken dofs split into interior (i), master (m) and slave (s) dofs; the
    slaves follow the masters through W_sm, P = [I_i 0; 0 I_m; 0 W_sm] maps the conforming
    unknowns (i and m) to the broken space, and C = [0 -W_sm I_s] (one multiplier per slave)
    has C P = 0 and ker C = range P.
  * Thm 2.1 (general equivalence): the hybridized system H lam = C A_hat^{-1} C^T lam =
    C A_hat^{-1} f_hat with x_hat = A_hat^{-1}(f_hat - C^T lam) gives x_hat = P x for the x of
    P^T A_hat P x = P^T f_hat (eq. 2.1-2.4); H is the sum of the element terms
    C_T A_T^{-1} C_T^T (A_hat block diagonal).
  * Sec. 1: the same eliminations over subdomains (unions of elements) instead of elements:
    inside a subdomain the slaves whose master lies in it are eliminated by assembly, and only
    the constraints across subdomains keep a multiplier (hybridization), or only the unknowns
    shared by several subdomains stay global (static condensation, Sec. 3.1).
  * Fig. 5.1 (right): a non-conforming mesh face, whose RT dofs are matched to the other side.

Readings where the paper is silent:
  * Mesh: the two-level mesh of inputs.two_level_problem. Every face dof is the reference
    normal component along the +axis (as in oracle.hybrid), elements of both blocks share the
    axis orientation, and every boundary face is natural (its dofs are interior dofs here).
  * Conforming faces: the dofs of the element below the face (along its axis) are the masters,
    those of the element above the slaves, W = I node by node.
  * Non-conforming faces: the coarse cell's top-face dofs are the masters; the bottom-face
    dofs of the four fine cells on it are the slaves. A face dof is the flux density of the
    normal component per unit reference face area (the Piola map keeps fluxes), the fine face
    (sub-square (a, b) of the coarse one) is the coarse face's parametrisation restricted to
    [a/2, (a+1)/2] x [b/2, (b+1)/2], so one unit of fine reference area is a quarter of the
    coarse one: slave (node (p, q) of sub-face (a, b)) = 1/4 sum over the coarse nodes (r, t)
    of L_r((a + g_p) / 2) L_t((b + g_q) / 2) master(r, t), with L the Lagrange basis on the
    k+1 Gauss-Legendre nodes g (the normal trace is in Q_k on both faces).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import lagrange
from .element import ElementIntegrator
from .quadrature import gauss_legendre


class TwoLevelDiscretization:
    """Element matrices, loads and the master / slave relations of a TwoLevelProblem."""

    def __init__(self, prob, nq1d=None):
        self.p = prob
        self.k = prob.order
        self.integ = ElementIntegrator(self.k, nq1d)
        b = self.basis = self.integ.basis
        self.n = b.n
        self.nfn = b.n_face_nodes
        nx, ny, nzc, nzf, mx, my = prob.nx, prob.ny, prob.nzc, prob.nzf, prob.mx, prob.my
        self.Ec, self.E = prob.n_coarse, prob.n_elem
        cv = prob.coarse_vertices.reshape(nzc + 1, ny + 1, nx + 1, 3)
        fv = prob.fine_vertices.reshape(nzf + 1, my + 1, mx + 1, 3)
        self.X8 = []
        self.cell = []                                   # (block, i, j, l)
        for blk, (V, ax, ay, az) in enumerate(((cv, nx, ny, nzc), (fv, mx, my, nzf))):
            for l in range(az):
                for j in range(ay):
                    for i in range(ax):
                        self.X8.append(np.array([V[l + u, j + t, i + s] for u in (0, 1) for t in (0, 1)
                                                 for s in (0, 1)]))
                        self.cell.append((blk, i, j, l))
        self.A, self.f = [], []
        for e in range(self.E):
            A, M = self.integ.matrices(self.X8[e], prob.alpha[e], prob.beta[e])
            self.A.append(A)
            self.f.append(M @ prob.load[e])
        self._relations()

    # ---- dof numbering ----------------------------------------------------------------------
    def elem_index(self, blk, i, j, l):
        p = self.p
        if blk == 0:
            return i + p.nx * (j + p.ny * l)
        return self.Ec + i + p.mx * (j + p.my * l)

    def face_dof(self, e, face, m):
        """Broken (global) index of node m of local face `face` (x0 x1 y0 y1 z0 z1) of element e."""
        return e * self.n + self.basis.n_interior + face * self.nfn + m

    def _relations(self):
        """Slave -> (master dofs, weights) for every interior face (Example 2.1's W_sm)."""
        p, k, nfn = self.p, self.k, self.nfn
        rows = []                                        # (slave, [(master, w), ...])
        for blk, (ax, ay, az) in enumerate(((p.nx, p.ny, p.nzc), (p.mx, p.my, p.nzf))):
            dims = (ax, ay, az)
            for l in range(az):
                for j in range(ay):
                    for i in range(ax):
                        lo = self.elem_index(blk, i, j, l)
                        pos = [i, j, l]
                        for d in range(3):
                            if pos[d] + 1 >= dims[d]:
                                continue
                            up = list(pos)
                            up[d] += 1
                            hi = self.elem_index(blk, *up)
                            for m in range(nfn):
                                rows.append((self.face_dof(hi, 2 * d, m), [(self.face_dof(lo, 2 * d + 1, m), 1.0)]))
        g, _ = gauss_legendre(k + 1)
        r = 2 if p.refine else 1
        for j in range(p.ny):
            for i in range(p.nx):
                ec = self.elem_index(0, i, j, p.nzc - 1)
                for b_ in range(r):
                    for a_ in range(r):
                        ef = self.elem_index(1, r * i + a_, r * j + b_, 0)
                        if r == 1:
                            for m in range(nfn):
                                rows.append((self.face_dof(ef, 4, m), [(self.face_dof(ec, 5, m), 1.0)]))
                            continue
                        # coarse-face parameters of the fine nodes (lower tangential axis x fastest)
                        Ls = lagrange(g, (a_ + g) / 2.0)[0]     # Ls[p, r] = L_r((a + g_p) / 2)
                        Lt = lagrange(g, (b_ + g) / 2.0)[0]
                        for q in range(k + 1):
                            for p_ in range(k + 1):
                                ms = []
                                for t in range(k + 1):
                                    for rr in range(k + 1):
                                        ms.append((self.face_dof(ec, 5, rr + (k + 1) * t),
                                                   0.25 * Ls[p_, rr] * Lt[q, t]))
                                rows.append((self.face_dof(ef, 4, p_ + (k + 1) * q), ms))
        rows.sort(key=lambda x: x[0])
        self.slaves = np.array([s for s, _ in rows], dtype=np.int64)
        self.relations = rows
        N = self.E * self.n
        self.N = N
        masters = sorted({m for _, ms in rows for m, _ in ms})
        self.masters = np.array(masters, dtype=np.int64)
        is_s = np.zeros(N, dtype=bool)
        is_s[self.slaves] = True
        assert not is_s[self.masters].any(), "a dof is both master and slave"
        self.kept = np.nonzero(~is_s)[0]                # columns of P: the i and m dofs
        col = np.full(N, -1, dtype=np.int64)
        col[self.kept] = np.arange(self.kept.size)
        self.col = col
        # P: identity on kept dofs, W_sm on slaves; C = [0 -W_sm I_s] (rows = slaves)
        PI, PJ, PV = list(self.kept), list(range(self.kept.size)), [1.0] * self.kept.size
        CI, CJ, CV = [], [], []
        for r_, (s, ms) in enumerate(rows):
            CI.append(r_)
            CJ.append(s)
            CV.append(1.0)
            for m, w in ms:
                PI.append(s)
                PJ.append(col[m])
                PV.append(w)
                CI.append(r_)
                CJ.append(m)
                CV.append(-w)
        self.P = sp.csr_matrix((PV, (PI, PJ)), shape=(N, self.kept.size))
        self.C = sp.csr_matrix((CV, (CI, CJ)), shape=(len(rows), N))
        self.n_lambda = len(rows)

    # ---- broken operators -------------------------------------------------------------------
    def A_hat(self):
        return sp.block_diag([sp.csr_matrix(a) for a in self.A], format="csr")

    def f_hat(self):
        return np.concatenate(self.f)

    # ---- conforming solve (eq. 2.1-2.2) -------------------------------------------------------
    def conforming_solve(self):
        """x of P^T A_hat P x = P^T f_hat, returned as the broken vector P x."""
        K = (self.P.T @ self.A_hat() @ self.P).tocsc()
        x = spla.spsolve(K, self.P.T @ self.f_hat())
        return self.P @ x

    # ---- element-level hybridization (Thm 2.1, eq. 2.4) ----------------------------------------
    def hybridize(self):
        """H = sum_T C_T A_T^{-1} C_T^T and g = sum_T C_T A_T^{-1} f_T (dense, small meshes)."""
        C = self.C.tocsc()
        H = np.zeros((self.n_lambda, self.n_lambda))
        g = np.zeros(self.n_lambda)
        self.chol = []
        for e in range(self.E):
            CT = C[:, e * self.n:(e + 1) * self.n]
            L = sla.cho_factor(self.A[e], lower=True)
            self.chol.append(L)
            rows = np.unique(CT.nonzero()[0])
            if rows.size == 0:
                continue
            Ct = CT[rows].toarray()
            X = sla.cho_solve(L, Ct.T)
            H[np.ix_(rows, rows)] += Ct @ X
            g[rows] += Ct @ sla.cho_solve(L, self.f[e])
        return H, g

    def recover(self, lam):
        """x_hat_T = A_T^{-1}(f_T - C_T^T lam) for every element; the broken vector."""
        C = self.C.tocsc()
        u = np.zeros(self.N)
        for e in range(self.E):
            CT = C[:, e * self.n:(e + 1) * self.n]
            u[e * self.n:(e + 1) * self.n] = sla.cho_solve(self.chol[e], self.f[e] - CT.T @ lam)
        return u

    def hybridized_solve(self):
        H, g = self.hybridize()
        lam = np.linalg.solve(H, g)
        return self.recover(lam), lam, H

    # ---- subdomain level (Sec. 1) ---------------------------------------------------------------
    def _subdomain_parts(self, part):
        """Per subdomain: its broken dofs, its local P_D (slaves with a master inside eliminated),
        and the cross-subdomain relations (their slave or masters inside)."""
        part = np.asarray(part)
        owner = np.repeat(part, self.n)                  # subdomain of every broken dof
        subs = []
        for D in np.unique(part):
            dofs = np.nonzero(owner == D)[0]
            loc = np.full(self.N, -1, dtype=np.int64)
            loc[dofs] = np.arange(dofs.size)
            internal = [(s, ms) for s, ms in self.relations
                        if owner[s] == D and all(owner[m] == D for m, _ in ms)]
            elim = np.zeros(dofs.size, dtype=bool)
            for s, _ in internal:
                elim[loc[s]] = True
            keep = np.nonzero(~elim)[0]
            kcol = np.full(dofs.size, -1, dtype=np.int64)
            kcol[keep] = np.arange(keep.size)
            PI, PJ, PV = list(keep), list(range(keep.size)), [1.0] * keep.size
            for s, ms in internal:
                for m, w in ms:
                    PI.append(loc[s])
                    PJ.append(kcol[loc[m]])
                    PV.append(w)
            PD = sp.csr_matrix((PV, (PI, PJ)), shape=(dofs.size, keep.size))
            elems = np.nonzero(part == D)[0]
            AD = sp.block_diag([sp.csr_matrix(self.A[e]) for e in elems], format="csr")
            fD = np.concatenate([self.f[e] for e in elems])
            subs.append(dict(D=D, dofs=dofs, loc=loc, kcol=kcol, P=PD, A=(PD.T @ AD @ PD).toarray(),
                             f=PD.T @ fD))
        return subs, owner

    def subdomain_hybridized_solve(self, part):
        """Hybridization over subdomains: multipliers only for the relations across subdomains."""
        subs, owner = self._subdomain_parts(part)
        cross = [(s, ms) for s, ms in self.relations if any(owner[m] != owner[s] for m, _ in ms)]
        nl = len(cross)
        index = {int(sd["D"]): i for i, sd in enumerate(subs)}
        # C_D: rows = cross relations, columns = the subdomain's kept unknowns
        CDs = [np.zeros((nl, sd["P"].shape[1])) for sd in subs]
        for r_, (s, ms) in enumerate(cross):
            sd = index[int(owner[s])]
            CDs[sd][r_, subs[sd]["kcol"][subs[sd]["loc"][s]]] += 1.0
            for m, w in ms:
                dm = index[int(owner[m])]
                CDs[dm][r_, subs[dm]["kcol"][subs[dm]["loc"][m]]] -= w
        H = np.zeros((nl, nl))
        g = np.zeros(nl)
        facs = []
        for sd, CD in zip(subs, CDs):
            L = sla.cho_factor(sd["A"], lower=True)
            facs.append(L)
            H += CD @ sla.cho_solve(L, CD.T)
            g += CD @ sla.cho_solve(L, sd["f"])
        lam = np.linalg.solve(H, g)
        u = np.zeros(self.N)
        for sd, CD, L in zip(subs, CDs, facs):
            y = sla.cho_solve(L, sd["f"] - CD.T @ lam)
            u[sd["dofs"]] = sd["P"] @ y
        return u, lam, H

    def subdomain_condensed_solve(self, part):
        """Static condensation over subdomains (Sec. 3.1 with subdomains as the blocks): the
        conforming unknowns (columns of P) touching one subdomain only are eliminated inside
        it; the Schur complement on those touching several is assembled subdomain by
        subdomain, solved, and the eliminated unknowns recovered."""
        part = np.asarray(part)
        owner = np.repeat(part, self.n)
        Pc = self.P.tocsc()
        touch = []                                       # subdomains touched by each column
        for j in range(Pc.shape[1]):
            rows = Pc.indices[Pc.indptr[j]:Pc.indptr[j + 1]]
            touch.append(set(owner[rows].tolist()))
        gamma = np.array([j for j, t in enumerate(touch) if len(t) > 1], dtype=np.int64)
        gpos = np.full(Pc.shape[1], -1, dtype=np.int64)
        gpos[gamma] = np.arange(gamma.size)
        S = np.zeros((gamma.size, gamma.size))
        r = np.zeros(gamma.size)
        blocks = []
        for D in np.unique(part):
            dofs = np.nonzero(owner == D)[0]
            elems = np.nonzero(part == D)[0]
            PD = self.P[dofs]                            # rows of P in D
            cols = np.unique(PD.nonzero()[1])
            inner = np.array([c for c in cols if gpos[c] < 0], dtype=np.int64)
            bnd = np.array([c for c in cols if gpos[c] >= 0], dtype=np.int64)
            AD = sp.block_diag([sp.csr_matrix(self.A[e]) for e in elems], format="csr")
            fD = np.concatenate([self.f[e] for e in elems])
            KD = (PD[:, cols].T @ AD @ PD[:, cols]).toarray()
            FD = PD[:, cols].T @ fD
            ii = np.searchsorted(cols, inner)
            bb = np.searchsorted(cols, bnd)
            Kii, Kib, Kbb = KD[np.ix_(ii, ii)], KD[np.ix_(ii, bb)], KD[np.ix_(bb, bb)]
            if ii.size:
                L = sla.cho_factor(Kii, lower=True)
                Sd = Kbb - Kib.T @ sla.cho_solve(L, Kib)
                rd = FD[bb] - Kib.T @ sla.cho_solve(L, FD[ii])
            else:
                L, Sd, rd = None, Kbb, FD[bb]
            S[np.ix_(gpos[bnd], gpos[bnd])] += Sd
            r[gpos[bnd]] += rd
            blocks.append((inner, bnd, L, Kib, FD[ii]))
        xg = np.linalg.solve(S, r)
        x = np.zeros(Pc.shape[1])
        x[gamma] = xg
        for inner, bnd, L, Kib, Fi in blocks:
            if inner.size:
                x[inner] = sla.cho_solve(L, Fi - Kib @ xg[gpos[bnd]])
        return self.P @ x, S
