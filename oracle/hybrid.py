"""Hybridization, static condensation and the conforming reference solve (oracle; test infrastructure only).

Definitions followed (arXiv:1801.08914):
  * A_hat = blockdiag(A_T), f_hat = element loads (Sec. 2.2).
  * Traditional assembly A = P^T A_hat P, f = P^T f_hat (eq. 2.1-2.2).
  * Hybridized saddle system [A_hat C^T; C 0][x_hat; lam] = [f_hat; 0] (Thm 2.1, eq. 2.3),
    its multiplier Schur complement H lam = C A_hat^{-1} C^T lam = C A_hat^{-1} f_hat (eq. 2.4)
    and the back substitution x_hat = A_hat^{-1}(f_hat - C^T lam).
  * C from the bilinear form c(u, lam) = int_I [u.n] lam (Example 2.2), weighted by the
    multiplier / normal-trace mass M_s.
  * Essential dofs are eliminated from the element matrices (Sec. 5).
  * Static condensation S_hat = A_bb - A_bi A_ii^{-1} A_ib, S = [I; W]^T S_hat [I; W] (Sec. 3.1, eq. 3.1-3.2).

Readings where the paper is silent:
  * Dof convention: every face dof is the reference normal component along the +axis
    of the face, identically parametrised from both neighbours on a structured mesh.
    The two copies of a shared dof are therefore equal (P copies with +1; the paper's
    W = -I is the same statement for outward-oriented dofs, Sec. 3.1).
  * C row (face f, node m): +w_m on the dof of the neighbour below f along its normal
    axis, -w_m on the neighbour above; w_m the tensor Gauss-Legendre weight on the
    reference face [0,1]^2 (M_s is diagonal: Q_k x Q_k is integrated exactly).
  * Element loads f_T = M_T c_T for f = sum_j c_j u_j given in the broken RT_k basis.
  * Boundary faces carry essential normal-trace data, or (natural=True) none: the weak form
    is then posed over all of H(div) (eq. 5.1 as the soft-hard test of Sec. 6.1 states it),
    the boundary-face dofs stay unknowns of their element and carry no multiplier.
    Static condensation is only defined here with essential boundary faces (its global
    unknowns are the interior faces' dofs).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .element import ElementIntegrator, MeshError, trilinear_jacobian
from .mesh import StructuredHexMesh
from .quadrature import gauss_legendre


class NotSPDError(ValueError):
    pass


class Discretization:
    """Mesh, basis, element data and the constraint pattern of one problem."""

    def __init__(self, nx, ny, nz, order, vertices, alpha, beta, load, ess=None, nq1d=None, natural=False):
        self.k = order
        self.natural = bool(natural)
        self.mesh = StructuredHexMesh(nx, ny, nz, vertices)
        self.integ = ElementIntegrator(order, nq1d)
        self.basis = self.integ.basis
        self.n = self.basis.n
        self.nfn = self.basis.n_face_nodes
        E = self.mesh.n_elem
        self.alpha = np.asarray(alpha, dtype=np.float64).reshape(E)
        self.beta = np.asarray(beta, dtype=np.float64).reshape(E)
        self.load = np.asarray(load, dtype=np.float64).reshape(E, self.n)
        self.ess = None if ess is None else np.asarray(ess, dtype=np.float64).reshape(E, self.n)
        g, w = gauss_legendre(order + 1)
        # face weights, node m = s0 + (k+1) s1 (lower tangential axis fastest)
        self.face_w = np.array([w[s0] * w[s1] for s1 in range(order + 1) for s0 in range(order + 1)])
        self.n_lambda = self.mesh.n_interior_faces * self.nfn

    @classmethod
    def from_problem(cls, p, nq1d=None):
        return cls(p.nx, p.ny, p.nz, p.order, p.vertices, p.alpha, p.beta, p.load, p.ess, nq1d,
                   getattr(p, "natural", False))

    # ---- one element -------------------------------------------------------------------------
    def element(self, e):
        """Element matrix and load with essential dofs eliminated, and the element's block of C.

        Returns a dict with A (free x free), f (free), free / edofs (local indices), ue,
        C (rows = the element's multipliers, cols = free dofs) and lam (global multiplier ids).
        """
        X8 = self.mesh.element_vertices(e)
        A, M = self.integ.matrices(X8, self.alpha[e], self.beta[e])
        f = M @ self.load[e]
        faces = self.mesh.element_faces(e)
        b = self.basis
        is_e = np.zeros(self.n, dtype=bool)
        for a, (_, fint) in enumerate(faces):
            if fint < 0 and not self.natural:
                is_e[b.n_interior + a * self.nfn: b.n_interior + (a + 1) * self.nfn] = True
        edofs = np.nonzero(is_e)[0]
        free = np.nonzero(~is_e)[0]
        ue = np.zeros(edofs.size) if self.ess is None else self.ess[e, edofs]
        f_free = f[free] - A[np.ix_(free, edofs)] @ ue
        A_free = A[np.ix_(free, free)]
        pos = {int(d): i for i, d in enumerate(free)}
        rows, lam = [], []
        for a, (_, fint) in enumerate(faces):
            if fint < 0:
                continue
            sign = 1.0 if a % 2 == 1 else -1.0
            for m in range(self.nfn):
                r = np.zeros(free.size)
                r[pos[b.n_interior + a * self.nfn + m]] = sign * self.face_w[m]
                rows.append(r)
                lam.append(fint * self.nfn + m)
        C = np.array(rows).reshape(len(rows), free.size)
        return dict(A=A_free, A_full=A, f=f_free, f_full=f, free=free, edofs=edofs, ue=ue,
                    C=C, lam=np.array(lam, dtype=np.int64), faces=faces)

    # ---- hybridization (Thm 2.1, eq. 2.4) ------------------------------------------------------
    def element_reduced(self, e):
        """S_T = C_T A_T^{-1} C_T^T and g_T = C_T A_T^{-1} f_T for element e (dense, general products)."""
        d = self.element(e)
        try:
            L = np.linalg.cholesky(d["A"])
        except np.linalg.LinAlgError as exc:
            raise NotSPDError(f"element {e}: A_T not SPD") from exc
        X = sla.cho_solve((L, True), d["C"].T)
        d["S"] = d["C"] @ X
        d["g"] = d["C"] @ sla.cho_solve((L, True), d["f"])
        d["L"] = L
        return d

    def mixed_form_blocks(self, e):
        """Blocks of the hybridized mixed form (Sec. 3.2, eq. 3.3-3.6) for element e.

        With q = beta div u in Q_k (Lagrange basis l_a at the (k+1)^3 Gauss-Legendre nodes),
        W_ab = sum_q w_q (beta / det J) l_a l_b and B_ai = sum_q w_q (beta / det J) l_a div_hat phi_i,
        so that A_T = M_T + B^T W^{-1} B exactly (div_hat phi_i lies in Q_k) with M_T the
        alpha-weighted mass. Returns M, B (restricted to free dofs), W and the element dict."""
        d = self.element(e)
        X8 = self.mesh.element_vertices(e)
        integ = self.integ
        M, _ = integ.matrices(X8, self.alpha[e], 0.0)
        from .basis import lagrange
        g, _ = gauss_legendre(self.k + 1)
        Ls = [lagrange(g, integ.pts[:, dd])[0] for dd in range(3)]            # (nq, k+1) each
        L = np.einsum("qa,qb,qc->qcba", Ls[0], Ls[1], Ls[2]).reshape(integ.pts.shape[0], -1)
        J = np.einsum("ci,qcd->qid", X8, integ.dN)
        wgt = integ.wts * self.beta[e] / np.linalg.det(J)
        W = L.T @ (wgt[:, None] * L)
        B = L.T @ (wgt[:, None] * integ.div)
        free = d["free"]
        return M[np.ix_(free, free)], B[:, free], W, d

    def element_reduced_mixed(self, e):
        """S_T and g_T from the mixed form: [C 0] [M B^T; B -W]^{-1} [C^T; 0] (Sec. 3.2, H = H~)."""
        M, B, W, d = self.mixed_form_blocks(e)
        nf, nq = M.shape[0], W.shape[0]
        K = np.block([[M, B.T], [B, -W]])
        rhs = np.zeros((nf + nq, d["C"].shape[0] + 1))
        rhs[:nf, :-1] = d["C"].T
        rhs[:nf, -1] = d["f"]
        X = np.linalg.solve(K, rhs)[:nf]
        d["S"] = d["C"] @ X[:, :-1]
        d["g"] = d["C"] @ X[:, -1]
        return d

    def hybridize(self, elements=None):
        """Assemble H and g (eq. 2.4); keeps per-element factors for the back substitution."""
        return self._assemble_reduced(self.element_reduced, elements)

    def hybridize_mixed(self, elements=None):
        """H~ and g~ of the hybridized mixed form (Sec. 3.2, eq. 3.3-3.6), element by element
        through element_reduced_mixed; H~ = H in exact arithmetic (end of Sec. 3.2).

        Why a second route: the primal route factors A_T = alpha M + beta K, whose condition
        number grows like (beta / alpha) h^-2, and forming its entries in FP64 already rounds
        away the divergence-free structure that A_T^{-1} C_T^T depends on, so at contrast
        1e6 its S_T carries errors of order kappa(A_T) eps_64 (1e-8..1e-7, measured against
        an extended-precision evaluation in the tests). The mixed form never forms
        alpha M + beta K: its saddle matrix [M B^T; B -W] is well conditioned at any
        contrast, and its FP64 result is the accurate reference at high contrast."""
        return self._assemble_reduced(self.element_reduced_mixed, elements)

    def recover_mixed(self, lam):
        """x_hat_T of the back substitution (Thm 2.1) through the mixed form: the element saddle
        system [M B^T; B -W][x; q] = [f_T - C_T^T lam_T; 0] (eq. 3.3 with q = W^{-1} B x,
        so that M x + B^T W^{-1} B x = A_T x), essential dofs re-inserted; returns (E, n)."""
        u = np.zeros((self.mesh.n_elem, self.n))
        for e in range(self.mesh.n_elem):
            u[e] = self.recover_mixed_element(e, lam)
        return u

    def recover_mixed_element(self, e, lam):
        """recover_mixed for the single element e; returns its n dofs."""
        M, B, W, d = self.mixed_form_blocks(e)
        nf = M.shape[0]
        K = np.block([[M, B.T], [B, -W]])
        rhs = np.zeros(nf + W.shape[0])
        rhs[:nf] = d["f"] - d["C"].T @ lam[d["lam"]]
        x = np.zeros(self.n)
        x[d["free"]] = np.linalg.solve(K, rhs)[:nf]
        x[d["edofs"]] = d["ue"]
        return x

    def _assemble_reduced(self, reduce_element, elements=None):
        """Sum the element contributions S_T, g_T of reduce_element into H and g (eq. 2.4)."""
        E = self.mesh.n_elem
        elems = range(E) if elements is None else elements
        I, J, V = [], [], []
        g = np.zeros(self.n_lambda)
        self.factors = {}
        for e in elems:
            d = reduce_element(e)
            lam = d["lam"]
            if lam.size:
                I.append(np.repeat(lam, lam.size))
                J.append(np.tile(lam, lam.size))
                V.append(d["S"].ravel())
                np.add.at(g, lam, d["g"])
            self.factors[e] = d
        if I:
            H = sp.coo_matrix((np.concatenate(V), (np.concatenate(I), np.concatenate(J))),
                              shape=(self.n_lambda, self.n_lambda)).tocsr()
        else:
            H = sp.csr_matrix((self.n_lambda, self.n_lambda))
        H.sum_duplicates()
        H.sort_indices()
        return H, g

    def recover(self, lam):
        """x_hat_T = A_T^{-1}(f_T - C_T^T lam_T) with essential dofs re-inserted; returns (E, n)."""
        u = np.zeros((self.mesh.n_elem, self.n))
        for e, d in self.factors.items():
            rhs = d["f"] - d["C"].T @ lam[d["lam"]]
            u[e, d["free"]] = sla.cho_solve((d["L"], True), rhs)
            u[e, d["edofs"]] = d["ue"]
        return u

    # ---- static condensation (Sec. 3.1) --------------------------------------------------------
    def static_condense(self):
        """Assemble S (eq. 3.2, +1 copies in this dof convention) and its right-hand side.

        Global unknowns: the face dofs of interior faces, numbered like the multipliers.
        """
        if self.natural:
            raise NotImplementedError("static condensation with natural boundary faces")
        E = self.mesh.n_elem
        b = self.basis
        I, J, V = [], [], []
        rhs = np.zeros(self.n_lambda)
        self.sc = {}
        for e in range(E):
            c = self.element_condensed(e)
            gidx, Shat, r = c["gidx"], c["Shat"], c["r"]
            if gidx.size:
                I.append(np.repeat(gidx, gidx.size))
                J.append(np.tile(gidx, gidx.size))
                V.append(Shat.ravel())
                np.add.at(rhs, gidx, r)
            self.sc[e] = c
        S = sp.coo_matrix((np.concatenate(V), (np.concatenate(I), np.concatenate(J))),
                          shape=(self.n_lambda, self.n_lambda)).tocsr()
        S.sum_duplicates()
        S.sort_indices()
        return S, rhs

    def element_condensed(self, e):
        """One element's static condensation (Sec. 3.1, eq. 3.1): S_hat = A_bb - A_bi A_ii^{-1} A_ib,
        r = f_b - A_bi A_ii^{-1} f_i, and the global index of each free face dof."""
        b = self.basis
        d = self.element(e)
        free = d["free"]
        ii = np.nonzero(free < b.n_interior)[0]      # positions (within free) of interior dofs
        bb = np.nonzero(free >= b.n_interior)[0]     # positions of free face dofs
        A = d["A"]
        Aii, Aib, Abi, Abb = A[np.ix_(ii, ii)], A[np.ix_(ii, bb)], A[np.ix_(bb, ii)], A[np.ix_(bb, bb)]
        fi, fb = d["f"][ii], d["f"][bb]
        if ii.size:
            Shat = Abb - Abi @ np.linalg.solve(Aii, Aib)
            r = fb - Abi @ np.linalg.solve(Aii, fi)
        else:
            Shat, r = Abb.copy(), fb.copy()
        gidx = []
        for p in bb:
            ldof = free[p]
            a = b.face_of_dof[ldof]
            m = b.face_node_of_dof[ldof]
            gidx.append(d["faces"][a][1] * self.nfn + m)
        return dict(d=d, ii=ii, bb=bb, gidx=np.array(gidx, dtype=np.int64), Shat=Shat, r=r)

    def sc_recover(self, ub):
        """u_i = A_ii^{-1}(f_i - A_ib u_b) per element; face dofs copied from ub, e-dofs from ue."""
        u = np.zeros((self.mesh.n_elem, self.n))
        for e, s in self.sc.items():
            d = s["d"]
            free, ii, bb = d["free"], s["ii"], s["bb"]
            A = d["A"]
            u_b = ub[s["gidx"]]
            if ii.size:
                u_i = np.linalg.solve(A[np.ix_(ii, ii)], d["f"][ii] - A[np.ix_(ii, bb)] @ u_b)
                u[e, free[ii]] = u_i
            u[e, free[bb]] = u_b
            u[e, d["edofs"]] = d["ue"]
        return u

    # ---- conforming assembly (eq. 2.1-2.2) -----------------------------------------------------
    def conforming_solve(self):
        """Solve P^T A_hat P x = P^T f_hat with essential face dofs fixed (natural: all face dofs
        unknown); returns P x as (E, n)."""
        E = self.mesh.n_elem
        b = self.basis
        nfd = self.mesh.n_faces * self.nfn
        ng = nfd + E * b.n_interior
        I, J, V = [], [], []
        f = np.zeros(ng)
        ess_val = np.zeros(ng)
        is_ess = np.zeros(ng, dtype=bool)
        P = np.zeros((E, self.n), dtype=np.int64)
        for e in range(E):
            X8 = self.mesh.element_vertices(e)
            A, M = self.integ.matrices(X8, self.alpha[e], self.beta[e])
            fe = M @ self.load[e]
            faces = self.mesh.element_faces(e)
            gl = np.empty(self.n, dtype=np.int64)
            gl[:b.n_interior] = nfd + e * b.n_interior + np.arange(b.n_interior)
            for a, (fid, fint) in enumerate(faces):
                sl = slice(b.n_interior + a * self.nfn, b.n_interior + (a + 1) * self.nfn)
                gl[sl] = fid * self.nfn + np.arange(self.nfn)
                if fint < 0 and not self.natural:
                    is_ess[gl[sl]] = True
                    if self.ess is not None:
                        ess_val[gl[sl]] = self.ess[e, sl]
            P[e] = gl
            I.append(np.repeat(gl, self.n))
            J.append(np.tile(gl, self.n))
            V.append(A.ravel())
            np.add.at(f, gl, fe)
        A = sp.coo_matrix((np.concatenate(V), (np.concatenate(I), np.concatenate(J))), shape=(ng, ng)).tocsr()
        used = np.zeros(ng, dtype=bool)
        used[P.ravel()] = True
        fr = np.nonzero(used & ~is_ess)[0]
        es = np.nonzero(is_ess)[0]
        rhs = f[fr] - A[fr][:, es] @ ess_val[es]
        x = np.zeros(ng)
        x[es] = ess_val[es]
        x[fr] = spla.spsolve(A[fr][:, fr].tocsc(), rhs)
        return x[P]

    # ---- dense saddle-point system (eq. 2.3), tiny meshes only --------------------------------
    def saddle_solve(self):
        E = self.mesh.n_elem
        blocks, offs = [], [0]
        for e in range(E):
            d = self.element(e)
            blocks.append(d)
            offs.append(offs[-1] + d["free"].size)
        nh = offs[-1]
        K = np.zeros((nh + self.n_lambda, nh + self.n_lambda))
        rhs = np.zeros(nh + self.n_lambda)
        for e, d in enumerate(blocks):
            s = slice(offs[e], offs[e + 1])
            K[s, s] = d["A"]
            rhs[s] = d["f"]
            for r, lidx in enumerate(d["lam"]):
                K[nh + lidx, s] = d["C"][r]
                K[s, nh + lidx] = d["C"][r]
        sol = np.linalg.solve(K, rhs)
        u = np.zeros((E, self.n))
        for e, d in enumerate(blocks):
            u[e, d["free"]] = sol[offs[e]:offs[e + 1]]
            u[e, d["edofs"]] = d["ue"]
        return u, sol[nh:]

    # ---- constraint residual C x_hat (second block row of eq. 2.3) ----------------------------
    def constraint_residual(self, u):
        """(C u)_(f,m) = w_m (u_low - u_high) on every interior face node."""
        r = np.zeros(self.n_lambda)
        b = self.basis
        for e in range(self.mesh.n_elem):
            for a, (_, fint) in enumerate(self.mesh.element_faces(e)):
                if fint < 0:
                    continue
                sign = 1.0 if a % 2 == 1 else -1.0
                sl = slice(b.n_interior + a * self.nfn, b.n_interior + (a + 1) * self.nfn)
                r[fint * self.nfn: (fint + 1) * self.nfn] += sign * self.face_w * u[e, sl]
        return r


# ---- reduced-system solvers --------------------------------------------------------------------
def solve_dense(H, g):
    """Dense Cholesky solve of the SPD reduced system (tiny problems)."""
    Hd = H.toarray() if sp.issparse(H) else np.asarray(H)
    c = sla.cho_factor(Hd, lower=True)
    return sla.cho_solve(c, g)


def pcg_diag(H, g, rtol=1e-12, maxit=100000, x0=None):
    """Preconditioned CG with the diagonal of H, x0 = 0, stop when ||r||_2 <= rtol ||r_0||_2 (Sec. 6.1)."""
    d = H.diagonal()
    x = np.zeros_like(g) if x0 is None else x0.copy()
    r = g - H @ x
    r0 = np.linalg.norm(r)
    if r0 == 0.0:
        return x, 0, 0.0
    z = r / d
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = H @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        rn = np.linalg.norm(r)
        if rn <= rtol * r0:
            return x, it, rn / r0
        z = r / d
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, np.linalg.norm(r) / r0


def solve_sparse_direct(H, g):
    return spla.spsolve(H.tocsc(), g)
