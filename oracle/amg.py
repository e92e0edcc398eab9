"""Aggregation multigrid preconditioner for the reduced system H (oracle; test infrastructure
only: nothing on the product path imports this module).

Sec. 4 shows that H = C A^{-1} C^T is spectrally equivalent to a mesh-dependent H^1-type norm
of the face functions, so an H^1-type algebraic multigrid preconditions it with iteration
counts independent of the mesh size; Sec. 6.1 uses BoomerAMG for this. The paper does not
define the multigrid itself; this is the method the GPU path implements, written out plainly:

* Aggregates: every interior face belongs to the 2 x 2 x 2 block of cells (i // 2, j // 2,
  l // 2), (i, j, l) being the face's grid position (its plane index along its normal axis,
  the cell indices across it). All face nodes of an aggregate share one coarse unknown: the
  tentative prolongation P_0 is 1 at (face node, its face's block), 0 elsewhere (the near-null
  vector of an H^1-type operator is the constant). Coarser levels aggregate the block grid the
  same way (point (I, J, K) -> (I // 2, J // 2, K // 2)) until at most `coarsest` unknowns
  remain or the grid is a single point.
* Coarse operators: Galerkin, A_{l+1} = P_l^T A_l P_l. A coarse unknown whose aggregate holds
  no face (possible on grids of one cell across) gets the equation x = 0 (diagonal 1).
* Smoother: Chebyshev iteration of degree `degree` for the Jacobi-preconditioned operator
  D^{-1} A on the interval [lmax / ratio, lmax], lmax = 1.1 x the estimate of the largest
  eigenvalue from `power_steps` steps of the power iteration in the D inner product started
  from s_i = ((7919 i) mod 101) / 101 - 1/2 (the Rayleigh quotient v.Av / v.Dv of the last
  iterate). The same polynomial before and after the coarse correction, so the V-cycle is a
  symmetric positive definite preconditioner.
* Coarsest level: exact solve (dense inverse).
* V-cycle: pre-smoothing from zero, residual, restriction P^T, coarse V-cycle, prolongation
  P, post-smoothing.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def face_positions(nx, ny, nz):
    """(axis, i, j, l) of every interior face in the multiplier face order (axis x, y, z, then
    plane fastest, then the cell indices across, lower axis first), (i, j, l) the face's grid
    position: along its axis the plane index, across it the cell indices."""
    dims = (nx, ny, nz)
    out = []
    for d in range(3):
        a_dim, b_dim = [dims[x] for x in range(3) if x != d]
        for b in range(b_dim):
            for a in range(a_dim):
                for plane in range(1, dims[d]):
                    pos = [0, 0, 0]
                    pos[d] = plane
                    across = [x for x in range(3) if x != d]
                    pos[across[0]] = a
                    pos[across[1]] = b
                    out.append((d, pos[0], pos[1], pos[2]))
    return out


def coarse_dims(dims):
    return tuple((n + 1) // 2 for n in dims)


def face_aggregates(nx, ny, nz):
    """Aggregate (block index, first axis fastest) of every interior face, and the block grid."""
    B = coarse_dims((nx, ny, nz))
    agg = np.array([(i // 2) + B[0] * ((j // 2) + B[1] * (l // 2)) for _, i, j, l in face_positions(nx, ny, nz)],
                   dtype=np.int64)
    return agg, B


def grid_aggregates(dims):
    """Parent of every point of the grid `dims` in the grid coarse_dims(dims)."""
    C = coarse_dims(dims)
    idx = np.arange(dims[0] * dims[1] * dims[2])
    i, j, l = idx % dims[0], (idx // dims[0]) % dims[1], idx // (dims[0] * dims[1])
    return (i // 2) + C[0] * ((j // 2) + C[1] * (l // 2)), C


def tentative_prolongation(agg, n_coarse, nfn=1):
    """P with P[(f, m), agg[f]] = 1 for every node m < nfn of every fine point f."""
    rows = np.arange(agg.size * nfn)
    cols = np.repeat(agg, nfn)
    return sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(agg.size * nfn, n_coarse))


def start_vector(n):
    i = np.arange(n, dtype=np.int64)
    return ((7919 * i) % 101) / 101.0 - 0.5


def chebyshev_coefficients(lmax, ratio, degree):
    """theta, delta and the recurrence factors rho_k of the Chebyshev iteration on [lmax/ratio, lmax]."""
    a, b = lmax / ratio, lmax
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    sigma = theta / delta
    rho = [1.0 / sigma]
    for _ in range(1, degree):
        rho.append(1.0 / (2.0 * sigma - rho[-1]))
    return theta, delta, rho


class AggregationAMG:
    def __init__(self, H, nx, ny, nz, nfn, degree=2, ratio=30.0, power_steps=12, coarsest=512):
        self.degree, self.ratio, self.power_steps, self.coarsest = degree, ratio, power_steps, coarsest
        A = sp.csr_matrix(H)
        self.A, self.P, self.dinv, self.lmax = [A], [], [], []
        if A.shape[0] > coarsest:
            agg, dims = face_aggregates(nx, ny, nz)
            while True:
                n_c = dims[0] * dims[1] * dims[2]
                P = tentative_prolongation(agg, n_c, nfn if not self.P else 1)
                Ac = sp.csr_matrix(P.T @ self.A[-1] @ P)
                d = Ac.diagonal()
                empty = d == 0.0
                if np.any(empty):
                    Ac = Ac + sp.diags(empty.astype(float))
                Ac.sort_indices()
                self.P.append(P)
                self.A.append(Ac)
                if n_c <= coarsest or dims == (1, 1, 1):
                    break
                agg, dims = grid_aggregates(dims)
        for A_l in self.A[:-1]:
            d = A_l.diagonal()
            self.dinv.append(1.0 / d)
            self.lmax.append(1.1 * self.power_estimate(A_l, d))
        self.coarse_inv = np.linalg.inv(self.A[-1].toarray())

    def power_estimate(self, A, d):
        """Largest eigenvalue of D^{-1} A: power iteration, Rayleigh quotient in the D inner product."""
        v = start_vector(A.shape[0])
        lam = 0.0
        for _ in range(self.power_steps):
            w = A @ v
            lam = (v @ w) / (v @ (d * v))
            v = w / d
            v = v / np.linalg.norm(v)
        return lam

    def smooth(self, level, b, x):
        """Chebyshev iteration on A x = b from x (a new array); also returns the final residual."""
        A, dinv = self.A[level], self.dinv[level]
        theta, delta, rho = chebyshev_coefficients(self.lmax[level], self.ratio, self.degree)
        r = b - A @ x
        dvec = dinv * r / theta
        x = x + dvec
        for k in range(1, self.degree):
            r = r - A @ dvec
            dvec = rho[k] * rho[k - 1] * dvec + (2.0 * rho[k] / delta) * (dinv * r)
            x = x + dvec
        r = r - A @ dvec
        return x, r

    def vcycle(self, b, level=0):
        if level == len(self.A) - 1:
            return self.coarse_inv @ b
        x, r = self.smooth(level, b, np.zeros_like(b))
        P = self.P[level]
        x = x + P @ self.vcycle(P.T @ r, level + 1)
        x, _ = self.smooth(level, b, x)
        return x

    def pcg(self, g, rtol=1e-12, maxit=1000, x0=None):
        """CG preconditioned by one V-cycle, stopping as pcg_diag does (||r|| <= rtol ||r_0||)."""
        H = self.A[0]
        x = np.zeros_like(g) if x0 is None else x0.copy()
        r = g - H @ x
        r0 = np.linalg.norm(r)
        if r0 == 0.0:
            return x, 0, 0.0
        z = self.vcycle(r)
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
            z = self.vcycle(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x, maxit, np.linalg.norm(r) / r0
