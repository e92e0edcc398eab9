"""Seeded synthetic inputs for the hybridization workloads.

This module is the only code shared by the CUDA path and the CPU oracle. It
holds no arithmetic of the method itself (no quadrature, no basis, no Piola
map, no elimination): it draws random numbers and lays out the structured
hexahedral mesh that both sides read.

Random numbers come from a counter-based SplitMix64 generator (Steele, Lea,
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): value i
of stream s under seed S is mix64(key(S, s) + (i + 1) * GOLDEN), where mix64 is
SplitMix64's finaliser. Uniforms on [0, 1) take the top 53 bits; normals use
the Box-Muller transform on consecutive pairs of uniforms.

Mesh recipe (the paper's soft-hard and SPE10 workloads use structured hex
meshes, Sec. 6.1 and 6.4; none of its geometries ship with it): an nx*ny*nz
grid on [0,1]^3 with vertex (i,j,l) at (i/nx, j/ny, l/nz); every coordinate of
every interior vertex moves by U(-gamma*h, +gamma*h) with h the grid spacing of
that axis, drawn in vertex-lexicographic order (i fastest), x then y then z.
Boundary vertices stay put, so boundary faces are planar axis-aligned
rectangles.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_FNV = np.uint64(0x100000001B3)

# stream ids
STREAM_JITTER = 1
STREAM_ALPHA = 2
STREAM_CONTRAST = 3
STREAM_LOAD = 4
STREAM_BATCH = 5
STREAM_LINES = 6


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Raw 64-bit draws number offset..offset+count-1 of (seed, stream)."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([np.uint64(seed) * _FNV + np.uint64(stream)], dtype=np.uint64))[0]
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix64(key + i * _GOLDEN)


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """U[0,1) in float64 from the top 53 bits of each draw."""
    r = splitmix64(seed, stream, count, offset)
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """N(0,1) by Box-Muller on consecutive uniform pairs (cos branch then sin branch)."""
    npair = (count + 1) // 2
    u = uniform(seed, stream, 2 * npair)
    u1 = 1.0 - u[0::2]            # (0, 1]: log is finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npair)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:count]


@dataclass
class Problem:
    """One hybridization problem: mesh, coefficients, load and boundary data.

    vertices : ((nz+1)*(ny+1)*(nx+1), 3) float64, vertex (i,j,l) at row i + (nx+1)*(j + (ny+1)*l)
    alpha    : (E,) mass coefficient per element, element (i,j,l) at i + nx*(j + ny*l)
    beta     : (E,) divergence coefficient per element
    load     : (E, n_loc) coefficients of f in the broken RT_k basis (element-local dof order)
    ess      : (E, n_loc) essential normal-trace values, read only at boundary-face dofs, or None (= 0)
    natural  : True when the boundary faces carry no essential data (their dofs stay unknowns)

    Element-local dof order (the contract both implementations read): the interior dofs of the
    x, y, z reference components (k (k+1)^2 each, component by component), then the face dofs
    of the faces x=0, x=1, y=0, y=1, z=0, z=1 ((k+1)^2 each); a face's dofs belong to the
    component normal to it.
    """
    nx: int
    ny: int
    nz: int
    order: int
    vertices: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    load: np.ndarray
    ess: np.ndarray | None
    name: str = ""
    natural: bool = False

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_loc(self) -> int:
        k = self.order
        return 3 * (k + 1) * (k + 1) * (k + 2)


def n_local_dofs(order: int) -> int:
    return 3 * (order + 1) ** 2 * (order + 2)


def mesh_vertices(nx: int, ny: int, nz: int, gamma: float, seed: int) -> np.ndarray:
    """Structured grid on [0,1]^3 with seeded jitter of interior vertices (recipe in the module doc)."""
    hx, hy, hz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    i = np.arange(nx + 1, dtype=np.float64)
    j = np.arange(ny + 1, dtype=np.float64)
    l = np.arange(nz + 1, dtype=np.float64)
    L, J, I = np.meshgrid(l, j, i, indexing="ij")          # i fastest when flattened
    v = np.stack([I.ravel() * hx, J.ravel() * hy, L.ravel() * hz], axis=1)
    if gamma != 0.0:
        interior = ((I > 0) & (I < nx) & (J > 0) & (J < ny) & (L > 0) & (L < nz)).ravel()
        nint = int(interior.sum())
        u = uniform(seed, STREAM_JITTER, 3 * nint).reshape(nint, 3)
        v[interior] += (2.0 * u - 1.0) * gamma * np.array([hx, hy, hz])
    return v


def random_problem(n: int, order: int, gamma: float, seed: int,
                   contrast_lo: float, contrast_hi: float,
                   lognormal_alpha: bool = True, name: str = "") -> Problem:
    """alpha ~ lognormal(0,1) per element, beta/alpha ~ 10^U(lo,hi), N(0,1) load coefficients, zero essential BC."""
    E = n * n * n
    nl = n_local_dofs(order)
    verts = mesh_vertices(n, n, n, gamma, seed)
    alpha = np.exp(normal(seed, STREAM_ALPHA, E)) if lognormal_alpha else np.ones(E)
    lo, hi = np.log10(contrast_lo), np.log10(contrast_hi)
    beta = alpha * 10.0 ** (lo + (hi - lo) * uniform(seed, STREAM_CONTRAST, E))
    load = normal(seed, STREAM_LOAD, E * nl).reshape(E, nl)
    return Problem(n, n, n, order, verts, alpha, beta, load, None, name)


def _u_exact(x, y, z):
    return np.stack([1.0 + 2.0 * x, 3.0 - y, 0.5 + z], axis=-1)


def manufactured_rt0_problem(n: int, gamma: float, seed: int) -> Problem:
    """RT_0 workload with u_exact = (1+2x, 3-y, 0.5+z), alpha = beta = 1.

    The RT_0 reference dofs sit at the face centres (closed nodes {0,1} along the
    component's axis, the open node 1/2 across it). Both the load coefficients
    and the essential values are h_a*h_b * u_exact(face centre of the unjittered
    grid) . e_axis, where h_a, h_b are the grid spacings across the face: the
    face's normal flux density. With gamma = 0 this is the exact RT_0
    interpolant of u_exact (the field is in RT_0 on affine cells), so the load
    f = sum c_j phi_j equals u_exact = alpha u - grad(beta div u). With
    gamma > 0 it is a smooth synthetic load; the boundary values stay exact
    because boundary faces are never jittered.
    """
    order = 0
    nx = ny = nz = n
    E = nx * ny * nz
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    verts = mesh_vertices(nx, ny, nz, gamma, seed)
    e = np.arange(E)
    ei, ej, el = e % nx, (e // nx) % ny, e // (nx * ny)
    load = np.zeros((E, 6))
    # local face order: x0, x1, y0, y1, z0, z1 (k = 0: no interior dofs)
    for f in range(6):
        axis, side = f // 2, f % 2
        c = np.stack([ei + 0.5, ej + 0.5, el + 0.5], axis=1).astype(np.float64)
        c[:, axis] = (np.stack([ei, ej, el], axis=1)[:, axis] + side)
        pos = c * h
        u = _u_exact(pos[:, 0], pos[:, 1], pos[:, 2])
        area = np.prod(np.delete(h, axis))
        load[:, f] = area * u[:, axis]
    ess = load.copy()
    return Problem(nx, ny, nz, order, verts, np.ones(E), np.ones(E), load, ess, "manufactured")


def dof_component(order: int) -> np.ndarray:
    """Reference component (0, 1, 2) of every element-local dof, in the order of Problem's doc."""
    k, p = order, order + 1
    ni = k * p * p
    comp = [c for c in range(3) for _ in range(ni)]
    comp += [f // 2 for f in range(6) for _ in range(p * p)]
    return np.array(comp, dtype=np.int64)


# mesh of the soft-hard test per order (Sec. 6.1, its table of initial meshes): nx = ny = 2 nz
SOFT_HARD_NZ = {0: 32, 1: 16, 2: 12, 3: 8}


def soft_hard_problem(order: int, p: float, nz: int | None = None) -> Problem:
    """The soft-hard materials test of Sec. 6.1 on an unjittered 2nz x 2nz x nz grid.

    The paper's coefficients, in this package's naming (alpha multiplies the mass term,
    beta the divergence term): beta = 1 everywhere and alpha = 10^p on the two cubes
    [1/4, 1/2]^3 and [1/2, 3/4]^3 (an element belongs to them when its centre does; nz a
    multiple of 4 makes the cubes unions of elements), 1 elsewhere. The source is the
    constant field g = (1, 1, 1) and no boundary face carries essential data. On the box
    cell [h_x] x [h_y] x [h_z] the reference field of a constant g under the Piola map is
    (h_y h_z g_x, h_x h_z g_y, h_x h_y g_z) at every point, so every dof of component c takes
    the product of the two other spacings: that is the load in the broken RT_k basis, exact.
    """
    nz = SOFT_HARD_NZ.get(order, 8) if nz is None else nz
    if nz % 4:
        raise ValueError("nz must be a multiple of 4")
    nx = ny = 2 * nz
    E = nx * ny * nz
    verts = mesh_vertices(nx, ny, nz, 0.0, 0)
    e = np.arange(E)
    cx = ((e % nx) + 0.5) / nx
    cy = (((e // nx) % ny) + 0.5) / ny
    cz = ((e // (nx * ny)) + 0.5) / nz
    inner = lambda lo, hi: (cx > lo) & (cx < hi) & (cy > lo) & (cy < hi) & (cz > lo) & (cz < hi)
    alpha = np.where(inner(0.25, 0.5) | inner(0.5, 0.75), 10.0 ** p, 1.0)
    beta = np.ones(E)
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    per_comp = np.array([h[1] * h[2], h[0] * h[2], h[0] * h[1]])
    load = np.tile(per_comp[dof_component(order)], (E, 1))
    return Problem(nx, ny, nz, order, verts, alpha, beta, load, None, f"softhard_p{p:g}", natural=True)


# The five workloads (sizes as the benchmark definitions state them).
CONFIGS = {
    1: dict(kind="manufactured", n=4, order=0, gamma=0.0, seed=1000),
    "1j": dict(kind="manufactured", n=4, order=0, gamma=0.15, seed=1000),
    2: dict(kind="random", n=32, order=1, gamma=0.2, seed=2000, contrast=(1e-2, 1e4)),
    3: dict(kind="random", n=96, order=2, gamma=0.2, seed=3000, contrast=(1e-2, 1e6)),
    5: dict(kind="random", n=64, order=3, gamma=0.2, seed=5000, contrast=(1e-2, 1e6)),
}


def make_config(cfg, n: int | None = None) -> Problem:
    """Build a named workload; n overrides the mesh size (scaled-down parity cases)."""
    c = CONFIGS[cfg]
    nn = c["n"] if n is None else n
    if c["kind"] == "manufactured":
        return manufactured_rt0_problem(nn, c["gamma"], c["seed"])
    lo, hi = c["contrast"]
    return random_problem(nn, c["order"], c["gamma"], c["seed"], lo, hi, name=f"config{cfg}")


def batch_problems(count: int = 256, seed0: int = 4000, nmin: int = 6, nmax: int = 24,
                   contrast=(1e-2, 1e4)) -> list[Problem]:
    """Many independent problems of uneven size and order: n ~ U{nmin..nmax}, k ~ U{0..3}."""
    return [batch_problem(p, seed0, nmin, nmax, contrast) for p in range(count)]


def batch_shape(p: int, seed0: int = 4000, nmin: int = 6, nmax: int = 24) -> tuple[int, int]:
    """(n, k) of problem p of the batched workload: n ~ U{nmin..nmax}, k ~ U{0..3}."""
    u = uniform(seed0 + p, STREAM_BATCH, 2)
    return nmin + int(u[0] * (nmax - nmin + 1)), int(u[1] * 4)


def batch_problem(p: int, seed0: int = 4000, nmin: int = 6, nmax: int = 24, contrast=(1e-2, 1e4)) -> Problem:
    """Problem p of the batched workload (seed seed0 + p)."""
    n, k = batch_shape(p, seed0, nmin, nmax)
    return random_problem(n, k, 0.2, seed0 + p, contrast[0], contrast[1], name=f"batch{p}")


@dataclass
class TwoLevelProblem:
    """A mesh with a non-conforming interface: a coarse block of nx x ny x nzc cells on z in
    [0, zI] under a fine block of mx x my x nzf cells on [zI, 1], with (mx, my) = (2 nx, 2 ny)
    when refine (each coarse top face meets four fine bottom faces) and (nx, ny) otherwise (a
    conforming interface, the same cells as one structured grid).

    coarse_vertices : ((nzc+1)(ny+1)(nx+1), 3), vertex (i,j,l) at i + (nx+1)(j + (ny+1) l)
    fine_vertices   : ((nzf+1)(my+1)(mx+1), 3), vertex (i,j,l) at i + (mx+1)(j + (my+1) l);
                      layer l = 0 lies on the interface
    alpha, beta     : (Ec + Ef,) per element: the coarse cells (i + nx (j + ny l)) first, then
                      the fine cells (i + mx (j + my l))
    load            : (Ec + Ef, n_loc) coefficients of f in the broken RT_k basis
    Every boundary face is natural (no essential data).
    """
    nx: int
    ny: int
    nzc: int
    nzf: int
    order: int
    refine: bool
    coarse_vertices: np.ndarray
    fine_vertices: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    load: np.ndarray
    z_interface: float = 0.5

    @property
    def mx(self) -> int:
        return 2 * self.nx if self.refine else self.nx

    @property
    def my(self) -> int:
        return 2 * self.ny if self.refine else self.ny

    @property
    def n_coarse(self) -> int:
        return self.nx * self.ny * self.nzc

    @property
    def n_fine(self) -> int:
        return self.mx * self.my * self.nzf

    @property
    def n_elem(self) -> int:
        return self.n_coarse + self.n_fine


def two_level_problem(nx: int, ny: int, nzc: int, nzf: int, order: int, seed: int, refine: bool = True,
                      lines: float = 0.0, gamma: float = 0.0, z_interface: float = 0.5,
                      contrast=(0.1, 10.0)) -> TwoLevelProblem:
    """Seeded two-level mesh (TwoLevelProblem) and its coefficients.

    Grid lines: x_i = i / nx, y_j = j / ny, the coarse z lines l zI / nzc and the fine ones
    zI + l (1 - zI) / nzf; with lines > 0 every interior line moves by U(-lines h, +lines h)
    (h its spacing; x, then y, then coarse z, then fine z lines), which keeps every cell a box.
    The fine x and y lines are the coarse ones and, when refine, their midpoints. With gamma > 0
    every vertex off the domain boundary then moves by U(-gamma h, +gamma h) per coordinate (h the
    block's spacing along that axis), except that coarse vertices on the interface move in x and
    y only and the fine interface vertices are placed at the bilinear points (parameters 0, 1/2,
    1) of the coarse top faces, so that four fine faces tile each coarse face exactly.
    alpha ~ lognormal(0, 1), beta / alpha ~ 10^U(log10 contrast), N(0, 1) load coefficients.
    """
    def line_set(n, lo, hi, offset):
        x = lo + (hi - lo) * np.arange(n + 1, dtype=np.float64) / n
        if lines > 0.0 and n > 1:
            u = uniform(seed, STREAM_LINES, n - 1, offset)
            x[1:-1] += (2.0 * u - 1.0) * lines * (hi - lo) / n
        return x

    zI = z_interface
    X = line_set(nx, 0.0, 1.0, 0)
    Y = line_set(ny, 0.0, 1.0, nx)
    Zc = line_set(nzc, 0.0, zI, nx + ny)
    Zf = line_set(nzf, zI, 1.0, nx + ny + nzc)

    def grid(xs, ys, zs):
        L, J, I = np.meshgrid(np.arange(zs.size), np.arange(ys.size), np.arange(xs.size), indexing="ij")
        return np.stack([xs[I.ravel()], ys[J.ravel()], zs[L.ravel()]], axis=1), I.ravel(), J.ravel(), L.ravel()

    cv, ci, cj, cl = grid(X, Y, Zc)
    if refine:
        Xf = np.sort(np.concatenate([X, 0.5 * (X[1:] + X[:-1])]))
        Yf = np.sort(np.concatenate([Y, 0.5 * (Y[1:] + Y[:-1])]))
    else:
        Xf, Yf = X, Y
    fv, fi, fj, fl = grid(Xf, Yf, Zf)
    mx, my = Xf.size - 1, Yf.size - 1
    if gamma > 0.0:
        h = np.array([1.0 / nx, 1.0 / ny, zI / nzc])
        inner = (ci > 0) & (ci < nx) & (cj > 0) & (cj < ny) & (cl > 0)
        n_in = int(inner.sum())
        u = uniform(seed, STREAM_JITTER, 3 * n_in).reshape(n_in, 3)
        mv = (2.0 * u - 1.0) * gamma * h
        mv[cl[inner] == nzc, 2] = 0.0                      # the interface stays the plane z = zI
        cv[inner] += mv
        hf = np.array([1.0 / mx, 1.0 / my, (1.0 - zI) / nzf])
        inner_f = (fi > 0) & (fi < mx) & (fj > 0) & (fj < my) & (fl > 0) & (fl < nzf)
        n_f = int(inner_f.sum())
        u = uniform(seed, STREAM_JITTER, 3 * n_f, 3 * n_in).reshape(n_f, 3)
        fv[inner_f] += (2.0 * u - 1.0) * gamma * hf
    # fine interface vertices on the coarse top faces (their bilinear points)
    top = cv.reshape(nzc + 1, ny + 1, nx + 1, 3)[nzc]
    fvr = fv.reshape(nzf + 1, my + 1, mx + 1, 3)
    r = 2 if refine else 1
    for q in range(my + 1):
        j = min(q // r, ny - 1)
        t = (q - r * j) / r
        for p_ in range(mx + 1):
            i = min(p_ // r, nx - 1)
            s_ = (p_ - r * i) / r
            fvr[0, q, p_] = ((1 - s_) * (1 - t) * top[j, i] + s_ * (1 - t) * top[j, i + 1] +
                             (1 - s_) * t * top[j + 1, i] + s_ * t * top[j + 1, i + 1])
    fv = fvr.reshape(-1, 3)
    E = nx * ny * nzc + mx * my * nzf
    nl = n_local_dofs(order)
    alpha = np.exp(normal(seed, STREAM_ALPHA, E))
    lo, hi = np.log10(contrast[0]), np.log10(contrast[1])
    beta = alpha * 10.0 ** (lo + (hi - lo) * uniform(seed, STREAM_CONTRAST, E))
    load = normal(seed, STREAM_LOAD, E * nl).reshape(E, nl)
    return TwoLevelProblem(nx, ny, nzc, nzf, order, refine, cv, fv, alpha, beta, load, zI)

