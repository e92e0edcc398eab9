"""Full-size workloads (32^3 RT_1, 96^3 RT_2, 64^3 RT_3) in the launch configuration the benchmark
times, FP64 and mixed precision, hybridization and static condensation, checked on sampled
outputs the oracle computes one element at a time:

* rows of H and g for every face of a few seeded elements: each such row is the sum of the
  S_T / g_T of the face's two neighbours (eq. 2.4), which the oracle forms independently;
* the back substitution with lambda = 0 on sampled elements, i.e. u_T = A_T^{-1} f_T;
* on the 32^3 case, the whole reduced solve: the true residual ||g - H lambda|| / ||g|| of the
  GPU's lambda, computed with torch's sparse product (a property at any size).
Tolerances are the conditioning-derived bound of the parity tests, per sampled element.
"""
from collections import defaultdict

import numpy as np
import pytest

from gpu_helpers import EPS, dev, kappa_w, rel_inf
from oracle.hybrid import Discretization
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu


def neighbours(n, e, a):
    i, j, l = e % n, (e // n) % n, e // (n * n)
    d, s = a // 2, a % 2
    pos = [i, j, l]
    pos[d] += 1 if s else -1
    if not 0 <= pos[d] < n:
        return None
    return pos[0] + n * (pos[1] + n * pos[2])


U32 = np.finfo(np.float32).eps / 2


def sampled_rows(ctx, p, D, sample, reduce_element, tol_S, tol_g):
    """Rows of the exported H (or S) and g for every interior face of the sampled elements,
    against the sum of the two neighbours' oracle contributions, entry-wise per row.
    reduce_element(e) -> dict(lam=global row ids, S=element block, g=element load)."""
    from paper_1801_08914_gb300 import hyb
    red = hyb.hyb_export_reduced(ctx)
    rp = red["row_ptr"]
    n, nfn = p.nx, (p.order + 1) ** 2
    worst_S = worst_g = 0.0
    checked = 0
    for e in sample:
        de = reduce_element(e)
        faces = D.mesh.element_faces(e)
        for a, (_, fint) in enumerate(faces):
            if fint < 0:
                continue
            e2 = neighbours(n, e, a)
            d2 = reduce_element(e2)
            rows, g = defaultdict(lambda: defaultdict(float)), defaultdict(float)
            for d in (de, d2):
                for i, r in enumerate(d["lam"]):
                    for j, c in enumerate(d["lam"]):
                        rows[r][c] += d["S"][i, j]
                    g[r] += d["g"][i]
            tS, tg = tol_S(e, e2), tol_g(e, e2)
            gv, gr = [], []
            for m in range(nfn):
                r = fint * nfn + m
                lo, hi = int(rp[r]), int(rp[r + 1])
                cols = red["col"][lo:hi].cpu().numpy()
                vals = red["val"][lo:hi].cpu().numpy()
                ref = np.array([rows[r][c] for c in cols])
                assert sorted(int(c) for c in rows[r].keys()) == [int(c) for c in cols]
                xr = rel_inf(vals, ref)                       # this row, against its largest entry
                worst_S = max(worst_S, xr / tS)
                assert xr <= tS, (e, a, m, xr, tS)
                gv.append(red["rhs"][r].item())
                gr.append(g[r])
                checked += 1
            xg = rel_inf(np.array(gv), np.array(gr))
            worst_g = max(worst_g, xg / tg)
            assert xg <= tg, (e, a, xg, tg)
    return checked, worst_S, worst_g


def hyb_reduce(D):
    return D.element_reduced


def sc_reduce(D):
    def f(e):
        c = D.element_condensed(e)
        return dict(lam=c["gidx"], S=c["Shat"], g=c["r"])
    return f


def kappa_T(D, *es):
    return max(np.linalg.cond(D.element(e)["A"]) for e in es)


@pytest.mark.parametrize("cfg,nsample", [(2, 6), (3, 3), (5, 2)])
def test_full_size_sampled_rows_and_recovery(cfg, nsample):
    """FP64 hybridization at full size: sampled rows of H and g, and u_T = A_T^{-1} f_T."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.make_config(cfg)
    E = p.n_elem
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta))
    hyb.hyb_assemble_reduced(ctx, dev(p.load), None)
    D = Discretization.from_problem(p)
    rng = np.random.default_rng(cfg)
    sample = [int(x) for x in rng.choice(E, size=nsample, replace=False)]
    tol = lambda *es: max(1e-12, kappa_T(D, *es) * EPS)
    checked, wS, wg = sampled_rows(ctx, p, D, sample, hyb_reduce(D), tol, tol)
    # back substitution with lambda = 0: u_T = A_T^{-1} f_T
    sz = ctx.sizes()
    lam0 = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    u = torch.empty(E, sz["n_loc"], dtype=torch.float64, device="cuda")
    hyb.hyb_recover(ctx, lam0, u)
    for e in sample:
        d = D.element(e)
        ref = np.zeros(D.n)
        ref[d["free"]] = np.linalg.solve(d["A"], d["f"])
        assert rel_inf(u[e].cpu().numpy(), ref) <= tol(e)
    print(f"config {cfg}: {checked} rows of H and g and {len(sample)} recovered elements match the oracle "
          f"(worst row at {wS:.2e} of its bound, g at {wg:.2e})")
    ctx.close()


@pytest.mark.parametrize("cfg,nsample", [(3, 3), (5, 2)])
def test_full_size_mixed_sampled_rows_and_recovery(cfg, nsample):
    """Mixed precision, autotuned threshold (all elements FP32 up to beta/alpha = 1e6) at the
    precision workloads 96^3 RT_2 and 64^3 RT_3. The reference is the oracle's mixed-form
    route (Sec. 3.2), accurate at this contrast. Bounds: S and g per row 100 u_32 kappa_w (the
    FP32 elimination of the well-conditioned M and Z); the refined element solve of the
    recovery (lambda = 0) (100 u_32 kappa_w)^2, one FP64-residual refinement step applied to
    an FP32 solve, floored at 1e-10."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.make_config(cfg)
    E = p.n_elem
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta),
                        precision=hyb.HYB_MIXED, contrast_threshold=0.0)
    n64, n32, theta = ctx.precision_split()
    print(f"config {cfg}: autotuned threshold {theta:g}: {n32} FP32 + {n64} FP64 elements")
    hyb.hyb_assemble_reduced(ctx, dev(p.load), None)
    D = Discretization.from_problem(p)
    rng = np.random.default_rng(10 + cfg)
    sample = [int(x) for x in rng.choice(E, size=nsample, replace=False)]
    bS = lambda *es: 100 * U32 * kappa_w(D, es)
    bg = lambda *es: max(1e-10, bS(*es) ** 2)
    checked, wS, wg = sampled_rows(ctx, p, D, sample, D.element_reduced_mixed, bS, bS)
    sz = ctx.sizes()
    lam0 = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    u = torch.empty(E, sz["n_loc"], dtype=torch.float64, device="cuda")
    hyb.hyb_recover(ctx, lam0, u)
    lam0h = np.zeros(sz["n_lambda"])
    worst_u = 0.0
    for e in sample:
        ref = D.recover_mixed_element(e, lam0h)
        xu = rel_inf(u[e].cpu().numpy(), ref)
        worst_u = max(worst_u, xu)
        assert xu <= bg(e), (e, xu, bg(e))
    print(f"config {cfg} mixed: {checked} rows of H and g, {len(sample)} recovered elements; worst row at "
          f"{wS:.2e} of its bound, g at {wg:.2e}, recovery max rel {worst_u:.1e}")
    ctx.close()


def test_full_size_static_condensation_rt3():
    """Static condensation at the 64^3 RT_3 workload: sampled rows of S and of its right-hand
    side against the oracle's per-element condensation (Sec. 3.1, eq. 3.1), and the interior
    recovery u_i = A_ii^{-1} f_i with zero face values."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.make_config(5)
    E = p.n_elem
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta))
    hyb.staticcond_assemble(ctx, dev(p.load), None)
    D = Discretization.from_problem(p)
    rng = np.random.default_rng(55)
    sample = [int(x) for x in rng.choice(E, size=2, replace=False)]
    tol = lambda *es: max(1e-12, kappa_T(D, *es) * EPS)
    checked, wS, wg = sampled_rows(ctx, p, D, sample, sc_reduce(D), tol, tol)
    sz = ctx.sizes()
    uf = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    u = torch.empty(E, sz["n_loc"], dtype=torch.float64, device="cuda")
    hyb.staticcond_recover(ctx, uf, u)
    for e in sample:
        c = D.element_condensed(e)
        d = c["d"]
        ref = np.zeros(D.n)
        ii = c["ii"]
        ref[d["free"][ii]] = np.linalg.solve(d["A"][np.ix_(ii, ii)], d["f"][ii])
        assert rel_inf(u[e].cpu().numpy(), ref) <= tol(e)
    print(f"64^3 RT_3 static condensation: {checked} rows of S and its load, {len(sample)} recovered elements "
          f"(worst row at {wS:.2e} of its bound, load at {wg:.2e})")
    ctx.close()


def test_full_size_reduced_solve_residual():
    """32^3 RT_1: diag-PCG to 1e-12 (the paper's stopping rule); the true residual of the GPU's
    lambda against the GPU's H, recomputed with an independent sparse product, meets it."""
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.make_config(2)
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta))
    hyb.hyb_assemble_reduced(ctx, dev(p.load), None)
    sz = ctx.sizes()
    lam = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    it, rr, st = hyb.hyb_solve_reduced(ctx, 1e-12, 100000, lam)
    red = hyb.hyb_export_reduced(ctx)
    H = torch.sparse_csr_tensor(red["row_ptr"], red["col"].to(torch.int64), red["val"],
                                size=(sz["n_lambda"], sz["n_lambda"]))
    res = torch.linalg.norm(red["rhs"] - H @ lam) / torch.linalg.norm(red["rhs"])
    print(f"32^3 RT_1: {it} PCG iterations, recursive residual {rr:.2e}, true residual {res.item():.2e}")
    assert st == hyb.HYB_OK and rr <= 1e-12 and res.item() <= 1e-11
    ctx.close()
