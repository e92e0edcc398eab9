"""Full-size workloads (32^3 RT_1, 96^3 RT_2, 64^3 RT_3) in the launch configuration the benchmark
times, checked on sampled outputs the oracle computes one element at a time:

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

from gpu_helpers import EPS, dev, rel
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


@pytest.mark.parametrize("cfg,nsample", [(2, 6), (3, 3), (5, 2)])
def test_full_size_sampled_rows_and_recovery(cfg, nsample):
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.make_config(cfg)
    n, E = p.nx, p.n_elem
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta))
    hyb.hyb_assemble_reduced(ctx, dev(p.load), None)
    red = hyb.hyb_export_reduced(ctx)
    rp = red["row_ptr"]
    D = Discretization.from_problem(p)
    rng = np.random.default_rng(cfg)
    sample = [int(x) for x in rng.choice(E, size=nsample, replace=False)]
    nfn = (p.order + 1) ** 2
    checked = 0
    for e in sample:
        de = D.element_reduced(e)
        faces = D.mesh.element_faces(e)
        for a, (_, fint) in enumerate(faces):
            if fint < 0:
                continue
            e2 = neighbours(n, e, a)
            d2 = D.element_reduced(e2)
            rows, g = defaultdict(lambda: defaultdict(float)), defaultdict(float)
            for d in (de, d2):
                for i, r in enumerate(d["lam"]):
                    for j, c in enumerate(d["lam"]):
                        rows[r][c] += d["S"][i, j]
                    g[r] += d["g"][i]
            kT = max(np.linalg.cond(de["A"]), np.linalg.cond(d2["A"]))
            tol = max(1e-12, kT * EPS)
            gv, gr = [], []
            for m in range(nfn):
                r = fint * nfn + m
                lo, hi = int(rp[r]), int(rp[r + 1])
                cols = red["col"][lo:hi].cpu().numpy()
                vals = red["val"][lo:hi].cpu().numpy()
                ref = np.array([rows[r][c] for c in cols])
                assert sorted(int(c) for c in rows[r].keys()) == [int(c) for c in cols]
                assert rel(vals, ref) <= tol, (e, a, m, rel(vals, ref), tol)
                gv.append(red["rhs"][r].item())
                gr.append(g[r])
                checked += 1
            assert rel(np.array(gv), np.array(gr)) <= tol
    # back substitution with lambda = 0: u_T = A_T^{-1} f_T
    sz = ctx.sizes()
    lam0 = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    u = torch.empty(E, sz["n_loc"], dtype=torch.float64, device="cuda")
    hyb.hyb_recover(ctx, lam0, u)
    for e in sample:
        d = D.element(e)
        ref = np.zeros(D.n)
        ref[d["free"]] = np.linalg.solve(d["A"], d["f"])
        assert rel(u[e].cpu().numpy(), ref) <= max(1e-12, np.linalg.cond(d["A"]) * EPS)
    print(f"config {cfg}: {checked} rows of H and g and {len(sample)} recovered elements match the oracle")
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
