"""Batched problems (uneven sizes and orders in one context) against solo contexts and the oracle.

The element phase of a batch runs the same element code as a solo context, so its reduced
systems must be bitwise identical; the batched PCG partitions its blocks per problem, so its
iterates differ from a solo solve only by the order of the reductions (compared at the
conditioning-derived bound of the parity tests)."""
import numpy as np
import pytest

from gpu_helpers import EPS, dev, element_kappa, gpu_run, rel, rel_inf
from oracle.hybrid import Discretization, solve_dense
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu


def make_batch(specs):
    return [inputs.random_problem(n, k, 0.2, 700 + i, 1e-2, 1e4, name=f"b{i}") for i, (n, k) in enumerate(specs)]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_solo_and_oracle(precision):
    import torch
    from paper_1801_08914_gb300 import hyb
    specs = [(3, 0), (4, 1), (2, 2), (3, 3), (5, 0), (2, 1)]
    probs = make_batch(specs)
    verts = [dev(p.vertices) for p in probs]
    alphas = [dev(p.alpha) for p in probs]
    betas = [dev(p.beta) for p in probs]
    b = hyb.hyb_setup_batch([(v, p.nx, p.ny, p.nz) for v, p in zip(verts, probs)], [p.order for p in probs],
                            alphas, betas, precision=precision, contrast_threshold=1e4)
    loads = [dev(p.load) for p in probs]
    hyb.hyb_assemble_reduced_batch(b, loads)
    sizes = [b.context(i).sizes() for i in range(len(probs))]
    lams = [torch.zeros(s["n_lambda"], dtype=torch.float64, device="cuda") for s in sizes]
    us = [torch.zeros(s["n_elem"], s["n_loc"], dtype=torch.float64, device="cuda") for s in sizes]
    its, rrs, st = hyb.hyb_solve_reduced_batch(b, 1e-14, 20000, lams)
    hyb.hyb_recover_batch(b, lams, us)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        red = {k: v.cpu().numpy() for k, v in hyb.hyb_export_reduced(b.context(i)).items()}
        # the batched PCG applies the FP64 values; so does the solo context compared with it
        solo = gpu_run(p, rtol=1e-14, maxit=20000, precision=precision, threshold=1e4,
                       op32=False if precision else None)
        assert np.array_equal(red["val"], solo["red"]["val"]) and np.array_equal(red["rhs"], solo["red"]["rhs"])
        D = Discretization.from_problem(p)
        H, g = D.hybridize()
        ev = np.linalg.eigvalsh(H.toarray())
        kH = ev[-1] / ev[0]
        el = rel(lams[i].cpu().numpy(), solo["lam"])
        eu = rel(us[i].cpu().numpy(), solo["u"])
        print(f"batch problem {i} (n={p.nx}, k={p.order}, prec={precision}): {its[i]} it, batch vs solo lam {el:.1e} u {eu:.1e}")
        assert el <= max(1e-12, kH * 100 * EPS) and eu <= max(1e-12, kH * 100 * EPS)
        if precision == 0:
            lam_o = solve_dense(H, g)
            assert rel_inf(lams[i].cpu().numpy(), lam_o) <= max(1e-12, max(kH, element_kappa(D)) * EPS)
    b.close()


def test_batch_graph_replay_matches_direct_launches():
    """The CUDA-graph replay of a PCG chunk runs the same kernels in the same order as the
    direct launches: iterates and counts are bitwise identical (also across an rtol change,
    which re-captures the graph)."""
    import torch
    from paper_1801_08914_gb300 import hyb
    probs = make_batch([(4, 1), (3, 2), (5, 0), (3, 3)])
    verts = [dev(p.vertices) for p in probs]
    b = hyb.hyb_setup_batch([(v, p.nx, p.ny, p.nz) for v, p in zip(verts, probs)], [p.order for p in probs],
                            [dev(p.alpha) for p in probs], [dev(p.beta) for p in probs], precision=0)
    hyb.hyb_assemble_reduced_batch(b, [dev(p.load) for p in probs])
    hyb.hyb_batch_set_pcg_fused(b, False)              # the default; graphs apply to this form
    sizes = [b.context(i).sizes() for i in range(len(probs))]
    for rtol in (1e-12, 1e-10):
        res = []
        for graphs in (True, False):
            hyb.hyb_batch_set_graphs(b, graphs)
            lams = [torch.zeros(s["n_lambda"], dtype=torch.float64, device="cuda") for s in sizes]
            its, rrs, st = hyb.hyb_solve_reduced_batch(b, rtol, 20000, lams)
            assert st == hyb.HYB_OK
            res.append((list(its), [l.clone() for l in lams]))
        assert res[0][0] == res[1][0] and max(res[0][0]) > 32
        assert all(torch.equal(x, y) for x, y in zip(res[0][1], res[1][1]))
    b.close()


def test_batch_team_fused_pcg():
    """The team-fused batched PCG against the three-launch form and solo fused solves: the
    same CG iterates up to the rounding of the reductions (iteration counts within 2, the
    solutions within the kappa(H) rtol bound), bitwise reproducible, and per-problem
    iteration counts (problems converge and leave their teams at different chunks)."""
    import torch
    from paper_1801_08914_gb300 import hyb
    probs = make_batch([(6, 1), (3, 2), (8, 0), (4, 3), (2, 1), (5, 2)])
    verts = [dev(p.vertices) for p in probs]
    b = hyb.hyb_setup_batch([(v, p.nx, p.ny, p.nz) for v, p in zip(verts, probs)], [p.order for p in probs],
                            [dev(p.alpha) for p in probs], [dev(p.beta) for p in probs], precision=0)
    hyb.hyb_assemble_reduced_batch(b, [dev(p.load) for p in probs])
    sizes = [b.context(i).sizes() for i in range(len(probs))]

    def run(fused):
        hyb.hyb_batch_set_pcg_fused(b, fused)
        lams = [torch.zeros(s["n_lambda"], dtype=torch.float64, device="cuda") for s in sizes]
        its, rrs, st = hyb.hyb_solve_reduced_batch(b, 1e-12, 20000, lams)
        assert st == hyb.HYB_OK and max(rrs) <= 1e-12
        return list(its), lams

    itf, lf = run(True)
    itf2, lf2 = run(True)
    itu, lu = run(False)
    assert itf == itf2 and all(torch.equal(x, y) for x, y in zip(lf, lf2))
    assert len(set(itf)) > 1
    for i, p in enumerate(probs):
        assert abs(itf[i] - itu[i]) <= 2, (i, itf[i], itu[i])
        d = rel(lf[i].cpu().numpy(), lu[i].cpu().numpy())
        print(f"team-fused problem {i} (n={p.nx}, k={p.order}): {itf[i]} it (three-launch {itu[i]}), rel diff {d:.1e}")
        assert d <= 1e-8
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_step_graph_matches_the_three_calls(precision):
    """hyb_batch_step (element phase, batched PCG with its loop as a device-driven WHILE node,
    recovery: one CUDA graph launch) against hyb_assemble_reduced_batch + hyb_solve_reduced_batch +
    hyb_recover_batch: the same reduced systems bitwise, the same iteration counts within 2 (the
    initialisation sums its reductions over other block ranges), lambda and u at the parity tests'
    conditioning bound; a second step with other loads reuses the graph; maxit is honoured
    inside the graph."""
    import torch
    from paper_1801_08914_gb300 import hyb
    probs = make_batch([(4, 1), (3, 2), (5, 0), (3, 3), (2, 2), (6, 1)])
    verts = [dev(p.vertices) for p in probs]
    b = hyb.hyb_setup_batch([(v, p.nx, p.ny, p.nz) for v, p in zip(verts, probs)], [p.order for p in probs],
                            [dev(p.alpha) for p in probs], [dev(p.beta) for p in probs], precision=precision,
                            contrast_threshold=1e4)
    sizes = [b.context(i).sizes() for i in range(len(probs))]
    zl = lambda: [torch.zeros(s["n_lambda"], dtype=torch.float64, device="cuda") for s in sizes]
    zu = lambda: [torch.zeros(s["n_elem"], s["n_loc"], dtype=torch.float64, device="cuda") for s in sizes]
    rng = np.random.default_rng(9)
    for step in range(2):
        loads = [dev(p.load * (1.0 if step == 0 else rng.uniform(0.5, 2.0))) for p in probs]
        hyb.hyb_assemble_reduced_batch(b, loads)
        ref_red = [{k: v.cpu().numpy() for k, v in hyb.hyb_export_reduced(b.context(i)).items()}
                   for i in range(len(probs))]
        l3, u3 = zl(), zu()
        it3, _, st = hyb.hyb_solve_reduced_batch(b, 1e-13, 20000, l3)
        assert st == hyb.HYB_OK
        hyb.hyb_recover_batch(b, l3, u3)
        ls, us = zl(), zu()
        its, rrs, st = hyb.hyb_batch_step(b, loads, 1e-13, 20000, ls, us)
        assert st == hyb.HYB_OK and max(rrs) <= 1e-13
        for i, p in enumerate(probs):
            red = {k: v.cpu().numpy() for k, v in hyb.hyb_export_reduced(b.context(i)).items()}
            assert np.array_equal(red["val"], ref_red[i]["val"]) and np.array_equal(red["rhs"], ref_red[i]["rhs"])
            D = Discretization.from_problem(p)
            H, g = D.hybridize()
            ev = np.linalg.eigvalsh(H.toarray())
            tol = max(1e-12, (ev[-1] / ev[0]) * 100 * EPS)
            el = rel_inf(ls[i].cpu().numpy(), l3[i].cpu().numpy())
            eu = rel_inf(us[i].cpu().numpy(), u3[i].cpu().numpy())
            print(f"step {step} problem {i} (n={p.nx}, k={p.order}, prec={precision}): graph {its[i]} it, "
                  f"three calls {it3[i]} it; lambda {el:.1e} u {eu:.1e}")
            assert abs(its[i] - it3[i]) <= 2 and el <= tol and eu <= tol
    for k in range(4):                       # the autotuner's choice per order bin and path
        for path in (0, 1):
            m, g = hyb.hyb_batch_get_autotune(b, k, path)
            assert m in (0, 1, 2, 4) and (g == 0) == (m == 0)
    outside, per_pass, ipp = hyb.hyb_batch_step_kernels(b)
    assert per_pass == 3 * ipp + 1 and outside > 0
    # maxit inside the graph: every problem stops after exactly 5 iterations
    its, rrs, st = hyb.hyb_batch_step(b, [dev(p.load) for p in probs], 1e-13, 5, zl(), zu(), check=False)
    assert st == hyb.HYB_ERR_NOT_CONVERGED and its == [5] * len(probs)
    b.close()
