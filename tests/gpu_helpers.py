"""Shared drivers for the GPU parity tests: run the CUDA path through the C ABI and the CPU oracle
on the same seeded inputs, and derive tolerances from the conditioning."""
import numpy as np
import scipy.sparse as sp

EPS = np.finfo(np.float64).eps


def dev(a, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def gpu_run(p, mode="hyb", rtol=1e-14, maxit=100000, solve=True, precision=0, threshold=0.0, op32=None):
    """setup -> assemble -> export reduced system -> PCG -> recover, all through libhyb.
    op32: for mixed contexts, the PCG operator (None: the library's default)."""
    import torch
    from paper_1801_08914_gb300 import hyb
    ctx = hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta),
                        precision=precision, contrast_threshold=threshold)
    if op32 is not None:
        hyb.hyb_set_mixed_operator(ctx, op32)
    if getattr(p, "natural", False):
        hyb.hyb_set_natural_bc(ctx, True)
    load = dev(p.load)
    ess = None if p.ess is None else dev(p.ess)
    if mode == "hyb":
        hyb.hyb_assemble_reduced(ctx, load, ess)
    else:
        hyb.staticcond_assemble(ctx, load, ess)
    red = {k: v.cpu().numpy() for k, v in hyb.hyb_export_reduced(ctx).items()}
    sz = ctx.sizes()
    out = dict(red=red, sizes=sz, split=ctx.precision_split())
    if solve:
        lam = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
        it, rr, st = hyb.hyb_solve_reduced(ctx, rtol, maxit, lam, check=False)
        u = torch.zeros(sz["n_elem"], sz["n_loc"], dtype=torch.float64, device="cuda")
        if mode == "hyb":
            hyb.hyb_recover(ctx, lam, u)
        else:
            hyb.staticcond_recover(ctx, lam, u)
        torch.cuda.synchronize()
        out.update(lam=lam.cpu().numpy(), u=u.cpu().numpy(), it=it, rr=rr, status=st)
    ctx.close()
    return out


def csr(red):
    n = red["row_ptr"].size - 1
    return sp.csr_matrix((red["val"], red["col"], red["row_ptr"]), shape=(n, n))


def rel(a, b):
    """Norm-wise relative difference ||a - b||_2 / ||b||_2 (printed beside the entry-wise ones)."""
    nb = np.linalg.norm(np.ravel(b))
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / (nb if nb > 0 else 1.0)


def rel_inf(a, b):
    """Entry-wise relative difference against the largest entry: max_i |a_i - b_i| / max_i |b_i|.
    A single wrong entry cannot hide under the norm of many right ones."""
    a, b = np.ravel(a), np.ravel(b)
    s = np.abs(b).max() if b.size else 0.0
    return (np.abs(a - b).max() / (s if s > 0 else 1.0)) if a.size else 0.0


def rel_groups(a, b, g):
    """Entry-wise relative difference per group of g consecutive entries (an element's dofs):
    max over groups of max |a - b| / max |b| within the group."""
    a, b = np.reshape(a, (-1, g)), np.reshape(b, (-1, g))
    d, s = np.abs(a - b).max(axis=1), np.abs(b).max(axis=1)
    return float((d / np.where(s > 0, s, 1.0)).max()) if d.size else 0.0


def rel_rows(val, ref, row_ptr):
    """Entry-wise relative difference per CSR row (same pattern on both sides): max over rows
    of max_j |val_rj - ref_rj| / max_j |ref_rj|."""
    val, ref = np.ravel(val), np.ravel(ref)
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    nonempty = row_ptr[1:] > row_ptr[:-1]
    starts = row_ptr[:-1][nonempty]
    d = np.maximum.reduceat(np.abs(val - ref), starts)
    s = np.maximum.reduceat(np.abs(ref), starts)
    return float((d / np.where(s > 0, s, 1.0)).max()) if d.size else 0.0


def element_kappa(D, elements=None):
    es = range(D.mesh.n_elem) if elements is None else elements
    return max(np.linalg.cond(D.element(e)["A"]) for e in es)


def kappa_w(D, elements=None):
    """Largest condition number of the factored matrices of the FP32 mixed form, M and
    Z = W^{-1} (W + B M^{-1} B^T) W^{-1}, over the elements (Sec. 3.2's blocks)."""
    out = 1.0
    es = range(D.mesh.n_elem) if elements is None else elements
    for e in es:
        M, B, W, _ = D.mixed_form_blocks(e)
        Wi = np.linalg.inv(W)
        Z = Wi @ (W + B @ np.linalg.solve(M, B.T)) @ Wi
        out = max(out, np.linalg.cond(M), np.linalg.cond(Z))
    return out
