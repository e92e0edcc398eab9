"""Thin ctypes binding of libhyb.so (include/hyb.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Arrays are torch tensors on the CUDA device (float64, contiguous); the binding
passes their data pointers and the current torch stream. There is no CPU
fallback: importing this module without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhyb.so")

HYB_OK = 0
HYB_ERR_INVALID_ARG = -1
HYB_ERR_UNSUPPORTED_ORDER = -2
HYB_ERR_MESH = -3
HYB_ERR_NOT_SPD = -4
HYB_ERR_NOT_CONVERGED = -5
HYB_ERR_BREAKDOWN = -6
HYB_ERR_CUDA = -7
HYB_ERR_OOM = -8
HYB_ERR_TIMEOUT = -9
HYB_FP64 = 0
HYB_MIXED = 1
HYB_PC_JACOBI = 0
HYB_PC_AMG = 1
KERNEL_CLASSES = {"element": 0, "spmv": 1, "pcg_vector": 2, "recover": 3, "setup": 4, "pcg_fused": 5, "step": 6}

EXPORTS = ["hyb_setup", "hyb_assemble_reduced", "hyb_solve_reduced", "hyb_recover",
           "staticcond_assemble", "staticcond_recover", "hyb_get_reduced", "hyb_export_reduced", "hyb_get_sizes",
           "hyb_set_profiling", "hyb_get_profile", "hyb_pcg_solve_noalloc", "hyb_measure_fma_peak",
           "hyb_get_precision_split", "hyb_setup_batch", "hyb_assemble_reduced_batch", "hyb_solve_reduced_batch",
           "hyb_recover_batch", "hyb_batch_context", "hyb_batch_set_profiling", "hyb_batch_get_profile",
           "hyb_destroy_batch", "hyb_set_mixed_operator", "hyb_batch_step", "hyb_batch_step_kernels", "hyb_batch_get_autotune",
           "hyb_set_preconditioner", "hyb_amg_apply", "hyb_amg_info", "hyb_two_level_layout",
           "hyb_last_error_element", "hyb_destroy", "hyb_status_string"]


class HybError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class _Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("vertices", ctypes.c_void_p)]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libhyb.so not built at {path}: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    lib.hyb_setup.argtypes = [ctypes.POINTER(_Mesh), I, P, P, I, D, P, ctypes.POINTER(P)]
    lib.hyb_assemble_reduced.argtypes = [P, P, P]
    lib.staticcond_assemble.argtypes = [P, P, P]
    lib.hyb_solve_reduced.argtypes = [P, D, I, P, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.hyb_recover.argtypes = [P, P, P]
    lib.staticcond_recover.argtypes = [P, P, P]
    lib.hyb_get_reduced.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                    ctypes.POINTER(P), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.hyb_export_reduced.argtypes = [P, P, P, P, P]
    lib.hyb_pcg_solve_noalloc.argtypes = [P, P, P, P, P, I64, I, D, I, P, ctypes.POINTER(I),
                                          ctypes.POINTER(D)]
    lib.hyb_measure_fma_peak.argtypes = [I, P, ctypes.POINTER(D)]
    lib.hyb_get_precision_split.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(D)]
    PP = ctypes.POINTER(P)
    lib.hyb_setup_batch.argtypes = [I, ctypes.POINTER(_Mesh), ctypes.POINTER(I), PP, PP, I, D, P, ctypes.POINTER(P)]
    lib.hyb_assemble_reduced_batch.argtypes = [P, PP, PP]
    lib.hyb_solve_reduced_batch.argtypes = [P, D, I, PP, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.hyb_recover_batch.argtypes = [P, PP, PP]
    lib.hyb_batch_context.argtypes = [P, I, ctypes.POINTER(P)]
    lib.hyb_batch_step.argtypes = [P, PP, PP, D, I, PP, PP, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.hyb_batch_step_kernels.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I)]
    lib.hyb_batch_get_autotune.argtypes = [P, I, I, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.hyb_batch_set_profiling.argtypes = [P, I]
    lib.hyb_batch_set_graphs.argtypes = [P, I]
    lib.hyb_batch_set_pcg_fused.argtypes = [P, I]
    lib.hyb_batch_get_profile.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(I64)]
    lib.hyb_destroy_batch.argtypes = [P]
    lib.hyb_destroy_batch.restype = None
    lib.hyb_set_profiling.argtypes = [P, I]
    lib.hyb_set_pcg_fused.argtypes = [P, I]
    lib.hyb_set_mixed_operator.argtypes = [P, I]
    lib.hyb_set_preconditioner.argtypes = [P, I, I, I]
    lib.hyb_amg_apply.argtypes = [P, P, P]
    lib.hyb_amg_info.argtypes = [P, ctypes.POINTER(I), P, P, I]
    lib.hyb_two_level_layout.argtypes = [I, I, I, I, I, I, ctypes.POINTER(I64), ctypes.POINTER(I64), P, P, P, P]
    lib.hyb_rsqrt_probe.argtypes = [ctypes.c_int64, P, P, P, P]
    lib.hyb_set_natural_bc.argtypes = [P, I]
    lib.hyb_refine.argtypes = [P, I, D, I, P, P, ctypes.POINTER(D)]
    lib.hyb_barrier_selftest.argtypes = [I, I, P]
    lib.hyb_get_profile.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(I64)]
    lib.hyb_get_sizes.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I), ctypes.POINTER(I64),
                                  ctypes.POINTER(I64)]
    lib.hyb_last_error_element.argtypes = [P, ctypes.POINTER(I64)]
    lib.hyb_destroy.argtypes = [P]
    lib.hyb_destroy.restype = None
    lib.hyb_status_string.argtypes = [I]
    lib.hyb_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("hyb_destroy", "hyb_status_string", "hyb_destroy_batch"):
            getattr(lib, name).restype = I
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def status_string(status: int) -> str:
    return lib().hyb_status_string(int(status)).decode()


def _ptr(t, name, dtype=torch.float64):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _need(t, name, count):
    """The library trusts the extents it is given (plain device pointers): a tensor shorter than
    the context's sizes would be read or written past its end, so lengths are checked here."""
    if t is not None and isinstance(t, torch.Tensor) and t.numel() != count:
        raise ValueError(f"{name} has {t.numel()} entries, expected {count}")
    return t


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(st: int, where: str, ok=(HYB_OK,)):
    if st not in ok:
        raise HybError(st, where)
    return st


class Context:
    """Owns a hyb_ctx* and keeps the tensors the library holds pointers to alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def sizes(self):
        E, L, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        n = ctypes.c_int()
        _check(lib().hyb_get_sizes(self.handle, ctypes.byref(E), ctypes.byref(n), ctypes.byref(L),
                                   ctypes.byref(nnz)), "hyb_get_sizes")
        return dict(n_elem=E.value, n_loc=n.value, n_lambda=L.value, nnz=nnz.value)

    def precision_split(self):
        """(elements on the FP64 path, elements on the FP32 path, contrast threshold)."""
        a, b, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib().hyb_get_precision_split(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(t)),
               "hyb_get_precision_split")
        return a.value, b.value, t.value

    def close(self):
        if self.handle:
            lib().hyb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hyb_setup(vertices, nx, ny, nz, order, alpha, beta, precision=HYB_FP64, contrast_threshold=0.0,
              stream=None, check=True):
    if min(int(nx), int(ny), int(nz)) > 0:              # otherwise the library reports HYB_ERR_INVALID_ARG
        E = int(nx) * int(ny) * int(nz)
        _need(vertices, "vertices", 3 * (int(nx) + 1) * (int(ny) + 1) * (int(nz) + 1))
        _need(alpha, "alpha", E)
        _need(beta, "beta", E)
    m = _Mesh(int(nx), int(ny), int(nz), _ptr(vertices, "vertices"))
    h = ctypes.c_void_p()
    st = lib().hyb_setup(ctypes.byref(m), int(order), _ptr(alpha, "alpha"), _ptr(beta, "beta"),
                         int(precision), float(contrast_threshold), _stream(stream), ctypes.byref(h))
    ctx = Context(h, (vertices, alpha, beta)) if h.value else None
    if check:
        _check(st, "hyb_setup")
        return ctx
    return ctx, st


def _need_elements(ctx, **tensors):
    if not ctx.handle:                                  # a closed context: the library reports it
        return
    z = ctx.sizes()
    for name, t in tensors.items():
        _need(t, name, z["n_elem"] * z["n_loc"])


def _need_lambda(ctx, **tensors):
    if not ctx.handle:
        return
    n = ctx.sizes()["n_lambda"]
    for name, t in tensors.items():
        _need(t, name, n)


def hyb_assemble_reduced(ctx, load, ess=None, check=True):
    _need_elements(ctx, load=load, ess=ess)
    st = lib().hyb_assemble_reduced(ctx.handle, _ptr(load, "load"), _ptr(ess, "ess"))
    return _check(st, "hyb_assemble_reduced") if check else st


def staticcond_assemble(ctx, load, ess=None, check=True):
    _need_elements(ctx, load=load, ess=ess)
    st = lib().staticcond_assemble(ctx.handle, _ptr(load, "load"), _ptr(ess, "ess"))
    return _check(st, "staticcond_assemble") if check else st


def hyb_solve_reduced(ctx, rtol, maxit, lam, check=True):
    """Returns (iterations, relative residual, status)."""
    _need_lambda(ctx, lam=lam)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().hyb_solve_reduced(ctx.handle, float(rtol), int(maxit), _ptr(lam, "lambda"),
                                 ctypes.byref(it), ctypes.byref(rr))
    if check:
        _check(st, "hyb_solve_reduced")
    return it.value, rr.value, st


def hyb_recover(ctx, lam, u, check=True):
    _need_lambda(ctx, lam=lam)
    _need_elements(ctx, u=u)
    st = lib().hyb_recover(ctx.handle, _ptr(lam, "lambda"), _ptr(u, "u"))
    return _check(st, "hyb_recover") if check else st


def staticcond_recover(ctx, u_face, u, check=True):
    _need_lambda(ctx, u_face=u_face)
    _need_elements(ctx, u=u)
    st = lib().staticcond_recover(ctx.handle, _ptr(u_face, "u_face"), _ptr(u, "u"))
    return _check(st, "staticcond_recover") if check else st


def hyb_get_reduced(ctx):
    """Borrowed device pointers and sizes of the context's reduced system (ints)."""
    P = ctypes.c_void_p
    rp, cl, vl, rh = P(), P(), P(), P()
    n, nnz = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().hyb_get_reduced(ctx.handle, ctypes.byref(rp), ctypes.byref(cl), ctypes.byref(vl),
                                 ctypes.byref(rh), ctypes.byref(n), ctypes.byref(nnz)), "hyb_get_reduced")
    return dict(row_ptr=rp.value, col=cl.value, val=vl.value, rhs=rh.value, n=n.value, nnz=nnz.value)


def hyb_export_reduced(ctx):
    """Copies of the reduced CSR system as CUDA tensors: row_ptr (int64), col (int32), val, rhs."""
    sz = ctx.sizes()
    n, nnz = sz["n_lambda"], sz["nnz"]
    out = dict(row_ptr=torch.empty(n + 1, dtype=torch.int64, device="cuda"),
               col=torch.empty(nnz, dtype=torch.int32, device="cuda"),
               val=torch.empty(nnz, dtype=torch.float64, device="cuda"),
               rhs=torch.empty(n, dtype=torch.float64, device="cuda"))
    torch.cuda.current_stream().synchronize()
    _check(lib().hyb_export_reduced(ctx.handle, _ptr(out["row_ptr"], "row_ptr", torch.int64),
                                    _ptr(out["col"], "col", torch.int32), _ptr(out["val"], "val"),
                                    _ptr(out["rhs"], "rhs")), "hyb_export_reduced")
    return out


def hyb_export_rhs(ctx, out):
    """Copy the reduced right-hand side g into the caller's device tensor `out` (N_lambda doubles)."""
    if out.numel() != ctx.sizes()["n_lambda"]:
        raise ValueError("out must hold N_lambda doubles")
    return _check(lib().hyb_export_reduced(ctx.handle, None, None, None, _ptr(out, "out")), "hyb_export_reduced")


def hyb_pcg_solve_noalloc(row_ptr, col, val, b, x, rows_per_face, rtol, maxit, stream=None, check=True):
    """Allocation-free PCG on a caller-supplied CSR system (see include/hyb.h).
    Returns (iterations, relative residual, status).

    The library trusts the sizes it is given, so they are checked here first: a short x,
    row_ptr or col would make the kernels read or write past the caller's buffers. The
    last check reads row_ptr[n] back to the host (one 8-byte copy)."""
    n = b.numel()
    if x.numel() != n:
        raise ValueError(f"x has {x.numel()} entries, b has {n}")
    if row_ptr.numel() != n + 1:
        raise ValueError(f"row_ptr has {row_ptr.numel()} entries, expected n + 1 = {n + 1}")
    if col.numel() != val.numel():
        raise ValueError(f"col ({col.numel()}) and val ({val.numel()}) differ in length")
    if n > 0 and int(row_ptr[n].item()) > col.numel():
        raise ValueError(f"row_ptr[n] = {int(row_ptr[n].item())} exceeds the {col.numel()} stored entries")
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = lib().hyb_pcg_solve_noalloc(_ptr(row_ptr, "row_ptr", torch.int64), _ptr(col, "col", torch.int32),
                                     _ptr(val, "val"), _ptr(b, "b"), _ptr(x, "x"), int(b.numel()),
                                     int(rows_per_face), float(rtol), int(maxit), _stream(stream),
                                     ctypes.byref(it), ctypes.byref(rr))
    if check:
        _check(st, "hyb_pcg_solve_noalloc")
    return it.value, rr.value, st


def hyb_measure_fma_peak(fp64=True, stream=None):
    """Measured FMA throughput of the current device, TFLOP/s."""
    v = ctypes.c_double()
    _check(lib().hyb_measure_fma_peak(int(bool(fp64)), _stream(stream), ctypes.byref(v)), "hyb_measure_fma_peak")
    return v.value


def hyb_refine(ctx, steps, inner_rtol, maxit, lam, u, check=True):
    """FP64 refinement steps on (lambda, u); returns (||C u|| / ||g|| per step, status)."""
    _need_lambda(ctx, lam=lam)
    _need_elements(ctx, u=u)
    jump = (ctypes.c_double * (int(steps) + 1))()
    st = lib().hyb_refine(ctx.handle, int(steps), float(inner_rtol), int(maxit), _ptr(lam, "lambda"),
                          _ptr(u, "u"), jump)
    if check:
        _check(st, "hyb_refine")
    return list(jump), st


def hyb_rsqrt_probe(x, out, positive_normal, stream=None):
    """Status; out / positive_normal receive the kernels' pivot inverse square root and check."""
    _need(out, "out", x.numel())
    _need(positive_normal, "positive_normal", x.numel())
    return lib().hyb_rsqrt_probe(int(x.numel()), _ptr(x, "x"), _ptr(out, "out"),
                                 _ptr(positive_normal, "positive_normal", torch.int32), _stream(stream))


def hyb_set_natural_bc(ctx, natural, check=True):
    """Boundary reading of the next assembly: False = essential data on every boundary face
    (default), True = natural (no boundary data, boundary-face dofs stay unknowns)."""
    st = lib().hyb_set_natural_bc(ctx.handle, int(bool(natural)))
    return _check(st, "hyb_set_natural_bc") if check else st


def hyb_set_pcg_fused(ctx, on):
    """PCG launch form: True = one cooperative launch per 64 iterations, False = 3 per iteration."""
    return _check(lib().hyb_set_pcg_fused(ctx.handle, int(bool(on))), "hyb_set_pcg_fused")


def hyb_set_mixed_operator(ctx, fp32, check=True):
    """Mixed contexts: the PCG applies H from its FP32 copy (True, default) or its FP64 values."""
    st = lib().hyb_set_mixed_operator(ctx.handle, int(bool(fp32)))
    return _check(st, "hyb_set_mixed_operator") if check else st


def hyb_set_preconditioner(ctx, kind, chebyshev_degree=2, coarsest=64, check=True):
    """PCG preconditioner: HYB_PC_JACOBI (the diagonal) or HYB_PC_AMG (aggregation multigrid)."""
    st = lib().hyb_set_preconditioner(ctx.handle, int(kind), int(chebyshev_degree), int(coarsest))
    return _check(st, "hyb_set_preconditioner") if check else st


def hyb_amg_apply(ctx, r, z, check=True):
    """z = M^{-1} r: one V-cycle of the context's multigrid (device tensors of n_lambda doubles)."""
    _need_lambda(ctx, r=r, z=z)
    st = lib().hyb_amg_apply(ctx.handle, _ptr(r, "r"), _ptr(z, "z"))
    return _check(st, "hyb_amg_apply") if check else st


def hyb_amg_info(ctx, cap=32):
    """(levels, sizes of the levels, power estimates of lmax(D^-1 A) per smoothed level)."""
    n = ctypes.c_int(0)
    sizes = (ctypes.c_int64 * cap)()
    lmax = (ctypes.c_double * cap)()
    _check(lib().hyb_amg_info(ctx.handle, ctypes.byref(n), ctypes.cast(sizes, ctypes.c_void_p),
                              ctypes.cast(lmax, ctypes.c_void_p), cap), "hyb_amg_info")
    k = min(n.value, cap)
    return n.value, [int(sizes[i]) for i in range(k)], [float(lmax[i]) for i in range(k)]


def hyb_two_level_layout(nx, ny, nzc, nzf, order, refine=True):
    """Host-only multiplier layout of a two-level mesh (see include/hyb.h): dict with n_lambda,
    elem_face (E x 6 int32), W ((4 (k+1)^2) x (k+1)^2, refine only), row_ptr and col (numpy)."""
    import numpy as np
    nl, nnz = ctypes.c_int64(), ctypes.c_int64()
    args = (int(nx), int(ny), int(nzc), int(nzf), int(order), int(bool(refine)))
    _check(lib().hyb_two_level_layout(*args, ctypes.byref(nl), ctypes.byref(nnz), None, None, None, None),
           "hyb_two_level_layout")
    r = 2 if refine else 1
    E = nx * ny * nzc + (r * nx) * (r * ny) * nzf
    nfn = (order + 1) ** 2
    ef = np.empty((E, 6), dtype=np.int32)
    W = np.zeros((4 * nfn, nfn)) if refine else None
    row_ptr = np.empty(nl.value + 1, dtype=np.int64)
    col = np.empty(nnz.value, dtype=np.int32)
    ptr = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
    _check(lib().hyb_two_level_layout(*args, ctypes.byref(nl), ctypes.byref(nnz), ptr(ef), ptr(W), ptr(row_ptr),
                                      ptr(col)), "hyb_two_level_layout")
    return dict(n_lambda=nl.value, elem_face=ef, W=W, row_ptr=row_ptr, col=col)


def hyb_barrier_selftest(absent, rounds, stream=None):
    """Status of the grid-barrier self-test (HYB_OK, or HYB_ERR_TIMEOUT when absent > 0)."""
    return lib().hyb_barrier_selftest(int(absent), int(rounds), _stream(stream))


def hyb_set_profiling(ctx, enable):
    return _check(lib().hyb_set_profiling(ctx.handle, int(bool(enable))), "hyb_set_profiling")


def hyb_get_profile(ctx):
    """{kernel class: (total ms, launches)} since profiling was enabled."""
    out = {}
    for name, cls in KERNEL_CLASSES.items():
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(lib().hyb_get_profile(ctx.handle, cls, ctypes.byref(ms), ctypes.byref(n)), "hyb_get_profile")
        out[name] = (ms.value, n.value)
    return out


def hyb_last_error_element(ctx):
    e = ctypes.c_int64()
    _check(lib().hyb_last_error_element(ctx.handle, ctypes.byref(e)), "hyb_last_error_element")
    return e.value


# ---------------------------------------------------------------- batches
def _ptr_array(tensors, name, allow_none=False):
    if tensors is None:
        if allow_none:
            return None
        raise TypeError(f"{name} required")
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        p = _ptr(t, f"{name}[{i}]")
        arr[i] = p.value if p is not None else None
    return arr


class Batch:
    """Owns a hyb_batch* (many problems); keeps the tensors it points to alive."""

    def __init__(self, handle, n, keep):
        self.handle = handle
        self.n = n
        self._keep = keep

    def context(self, i):
        """Borrowed single-problem context of problem i (owned by the batch)."""
        h = ctypes.c_void_p()
        _check(lib().hyb_batch_context(self.handle, int(i), ctypes.byref(h)), "hyb_batch_context")
        c = Context(h, None)
        c.close = lambda: None           # owned by the batch
        return c

    def close(self):
        if self.handle:
            lib().hyb_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hyb_setup_batch(meshes, orders, alphas, betas, precision=HYB_FP64, contrast_threshold=0.0, stream=None):
    """meshes: list of (vertices tensor, nx, ny, nz); orders: ints; alphas, betas: lists of tensors."""
    n = len(meshes)
    ms = (_Mesh * n)(*[_Mesh(int(nx), int(ny), int(nz), _ptr(v, "vertices")) for v, nx, ny, nz in meshes])
    ords = (ctypes.c_int * n)(*[int(k) for k in orders])
    h = ctypes.c_void_p()
    st = lib().hyb_setup_batch(n, ms, ords, _ptr_array(alphas, "alphas"), _ptr_array(betas, "betas"),
                               int(precision), float(contrast_threshold), _stream(stream), ctypes.byref(h))
    _check(st, "hyb_setup_batch")
    return Batch(h, n, (meshes, alphas, betas))


def hyb_assemble_reduced_batch(batch, loads, ess=None, check=True):
    st = lib().hyb_assemble_reduced_batch(batch.handle, _ptr_array(loads, "loads"), _ptr_array(ess, "ess", True))
    return _check(st, "hyb_assemble_reduced_batch") if check else st


def hyb_solve_reduced_batch(batch, rtol, maxit, lambdas, check=True):
    """Returns (iterations per problem, relative residual per problem, status)."""
    its = (ctypes.c_int * batch.n)()
    rr = (ctypes.c_double * batch.n)()
    st = lib().hyb_solve_reduced_batch(batch.handle, float(rtol), int(maxit), _ptr_array(lambdas, "lambdas"), its, rr)
    if check:
        _check(st, "hyb_solve_reduced_batch")
    return list(its), list(rr), st


def hyb_recover_batch(batch, lambdas, us, check=True):
    st = lib().hyb_recover_batch(batch.handle, _ptr_array(lambdas, "lambdas"), _ptr_array(us, "us"))
    return _check(st, "hyb_recover_batch") if check else st


def hyb_batch_step(batch, loads, rtol, maxit, lambdas, us, ess=None, check=True):
    """The whole batched step as one CUDA graph launch; returns (iterations, rel. residuals, status)."""
    its = (ctypes.c_int * batch.n)()
    rr = (ctypes.c_double * batch.n)()
    st = lib().hyb_batch_step(batch.handle, _ptr_array(loads, "loads"), _ptr_array(ess, "ess", True), float(rtol),
                              int(maxit), _ptr_array(lambdas, "lambdas"), _ptr_array(us, "us"), its, rr)
    if check:
        _check(st, "hyb_batch_step")
    return list(its), list(rr), st


def hyb_batch_step_kernels(batch):
    """(kernel nodes outside the PCG loop, kernel nodes per loop pass, PCG iterations per pass)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(lib().hyb_batch_step_kernels(batch.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "hyb_batch_step_kernels")
    return a.value, b.value, c.value


def hyb_batch_get_autotune(batch, order, path):
    """(multiple of resident CTAs or 0 = one CTA per element, grid) of an order bin and path."""
    m, g = ctypes.c_int(), ctypes.c_int()
    _check(lib().hyb_batch_get_autotune(batch.handle, int(order), int(path), ctypes.byref(m), ctypes.byref(g)),
           "hyb_batch_get_autotune")
    return m.value, g.value


def hyb_batch_set_pcg_fused(batch, on):
    """True (default): team-fused cooperative PCG per order; False: three launches per iteration."""
    return _check(lib().hyb_batch_set_pcg_fused(batch.handle, int(bool(on))), "hyb_batch_set_pcg_fused")


def hyb_batch_set_graphs(batch, on):
    """True (default): batched PCG chunks replay as one CUDA graph; False: direct launches."""
    return _check(lib().hyb_batch_set_graphs(batch.handle, int(bool(on))), "hyb_batch_set_graphs")


def hyb_batch_set_profiling(batch, enable):
    return _check(lib().hyb_batch_set_profiling(batch.handle, int(bool(enable))), "hyb_batch_set_profiling")


def hyb_batch_get_profile(batch):
    out = {}
    for name, cls in KERNEL_CLASSES.items():
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(lib().hyb_batch_get_profile(batch.handle, cls, ctypes.byref(ms), ctypes.byref(n)),
               "hyb_batch_get_profile")
        out[name] = (ms.value, n.value)
    return out
