"""Error paths of the C ABI: every failure is a status code (no exception crosses the ABI),
and the two data-dependent ones name the element that caused them. The failing inputs are
caught by host checks or by the kernels' own checks (det J <= 0 at a corner or Gauss point,
a non-positive Cholesky pivot), which record the element and skip its work."""
import numpy as np
import pytest

from gpu_helpers import dev
from paper_1801_08914_gb300 import inputs

pytestmark = pytest.mark.gpu


def setup(p, **kw):
    from paper_1801_08914_gb300 import hyb
    return hyb.hyb_setup(dev(p.vertices), p.nx, p.ny, p.nz, p.order, dev(p.alpha), dev(p.beta), check=False, **kw)


def test_invalid_arguments_and_order():
    from paper_1801_08914_gb300 import hyb
    p = inputs.random_problem(2, 1, 0.2, 900, 1e-2, 1e2)
    for order in (-1, 4):
        q = inputs.random_problem(2, 1, 0.2, 900, 1e-2, 1e2)
        q.order = order
        ctx, st = setup(q)
        assert ctx is None and st == hyb.HYB_ERR_UNSUPPORTED_ORDER
    ctx, st = setup(p, precision=7)
    assert ctx is None and st == hyb.HYB_ERR_INVALID_ARG
    ctx, st = setup(p, precision=hyb.HYB_MIXED, contrast_threshold=-1.0)
    assert ctx is None and st == hyb.HYB_ERR_INVALID_ARG
    q = inputs.random_problem(2, 1, 0.2, 900, 1e-2, 1e2)
    q.nx = 0
    ctx, st = setup(q)
    assert ctx is None and st == hyb.HYB_ERR_INVALID_ARG


def test_calls_out_of_order_and_wrong_mode():
    import torch
    from paper_1801_08914_gb300 import hyb
    p = inputs.random_problem(3, 1, 0.2, 901, 1e-2, 1e2)
    ctx, st = setup(p)
    assert st == hyb.HYB_OK
    sz = ctx.sizes()
    lam = torch.zeros(sz["n_lambda"], dtype=torch.float64, device="cuda")
    u = torch.zeros(sz["n_elem"], sz["n_loc"], dtype=torch.float64, device="cuda")
    assert hyb.hyb_solve_reduced(ctx, 1e-12, 100, lam, check=False)[2] == hyb.HYB_ERR_INVALID_ARG
    assert hyb.hyb_recover(ctx, lam, u, check=False) == hyb.HYB_ERR_INVALID_ARG
    hyb.staticcond_assemble(ctx, dev(p.load))
    assert hyb.hyb_recover(ctx, lam, u, check=False) == hyb.HYB_ERR_INVALID_ARG     # SC assembled
    assert hyb.hyb_solve_reduced(ctx, 1e-12, 20000, lam, check=False)[2] == hyb.HYB_OK
    ctx.close()
    ctxm, st = setup(p, precision=hyb.HYB_MIXED, contrast_threshold=1e300)
    assert st == hyb.HYB_OK
    assert hyb.staticcond_assemble(ctxm, dev(p.load), check=False) == hyb.HYB_ERR_INVALID_ARG
    ctxm.close()


def test_inverted_element_is_a_mesh_error():
    """Moving an interior vertex beyond its neighbour inverts the elements around it:
    set-up reports HYB_ERR_MESH and names one of the eight elements sharing that vertex."""
    from paper_1801_08914_gb300 import hyb
    p = inputs.random_problem(4, 1, 0.0, 902, 1e-2, 1e2)
    n = p.nx
    i, j, l = 2, 2, 2
    v = i + (n + 1) * (j + (n + 1) * l)
    verts = np.array(p.vertices, copy=True).reshape(-1, 3)
    verts[v, 0] += 1.6 / n                            # past the vertex at i + 1
    p.vertices = verts.reshape(p.vertices.shape)
    ctx, st = setup(p)
    assert st == hyb.HYB_ERR_MESH and ctx is not None
    e = hyb.hyb_last_error_element(ctx)
    ei, ej, el = e % n, (e // n) % n, e // (n * n)
    assert ei in (i - 1, i) and ej in (j - 1, j) and el in (l - 1, l), e
    ctx.close()


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_non_spd_element_is_reported(precision, order):
    """alpha < 0 on one element makes its local matrix (and, in the mixed form, its alpha
    mass) indefinite: the factorisation (RT_3: the tiled look-ahead one) reports
    HYB_ERR_NOT_SPD with that element."""
    from paper_1801_08914_gb300 import hyb
    p = inputs.random_problem(3, order, 0.2, 903, 1e-2, 1e2)
    bad = 13
    p.alpha = np.array(p.alpha, copy=True)
    p.alpha[bad] = -1.0
    ctx, st = setup(p, precision=precision, contrast_threshold=1e300 if precision else 0.0)
    assert st == hyb.HYB_OK
    st = hyb.hyb_assemble_reduced(ctx, dev(p.load), check=False)
    assert st == hyb.HYB_ERR_NOT_SPD
    assert hyb.hyb_last_error_element(ctx) == bad
    assert "NOT_SPD" in hyb.status_string(st)
    ctx.close()


def test_pivot_rsqrt_accuracy():
    """The element kernels' pivot inverse square root (integer-built FP32 seed, one third-order
    correction) against the correctly rounded value computed on the host in extended
    precision: within 2 ulp of a double for positive normal inputs over the whole exponent
    range; the check flags zero, negatives, denormals, infinities and NaN."""
    import torch
    from paper_1801_08914_gb300 import hyb
    rng = np.random.default_rng(7)
    x = np.ldexp(rng.uniform(1.0, 2.0, 200000), rng.integers(-1021, 1023, 200000))
    x = np.concatenate([x, [1.0, 2.0, 4.0, 0.25, 3.999999999999, np.nextafter(4.0, 0.0), 2.2250738585072014e-308,
                            1.7976931348623157e308]])
    bad = np.array([0.0, -0.0, -1.0, 1e-310, np.inf, -np.inf, np.nan])
    xs = np.concatenate([x, bad])
    xd = torch.tensor(xs, dtype=torch.float64, device="cuda")
    out = torch.empty_like(xd)
    ok = torch.empty(xs.size, dtype=torch.int32, device="cuda")
    assert hyb.hyb_rsqrt_probe(xd, out, ok) == hyb.HYB_OK
    r, okh = out.cpu().numpy(), ok.cpu().numpy()
    assert np.all(okh[:x.size] == 1) and np.all(okh[x.size:] == 0)
    exact = 1.0 / np.sqrt(x.astype(np.longdouble))
    ulp = np.spacing(np.abs(exact.astype(np.float64)))
    err = np.abs(r[:x.size].astype(np.longdouble) - exact) / ulp
    print(f"pivot rsqrt: max error {float(err.max()):.2f} ulp over {x.size} inputs")
    assert float(err.max()) <= 2.0
