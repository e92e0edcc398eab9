"""The bench's workload descriptions (host logic only, no GPU): every workload it can run is
named by what it is, with its sizes, and the default one matches the reference arm's."""
import bench
from paper_1801_08914_gb300 import inputs


def test_workload_names():
    args = bench.parse_args(["--config", "2"])
    p = inputs.make_config(2)
    assert bench.workload_name(2, p, args) == bench.WORKLOAD
    for cfg, n in ((3, 6), (5, 4), (2, 8)):
        p = inputs.make_config(cfg, n=n)
        w = bench.workload_name(cfg, p, args)
        assert w.startswith(f"{n}x{n}x{n} jittered hex mesh") and f"RT_{p.order}" in w and "config" not in w
        wm = bench.workload_name(cfg, p, bench.parse_args(["--precision", "mixed", "--refine", "2"]), True, False, 1e6, 10, 2)
        assert "mixed FP32/FP64 (autotuned threshold 1e+06: 10 FP32 + 2 FP64 elements)" in wm and "2 FP64 refinement" in wm
        ws = bench.workload_name(cfg, p, bench.parse_args(["--mode", "sc", "--assembly-only"]), False, True)
        assert "static condensation" in ws and ws.endswith("(element phase only: assemble + recover)")
    p = inputs.soft_hard_problem(1, -8.0, nz=4)
    w = bench.workload_name("softhard", p, bench.parse_args(["--config", "softhard", "--sh-p", "-8"]))
    assert w.startswith("soft-hard (Sec. 6.1): 8x8x4 hex mesh, RT_1, mass coefficient 10^-8")


def test_recover_roofline_arithmetic():
    """The FP64 recovery per element reads the interior rows of the factor (L_ii packed: n_i(n_i+1)/2,
    L_bi: n_b n_i), P = (A^{-1})_bb as a full square (n_b^2), z (n) and lambda_T (n_b), writes u (n):
    8 bytes each, one FMA per stored double. RT_3: n_i = 144, n_b = 96; RT_0: n_i = 0, n_b = 6."""
    assert bench.recover_bytes_per_element(3) == 8 * (144 * 145 // 2 + 96 * 144 + 96 * 96 + 2 * 240 + 96)
    assert bench.recover_flops_per_element(3) == 2 * (144 * 145 // 2 + 96 * 144 + 96 * 96)
    assert bench.recover_bytes_per_element(0) == 8 * (36 + 12 + 6)
    r = bench.recover_roofline_of(3, 1000, 2.0, 6771.0)
    assert r["bound"] == "hbm" and abs(r["achieved"] - 1000 * bench.recover_bytes_per_element(3) / 2e-3 / 1e9) < 1e-9
    # with the FP64 peak known, the larger of the two times names the bound: at 1.25 TFLOP/s the
    # FMAs (one per 8 bytes) take longer than the bytes at 6771 GB/s
    r = bench.recover_roofline_of(3, 1000, 2.0, 6771.0, 1.25)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 1000 * bench.recover_flops_per_element(3) / 2e-3 / 1e12) < 1e-12
    assert abs(r["hbm_frac"] * 6771.0 - 1000 * bench.recover_bytes_per_element(3) / 2e-3 / 1e9) < 1e-6
    assert bench.recover_roofline_of(3, 1000, 0.0, 6771.0) is None


def test_precision_workload_defaults():
    """The default run is the precision workload (96^3 RT_2, contrast up to 1e6) with both arms and
    up to four refinement steps on the mixed arm; its name states the mesh, order, coefficients and step."""
    args = bench.parse_args([])
    assert str(args.config) == "3" and not args.single_arm and args.refine == 4 and args.refine_rtol == 1e-4
    w = bench.precision_workload_name(3)
    assert w.startswith("96x96x96 jittered hex mesh (+-0.2h), RT_2") and "beta/alpha 10^U(-2,6)" in w
    assert "element phase a1-a6" in w and "config" not in w
    assert bench.precision_workload_name(5).startswith("64x64x64 jittered hex mesh (+-0.2h), RT_3")
    assert bench.parse_args(["--config", "2"]).refine == 0
    assert bench.parse_args(["--config", "3", "--single-arm"]).refine == 0
