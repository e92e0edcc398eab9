#!/usr/bin/env python
"""Benchmark: hybridized elements/s on one GB300, FP64 against mixed precision (per rank).

Default workload (the precision workload): a 96x96x96 hex mesh jittered by +-0.2h, RT_2
(108 dofs and 54 multipliers per element), alpha lognormal(0,1), beta/alpha log-uniform in
[1e-2, 1e6], N(0,1) load coefficients, zero normal essential data. A timed step is the
element phase a1-a6, hyb_assemble_reduced: per element the local matrix by quadrature
through the Piola map, the elimination and S_T, g_T, scattered without atomics into the CSR
reduced system. value = elements / that time, for the mixed-precision context (contrast
threshold autotuned by the library: elements up to beta/alpha = 1e6 eliminated in FP32 through
the hybridized mixed form, the reduced system, PCG and recovery FP64); the FP64 context is timed
the same way in the same run. Once per arm the rest of the path follows (diagonal PCG to
1e-12, back substitution, and for the mixed arm two FP64 refinement steps), timed per phase.
Relative errors of S, lambda and u of both arms are measured on an 8^3 mesh of the same recipe
against the CPU FP64 oracle's two routes (primal, and the hybridized mixed form that stays
accurate at this contrast). Inputs are resident in HBM; L2 is flushed (a 512 MiB write)
before every timed step, outside its events.

--config 2 (32^3 RT_1, FP64 full step), 4 (256-problem batch), 5 (64^3 RT_3, the precision
workload with RT_3) and softhard select the other workloads.

Output: one JSON line (rank 0). Under torchrun every rank runs an independent replica (the
path has no exchange step on one GPU per problem) and the slowest rank's time is reported;
value = all ranks' elements / that time.

--impl reference times the CPU FP64 oracle, as it stands, on the host cores: the element phase
of the same recipe on a bounded sample mesh, one worker process per core.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "32x32x32 jittered hex mesh (+-0.2h), RT_1, FP64 hybridization: assemble + diag-PCG 1e-12 + recover"
METRIC = "hybridized elements/s (FP64 GPU path)"
PRECISION_METRIC = "hybridized elements/s, FP64 vs mixed (same GB300), rel err vs FP64 oracle"
SAMPLE_N = 20          # oracle sample mesh of the 32^3 RT_1 workload (same recipe, 8000 elements)
# oracle element-phase samples of the precision workloads: (mesh size, element stride) for the
# one-core leg and the mesh size of the all-core leg (every core takes a strided share)
PHASE_SAMPLE = {3: dict(one=(12, 2), all_n=24), 5: dict(one=(6, 2), all_n=12)}
ERR_N = 8              # mesh size of the error measurement (same recipe as the workload)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rtol", type=float, default=1e-12)
    ap.add_argument("--maxit", type=int, default=100000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="mesh size override (parity / profiling runs)")
    ap.add_argument("--config", default="3",
                    help="workload: 3 (96^3 RT_2, default) and 5 (64^3 RT_3): the precision workloads, mixed and "
                         "FP64 arms in one run; 2 (32^3 RT_1, FP64 full step), 4 (256-problem batch), softhard "
                         "(Sec. 6.1's two-cube inclusion, natural boundary, --sh-order / --sh-p)")
    ap.add_argument("--single-arm", action="store_true",
                    help="configs 3/5: the one-arm full-step measurement (--precision) instead of both arms")
    ap.add_argument("--no-full", action="store_true", help="configs 3/5: skip the one-pass full-path timing")
    ap.add_argument("--no-amg", action="store_true",
                    help="configs 3/5: skip the full-path pass with the multigrid-preconditioned solves")
    ap.add_argument("--pc", choices=("jacobi", "amg"), default="jacobi",
                    help="configs 1/2/softhard: PCG preconditioner of the timed step (default: the diagonal)")
    ap.add_argument("--no-errors", action="store_true", help="configs 3/5: skip the error measurement")
    ap.add_argument("--sh-order", type=int, default=1, help="softhard: RT order (mesh 2n x 2n x n of the paper's table)")
    ap.add_argument("--sh-p", type=float, default=-8.0, help="softhard: mass coefficient 10^p in the inclusion")
    ap.add_argument("--batch-count", type=int, default=256, help="problems in the batched workload")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="fp64, or mixed: FP32 mixed-form elimination below the contrast threshold")
    ap.add_argument("--threshold", type=float, default=0.0,
                    help="mixed: contrast above which elements stay FP64 (0: autotuned by the library)")
    ap.add_argument("--mode", choices=["hyb", "sc"], default="hyb",
                    help="hybridization, or static condensation of the interior dofs (FP64 only)")
    ap.add_argument("--refine", type=int, default=None,
                    help="FP64 refinement steps after the solve (hyb_refine; for --precision mixed)")
    ap.add_argument("--refine-rtol", type=float, default=None,
                    help="inner PCG tolerance of a refinement step (configs 3/5: 1e-4, else 1e-6)")
    ap.add_argument("--mixed-rtol", type=float, default=1e-4,
                    help="configs 3/5: PCG tolerance of the mixed arm's first solve (its refinement steps then "
                         "run until ||C u|| / ||g|| <= --rtol, at most --refine steps)")
    ap.add_argument("--pcg", choices=["fused", "split"], default="fused",
                    help="PCG launch form: one cooperative launch per 64 iterations, or 3 launches per iteration")
    ap.add_argument("--assembly-only", action="store_true",
                    help="time only the element phase (assemble + recover with lambda = 0); per-config rates")
    args = ap.parse_args(argv)
    precision = str(args.config) in ("3", "5") and not args.single_arm
    if args.refine is None:          # the precision workloads refine the mixed arm (at most 4 steps)
        args.refine = 4 if precision else 0
    if args.refine_rtol is None:
        args.refine_rtol = 1e-4 if precision else 1e-6
    return args


# ---------------------------------------------------------------- distributed plumbing
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def dist_init(backend):
    import torch.distributed as dist
    rank, local, world = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return rank, local, world


def build_once(local):
    """Compile the library on the node's first rank only (the others would write the same
    files), then load it everywhere."""
    import __graft_entry__
    if local == 0:
        __graft_entry__.build()
    barrier()
    if local != 0:
        __graft_entry__.build()          # up to date by now: loads the library


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device="cpu") -> float:
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return x


def aggregate(units_per_rank: int, times_ms_rank: float, world: int, device="cpu"):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    t = max_over_ranks(times_ms_rank, device)
    return world * units_per_rank / (t * 1e-3), t


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.halt()
        return self.summarize(self.lines)

    def halt(self):
        """Stop sampling and keep the lines (summarize several samplers' lines together)."""
        if self.proc is None:
            return []
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return self.lines

    @staticmethod
    def summarize(lines):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle sample
def oracle_sample_step(n=SAMPLE_N):
    """One full step of the CPU FP64 oracle (hybridize, diag-PCG 1e-12, recover) on the n^3 sample."""
    from oracle.hybrid import Discretization, pcg_diag
    from paper_1801_08914_gb300 import inputs
    p = inputs.make_config(2, n=n)
    t0 = time.perf_counter()
    D = Discretization.from_problem(p)
    H, g = D.hybridize()
    lam, it, _ = pcg_diag(H, g, rtol=1e-12)
    D.recover(lam)
    return p.n_elem, time.perf_counter() - t0, it


def _oracle_worker(n, steps):
    out = []
    for _ in range(steps):
        E, t, it = oracle_sample_step(n)
        out.append((E, t, it))
    print(json.dumps(out))


def run_oracle_subprocess(n, steps):
    """Runs the oracle in a fresh single-threaded process (1 core, BLAS threads pinned to 1)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"import bench; bench._oracle_worker({n}, {steps})"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(steps=1):
    res = run_oracle_subprocess(SAMPLE_N, steps)
    E = sum(r[0] for r in res)
    t = sum(r[1] for r in res)
    return {"value": E / t, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": f"full step (hybridize, diag-PCG 1e-12 [{res[0][2]} it], recover) on the "
                      f"{SAMPLE_N}^3 mesh of the same recipe ({res[0][0]} elements), {len(res)} run(s), "
                      f"{t:.1f} s on 1 host core"}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "processor name"):
                    return ln.split(":", 1)[1].strip()
        with open("/proc/cpuinfo") as f:          # Arm: implementer / part numbers only
            parts = {}
            for ln in f:
                if ":" in ln:
                    k, v = (x.strip() for x in ln.split(":", 1))
                    if k in ("CPU implementer", "CPU part") and k not in parts:
                        parts[k] = v
            if parts:
                return "Arm " + ", ".join(f"{k} {v}" for k, v in parts.items())
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_phase_worker(cfg, n, first, stride, steps):
    """Element phase of the CPU FP64 oracle (A_T by quadrature, Cholesky, S_T = C A^-1 C^T, g_T,
    assembly of H and g: a1-a6) over elements first, first + stride, ... of the n^3 mesh of
    workload cfg, `steps` times; prints [(elements, seconds)] per step."""
    from oracle.hybrid import Discretization
    from paper_1801_08914_gb300 import inputs
    p = inputs.make_config(cfg, n=n)
    D = Discretization.from_problem(p)
    els = list(range(first, p.n_elem, stride))
    out = []
    for _ in range(steps):
        t0 = time.perf_counter()
        D.hybridize(elements=els)
        out.append((len(els), time.perf_counter() - t0))
    print(json.dumps(out))


def oracle_phase_rate(cfg, n, workers, stride=1, steps=1):
    """Runs `workers` single-threaded oracle processes at once (BLAS threads pinned to 1);
    worker w takes elements w, w + workers * stride, ... Returns per step (elements, seconds):
    all workers' elements over the slowest worker's time."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = [subprocess.Popen([sys.executable, "-c", f"import bench; bench._oracle_phase_worker("
                               f"{cfg}, {n}, {w * stride}, {workers * stride}, {steps})"],
                              cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for w in range(workers)]
    res = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    return [(sum(r[k][0] for r in res), max(r[k][1] for r in res)) for k in range(steps)]


def cpu_baseline_phase(cfg):
    """The oracle's element phase timed on the host cores: all cores (one worker process per
    core, strided shares of the all-core sample mesh) and one core (the one-core sample)."""
    smp = PHASE_SAMPLE[cfg]
    n1, m1 = smp["one"]
    E1, t1 = oracle_phase_rate(cfg, n1, 1, stride=m1)[0]
    C = host_cores()
    Ea, ta = oracle_phase_rate(cfg, smp["all_n"], C)[0]
    return {"value": Ea / ta, "unit": "elements/s", "cores": C, "kind": "oracle",
            "sample": f"element phase a1-a6 (hybridize: A_T, Cholesky, S_T, g_T, assembly) of the same recipe: "
                      f"all {C} cores on the {smp['all_n']}^3 mesh ({Ea} elements, {ta:.1f} s, one process per core), "
                      f"one core on every {m1}-th element of the {n1}^3 mesh ({E1} elements, {t1:.1f} s)",
            "one_core": {"value": E1 / t1, "unit": "elements/s", "cores": 1},
            "nproc": os.cpu_count(), "cpu_model": cpu_model()}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    if str(args.config) in ("3", "5"):
        cfg = int(args.config)
        W, K = args.warmup, args.steps
        n = PHASE_SAMPLE[cfg]["one"][0]
        C = host_cores()
        res = oracle_phase_rate(cfg, n, C, steps=W + K)[W:]
        E = sum(r[0] for r in res)
        t = sum(r[1] for r in res)
        v = E / t
        line = {"impl": "reference", "metric": PRECISION_METRIC, "value": v, "unit": "elements/s",
                "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": 1e3 * t / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": precision_workload_name(cfg),
                           "sample": f"{n}^3 mesh of the same recipe per step, element phase a1-a6, "
                                     f"one oracle process per core", "parallelism": "none"},
                "cpu_baseline": {"value": v, "unit": "elements/s", "cores": C, "kind": "oracle",
                                 "sample": f"element phase of the {n}^3 mesh of the same recipe per step",
                                 "nproc": os.cpu_count(), "cpu_model": cpu_model()},
                "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    W, K = args.warmup, args.steps
    res = run_oracle_subprocess(SAMPLE_N, W + K)[W:]
    E = sum(r[0] for r in res)
    t = sum(r[1] for r in res)
    v = E / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "elements/s", "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * t / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{SAMPLE_N}^3 mesh of the same recipe", "parallelism": "none"},
            "cpu_baseline": {"value": v, "unit": "elements/s", "cores": 1, "kind": "oracle",
                             "sample": f"{SAMPLE_N}^3 mesh, full step per sample"},
            "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def spmv_bytes(n, nnz, nfn):
    """Algorithmic bytes of one SpMV launch: the values (8 B per nonzero), the shared column
    list of each face (4 B per nonzero / rows per face), two row pointers per face, one read
    of the gathered vector and of p_i, one write of the result."""
    return 8 * nnz + 4 * nnz // nfn + 16 * (n // nfn) + 8 * n + 8 * n


# DRAM bytes per PCG iteration of pcg_fused_kernel from one ncu capture of the unchanged kernel,
# keyed by (config, mesh size, order); remove an entry when the kernel changes.
FUSED_TRAFFIC = {(2, 32, 1): 163.0e6}
# DRAM bytes per element of the FP64 element kernel (hybridization), from one ncu capture of
# a smaller mesh of the same order (profiles/element_kernel_fp64.md: 16^3 RT_3, 2,048 elements
# per launch, 23.6 MB read + 578.2 MB written); per-element work is uniform, so a launch's
# traffic is this times its elements
ELEMENT_TRAFFIC_PER_ELEMENT = {3: 293.8e3}
# DRAM bytes per element of the mixed element phase (mixed_load_kernel<k> + element_tiled_kernel<k>),
# from ncu captures of the unchanged kernels on a smaller mesh of the same order (RT_2: 32^3,
# colour 0, 16,384 elements: 18.28 + 10.72 MB and 205.49 + 1053.07 MB read + written;
# profiles/element_tiled_kernel_rt2_32cube_mixed.md)
MIXED_ELEMENT_TRAFFIC_PER_ELEMENT = {2: 78.6e3}


def pcg_iteration_flops(n, nnz):
    """FP64 flops of one PCG iteration: SpMV (2 per nonzero), p^T q (2n), x and r updates (4n),
    z = D^-1 r (n), r^T z and r^T r (4n), p = z + beta p (2n)."""
    return 2 * nnz + 13 * n


def pcg_iteration_bytes(n, nnz, nfn):
    """Algorithmic bytes of one PCG iteration: the SpMV's, then x, p, r, q, D^-1 read and x, r, z
    written by the update, p and z read and p written by the direction update."""
    return spmv_bytes(n, nnz, nfn) + 8 * 8 * n + 3 * 8 * n


def element_flops(k, condense=False):
    """Algorithmic FP64 flops of one element elimination (what the method needs, not what a
    kernel issues): sum-factorised A_T (6 blocks, 3 stages, mass + divergence terms),
    the load f = M c, Cholesky n^3/3, z = L^{-1} f, Y = L_bb^{-1} (n_b^3/3),
    Y^T Y (n_b^3/3), g = Y^T z_b. Static condensation stops the Cholesky before the face
    block (n^3/3 - n_b^3/3) and forms the condensed load f_b - L_bi z_i instead."""
    P, p, Q = k + 2, k + 1, k + 2
    nfn, ni = p * p, 3 * k * p * p
    nb = 6 * nfn
    n = ni + nb
    nc = P * p * p
    asm = 0
    for diag in (True, True, True, False, False, False):
        nja, njb = (P, p) if diag else (p, P)
        st1 = Q * Q * P * nja * Q * 2 * 2
        st2 = Q * P * nja * p * njb * Q * 2 * (1 if diag else 2)
        st3 = P * nja * p * njb * p * p * Q * 2 // (2 if diag else 1)
        asm += st1 + st2 + st3
    load = 2 * 3 * 2 * (nc * Q + nc * Q + nc * Q)
    if condense:
        return asm + load + n ** 3 // 3 - nb ** 3 // 3 + ni * ni + 2 * ni * nb
    chol = n ** 3 // 3 + n * n
    inv = nb ** 3 // 3
    gram = nb ** 3 // 3
    return asm + load + chol + inv + gram + nb * nb


def element_flops_mixed(k):
    """Algorithmic FP32 flops of one element on the mixed path (hybridized mixed form):
    alpha-mass by sum factorisation, G and G^{-1}, chol(M), Xd = L_M^{-1} D, Z = G^{-1} + Xd^T Xd,
    chol(Z), Y = L_M,bb^{-1}, P = Xd_b^T Y, V = L_Z^{-1} P, S = Y^T Y - V^T V, two FP32 solves."""
    P, p, Q = k + 2, k + 1, k + 2
    nfn, ni = p * p, 3 * k * p * p
    nb = 6 * nfn
    n = ni + nb
    nq = p ** 3
    mass = 0
    for diag in (True, True, True, False, False, False):
        nja, njb = (P, p) if diag else (p, P)
        mass += 2 * (Q * Q * P * nja * Q + Q * P * nja * p * njb * Q + P * nja * p * njb * p * p * Q // (2 if diag else 1))
    g = 2 * (Q * Q * p * p * Q + Q * p ** 4 * Q + p ** 6 * Q) + 2 * nq ** 3
    return (mass + g + n ** 3 // 3 + n * n * nq + nq * nq * n + nq ** 3 // 3 + nb ** 3 // 3 + nq * nb * nb
            + nq * nq * nb + nb ** 3 // 3 + nb * nb * nq + 2 * 2 * (2 * n * n + 2 * n * nq + 2 * nq * nq))


def measured_hbm_peak():
    """HBM copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the recipe's fallback 6800."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
    except (OSError, ValueError):
        return 6800.0


def recover_bytes_per_element(k):
    """Algorithmic DRAM bytes of one FP64 hybridization recovery: the interior rows of the stored
    factor (L_ii packed, L_bi), P = (A_T^{-1})_bb as a full square, z read, lambda_T gathered, u
    written."""
    p = k + 1
    ni, nb = 3 * k * p * p, 6 * p * p
    n = ni + nb
    return 8 * (ni * (ni + 1) // 2 + nb * ni + nb * nb + 2 * n + nb)


def recover_flops_per_element(k):
    """FP64 flops of one recovery: one FMA per stored double read (L_ii, L_bi, P)."""
    p = k + 1
    ni, nb = 3 * k * p * p, 6 * p * p
    return 2 * (ni * (ni + 1) // 2 + nb * ni + nb * nb)


def recover_roofline_of(k, E, rec_ms, hbm_peak, fp64_peak=None):
    """Roofline of the FP64 recovery phase (None when it did not run): its bytes against HBM and
    its FMAs against the FP64 peak; `bound` names the larger of the two times."""
    if not rec_ms or rec_ms <= 0:
        return None
    bpe, fpe = recover_bytes_per_element(k), recover_flops_per_element(k)
    gbs = E * bpe / (rec_ms * 1e-3) / 1e9
    out = {"kernel": f"recover_kernel<{k}> (FP64)", "bound": "hbm", "achieved": gbs, "peak": hbm_peak,
           "unit": "GB/s", "frac": gbs / hbm_peak, "algorithmic_bytes_per_element": bpe,
           "algorithmic_flops_per_element": fpe, "ms": rec_ms,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    if fp64_peak:
        tf = E * fpe / (rec_ms * 1e-3) / 1e12
        out["fp64_tflops"] = tf
        out["fp64_frac"] = tf / fp64_peak
        out["hbm_frac"] = gbs / hbm_peak
        if E * fpe / (fp64_peak * 1e12) > E * bpe / (hbm_peak * 1e9):
            out.update(bound="alu", achieved=tf, peak=fp64_peak, unit="TFLOP/s", frac=tf / fp64_peak,
                       peak_source="FP64 FMA throughput measured in this run (hyb_measure_fma_peak)")
    return out


def workload_name(cfg, p, args, mixed=False, sc=False, theta=0.0, n32=0, n64=0):
    """The workload as what it is, with its sizes: mesh, order, coefficients, precision, phases."""
    import math
    from paper_1801_08914_gb300 import inputs
    if cfg == "softhard":
        w = (f"soft-hard (Sec. 6.1): {p.nx}x{p.ny}x{p.nz} hex mesh, RT_{p.order}, mass coefficient "
             f"10^{args.sh_p:g} on [1/4,1/2]^3 u [1/2,3/4]^3, g = (1,1,1), natural boundary, FP64 hybridization: "
             f"assemble + diag-PCG {args.rtol:g} + recover")
    elif cfg == 2 and p.nx == 32:
        w = WORKLOAD
    else:
        c = inputs.CONFIGS[cfg]
        lo, hi = (math.log10(v) for v in c["contrast"])
        w = (f"{p.nx}x{p.ny}x{p.nz} jittered hex mesh (+-{c['gamma']:g}h), RT_{p.order}, alpha lognormal(0,1), "
             f"beta/alpha 10^U({lo:g},{hi:g}), N(0,1) loads, FP64 hybridization: assemble + diag-PCG "
             f"{args.rtol:g} + recover")
    if mixed:
        how = "autotuned " if args.threshold == 0 else ""
        w = w.replace("FP64", f"mixed FP32/FP64 ({how}threshold {theta:g}: {n32} FP32 + {n64} FP64 elements)", 1)
    if args.refine and not args.assembly_only:
        w += f", {args.refine} FP64 refinement steps"
    if getattr(args, "pc", "jacobi") == "amg" and not args.assembly_only:
        w = w.replace("diag-PCG", "AMG-PCG (aggregation multigrid V-cycle)")
    if sc:
        w = w.replace("hybridization", "static condensation")
    if args.assembly_only:
        w += " (element phase only: assemble + recover)"
    return w


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    rank, local, world = dist_init("nccl" if int(os.environ.get("WORLD_SIZE", 1)) > 1 else "gloo")
    torch.cuda.set_device(local)
    build_once(local)
    from paper_1801_08914_gb300 import hyb, inputs

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    cfg = str(args.config)
    if cfg == "softhard":
        p = inputs.soft_hard_problem(args.sh_order, args.sh_p, nz=args.n)
    else:
        cfg = int(cfg)
        p = inputs.make_config(cfg, n=args.n)
    tt = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    verts, alpha, beta, load = tt(p.vertices), tt(p.alpha), tt(p.beta), tt(p.load)
    mixed = args.precision == "mixed"
    ctx = hyb.hyb_setup(verts, p.nx, p.ny, p.nz, p.order, alpha, beta,
                        precision=hyb.HYB_MIXED if mixed else hyb.HYB_FP64,
                        contrast_threshold=args.threshold if mixed else 0.0)
    hyb.hyb_set_pcg_fused(ctx, args.pcg == "fused")
    if args.pc == "amg":
        hyb.hyb_set_preconditioner(ctx, hyb.HYB_PC_AMG, 2, 64)
    if p.natural:
        hyb.hyb_set_natural_bc(ctx, True)
    n64, n32, theta = ctx.precision_split()
    sz = ctx.sizes()
    E, n_loc, N, nnz = sz["n_elem"], sz["n_loc"], sz["n_lambda"], sz["nnz"]
    lam = torch.zeros(N, dtype=torch.float64, device=dev)
    u = torch.zeros(E, n_loc, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    iters = []
    jumps = []

    sc = args.mode == "sc"
    if sc and mixed:
        raise SystemExit("static condensation runs in FP64 contexts only")

    def step(load_dev):
        (hyb.staticcond_assemble if sc else hyb.hyb_assemble_reduced)(ctx, load_dev, None)
        if args.assembly_only:
            iters.append(0)
        else:
            it, rr, st = hyb.hyb_solve_reduced(ctx, args.rtol, args.maxit, lam, check=False)
            if st not in (hyb.HYB_OK,):
                raise hyb.HybError(st, "hyb_solve_reduced")
            iters.append(it)
        (hyb.staticcond_recover if sc else hyb.hyb_recover)(ctx, lam, u)
        if args.refine and not args.assembly_only:
            j, _ = hyb.hyb_refine(ctx, args.refine, args.refine_rtol, args.maxit, lam, u)
            jumps.append(j)

    for _ in range(args.warmup):
        step(load)
    torch.cuda.synchronize()
    fp64_peak = hyb.hyb_measure_fma_peak(True)            # TFLOP/s, this GPU, now
    fp32_peak = hyb.hyb_measure_fma_peak(False)
    hyb.hyb_set_profiling(ctx, True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters.clear()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        step(load)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    it_total = sum(iters)
    iters_timed = list(iters)
    ck = clocks.stop()
    prof = hyb.hyb_get_profile(ctx)
    hyb.hyb_set_profiling(ctx, False)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    value, ms_max = aggregate(E * args.steps, ms, world, device=dev)

    # end to end through the C ABI with host buffers: H2D of the load, D2H of u, every step
    load_h = torch.from_numpy(np.ascontiguousarray(p.load)).pin_memory()
    u_h = torch.empty(E, n_loc, dtype=torch.float64).pin_memory()
    load_d = torch.empty_like(load)
    ke = max(1, min(args.steps, 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    for _ in range(ke):
        load_d.copy_(load_h, non_blocking=True)
        step(load_d)
        u_h.copy_(u, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_value, _ = aggregate(E * ke, e2e_ms, world, device=dev)

    # roofline of the dominant kernel class
    spmv_ms, spmv_launches = prof["spmv"]
    fused_ms, fused_launches = prof["pcg_fused"]
    dominant = max(prof, key=lambda k: prof[k][0])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    per_launch_ms = spmv_ms / it_total if it_total and spmv_ms > 0 else float("nan")   # no-op launches charged to real ones
    nfn = (p.order + 1) ** 2
    gbs = spmv_bytes(N, nnz, nfn) / (per_launch_ms * 1e-3) / 1e9
    tflops = 2.0 * nnz / (per_launch_ms * 1e-3) / 1e12
    # On this part the SpMV's FMAs (2 nnz FP64 flops) take longer at the FP64 peak than its
    # bytes take at the HBM peak, so the FP64 pipe is the bound; the HBM view is reported too.
    roof = {"kernel": "spmv_face_kernel (CSR SpMV fused with p^T H p)", "bound": "alu", "achieved": tflops,
            "peak": fp64_peak, "unit": "TFLOP/s", "frac": tflops / fp64_peak,
            "peak_source": "FP64 FMA throughput measured in this run (hyb_measure_fma_peak)",
            "traffic": None, "algorithmic_flops_per_launch": 2 * nnz,
            "algorithmic_bytes_per_launch": spmv_bytes(N, nnz, nfn), "achieved_gbs": gbs, "hbm_peak_gbs": hbm_peak,
            "hbm_frac": gbs / hbm_peak,
            "hbm_peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
            "avg_launch_ms": per_launch_ms, "dominant_class": dominant,
            "fp64_peak_tflops": fp64_peak, "fp32_peak_tflops": fp32_peak}
    if fused_ms > 0 and it_total and args.pc == "amg":
        # one unit = one multigrid-preconditioned iteration: the PCG's own product and updates plus
        # the V-cycle's four level-0 products (Chebyshev degree 2 before and after the coarse
        # correction; the coarse levels are ~1/100 of level 0 and left out)
        it_ms = fused_ms / it_total
        flops_it = pcg_iteration_flops(N, nnz) + 4 * 2 * nnz
        bytes_it = pcg_iteration_bytes(N, nnz, nfn) + 4 * spmv_bytes(N, nnz, nfn)
        tf, gb = flops_it / (it_ms * 1e-3) / 1e12, bytes_it / (it_ms * 1e-3) / 1e9
        roof = {"kernel": "AMG-PCG iteration (face_kernel products of level 0, V-cycle, PCG updates)",
                "bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s", "frac": tf / fp64_peak,
                "peak_source": "FP64 FMA throughput measured in this run (hyb_measure_fma_peak)",
                "traffic": None, "unit_of_work": "one AMG-preconditioned PCG iteration",
                "algorithmic_flops_per_iteration": flops_it, "algorithmic_bytes_per_iteration": bytes_it,
                "achieved_gbs": gb, "hbm_peak_gbs": hbm_peak, "hbm_frac": gb / hbm_peak,
                "avg_iteration_ms": it_ms, "dominant_class": dominant,
                "fp64_peak_tflops": fp64_peak, "fp32_peak_tflops": fp32_peak}
    elif fused_ms > 0 and it_total:
        # one unit = one PCG iteration (SpMV + p^T q, the x/r/z update with r^T z and r^T r,
        # the direction update); a launch runs up to 64 of them
        it_ms = fused_ms / it_total
        flops_it, bytes_it = pcg_iteration_flops(N, nnz), pcg_iteration_bytes(N, nnz, nfn)
        tf, gb = flops_it / (it_ms * 1e-3) / 1e12, bytes_it / (it_ms * 1e-3) / 1e9
        roof = {"kernel": "pcg_fused_kernel (cooperative: SpMV + p^T H p, updates, reductions)", "bound": "alu",
                "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s", "frac": tf / fp64_peak,
                "peak_source": "FP64 FMA throughput measured in this run (hyb_measure_fma_peak)",
                "traffic": FUSED_TRAFFIC.get((cfg, p.nx, p.order)), "unit_of_work": "one PCG iteration",
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 64-iteration launch / 64 "
                                  "(profiles/pcg_fused_kernel_32cube_rt1.md)" if (cfg, p.nx, p.order) in FUSED_TRAFFIC
                                  else None,
                "iterations_per_launch": it_total / max(1, fused_launches),
                "algorithmic_flops_per_iteration": flops_it, "algorithmic_bytes_per_iteration": bytes_it,
                "achieved_gbs": gb, "hbm_peak_gbs": hbm_peak, "hbm_frac": gb / hbm_peak,
                "hbm_peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
                "avg_launch_ms": fused_ms / max(1, fused_launches), "avg_iteration_ms": it_ms,
                "dominant_class": dominant, "fp64_peak_tflops": fp64_peak, "fp32_peak_tflops": fp32_peak}
    launches = sum(v[1] for v in prof.values())
    phases = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps} for k, v in prof.items()}
    elem_ms = prof["element"][0] / args.steps
    elem_flops = element_flops(p.order, condense=args.mode == "sc")
    if not mixed:
        elem_tflops = E * elem_flops / (elem_ms * 1e-3) / 1e12 if elem_ms > 0 else None
        element_roofline = {"kernel": f"element_kernel<{p.order}> (FP64)", "bound": "alu",
                            "achieved": elem_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                            "frac": elem_tflops / fp64_peak if elem_tflops else None,
                            "algorithmic_flops_per_element": elem_flops}
        tpe = ELEMENT_TRAFFIC_PER_ELEMENT.get(p.order) if not sc else None
        el_launches = prof["element"][1] / args.steps
        element_roofline["traffic"] = tpe * E / el_launches if tpe and el_launches else None
        element_roofline["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per element x elements "
                                              "per launch (profiles/element_kernel_fp64.md)" if tpe else None)
    else:
        f32 = element_flops_mixed(p.order)
        # FP32 elements at the FP32 peak plus FP64 elements at the FP64 peak bound the phase from below
        t_min = (n32 * f32 / (fp32_peak * 1e12) + n64 * elem_flops / (fp64_peak * 1e12))
        element_roofline = {"kernel": f"element_tiled_kernel<{p.order}> (FP32) + element_kernel<{p.order}> (FP64)",
                            "bound": "alu", "achieved": (n32 * f32 + n64 * elem_flops) / (elem_ms * 1e-3) / 1e12,
                            "peak": (n32 * f32 + n64 * elem_flops) / t_min / 1e12 if t_min > 0 else None,
                            "unit": "TFLOP/s", "frac": t_min / (elem_ms * 1e-3) if elem_ms > 0 else None,
                            "algorithmic_flops_per_element_fp32": f32, "algorithmic_flops_per_element_fp64": elem_flops,
                            "elements_fp64": n64, "elements_fp32": n32, "contrast_threshold": theta}
    workload = workload_name(cfg, p, args, mixed, sc, theta, n32, n64)
    line = {
        "metric": (METRIC.replace("hybridized", "statically condensed") if sc else
                   METRIC.replace("FP64 GPU path", "mixed FP32/FP64 GPU path") if mixed else METRIC),
        "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": workload, "elements": E, "order": p.order, "n_loc": n_loc, "n_lambda": N,
                   "nnz": nnz, "pcg_rtol": args.rtol, "pcg_iterations": iters_timed[0] if iters_timed else None,
                   "parallelism": f"replicas x{world}", "l2": "flushed (512 MiB write) before each step"},
        "e2e": {"value": e2e_value, "unit": "elements/s", "h2d_bytes_per_step": int(p.load.nbytes),
                "d2h_bytes_per_step": int(E * n_loc * 8)},
        "gpu_launches": int(launches),
        "roofline": roof if not args.assembly_only else element_roofline,
        "element_roofline": element_roofline,
        "recover_roofline": (recover_roofline_of(p.order, E, prof["recover"][0] / args.steps, hbm_peak, fp64_peak)
                             if not mixed and not sc else None),
        "phases": phases,
        "assembly_elements_per_s": E / (elem_ms * 1e-3) if elem_ms > 0 else None,
        "pcg_ms_per_iteration": ((prof["spmv"][0] + prof["pcg_vector"][0] + prof["pcg_fused"][0]) / it_total
                                 if it_total else None),
        "reduced_dofs_per_s": (N * args.steps / ((prof["spmv"][0] + prof["pcg_vector"][0] + prof["pcg_fused"][0]) * 1e-3)
                               if it_total and prof["spmv"][0] + prof["pcg_vector"][0] + prof["pcg_fused"][0] > 0
                               else None),
        "clocks": ck,
        "wall_s": t_wall,
    }
    if args.refine and jumps:
        line["refinement"] = {"steps": args.refine, "inner_rtol": args.refine_rtol,
                              "jump_per_step": jumps[-1],
                              "note": "||C u|| / ||g|| before each FP64 refinement step and after the last"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline()
        except Exception as exc:  # reported, not fatal
            line["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def precision_workload_name(cfg, n=None):
    import math
    from paper_1801_08914_gb300 import inputs
    c = inputs.CONFIGS[cfg]
    n = c["n"] if n is None else n
    lo, hi = (math.log10(v) for v in c["contrast"])
    return (f"{n}x{n}x{n} jittered hex mesh (+-{c['gamma']:g}h), RT_{c['order']}, alpha lognormal(0,1), "
            f"beta/alpha 10^U({lo:g},{hi:g}), N(0,1) loads, zero essential BC; timed step: element phase a1-a6 "
            f"(hyb_assemble_reduced), mixed FP32/FP64 (autotuned contrast threshold) against FP64")


def _event_pair():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_element_phase(hyb, ctx, load, warmup, steps, flush, stream):
    """W untimed and K timed hyb_assemble_reduced calls (L2 flushed before each, outside the
    events); returns the per-step device times (ms) and the launch profile of the timed steps."""
    import torch
    for _ in range(warmup):
        hyb.hyb_assemble_reduced(ctx, load)
    torch.cuda.synchronize()
    hyb.hyb_set_profiling(ctx, True)
    ev = [_event_pair() for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        hyb.hyb_assemble_reduced(ctx, load)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    prof = hyb.hyb_get_profile(ctx)
    hyb.hyb_set_profiling(ctx, False)
    return [a.elapsed_time(b) for a, b in ev], prof


def time_full_path(hyb, ctx, load, lam, u, args, refine, flush, stream):
    """One pass of the whole path: assemble, diagonal PCG (rtol), recover, and `refine` FP64
    refinement steps; device time per phase (ms) from events on the library's stream."""
    import torch
    flush.fill_(7)
    ev = [_event_pair()[0] for _ in range(5)]
    hyb.hyb_set_profiling(ctx, True)
    rtol0 = args.mixed_rtol if refine else args.rtol
    ev[0].record(stream)
    hyb.hyb_assemble_reduced(ctx, load)
    ev[1].record(stream)
    it, rr, st = hyb.hyb_solve_reduced(ctx, rtol0, args.maxit, lam, check=False)
    if st != hyb.HYB_OK:
        raise hyb.HybError(st, "hyb_solve_reduced")
    ev[2].record(stream)
    hyb.hyb_recover(ctx, lam, u)
    ev[3].record(stream)
    jumps, steps = None, 0
    if refine:
        # FP64 refinement steps until the jump ||C u|| / ||g|| (the reduced residual with the exact
        # H) meets the FP64 arm's stopping rule rtol, at most `refine` steps
        jumps = refine_until(hyb, ctx, args, lam, u)
        steps = len(jumps) - 1
    ev[4].record(stream)
    torch.cuda.synchronize()
    prof = hyb.hyb_get_profile(ctx)
    hyb.hyb_set_profiling(ctx, False)
    ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
    total = sum(ms)
    E = ctx.sizes()["n_elem"]
    out = {"elements_per_s": E / (total * 1e-3), "ms": total, "assemble_ms": ms[0], "pcg_ms": ms[1],
           "pcg_iterations": it, "pcg_rel_res": rr, "recover_ms": ms[2],
           "launches": int(sum(v[1] for v in prof.values())),
           "pcg_ms_per_iteration": None}
    if refine:
        out.update(pcg_rtol=rtol0, refine_ms=ms[3], refine_steps=steps, refine_inner_rtol=args.refine_rtol,
                   jump_per_step=jumps, jump_target=args.rtol)
    pcg_dev = prof["spmv"][0] + prof["pcg_vector"][0] + prof["pcg_fused"][0]
    out["pcg_ms_per_iteration"] = ms[1] / it if it else None
    out["reduced_dofs_per_s"] = ctx.sizes()["n_lambda"] / (ms[1] * 1e-3) if ms[1] > 0 else None
    out["pcg_device_ms_all_solves"] = pcg_dev
    return out


def refine_until(hyb, ctx, args, lam, u):
    """FP64 refinement steps (hyb_refine) until ||C u|| / ||g|| <= args.rtol, at most args.refine.
    Each step's inner PCG tolerance is args.refine_rtol, loosened to half the reduction still
    needed when that is less (each step contracts the jump by about its inner tolerance).
    Returns the jump before the first step and after every step."""
    jumps = []
    j = None
    for _ in range(args.refine):
        inner = args.refine_rtol if j is None else max(args.refine_rtol, min(0.5, 0.5 * args.rtol / j))
        jj, _ = hyb.hyb_refine(ctx, 1, inner, args.maxit, lam, u)
        if not jumps:
            jumps.append(jj[0])
        jumps.append(jj[1])
        j = jj[1]
        if j <= args.rtol:
            break
    return jumps


def _err_oracle_worker(cfg, n, route, path):
    """CPU FP64 oracle on the n^3 mesh of workload cfg through one route (primal: A_T and its
    Cholesky; mixed: the hybridized mixed form of Sec. 3.2); saves H values, g, lambda, u."""
    import numpy as np
    from oracle.hybrid import Discretization, solve_sparse_direct
    from paper_1801_08914_gb300 import inputs
    p = inputs.make_config(cfg, n=n)
    D = Discretization.from_problem(p)
    H, g = D.hybridize_mixed() if route == "mixed" else D.hybridize()
    lam = solve_sparse_direct(H, g)
    u = D.recover_mixed(lam) if route == "mixed" else D.recover(lam)
    np.savez(path, val=H.data, indptr=H.indptr, indices=H.indices, g=g, lam=lam, u=u)


def start_error_oracle(cfg, n, tmpdir):
    env = dict(os.environ, OMP_NUM_THREADS="2", OPENBLAS_NUM_THREADS="2", MKL_NUM_THREADS="2")
    procs = {}
    for route in ("primal", "mixed"):
        path = os.path.join(tmpdir, f"oracle_{route}.npz")
        procs[route] = (subprocess.Popen([sys.executable, "-c", f"import bench; bench._err_oracle_worker("
                                          f"{cfg}, {n}, {route!r}, {path!r})"], cwd=ROOT, env=env,
                                         stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True), path)
    return procs


def measure_errors(hyb, cfg, n, args, oracle_procs, dev):
    """Relative errors of both GPU arms on the n^3 mesh of the workload against both oracle routes:
    S entry-wise per CSR row (max |S - S_o| / max |S_o| over a row, worst row) and norm-wise,
    lambda entry-wise (against max |lambda_o|) and norm-wise, u entry-wise per element and norm-wise."""
    import numpy as np
    import torch
    from paper_1801_08914_gb300 import inputs
    p = inputs.make_config(cfg, n=n)
    tt = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    gpu = {}
    for arm in ("mixed", "fp64"):
        mixed = arm == "mixed"
        ctx = hyb.hyb_setup(tt(p.vertices), p.nx, p.ny, p.nz, p.order, tt(p.alpha), tt(p.beta),
                            precision=hyb.HYB_MIXED if mixed else hyb.HYB_FP64, contrast_threshold=0.0)
        hyb.hyb_assemble_reduced(ctx, tt(p.load))
        red = {k: v.cpu().numpy() for k, v in hyb.hyb_export_reduced(ctx).items()}
        sz = ctx.sizes()
        lam = torch.zeros(sz["n_lambda"], dtype=torch.float64, device=dev)
        u = torch.zeros(sz["n_elem"], sz["n_loc"], dtype=torch.float64, device=dev)
        # the schedule of the timed full path: the mixed arm's first solve to --mixed-rtol, then
        # refinement steps until ||C u|| / ||g|| <= --rtol
        hyb.hyb_solve_reduced(ctx, args.mixed_rtol if mixed and args.refine else args.rtol, args.maxit, lam)
        hyb.hyb_recover(ctx, lam, u)
        g0 = dict(lam=lam.cpu().numpy().copy(), u=u.cpu().numpy().copy())
        jumps = refine_until(hyb, ctx, args, lam, u) if mixed and args.refine else []
        torch.cuda.synchronize()
        gpu[arm] = dict(red=red, lam=lam.cpu().numpy(), u=u.cpu().numpy(), unrefined=g0, split=ctx.precision_split(),
                        jumps=jumps)
        ctx.close()
    ref = {}
    for route, (pr, path) in oracle_procs.items():
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        ref[route] = dict(np.load(path))

    def rn(a, b):
        return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))

    def rinf(a, b):
        return float(np.abs(np.ravel(a) - np.ravel(b)).max() / np.abs(b).max())

    def rgroups(a, b, g):
        a, b = np.reshape(a, (-1, g)), np.reshape(b, (-1, g))
        return float((np.abs(a - b).max(1) / np.abs(b).max(1)).max())

    def rrows(a, b, rp):
        st = rp[:-1][rp[1:] > rp[:-1]]
        return float((np.maximum.reduceat(np.abs(a - b), st) / np.maximum.reduceat(np.abs(b), st)).max())

    nloc = p.load.shape[1]
    out = {"mesh": f"{n}^3 mesh of the same recipe ({p.n_elem} elements, "
                   f"{ref['primal']['g'].size} multipliers, seed {inputs.CONFIGS[cfg]['seed']})",
           "note": "S: worst CSR row of max|S - S_o| / max|S_o| (entry-wise) and ||S - S_o|| / ||S_o||; lambda: "
                   "max|d| / max|lambda_o| and norm-wise; u: worst element of max|d| / max|u_o| and norm-wise. "
                   "primal oracle = A_T = alpha M + beta K and its Cholesky (FP64, accurate to kappa(A_T) eps: "
                   "~1e-7 in u at this contrast); mixed-form oracle = Sec. 3.2's saddle route (FP64, accurate "
                   "at any contrast)",
           "solve": {"pcg_rtol": args.rtol, "mixed_first_rtol": args.mixed_rtol, "refine_max_steps": args.refine,
                     "refine_inner_rtol": args.refine_rtol}}
    for arm, gv in gpu.items():
        red = gv["red"]
        for route, r in ref.items():
            assert np.array_equal(red["row_ptr"], r["indptr"]) and np.array_equal(red["col"], r["indices"])
            e = {"S_row": rrows(red["val"], r["val"], r["indptr"]), "S_norm": rn(red["val"], r["val"]),
                 "g_inf": rinf(red["rhs"], r["g"]),
                 "lambda_inf": rinf(gv["lam"], r["lam"]), "lambda_norm": rn(gv["lam"], r["lam"]),
                 "u_element": rgroups(gv["u"], r["u"], nloc), "u_norm": rn(gv["u"], r["u"])}
            if arm == "mixed" and args.refine:
                e["u_element_before_refinement"] = rgroups(gv["unrefined"]["u"], r["u"], nloc)
                e["lambda_inf_before_refinement"] = rinf(gv["unrefined"]["lam"], r["lam"])
            out[f"{arm}_vs_{route}_oracle"] = e
    out["mixed_jumps"] = gpu["mixed"]["jumps"]
    out["mixed_split"] = {"fp64_elements": gpu["mixed"]["split"][0], "fp32_elements": gpu["mixed"]["split"][1],
                          "threshold": gpu["mixed"]["split"][2]}
    return out


def run_precision(args):
    """The precision workloads (96^3 RT_2; 64^3 RT_3): mixed and FP64 arms in one run."""
    import tempfile

    import numpy as np
    import torch

    rank, local, world = dist_init("nccl" if int(os.environ.get("WORLD_SIZE", 1)) > 1 else "gloo")
    torch.cuda.set_device(local)
    cfg = int(args.config)
    tmpdir = tempfile.mkdtemp(prefix="hyb_bench_")
    measure_err = rank == 0 and not args.no_errors
    oracle_procs = start_error_oracle(cfg, ERR_N, tmpdir) if measure_err else None
    build_once(local)
    from paper_1801_08914_gb300 import hyb, inputs

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    p = inputs.make_config(cfg, n=args.n)
    tt = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    verts, alpha, beta, load = tt(p.vertices), tt(p.alpha), tt(p.beta), tt(p.load)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    fp64_peak = hyb.hyb_measure_fma_peak(True)
    hbm_peak = measured_hbm_peak()
    fp32_peak = hyb.hyb_measure_fma_peak(False)
    clock_lines = []

    def sampled(fn):
        """Run fn with nvidia-smi sampling the clocks (only the timed regions are sampled)."""
        c = ClockSampler(local)
        c.start()
        try:
            return fn()
        finally:
            clock_lines.extend(c.halt())

    arms = {}
    for arm in ("mixed", "fp64"):
        mixed = arm == "mixed"
        t0 = time.perf_counter()
        ctx = hyb.hyb_setup(verts, p.nx, p.ny, p.nz, p.order, alpha, beta,
                            precision=hyb.HYB_MIXED if mixed else hyb.HYB_FP64,
                            contrast_threshold=args.threshold if mixed else 0.0)
        t_setup = time.perf_counter() - t0
        n64, n32, theta = ctx.precision_split()
        sz = ctx.sizes()
        E, n_loc, N, nnz = sz["n_elem"], sz["n_loc"], sz["n_lambda"], sz["nnz"]
        barrier()
        ms, prof = sampled(lambda: time_element_phase(hyb, ctx, load, args.warmup, args.steps, flush, stream))
        barrier()
        a = {"ms_steps": ms, "prof": prof, "setup_s": t_setup, "split": (n64, n32, theta)}
        if mixed:
            # end to end through the C ABI from host memory: pinned load -> device, the element
            # phase, the reduced right-hand side g -> pinned host buffer, every step
            load_h = torch.from_numpy(np.ascontiguousarray(p.load)).pin_memory()
            g_h = torch.empty(N, dtype=torch.float64).pin_memory()
            load_d = torch.empty_like(load)
            g_dev = torch.empty(N, dtype=torch.float64, device=dev)
            ke = max(1, min(args.steps, 5))
            e0, e1 = _event_pair()
            torch.cuda.synchronize()
            barrier()
            e0.record(stream)
            for _ in range(ke):
                load_d.copy_(load_h, non_blocking=True)
                hyb.hyb_assemble_reduced(ctx, load_d)
                hyb.hyb_export_rhs(ctx, g_dev)
                g_h.copy_(g_dev, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            a["e2e_ms"] = e0.elapsed_time(e1) / ke
            a["e2e_bytes"] = (int(p.load.nbytes), int(N * 8))
            del load_h, g_h, load_d, g_dev
        if not args.no_full:
            lam = torch.zeros(N, dtype=torch.float64, device=dev)
            u = torch.zeros(E, n_loc, dtype=torch.float64, device=dev)
            a["full"] = sampled(lambda: time_full_path(hyb, ctx, load, lam, u, args, args.refine if mixed else 0,
                                                       flush, stream))
            if not args.no_amg:
                # the same pass with the reduced solves preconditioned by the aggregation multigrid
                hyb.hyb_set_preconditioner(ctx, hyb.HYB_PC_AMG, 2, 64)
                a["full_amg"] = sampled(lambda: time_full_path(hyb, ctx, load, lam, u, args,
                                                               args.refine if mixed else 0, flush, stream))
                a["full_amg"]["amg_levels"] = hyb.hyb_amg_info(ctx)[1]
                hyb.hyb_set_preconditioner(ctx, hyb.HYB_PC_JACOBI, 2, 64)
            del lam, u
        ctx.close()
        torch.cuda.synchronize()
        arms[arm] = a
    ck = ClockSampler.summarize(clock_lines) if clock_lines else \
        {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}

    E = p.n_elem
    res = {}
    for arm, a in arms.items():
        ms = sum(a["ms_steps"])
        value, ms_max = aggregate(E * args.steps, ms, world, device=dev)
        res[arm] = (value, ms_max)
    value, ms_max = res["mixed"]
    fp64_value = res["fp64"][0]
    n64, n32, theta = arms["mixed"]["split"]
    f32 = element_flops_mixed(p.order)
    f64 = element_flops(p.order)
    pm = arms["mixed"]["prof"]
    el_ms_m = pm["element"][0] / args.steps
    el_launch_m = pm["element"][1] / args.steps
    # the dominant kernel of the timed step: the FP32 mixed-form element kernel (every element
    # of contrast <= the threshold). Its profile class also holds mixed_load_kernel (the FP64
    # load and G^{-1}, one launch before every element_tiled_kernel launch: ~10% of the phase in
    # the ncu launch list), so the unit is that pair of launches per colour: algorithmic flops
    # per pair over the pair's average time
    tflops = (n32 * f32 + n64 * f64) / (el_ms_m * 1e-3) / 1e12 if el_ms_m > 0 else None
    pairs = el_launch_m / 2 if n64 == 0 else el_launch_m
    roof = {"kernel": f"element_tiled_kernel<{p.order}> (FP32 mixed-form elimination"
                      + (f") + element_kernel<{p.order}> (FP64)" if n64 else ")"),
            "bound": "alu", "achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": tflops / fp32_peak if tflops else None,
            "peak_source": "FP32 FMA throughput measured in this run (hyb_measure_fma_peak: independent FMA "
                           "chains on every SM)",
            "traffic": MIXED_ELEMENT_TRAFFIC_PER_ELEMENT.get(p.order) and n64 == 0 and
                       MIXED_ELEMENT_TRAFFIC_PER_ELEMENT[p.order] * E / pairs,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per element x elements per launch "
                               "(profiles/element_tiled_kernel_rt2_32cube_mixed.md)"
                               if p.order in MIXED_ELEMENT_TRAFFIC_PER_ELEMENT else None),
            "algorithmic_flops_per_element": f32, "unit_of_work": "one colour: mixed_load_kernel + element_tiled_kernel",
            "elements_per_launch": E / pairs, "avg_launch_ms": el_ms_m / pairs,
            "fp64_peak_tflops": fp64_peak, "fp32_peak_tflops": fp32_peak}
    pf = arms["fp64"]["prof"]
    el_ms_f = pf["element"][0] / args.steps
    tf64 = E * f64 / (el_ms_f * 1e-3) / 1e12 if el_ms_f > 0 else None
    fp64_roof = {"kernel": f"element_kernel<{p.order}> (FP64)", "bound": "alu", "achieved": tf64, "peak": fp64_peak,
                 "unit": "TFLOP/s", "frac": tf64 / fp64_peak if tf64 else None,
                 "algorithmic_flops_per_element": f64, "avg_launch_ms": el_ms_f / max(1, pf["element"][1] / args.steps)}
    workload = precision_workload_name(cfg, p.nx)
    line = {
        "metric": PRECISION_METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload, "elements": E, "order": p.order, "n_loc": p.load.shape[1],
                   "step": "element phase a1-a6 of the mixed-precision context (hyb_assemble_reduced)",
                   "contrast_threshold": theta, "elements_fp32": n32, "elements_fp64": n64,
                   "parallelism": f"replicas x{world}", "l2": "flushed (512 MiB write) before each timed step"},
        "fp64": {"value": fp64_value, "unit": "elements/s", "ms_per_step": res["fp64"][1] / args.steps,
                 "step": "element phase a1-a6 of the FP64 context", "element_roofline": fp64_roof},
        "mixed_over_fp64": value / fp64_value,
        "e2e": {"value": E / (arms["mixed"]["e2e_ms"] * 1e-3), "unit": "elements/s",
                "h2d_bytes_per_step": arms["mixed"]["e2e_bytes"][0], "d2h_bytes_per_step": arms["mixed"]["e2e_bytes"][1],
                "path": "pinned host load -> hyb_assemble_reduced (mixed) -> reduced right-hand side to pinned host"},
        "gpu_launches": int(sum(v[1] for v in pm.values())),
        "roofline": roof,
        "clocks": ck,
        "setup_s": {arm: a["setup_s"] for arm, a in arms.items()},
    }
    if not args.no_full:
        line["full_step"] = {arm: a["full"] for arm, a in arms.items()}
        line["full_step"]["note"] = ("one pass of the whole path per arm: assemble, diagonal PCG to rtol, back "
                                     "substitution; the mixed arm adds FP64 refinement steps (hyb_refine)")
        fm, ff = arms["mixed"]["full"], arms["fp64"]["full"]
        line["full_step"]["mixed_over_fp64"] = fm["elements_per_s"] / ff["elements_per_s"]
        line["fp64"]["recover_roofline"] = recover_roofline_of(p.order, E, ff["recover_ms"], hbm_peak, fp64_peak)
        if "full_amg" in arms["mixed"]:
            am, af = arms["mixed"]["full_amg"], arms["fp64"]["full_amg"]
            line["full_step_amg"] = {"mixed": am, "fp64": af, "mixed_over_fp64": am["elements_per_s"] / af["elements_per_s"],
                                     "note": "the full_step pass with every reduced solve preconditioned by one V-cycle "
                                             "of the aggregation multigrid (HYB_PC_AMG: Chebyshev degree 2, coarsest "
                                             "<= 64 unknowns), its set-up inside the first solve"}
    if measure_err:
        try:
            line["errors"] = measure_errors(hyb, cfg, ERR_N, args, oracle_procs, dev)
        except Exception as exc:  # reported, not fatal
            line["errors"] = {"error": str(exc)[:300]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline_phase(cfg)
        except Exception as exc:  # reported, not fatal
            line["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def _oracle_batch_worker(problems, stride, first):
    """Element phase of the CPU FP64 oracle on every `stride`-th element (from `first`) of the given
    problems of the batched workload; prints {order: [elements, seconds]}."""
    from oracle.hybrid import Discretization
    from paper_1801_08914_gb300 import inputs
    out = {}
    for pidx in problems:
        p = inputs.batch_problem(pidx)
        D = Discretization.from_problem(p)
        els = list(range(first, p.n_elem, stride))
        t0 = time.perf_counter()
        D.hybridize(elements=els)
        dt = time.perf_counter() - t0
        e, t = out.get(p.order, (0, 0.0))
        out[p.order] = (e + len(els), t + dt)
    print(json.dumps(out))


def cpu_baseline_batch(probs_orders, E_per_order, sample=16):
    """The oracle's element phase on the batched workload: `sample` problems, every stride-th
    element, one worker process per core; per-order rates weighted by the batch's element counts."""
    from paper_1801_08914_gb300 import inputs
    C = host_cores()
    count = len(probs_orders)
    per = max(1, sample // 4)
    picks, seen = [], {k: 0 for k in range(4)}
    for pidx in range(count):                       # the first `per` problems of every order
        k = probs_orders[pidx]
        if seen[k] < per:
            picks.append(pidx)
            seen[k] += 1
    stride = 23
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs = [subprocess.Popen([sys.executable, "-c", f"import bench; bench._oracle_batch_worker({picks!r}, "
                               f"{stride * C}, {w * stride})"], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for w in range(C)]
    t_start = time.perf_counter()
    tot = {}
    tmax = 0.0
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        d = json.loads(out.strip().splitlines()[-1])
        for k, (e, t) in d.items():
            a = tot.get(int(k), [0, 0.0])
            tot[int(k)] = [a[0] + e, a[1] + t]
    wall = time.perf_counter() - t_start
    rate_core = {k: e / t for k, (e, t) in tot.items() if t > 0}      # elements per core-second, per order
    # all cores: the batch's per-order element counts at C times the one-core rates
    t_batch = sum(E_per_order[k] / (C * rate_core[k]) for k in E_per_order if E_per_order[k] and k in rate_core)
    E = sum(E_per_order.values())
    return {"value": E / t_batch if t_batch > 0 else None, "unit": "elements/s", "cores": C, "kind": "oracle",
            "sample": f"element phase a1-a6 of every {stride}-th element of problems {picks} (the first {per} of each order), "
                      f"{sum(e for e, _ in tot.values())} elements in {wall:.1f} s on {C} worker processes; "
                      f"per-order core rates {({k: round(v, 1) for k, v in rate_core.items()})} el/s weighted by the "
                      f"batch's elements per order",
            "nproc": os.cpu_count(), "cpu_model": cpu_model()}


def run_batch(args):
    """The batched workload: 256 independent problems, n ~ U{6..24}, k ~ U{0..3}, one batch.
    A timed step is hyb_batch_step: the element phase, the batched diagonal PCG (its loop a
    device-driven WHILE node) and the recovery of every problem as one CUDA graph launch."""
    import numpy as np
    import torch

    import __graft_entry__
    rank, local, world = dist_init("nccl" if int(os.environ.get("WORLD_SIZE", 1)) > 1 else "gloo")
    torch.cuda.set_device(local)
    build_once(local)
    from paper_1801_08914_gb300 import hyb, inputs

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    probs = inputs.batch_problems(count=args.batch_count)
    tt = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    verts = [tt(p.vertices) for p in probs]
    alphas = [tt(p.alpha) for p in probs]
    betas = [tt(p.beta) for p in probs]
    loads = [tt(p.load) for p in probs]
    mixed = args.precision == "mixed"
    t0 = time.perf_counter()
    b = hyb.hyb_setup_batch([(v, p.nx, p.ny, p.nz) for v, p in zip(verts, probs)], [p.order for p in probs],
                            alphas, betas, precision=hyb.HYB_MIXED if mixed else hyb.HYB_FP64,
                            contrast_threshold=args.threshold if mixed else 0.0)
    t_setup = time.perf_counter() - t0
    sizes = [b.context(i).sizes() for i in range(len(probs))]
    E = sum(s["n_elem"] for s in sizes)
    N = sum(s["n_lambda"] for s in sizes)
    nnz = sum(s["nnz"] for s in sizes)
    orders = [p.order for p in probs]
    tuned = {}
    for k in sorted(set(orders)):
        for path, name in ((0, "fp64"), (1, "fp32")):
            m, g = hyb.hyb_batch_get_autotune(b, k, path)
            if m or g or (path == 1) == mixed:
                tuned[f"RT_{k} {name}"] = ("one CTA per element" if m == 0 else
                                           f"{g} persistent CTAs ({m} x resident)")
    E_per_order = {k: sum(s["n_elem"] for s, o in zip(sizes, orders) if o == k) for k in range(4)}
    lams = [torch.zeros(s["n_lambda"], dtype=torch.float64, device=dev) for s in sizes]
    us = [torch.zeros(s["n_elem"], s["n_loc"], dtype=torch.float64, device=dev) for s in sizes]
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    its_last = []

    def step(lds):
        its, rr, st = hyb.hyb_batch_step(b, lds, args.rtol, args.maxit, lams, us, check=False)
        if st != hyb.HYB_OK:
            raise hyb.HybError(st, "hyb_batch_step")
        its_last[:] = its

    for _ in range(args.warmup):
        step(loads)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        step(loads)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = sum(a.elapsed_time(c) for a, c in ev)
    value, ms_max = aggregate(E * args.steps, ms, world, device=dev)
    outside, per_pass, ipp = hyb.hyb_batch_step_kernels(b)
    passes = max(1, -(-max(its_last) // ipp))
    launches_per_step = outside + passes * per_pass

    # per-phase attribution of the same work (the three calls, profiled per kernel class)
    hyb.hyb_batch_set_profiling(b, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hyb.hyb_assemble_reduced_batch(b, loads)
    e1.record(stream)
    its, rr, st = hyb.hyb_solve_reduced_batch(b, args.rtol, args.maxit, lams, check=False)
    hyb.hyb_recover_batch(b, lams, us)
    torch.cuda.synchronize()
    ck = clocks.stop()
    prof = hyb.hyb_batch_get_profile(b)
    hyb.hyb_batch_set_profiling(b, False)
    elem_ms = e0.elapsed_time(e1)
    pcg_ms = prof["spmv"][0] + prof["pcg_vector"][0] + prof["pcg_fused"][0]
    it_max = max(its)
    # roofline of the dominant phase, the batched PCG: one iteration of every problem moves the
    # SpMV's bytes plus the vector updates' (FP64: 2 nnz flops at the FP64 pipe's rate)
    fp64_peak = hyb.hyb_measure_fma_peak(True)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    it_ms = pcg_ms / it_max if it_max else float("nan")
    flops_it = sum(pcg_iteration_flops(s["n_lambda"], s["nnz"]) for s in sizes)
    bytes_it = sum(pcg_iteration_bytes(s["n_lambda"], s["nnz"], (o + 1) ** 2) for s, o in zip(sizes, orders))
    tf, gb = flops_it / (it_ms * 1e-3) / 1e12, bytes_it / (it_ms * 1e-3) / 1e9
    roof = {"kernel": "spmv_batch_kernel + update_batch_kernel + direction_batch_kernel (one batched PCG iteration)",
            "bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s", "frac": tf / fp64_peak,
            "peak_source": "FP64 FMA throughput measured in this run (hyb_measure_fma_peak)", "traffic": None,
            "unit_of_work": "one iteration of every problem (the last problems converge later: iterations of "
                            "converged problems are no-ops, so this is a lower bound)",
            "algorithmic_flops_per_iteration": flops_it, "algorithmic_bytes_per_iteration": bytes_it,
            "achieved_gbs": gb, "hbm_peak_gbs": hbm_peak, "hbm_frac": gb / hbm_peak, "avg_iteration_ms": it_ms}

    # end to end: pinned host loads -> the step -> every problem's u to pinned host memory
    loads_h = [torch.from_numpy(np.ascontiguousarray(p.load)).pin_memory() for p in probs]
    us_h = [torch.empty(s["n_elem"], s["n_loc"], dtype=torch.float64).pin_memory() for s in sizes]
    loads_d = [torch.empty_like(l) for l in loads]
    ke = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(ke):
        for h, d in zip(loads_h, loads_d):
            d.copy_(h, non_blocking=True)
        step(loads_d)
        for d, h in zip(us, us_h):
            h.copy_(d, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / ke
    line = {
        "metric": "hybridized elements/s, batched (" + ("mixed" if mixed else "FP64") + "), whole step",
        "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": f"{len(probs)} independent problems, n ~ U{{6..24}}, k ~ U{{0..3}}, jitter 0.2h, "
                               f"alpha lognormal(0,1), beta/alpha 10^U(-2,4), N(0,1) loads; timed step: "
                               f"hyb_batch_step (element phase, batched diagonal PCG to {args.rtol:g}, recovery) "
                               f"as one CUDA graph launch",
                   "elements": E, "n_lambda": N, "nnz": nnz, "problems_per_order": [orders.count(k) for k in range(4)],
                   "elements_per_order": [E_per_order[k] for k in range(4)], "pcg_iterations_max": max(its_last),
                   "setup_s": t_setup, "parallelism": f"replicas x{world}",
                   "l2": "flushed (512 MiB write) before each step"},
        "e2e": {"value": E / (e2e_ms * 1e-3), "unit": "elements/s",
                "h2d_bytes_per_step": int(sum(p.load.nbytes for p in probs)),
                "d2h_bytes_per_step": int(sum(s["n_elem"] * s["n_loc"] * 8 for s in sizes)),
                "path": "pinned host loads -> hyb_batch_step -> every problem's u to pinned host memory"},
        "gpu_launches": int(launches_per_step * args.steps),
        "autotuned_element_launches": tuned,
        "graph": {"kernel_nodes_outside_loop": outside, "kernel_nodes_per_loop_pass": per_pass,
                  "iterations_per_pass": ipp, "loop_passes_per_step": passes, "graph_launches_per_step": 1},
        "phases": {"element_ms": elem_ms, "pcg_ms": pcg_ms, "pcg_iterations_max": it_max,
                   "recover_ms": prof["recover"][0],
                   "note": "the same work through the three calls, profiled (CUDA events per launch class)"},
        "assembly_elements_per_s": E / (elem_ms * 1e-3) if elem_ms > 0 else None,
        "roofline": roof,
        "clocks": ck,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline_batch(orders, E_per_order)
        except Exception as exc:  # reported, not fatal
            line["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif str(args.config) == "4":
        run_batch(args)
    elif str(args.config) in ("3", "5") and not args.single_arm:
        run_precision(args)
    else:
        run_ours(args)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
