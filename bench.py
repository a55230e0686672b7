"""Benchmark of the PF-MP hot path on GB300.

Workload (one "step"): solve K x = b to a true relative residual of 1e-10 on a
16^3 x 32 lattice -- SU(3) links U = exp(i 0.5 H) with Gaussian H (seed 1),
Wilson-clover c_sw = 1.0, kappa = 0.130, even-odd preconditioned, Gaussian complex
right-hand side (seed 100) -- with the mixed-precision CG (FP32 iterations, FP64
reliable updates whose true residual is computed to FP64 accuracy in double-float).
Inputs are resident in HBM when the timed region starts; L2 is flushed (a 512 MiB
write) before every timed step.

Also reported on the same line:
  fp64_cg    the same solve with CG in FP64 throughout (the baseline the mixed solver
             is compared against), and the speedup;
  e2e        the same solve through the host-memory entry point pfmp_solve_host
             (H2D of b and D2H of x inside the timed region), wall clock;
  roofline   the stencil kernels (Wilson hop with fused clover epilogues, FP32) timed
             by CUDA events inside the library over R applications of K on a
             32^3 x 64 lattice (1.7 GB of FP32 operator data, far above the 129 MB L2),
             algorithmic bytes / time against the measured HBM copy bandwidth;
  cpu_baseline  one complete solve of the same system by the FP64 CPU oracle on the
             host's cores (wall clock, not extrapolated), with the CPU model.
With --impl reference the same oracle solve is the reference arm: one complete solve
split over the timed steps.  --cpu-full adds the oracle's single-thread solve and its
4^4 PF-MP trajectory.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank solves its own copy (replicas, weak scaling).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (16, 16, 16, 32)
EPS, KAPPA, CSW, TOL = 0.5, 0.130, 1.0, 1e-10
GAUGE_SEED, RHS_SEED = 1, 100
ROOF_DIMS = (32, 32, 32, 64)
METRIC = "PF-MP traj & solve time: mixed+learned vs FP64 CG at 1e-10; dslash HBM GB/s"
UNIT = "ms per solve (16^3x32 K x = b to 1e-10 true residual)"
WORKLOAD = "Dslash + solver at 16^3x32: eps=0.5 random SU(3), c_sw=1.0, kappa=0.130, Gaussian RHS, 1e-10"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ distributed plumbing
def dist_setup(n):
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if os.environ.get("PFMP_BENCH_GLOO") is None else "gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allmax(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle (CPU) timing
def cpu_model():
    """CPU model name and logical core count of this host."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if name is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        name = line.split(":", 1)[1].strip()
                        break
        except Exception:
            name = "unknown"
    return {"model": name, "nproc": os.cpu_count()}


class OracleCG:
    """The FP64 CPU oracle's CG on the benchmark system (the same K, b and stopping rule as
    the GPU solve: zero start, stop when the recursive residual is below 1e-10 |b|, then
    the true residual b - K x recomputed), advanced a given number of iterations at a
    time so that one full solve can be split over timed steps."""

    def __init__(self, threads=None):
        import torch

        import pfmp_inputs as pin
        from oracle.dirac import WilsonClover
        from oracle.lattice import Lattice, algebra_to_matrix, expi_hermitian

        # rank 0 runs the oracle alone: all host cores (torchrun sets OMP_NUM_THREADS=1)
        torch.set_num_threads(threads if threads is not None else (os.cpu_count() or 1))
        self.threads = torch.get_num_threads()
        lat = Lattice(DIMS, bc_t=-1)
        h = torch.tensor(pin.gauge_algebra(DIMS, GAUGE_SEED)).reshape(*lat.shape, 4, 8)
        U = expi_hermitian(algebra_to_matrix(h), EPS)
        self.W = WilsonClover(lat, U, KAPPA, CSW)
        _ = self.W.Ainv
        self.b = torch.tensor(pin.spinor(DIMS, RHS_SEED)).reshape(*lat.shape, 4, 3) * lat.even
        self.bb = (self.b.conj() * self.b).sum().real.item()
        self.restart()

    def restart(self):
        self.x = self.b.new_zeros(self.b.shape)
        self.r = self.b.clone()
        self.p = self.r.clone()
        self.rr = self.bb
        self.iters = 0

    def done(self):
        return self.rr < TOL * TOL * self.bb

    def advance(self, n):
        K = self.W.K
        for _ in range(n):
            if self.done():
                break
            Ap = K(self.p)
            a = self.rr / (self.p.conj() * Ap).sum().real.item()
            self.x = self.x + a * self.p
            self.r = self.r - a * Ap
            rn = (self.r.conj() * self.r).sum().real.item()
            self.p = self.r + (rn / self.rr) * self.p
            self.rr = rn
            self.iters += 1

    def true_residual(self):
        d = self.b - self.W.K(self.x)
        return math.sqrt((d.conj() * d).sum().real.item() / self.bb)


def oracle_iterations():
    """Iterations the oracle's FP64 CG needs on this system (stored by
    tests/golden/make_cg_iterations.py, which runs only the oracle)."""
    p = os.path.join(ROOT, "tests", "golden", "cg_iterations_16x16x16x32.json")
    if os.path.exists(p):
        with open(p) as f:
            return int(json.load(f)["iterations"])
    return 100


def oracle_full_solve(threads=None):
    """One full oracle FP64 CG solve to the 1e-10 true residual, wall clock."""
    cg = OracleCG(threads)
    t0 = time.perf_counter()
    cg.advance(100000)
    dt = time.perf_counter() - t0
    return {"ms": dt * 1e3, "iterations": cg.iters, "true_rel_res": cg.true_residual(), "threads": cg.threads}


def run_reference(args, rank, world):
    """The oracle's full FP64 CG solve of the benchmark system, split over the timed steps:
    every step advances the same CG by ceil(n / steps) iterations (n the oracle's stored
    iteration count) until it has converged; value = the sum of the step times, i.e. one
    complete solve measured, not extrapolated.  Warm-up steps run single iterations of a
    separate start that is discarded."""
    if rank != 0:
        return
    cg = OracleCG()
    for _ in range(args.warmup):
        cg.advance(1)
    cg.restart()
    per = max(1, -(-oracle_iterations() // max(args.steps, 1)))
    steps = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cg.advance(per)
        steps.append((time.perf_counter() - t0) * 1e3)
    while not cg.done():   # the stored count was short: finish the solve, timed too
        t0 = time.perf_counter()
        cg.advance(per)
        steps[-1] += (time.perf_counter() - t0) * 1e3
    value = sum(steps)
    res = cg.true_residual()
    sample = (f"one complete FP64 oracle CG solve of the 16^3x32 system ({cg.iters} iterations, true residual "
              f"{res:.2e}) split over the {args.steps} timed steps ({per} iterations per step); value = its total "
              f"wall time on {cg.threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(steps),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "implementation": "FP64 CPU oracle (PyTorch CPU ops)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cg.threads, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_full():
    """The oracle's CPU timings beyond the default line: the full FP64 CG solve on one
    thread and on every host core, and one config-1 PF-MP trajectory (4^4, order-8 filter,
    two-level 2MN 8 x 2 steps, tau 0.5, CG to 1e-12) on every core."""
    import torch

    import pfmp_inputs as pin
    from oracle.action import PFMP, PFMPParams
    from oracle.integrator import merge, trajectory, two_mn
    from oracle.lattice import Lattice, algebra_to_matrix, expi_hermitian

    ncores = os.cpu_count()
    out = {"cpu": cpu_model(), "solve_all_cores": oracle_full_solve(ncores), "solve_one_thread": oracle_full_solve(1)}
    torch.set_num_threads(ncores)
    dims = (4, 4, 4, 4)
    lat = Lattice(dims, bc_t=-1)
    U = expi_hermitian(algebra_to_matrix(torch.tensor(pin.gauge_algebra(dims, 1)).reshape(*lat.shape, 4, 8)), 0.3)
    act = PFMP(lat, PFMPParams(beta=5.5, kappa=0.120, kappa_h=0.110, csw=1.0, n=8, mu=1.2, nu=0.9, tol=1e-12))
    xi = [torch.tensor(pin.spinor(dims, 10 + i)).reshape(*lat.shape, 4, 3) * lat.even for i in range(3)]
    p0 = torch.tensor(pin.momenta(dims, 5)).reshape(*lat.shape, 4, 8)
    sched = merge([two_mn(8, 0.5), two_mn(16, 0.5)])
    t0 = time.perf_counter()
    r = trajectory(act, U, p0, xi, float(pin.uniform(6)[0]), [["polycorr", "hasen"], ["gauge", "det", "poly"]], sched)
    out["trajectory_4x4x4x4"] = {"ms": (time.perf_counter() - t0) * 1e3, "dH": r["dH"], "threads": ncores}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(args, rank, world):
    import torch

    import pfmp_inputs as pin
    from paper_1609_02652_gb300 import capi

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def l2_flush():
        with torch.cuda.stream(stream):
            flush.zero_()

    ctx = capi.pfmp_ctx_create(DIMS, -1, stream.cuda_stream)
    h = torch.tensor(np.ascontiguousarray(pin.gauge_algebra(DIMS, GAUGE_SEED)).reshape(-1), device="cuda")
    bcan = torch.tensor(np.ascontiguousarray(pin.spinor(DIMS, RHS_SEED)).view(np.float64).reshape(-1), device="cuda")
    torch.cuda.synchronize()
    capi.pfmp_gauge_from_algebra(ctx, h, EPS, capi.PFMP_DEVICE)
    op = capi.pfmp_op_create(ctx, KAPPA, CSW)
    nb64 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F64) // 8
    b = torch.zeros(nb64, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    capi.pfmp_spinor_pack(ctx, b, capi.PFMP_F64, bcan, capi.PFMP_DEVICE, 0)
    mixed = capi.SolverParams(method=capi.PFMP_SOLVER_CG_MIXED, tol=TOL, max_iter=20000, delta=args.delta,
                              check_every=args.chunk)
    plain = capi.SolverParams(method=capi.PFMP_SOLVER_CG64, tol=TOL, max_iter=20000, delta=0.1, check_every=args.chunk)

    def timed(params, steps, profile=False):
        times, infos = [], []
        for _ in range(steps):
            l2_flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(capi.pfmp_solve(op, params, x, b))
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times, infos

    for _ in range(args.warmup):
        capi.pfmp_solve(op, mixed, x, b)
    torch.cuda.synchronize()
    barrier(world)
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if "CUDA_VISIBLE_DEVICES" in os.environ else local
    clk = Clocks(gpu_index)
    launches0 = capi.pfmp_launch_count()
    t_mixed, info_mixed = timed(mixed, args.steps)
    launches = capi.pfmp_launch_count() - launches0
    clocks = clk.stop()
    # the same solve once more with the stencil launches bracketed by CUDA events
    # (profiling replaces the CUDA-graph replay by direct launches)
    capi.pfmp_profile_begin(ctx)
    capi.pfmp_solve(op, mixed, x, b)
    n_cg, cg_ms, cg_bytes = capi.pfmp_profile_end(ctx, capi.PFMP_KERNEL_CG_F32)
    n_df, df_ms, _ = capi.pfmp_profile_end(ctx, capi.PFMP_KERNEL_HOP_DF)
    torch.cuda.synchronize()
    barrier(world)
    ms_step = allmax(sum(t_mixed), world) / args.steps
    value = ms_step / world  # whole-job ms per solve (replicas)

    # the same solve with the stencil on FP16 storage, a few reliable-update thresholds
    half_res = {}
    for dl in (1e-1, 3e-2, 1e-2):
        hp = capi.SolverParams(method=capi.PFMP_SOLVER_CG_HALF, tol=TOL, max_iter=20000, delta=dl, check_every=8)
        capi.pfmp_solve(op, hp, x, b)
        t_h, info_h = timed(hp, 3)
        half_res[f"delta_{dl:g}"] = {"ms": statistics.median(t_h), "iterations": info_h[-1].iters,
                                     "reliable_updates": info_h[-1].reliable_updates,
                                     "true_rel_res": info_h[-1].true_rel_res}

    # FP64 CG baseline (same system, same flush)
    for _ in range(1):
        capi.pfmp_solve(op, plain, x, b)
    t_plain, info_plain = timed(plain, 3)
    fp64_ms = statistics.median(t_plain)
    # the FP64 stencil inside the FP64 CG against the measured FP64 FMA rate (its roofline):
    # 1320 flops of the hop and 2 x 288 of the two 6x6 clover blocks per output site
    capi.pfmp_profile_begin(ctx)
    capi.pfmp_solve(op, plain, x, b)
    n64, ms64, _ = capi.pfmp_profile_end(ctx, capi.PFMP_KERNEL_HOP_F64)
    vh = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] // 2
    fp64_rate = capi.pfmp_fma_rate(ctx, capi.PFMP_F64)
    fp32_rate = capi.pfmp_fma_rate(ctx, capi.PFMP_F32)
    stencil64 = n64 * vh * (1320 + 576) / (ms64 * 1e-3) / 1e12 if ms64 > 0 else None
    alu = {"fp64_fma_tflops": fp64_rate, "fp32_fma_tflops": fp32_rate,
           "fp64_stencil": {"launches": n64, "avg_us": ms64 * 1e3 / max(n64, 1), "tflops": stencil64,
                            "frac_of_fp64_fma": stencil64 / fp64_rate if stencil64 else None,
                            "flops_per_site": 1896},
           "note": "measured by pfmp_fma_rate (independent register FMA chains); the FP64 stencil of the "
                   "FP64 CG baseline, timed by CUDA events inside one FP64 solve"}

    # end to end through host memory (pinned), wall clock
    bh = torch.empty(DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3] * 24, dtype=torch.float64, pin_memory=True)
    bh.copy_(bcan.cpu())
    xh = torch.empty_like(bh).pin_memory()
    capi.pfmp_solve_host(op, mixed, xh.data_ptr(), bh.data_ptr())
    e2e = []
    for _ in range(args.steps):
        l2_flush()
        stream.synchronize()
        t0 = time.perf_counter()
        capi.pfmp_solve_host(op, mixed, xh.data_ptr(), bh.data_ptr())
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = allmax(statistics.mean(e2e), world) / world
    learn = None if args.no_learned else learned(capi, stream, l2_flush, args, ctx, op, b, x)
    traj = trajectory_4x4x4x4(capi, stream)
    traj_big = None if args.no_big_trajectory else {
        "fp64_forces": guarded(trajectory_16x16x16x32, capi, stream, capi.PFMP_F64),
        "fp32_forces": guarded(trajectory_16x16x16x32, capi, stream, capi.PFMP_F32)}
    prod = None if args.no_production else guarded(production_24x24x24x48, capi, stream, 1, 40, False)
    tuning = None if args.no_tuning else guarded(tuning_4x4x4x4, capi, stream)
    capi.pfmp_op_destroy(op)
    capi.pfmp_ctx_destroy(ctx)

    # roofline of the stencil kernels on a lattice far larger than L2
    roof, roof_h16 = roofline(capi, stream, l2_flush)
    batched = None if args.no_batched else batched_96(capi, stream, l2_flush, args)

    hbm, src = peaks()
    cg_gbs_l2 = cg_bytes / (cg_ms * 1e-3) / 1e9 if cg_ms > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": "16x16x16x32", "solver": "mixed CG, FP32 + FP64 reliable updates",
                   "l2": "flushed (512 MiB write) before every timed step", "parallelism": f"replicas x{world}"},
        "iterations": info_mixed[-1].iters, "reliable_updates": info_mixed[-1].reliable_updates,
        "true_rel_res": info_mixed[-1].true_rel_res,
        "roofline_h16": roof_h16,
        "half_cg": half_res,
        "fp64_cg": {"ms": fp64_ms, "iterations": info_plain[-1].iters, "true_rel_res": info_plain[-1].true_rel_res,
                    "speedup_mixed_vs_fp64": fp64_ms / ms_step},
        "e2e": {"value": e2e_ms, "unit": UNIT, "h2d_bytes_per_step": int(bh.numel() * 8),
                "d2h_bytes_per_step": int(xh.numel() * 8)},
        "roofline": roof,
        "learned": learn,
        "trajectory_4x4x4x4": traj,
        "trajectory_16x16x16x32": traj_big,
        "production_24x24x24x48": prod,
        "tuning_4x4x4x4": tuning,
        "batched": batched,
        "alu_rates": alu,
        "cg_in_solve": {"launches": n_cg, "avg_us": cg_ms * 1e3 / max(n_cg, 1), "algorithmic_gbs": cg_gbs_l2,
                        "kernel_ms": cg_ms, "df_residual_launches": n_df, "df_residual_ms": df_ms,
                        "note": "the FP32 CG iteration's four stencil kernels with the vector updates fused in "
                                "(bytes include the CG vectors); 16^3x32 FP32 working set (~75 MB) is L2-resident"},
        "gpu_launches": int(launches),
        "gpu_launches_note": "kernels launched by libpfmp in the timed steps, graph-replayed kernels included",
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        full = oracle_full_solve()
        line["cpu_baseline"] = {
            "value": full["ms"], "unit": UNIT, "cores": full["threads"], "kind": "oracle",
            "sample": f"one complete FP64 oracle CG solve of the same 16^3x32 system ({full['iterations']} "
                      f"iterations, true residual {full['true_rel_res']:.2e}), wall clock, not extrapolated",
            "cpu": cpu_model()}
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_96(capi, stream, l2_flush, args):
    """96 systems -- 32 each on 8^4, 12^3x24 and 16^3x32, eps = 0.4, kappa ~ U[0.120, 0.134]
    (seed 7), c_sw = 1.0, 1..8 Gaussian right-hand sides each (seed 8) -- solved to 1e-10 by
    the batched solver (one persistent launch), against the same solves one after another with the
    single-system mixed solver."""
    import torch

    import pfmp_inputs as pin

    lattices = [(8, 8, 8, 8)] * 32 + [(12, 12, 12, 24)] * 32 + [(16, 16, 16, 32)] * 32
    kappas = pin.uniform_range(7, 0.120, 0.134, 96)
    nrhs = [int(v) for v in pin.integers(8, 1, 8, 96)]
    ctxs, ops, bs, xs = [], [], [], []
    for s, dims in enumerate(lattices):
        ctx = capi.pfmp_ctx_create(dims, -1, stream.cuda_stream)
        h = torch.tensor(np.ascontiguousarray(pin.gauge_algebra(dims, 1000 + s)).reshape(-1), device="cuda")
        torch.cuda.synchronize()
        capi.pfmp_gauge_from_algebra(ctx, h, 0.4, capi.PFMP_DEVICE)
        del h
        op = capi.pfmp_op_create(ctx, float(kappas[s]), 1.0)
        n64 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F64) // 8
        for r in range(nrhs[s]):
            bc = torch.tensor(np.ascontiguousarray(pin.spinor(dims, 2000 + 10 * s + r)).view(np.float64).reshape(-1),
                              device="cuda")
            b = torch.zeros(n64, dtype=torch.float64, device="cuda")
            capi.pfmp_spinor_pack(ctx, b, capi.PFMP_F64, bc, capi.PFMP_DEVICE, 0)
            bs.append(b)
            xs.append(torch.zeros_like(b))
        ctxs.append(ctx)
        ops.append(op)
    prm = capi.SolverParams(method=capi.PFMP_SOLVER_CG_MIXED, tol=TOL, max_iter=20000, delta=args.delta,
                            check_every=args.chunk)
    B = capi.pfmp_batch_create(ops, nrhs)
    block, _ = capi.pfmp_batch_tune(B, args.chunk)
    capi.pfmp_batch_solve(B, prm, xs, bs)  # warm-up
    times = []
    for _ in range(2):
        l2_flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = capi.pfmp_batch_solve(B, prm, xs, bs)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    capi.pfmp_batch_destroy(B)
    worst = max(i.true_rel_res for i in infos)
    # the same solves one by one
    k = 0
    for s, op in enumerate(ops):
        for r in range(nrhs[s]):
            capi.pfmp_solve(op, prm, xs[k], bs[k])
            k += 1
    l2_flush()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    k = 0
    for s, op in enumerate(ops):
        for r in range(nrhs[s]):
            capi.pfmp_solve(op, prm, xs[k], bs[k])
            k += 1
    e1.record(stream)
    e1.synchronize()
    seq = e0.elapsed_time(e1)
    for op in ops:
        capi.pfmp_op_destroy(op)
    for ctx in ctxs:
        capi.pfmp_ctx_destroy(ctx)
    bt = min(times)
    return {"systems": 96, "rhs": int(sum(nrhs)), "batched_ms": bt, "sequential_ms": seq, "speedup": seq / bt,
            "block": block, "worst_true_rel_res": worst,
            "workload": "32x 8^4 + 32x 12^3x24 + 32x 16^3x32, eps=0.4, kappa~U[0.120,0.134], 1-8 rhs, 1e-10"}


def learned(capi, stream, l2_flush, args, ctx, op, b, x):
    """Mixed + learned: a [1,8,8,8,1] network (4 layers, 8 hidden channels) trained
    (residual loss, Adam, the project's FP32 kernels) on (b, K^{-1} b) pairs from the
    mixed solver on a held-out 8^3x16 gauge field (eps = 0.5, seed 2, same kappa and c_sw),
    then used as the FGCR preconditioner on the 16^3x32 benchmark system with its 8 -> 8
    layers on the tensor cores; the same network on the FP32 kernels and GCR (no network)
    alongside, and the time of one network application each way."""
    import torch

    import pfmp_inputs as pin

    tdims = (8, 8, 8, 16)
    tctx = capi.pfmp_ctx_create(tdims, -1, stream.cuda_stream)
    h = torch.tensor(np.ascontiguousarray(pin.gauge_algebra(tdims, 2)).reshape(-1), device="cuda")
    torch.cuda.synchronize()
    capi.pfmp_gauge_from_algebra(tctx, h, EPS, capi.PFMP_DEVICE)
    top = capi.pfmp_op_create(tctx, KAPPA, CSW)
    n64 = capi.pfmp_spinor_bytes(tctx, capi.PFMP_F64) // 8
    mixed = capi.SolverParams(method=capi.PFMP_SOLVER_CG_MIXED, tol=TOL, max_iter=20000, delta=1e-4, check_every=8)
    bs, xs = [], []
    t0 = time.perf_counter()
    for i in range(16):
        bc = torch.tensor(np.ascontiguousarray(pin.spinor(tdims, 3000 + i)).view(np.float64).reshape(-1), device="cuda")
        bb = torch.zeros(n64, dtype=torch.float64, device="cuda")
        capi.pfmp_spinor_pack(tctx, bb, capi.PFMP_F64, bc, capi.PFMP_DEVICE, 0)
        xx = torch.zeros_like(bb)
        capi.pfmp_solve(top, mixed, xx, bb)
        bs.append(bb)
        xs.append(xx)
    t_pairs = time.perf_counter() - t0
    ch = [1, 8, 8, 8, 1]
    net = capi.pfmp_nn_create(tctx, ch, capi.PFMP_F32)
    capi.pfmp_nn_set_weights(net, pin.nn_weights(ch, 5))
    t0 = time.perf_counter()
    loss = capi.pfmp_nn_train(net, bs, xs, steps=args.nn_steps, batch=4, lr=5e-3, op=top,
                              kind=capi.PFMP_NN_LOSS_RESIDUAL)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    shapes = [(9, co, ci, 4, 4) for ci, co in zip(ch[:-1], ch[1:])]
    w = capi.pfmp_nn_get_weights(net, shapes)
    capi.pfmp_nn_destroy(net)
    capi.pfmp_op_destroy(top)
    capi.pfmp_ctx_destroy(tctx)
    net = capi.pfmp_nn_create(ctx, ch, capi.PFMP_F32)
    capi.pfmp_nn_set_weights(net, w)
    prm = capi.SolverParams(method=0, tol=TOL, max_iter=20000, delta=1e-3, check_every=8, restart=16)
    out = {"train_lattice": "8x8x8x16 (held-out field, seed 2)", "pairs": 16, "pairs_s": t_pairs,
           "train_steps": args.nn_steps, "train_s": t_train, "final_train_loss": loss, "network": ch}
    for name, n, tc in (("fgcr_nn", net, 1), ("fgcr_nn_fp32_layers", net, 0), ("gcr", None, 0)):
        if n is not None:
            capi.pfmp_nn_set_tensor_cores(n, tc)
        capi.pfmp_solve_fgcr(op, n, prm, x, b)  # warm
        l2_flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = capi.pfmp_solve_fgcr(op, n, prm, x, b)
        e1.record(stream)
        e1.synchronize()
        out[name] = {"ms": e0.elapsed_time(e1), "iterations": info.iters, "cg_fallback_iterations": info.reliable_updates,
                     "true_rel_res": info.true_rel_res}
    # one network application on an FP32 even field, tensor-core and FP32 layers
    n32 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F32) // 4
    vin = torch.randn(n32, dtype=torch.float32, device="cuda")
    vout = torch.zeros_like(vin)
    for tc in (1, 0):
        capi.pfmp_nn_set_tensor_cores(net, tc)
        capi.pfmp_nn_apply(net, capi.PFMP_F32, vout, vin)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            capi.pfmp_nn_apply(net, capi.PFMP_F32, vout, vin)
        e1.record(stream)
        e1.synchronize()
        out["apply_ms_tensor_cores" if tc else "apply_ms_fp32_layers"] = e0.elapsed_time(e1) / 10
    capi.pfmp_nn_set_tensor_cores(net, 1)
    capi.pfmp_nn_destroy(net)
    return out


def learned_32x32x32x64(capi, stream, npairs=256, steps=300, ntherm=60):
    """The learned preconditioner at scale.  Training field: 24^3 x 48 thermalised by
    ntherm pure-gauge HMC trajectories at beta = 5.5 (seed 5), Wilson-clover c_sw = 1.6;
    kappa: the lightest of 0.125 .. 0.135 (steps of 0.0025) at which the mixed CG reaches
    1e-10 within 20000 iterations on it.  npairs (b, x = K^{-1} b) pairs from the mixed
    solver (Gaussian b), a [1, 8, 8, 8, 1] network trained on them (residual loss, Adam,
    batch 4).  Evaluation field: 32^3 x 64 thermalised the same way (seed 6), a Gaussian
    right-hand side: FGCR with the network (tensor-core layers), GCR without it, the mixed
    CG and the FP64 CG, all to a 1e-10 FP64 true residual; wall times by CUDA events."""
    import torch

    import pfmp_inputs as pin

    csw, tol = 1.6, 1e-10
    out = {"csw": csw, "beta": 5.5}
    mixed = capi.SolverParams(method=capi.PFMP_SOLVER_CG_MIXED, tol=tol, max_iter=20000, delta=1e-4, check_every=16)
    # ---- training field and the kappa scan
    tdims = (24, 24, 24, 48)
    tctx = capi.pfmp_ctx_create(tdims, -1, stream.cuda_stream)
    out["train_thermalisation"] = thermalise(capi, tctx, tdims, ntherm, 5)
    n64 = capi.pfmp_spinor_bytes(tctx, capi.PFMP_F64) // 8

    def rhs(ctx, dims, seed, n):
        bc = torch.tensor(np.ascontiguousarray(pin.spinor(dims, seed)).view(np.float64).reshape(-1), device="cuda")
        bb = torch.zeros(n, dtype=torch.float64, device="cuda")
        capi.pfmp_spinor_pack(ctx, bb, capi.PFMP_F64, bc, capi.PFMP_DEVICE, 0)
        return bb

    b0 = rhs(tctx, tdims, 7000, n64)
    x0 = torch.zeros_like(b0)
    scan, kappa = [], None
    for kap in (0.125, 0.1275, 0.130, 0.1325, 0.135):
        op = capi.pfmp_op_create(tctx, kap, csw)
        t0 = time.perf_counter()
        info = capi.pfmp_solve(op, mixed, x0, b0, raise_on_error=False)
        scan.append({"kappa": kap, "iterations": info.iters, "status": info.status, "s": time.perf_counter() - t0,
                     "true_rel_res": info.true_rel_res})
        capi.pfmp_op_destroy(op)
        if info.status == 0:
            kappa = kap
        else:
            break
    out["kappa_scan"] = scan
    out["kappa"] = kappa
    if kappa is None:
        capi.pfmp_ctx_destroy(tctx)
        return out
    top = capi.pfmp_op_create(tctx, kappa, csw)
    bs, xs = [], []
    t0 = time.perf_counter()
    for i in range(npairs):
        bb = rhs(tctx, tdims, 8000 + i, n64)
        xx = torch.zeros_like(bb)
        capi.pfmp_solve(top, mixed, xx, bb)
        bs.append(bb)
        xs.append(xx)
    torch.cuda.synchronize()
    out["pairs"] = npairs
    out["pairs_s"] = time.perf_counter() - t0
    ch = [1, 8, 8, 8, 1]
    net = capi.pfmp_nn_create(tctx, ch, capi.PFMP_F32)
    capi.pfmp_nn_set_weights(net, pin.nn_weights(ch, 5))
    t0 = time.perf_counter()
    loss = capi.pfmp_nn_train(net, bs, xs, steps=steps, batch=4, lr=5e-3, op=top, kind=capi.PFMP_NN_LOSS_RESIDUAL)
    torch.cuda.synchronize()
    out.update({"train_steps": steps, "train_s": time.perf_counter() - t0, "final_train_loss": loss, "network": ch})
    w = capi.pfmp_nn_get_weights(net, [(9, co, ci, 4, 4) for ci, co in zip(ch[:-1], ch[1:])])
    capi.pfmp_nn_destroy(net)
    del bs, xs
    capi.pfmp_op_destroy(top)
    capi.pfmp_ctx_destroy(tctx)
    # ---- evaluation at 32^3 x 64
    edims = (32, 32, 32, 64)
    ctx = capi.pfmp_ctx_create(edims, -1, stream.cuda_stream)
    try:
        out["eval_thermalisation"] = thermalise(capi, ctx, edims, ntherm, 6)
        op = capi.pfmp_op_create(ctx, kappa, csw)
        n64 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F64) // 8
        b = rhs(ctx, edims, 9000, n64)
        x = torch.zeros_like(b)
        net = capi.pfmp_nn_create(ctx, ch, capi.PFMP_F32)
        capi.pfmp_nn_set_weights(net, w)
        capi.pfmp_nn_set_tensor_cores(net, 1)

        def timed(fn):
            fn()  # warm
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = fn()
            e1.record(stream)
            e1.synchronize()
            return {"ms": e0.elapsed_time(e1), "iterations": info.iters, "true_rel_res": info.true_rel_res,
                    "status": info.status}

        prm = capi.SolverParams(method=0, tol=tol, max_iter=20000, delta=1e-3, check_every=8, restart=16)
        plain = capi.SolverParams(method=capi.PFMP_SOLVER_CG64, tol=tol, max_iter=40000, delta=0.1, check_every=16)
        res = {"fgcr_nn": timed(lambda: capi.pfmp_solve_fgcr(op, net, prm, x, b, raise_on_error=False)),
               "gcr": timed(lambda: capi.pfmp_solve_fgcr(op, None, prm, x, b, raise_on_error=False)),
               "mixed_cg": timed(lambda: capi.pfmp_solve(op, mixed, x, b, raise_on_error=False)),
               "fp64_cg": timed(lambda: capi.pfmp_solve(op, plain, x, b, raise_on_error=False))}
        n32 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F32) // 4
        vin = torch.randn(n32, dtype=torch.float32, device="cuda")
        vout = torch.zeros_like(vin)
        capi.pfmp_nn_apply(net, capi.PFMP_F32, vout, vin)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            capi.pfmp_nn_apply(net, capi.PFMP_F32, vout, vin)
        e1.record(stream)
        e1.synchronize()
        res["network_apply_ms"] = e0.elapsed_time(e1) / 5
        res["speedup_fgcr_nn_vs_fp64_cg"] = res["fp64_cg"]["ms"] / res["fgcr_nn"]["ms"]
        res["speedup_mixed_cg_vs_fp64_cg"] = res["fp64_cg"]["ms"] / res["mixed_cg"]["ms"]
        out["eval_32x32x32x64"] = res
        capi.pfmp_nn_destroy(net)
        capi.pfmp_op_destroy(op)
    finally:
        capi.pfmp_ctx_destroy(ctx)
    return out


def guarded(fn, *a):
    """A secondary measurement that must not take the headline line down with it."""
    try:
        return fn(*a)
    except Exception as e:  # reported in the JSON line instead
        return {"error": f"{type(e).__name__}: {e}"}


def trajectory_16x16x16x32(capi, stream, force_prec=0):
    """One PF-MP trajectory on the paper's lattice size, 16^3x32 (synthetic field eps 0.3,
    seed 1; beta 5.5, c_sw 1, kappa 0.125, kappa' 0.110, order-8 filter, (mu, nu) = (1.2,
    0.9)), the action's CG in mixed precision and the multi-shift in FP64, all solves to
    1e-10 (force_prec = PFMP_F32: the MD forces in FP32 with solves to 1e-6); 2-level 2MN,
    2 coarse (correction + Hasenbusch ratio) x 4 fine (gauge, clover determinant,
    filter) steps over tau = 0.1.  Wall time of the whole trajectory
    (heatbath, both Hamiltonians, MD, accept/reject) with per-term K counts and forces."""
    import torch

    import pfmp_inputs as pin

    dims = (16, 16, 16, 32)
    V = 16 * 16 * 16 * 32
    ctx = capi.pfmp_ctx_create(dims, -1, stream.cuda_stream)
    h = torch.tensor(np.ascontiguousarray(pin.gauge_algebra(dims, 1)).reshape(-1), device="cuda")
    torch.cuda.synchronize()
    capi.pfmp_gauge_from_algebra(ctx, h, 0.3, capi.PFMP_DEVICE)
    d = capi.ActionDef()
    d.beta, d.csw, d.nkappa = 5.5, 1.0, 2
    d.kappa[0], d.kappa[1] = 0.125, 0.110
    d.mu, d.nu, d.tol, d.max_iter = 1.2, 0.9, 1e-10, 20000
    d.solver = capi.PFMP_SOLVER_CG_MIXED
    d.force_prec, d.md_tol = force_prec, (1e-6 if force_prec == capi.PFMP_F32 else 0.0)
    capi.pfmp_action_scheme(capi.PFMP_SCHEME_PFMP, 0, 8, d)
    A = capi.pfmp_action_create_def(ctx, d)
    lam = 0.1931833275037836
    T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(2, 0.1, lam), capi.pfmp_schedule_2mn(4, 0.1, lam)])
    xi = np.concatenate([np.ascontiguousarray(pin.spinor(dims, 10 + i)).view(np.float64).reshape(-1) for i in range(3)])
    mom = np.ascontiguousarray(pin.momenta(dims, 5)).reshape(-1)
    levels = [1, 1, 1, 0, 0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = capi.pfmp_trajectory(A, T, S, levels, mom, xi, float(pin.uniform(6)[0]))
    ms = (time.perf_counter() - t0) * 1e3
    names = ["gauge", "det", "filter", "filtercorr", "ratio"]
    out = {"ms": ms, "dH": info.dH, "accepted": bool(info.accepted), "k_apply": int(info.k_apply),
           "force_evals": int(info.force_evals), "steps": len(T), "sites": V,
           "per_term": {n: {"k_apply": int(info.k_apply_term[t]), "forces": int(info.nforce[t]),
                            "fmax": info.fmax[t], "favg": info.favg[t]} for t, n in enumerate(names)}}
    capi.pfmp_action_destroy(A)
    capi.pfmp_ctx_destroy(ctx)
    return out


def thermalise(capi, ctx, dims, ntherm, seed, beta=5.5):
    """A random start (U = exp(i H), H from seed) thermalised by ntherm pure-gauge HMC
    trajectories at beta (2MN, 10 steps over tau = 1; the first half accepted
    unconditionally, the rest with the Metropolis test); returns the plaquette history
    (thinned) and the acceptance of the second half."""
    import torch

    import pfmp_inputs as pin

    lam = 0.1931833275037836
    h = torch.tensor(np.ascontiguousarray(pin.gauge_algebra(dims, seed)).reshape(-1), device="cuda")
    torch.cuda.synchronize()
    capi.pfmp_gauge_from_algebra(ctx, h, 1.0, capi.PFMP_DEVICE)
    del h
    dq = capi.ActionDef()
    dq.beta, dq.csw, dq.nkappa = beta, 0.0, 1   # no fermion term: no clover needed
    dq.kappa[0] = 0.1
    dq.mu, dq.nu, dq.tol, dq.max_iter = 1.2, 0.9, 1e-10, 20000
    dq.nterms = 1
    dq.term[0] = capi.Term(capi.PFMP_KIND_GAUGE, 0, 0, 0, 0)
    Aq = capi.pfmp_action_create_def(ctx, dq)
    Tq, Sq = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(10, 1.0, lam)])
    plaq, accq = [capi.pfmp_plaquette(ctx)], []
    t0 = time.perf_counter()
    try:
        for k in range(ntherm):
            u = 0.0 if k < ntherm // 2 else float(pin.uniform(1000 * seed + 31000 + k)[0])
            mom = np.ascontiguousarray(pin.momenta(dims, 1000 * seed + 30000 + k)).reshape(-1)
            info = capi.pfmp_trajectory(Aq, Tq, Sq, [0], mom, np.zeros(1), u)
            plaq.append(info.plaquette)
            if k >= ntherm // 2:
                accq.append(int(info.accepted))
    finally:
        capi.pfmp_action_destroy(Aq)
    return {"trajectories": ntherm, "s": time.perf_counter() - t0, "beta": beta,
            "acceptance": float(np.mean(accq)) if accq else None,
            "plaquette_history": plaq[:: max(1, len(plaq) // 25)] + [plaq[-1]]}


PROD_DIMS = (24, 24, 24, 48)
PROD = dict(beta=5.5, csw=1.6, kappa=0.134, kappa1=0.120, kappa2=0.130, p1=12, p2=64, steps=(60, 24, 10, 4), tau=1.0)


def production_24x24x24x48(capi, stream, ntraj=10, ntherm=100, reversibility=True, force_prec=None):
    """The production PF-MP run at 24^3 x 48 (Nf = 2 Wilson-clover c_sw = 1.6, Wilson gauge
    beta = 5.5; kappa = 0.134 with Hasenbusch kappas 0.120 and 0.130).

    Start: a random field (U = exp(i H), seed 3) thermalised by ntherm pure-gauge HMC
    trajectories at beta = 5.5 (2MN, 10 steps over tau = 1; the first half accepted
    unconditionally, the rest with the Metropolis test), the plaquette logged.  The
    filter ellipse is fitted to the spectrum of J_1 (Lanczos, 60 steps): (mu, nu) =
    s (1.2, 0.9) with s = max(1, 1.02 lambda_max / 2.1).  Action: S_G, S_det, P_12(J_1),
    Q = P_64 / P_12 (J_1), [J_1 P_64(J_1)]^{-1}, J_1 J_2^{-1}, J_2 K^{-1} (the filters of
    orders 12 and 64 = the smallest even order >= 48 that P_12 divides, and two
    Hasenbusch ratios), on a 4-level generalised 2MN with n = (60, 24, 10, 4) over tau = 1
    (step ratios 1 : 2.5 : 6 : 15): level 0 gauge + determinant, 1 the P_12 filter, 2 the
    Q filter, 3 the correction and both ratios.  Solves: mixed CG and FP64 multi-shift to
    1e-10 for the heatbath and the actions; MD forces in FP32 with solves to 1e-6.
    Reports per trajectory the wall time, dH, acceptance, plaquette and the K/J
    applications and forces per term; the reversibility of the first trajectory's MD
    (forward, momenta flipped, forward: |U - U_0| and |p + p_0|)."""
    import torch

    import pfmp_inputs as pin

    dims = PROD_DIMS
    V = int(np.prod(dims))
    lam = 0.1931833275037836
    fp = capi.PFMP_F32 if force_prec is None else force_prec
    ctx = capi.pfmp_ctx_create(dims, -1, stream.cuda_stream)
    out = {"lattice": "24x24x24x48", "params": dict(PROD, force_prec="f32" if fp == capi.PFMP_F32 else "f64")}
    try:
        out["thermalisation"] = thermalise(capi, ctx, dims, ntherm, 3)
        # spectrum of J_1 and an estimate for K (Lanczos: lmax converges, lmin from above)
        nb = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F64) // 8
        v0 = torch.zeros(nb, dtype=torch.float64, device="cuda")
        vc = torch.tensor(np.ascontiguousarray(pin.spinor(dims, 33)).view(np.float64).reshape(-1), device="cuda")
        capi.pfmp_spinor_pack(ctx, v0, capi.PFMP_F64, vc, capi.PFMP_DEVICE, 0)
        del vc
        spec = {}
        for name, kap in (("J1", PROD["kappa1"]), ("J2", PROD["kappa2"]), ("K", PROD["kappa"])):
            op = capi.pfmp_op_create(ctx, kap, PROD["csw"])
            lo, hi, _, _ = capi.pfmp_spectrum(op, 60, v0)
            spec[name] = {"lambda_min_upper": lo, "lambda_max": hi}
            capi.pfmp_op_destroy(op)
        del v0
        sc = max(1.0, 1.02 * spec["J1"]["lambda_max"] / 2.1)
        mu, nu = 1.2 * sc, 0.9 * sc
        out["spectrum"] = spec
        out["ellipse"] = {"mu": mu, "nu": nu}
        # the production action
        d = capi.ActionDef()
        d.beta, d.csw, d.nkappa = PROD["beta"], PROD["csw"], 3
        d.kappa[0], d.kappa[1], d.kappa[2] = PROD["kappa"], PROD["kappa1"], PROD["kappa2"]
        d.mu, d.nu, d.tol, d.max_iter = mu, nu, 1e-10, 40000
        d.solver, d.force_prec, d.md_tol = capi.PFMP_SOLVER_CG_MIXED, fp, 1e-6
        terms = [(capi.PFMP_KIND_GAUGE, 0, 0, 0, 0), (capi.PFMP_KIND_DET, 0, 0, 0, 0),
                 (capi.PFMP_KIND_FILTER, 1, 0, 0, PROD["p1"]), (capi.PFMP_KIND_FILTER, 1, 0, PROD["p1"], PROD["p2"]),
                 (capi.PFMP_KIND_FILTERCORR, 1, 0, 0, PROD["p2"]), (capi.PFMP_KIND_RATIO, 1, 2, 0, 0),
                 (capi.PFMP_KIND_RATIO, 2, 0, 0, 0)]
        names = ["gauge", "det", "P12(J1)", "Q=P64/P12(J1)", "[J1 P64(J1)]^-1", "J1 J2^-1", "J2 K^-1"]
        levels = [0, 0, 1, 2, 3, 3, 3]
        d.nterms = len(terms)
        for i, t in enumerate(terms):
            d.term[i] = capi.Term(*t)
        A = capi.pfmp_action_create_def(ctx, d)
        T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(n, PROD["tau"], lam) for n in PROD["steps"]])
        out["schedule_len"] = len(T)
        npf = capi.pfmp_action_counts(A)[1]

        def noise(seed):
            return np.concatenate([np.ascontiguousarray(pin.spinor(dims, seed + i)).view(np.float64).reshape(-1)
                                   for i in range(npf)])

        if reversibility:
            U0 = np.zeros(V * 72)
            capi.pfmp_gauge_get(ctx, U0, capi.PFMP_HOST)
            capi.pfmp_action_heatbath(A, noise(40000))
            p0 = np.ascontiguousarray(pin.momenta(dims, 40100)).reshape(-1).copy()
            p = p0.copy()
            t0 = time.perf_counter()
            capi.pfmp_md(A, T, S, levels, p)
            t_md = time.perf_counter() - t0
            U1 = np.zeros(V * 72)
            capi.pfmp_gauge_get(ctx, U1, capi.PFMP_HOST)
            moved = float(np.abs(U1 - U0).max())
            del U1
            p = -p
            capi.pfmp_md(A, T, S, levels, p)
            U2 = np.zeros(V * 72)
            capi.pfmp_gauge_get(ctx, U2, capi.PFMP_HOST)
            out["reversibility"] = {"md_s": t_md, "max_dU_forward": moved, "max_dU_after_return": float(np.abs(U2 - U0).max()),
                                    "max_dp_after_return": float(np.abs(p + p0).max())}
            del U2
            capi.pfmp_gauge_set(ctx, U0, capi.PFMP_HOST)
            capi.pfmp_action_refresh(A)
            del U0
        trajs = []
        for k in range(ntraj):
            xi = noise(50000 + 10 * k)
            mom = np.ascontiguousarray(pin.momenta(dims, 60000 + k)).reshape(-1)
            u = float(pin.uniform(61000 + k)[0])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = capi.pfmp_trajectory(A, T, S, levels, mom, xi, u)
            ms = (time.perf_counter() - t0) * 1e3
            trajs.append({"ms": ms, "dH": info.dH, "accepted": bool(info.accepted), "plaquette": info.plaquette,
                          "k_apply": int(info.k_apply), "force_evals": int(info.force_evals),
                          "ms_link_updates": info.ms_update,
                          "per_term": {n: {"k_apply": int(info.k_apply_term[t]), "forces": int(info.nforce[t]),
                                           "fmax": info.fmax[t], "favg": info.favg[t], "ms": info.ms_force[t]}
                                       for t, n in enumerate(names)}})
        out["trajectories"] = trajs
        if trajs:
            out["summary"] = {"ms_per_trajectory": statistics.mean(t["ms"] for t in trajs),
                              "acceptance": float(np.mean([t["accepted"] for t in trajs])),
                              "dH": [t["dH"] for t in trajs],
                              "exp_minus_dH": float(np.mean([math.exp(-t["dH"]) for t in trajs])),
                              "n_mat_per_term": {n: float(np.mean([t["per_term"][n]["k_apply"] for t in trajs]))
                                                 for n in names},
                              "ms_per_term": {n: float(np.mean([t["per_term"][n]["ms"] for t in trajs])) for n in names},
                              "ms_link_updates": float(np.mean([t["ms_link_updates"] for t in trajs]))}
        capi.pfmp_action_destroy(A)
    finally:
        capi.pfmp_ctx_destroy(ctx)
    return out


def tuning_4x4x4x4(capi, stream, ntraj=6):
    """The paper's step-size method (Sec. 2.4, Sec. 3.1) on the 4^4 parity configuration:
    one PF-MP trajectory (2MN 4 x 8 steps, tau 0.5) measures the maximal force of each
    level, F_l h_l = const gives the step counts (4 on the level with the smaller force),
    then ntraj trajectories from the same field with fresh momenta and noise give P_acc,
    N_mat and C = N_mat / P_acc with the autocorrelation-corrected errors (tau_int 12.5)."""
    import pfmp_inputs as pin

    dims = (4, 4, 4, 4)
    V = 256
    ctx = capi.pfmp_ctx_create(dims, -1, stream.cuda_stream)
    capi.pfmp_gauge_from_algebra(ctx, np.ascontiguousarray(pin.gauge_algebra(dims, 1)).reshape(-1), 0.3, capi.PFMP_HOST)
    U0 = np.zeros(V * 72)
    capi.pfmp_gauge_get(ctx, U0, capi.PFMP_HOST)
    d = capi.ActionDef()
    d.beta, d.csw, d.nkappa = 5.5, 1.0, 2
    d.kappa[0], d.kappa[1] = 0.120, 0.110
    d.mu, d.nu, d.tol, d.max_iter = 1.2, 0.9, 1e-12, 5000
    capi.pfmp_action_scheme(capi.PFMP_SCHEME_PFMP, 0, 8, d)
    A = capi.pfmp_action_create_def(ctx, d)
    lam = 0.1931833275037836
    levels = [1, 1, 1, 0, 0]
    noise = lambda s: np.concatenate([np.ascontiguousarray(pin.spinor(dims, s + i)).view(np.float64).reshape(-1)
                                      for i in range(3)])
    T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(n, 0.5, lam) for n in (4, 8)])
    info = capi.pfmp_trajectory(A, T, S, levels, np.ascontiguousarray(pin.momenta(dims, 500)).reshape(-1),
                                noise(510), 2.0)
    fl = [max(info.fmax[t] for t in range(5) if levels[t] == lv) for lv in (0, 1)]
    n = capi.pfmp_balance_steps(fl, 4)
    T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(k, 0.5, lam) for k in n])
    acc, nmat, dh = [], [], []
    t0 = time.perf_counter()
    for k in range(ntraj):
        capi.pfmp_gauge_set(ctx, U0, capi.PFMP_HOST)
        capi.pfmp_action_refresh(A)
        r = capi.pfmp_trajectory(A, T, S, levels, np.ascontiguousarray(pin.momenta(dims, 520 + k)).reshape(-1),
                                 noise(530 + 3 * k), float(pin.uniform(560 + k)[0]))
        acc.append(r.accepted)
        nmat.append(r.k_apply)
        dh.append(r.dH)
    s = time.perf_counter() - t0
    c = capi.pfmp_cost(acc, nmat, dh, 12.5)
    capi.pfmp_action_destroy(A)
    capi.pfmp_ctx_destroy(ctx)
    return {"level_fmax": fl, "steps": n, "trajectories": ntraj, "s_per_trajectory": s / ntraj,
            "p_acc": [c.p_acc, c.p_acc_err], "n_mat": [c.nmat, c.nmat_err], "cost": [c.cost, c.cost_err],
            "exp_minus_dH": [c.exp_mdh, c.exp_mdh_err], "dH": dh}


def trajectory_4x4x4x4(capi, stream):
    """One PF-MP trajectory of the 4^4 parity configuration (eps 0.3, beta 5.5, c_sw 1,
    kappa 0.120, kappa' 0.110, order-8 filter, 2MN 8 x 16 steps, tau 0.5, FP64, CG 1e-12)."""
    import torch

    import pfmp_inputs as pin

    dims = (4, 4, 4, 4)
    V = 256
    ctx = capi.pfmp_ctx_create(dims, -1, stream.cuda_stream)
    capi.pfmp_gauge_from_algebra(ctx, np.ascontiguousarray(pin.gauge_algebra(dims, 1)).reshape(-1), 0.3, capi.PFMP_HOST)
    ap = capi.ActionParams(beta=5.5, kappa=0.120, kappa_h=0.110, csw=1.0, n=8, mu=1.2, nu=0.9, tol=1e-12,
                           max_iter=5000)
    A = capi.pfmp_action_create(ctx, ap)
    lam = 0.1931833275037836
    T, S = capi.pfmp_schedule_merge([capi.pfmp_schedule_2mn(8, 0.5, lam), capi.pfmp_schedule_2mn(16, 0.5, lam)])
    xi = np.concatenate([np.ascontiguousarray(pin.spinor(dims, 10 + i)).view(np.float64).reshape(-1) for i in range(3)])
    mom = np.ascontiguousarray(pin.momenta(dims, 5)).reshape(-1)
    U0 = np.zeros(V * 72)
    capi.pfmp_gauge_get(ctx, U0, capi.PFMP_HOST)
    capi.pfmp_trajectory(A, T, S, [1, 1, 1, 0, 0], mom, xi, 2.0)  # warm (u = 2: reject, U restored)
    capi.pfmp_gauge_set(ctx, U0, capi.PFMP_HOST)
    capi.pfmp_action_refresh(A)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = capi.pfmp_trajectory(A, T, S, [1, 1, 1, 0, 0], mom, xi, float(pin.uniform(6)[0]))
    ms = (time.perf_counter() - t0) * 1e3
    capi.pfmp_action_destroy(A)
    capi.pfmp_ctx_destroy(ctx)
    return {"ms": ms, "dH": info.dH, "accepted": bool(info.accepted), "k_apply": int(info.k_apply),
            "force_evals": int(info.force_evals), "steps": len(T)}


def kernel_source():
    """Bytes of the sources that define the FP32 stencil kernels (for the traffic record)."""
    csrc = os.path.join(ROOT, "paper_1609_02652_gb300", "csrc")
    return b"".join(open(os.path.join(csrc, f), "rb").read()
                    for f in ("dslash_kernels.cuh", "hop.cuh", "fields.cuh", "spin.cuh", "pfmp_internal.cuh"))


def recorded_traffic():
    """DRAM bytes per launch of the FP32 stencil at 32^3x64 from the committed ncu summary,
    or None when the kernel source changed since those counters were taken."""
    import hashlib
    import re

    path = os.path.join(ROOT, "profiles", "hop_f32_24x24x24x48_full.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"bytes_per_launch_32x32x32x64: (\d+)", txt)
    h = re.search(r"kernel_source_sha256: ([0-9a-f]+)", txt)
    src = kernel_source()
    if not m or not h or h.group(1) != hashlib.sha256(src).hexdigest():
        return None
    return int(m.group(1))


def roofline(capi, stream, l2_flush, reps=12):
    import torch

    import pfmp_inputs as pin

    ctx = capi.pfmp_ctx_create(ROOF_DIMS, -1, stream.cuda_stream)
    V = ROOF_DIMS[0] * ROOF_DIMS[1] * ROOF_DIMS[2] * ROOF_DIMS[3]
    h = torch.tensor(np.ascontiguousarray(pin.gauge_algebra(ROOF_DIMS, GAUGE_SEED)).reshape(-1), device="cuda")
    torch.cuda.synchronize()
    capi.pfmp_gauge_from_algebra(ctx, h, EPS, capi.PFMP_DEVICE)
    del h
    op = capi.pfmp_op_create(ctx, KAPPA, CSW)
    n32 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F32) // 4
    a = torch.randn(n32, dtype=torch.float32, device="cuda")
    o = torch.zeros_like(a)
    for _ in range(3):
        capi.pfmp_kop(op, capi.PFMP_F32, o, a)
    capi.pfmp_profile_begin(ctx)
    for _ in range(reps):
        l2_flush()
        capi.pfmp_kop(op, capi.PFMP_F32, o, a)
    n, ms, by = capi.pfmp_profile_end(ctx, capi.PFMP_KERNEL_HOP_F32)
    # the same K on FP16 storage (spinors with per-site FP32 scales, links and clover FP16)
    nh = capi.pfmp_spinor_bytes(ctx, capi.PFMP_H16) // 4
    ah = torch.zeros(nh, dtype=torch.float32, device="cuda")
    oh = torch.zeros_like(ah)
    capi.pfmp_convert(ctx, ah, capi.PFMP_H16, a, capi.PFMP_F32)
    for _ in range(3):
        capi.pfmp_kop(op, capi.PFMP_H16, oh, ah)
    capi.pfmp_profile_begin(ctx)
    for _ in range(reps):
        l2_flush()
        capi.pfmp_kop(op, capi.PFMP_H16, oh, ah)
    n16, ms16, by16 = capi.pfmp_profile_end(ctx, capi.PFMP_KERNEL_HOP_H16)
    # the solves on the same 32^3x64 system, where the stencil is HBM-bound: mixed CG on
    # the FP32 stencil and on FP16 storage, the FP64 CG (a Gaussian rhs, 1e-10, L2 flushed)
    n64 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F64) // 8
    bcan = torch.tensor(np.ascontiguousarray(pin.spinor(ROOF_DIMS, RHS_SEED)).view(np.float64).reshape(-1), device="cuda")
    b = torch.zeros(n64, dtype=torch.float64, device="cuda")
    capi.pfmp_spinor_pack(ctx, b, capi.PFMP_F64, bcan, capi.PFMP_DEVICE, 0)
    del bcan
    x = torch.zeros_like(b)
    solves = {}
    for name, method, delta in (("mixed_cg", capi.PFMP_SOLVER_CG_MIXED, 1e-4), ("half_cg", capi.PFMP_SOLVER_CG_HALF, 0.03),
                                ("fp64_cg", capi.PFMP_SOLVER_CG64, 0.1)):
        prm = capi.SolverParams(method=method, tol=TOL, max_iter=20000, delta=delta, check_every=8)
        capi.pfmp_solve(op, prm, x, b)
        l2_flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = capi.pfmp_solve(op, prm, x, b)
        e1.record(stream)
        e1.synchronize()
        solves[name] = {"ms": e0.elapsed_time(e1), "iterations": info.iters, "true_rel_res": info.true_rel_res}
    solves["speedup_half_vs_mixed"] = solves["mixed_cg"]["ms"] / solves["half_cg"]["ms"]
    capi.pfmp_op_destroy(op)
    capi.pfmp_ctx_destroy(ctx)
    hbm, src = peaks()
    achieved = by / (ms * 1e-3) / 1e9
    traffic = recorded_traffic()
    a16 = by16 / (ms16 * 1e-3) / 1e9
    h16 = {"bound": "hbm", "achieved": a16, "peak": hbm, "unit": "GB/s", "frac": a16 / hbm, "peak_source": src,
           "kernel": "k_hop FP16 storage (half2 projection and link multiply, FP32 sums), 4 launches per K", "launches": n16,
           "avg_us": ms16 * 1e3 / n16, "bytes_per_launch": by16 / n16,
           "k_time_ratio_f32_over_h16": (ms / n) / (ms16 / n16), "solves_32x32x32x64": solves}
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "peak_source": src,
            "kernel": "k_hop FP32 (Wilson hop + fused clover epilogues), 4 launches per K",
            "workload": "K applications on 32^3x64, FP32, L2 flushed before each K",
            "launches": n, "avg_us": ms * 1e3 / n, "bytes_per_launch": by / n}, h16


def kernel_only(dims, reps, prec="f32"):
    """K = M-hat^dag M-hat applications in FP32 (or on FP16 storage) on `dims`, or true
    residuals b - K x of FP64 fields in FP64 or double-float arithmetic (prec "f64",
    "df"), with no timing: the case the ncu captures of the stencil kernels run."""
    import torch

    import pfmp_inputs as pin
    from paper_1609_02652_gb300 import capi

    torch.cuda.set_device(0)
    ctx = capi.pfmp_ctx_create(dims, -1, None)
    h = torch.tensor(np.ascontiguousarray(pin.gauge_algebra(dims, GAUGE_SEED)).reshape(-1), device="cuda")
    torch.cuda.synchronize()
    capi.pfmp_gauge_from_algebra(ctx, h, EPS, capi.PFMP_DEVICE)
    op = capi.pfmp_op_create(ctx, KAPPA, CSW)
    if prec in ("f64", "df"):
        n64 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F64) // 8
        x = torch.randn(n64, dtype=torch.float64, device="cuda")
        b = torch.randn_like(x)
        r = torch.zeros_like(x)
        ar = capi.PFMP_F64 if prec == "f64" else capi.PFMP_DF
        for _ in range(reps):
            capi.pfmp_true_residual(op, ar, r, x, b)
        torch.cuda.synchronize()
        capi.pfmp_op_destroy(op)
        capi.pfmp_ctx_destroy(ctx)
        print(json.dumps({"kernel_only": list(dims), "reps": reps, "launches_per_rep": 4, "prec": prec}))
        return
    n32 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F32) // 4
    a = torch.randn(n32, dtype=torch.float32, device="cuda")
    pr = capi.PFMP_F32
    if prec == "h16":
        pr = capi.PFMP_H16
        ah = torch.zeros(capi.pfmp_spinor_bytes(ctx, pr) // 4, dtype=torch.float32, device="cuda")
        capi.pfmp_convert(ctx, ah, pr, a, capi.PFMP_F32)
        a = ah
    o = torch.zeros_like(a)
    for _ in range(reps):
        capi.pfmp_kop(op, pr, o, a)
    torch.cuda.synchronize()
    capi.pfmp_op_destroy(op)
    capi.pfmp_ctx_destroy(ctx)
    print(json.dumps({"kernel_only": list(dims), "reps": reps, "launches_per_rep": 4, "prec": prec}))


def nn_only(reps, timed=0):
    """Applications of a [1,8,8,8,1] network (weights pfmp_inputs.nn_weights(ch, 5)) on the
    16^3x32 benchmark field through the tensor-core path: the case the ncu captures of the
    network kernels run; with timed > 0, that many more applications timed by CUDA events
    on the default stream (not for runs under ncu)."""
    import torch

    import pfmp_inputs as pin
    from paper_1609_02652_gb300 import capi

    torch.cuda.set_device(0)
    ctx = capi.pfmp_ctx_create(DIMS, -1, None)
    h = torch.tensor(np.ascontiguousarray(pin.gauge_algebra(DIMS, GAUGE_SEED)).reshape(-1), device="cuda")
    torch.cuda.synchronize()
    capi.pfmp_gauge_from_algebra(ctx, h, EPS, capi.PFMP_DEVICE)
    ch = [1, 8, 8, 8, 1]
    net = capi.pfmp_nn_create(ctx, ch, capi.PFMP_F32)
    capi.pfmp_nn_set_weights(net, pin.nn_weights(ch, 5))
    n32 = capi.pfmp_spinor_bytes(ctx, capi.PFMP_F32) // 4
    a = torch.randn(n32, dtype=torch.float32, device="cuda")
    o = torch.zeros_like(a)
    for _ in range(reps):
        capi.pfmp_nn_apply(net, capi.PFMP_F32, o, a)
    torch.cuda.synchronize()
    ms = None
    if timed > 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(timed):
            capi.pfmp_nn_apply(net, capi.PFMP_F32, o, a)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / timed
    capi.pfmp_nn_destroy(net)
    capi.pfmp_ctx_destroy(ctx)
    print(json.dumps({"nn_only": list(DIMS), "reps": reps, "network": ch, "ms_per_application": ms}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--production", action="store_true",
                    help="only the 24^3x48 production PF-MP run (thermalisation, reversibility, trajectories)")
    ap.add_argument("--prod-traj", type=int, default=10)
    ap.add_argument("--learned-scale", action="store_true",
                    help="only the learned preconditioner at scale (train on 24^3x48, FGCR at 32^3x64)")
    ap.add_argument("--pairs", type=int, default=256)
    ap.add_argument("--prod-therm", type=int, default=100)
    ap.add_argument("--cpu-full", action="store_true",
                    help="only the oracle's CPU timings: full solve on one thread and on all cores, 4^4 trajectory")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-big-trajectory", action="store_true")
    ap.add_argument("--no-production", action="store_true", help="skip the 24^3x48 production trajectory")
    ap.add_argument("--no-tuning", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 96-system batched-solve measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner measurement")
    ap.add_argument("--nn-steps", type=int, default=300, help="training steps of the learned preconditioner")
    ap.add_argument("--delta", type=float, default=1e-4, help="reliable-update threshold of the mixed solver")
    ap.add_argument("--chunk", type=int, default=8, help="CG iterations per CUDA-graph chunk")
    ap.add_argument("--nn-only", action="store_true",
                    help="three applications of the [1,8,8,8,1] network at 16^3x32 (for ncu captures)")
    ap.add_argument("--nn-timed", type=int, default=0, help="with --nn-only: applications timed by CUDA events")
    ap.add_argument("--kernel-prec", default="f32", choices=["f32", "h16", "f64", "df"])
    ap.add_argument("--kernel-only", action="store_true",
                    help="only apply K (FP32) --kernel-reps times on --kernel-dims: the small case for ncu")
    ap.add_argument("--kernel-dims", default="24,24,24,48")
    ap.add_argument("--kernel-reps", type=int, default=8)
    args = ap.parse_args()
    if args.cpu_full:
        cpu_full()
        return
    if args.learned_scale:
        import torch

        from paper_1609_02652_gb300 import capi

        stream = torch.cuda.Stream()
        print(json.dumps(learned_32x32x32x64(capi, stream, args.pairs, args.nn_steps)), flush=True)
        return
    if args.production:
        import torch

        from paper_1609_02652_gb300 import capi

        stream = torch.cuda.Stream()
        print(json.dumps(production_24x24x24x48(capi, stream, args.prod_traj, args.prod_therm)), flush=True)
        return
    if args.nn_only:
        nn_only(3, args.nn_timed)
        return
    if args.kernel_only:
        kernel_only(tuple(int(v) for v in args.kernel_dims.split(",")), args.kernel_reps, args.kernel_prec)
        return
    rank, world = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
