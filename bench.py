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
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the same solve.

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
def oracle_sample(iters):
    """The FP64 CPU oracle's CG on the same system, stopped after `iters` iterations.

    Returns (seconds per iteration, estimated iterations to 1e-10 from the oracle's own
    residual decay, threads)."""
    import torch

    import pfmp_inputs as pin
    from oracle.dirac import WilsonClover
    from oracle.lattice import Lattice, algebra_to_matrix, expi_hermitian

    lat = Lattice(DIMS, bc_t=-1)
    U = expi_hermitian(algebra_to_matrix(torch.tensor(pin.gauge_algebra(DIMS, GAUGE_SEED)).reshape(*lat.shape, 4, 8)), EPS)
    W = WilsonClover(lat, U, KAPPA, CSW)
    _ = W.Ainv
    b = torch.tensor(pin.spinor(DIMS, RHS_SEED)).reshape(*lat.shape, 4, 3) * lat.even
    x = torch.zeros_like(b)
    r = b.clone()
    p = r.clone()
    rr = (r.conj() * r).sum().real
    bb = rr
    t0 = time.perf_counter()
    res = []
    for _ in range(iters):
        Ap = W.K(p)
        a = rr / (p.conj() * Ap).sum().real
        x = x + a * p
        r = r - a * Ap
        rn = (r.conj() * r).sum().real
        p = r + (rn / rr) * p
        rr = rn
        res.append(math.sqrt(rr / bb))
    dt = (time.perf_counter() - t0) / iters
    rate = math.log(res[-1]) / iters
    est = int(math.ceil(math.log(TOL) / rate)) if rate < 0 else None
    return dt, est, torch.get_num_threads()


def oracle_iterations():
    """Iterations the oracle's FP64 CG needs on this system (stored by
    tests/golden/make_cg_iterations.py, which runs only the oracle)."""
    p = os.path.join(ROOT, "tests", "golden", "cg_iterations_16x16x16x32.json")
    if os.path.exists(p):
        with open(p) as f:
            return int(json.load(f)["iterations"]), "the oracle's full FP64 CG run (stored)"
    return None, None


def run_reference(args, rank, world):
    if rank != 0:
        return
    per_step = []
    est = None
    thr = None
    for _ in range(args.warmup + args.steps):
        dt, est, thr = oracle_sample(2)
        per_step.append(dt)
    per_it = statistics.mean(per_step[args.warmup:])
    n_it, how = oracle_iterations()
    if n_it is None:
        n_it, how = est, "extrapolated from the sample's residual decay"
    value = per_it * n_it * 1e3
    sample = (f"{2 * args.steps} FP64 oracle CG iterations (2 per step) on the full 16^3x32 system; ms/solve = "
              f"s/iteration x {n_it} iterations ({how})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "implementation": "FP64 CPU oracle (PyTorch CPU ops)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    n_hop, hop_ms, hop_bytes = capi.pfmp_profile_end(ctx, capi.PFMP_KERNEL_HOP_F32)
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
    traj_big = None if args.no_big_trajectory else guarded(trajectory_16x16x16x32, capi, stream)
    tuning = None if args.no_tuning else guarded(tuning_4x4x4x4, capi, stream)
    capi.pfmp_op_destroy(op)
    capi.pfmp_ctx_destroy(ctx)

    # roofline of the stencil kernels on a lattice far larger than L2
    roof, roof_h16 = roofline(capi, stream, l2_flush)
    batched = None if args.no_batched else batched_96(capi, stream, l2_flush, args)

    hbm, src = peaks()
    hop_gbs_l2 = hop_bytes / (hop_ms * 1e-3) / 1e9 if hop_ms > 0 else None
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
        "tuning_4x4x4x4": tuning,
        "batched": batched,
        "hop_in_solve": {"launches": n_hop, "avg_us": hop_ms * 1e3 / max(n_hop, 1), "algorithmic_gbs": hop_gbs_l2,
                         "note": "16^3x32 FP32 working set (~75 MB) is L2-resident inside a solve"},
        "gpu_launches": int(launches),
        "gpu_launches_note": "kernels launched by libpfmp in the timed steps, graph-replayed kernels included",
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        per_it, est, thr = oracle_sample(args.cpu_iters)
        n_it, how = oracle_iterations()
        if n_it is None:
            n_it, how = info_plain[-1].iters, "the FP64 CG iteration count of the GPU run"
        line["cpu_baseline"] = {
            "value": per_it * n_it * 1e3, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"{args.cpu_iters} FP64 oracle CG iterations on the full 16^3x32 system; ms/solve = "
                      f"s/iteration x {n_it} iterations ({how})"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_96(capi, stream, l2_flush, args):
    """96 systems -- 32 each on 8^4, 12^3x24 and 16^3x32, eps = 0.4, kappa ~ U[0.120, 0.134]
    (seed 7), c_sw = 1.0, 1..8 Gaussian right-hand sides each (seed 8) -- solved to 1e-10 by
    the batched grouped-kernel solver, against the same solves one after another with the
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


def guarded(fn, *a):
    """A secondary measurement that must not take the headline line down with it."""
    try:
        return fn(*a)
    except Exception as e:  # reported in the JSON line instead
        return {"error": f"{type(e).__name__}: {e}"}


def trajectory_16x16x16x32(capi, stream):
    """One PF-MP trajectory on the paper's lattice size, 16^3x32 (synthetic field eps 0.3,
    seed 1; beta 5.5, c_sw 1, kappa 0.125, kappa' 0.110, order-8 filter, (mu, nu) = (1.2,
    0.9)), the action's CG in mixed precision and the multi-shift in FP64, all solves to
    1e-10; 2-level 2MN, 2 coarse (correction + Hasenbusch ratio) x 4 fine (gauge, clover
    determinant, filter) steps over tau = 0.1.  Wall time of the whole trajectory
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
                    for f in ("dslash.cu", "hop.cuh", "fields.cuh", "spin.cuh", "pfmp_internal.cuh"))


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
    capi.pfmp_op_destroy(op)
    capi.pfmp_ctx_destroy(ctx)
    hbm, src = peaks()
    achieved = by / (ms * 1e-3) / 1e9
    traffic = recorded_traffic()
    a16 = by16 / (ms16 * 1e-3) / 1e9
    h16 = {"bound": "hbm", "achieved": a16, "peak": hbm, "unit": "GB/s", "frac": a16 / hbm, "peak_source": src,
           "kernel": "k_hop FP16 storage (FP32 arithmetic), 4 launches per K", "launches": n16,
           "avg_us": ms16 * 1e3 / n16, "bytes_per_launch": by16 / n16,
           "k_time_ratio_f32_over_h16": (ms / n) / (ms16 / n16)}
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


def nn_only(reps):
    """Applications of a [1,8,8,8,1] network (weights pfmp_inputs.nn_weights(ch, 5)) on the
    16^3x32 benchmark field through the tensor-core path (no timing): the case the ncu
    captures of the network kernels run."""
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
    capi.pfmp_nn_destroy(net)
    capi.pfmp_ctx_destroy(ctx)
    print(json.dumps({"nn_only": list(DIMS), "reps": reps, "network": ch}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-big-trajectory", action="store_true")
    ap.add_argument("--no-tuning", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 96-system batched-solve measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner measurement")
    ap.add_argument("--nn-steps", type=int, default=300, help="training steps of the learned preconditioner")
    ap.add_argument("--delta", type=float, default=1e-4, help="reliable-update threshold of the mixed solver")
    ap.add_argument("--chunk", type=int, default=8, help="CG iterations per CUDA-graph chunk")
    ap.add_argument("--nn-only", action="store_true",
                    help="three applications of the [1,8,8,8,1] network at 16^3x32 (for ncu captures)")
    ap.add_argument("--kernel-prec", default="f32", choices=["f32", "h16", "f64", "df"])
    ap.add_argument("--kernel-only", action="store_true",
                    help="only apply K (FP32) --kernel-reps times on --kernel-dims: the small case for ncu")
    ap.add_argument("--kernel-dims", default="24,24,24,48")
    ap.add_argument("--kernel-reps", type=int, default=8)
    args = ap.parse_args()
    if args.nn_only:
        nn_only(3)
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
