#!/usr/bin/env python
"""Throughput of the implicit q-LSKUM hot path on GB300, in point-iterations/s,
and the wall time of whole solves to a 1e-8 residual drop.

One step = one pseudo-time iteration (q-derivatives with K = 2 inner
iterations, second-order split-flux residual, residual norm, forward and
backward LU-SGS sweeps with exact-AD Jacobian products, state update) of the
plain FP64 solver.  Default workload: the jittered NACA 0012 cloud of
2560x2048 nodes (5,242,880 points, stencils in the index-normalised metric),
M = 0.8, AoA = 1.25 deg, CFL 100.  The solve starts with START first-order
iterations (untimed set-up, before the warm-up); every timed step is a full
second-order iteration.

At N = 1 the default run also times two whole solves to a 1e-8 drop of the
density residual on the 147,584-point cloud (the largest whose two solves fit
a few minutes; a 1e-8 solve of the 5.24M-point cloud takes ~1e5 iterations):
plain FP64 from the free stream, and FP32 sweeps from the learned warm start
judged by the residual (the network trained first on the solver's own
batched solutions, training time reported apart) -- the `solve` block.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload W] [--solve on|off]

--workload naca0012_640x256_jit runs the 147,584-point cloud (M 0.85, AoA 1);
naca0012_160x64 the 10,240-point O-grid (M 0.63, AoA 2); naca0012_1280x1024_jit
the quarter-size stand-in of the default cloud (profiling);
naca0012_640x256_jit_m1.2 the paper's supersonic case (M 1.2, AoA 0) on the
same cloud with the kinetic far field (and a whole solve, --solve-iters caps
it); naca0012_batch64 the 64-cloud batch; naca0012_warmstart the warm-start
study on the 160x64 cloud.

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded number of iterations of the same workload.  Under torchrun (N > 1)
every rank runs an independent replica (the single-cloud solve has no
data-parallel split; see the design notes), value = total point-iterations
of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "naca0012_2560x2048_jit"      # default: 5,242,880 points
MID_WORKLOAD = "naca0012_640x256_jit"    # 147,584 points
PROF_WORKLOAD = "naca0012_1280x1024_jit"  # 1,310,720 points, the default's construction (profiling)
SUPER_WORKLOAD = "naca0012_640x256_jit_m1.2"
SMALL_WORKLOAD = "naca0012_160x64"        # 10,240 points, 3x3 index-block stencils
# K = 2 inner iterations everywhere: with 3 the unlimited reconstruction
# diverges in the coarse far field in long runs from the free stream, so
# the solves to a 1e-8 drop use 2 and the timed steps do the same
CASES = {WORKLOAD: dict(mach=0.8, aoa=1.25, K=2, farfield=0),
         MID_WORKLOAD: dict(mach=0.85, aoa=1.0, K=2, farfield=0),
         PROF_WORKLOAD: dict(mach=0.8, aoa=1.25, K=2, farfield=0),
         SUPER_WORKLOAD: dict(mach=1.2, aoa=0.0, K=2, farfield=1),
         SMALL_WORKLOAD: dict(mach=0.63, aoa=2.0, K=2, farfield=0)}
SOLVE_WORKLOAD = MID_WORKLOAD
METRIC = "point-iter/s; wall time to 1e-8 residual drop, plain FP64 vs FP32+warm start"
UNIT = "point-iter/s"
L2_BYTES = 129 * 2**20
# FP64 peak derived from unit counts and clock: 152 SMs x 2 DFMA/clk/SM x 2 flop
# x 2070 MHz = 1.259 TFLOP/s (a DFMA-chain probe measured 1.196 at ~2.0 GHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# The residual's algorithmic arithmetic per neighbour slot that joins a split
# sub-stencil, in FP64 flops (DFMA = 2): what the method's formulas cost when
# every operation runs on the FP64 unit, counted by ncu (2 x dfma + dmul +
# dadd thread instructions of one launch / such slots) on the all-FP64 form
# of this kernel (the same exp, erfcx and reconstruction formulas): the
# 147,584-point cloud's Euclidean stencils (2,926,611 slots at 2 threads per
# point), and the cone-completed stencils of the 1,310,720-point cloud
# (26,159,870 slots at 1 thread per point: 2 x 3,240,043,812 + 1,797,370,444
# + 477,404,332), which stand for the 5,242,880-point cloud of the same
# construction (the count depends on the mix of slots joining one or two
# sub-stencils)
RES_FLOPS_PER_SLOT = {MID_WORKLOAD: 336.07, SUPER_WORKLOAD: 336.07, PROF_WORKLOAD: 334.668, WORKLOAD: 334.668}
# The current kernel runs exp and erfcx in fixed point and the split fluxes'
# multiplications as correctly rounded integer multiplies on the integer
# pipes, beside the FP64 unit; the FP64 flops it still executes on the FP64
# unit per slot (ncu, the same counting; profiles/)
RES_FP64_UNIT_FLOPS_PER_SLOT = {MID_WORKLOAD: 154.72, SUPER_WORKLOAD: 154.72, PROF_WORKLOAD: 154.67,
                                WORKLOAD: 154.67}
START = 50  # first-order start-up iterations before warm-up and timing
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one residual
# launch, from one ncu capture of the current kernel (profiles/), per
# workload and threads per point; reported only for that launch shape and FP64
RES_TRAFFIC = {MID_WORKLOAD: {1: 163.482624e6}, PROF_WORKLOAD: {1: 3.407065856e9},
               WORKLOAD: {1: 14.584e9}}  # the last from a one-pass capture of the full-size launch
# Unit utilisation of that launch (fraction of peak sustained, ncu): the FP64
# pipe is the binding unit; the integer pipes (ALU, FMA-heavy: IMAD) carry
# the fixed-point functions and the integer multiplies
RES_UNITS_NCU = {MID_WORKLOAD: {"fp64_pipe": 0.8058, "alu_pipe": 0.3980, "fmaheavy_pipe": 0.3469, "issue": 0.4153},
                 PROF_WORKLOAD: {"fp64_pipe": 0.8342, "alu_pipe": 0.4119, "fmaheavy_pipe": 0.3591,
                                 "issue": 0.4282}}
RES_UNITS_NCU[SUPER_WORKLOAD] = RES_UNITS_NCU[MID_WORKLOAD]
RES_UNITS_NCU[WORKLOAD] = RES_UNITS_NCU[PROF_WORKLOAD]
ROOFLINE_NOTE = ("achieved counts the method's FP64 arithmetic as the all-FP64 form executes it "
                 "(flops_per_active_slot); frac can exceed 1 because exp and erfcx run in 64-bit fixed point "
                 "and the split fluxes' multiplications as correctly rounded integer multiplies on the integer "
                 "pipes, beside the FP64 unit; fp64_unit gives the FP64 unit's own share and utilisation")


def _sweep_form(lanes):
    """What the library's sweep launch-shape value means."""
    if lanes == 32:
        return ("packed: each point's axis Jacobian products formed once and gathered, 4 lanes per "
                "interior point, one lane per slot for wall points")
    return f"{lanes} lanes per point, products per slot"


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.p = None
        self.gpu_id = gpu_id

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else f"GPU-{u}"
    except Exception:
        return str(dev)


def cpu_baseline(cloud, iters, warm=0, mach=0.85, aoa=1.0, K=2, farfield=0, startup=1, jvp=0):
    """The FP64 oracle, as it stands, on one host core: `iters` iterations
    timed after `startup` first-order start-up and `warm` warm-up iterations
    (startup = 0: the first `iters` iterations from the free stream, all
    first-order -- the same arithmetic with the reconstruction's gradients
    zero)."""
    import oracle as O
    o = O.Oracle(cloud, farfield=farfield, mach=mach, aoa_deg=aoa)
    U = o.initial_state(mach, aoa)
    n0, hist0 = 0, 0.0
    if startup + warm > 0:
        r0 = o.run(U, startup + warm, cfl=100.0, K=K, first_order=startup, jvp=jvp)
        U, n0, hist0 = r0["U"], startup + warm, r0["hist0"]
    t0 = time.perf_counter()
    r = o.run(U, iters, cfl=100.0, K=K, n0=n0, hist0=hist0, first_order=startup if startup else iters, jvp=jvp)
    dt = time.perf_counter() - t0
    return cloud.n * r["done"] / dt, dt, r["done"]


def _cpu_sample(wl, steps, warm):
    """(iterations, warm-up, start-up) of a bounded oracle sample: about 10-30 s
    of one core per iteration on the 5.24M-point cloud, so one to three
    iterations from the free stream there; up to 10 second-order ones on the
    smaller clouds."""
    if wl in (WORKLOAD, PROF_WORKLOAD):
        return max(1, min(steps, 3 if wl == PROF_WORKLOAD else 2)), 0, 0
    return max(1, min(steps, 10)), min(warm, 1), 1


def _sample_text(done, warm, startup, n):
    if startup == 0:
        return (f"{done} FP64 oracle iteration(s) from the free stream on the full {n}-point cloud (first-order "
                f"start-up: the arithmetic of a second-order iteration with the reconstruction's gradients zero), "
                f"one thread")
    return (f"{done} second-order FP64 oracle iterations on the full {n}-point cloud after {startup} first-order "
            f"start-up and {warm} warm-up iterations, one thread")


def run_reference(args, rank):
    from paper_2406_07441_gb300 import cloudgen as cg
    if rank != 0:
        return
    wl = args.workload if args.workload in CASES else WORKLOAD
    case = CASES[wl]
    cloud = cg.build_workload(wl)
    steps, warm, startup = _cpu_sample(wl, args.steps, args.warmup)
    val, dt, done = cpu_baseline(cloud, steps, warm, mach=case["mach"], aoa=case["aoa"], K=case["K"],
                                 farfield=case["farfield"], startup=startup)
    sample = _sample_text(done, warm, startup, cloud.n)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": done,
            "warmup": warm, "ms_per_step": dt * 1e3 / done, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl, "points": cloud.n, "mach": case["mach"], "aoa_deg": case["aoa"], "cfl": 100.0,
                       "inner_iters": case["K"], "jvp": "exact-AD",
                       "order": "first (start-up from the free stream)" if startup == 0 else "second (after start-up)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _shared_cloud(wl, rank, world, dist):
    """The workload's cloud; with several ranks rank 0 builds it once and the
    others load it from a temporary file (a 5.24M-point build holds ~10 GB of
    host memory)."""
    import numpy as np

    from paper_2406_07441_gb300 import cloudgen as cg
    if world == 1 or dist is None:
        return cg.build_workload(wl)
    path = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"lskum_cloud_{wl}_{os.getppid()}.npz")
    if rank == 0:
        c = cg.build_workload(wl)
        np.savez(path + ".tmp.npz", x=c.x, y=c.y, flag=c.flag, nx=c.nx, ny=c.ny, off=c.nbr_off, idx=c.nbr_idx)
        os.replace(path + ".tmp.npz", path)
    dist.barrier()
    if rank != 0:
        z = np.load(path)
        c = cg.Cloud(z["x"], z["y"], z["flag"], z["nx"], z["ny"], z["off"], z["idx"], {"workload": wl})
    dist.barrier()
    if rank == 0:
        os.remove(path)
    return c


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2406_07441_gb300 import lskum

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    wl = args.workload
    case = CASES[wl]
    mach, aoa, K, kinetic = case["mach"], case["aoa"], case["K"], case["farfield"] == 1
    cloud = _shared_cloud(wl, rank, world, dist)
    n = cloud.n
    explicit = args.scheme == "explicit"
    cfl = 0.3 if explicit else 100.0
    jvp = lskum.JVP_INCREMENT if args.jvp == "increment" else lskum.JVP_EXACT
    kw = dict(cfl=cfl, inner_iters=K, jvp=jvp, first_order_iters=START, precision=args.precision,
              scheme=lskum.SCHEME_EXPLICIT if explicit else lskum.SCHEME_LUSGS, farfield=case["farfield"])
    s = lskum.Solver(cloud, mach, aoa, **kw)
    nslots = int(np.count_nonzero(_memberships(cloud, kinetic)))
    # first-order start-up, then warm-up iterations (untimed)
    assert s.run(START) == START
    # launch shape chosen by the library's autotuner (real iterations, state
    # restored), or given (e.g. for a profiler run with a known launch count)
    if args.launch_shape:
        tpp, lanes = (int(t) for t in args.launch_shape.split(","))
        s.set_launch_shape(tpp, lanes)
    else:
        tpp, lanes, _ = s.autotune(3 if n > 1_000_000 else 5)
    info = s.info()  # launches per iteration in the chosen launch shape
    assert s.run(args.warmup) == args.warmup
    stream = torch.cuda.ExternalStream(s.stream())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(_gpu_id(torch, local_rank)) as clk:
        e0.record(stream)
        s.enqueue(args.steps)
        e1.record(stream)
        done = s.wait()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    if done != args.steps:
        raise RuntimeError(f"only {done} of {args.steps} iterations ran")
    ms = e0.elapsed_time(e1)
    ms_max, (work_all,) = combine_over_ranks(dist, ms, [float(n) * args.steps], "cuda")
    value = work_all / (ms_max / 1e3)

    # live per-phase timing (CUDA events on the library stream) for the roofline
    phases = s.time_phases(5)
    res_ms = phases["residual"]
    flops_slot = RES_FLOPS_PER_SLOT.get(wl)
    achieved = flops_slot * nslots / (res_ms / 1e3) / 1e12 if flops_slot else None
    unit_slot = RES_FP64_UNIT_FLOPS_PER_SLOT.get(wl)
    unit_tf = unit_slot * nslots / (res_ms / 1e3) / 1e12 if unit_slot else None

    # end to end through the C-ABI with host buffers: state in (H2D), one
    # iteration, state out (D2H) every step
    e2e_steps = min(args.steps, 20 if n < 1_000_000 else 10)
    U = s.field(lskum.FIELD_U)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_conserved(U)
        s.run(1)
        U = s.field(lskum.FIELD_U)
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": n * e2e_steps / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": int(U.nbytes),
           "d2h_bytes_per_step": int(U.nbytes) + 8}
    del U

    whole = None
    if args.solve_iters > 0:
        # wall time of a whole solve from the free stream to the drop target
        # on this workload (host clock around the C-ABI call; the launch shape
        # of the timed steps)
        s2 = lskum.Solver(cloud, mach, aoa, **kw)
        s2.set_launch_shape(tpp, lanes)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it = s2.run(args.solve_iters, target_drop=1e-8)
        sec = time.perf_counter() - t0
        h = s2.residuals()
        cl, cd = s2.forces()
        whole = {"target_drop": 1e-8, "iterations": int(it), "seconds": sec, "reached": bool(h[-1] / h[0] <= 1e-8),
                 "final_drop": float(h[-1] / h[0]), "cl": cl, "cd": cd, "max_iters": args.solve_iters}
        s2.close()
    s.close()

    solve = None
    if world == 1 and args.solve == "on":
        solve = solve_block(args, torch)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1:
        steps, warm, startup = _cpu_sample(wl, 1 if wl == WORKLOAD else 10, 0)
        cv, cdt, cdone = cpu_baseline(cloud, steps, warm, mach=mach, aoa=aoa, K=K, farfield=case["farfield"],
                                      startup=startup, jvp=jvp)
        cpu = {"value": cv, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": _sample_text(cdone, warm, startup, n)}
    ws = _working_set_bytes(cloud)
    traffic = RES_TRAFFIC.get(wl, {}).get(tpp) if args.precision == 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f64+f32", "data": "synthetic",
        "config": {"workload": wl, "points": n, "neighbour_slots": int(cloud.nnz),
                   "precision": "fp64" if args.precision == 0 else "fp32 sweeps, fp64 residual/update",
                   "mach": mach, "aoa_deg": aoa, "cfl": cfl, "inner_iters": K,
                   "far_field": "kinetic (outer points updated, free-stream ghosts)" if kinetic
                   else "free stream held at the outer points",
                   "scheme": "explicit (forward Euler, no sweeps)" if explicit else "implicit LU-SGS",
                   "jvp": "increment (split-flux differences)" if args.jvp == "increment" else "exact-AD",
                   "order": f"second (timed steps follow {START} untimed first-order start-up iterations)",
                   "colours": info["n_colours"],
                   "launch_shape": {"threads_per_point": tpp, "sweep_lanes_per_point": lanes,
                                    "sweep_form": _sweep_form(lanes),
                                    "by": "given" if args.launch_shape else "autotune"},
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"inputs larger than L2: device working set {ws / 2**20:.0f} MiB > 129 MiB L2"},
        "roofline": {"bound": "alu", "kernel": "k_residual", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                     "traffic": traffic, "traffic_unit": "bytes per launch (ncu)",
                     "algorithmic_bytes_per_launch": int(cloud.nnz) * 37 + n * 360,
                     "algorithmic_bytes_rule": "37 B per neighbour slot (index, membership, dx, dy, 2 weights) "
                                               "+ 360 B per point (q, grad q, frame, geometry, state, R, D)",
                     "flops_per_active_slot": flops_slot, "active_slots": nslots,
                     "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz (the FP64 unit)",
                     "note": ROOFLINE_NOTE,
                     "fp64_unit": {"flops_per_active_slot": unit_slot, "achieved": unit_tf,
                                   "frac": unit_tf / FP64_PEAK_TFLOPS if unit_tf else None},
                     "units_active_ncu": RES_UNITS_NCU.get(wl) if args.precision == 0 else None,
                     "launch_ms": res_ms, "phase_ms": phases},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": info["launches_per_iter"] * args.steps,
        "clocks": clk.summary(),
    }
    if whole is not None:
        line["whole_solve"] = whole
    if solve is not None:
        line["solve"] = solve
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


FWD_POINTS = 131072  # points of the timed forward pass of the network (one launch)


def train_network(n_solves, seed, K=2):
    """The warm-start network trained on the solver's own solutions: batched
    FP32-sweep solves of the 160x64 cloud at n_solves random (M, AoA)
    (3,000 iterations each, 4,096 points sampled per solve), then Adam.
    Returns (network, facts)."""
    import numpy as np
    import torch

    from paper_2406_07441_gb300 import cloudgen as cg
    from paper_2406_07441_gb300 import lskum
    cloud = cg.build_workload("naca0012_160x64")
    rng = np.random.default_rng(seed)
    train = [(float(rng.uniform(0.3, 0.85)), float(rng.uniform(-4, 6))) for _ in range(n_solves)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net = lskum.Mlp(seed=cg.BASE_SEED, max_batch=FWD_POINTS)  # buffers for one forward tile set
    failed = 0
    for g0 in range(0, len(train), 64):
        conds = train[g0:g0 + 64]
        b = lskum.Solver.batch([cloud] * len(conds), conds, first_order_iters=START, inner_iters=K, precision=1)
        b.run(3000)
        failed += sum(1 for k in range(len(conds)) if b.case_info(k)["status"] != 0)
        net.add_samples(b, 4096, seed=g0)
        del b
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    n_samp = net.n_samples()
    epochs = max(10, min(200, int(100 * 262144 / max(n_samp, 1))))
    t0 = time.perf_counter()
    losses = net.train(epochs, 512, 1e-3, seed=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    return net, {"train_cloud": "naca0012_160x64", "train_solves": len(train), "train_iters": 3000,
                 "train_failed": failed, "samples": n_samp, "epochs": epochs, "data_s": t_data, "train_s": t_train,
                 "final_loss": float(losses[-1]), "conditions": "M ~ U[0.3, 0.85], AoA ~ U[-4, 6] deg"}


def solve_block(args, torch):
    """Wall time to a 1e-8 drop of the density residual on SOLVE_WORKLOAD:
    plain FP64 from the free stream, then FP32 sweeps from the judged warm
    start to the plain run's final absolute norm (1e-8 x its first norm).
    Host clock around the C-ABI runs (set-up, autotuning and the network's
    training outside; the prediction and its judging inside)."""
    from paper_2406_07441_gb300 import cloudgen as cg
    from paper_2406_07441_gb300 import lskum
    case = CASES[SOLVE_WORKLOAD]
    mach, aoa, K = case["mach"], case["aoa"], case["K"]
    cloud = cg.build_workload(SOLVE_WORKLOAD)
    drop, max_iters = 1e-8, args.solve_max
    sp = lskum.Solver(cloud, mach, aoa, inner_iters=K, first_order_iters=START, precision=0)
    tp_shape = sp.autotune(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it_p = sp.run(max_iters, target_drop=drop)
    torch.cuda.synchronize()
    sec_p = time.perf_counter() - t0
    hp = sp.residuals()
    clp, cdp = sp.forces()
    target = hp[0] * drop
    sp.close()
    net, facts = train_network(args.train_solves, cg.BASE_SEED + 5, K=K)
    sw = lskum.Solver(cloud, mach, aoa, inner_iters=K, first_order_iters=0, precision=1)
    tw_shape = sw.autotune(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kept = bool(net.predict(sw)[0])
    if not kept:
        sw.set_start_iters(START)  # the free stream needs the first-order start-up
    st_w, it_w, hw = _drop_run(sw, target, 20000, max_iters)
    torch.cuda.synchronize()
    sec_w = time.perf_counter() - t0
    clw, cdw = sw.forces()
    sw.close()
    net.time_forward(FWD_POINTS, 3)
    fwd_ms = net.time_forward(FWD_POINTS, 20)
    net.close()
    ok_p = bool(hp[-1] <= target)
    ok_w = bool(st_w == 0 and hw[-1] <= target)
    return {
        "cloud": SOLVE_WORKLOAD, "points": cloud.n, "mach": mach, "aoa_deg": aoa, "inner_iters": K, "cfl": 100.0,
        "target_drop": drop, "max_iters": max_iters,
        "plain": {"precision": "fp64", "start": f"free stream, {START} first-order start-up iterations",
                  "iterations": int(it_p), "seconds": sec_p, "reached": ok_p, "final_drop": float(hp[-1] / hp[0]),
                  "cl": clp, "cd": cdp, "launch_shape": list(tp_shape[:2])},
        "warm": {"precision": "fp32 sweeps, fp64 residual/update",
                 "start": "network prediction judged by the first residual (second order from iteration 1)"
                 if kept else f"free stream (prediction rejected by the judge), {START} first-order iterations",
                 "prediction_kept": kept, "iterations": int(it_w), "seconds": sec_w, "reached": ok_w,
                 "first_norm_ratio": float(hw[0] / hp[0]), "final_norm_vs_plain_first": float(hw[-1] / hp[0]),
                 "cl": clw, "cd": cdw, "launch_shape": list(tw_shape[:2]),
                 "network_forward_ms_per_131072_points": fwd_ms},
        "time_ratio": sec_w / sec_p if ok_p and ok_w else None,
        "iteration_ratio": it_w / it_p if ok_p and ok_w else None,
        "dcl": abs(clw - clp), "dcd": abs(cdw - cdp),
        "network": facts,
        "reference": "the plain FP64 GPU path is the one checked against the FP64 oracle (parity tests: history "
                     "1e-10 per entry, final fields 1e-9); dcl and dcd compare the warm arm with it",
    }


BATCH_WORKLOAD = "naca0012_batch64"


def combine_over_ranks(dist, ms, counts, device):
    """The job's time is the slowest rank's, its work the sum of the ranks'
    (dist = torch.distributed or None for one process)."""
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    c = torch.tensor([float(x) for x in counts], device=device, dtype=torch.float64)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(x) for x in c.tolist()]


def _shard(cases, rank, world):
    """Longest-processing-time split of the cases over the ranks (cost = points)."""
    loads = [0] * world
    mine = []
    for k in sorted(range(len(cases)), key=lambda k: -cases[k]["n_i"] * cases[k]["n_j"]):
        r = loads.index(min(loads))
        loads[r] += cases[k]["n_i"] * cases[k]["n_j"]
        if r == rank:
            mine.append(k)
    return sorted(mine)


def _build_clouds(cases):
    """Generate the clouds on the host cores (spawned workers, before any CUDA call)."""
    import multiprocessing as mp

    from paper_2406_07441_gb300 import cloudgen as cg
    procs = max(1, min(len(cases), os.cpu_count() or 1, 16))
    if procs == 1:
        return [cg.build_case(c) for c in cases]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(cg.build_case, cases, chunksize=1)


def run_batch(args, rank, world, local_rank):
    """64 clouds x free-stream conditions solved as one batched context:
    FP32 sweeps, FP64 residual and update, cases sharded over the ranks."""
    import numpy as np
    import torch

    from paper_2406_07441_gb300 import cloudgen as cg

    cases_all = cg.batch_cases()
    mine = _shard(cases_all, rank, world)
    cases = [cases_all[k] for k in mine]
    clouds = _build_clouds(cases)
    from paper_2406_07441_gb300 import lskum

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    n = sum(c.n for c in clouds)
    conds = [(c["mach"], c["aoa_deg"]) for c in cases]
    s = lskum.Solver.batch(clouds, conds, cfl=100.0, inner_iters=2, jvp=lskum.JVP_EXACT, first_order_iters=START,
                           precision=args.precision)
    info = s.info()
    nslots = int(sum(np.count_nonzero(_memberships(c)) for c in clouds))
    assert s.run(START) == START
    tpp, lanes, _ = s.autotune(5)
    info = s.info()  # launches per iteration in the chosen launch shape
    assert s.run(args.warmup) == args.warmup
    it0 = [s.case_info(k)["iters"] for k in range(len(cases))]
    stream = torch.cuda.ExternalStream(s.stream())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(_gpu_id(torch, local_rank)) as clk:
        e0.record(stream)
        s.enqueue(args.steps)
        e1.record(stream)
        done = s.wait()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    if done != args.steps:
        raise RuntimeError(f"only {done} of {args.steps} iterations ran")
    ms = e0.elapsed_time(e1)
    infos = [s.case_info(k) for k in range(len(cases))]
    # only the point-iterations of cases still running count: a case that
    # failed (non-physical update or non-finite norm) is frozen and skipped
    work = sum(c.n * (inf["iters"] - i0) for c, inf, i0 in zip(clouds, infos, it0))
    failed = sum(1 for inf in infos if inf["status"] != 0)
    ms_max, (n_all, work_all, failed_all) = combine_over_ranks(dist, ms, [float(n), float(work), float(failed)],
                                                               "cuda")
    value = work_all / (ms_max / 1e3)
    drops = [float(h[-1] / h[0]) for k, h in enumerate(s.case_residuals(k) for k in range(len(cases)))
             if infos[k]["status"] == 0]

    phases = s.time_phases(5)
    res_ms = phases["residual"]
    achieved = RES_FLOPS_PER_SLOT[MID_WORKLOAD] * nslots / (res_ms / 1e3) / 1e12

    e2e_steps = min(args.steps, 10)
    U = s.field(lskum.FIELD_U)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_conserved(U)
        s.run(1)
        U = s.field(lskum.FIELD_U)
    torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": world * work / args.steps * e2e_steps / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": int(U.nbytes),
           "d2h_bytes_per_step": int(U.nbytes) + 8}
    rates = None
    if args.solve_iters > 0:
        # per-case convergence: run on, then extrapolate each running case's
        # iterations to a 1e-8 drop from its rate over the last half
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.run(args.solve_iters)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        per = []
        for k in range(len(cases)):
            inf = s.case_info(k)
            h = s.case_residuals(k)
            if inf["status"] != 0 or len(h) < 200:
                per.append({"case": k, "status": inf["status"], "iters": inf["iters"]})
                continue
            m = len(h) // 2
            r = (h[-1] / h[m]) ** (1.0 / (len(h) - 1 - m))
            drop = h[-1] / h[0]
            est = len(h) + (np.log(1e-8 / drop) / np.log(r) if r < 1.0 and drop > 1e-8 else 0.0)
            per.append({"case": k, "points": clouds[k].n, "iters": len(h), "drop": float(drop), "rate": float(r),
                        "iters_to_1e-8_est": float(est) if r < 1.0 else None})
        ok = [q for q in per if q.get("iters_to_1e-8_est")]
        rates = {"extra_iters": args.solve_iters, "seconds": sec, "cases": per,
                 "est_iters_to_1e-8_median": float(np.median([q["iters_to_1e-8_est"] for q in ok])) if ok else None,
                 "est_iters_to_1e-8_max": float(max(q["iters_to_1e-8_est"] for q in ok)) if ok else None,
                 "estimate": "iterations so far + log(1e-8 / drop) / log(rate), rate per iteration over the last "
                             "half of the history"}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1:
        k0 = int(np.argmin([c.n for c in clouds]))
        cv, cdt, cdone = cpu_baseline(clouds[k0], 10, mach=cases[k0]["mach"], aoa=cases[k0]["aoa_deg"], K=2)
        cpu = {"value": cv, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{cdone} FP64 oracle iterations on the smallest case ({clouds[k0].n} points), one thread"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f64+f32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "cases": len(cases_all), "cases_this_rank": len(cases),
                   "points": int(n_all), "failed_cases": int(failed_all),
                   "point_iterations_timed": int(work_all), "precision": "fp64" if args.precision == 0 else
                   "fp32 sweeps, fp64 residual/update", "cfl": 100.0, "inner_iters": 2, "jvp": "exact-AD",
                   "order": f"second (timed steps follow {START} untimed first-order start-up iterations)",
                   "colours": info["n_colours"],
                   "launch_shape": {"threads_per_point": tpp, "sweep_lanes_per_point": lanes,
                                    "sweep_form": _sweep_form(lanes), "by": "autotune"},
                   "parallelism": f"cases sharded over {world} ranks" if world > 1 else "single",
                   "residual_drop_min_max": [min(drops), max(drops)] if drops else None,
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "alu", "kernel": "k_residual", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                     "flops_per_active_slot": RES_FLOPS_PER_SLOT[MID_WORKLOAD],
                     "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz (the FP64 unit)",
                     "note": ROOFLINE_NOTE,
                     "launch_ms": res_ms, "phase_ms": phases},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": info["launches_per_iter"] * args.steps,
        "clocks": clk.summary(),
    }
    if rates is not None:
        line["per_case_convergence"] = rates
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


WARM_WORKLOAD = "naca0012_warmstart"


def _drop_run(solver, target_abs, chunk, max_iters):
    """Run until the residual norm is at or below target_abs (absolute), in
    chunks of `chunk` iterations; returns (status, iterations, history)."""
    done, st = 0, 0
    h0 = None
    while done < max_iters:
        n = min(chunk, max_iters - done)
        if h0 is None:
            st, d = solver.run(1, check=False)
            done += d
            if st != 0 or d == 0:
                break
            h0 = solver.residuals()[0]
            if h0 <= target_abs:
                break
            continue
        st, d = solver.run(n, target_drop=target_abs / h0, check=False)
        done += d
        if st != 0 or d < n:
            break
    return st, done, solver.residuals()


def run_warmstart(args, rank, world, local_rank):
    """Wall time to a 1e-8 residual drop: plain FP64 from the free stream vs
    FP32 sweeps from the learned warm start, on the 160x64 NACA 0012 cloud at
    unseen (M, AoA).  The network is trained on the solver's own solutions at
    --train-solves random (M, AoA) (batched FP32-sweep solves, 3,000
    iterations each, 4,096 points sampled per solve).  Both arms use K = 2
    inner iterations (K = 3 diverges in the coarse far field in long runs).
    The warm arm must reach the plain arm's absolute final norm
    (1e-8 x the plain run's first norm)."""
    import numpy as np
    import torch

    from paper_2406_07441_gb300 import cloudgen as cg
    from paper_2406_07441_gb300 import lskum

    torch.cuda.set_device(local_rank)
    if rank != 0:
        return
    wl = "naca0012_160x64"
    cloud = cg.build_workload(wl)
    K, drop, max_iters = 2, 1e-8, 60000
    rng = np.random.default_rng(cg.BASE_SEED + 5)
    for _ in range(args.train_solves):  # the training draws come first from this generator
        rng.uniform(0.3, 0.85), rng.uniform(-4, 6)
    test = [(float(rng.uniform(0.3, 0.85)), float(rng.uniform(-4, 6))) for _ in range(args.test_conditions)]
    net, facts = train_network(args.train_solves, cg.BASE_SEED + 5, K=K)
    failed_train, n_samp, epochs = facts["train_failed"], facts["samples"], facts["epochs"]
    t_data, t_train = facts["data_s"], facts["train_s"]

    rows = []
    for (m, a) in test:
        sp = lskum.Solver(cloud, m, a, first_order_iters=START, inner_iters=K, precision=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st_p, it_p, hp = _drop_run(sp, np.inf, 5000, 1)  # first norm
        target = hp[0] * drop
        st_p, it_p2, hp = _drop_run(sp, target, 5000, max_iters - 1)
        torch.cuda.synchronize()
        tp = time.perf_counter() - t0
        it_p += it_p2
        ok_p = st_p == 0 and hp[-1] <= target
        sw = lskum.Solver(cloud, m, a, first_order_iters=0, inner_iters=K, precision=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kept = bool(net.predict(sw)[0])
        st_w, it_w, hw = _drop_run(sw, target, 5000, max_iters)
        torch.cuda.synchronize()
        tw = time.perf_counter() - t0
        ok_w = st_w == 0 and hw[-1] <= target
        clp, cdp = sp.forces()
        clw, cdw = sw.forces()
        rows.append(dict(mach=m, aoa=a, plain_ok=bool(ok_p), warm_ok=bool(ok_w), kept=kept, plain_iters=int(it_p),
                         warm_iters=int(it_w), plain_s=tp, warm_s=tw, h0_ratio=float(hw[0] / hp[0]),
                         dcl=abs(clw - clp), dcd=abs(cdw - cdp)))
        del sp, sw
    both = [r for r in rows if r["plain_ok"] and r["warm_ok"]]
    ratio = np.array([r["warm_s"] / r["plain_s"] for r in both]) if both else np.array([np.inf])
    it_ratio = np.array([r["warm_iters"] / r["plain_iters"] for r in both]) if both else np.array([np.inf])
    net.time_forward(FWD_POINTS, 3)
    fwd_ms = net.time_forward(FWD_POINTS, 20)
    mlp_flops = 2.0 * (34 * 128 + 3 * 128 * 128 + 128 * 4) * FWD_POINTS
    bf16_peak, peak_src = _bf16_peak()
    line = {
        "metric": "wall time to a 1e-8 residual drop, FP32 sweeps + learned warm start vs plain FP64 from the "
                  "free stream (ratio, median over unseen conditions)",
        "value": float(np.median(ratio)), "unit": "ratio", "higher_is_better": False, "n_gpus": 1,
        "steps": max_iters, "warmup": 0, "dtype": "f64 (plain) / f64 + f32 sweeps + bf16 network (warm)",
        "data": "synthetic",
        "config": {"workload": WARM_WORKLOAD, "cloud": wl, "points": cloud.n, "inner_iters": K, "cfl": 100.0,
                   "drop": drop, "train_solves": facts["train_solves"], "train_iters": 3000,
                   "train_failed": failed_train,
                   "samples": n_samp, "epochs": epochs, "test_conditions": len(test),
                   "plain": f"FP64, {START} first-order start-up iterations, then second order, to 1e-8 x first norm",
                   "warm": "FP32 sweeps, prediction judged by the residual, second order from iteration 1, "
                           "to the plain run's final absolute norm"},
        "warm_start": {
            "time_ratio_median": float(np.median(ratio)), "time_ratio_worst": float(np.max(ratio)),
            "iteration_ratio_median": float(np.median(it_ratio)), "iteration_ratio_worst": float(np.max(it_ratio)),
            "plain_s_median": float(np.median([r["plain_s"] for r in both])) if both else None,
            "warm_s_median": float(np.median([r["warm_s"] for r in both])) if both else None,
            "plain_iters_median": float(np.median([r["plain_iters"] for r in both])) if both else None,
            "warm_iters_median": float(np.median([r["warm_iters"] for r in both])) if both else None,
            "first_norm_ratio_median": float(np.median([r["h0_ratio"] for r in rows])),
            "prediction_kept": int(sum(r["kept"] for r in rows)),
            "plain_not_converged": int(sum(1 for r in rows if not r["plain_ok"])),
            "warm_not_converged": int(sum(1 for r in rows if r["plain_ok"] and not r["warm_ok"])),
            "cl_diff_max": float(max([r["dcl"] for r in both], default=float("nan"))),
            "cd_diff_max": float(max([r["dcd"] for r in both], default=float("nan"))),
            "data_s": t_data, "train_s": t_train, "final_loss": facts["final_loss"],
        },
        "cases": rows,
        "roofline": {"bound": "tensor", "kernel": "k_mlp_fused (network forward, all five layers)",
                     "achieved": mlp_flops / (fwd_ms / 1e3) / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": mlp_flops / (fwd_ms / 1e3) / 1e12 / bf16_peak, "traffic": None,
                     "forward_ms": fwd_ms, "points": FWD_POINTS, "flops": mlp_flops, "peak_source": peak_src},
    }
    print(json.dumps(line), flush=True)


def _bf16_peak():
    """Dense bf16 peak (TFLOP/s) for a kernel timed alone: the burst figure of
    MEASURED_PEAKS.json when present, else the profiling fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["bf16_tflops"])
        return v, "measured: MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback: 1.9 PFLOP/s bf16 burst"


def _memberships(cloud, kinetic=False):
    """Neighbour slots that join a split sub-stencil of a swept point (wall,
    interior and, under the kinetic far field, outer points)."""
    import numpy as np
    deg = np.diff(cloud.nbr_off)
    owner = np.repeat(np.arange(cloud.n), deg)
    dx = cloud.x[cloud.nbr_idx] - cloud.x[owner]
    dy = cloud.y[cloud.nbr_idx] - cloud.y[owner]
    wall = cloud.flag[owner] == 1
    outer = cloud.flag[owner] == 2
    framed = wall | (outer & kinetic)
    a = np.where(framed, dx * cloud.ny[owner] - dy * cloud.nx[owner], dx)
    b = np.where(framed, dx * cloud.nx[owner] + dy * cloud.ny[owner], dy)
    active = ~outer | kinetic
    return active & ((a != 0) | ((b > 0) & ~outer) | ((b < 0) & ~wall))


def _working_set_bytes(cloud):
    n, nnz = cloud.n, cloud.nnz
    per_slot = 4 + 1 + 6 * 8
    per_point = 8 * (2 * (4 + 4 + 20) + 4 * 4 + 4 + 1 + 4 + 4 + 13)
    return nnz * per_slot + n * per_point


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", type=int, choices=[0, 1], default=None,
                    help="0: plain FP64 (default for the single cloud); 1: FP32 sweeps with FP64 residual "
                         "and update (default for the batch)")
    ap.add_argument("--workload", choices=[WORKLOAD, MID_WORKLOAD, PROF_WORKLOAD, SMALL_WORKLOAD, SUPER_WORKLOAD,
                                           BATCH_WORKLOAD, WARM_WORKLOAD], default=WORKLOAD)
    ap.add_argument("--solve", choices=["on", "off"], default=None,
                    help="time the two solves to a 1e-8 drop on the 147,584-point cloud (default: on for the "
                         "default workload at N = 1)")
    ap.add_argument("--solve-max", type=int, default=80000, help="iteration cap of each of those solves")
    ap.add_argument("--solve-iters", type=int, default=-1,
                    help="single-cloud workloads: also time a whole solve of the workload itself to a 1e-8 drop, "
                         "at most this many iterations (default: 30000 for the supersonic one, else 0)")
    ap.add_argument("--train-solves", type=int, default=None,
                    help="warm-start network: training solves (default 256 for the solve block, 512 for the "
                         "warm-start study)")
    ap.add_argument("--test-conditions", type=int, default=16, help="warm-start workload: unseen conditions")
    ap.add_argument("--jvp", choices=["exact", "increment"], default="exact",
                    help="single-cloud workloads: exact (forward-mode AD) or increment Jacobian-vector products")
    ap.add_argument("--scheme", choices=["lusgs", "explicit"], default="lusgs",
                    help="single-cloud workloads: the implicit LU-SGS solver or the paper's explicit solver")
    ap.add_argument("--launch-shape", default="",
                    help="T,L: threads per point and sweep lanes per point instead of autotuning")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.precision is None:
        args.precision = 1 if args.workload == BATCH_WORKLOAD else 0
    if args.solve_iters < 0:
        args.solve_iters = 30000 if args.workload == SUPER_WORKLOAD else 0
    if args.train_solves is None:
        args.train_solves = 512 if args.workload == WARM_WORKLOAD else 256
    if args.solve is None:
        args.solve = "on" if (args.workload == WORKLOAD and args.scheme == "lusgs" and args.precision == 0
                              and args.jvp == "exact" and not args.launch_shape) else "off"
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.workload == BATCH_WORKLOAD:
        run_batch(args, rank, world, local_rank)
    elif args.workload == WARM_WORKLOAD:
        run_warmstart(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
