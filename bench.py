#!/usr/bin/env python3
"""Benchmark of the immersed-FSI hot path on GB300.

One step = one pass of the operator path over the 64^3 workload (background
hex grid 64^3 = 262,144 elements, 274,625 nodes, 1,098,500 DOFs; smooth
seeded Fourier velocity/pressure plus noise; three thin leaflets sampled as
200,000 solid points):

  stage (generalized alpha) -> VMS residual and Jacobian apply (one fused
  pass, fsi_residual_jacobian_apply) -> locate + cell table ->
  interpolation C^T V -> spreading C lambda

in native FP64 arithmetic throughout, on FP64 arrays (the location,
interpolation and spreading run on a second stream, concurrently with the VMS
pass; "ms_per_step_one_stream" and "ops_step" time the operators one after the
other).  value = DOFs (4 per node) passed through the step per second, in
GDOF/s.  The same step with the VMS operators, interpolation and spreading in
double-float arithmetic (pairs of floats on the FP32 pipe; "step_df64", with
its difference from the FP64 step), the operators in FP32 ("ops_f32") and the
extra sections (Newton step, ensemble, network, solid, mapped and tetrahedral
meshes) are timed in further loops.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own replica (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GDOF/s VMS Jacobian apply; s/Newton step at 1e-8 resid, mixed+learned vs FP64"
UNIT = "GDOF/s"
WORKLOAD = "64^3 Q1-Q1 VMS grid + 200k leaflet points (stage, residual, Jacobian apply, locate, interp, spread)"
N_GRID = 64
M_POINTS = 200_000
SEED = 2026
# Kernel launches per step issued by the library (stage 1, residual + Jacobian
# fused 2, locate 1 + scan 3 + scatter 1 + sort 1, interp 1, spread 2).
LAUNCHES_PER_STEP = 12
# dram__bytes_read.sum + dram__bytes_write.sum of one fused native FP64
# residual + Jacobian launch on the 64^3 workload, per brick schedule the
# autotuner picks (4x4x4 bricks, 128 threads: brick 26.43 + 0.23 MB, gather
# 32.79 + 0 MB; 8x4x2, 128 threads: brick 26.43 + 0.40 MB, gather 35.41 +
# 0.004 MB), from ncu captures of the current kernels with a cache flush
# between the two (profiles/vms_fused_f64_64cubed_ncu.md)
TRAFFIC_FUSED_F64_64 = {(4, 4, 4, 128): 26_429_696 + 226_304 + 32_786_432 + 0,
                        (8, 4, 2, 128): 26_429_952 + 403_712 + 35_407_616 + 4_096}
# FP64 operations the fused FP64 brick kernel executes per element (ncu,
# same capture: DFMA 1,808 (x2), DMUL 1,232, DADD 950): context for the
# roofline, whose achieved rate counts the oracle's operations
KERNEL_FP64_FLOPS_PER_ELEM = 2 * 1808 + 1232 + 950


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(ms_step, e2e_ms, units_per_rank, ws, device):
    """Weak scaling over replicas: the step time is the maximum over ranks (a
    collective MAX when ws > 1), and the whole-job value is the units all ranks
    processed (ws x units_per_rank) per second of that time, in G units/s.
    Returns (max step ms, max e2e ms, value, e2e value or None)."""
    import torch
    if ws > 1:
        t = torch.tensor([ms_step, e2e_ms], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step, e2e_ms = float(t[0]), float(t[1])
    value = ws * units_per_rank / (ms_step * 1e-3) / 1e9
    e2e_val = ws * units_per_rank / (e2e_ms * 1e-3) / 1e9 if math.isfinite(e2e_ms) else None
    return ms_step, e2e_ms, value, e2e_val


def make_workload(N=N_GRID, m=M_POINTS, seed=SEED):
    from paper_2601_08266_gb300 import inputs
    n = inputs.n_nodes(N)
    Vn = inputs.fourier_field(N, seed=seed)
    An = inputs.fourier_field(N, seed=seed + 1)
    y = inputs.fourier_field(N, seed=seed + 2)
    x = inputs.uniform_nodal(N, seed=seed + 3)
    X = inputs.leaflet_points(m, seed=seed + 4)
    lam = inputs.multipliers(m, seed=seed + 5)
    return dict(N=N, n=n, m=m, y=y, Vn=Vn, An=An, x=x, X=X, lam=lam)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def local_rel(a, b):
    """Largest relative difference of a from b over the momentum and the
    continuity slots of a nodal field (or the whole of a point array), both
    norm-wise and for the largest entry."""
    a, b = a.double(), b.double()
    groups = [slice(0, 3), slice(3, 4)] if b.shape[-1] == 4 else [slice(None)]
    worst = 0.0
    for g in groups:
        r = b[..., g]
        n2 = float(r.norm())
        if n2 == 0.0:
            continue
        d = a[..., g] - r
        worst = max(worst, float(d.norm()) / n2, float(d.abs().max()) / float(r.abs().max()))
    return worst


def vms_flops():
    """The oracle's operation count per element of the VMS operators, stored
    by tests/golden/make_vms_flops.py (read here as data)."""
    with open(os.path.join(ROOT, "tests", "golden", "vms_flops.json")) as f:
        return json.load(f)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ oracle arm
def oracle_pass(W, grid, phys, c_a, c_v, nthreads=0):
    import oracle.core as oc
    import oracle.timeint as ot
    U, A = ot.stage(W["y"], W["Vn"], W["An"], phys["dt"], phys["rho_inf"])
    oc.residual(grid, phys, U, A, nthreads=nthreads)
    oc.jacobian_apply(grid, phys, U, A, W["x"], c_a, c_v, nthreads=nthreads)
    elem, xi, _ = oc.locate(grid, W["X"])
    oc.cell_hash(grid, elem)
    oc.interp(grid, elem, xi, U)
    oc.spread(grid, elem, xi, W["lam"])


def cpu_oracle_rate(W, max_seconds=20.0, min_passes=1, nthreads=0):
    """Oracle FP64 passes over the full workload (nthreads OpenMP threads; 0 =
    the runtime's default, all host cores)."""
    import oracle.core as oc
    import oracle.timeint as ot
    oc.build()
    grid = oc.Grid(W["N"])
    phys = dict(rho=1.0, mu=0.01, dt=1e-3, rho_inf=0.5)
    c_a, c_v = ot.chain_factors(0.5, 1e-3)
    passes, t0 = 0, time.perf_counter()
    while passes < min_passes or time.perf_counter() - t0 < max_seconds * 0.5:
        oracle_pass(W, grid, phys, c_a, c_v, nthreads=nthreads)
        passes += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    el = time.perf_counter() - t0
    return 4.0 * W["n"] * passes / el / 1e9, passes, el


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    W = make_workload()
    import oracle.core as oc
    import oracle.timeint as ot
    oc.build()
    grid = oc.Grid(W["N"])
    phys = dict(rho=1.0, mu=0.01, dt=1e-3, rho_inf=0.5)
    c_a, c_v = ot.chain_factors(0.5, 1e-3)
    for _ in range(args.warmup):
        oracle_pass(W, grid, phys, c_a, c_v)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_pass(W, grid, phys, c_a, c_v)
    el = time.perf_counter() - t0
    value = 4.0 * W["n"] * args.steps / el / 1e9
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [W["N"]] * 3, "points": W["m"],
                   "l2": "CPU run"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full FP64 oracle passes over the workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    import paper_2601_08266_gb300 as fsi
    from paper_2601_08266_gb300 import _binding as B

    W = make_workload(N=args.grid, m=args.points, seed=SEED + rank)
    N, n, m = W["N"], W["n"], W["m"]
    stream = torch.cuda.Stream(device=dev)
    mesh = fsi.Mesh(N, rho=1.0, mu=0.01, dt=1e-3, rho_inf=0.5, device=local,
                    stream=stream.cuda_stream)
    # brick schedules of the VMS operators, one per compute type: the
    # library's autotuner times its candidate shapes on this grid
    schedule = W["schedule"] = {"autotuned": not args.no_autotune}
    for prec, tag in ((fsi.FSI_F64, "f64"), (fsi.FSI_DF64, "df64")):
        for op, name in ((0, "residual"), (1, "jacobian"), (2, "vms")):
            key = f"{name}_{tag}"
            if args.no_autotune:
                schedule[key] = {"brick": [8, 4, 4] if op == 2 else [8, 8, 4], "threads": 256}
            else:
                t = fsi.fsi_mesh_autotune(mesh, op, prec, reps=3 if tag == "f64" else 5)
                schedule[key] = {"brick": list(t["brick"]), "threads": t["threads"],
                                 "ms": round(t["seconds"] * 1e3, 4)}

    def buffers(dtype):
        b = {}
        with torch.cuda.stream(stream):
            for k in ("y", "Vn", "An", "x"):
                b[k] = torch.as_tensor(W[k], device=dev).to(dtype).contiguous()
            b["X"] = torch.as_tensor(W["X"], device=dev).contiguous()
            b["lam"] = torch.as_tensor(W["lam"], device=dev).to(dtype).contiguous()
            for k in ("U", "A", "R", "Jx", "F"):
                b[k] = torch.zeros((n, 4), dtype=dtype, device=dev)
            b["elem"] = torch.empty(m, dtype=torch.int32, device=dev)
            b["xi"] = torch.empty((m, 3), dtype=torch.float64, device=dev)
            b["cs"] = torch.empty(N ** 3 + 1, dtype=torch.int32, device=dev)
            b["perm"] = torch.empty(m, dtype=torch.int32, device=dev)
            b["u"] = torch.empty((m, 3), dtype=dtype, device=dev)
        stream.synchronize()
        return b

    b64 = buffers(torch.float64)
    P64 = fsi.FSI_F64
    # vms: the residual and the Jacobian apply, one fused pass
    ops = ["stage", "vms", "locate", "interp", "spread"]

    def step(b, P, ev=None, vms=fsi.FSI_F64, dlm=fsi.FSI_F64):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        fsi.fsi_stage(mesh, P, b["y"], b["Vn"], b["An"], None, b["U"], b["A"])
        mark(1)
        fsi.fsi_residual_jacobian_apply(mesh, vms, b["U"], b["A"], None, b["x"], b["R"], b["Jx"])
        mark(2)
        fsi.fsi_locate(mesh, b["X"], b["elem"], b["xi"], b["cs"], b["perm"], want_outside=False)
        mark(3)
        fsi.fsi_dlm_interp(mesh, dlm, b["elem"], b["xi"], b["U"], b["u"])
        mark(4)
        fsi.fsi_dlm_spread(mesh, dlm, b["elem"], b["xi"], b["cs"], b["perm"], b["lam"], None,
                           b["F"], False)
        mark(5)

    # The timed step runs the operators that do not depend on one another on two
    # streams: stage -> VMS pass on the mesh's stream; location (needs only the
    # points), then interpolation (after the stage) and spreading on a
    # higher-priority side stream, whose latency-bound kernels take SM slots as
    # the VMS pass's CTAs retire.  The mesh handle is switched between the
    # streams (fsi_mesh_set_stream); the operators use disjoint scratch.
    side = torch.cuda.Stream(device=dev, priority=-1)
    ev_start, ev_staged, ev_side = (torch.cuda.Event() for _ in range(3))

    def step_cc(b, P, vms=fsi.FSI_F64, dlm=fsi.FSI_F64):
        ev_start.record(stream)
        fsi.fsi_stage(mesh, P, b["y"], b["Vn"], b["An"], None, b["U"], b["A"])
        ev_staged.record(stream)
        side.wait_event(ev_start)
        mesh.set_stream(side.cuda_stream)
        fsi.fsi_locate(mesh, b["X"], b["elem"], b["xi"], b["cs"], b["perm"], want_outside=False)
        side.wait_event(ev_staged)
        fsi.fsi_dlm_interp(mesh, dlm, b["elem"], b["xi"], b["U"], b["u"])
        fsi.fsi_dlm_spread(mesh, dlm, b["elem"], b["xi"], b["cs"], b["perm"], b["lam"], None,
                           b["F"], False)
        ev_side.record(side)
        mesh.set_stream(stream.cuda_stream)
        fsi.fsi_residual_jacobian_apply(mesh, vms, b["U"], b["A"], None, b["x"], b["R"], b["Jx"])
        stream.wait_event(ev_side)

    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device=dev)

    def timed_total(run_step, K, Wm):
        """Mean step time between events on the mesh's stream (the side
        stream joins it before the end event)."""
        for _ in range(Wm):
            run_step()
        stream.synchronize()
        total = 0.0
        for _ in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)          # evict the working set from L2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run_step()
            e1.record(stream)
            stream.synchronize()
            total += e0.elapsed_time(e1)
        return total / K

    def timed(run_step, K, Wm):
        for _ in range(Wm):
            run_step(None)
        stream.synchronize()
        per_op = np.zeros(len(ops))
        total = 0.0
        for _ in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)          # evict the working set from L2
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(ops) + 1)]
            run_step(ev)
            stream.synchronize()
            d = [ev[i].elapsed_time(ev[i + 1]) for i in range(len(ops))]
            per_op += d
            total += ev[0].elapsed_time(ev[-1])
        return total / K, per_op / K

    sampler = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    # the two-stream step must give bitwise the one-stream step's results
    keys = ("U", "A", "R", "Jx", "elem", "xi", "cs", "perm", "u", "F")
    step(b64, P64)
    stream.synchronize()
    ref = [b64[k].clone() for k in keys]
    step_cc(b64, P64)
    stream.synchronize()
    for k, r in zip(keys, ref):
        if not torch.equal(b64[k], r):
            raise RuntimeError(f"two-stream step: {k} differs from the one-stream step")
    # the headline: the step in native FP64 arithmetic throughout
    ms64 = timed_total(lambda: step_cc(b64, P64), args.steps, args.warmup)
    # the operators one after the other on one stream, for the per-operator split
    ms64_seq, per64 = timed(lambda ev: step(b64, P64, ev), args.steps, args.warmup)
    W["ms_seq"] = ms64_seq
    torch.cuda.synchronize()
    fp64_out = {k: b64[k].clone() for k in ("R", "Jx", "u", "F")}
    # the same step with the VMS operators, interpolation and spreading in
    # double-float arithmetic (FP64 arrays), and how far it is from FP64
    df = dict(vms=fsi.FSI_DF64, dlm=fsi.FSI_DF64)
    msnat = timed_total(lambda: step_cc(b64, P64, **df), args.steps, args.warmup)
    _, pernat = timed(lambda ev: step(b64, P64, ev, **df), args.steps, args.warmup)
    torch.cuda.synchronize()
    W["df64_vs_f64"] = {k: local_rel(b64[k], fp64_out[k]) for k in fp64_out}
    # FP32 operators (xi cast once outside the timed loop)
    b32 = buffers(torch.float32)
    fsi.fsi_locate(mesh, b32["X"], b32["elem"], b32["xi"], b32["cs"], b32["perm"],
                   want_outside=False)
    xi32 = b32["xi"].to(torch.float32)
    ops32 = ["residual", "jacobian", "interp", "spread"]

    def step32(ev):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        fsi.fsi_residual(mesh, fsi.FSI_F32, b32["U"], b32["A"], None, b32["R"])
        mark(1)
        fsi.fsi_jacobian_apply(mesh, fsi.FSI_F32, b32["U"], b32["A"], None, b32["x"], b32["Jx"])
        mark(2)
        fsi.fsi_dlm_interp(mesh, fsi.FSI_F32, b32["elem"], xi32, b32["U"], b32["u"])
        mark(3)
        fsi.fsi_dlm_spread(mesh, fsi.FSI_F32, b32["elem"], xi32, b32["cs"], b32["perm"],
                           b32["lam"], None, b32["F"], False)
        mark(4)
        for i in range(4, len(ops) + 1):
            mark(i)

    fsi.fsi_stage(mesh, fsi.FSI_F32, b32["y"], b32["Vn"], b32["An"], None, b32["U"], b32["A"])
    ms32, per32 = timed(step32, args.steps, args.warmup)

    # FP64-accurate VMS operators in double-float arithmetic (FP64 arrays)
    def stepdf(ev):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        fsi.fsi_residual(mesh, fsi.FSI_DF64, b64["U"], b64["A"], None, b64["R"])
        mark(1)
        fsi.fsi_jacobian_apply(mesh, fsi.FSI_DF64, b64["U"], b64["A"], None, b64["x"], b64["Jx"])
        for i in range(2, len(ops) + 1):
            mark(i)
    msdf, perdf = timed(stepdf, args.steps, args.warmup)
    per32 = np.concatenate([per32[:4], perdf[:2]])

    # the native FP64 residual and Jacobian apply, one after the other
    def stepnat(ev):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        fsi.fsi_residual(mesh, fsi.FSI_F64, b64["U"], b64["A"], None, b64["R"])
        mark(1)
        fsi.fsi_jacobian_apply(mesh, fsi.FSI_F64, b64["U"], b64["A"], None, b64["x"], b64["Jx"])
        for i in range(2, len(ops) + 1):
            mark(i)
    _, pernatops = timed(stepnat, args.steps, args.warmup)
    pernat = np.concatenate([pernat, pernatops[:2]])
    # the e2e arm below runs the headline (native FP64) step
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if args.no_e2e:
        return finish(args, W, ws, rank, local, mesh, ms64, per64, ms32, per32, ops, ops32,
                      clocks, None, 0, 0, (msnat, pernat))

    # end to end through host buffers (pinned), FP64 step
    h_in = {k: torch.as_tensor(W[k]).pin_memory() for k in ("y", "Vn", "An", "x", "X", "lam")}
    h_out = {k: torch.empty(tuple(b64[k].shape), dtype=b64[k].dtype).pin_memory()
             for k in ("R", "Jx", "u", "F")}
    h2d = sum(t.numel() * t.element_size() for t in h_in.values())
    d2h = sum(t.numel() * t.element_size() for t in h_out.values())

    # Two device buffer sets and a copy stream: the upload of step k+1's inputs
    # and the download of step k's results overlap step k's kernels.  Every
    # step still moves all its inputs in and its results out.
    copy_s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        sets = [b64, {k: v.clone() for k, v in b64.items()}]
    stream.synchronize()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]

    def upload(k):
        b = sets[k % 2]
        with torch.cuda.stream(copy_s):
            for key, t in h_in.items():
                b[key].copy_(t, non_blocking=True)
        ev_in[k % 2].record(copy_s)

    def compute_and_download(k):
        b = sets[k % 2]
        stream.wait_event(ev_in[k % 2])
        step_cc(b, P64)
        ev_done[k % 2].record(stream)
        copy_s.wait_event(ev_done[k % 2])
        with torch.cuda.stream(copy_s):
            for key, t in h_out.items():
                t.copy_(b[key], non_blocking=True)

    def e2e_run(K, e0=None, e1=None):
        # copy-stream order: up(0), up(1), down(0), up(2), down(1), ...; up(k+1)
        # reuses the set of step k-1, whose download precedes it on the stream
        if e0 is not None:
            e0.record(copy_s)
        upload(0)
        for k in range(K):
            if k + 1 < K:
                upload(k + 1)
            compute_and_download(k)
        if e1 is not None:
            e1.record(copy_s)
        copy_s.synchronize()
        stream.synchronize()

    e2e_run(args.warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_run(args.steps, e0, e1)
    e2e_ms = e0.elapsed_time(e1) / args.steps
    return finish(args, W, ws, rank, local, mesh, ms64, per64, ms32, per32, ops, ops32, clocks,
                  e2e_ms, h2d, d2h, (msnat, pernat))


def finish(args, W, ws, rank, local, mesh, ms64, per64, ms32, per32, ops, ops32, clocks, e2e_ms,
           h2d, d2h, native):
    import torch
    import paper_2601_08266_gb300 as fsi
    from paper_2601_08266_gb300 import _binding as B
    N, n, m = W["N"], W["n"], W["m"]
    dev = torch.device(f"cuda:{local}")
    if e2e_ms is None:
        e2e_ms = float("nan")
    t_step, e2e_ms, value, e2e_val = aggregate_over_ranks(ms64, e2e_ms, 4.0 * n, ws, dev)

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
        return 0

    # roofline of the dominant kernel of the FP64 step: the fused native FP64
    # residual + Jacobian pass (brick + gather), bound by the FP64 pipe (plain
    # ALU arithmetic, no tensor cores; the HBM bytes take microseconds).
    # achieved = the oracle's operation count per element (one element's
    # computation, constants folded, common subexpressions merged) x elements
    # / the pass's CUDA-event time; peak = the FP64 FMA rate probed in this run
    # (MEASURED_PEAKS.json has no FP64 figure)
    fma64 = B.fsi_measure_fma_peak(local, fsi.FSI_F64)
    fma32 = B.fsi_measure_fma_peak(local, fsi.FSI_F32)
    E = N ** 3
    fl = vms_flops()
    asm_ = (32.0 * E - 4.0 * n) / E
    flops_elem = {k: fl["per_element"][k]["element"] + (2 if k == "fused" else 1) * asm_
                  for k in ("residual", "jacobian", "fused")}
    vms_ms = per64[ops.index("vms")]
    schedule = W["schedule"]
    achieved = flops_elem["fused"] * E / (vms_ms * 1e-3)
    # DRAM bytes of one fused FP64 launch (brick + gather kernels), from an
    # ncu capture of this workload; only meaningful for the 64^3 grid
    vms_sched = tuple(schedule["vms_f64"]["brick"]) + (schedule["vms_f64"]["threads"],)
    traffic = TRAFFIC_FUSED_F64_64.get(vms_sched) if N == N_GRID else None
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)

    def gdofs(ms):
        return 4.0 * n / (ms * 1e-3) / 1e9

    op_tab = {o: {"ms": round(float(t), 5), "gdof_s": round(gdofs(t), 4)} for o, t in zip(ops, per64)}
    # the double-float step: per-operator split and native residual / Jacobian alone
    df_step_ops = {o: {"ms": round(float(t), 5)} for o, t in zip(ops, native[1][:len(ops)])}
    nat_res, nat_jac = native[1][len(ops)], native[1][len(ops) + 1]
    op_nat = {o: {"ms": round(float(t), 5), "gdof_s": round(gdofs(t), 4)}
              for o, t in zip(("residual", "jacobian"), (nat_res, nat_jac))}
    for o, t in (("residual", nat_res), ("jacobian", nat_jac)):
        r = flops_elem[o] * E / (t * 1e-3)
        op_nat[o]["method_tflop_s"] = round(r / 1e12, 4)
        op_nat[o]["frac_of_fp64_fma_peak"] = round(r / fma64, 4)
    op_tab32 = {o: {"ms": round(float(t), 5), "gdof_s": round(gdofs(t), 4)}
                for o, t in zip(ops32, per32[:4])}
    op_tabdf = {o: {"ms": round(float(t), 5), "gdof_s": round(gdofs(t), 4),
                    "method_tflop_s": round(flops_elem[o] * E / (t * 1e-3) / 1e12, 3),
                    "frac_of_fp32_fma_peak": round(flops_elem[o] * E / (t * 1e-3) / fma32, 4)}
                for o, t in zip(("residual", "jacobian"), per32[4:6])}
    # HBM-bound DLM operators: algorithmic bytes per launch
    bytes_interp64 = m * (4 + 24 + 24)
    bytes_spread64 = m * (4 + 4 + 24 + 24) + (E + 1) * 4 + n * 24
    # algorithmic bytes of the operators (every array touched once; the fused
    # VMS pass reads U, A, x and writes R, Jx)
    alg_bytes = {"stage": n * 160, "vms": n * 160,
                 "locate": m * (24 + 28 + 8) + (E + 1) * 4,
                 "interp": bytes_interp64, "spread": bytes_spread64}
    for o, t in zip(ops, per64):
        gbs = alg_bytes[o] / (t * 1e-3) / 1e9
        op_tab[o]["gb_s"] = round(gbs, 1)
        op_tab[o]["hbm_frac"] = round(gbs / hbm, 4)
        if o in ("locate", "interp", "spread"):
            op_tab[o]["points_per_s"] = round(m / (t * 1e-3), 1)
    for o, t in zip(ops, native[1][:len(ops)]):
        if o in ("locate", "interp", "spread"):
            df_step_ops[o]["hbm_frac"] = round(alg_bytes[o] / (t * 1e-3) / 1e9 / hbm, 4)
    op_tab32["jacobian"]["method_tflop_s"] = round(flops_elem["jacobian"] * E / (per32[1] * 1e-3) / 1e12, 3)
    op_tab32["jacobian"]["frac_of_fp32_fma_peak"] = round(
        flops_elem["jacobian"] * E / (per32[1] * 1e-3) / fma32, 4)
    op_tab["vms"]["method_tflop_s"] = round(achieved / 1e12, 4)
    df_vms_ms = native[1][ops.index("vms")]
    df_rate = flops_elem["fused"] * E / (df_vms_ms * 1e-3)

    cpu = None
    if ws == 1 and not args.no_cpu_baseline and N == N_GRID and m == M_POINTS:
        cores = os.cpu_count()
        rate, passes, el = cpu_oracle_rate(W, max_seconds=args.cpu_seconds, nthreads=cores)
        rate1, passes1, el1 = cpu_oracle_rate(W, max_seconds=args.cpu_seconds / 2, nthreads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "value_1_thread": rate1,
               "sample_1_thread": f"{passes1} pass(es), {el1:.1f} s",
               "sample": f"{passes} full FP64 oracle pass(es) of the step on the 64^3 workload "
                         f"({el:.1f} s, OpenMP over elements)"}

    extras = {}
    if not args.no_extras:
        stream2 = torch.cuda.Stream(device=dev)
        sections = args.sections.split(",")
        if "newton" in sections:
            extras["newton"] = newton_section(args, dev, stream2)
        if "batch" in sections:
            extras["batch"] = batch_section(args, dev, stream2)
        if "mlp" in sections:
            extras["mlp_inference"] = mlp_section(args, dev, stream2, W)
        if "solid" in sections:
            extras["solid"] = solid_section(args, dev, stream2)
        if "dlm" in sections:
            extras["dlm_128"] = dlm_section(args, dev, stream2)
        if "mapped" in sections:
            extras["mapped"] = mapped_section(args, dev, stream2)
        if "tet" in sections:
            extras["tet"] = tet_section(args, dev, stream2)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
        "ms_per_step_one_stream": W.get("ms_seq"),
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "arithmetic": "native IEEE FP64 throughout: stage, VMS residual + Jacobian apply (one "
                      "fused pass), location, interpolation, spreading",
        "config": {"workload": WORKLOAD if (N, m) == (N_GRID, M_POINTS) else
                   f"{N}^3 grid + {m} leaflet points (profiling case)",
                   "grid": [N, N, N], "dofs": 4 * n, "points": m,
                   "l2": "flushed between timed steps (write of a buffer > L2)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "roofline": {"bound": "alu",
                     "kernel": "vms residual + Jacobian apply, native FP64, fused (brick + gather)",
                     "achieved": achieved / 1e12, "peak": fma64 / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / fma64,
                     "traffic": traffic,
                     "flops_per_element": flops_elem["fused"],
                     "flops_source": "tests/golden/vms_flops.json: the oracle's operations for one "
                                     "element's residual and Jacobian apply (oracle/flops.cpp: "
                                     "constants folded, common subexpressions merged) + the "
                                     "assembly additions; the oracle sums over the 8 nodes where "
                                     "the kernel uses the tensor-product butterflies, so the "
                                     "kernel executes fewer operations than this count",
                     "peak_source": "FP64 FMA rate probed in this run (fsi_measure_fma_peak; "
                                    "MEASURED_PEAKS.json has no FP64 figure)",
                     "kernel_flops_per_element": KERNEL_FP64_FLOPS_PER_ELEM,
                     "kernel_flop_frac": KERNEL_FP64_FLOPS_PER_ELEM * E / (vms_ms * 1e-3) / fma64,
                     "kernel_flops_source": "ncu FP64 instruction counts of the fused brick kernel "
                                            "at 64^3 (DFMA x 2 + DMUL + DADD); its FP64 pipe is "
                                            "85 % active"},
        "schedule": schedule,
        "step_df64": {
            "ms": native[0], "gdof_s": gdofs(native[0]),
            "arithmetic": "VMS, interpolation and spreading in double-float (pairs of FP32, "
                          "~48-bit significand, FP32 exponent range) on FP64 arrays; stage and "
                          "location in FP64",
            "rel_diff_vs_f64_step": W.get("df64_vs_f64"),
            "ops": df_step_ops,
            "vms_method_tflop_s": df_rate / 1e12,
            "vms_frac_of_fp32_fma_peak": df_rate / fma32},
        "cpu_baseline": cpu,
        "e2e": None if e2e_val is None else {
            "value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "copies": "pinned host buffers; a copy stream uploads step k+1's inputs and "
                      "downloads step k's results while step k computes (two device "
                      "buffer sets); first upload and last download inside the timed region"},
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "clocks": clocks,
        "ops_step": op_tab,
        "ops_native_f64_alone": op_nat,
        "ops_f32": op_tab32,
        "ops_df64": op_tabdf,
        "ms_per_step_f32_ops": ms32,
        "alu_peaks_tflop_s": {"f64": fma64 / 1e12, "f32": fma32 / 1e12},
        "hbm_peak_gbs": hbm,
    }
    line.update(extras)
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.barrier()
    mesh.close()
    return 0

# ------------------------------------------------------------------ Newton section
class Channel:
    """Channel-like flow on an N^3 unit-cube grid (Re ~ 1000: mu = 1e-3, peak
    inflow 1): inflow v_x = 16 y(1-y) z(1-z) at x = 0, no-slip walls at y, z in
    {0, 1}, traction-free outflow at x = 1; initial velocity = the inflow
    profile plus 0.01 x a seeded smooth Fourier perturbation.  Three leaflets
    of m volume-weighted points (total volume 0.024, rho_s - rho_f = 0.5)."""

    def __init__(self, fsi, dev, stream, N, m, leaflet_seed, dt=1e-3, mu=1e-3, bubble=0.0):
        import torch
        from paper_2601_08266_gb300 import inputs
        self.fsi, self.dev, self.stream, self.N, self.m, self.dt = fsi, dev, stream, N, m, dt
        self.mesh = fsi.Mesh(N, rho=1.0, mu=mu, dt=dt, rho_inf=0.5, device=dev.index,
                             stream=stream.cuda_stream)
        n = self.n = self.mesh.n_nodes
        ax = np.arange(N + 1) / N
        Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
        X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
        if bubble:
            # a mapped grid: the faces of the cube stay in place (same masks)
            with torch.cuda.stream(stream):
                self.mesh.set_coordinates(torch.as_tensor(bubble_map(np.stack([X, Y, Z], 1),
                                                                     bubble), device=dev))
        prof = 16.0 * Y * (1 - Y) * Z * (1 - Z)
        wall = (Y < 1e-12) | (Y > 1 - 1e-12) | (Z < 1e-12) | (Z > 1 - 1e-12)
        inflow = (X < 1e-12) & ~wall
        mask = np.zeros((n, 4), dtype=np.uint8)
        mask[wall | inflow, :3] = 1
        V0 = np.zeros((n, 4))
        V0[:, 0] = prof
        V0[:, :3] += 0.01 * inputs.fourier_field(N, seed=SEED + 30, noise=0.0, ncomp=3)
        V0[mask[:, 0].astype(bool), :3] = 0.0
        V0[inflow, 0] = prof[inflow]
        g = np.zeros((n, 3))
        g[inflow, 0] = prof[inflow]
        self.gamma = 2.0 / 3.0
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
        with torch.cuda.stream(stream):
            self.Vn = T(V0)
            self.An = torch.zeros_like(self.Vn)
            self.yn, self.d1, self.d2 = (torch.zeros_like(self.Vn) for _ in range(3))
            self.g = T(g)
            self.mask = T(mask)
            self.maskb = self.mask.bool()
            self.e = torch.empty(m, dtype=torch.int32, device=dev)
            self.xi = torch.empty((m, 3), dtype=torch.float64, device=dev)
            self.cs = torch.empty(self.mesh.n_elems + 1, dtype=torch.int32, device=dev)
            self.pm = torch.empty(m, dtype=torch.int32, device=dev)
            self.w = torch.full((m,), 0.024 / m, dtype=torch.float64, device=dev)
        fsi.fsi_locate(self.mesh, T(inputs.leaflet_points(m, seed=leaflet_seed)), self.e,
                       self.xi, self.cs, self.pm)
        self.k = 0

    def dirichlet(self):
        """y_D for the unknown V_dot_{n+1}: the velocity update reaches g."""
        import torch
        with torch.cuda.stream(self.stream):
            yD = torch.zeros_like(self.Vn)
            yD[:, :3] = (self.g - self.Vn[:, :3] - self.dt * (1 - self.gamma) * self.An[:, :3]) / (
                self.gamma * self.dt)
        return yD

    def state(self, guess="extrapolated"):
        """Predictor y (extrapolated increment or zero increment) and its step state."""
        import torch
        yD = self.dirichlet()
        with torch.cuda.stream(self.stream):
            y = self.yn + 2 * self.d1 - self.d2 if guess == "extrapolated" else self.yn.clone()
            y[self.maskb] = yD[self.maskb]
        st = self.fsi.StepState(y, self.Vn, self.An, mask=self.mask, yD=yD, elem=self.e,
                                xi=self.xi, cell_start=self.cs, perm=self.pm, w=self.w,
                                drho_s=0.5)
        return y, st

    def advance(self, y):
        """Accept y as the step's solution: increments and history move on."""
        import torch
        with torch.cuda.stream(self.stream):
            dn = y - self.yn
            self.d2, self.d1, self.yn = self.d1, dn, y.clone()
        self.fsi.fsi_advance_history(self.mesh, self.fsi.FSI_F64, y, self.Vn, self.An)
        self.k += 1

    def close(self):
        self.mesh.close()


def train_network(args, dev, stream, fsi, feats, targs, gen):
    """Adam on the GPU (BF16 tensor-core forward/backward) over the collected
    (features, correction) pairs; per-channel normalisation from the pairs."""
    import torch
    with torch.cuda.stream(stream):
        Xa = torch.cat(feats)[:args.train_samples]
        Ca = torch.cat(targs)[:args.train_samples].float()
        im, isd = Xa.mean(0), Xa.std(0) + 1e-6
        om, osd = Ca.mean(0), Ca.std(0) + 1e-12
        Xn = ((Xa - im) / isd).contiguous()
        Cn = ((Ca - om) / osd).contiguous()
        P = torch.zeros(fsi.fsi_mlp_num_params(), device=dev)
        off = 0
        for fan_in, size in ((112, 112 * 256), (0, 256), (256, 256 * 256), (0, 256), (256, 1024),
                             (0, 4)):
            if fan_in:
                P[off:off + size] = torch.randn(size, device=dev, generator=gen) * (2.0 / fan_in) ** 0.5
            off += size
        Mo, Vo, G = torch.zeros_like(P), torch.zeros_like(P), torch.empty_like(P)
        loss = torch.empty(1, dtype=torch.float32, device=dev)
    h = fsi.Mlp(65536, device=dev.index, stream=stream.cuda_stream)
    losses = []
    for it in range(1, args.mlp_iters + 1):
        with torch.cuda.stream(stream):
            idx = torch.randint(0, Xn.shape[0], (4096,), device=dev, generator=gen)
            xb, cb = Xn[idx].contiguous(), Cn[idx].contiguous()
        fsi.fsi_mlp_loss_grad(h, P, xb, cb, loss, G)
        fsi.fsi_mlp_adam(h, P, G, Mo, Vo, it, lr=1e-3)
        if it in (1, args.mlp_iters):
            stream.synchronize()
            losses.append(float(loss.item()))
    h.check()  # no tensor-core wait ran out
    return h, P, im, isd, om, osd, Xn, losses


def newton_section(args, dev, stream):
    """Implicit steps of the channel flow with leaflets (Re ~ 1000, dt = 1e-3).
    A BF16 network is trained on the GPU on node samples from plain-solver runs
    on 64^3 grids with seeded leaflet positions, then applied on the 128^3 grid
    with 1M points.  One step there is solved to ||R|| <= 1e-8 r_ref (r_ref =
    residual of the extrapolated predictor) by plain FP64 Newton-GMRES, by the
    mixed FP32/FP64 solver from the zero and the extrapolated guess, and by the
    mixed solver from the learned guess."""
    import torch
    import paper_2601_08266_gb300 as fsi
    # krylov_rtol is the floor of the target-aware forcing (see fsi_newton_step)
    solve = dict(restart=50, max_newton=10, max_krylov=4000, newton_rtol=1e-8,
                 krylov_rtol=args.krylov_floor)
    wanted = set(args.newton_variants.split(","))
    learned = "mixed_learned" in wanted
    zeros = torch.zeros(112, dtype=torch.float32, device=dev)
    ones = torch.ones(112, dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev).manual_seed(SEED)
    # 1) training pairs from plain-solver runs on the training grid
    t0 = time.perf_counter()
    feats, targs = [], []
    runs, steps = (args.train_runs, args.train_steps) if learned else (0, 3)
    per_step = -(-args.train_samples // (runs * (steps - 2))) if runs else 0
    for r in range(runs):
        ch = Channel(fsi, dev, stream, args.train_grid, args.train_points, SEED + 40 + r)
        for k in range(steps):
            y, st = ch.state()
            if k >= 2:
                with torch.cuda.stream(stream):
                    idx = torch.randint(0, ch.n, (per_step,), device=dev, generator=gen,
                                        dtype=torch.int64).to(torch.int32)
                    Xf = torch.empty((per_step, 112), dtype=torch.float32, device=dev)
                fsi.fsi_mlp_features(ch.mesh, ch.Vn, ch.yn, ch.d1, ch.d2, idx, zeros, ones, Xf)
            fsi.fsi_newton_step(ch.mesh, st, mixed=True, residual_prec=fsi.FSI_DF64, **solve)
            if k >= 2:
                with torch.cuda.stream(stream):
                    dn = (y - ch.yn)[idx.long()]
                    tg = dn - (2 * ch.d1 - ch.d2)[idx.long()]
                    tg[ch.maskb[idx.long()]] = 0.0
                    feats.append(Xf)
                    targs.append(tg)
            ch.advance(y)
        ch.close()
    stream.synchronize()
    gen_s = time.perf_counter() - t0
    # 2) training on the GPU (BF16 tensor-core forward/backward, Adam)
    t0 = time.perf_counter()
    h = None
    losses = []
    Xn = torch.empty((0, 112), device=dev)
    im = isd = om = osd = P = None
    if learned:
        h, P, im, isd, om, osd, Xn, losses = train_network(args, dev, stream, fsi, feats, targs,
                                                          gen)
    train_s = time.perf_counter() - t0
    # 3) the evaluation grid: warm steps, then one step four ways
    ch = Channel(fsi, dev, stream, args.newton_grid, args.newton_points, SEED + 60)
    # brick schedules of the operators the mixed step runs most: the FP32
    # Jacobian apply of the Krylov iterations and the double-float residual
    schedule = {}
    if not args.no_autotune:
        for op, prec, name in ((1, fsi.FSI_F32, "jacobian_f32"), (0, fsi.FSI_DF64, "residual_df64")):
            t = fsi.fsi_mesh_autotune(ch.mesh, op, prec, reps=3)
            schedule[name] = {"brick": list(t["brick"]), "threads": t["threads"],
                              "ms": round(t["seconds"] * 1e3, 4)}
    for _ in range(args.newton_warm):
        y, st = ch.state()
        fsi.fsi_newton_step(ch.mesh, st, mixed=True, residual_prec=fsi.FSI_DF64, **solve)
        ch.advance(y)
    work = torch.empty((5, ch.n, 4), dtype=torch.float64, device=dev)
    out = {"grid": [ch.N] * 3, "dofs": 4 * ch.n, "points": ch.m, "dt": ch.dt, "mu": 1e-3,
           "history_steps": ch.k, "schedule": schedule,
           "training": {"grid": [args.train_grid] * 3, "points": args.train_points,
                        "runs": runs, "steps_per_run": steps,
                        "samples": int(Xn.shape[0]), "generate_seconds": gen_s,
                        "train_seconds": train_s, "iters": args.mlp_iters, "loss": losses}}
    S, BJ = fsi.PRECOND_SCHUR, fsi.PRECOND_BLOCK_JACOBI
    variants = [("fp64", False, "extrapolated", S), ("mixed_zero_guess", True, "zero", S),
                ("mixed", True, "extrapolated", S), ("mixed_learned", True, "learned", S),
                ("mixed_block_jacobi", True, "extrapolated", BJ)]
    variants = [v for v in variants if v[0] in wanted]
    out["preconditioner"] = ("block-diagonal Schur complement: 3x3 velocity blocks + one "
                             "pressure multigrid V-cycle (mixed_block_jacobi: nodal 4x4 "
                             "block-Jacobi)")
    out["residual"] = ("fp64: native FP64 residual; mixed variants: FP64-accurate double-float "
                       "residual (VMS, interp, spread; ~1e-14 vs FP64), also for the predictor's "
                       "judge")
    r_ref = None
    im_f = isd_f = om_c = osd_c = None
    if im is not None:  # the network was trained (the learned variant is wanted)
        im_f, isd_f = im.float().contiguous(), isd.float().contiguous()
        om_c, osd_c = om.contiguous(), osd.contiguous()
    # the same step from the same state, repeated (median wall time): the
    # mixed variants --newton-reps times, the slow FP64 one once
    for name, mixed, guess_kind, pc in variants:
        times, preds = [], []
        for rep_i in range(args.newton_reps if mixed else 1):
            y, st = ch.state("zero" if guess_kind == "zero" else "extrapolated")
            stream.synchronize()
            torch.cuda.nvtx.range_push(f"newton_{name}")
            t0 = time.perf_counter()
            guess = None
            R0 = None
            if guess_kind == "learned":
                guess = fsi.fsi_mlp_guess(h, ch.mesh, P, im_f, isd_f, om_c, osd_c,
                                          st, ch.yn, ch.d1, ch.d2, 0, work,
                                          judge_prec=fsi.FSI_DF64)
                # the judge's residual of the returned predictor is Newton's first
                R0 = work[0]
                preds.append(time.perf_counter() - t0)
            code, rep = fsi.fsi_newton_step(ch.mesh, st, mixed=mixed, r_ref=r_ref or 0.0,
                                            check=False, precond=pc,
                                            residual_prec=fsi.FSI_DF64 if mixed else fsi.FSI_F64,
                                            R0=R0, **solve)
            stream.synchronize()
            times.append(time.perf_counter() - t0)
            torch.cuda.nvtx.range_pop()
        if r_ref is None:
            r_ref = rep["r_ref"]
        out[name] = {"seconds": float(np.median(times)), "seconds_all": times,
                     "newton_iters": rep["newton_iters"],
                     "krylov_iters": rep["krylov_iters"], "r0_over_ref": rep["r0"] / r_ref,
                     "r_final_over_ref": rep["r_final"] / r_ref,
                     "converged": bool(rep["converged"]), "status": code}
        if guess is not None:
            out[name]["predictor"] = {k2: guess[k2] for k2 in (
                "r_fallback", "r_learned", "r_history_fit", "r_combined", "used",
                "c_d1", "c_d2", "c_net")}
            out[name]["predictor"]["seconds"] = float(np.median(preds))
    if {"fp64", "mixed"} <= wanted:
        out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    if {"fp64", "mixed_learned"} <= wanted:
        out["speedup_mixed_learned_vs_fp64"] = (out["fp64"]["seconds"] /
                                                out["mixed_learned"]["seconds"])
    if {"mixed", "mixed_learned"} <= wanted:
        out["speedup_learned_vs_extrapolated"] = (out["mixed"]["seconds"] /
                                                  out["mixed_learned"]["seconds"])
    if {"mixed_zero_guess", "mixed_learned"} <= wanted:
        out["speedup_learned_vs_zero"] = (out["mixed_zero_guess"]["seconds"] /
                                          out["mixed_learned"]["seconds"])
    if h is not None:
        h.close()
    # the Krylov BLAS-1 kernels on vectors of this grid's size (FP32, as in the
    # mixed solve): algorithmic bytes per call / CUDA-event time
    from paper_2601_08266_gb300 import _binding as B
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    length = 4 * ch.n
    blas = {"vector_mb_f32": length * 4 / 1e6}
    for nvec in (8, 24, 48):
        td, ta = B.fsi_measure_blas1(dev.index, fsi.FSI_F32, length, nvec, reps=10)
        bd = (nvec + -(-nvec // 8)) * length * 4
        ba = (nvec + 2) * length * 4
        blas[str(nvec)] = {"dot_ms": td * 1e3, "dot_gb_s": bd / td / 1e9,
                           "dot_hbm_frac": bd / td / 1e9 / hbm,
                           "update_ms": ta * 1e3, "update_gb_s": ba / ta / 1e9,
                           "update_hbm_frac": ba / ta / 1e9 / hbm}
    out["krylov_blas1"] = blas
    ch.close()
    return out


# ------------------------------------------------------------------ batched ensemble
def batch_section(args, dev, stream):
    """64 independent instances (N ~ U{16..48}, mu ~ logU[1e-3, 1e-1], 10k-150k
    leaflet points each): per-instance launches vs persistent grids vs the CUDA
    graph of the persistent step, FP32 and FP64.  One step = location and cell
    table of the raw points, residual, Jacobian apply, interpolation and
    spreading of every instance."""
    import torch
    import paper_2601_08266_gb300 as fsi
    from paper_2601_08266_gb300 import inputs
    rng = np.random.default_rng(SEED + 50)
    count = args.batch_count
    Ns = rng.integers(16, 49, size=count)
    mus = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), size=count))
    ms = rng.integers(10_000, 150_001, size=count)
    out = {"instances": count, "dofs_total": int(sum(4 * (N + 1) ** 3 for N in Ns)),
           "points_total": int(ms.sum()),
           "step": "locate + cell table, residual, Jacobian apply, interp, spread"}
    for prec_name, dt_t, P in (("f32", torch.float32, fsi.FSI_F32), ("f64", torch.float64, fsi.FSI_F64)):
        meshes, items = [], []
        for i in range(count):
            N, m = int(Ns[i]), int(ms[i])
            mesh = fsi.Mesh(N, rho=1.0, mu=float(mus[i]), dt=1e-3, rho_inf=0.5, device=dev.index,
                            stream=stream.cuda_stream)
            n = mesh.n_nodes
            with torch.cuda.stream(stream):
                g = torch.Generator(device=dev).manual_seed(SEED + i)
                it = {k: (torch.rand((n, 4), device=dev, generator=g) * 2 - 1).to(dt_t)
                      for k in ("U", "A", "x")}
                it.update(R=torch.empty((n, 4), dtype=dt_t, device=dev),
                          Jx=torch.empty((n, 4), dtype=dt_t, device=dev),
                          F=torch.empty((n, 4), dtype=dt_t, device=dev),
                          cell_start=torch.empty(N ** 3 + 1, dtype=torch.int32, device=dev),
                          elem=torch.empty(m, dtype=torch.int32, device=dev),
                          perm=torch.empty(m, dtype=torch.int32, device=dev),
                          lam=torch.randn((m, 3), device=dev, generator=g).to(dt_t),
                          u=torch.empty((m, 3), dtype=dt_t, device=dev))
                # raw points: every batched step locates them and builds the
                # instance's cell table itself (elem, xi, cell_start, perm are
                # outputs of the step)
                it["X"] = torch.as_tensor(inputs.leaflet_points(m, seed=SEED + 100 + i),
                                          device=dev)
                it["xi"] = torch.empty((m, 3), dtype=dt_t, device=dev)
            meshes.append(mesh)
            items.append(it)
        stream.synchronize()
        b = fsi.Batch(meshes, items, P, stream.cuda_stream)
        res = {}
        if prec_name == "f32" or args.batch_tune_f64:
            tune = b.autotune(reps=1)
            res["autotuned"] = {"brick": tune["brick"], "threads": tune["threads"],
                                "ctas_per_sm": tune["ctas_per_sm"]}
        for name, mode in (("per_instance", fsi.FSI_BATCH_PER_INSTANCE),
                           ("persistent", fsi.FSI_BATCH_PERSISTENT), ("graph", fsi.FSI_BATCH_GRAPH)):
            t = b.time(mode, reps=args.batch_reps)
            res[name] = {"ms": t * 1e3, "gdof_s": out["dofs_total"] / t / 1e9}
        res["speedup_graph_vs_per_instance"] = res["per_instance"]["ms"] / res["graph"]["ms"]
        out[prec_name] = res
        b.close()
        for mm in meshes:
            mm.close()
    return out


# ------------------------------------------------------------------ hyperelastic solid
def solid_section(args, dev, stream):
    """The three leaflets as neo-Hookean hexahedral solids (Sec. 2.2): the
    element residual and tangent kernels alone, and one implicit step of the
    64^3 channel with the body coupled through C (plain FP64 vs mixed)."""
    import torch
    import paper_2601_08266_gb300 as fsi
    from paper_2601_08266_gb300 import inputs
    X, conn = inputs.leaflet_hex_mesh(2, 96, 128, seed=SEED + 70)
    ns, es = X.shape[0], conn.shape[0]
    out = {"elements": int(es), "nodes": int(ns), "material": "neo-Hookean mu_s 50, lambda_s 500, "
           "rho_s 1.2 (fluid rho 1, mu 1e-3)"}
    ch = Channel(fsi, dev, stream, 64, 1, SEED + 71)
    with torch.cuda.stream(stream):
        Xd = torch.as_tensor(X, device=dev)
        body = fsi.Solid(ch.mesh, Xd, torch.as_tensor(conn, device=dev), 1.2, 50.0, 500.0)
        g = torch.Generator(device=dev).manual_seed(SEED + 72)
        st3 = [0.001 * torch.randn((ns, 3), dtype=torch.float64, device=dev, generator=g)
               for _ in range(4)]
        R = torch.empty((ns, 3), dtype=torch.float64, device=dev)
        x = torch.randn((ns, 3), dtype=torch.float64, device=dev, generator=g)
        Jx = torch.empty_like(R)
        x32, u32, J32 = x.float(), st3[0].float(), torch.empty((ns, 3), dtype=torch.float32,
                                                                device=dev)

    def timeit(fn, reps=10):
        for _ in range(2):
            fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = {
        "residual_f64": timeit(lambda: fsi.fsi_solid_residual(body, st3[0], st3[1], st3[2], st3[3],
                                                              (0.0, 0.0, -1.0), R)),
        "tangent_f64": timeit(lambda: fsi.fsi_solid_tangent_apply(body, fsi.FSI_F64, st3[0],
                                                                  st3[3], x, Jx)),
        "tangent_f32": timeit(lambda: fsi.fsi_solid_tangent_apply(body, fsi.FSI_F32, u32, st3[3],
                                                                  x32, J32)),
    }
    out["kernels"] = {k: {"ms": v, "elements_per_s": es / (v * 1e-3)} for k, v in ms.items()}
    # one implicit step of the channel with the body as the immersed solid
    with torch.cuda.stream(stream):
        us, vs, as_ = (torch.zeros((ns, 3), dtype=torch.float64, device=dev) for _ in range(3))
        xs = torch.empty((ns, 3), dtype=torch.float64, device=dev)
        e = torch.empty(ns, dtype=torch.int32, device=dev)
        xi = torch.empty((ns, 3), dtype=torch.float64, device=dev)
        cs = torch.empty(ch.mesh.n_elems + 1, dtype=torch.int32, device=dev)
        pm = torch.empty(ns, dtype=torch.int32, device=dev)
    fsi.fsi_solid_positions(body, us, xs)
    fsi.fsi_locate(ch.mesh, xs, e, xi, cs, pm)
    solve = dict(restart=50, max_newton=10, max_krylov=4000, newton_rtol=1e-8, krylov_rtol=1e-3)
    r_ref = None
    for name, mixed in (("fp64", False), ("mixed", True)):
        yD = ch.dirichlet()
        with torch.cuda.stream(stream):
            y = ch.yn.clone()
            y[ch.maskb] = yD[ch.maskb]
        st = fsi.StepState(y, ch.Vn, ch.An, mask=ch.mask, yD=yD, elem=e, xi=xi, cell_start=cs,
                           perm=pm, g_s=(0.0, 0.0, -1.0), body=body, us=us, vs=vs, as_=as_)
        stream.synchronize()
        t0 = time.perf_counter()
        code, rep = fsi.fsi_newton_step(ch.mesh, st, mixed=mixed, r_ref=r_ref or 0.0, check=False,
                                        residual_prec=fsi.FSI_DF64 if mixed else fsi.FSI_F64,
                                        **solve)
        stream.synchronize()
        el = time.perf_counter() - t0
        r_ref = r_ref or rep["r_ref"]
        out["newton_" + name] = {"seconds": el, "newton_iters": rep["newton_iters"],
                                 "krylov_iters": rep["krylov_iters"],
                                 "r_final_over_ref": rep["r_final"] / r_ref,
                                 "converged": bool(rep["converged"]), "status": code}
    out["newton_speedup_mixed_vs_fp64"] = out["newton_fp64"]["seconds"] / out["newton_mixed"]["seconds"]
    body.close()
    ch.close()
    return out


# ------------------------------------------------------------------ mapped grids
def bubble_map(X, delta):
    """Smooth map of the unit cube onto itself, identity on its faces."""
    b = np.sin(2 * np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1]) * np.sin(2 * np.pi * X[:, 2])
    return X + delta * b[:, None] * np.array([1.0, -0.7, 0.4])[None, :]


def dlm_section(args, dev, stream):
    """The coupling operators on the 128^3 grid with 1M leaflet points (the
    mixed Newton step's workload): location with the cell table (FP64),
    interpolation and spreading in FP32, double-float and FP64.  Each call is
    timed alone with CUDA events on the library's stream, L2 flushed (write of
    a buffer > L2) before it, median of the repetitions; achieved = the
    operator's algorithmic bytes (every input and output array touched once;
    the velocity rows of the nodes of occupied cells for interpolation) / time,
    against the measured HBM copy bandwidth."""
    import torch
    import paper_2601_08266_gb300 as fsi
    from paper_2601_08266_gb300 import inputs
    N, m = args.newton_grid, args.newton_points
    mesh = fsi.Mesh(N, device=dev.index, stream=stream.cuda_stream)
    n, E = mesh.n_nodes, mesh.n_elems
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    g = torch.Generator(device=dev).manual_seed(SEED + 90)
    with torch.cuda.stream(stream):
        flush = torch.empty(max(2 * l2, 256 << 20) // 4, dtype=torch.float32, device=dev)
        X = torch.as_tensor(inputs.leaflet_points(m, seed=SEED + 91), device=dev)
        elem = torch.empty(m, dtype=torch.int32, device=dev)
        xi = torch.empty((m, 3), dtype=torch.float64, device=dev)
        cs = torch.empty(E + 1, dtype=torch.int32, device=dev)
        perm = torch.empty(m, dtype=torch.int32, device=dev)
    fsi.fsi_locate(mesh, X, elem, xi, cs, perm)
    stream.synchronize()
    # nodes of occupied cells (the rows interpolation reads)
    occ = torch.nonzero(cs[1:] > cs[:-1]).flatten().long()
    ex, ey, ez = occ % N, (occ // N) % N, occ // (N * N)
    nodes = torch.cat([(ex + dx) + (N + 1) * ((ey + dy) + (N + 1) * (ez + dz))
                       for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]).unique().numel()

    def timed(fn, reps=10):
        ts = []
        for r in range(reps + 2):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            stream.synchronize()
            if r >= 2:
                ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    def entry(ms, nbytes):
        return {"ms": round(ms, 5), "gb_s": round(nbytes / (ms * 1e-3) / 1e9, 1),
                "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / hbm, 4),
                "points_per_s": round(m / (ms * 1e-3), 1), "bytes": int(nbytes)}

    out = {"grid": [N, N, N], "points": m, "occupied_cells": int(occ.numel()),
           "nodes_of_occupied_cells": int(nodes)}
    t = timed(lambda: fsi.fsi_locate(mesh, X, elem, xi, cs, perm, want_outside=False))
    out["locate_f64"] = entry(t, m * (24 + 4 + 24 + 4) + (E + 1) * 4)
    for name, P, dt, sz in (("f32", fsi.FSI_F32, torch.float32, 4),
                            ("df64", fsi.FSI_DF64, torch.float64, 8),
                            ("f64", fsi.FSI_F64, torch.float64, 8)):
        with torch.cuda.stream(stream):
            U = torch.randn((n, 4), dtype=dt, device=dev, generator=g)
            F = torch.zeros((n, 4), dtype=dt, device=dev)
            lam = torch.randn((m, 3), dtype=dt, device=dev, generator=g)
            u = torch.empty((m, 3), dtype=dt, device=dev)
            xw = xi.to(dt).contiguous()
        t = timed(lambda: fsi.fsi_dlm_interp(mesh, P, elem, xw, U, u))
        out[f"interp_{name}"] = entry(t, m * (4 + 3 * sz + 3 * sz) + nodes * 4 * sz)
        t = timed(lambda: fsi.fsi_dlm_spread(mesh, P, elem, xw, cs, perm, lam, None, F, False))
        out[f"spread_{name}"] = entry(t, m * (4 + 3 * sz + 3 * sz) + (E + 1) * 4 + n * 3 * sz)
        del U, F, lam, u, xw
    mesh.close()
    return out


def mapped_section(args, dev, stream):
    """Mapped (curvilinear) structured grids: the VMS kernels with per-Gauss-point
    geometry against the uniform kernels on the same 128^3 grid, point location
    by the element walk, and the mixed Newton step of the 64^3 channel on a
    bubble-mapped grid, with the Schur preconditioner's pressure block either
    the geometric multigrid of the nominal uniform operator or the algebraic
    multigrid of the operator assembled on the mapped grid (its host
    set-up timed apart)."""
    import torch
    import paper_2601_08266_gb300 as fsi
    N = 128
    out = {"grid": [N, N, N], "map": "x + 0.02 sin(2 pi x) sin(2 pi y) sin(2 pi z) (1, -0.7, 0.4)"}
    mesh = fsi.Mesh(N, rho=1.0, mu=1e-3, dt=1e-3, rho_inf=0.5, device=dev.index,
                    stream=stream.cuda_stream)
    n = mesh.n_nodes
    ax = np.arange(N + 1) / N
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    Xm = bubble_map(np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1), 0.02)
    g = torch.Generator(device=dev).manual_seed(SEED + 80)
    with torch.cuda.stream(stream):
        Xd = torch.as_tensor(Xm, device=dev)
        U = 0.5 * torch.randn((n, 4), dtype=torch.float64, device=dev, generator=g)
        A = 0.5 * torch.randn((n, 4), dtype=torch.float64, device=dev, generator=g)
        x = torch.randn((n, 4), dtype=torch.float64, device=dev, generator=g)
        R = torch.empty_like(U)
        U32, A32, x32, R32 = U.float(), A.float(), x.float(), torch.empty((n, 4),
                                                                           dtype=torch.float32,
                                                                           device=dev)

    def timeit(fn, reps=10):
        for _ in range(3):
            fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    cases = {
        "residual_f32": lambda: fsi.fsi_residual(mesh, fsi.FSI_F32, U32, A32, None, R32),
        "jacobian_f32": lambda: fsi.fsi_jacobian_apply(mesh, fsi.FSI_F32, U32, A32, None, x32, R32),
        "residual_df64": lambda: fsi.fsi_residual(mesh, fsi.FSI_DF64, U, A, None, R),
        "jacobian_df64": lambda: fsi.fsi_jacobian_apply(mesh, fsi.FSI_DF64, U, A, None, x, R),
        "residual_f64": lambda: fsi.fsi_residual(mesh, fsi.FSI_F64, U, A, None, R),
        "jacobian_f64": lambda: fsi.fsi_jacobian_apply(mesh, fsi.FSI_F64, U, A, None, x, R),
    }
    uni = {k: timeit(f) for k, f in cases.items()}
    with torch.cuda.stream(stream):
        mesh.set_coordinates(Xd)
    mapped = {k: timeit(f) for k, f in cases.items()}
    out["vms_kernels"] = {k: {"uniform_ms": uni[k], "mapped_ms": mapped[k],
                              "mapped_gdof_per_s": 4 * n / (mapped[k] * 1e-3) / 1e9,
                              "mapped_over_uniform": mapped[k] / uni[k]} for k in cases}
    # location of 2^20 points spread over the interior
    m = 1 << 20
    with torch.cuda.stream(stream):
        P = 0.02 + 0.96 * torch.rand((m, 3), dtype=torch.float64, device=dev, generator=g)
        e = torch.empty(m, dtype=torch.int32, device=dev)
        xi = torch.empty((m, 3), dtype=torch.float64, device=dev)
        cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device=dev)
        pm = torch.empty(m, dtype=torch.int32, device=dev)
    loc = lambda: fsi.fsi_locate(mesh, P, e, xi, cs, pm, want_outside=False)
    t_m = timeit(loc)
    with torch.cuda.stream(stream):
        mesh.set_coordinates(None)
    t_u = timeit(loc)
    out["locate"] = {"points": m, "uniform_ms": t_u, "mapped_ms": t_m,
                     "mapped_points_per_s": m / (t_m * 1e-3)}
    mesh.close()
    # the mixed Newton step of the 64^3 channel, uniform against mapped
    solve = dict(restart=50, max_newton=10, max_krylov=4000, newton_rtol=1e-8, krylov_rtol=1e-3)
    for name, bub, amg in (("uniform", 0.0, False), ("mapped", 0.02, False),
                           ("mapped_amg", 0.02, True)):
        ch = Channel(fsi, dev, stream, 64, M_POINTS, SEED + 81, bubble=bub)
        y, st = ch.state(guess="zero")
        setup = None
        if amg:
            # one untimed step builds the hierarchy for the step's elimination
            # set (the host set-up, timed apart); the timed step reuses it
            fsi.fsi_pressure_use_amg(ch.mesh, True)
            stream.synchronize()
            t0 = time.perf_counter()
            fsi.fsi_newton_step(ch.mesh, st, mixed=True, check=False,
                                residual_prec=fsi.FSI_DF64, **solve)
            stream.synchronize()
            setup = time.perf_counter() - t0
            y, st = ch.state(guess="zero")
        stream.synchronize()
        t0 = time.perf_counter()
        code, rep = fsi.fsi_newton_step(ch.mesh, st, mixed=True, check=False,
                                        residual_prec=fsi.FSI_DF64, **solve)
        stream.synchronize()
        out["newton_mixed_64cubed_" + name] = {
            "seconds": time.perf_counter() - t0, "newton_iters": rep["newton_iters"],
            "krylov_iters": rep["krylov_iters"], "r_final_over_r0": rep["r_final"] / rep["r0"],
            "converged": bool(rep["converged"]), "status": code}
        if amg:
            out["newton_mixed_64cubed_" + name]["first_step_with_amg_setup_seconds"] = setup
            out["newton_mixed_64cubed_" + name]["amg_levels"] = fsi.fsi_pressure_level_sizes(ch.mesh)
        ch.close()
    return out


# ------------------------------------------------------------------ tetrahedral meshes
def tet_section(args, dev, stream):
    """Unstructured tetrahedral meshes: the 64^3 grid split into 1,572,864
    linear tetrahedra (nodes moved by up to 0.2 h, node and element numbers
    shuffled), the same 274,625 nodes as the 64^3 step.  VMS residual and
    Jacobian apply in the three precisions, location of the 200k leaflet
    points, interpolation and spreading."""
    import torch
    import paper_2601_08266_gb300 as fsi
    from paper_2601_08266_gb300 import inputs
    N = 64
    X, Tt = inputs.tet_box_mesh(N, seed=SEED + 90, perturb=0.2)
    with torch.cuda.stream(stream):
        Xd, Td = torch.as_tensor(X, device=dev), torch.as_tensor(Tt, device=dev)
    stream.synchronize()
    t0 = time.perf_counter()
    mesh = fsi.TetMesh(Xd, Td, rho=1.0, mu=1e-3, dt=1e-3, rho_inf=0.5, device=dev.index,
                       stream=stream.cuda_stream)
    create_s = time.perf_counter() - t0
    n, E = mesh.n_nodes, mesh.n_elems
    out = {"elements": E, "nodes": n, "dofs": 4 * n, "mesh": "64^3 cubes x 6 tetrahedra, "
           "interior nodes moved by up to 0.2 h, numbering shuffled", "create_seconds": create_s}
    g = torch.Generator(device=dev).manual_seed(SEED + 91)
    with torch.cuda.stream(stream):
        U = 0.5 * torch.randn((n, 4), dtype=torch.float64, device=dev, generator=g)
        A = 0.5 * torch.randn((n, 4), dtype=torch.float64, device=dev, generator=g)
        x = torch.randn((n, 4), dtype=torch.float64, device=dev, generator=g)
        R = torch.empty_like(U)
        U32, A32, x32, R32 = U.float(), A.float(), x.float(), R.float()

    def timeit(fn, reps=10):
        for _ in range(3):
            fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    cases = {
        "residual_f32": lambda: fsi.fsi_tet_residual(mesh, fsi.FSI_F32, U32, A32, None, R32),
        "jacobian_f32": lambda: fsi.fsi_tet_jacobian_apply(mesh, fsi.FSI_F32, U32, A32, None, x32,
                                                           R32),
        "residual_df64": lambda: fsi.fsi_tet_residual(mesh, fsi.FSI_DF64, U, A, None, R),
        "jacobian_df64": lambda: fsi.fsi_tet_jacobian_apply(mesh, fsi.FSI_DF64, U, A, None, x, R),
        "residual_f64": lambda: fsi.fsi_tet_residual(mesh, fsi.FSI_F64, U, A, None, R),
        "jacobian_f64": lambda: fsi.fsi_tet_jacobian_apply(mesh, fsi.FSI_F64, U, A, None, x, R),
    }
    out["vms_kernels"] = {}
    for k, f in cases.items():
        ms = timeit(f)
        out["vms_kernels"][k] = {"ms": ms, "gdof_s": 4 * n / (ms * 1e-3) / 1e9,
                                 "elements_per_s": E / (ms * 1e-3)}
    m = M_POINTS
    with torch.cuda.stream(stream):
        P = torch.as_tensor(inputs.leaflet_points(m, seed=SEED + 92), device=dev)
        e = torch.empty(m, dtype=torch.int32, device=dev)
        lam = torch.empty((m, 3), dtype=torch.float64, device=dev)
        cs = torch.empty(E + 1, dtype=torch.int32, device=dev)
        pm = torch.empty(m, dtype=torch.int32, device=dev)
        lv = torch.randn((m, 3), dtype=torch.float64, device=dev, generator=g)
        u = torch.empty((m, 3), dtype=torch.float64, device=dev)
        F = torch.zeros((n, 4), dtype=torch.float64, device=dev)
    nout = fsi.fsi_tet_locate(mesh, P, e, lam, cs, pm)
    out["points"] = {"m": m, "outside": nout}
    out["locate_ms"] = timeit(lambda: fsi.fsi_tet_locate(mesh, P, e, lam, cs, pm,
                                                         want_outside=False))
    out["interp_df64_ms"] = timeit(lambda: fsi.fsi_tet_interp(mesh, fsi.FSI_DF64, e, lam, U, u))
    out["spread_df64_ms"] = timeit(lambda: fsi.fsi_tet_spread(mesh, fsi.FSI_DF64, e, lam, cs, pm,
                                                              lv, None, F, False))
    mesh.close()
    out["newton_channel"] = tet_newton(fsi, dev, stream,
                                       variants=args.tet_newton_variants.split(","))
    return out


def tet_newton(fsi, dev, stream, N=32, m=50_000, variants=("fp64", "mixed", "schur_fp64",
                                                          "schur_mixed")):
    """One implicit step of the channel flow (inflow 16 y(1-y) z(1-z) at x = 0,
    no-slip walls, traction-free outflow, mu = 1e-3, dt = 1e-3) on a
    tetrahedral mesh (32^3 cubes x 6, shuffled numbering) with leaflet points:
    plain FP64 against mixed FP32/FP64 Newton-GMRES, with block-Jacobi and
    with the Schur-complement preconditioner (algebraic multigrid for the
    pressure; its host set-up for the step's elimination set is timed apart)."""
    import torch
    from paper_2601_08266_gb300 import inputs
    X, Tt = inputs.tet_box_mesh(N, seed=SEED + 95, perturb=0.1)
    n = X.shape[0]
    dt, mu, gamma = 1e-3, 1e-3, 2.0 / 3.0
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    prof = 16.0 * y * (1 - y) * z * (1 - z)
    wall = (y < 1e-12) | (y > 1 - 1e-12) | (z < 1e-12) | (z > 1 - 1e-12)
    inflow = (x < 1e-12) & ~wall
    mask = np.zeros((n, 4), dtype=np.uint8)
    mask[wall | inflow, :3] = 1
    Vn = np.zeros((n, 4))
    Vn[:, 0] = prof * (1.0 + 0.05 * np.sin(2 * np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z))
    Vn[mask[:, 0].astype(bool), :3] = 0.0
    Vn[inflow, 0] = prof[inflow]
    g = np.zeros((n, 3))
    g[inflow, 0] = prof[inflow]
    yD = np.zeros((n, 4))
    yD[:, :3] = (g - Vn[:, :3]) / (gamma * dt)
    out = {"elements": int(Tt.shape[0]), "nodes": int(n), "dofs": 4 * int(n), "points": m,
           "preconditioner": "fp64/mixed: nodal 4x4 block-Jacobi (probed with a distance-2 "
                             "colouring); schur_*: 3x3 velocity blocks + sigma (K + kappa M) "
                             "by one smoothed-aggregation AMG V-cycle"}
    with torch.cuda.stream(stream):
        mesh = fsi.MeshTet(torch.as_tensor(X, device=dev), torch.as_tensor(Tt, device=dev),
                           rho=1.0, mu=mu, dt=dt, rho_inf=0.5, device=dev.index,
                           stream=stream.cuda_stream)
        P = torch.as_tensor(inputs.leaflet_points(m, seed=SEED + 96), device=dev)
        e = torch.empty(m, dtype=torch.int32, device=dev)
        xi = torch.empty((m, 3), dtype=torch.float64, device=dev)
        cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device=dev)
        pm = torch.empty(m, dtype=torch.int32, device=dev)
        w = torch.full((m,), 0.024 / m, dtype=torch.float64, device=dev)
        Vd, Ad = torch.as_tensor(Vn, device=dev), torch.zeros((n, 4), dtype=torch.float64,
                                                              device=dev)
        md, yDd = torch.as_tensor(mask, device=dev), torch.as_tensor(yD, device=dev)
    fsi.fsi_locate(mesh, P, e, xi, cs, pm)
    r_ref = None
    # the Schur runs eliminate the outflow nodes (boundary, velocity free); the
    # hierarchy for that set is built here, timed apart, and reused by both
    outflow = (x > 1 - 1e-12) & ~wall
    with torch.cuda.stream(stream):
        elim = torch.as_tensor(outflow.astype(np.uint8), device=dev)
    stream.synchronize()
    t0 = time.perf_counter()
    fsi.fsi_pressure_set_eliminated(mesh, elim)
    stream.synchronize()
    out["schur_amg_setup_seconds"] = time.perf_counter() - t0
    runs = (("fp64", False, fsi.PRECOND_BLOCK_JACOBI), ("mixed", True, fsi.PRECOND_BLOCK_JACOBI),
            ("schur_fp64", False, fsi.PRECOND_SCHUR), ("schur_mixed", True, fsi.PRECOND_SCHUR))
    for name, mixed, precond in runs:
        if name not in variants:
            continue
        with torch.cuda.stream(stream):
            yv = torch.zeros((n, 4), dtype=torch.float64, device=dev)
            yv[md.bool()] = yDd[md.bool()]
        st = fsi.StepState(yv, Vd, Ad, mask=md, yD=yDd, elem=e, xi=xi, cell_start=cs, perm=pm,
                           w=w, drho_s=0.5)
        stream.synchronize()
        t0 = time.perf_counter()
        code, rep = fsi.fsi_newton_step(mesh, st, mixed=mixed, restart=50, max_newton=10,
                                        max_krylov=20000, newton_rtol=1e-8, krylov_rtol=1e-3,
                                        r_ref=r_ref or 0.0, check=False, precond=precond,
                                        residual_prec=fsi.FSI_DF64 if mixed else fsi.FSI_F64)
        stream.synchronize()
        r_ref = r_ref or rep["r_ref"]
        out[name] = {"seconds": time.perf_counter() - t0, "newton_iters": rep["newton_iters"],
                     "krylov_iters": rep["krylov_iters"],
                     "r_final_over_ref": rep["r_final"] / r_ref,
                     "converged": bool(rep["converged"]), "status": code}
    if "fp64" in out and "mixed" in out:
        out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    if "fp64" in out and "schur_mixed" in out:
        out["speedup_schur_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["schur_mixed"]["seconds"]
    out["pressure_levels"] = fsi.fsi_pressure_level_sizes(mesh)
    mesh.close()
    return out


# ------------------------------------------------------------------ MLP inference
def mlp_section(args, dev, stream, W):
    """Per-node inference of the initial-guess network over whole grids: the
    fused tcgen05 predictor (features, three layers, predictor in one
    persistent kernel) against the unfused path of the training kernels
    (features to HBM, then the training GEMMs per chunk); and one training
    step (forward, loss, backward) on a batch of 4096 samples."""
    import torch
    import paper_2601_08266_gb300 as fsi
    out = {"kernel": "fused: tcgen05.mma kind::f16 (BF16 in, FP32 accumulate in TMEM), weights "
                     "resident in shared memory via cp.async.bulk; unfused and training: the "
                     "tcgen05 GEMM kernel (BF16 operands staged from FP32, TMEM accumulators, "
                     "split-K weight gradients)"}
    peaks = measured_peaks()
    bf16_peak = peaks.get("bf16_tflops", 1865.6)
    # one training step: 3 forward GEMMs, 5 backward GEMMs (2 x the forward
    # flops), bias sums and the loss; CUDA events over 20 steps
    B = 4096
    g = torch.Generator(device=dev).manual_seed(SEED + 7)
    with torch.cuda.stream(stream):
        P = torch.randn(fsi.fsi_mlp_num_params(), device=dev, generator=g) * 0.05
        Xb = torch.randn((B, 112), device=dev, generator=g)
        Tb = torch.randn((B, 4), device=dev, generator=g)
        G = torch.empty_like(P)
        loss = torch.empty(1, device=dev)
    h = fsi.Mlp(B, device=dev.index, stream=stream.cuda_stream)
    for _ in range(3):
        fsi.fsi_mlp_loss_grad(h, P, Xb, Tb, loss, G)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(20):
        fsi.fsi_mlp_loss_grad(h, P, Xb, Tb, loss, G)
    e1.record(stream)
    stream.synchronize()
    h.check()
    ms = e0.elapsed_time(e1) / 20
    tflop = 3 * 2.0 * B * (112 * 256 + 256 * 256 + 256 * 4) / 1e12
    out["training_step"] = {"batch": B, "ms": ms, "tflop_s": tflop / (ms * 1e-3),
                            "frac_of_bf16_peak": tflop / (ms * 1e-3) / bf16_peak,
                            "flops": "3 x 2 B (112 x 256 + 256 x 256 + 256 x 4)"}
    h.close()
    for N in (64, 128):
        mesh = fsi.Mesh(N, device=dev.index, stream=stream.cuda_stream)
        n = mesh.n_nodes
        g = torch.Generator(device=dev).manual_seed(SEED + N)
        with torch.cuda.stream(stream):
            P = torch.randn(fsi.fsi_mlp_num_params(), device=dev, generator=g) * 0.05
            st = [torch.randn((n, 4), dtype=torch.float64, device=dev, generator=g)
                  for _ in range(4)]
            stats = [torch.zeros(112, device=dev), torch.ones(112, device=dev),
                     torch.zeros(4, device=dev), torch.ones(4, device=dev)]
            y0 = torch.empty((n, 4), dtype=torch.float64, device=dev)
        chunk = 131072
        h = fsi.Mlp(chunk, device=dev.index, stream=stream.cuda_stream)
        flops = 2.0 * n * (112 * 256 + 256 * 256 + 256 * 4)

        def fused():
            fsi.fsi_mlp_predict(h, mesh, P, *stats, st[0], st[1], st[2], st[3], y0)

        with torch.cuda.stream(stream):
            Xc = torch.empty((chunk, 112), dtype=torch.float32, device=dev)
            Oc = torch.empty((chunk, 4), dtype=torch.float32, device=dev)
            idxs = [torch.arange(b0, min(n, b0 + chunk), dtype=torch.int32, device=dev)
                    for b0 in range(0, n, chunk)]

        def unfused():
            for idx in idxs:
                k = idx.shape[0]
                fsi.fsi_mlp_features(mesh, st[0], st[1], st[2], st[3], idx, stats[0], stats[1],
                                     Xc[:k])
                fsi.fsi_mlp_forward(h, P, Xc[:k], Oc[:k])
        res = {"nodes": n}
        for name, fn in (("fused_tcgen05", fused), ("unfused", unfused)):
            for _ in range(2):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[name] = {"ms": ms, "tflop_s": flops / (ms * 1e-3) / 1e12,
                         "frac_of_bf16_peak": flops / (ms * 1e-3) / 1e12 / bf16_peak}
        out[f"{N}^3"] = res
        h.close()
        mesh.close()
    out["bf16_peak_tflop_s"] = bf16_peak
    return out


def profile_case(args):
    """Small fixed cases for ncu captures (nothing is timed): 'vms_f64' runs the
    fused FP64 residual + Jacobian pass twice on the --grid grid with the
    --profile-brick schedule (default 4x4x4 bricks of 128 threads); 'vms_f32' runs the FP32 Jacobian apply twice on
    the --grid grid with the default schedule; 'dlm' runs location with the cell table, and FP32
    and double-float interpolation and spreading, twice, on the --grid grid
    with --points leaflet points; 'blas1' runs the Krylov multi-dot and
    multi-update kernels twice each on 8 FP32 vectors of the --grid grid's
    4 (N+1)^3 entries; 'pmg' runs two FP32 pressure V-cycles on the --grid
    grid (no eliminated faces)."""
    import torch
    import paper_2601_08266_gb300 as fsi
    from paper_2601_08266_gb300 import inputs
    dev = torch.device("cuda:0")
    N = args.grid
    if args.profile_case == "pmg":
        mesh = fsi.Mesh(N, device=0)
        bp = torch.randn(mesh.n_nodes, dtype=torch.float32, device=dev)
        xp = torch.empty_like(bp)
        for _ in range(2):
            fsi.fsi_pressure_vcycle(mesh, bp, xp)
        torch.cuda.synchronize()
        mesh.close()
        print(json.dumps({"profile_case": "pmg", "grid": N, "ok": True}))
        return 0
    if args.profile_case == "blas1":
        from paper_2601_08266_gb300 import _binding as B
        B.fsi_measure_blas1(0, fsi.FSI_F32, 4 * (N + 1) ** 3, 8, reps=1)
        print(json.dumps({"profile_case": "blas1", "grid": N, "ok": True}))
        return 0
    mesh = fsi.Mesh(N, device=0)
    n = mesh.n_nodes
    if args.profile_case == "vms_f32":
        # the FP32 Jacobian apply of the mixed Newton step, default schedule
        U = torch.as_tensor(inputs.fourier_field(N, seed=1), device=dev).float()
        A = torch.as_tensor(inputs.fourier_field(N, seed=2), device=dev).float()
        A[:, 3] = 1.0
        x = torch.as_tensor(inputs.uniform_nodal(N, seed=3), device=dev).float()
        J = torch.empty_like(U)
        for _ in range(2):
            fsi.fsi_jacobian_apply(mesh, fsi.FSI_F32, U, A, None, x, J)
    elif args.profile_case == "vms_f64":
        bx, by, bz, th = (int(v) for v in args.profile_brick.split(","))
        fsi.fsi_mesh_set_brick(mesh, 2, fsi.FSI_F64, bx, by, bz, th)
        U = torch.as_tensor(inputs.fourier_field(N, seed=1), device=dev)
        A = torch.as_tensor(inputs.fourier_field(N, seed=2), device=dev)
        A[:, 3] = 1.0
        x = torch.as_tensor(inputs.uniform_nodal(N, seed=3), device=dev)
        R, J = torch.empty_like(U), torch.empty_like(U)
        for _ in range(2):
            fsi.fsi_residual_jacobian_apply(mesh, fsi.FSI_F64, U, A, None, x, R, J)
    else:
        m = args.points
        X = torch.as_tensor(inputs.leaflet_points(m, seed=7), device=dev)
        elem = torch.empty(m, dtype=torch.int32, device=dev)
        xi = torch.empty((m, 3), dtype=torch.float64, device=dev)
        cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device=dev)
        perm = torch.empty(m, dtype=torch.int32, device=dev)
        bufs = {}
        for name, P, dt in (("f32", fsi.FSI_F32, torch.float32),
                            ("df64", fsi.FSI_DF64, torch.float64)):
            bufs[name] = (P, torch.randn((n, 4), dtype=dt, device=dev),
                          torch.zeros((n, 4), dtype=dt, device=dev),
                          torch.randn((m, 3), dtype=dt, device=dev),
                          torch.empty((m, 3), dtype=dt, device=dev))
        for _ in range(2):
            fsi.fsi_locate(mesh, X, elem, xi, cs, perm, want_outside=False)
            for name in ("f32", "df64"):
                P, U, F, lam, u = bufs[name]
                xw = xi.to(U.dtype).contiguous()
                fsi.fsi_dlm_interp(mesh, P, elem, xw, U, u)
                fsi.fsi_dlm_spread(mesh, P, elem, xw, cs, perm, lam, None, F, False)
    torch.cuda.synchronize()
    mesh.close()
    print(json.dumps({"profile_case": args.profile_case, "grid": N, "ok": True}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--grid", type=int, default=N_GRID, help="elements per axis (profiling)")
    ap.add_argument("--points", type=int, default=M_POINTS, help="solid points (profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default brick schedules of the VMS operators (8x8x4; 8x4x4 "
                         "for the fused pass)")
    ap.add_argument("--no-extras", action="store_true", help="skip Newton, batch and MLP sections")
    ap.add_argument("--sections", default="newton,dlm,batch,mlp,solid,mapped,tet",
                    help="comma-separated extra sections to run")
    ap.add_argument("--newton-grid", type=int, default=128)
    ap.add_argument("--newton-points", type=int, default=1_000_000)
    ap.add_argument("--newton-reps", type=int, default=3,
                    help="repetitions of each mixed Newton variant (median time)")
    ap.add_argument("--newton-warm", type=int, default=3)
    ap.add_argument("--krylov-floor", type=float, default=1e-4,
                    help="floor of the Newton solver's target-aware inner tolerance")
    ap.add_argument("--train-grid", type=int, default=64)
    ap.add_argument("--train-points", type=int, default=200_000)
    ap.add_argument("--train-runs", type=int, default=2)
    ap.add_argument("--train-steps", type=int, default=6)
    ap.add_argument("--train-samples", type=int, default=50_000)
    ap.add_argument("--mlp-iters", type=int, default=600)
    ap.add_argument("--newton-variants",
                    default="fp64,mixed_zero_guess,mixed,mixed_learned,mixed_block_jacobi",
                    help="comma-separated Newton variants to time")
    ap.add_argument("--tet-newton-variants", default="fp64,mixed,schur_fp64,schur_mixed",
                    help="comma-separated Newton runs of the tetrahedral channel step")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--batch-tune-f64", action="store_true")
    ap.add_argument("--profile-brick", default="4,4,4,128",
                    help="brick schedule bx,by,bz,threads of the vms_f64 profile case")
    ap.add_argument("--profile-case", choices=["vms_f64", "vms_f32", "dlm", "blas1", "pmg"],
                    default=None,
                    help="run one small fixed case for an ncu capture and exit")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
