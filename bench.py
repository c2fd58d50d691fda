#!/usr/bin/env python
"""Benchmark of the per-step solves at the 1024 x 1024 two-protrusion
workload (domain [0,4]x[0,1], r = 0.08 at x = 1.3 and 2.7, dt = 1e-4,
GMRES(30), synthetic seeded input): time steps per second on the GPU, plus
the end-to-end rate through the C ABI with host buffers, the roofline of
the dominant kernel and the FP64 CPU oracle as a reported baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   (the CPU oracle, rank 0 only)

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time steps/sec and solver HBM GB/s at 1024^2, mixed vs FP64 at 1e-6 rel err"
UNIT = "steps/s"

# FP64 FMA rate: 152 SMs x 2 FP64 FMA / clock / SM x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Algorithmic FP64 flops per node of one operator apply (FMA = 2)
FLOPS_PER_NODE = {"phi": 26.0, "p": 7.0, "u": 7.0}
# Algorithmic HBM bytes per node of one apply: read x (+ a), write y
BYTES_PER_NODE = {"phi": 24.0, "p": 16.0, "u": 16.0}
BYTES_PER_NODE_F32 = {"phi": 12.0, "p": 8.0, "u": 8.0}
# One FP32 Chebyshev-Jacobi smoother step with k >= 1 (d read): x, b, d read,
# d and y written (5-point: D^-1 formed per row); the 13-point step also
# reads a and D^-1
BYTES_PER_NODE_CHEB_F32 = {"phi": 28.0, "u": 20.0, "p": 20.0}

# Modelled algorithmic bytes per fine node of the mixed-precision step (the
# solver GB/s of the metric; derivation in the design notes): FP32 Krylov
# iterations (flexible GMRES inside one restart cycle; Chronopoulos-Gear CG:
# the apply with both dots 12, the update of p, s, x, r 40), FP32 V-cycles
# (temporally blocked passes: per level the down pass reads b and writes x
# and the coarse rhs, the up pass reads b, x and x_c and writes x; the
# 13-point passes also read a and D^-1; summed over the semicoarsened
# levels; the nutrient's V-cycle runs separate launches), the FP64
# refinement sweeps and the explicit FP64 step kernels.
MODEL_B_KRYLOV = {"phi": 76.0, "u": 52.0, "v": 52.0, "p": 52.0, "c": 52.0}
MODEL_B_VCYCLE = {"phi": 73.0, "u": 43.0, "v": 43.0, "p": 43.0, "c": 200.0}
MODEL_B_IR_SWEEP = 64.0
MODEL_IR_SWEEPS_PER_SOLVE = 2.0
MODEL_B_EXPLICIT = 240.0


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of a per-rank number over all ranks (identity at N=1)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank advances its own replica)."""
    return world * units_per_rank / seconds


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle
def oracle_sample(prm, geo, warmup: int, steps: int):
    """The FP64 CPU oracle on the same workload: `warmup` untimed steps then
    `steps` timed steps, single-threaded."""
    try:
        from threadpoolctl import threadpool_limits
        limiter = threadpool_limits(limits=1)
    except Exception:
        limiter = None
    from oracle import cahn_oracle as O
    from paper_1811_11842_gb300 import inputs
    c0 = inputs.initial_nutrient(prm) if prm.nutrient else None
    st = O.init_state(prm, *inputs.initial_state(prm, geo), c0)
    for _ in range(warmup):
        st = O.step(prm, st)
    t0 = time.perf_counter()
    for _ in range(steps):
        st = O.step(prm, st)
    dt = time.perf_counter() - t0
    if limiter is not None:
        limiter.unregister()
    return steps / dt, dt


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def host_cores():
    """Cores this process may run on (the oracle itself uses one)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


# ------------------------------------------------------------------ roofline
def time_apply(torch, fn, stream, dev, reps=50):
    """Mean device time of one launch of fn, L2-cold: before each launch a
    256 MB buffer (twice the 129 MB L2) is read on the same stream (a sum
    into a preallocated scalar), which leaves the L2 holding clean lines of
    that buffer -- no dirty line of an earlier write is left to drain during
    the timed launch -- and lets the host queue the launch and its events
    before the GPU reaches them; each launch is bracketed by its own event
    pair."""
    flush = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    acc = torch.empty((), dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            fn()
        for a0, a1 in ev:
            torch.sum(flush, dim=0, out=acc)
            a0.record(stream)
            fn()
            a1.record(stream)
    torch.cuda.synchronize()
    ts = sorted(a0.elapsed_time(a1) for a0, a1 in ev)
    del flush
    return sum(ts) / len(ts) / 1e3


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch on the
# 1024^2 workload, from one-kernel ncu captures of the current kernels
# (python bench.py --profile-kernel <which> under ncu --set full, three
# launches, L2 flushed by ncu before each pass); None where no capture of the
# current kernel exists.
NCU_TRAFFIC = {"k_mg_fused<float> down pass (H)": 4213760.0, "k_ch13v<float> apply": None,
               "k_ch13v<float> chebyshev": None, "k_lap5v<float> chebyshev (H)": None}


def level1_nodes(prm):
    """Nodes of the second level of the 5-point hierarchies: the grid is
    halved in y only while hx > sqrt(2) hy (or x cannot be halved), else in
    both directions (the library's coarsening rule)."""
    hx, hy = prm.lx / prm.nx, prm.ly / prm.ny
    can_x = prm.nx % 2 == 0 and prm.nx // 2 >= 4
    nx1 = prm.nx if (hx > 1.41421356 * hy or not can_x) else prm.nx // 2
    return nx1 * (prm.ny // 2 + 1)


def roofline_of(binding, sim, prm, precision, stream, dev):
    """Rooflines of the fine-level kernels, each timed live with CUDA events
    on the library's stream (L2 flushed before every launch); the first is
    the kernel family that leads the step's launch list (the temporally
    blocked down pass of the predictor's V-cycle)."""
    import torch
    n = prm.nx * (prm.ny + 1)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6793.4)
    shape = (prm.ny + 1, prm.nx)
    note = ("measured HBM copy bandwidth (MEASURED_PEAKS.json); L2 flushed by a 256 MB read "
            "before each launch")
    if precision == "mixed":
        f32 = lambda: torch.rand(shape, dtype=torch.float32, device=dev)
        x, b, d, y = f32(), f32(), f32(), f32()
        out = []

        def entry(name, fn, bpn, desc):
            t = time_apply(torch, fn, stream, dev)
            ach = bpn * n / t / 1e9
            bpn = round(bpn, 3)
            out.append({"bound": "hbm", "kernel": name, "what": desc, "achieved": ach,
                        "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                        "traffic": NCU_TRAFFIC.get(name), "peak_note": note,
                        "us_per_launch": t * 1e6, "bytes_per_node": bpn, "nodes": n})

        # b read, x written (4 B each), the level-1 right-hand side written
        entry("k_mg_fused<float> down pass (H)",
              lambda: binding.cahn_mg_down32(sim.ctx, 0, binding.SYS_U, b.data_ptr(),
                                             y.data_ptr()),
              8.0 + 4.0 * level1_nodes(prm) / n,
              "the V-cycle's first pass on the velocity predictor's fine level: three "
              "Chebyshev-Jacobi steps from zero, the residual and its restriction, one launch")
        entry("k_lap5v<float> chebyshev (H)",
              lambda: binding.cahn_smooth32(sim.ctx, 0, binding.SYS_U, 1, x.data_ptr(),
                                            b.data_ptr(), d.data_ptr(), y.data_ptr()),
              BYTES_PER_NODE_CHEB_F32["u"],
              "FP32 Chebyshev-Jacobi step (k = 1) of the velocity predictor's fine level")
        entry("k_ch13v<float> chebyshev",
              lambda: binding.cahn_smooth32(sim.ctx, 0, binding.SYS_PHI, 1, x.data_ptr(),
                                            b.data_ptr(), d.data_ptr(), y.data_ptr()),
              BYTES_PER_NODE_CHEB_F32["phi"],
              "FP32 Chebyshev-Jacobi step (k = 1) of the phase-field fine level")
        entry("k_ch13v<float> apply",
              lambda: binding.cahn_apply32(sim.ctx, 0, 0, x.data_ptr(), y.data_ptr()),
              BYTES_PER_NODE_F32["phi"], "FP32 13-point phase-field operator y = A x")
        main = dict(out[0])
        main["kernels"] = out[1:]
        return main
    x = torch.rand(shape, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    t = time_apply(torch, lambda: binding.cahn_apply(sim.ctx, 0, 0, x.data_ptr(), y.data_ptr()),
                   stream, dev)
    achieved = FLOPS_PER_NODE["phi"] * n / t / 1e12
    return {"bound": "alu", "kernel": "k_ch13v<double>: 13-point phase-field operator, FP64",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
            "peak_note": "FP64 FMA units x clock (152 x 2 x 2 flop x 2.07 GHz)",
            "us_per_launch": t * 1e6,
            "hbm_gbs_algorithmic": BYTES_PER_NODE["phi"] * n / t / 1e9}


def solver_bytes_model(iters, nodes, names):
    """Modelled algorithmic bytes of one mixed step (see MODEL_*)."""
    per_node = MODEL_B_EXPLICIT
    for k in names:
        per_node += iters[k] * (MODEL_B_KRYLOV[k] + MODEL_B_VCYCLE[k])
        per_node += MODEL_IR_SWEEPS_PER_SOLVE * MODEL_B_IR_SWEEP
    return per_node * nodes, per_node


def profile_kernel(which="ch13", nutrient_bc=0, n=1024):
    """Three launches of one FP32 kernel on the two-protrusion workload at
    n x n intervals (1024 by default), for an ncu capture with -c 3:
    ch13 / nut5 / lap5 the operator applies y = A x of the phase field, the
    nutrient and the velocity predictor H (regex k_ch13 / k_lap5); ch13cheb
    and lap5cheb one fine-level smoother step (k = 1) of the phase-field and
    predictor V-cycles; lap5down the predictor V-cycle's first pass on the
    fine level (regex k_mg_fused).  Above 1024^2 the instance is built with GMRES(2)
    and Jacobi scaling, so that it holds a few GB of device memory only (the
    applies only).  With CAHN_TILE=32 in the environment the tile autotuner
    launches nothing, so these are the first launches of the kernel."""
    import torch
    from paper_1811_11842_gb300 import binding, inputs
    from paper_1811_11842_gb300 import build as B
    B.build()
    prm, geo, _ = inputs.config_large()
    prm = prm.replace(precision=inputs.MIXED, rtol=1e-10, nutrient=1 if which == "nut5" else 0,
                      nutrient_bc=nutrient_bc, nx=n, ny=n)
    cheb = which.endswith("cheb")
    down = which == "lap5down"
    if n > 1024:
        if cheb:
            raise SystemExit("--profile-kernel %s: 1024^2 and below" % which)
        prm = prm.replace(restart=2, precond=1)
    sim = binding.Simulation([prm], [inputs.initial_state(prm, geo)])
    f32 = lambda: torch.rand((prm.ny + 1, prm.nx), dtype=torch.float32, device="cuda")
    x, y, b, d = f32(), f32(), f32(), f32()
    sysid = {"nut5": binding.SYS_C, "lap5": binding.SYS_U, "lap5cheb": binding.SYS_U,
             "lap5down": binding.SYS_U}.get(which, binding.SYS_PHI)
    for _ in range(3):
        if down:
            binding.cahn_mg_down32(sim.ctx, 0, sysid, b.data_ptr(), y.data_ptr())
        elif cheb:
            binding.cahn_smooth32(sim.ctx, 0, sysid, 1, x.data_ptr(), b.data_ptr(), d.data_ptr(),
                                  y.data_ptr())
        else:
            binding.cahn_apply32(sim.ctx, 0, sysid, x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    sim.close()
    print("profile-kernel done")


def batch_measure(count, steps, warmup, seq_steps=2):
    """`count` independent instances (sizes {128..512}^2, chi ~ U[2,3],
    log10 M ~ U[-4,-2], r ~ U[0.05,0.15]; mixed precision) advanced together
    by one CUDA graph per step, against the same instances stepped one at a
    time in graph mode, mixed and plain FP64 (seq_steps timed steps each,
    after one warm-up step).  Device time with CUDA events."""
    import torch
    from paper_1811_11842_gb300 import binding, inputs
    from paper_1811_11842_gb300 import build as B
    B.build()
    dev = torch.device("cuda", 0)
    cfgs = inputs.config_batch(count)
    prms = [p.replace(use_graph=1, precision=inputs.MIXED, rtol=1e-10) for p, _ in cfgs]
    states = [inputs.initial_state(p, g) for p, g in cfgs]
    stream = torch.cuda.Stream(dev)
    sim = binding.Simulation(prms, states, stream=stream)
    tiles = {}
    for k, p in enumerate(prms):
        tiles.setdefault(f"{p.nx}x{p.ny}", binding.tile_heights(sim.ctx, k))
    for _ in range(warmup):
        sim.step(1)
    torch.cuda.synchronize()
    launches = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    launches = binding.cahn_last_launch_count(sim.ctx)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sim.close()
    value = count * steps / (ms / 1e3)

    def sequential(precision, rtol):
        total = 0.0
        for p, st in zip(prms, states):
            s1 = binding.Simulation([p.replace(precision=precision, rtol=rtol)], [st],
                                    stream=stream)
            s1.step(1)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            s1.step(seq_steps)
            a1.record(stream)
            torch.cuda.synchronize()
            total += a0.elapsed_time(a1) / seq_steps
            s1.close()
        return count / (total / 1e3)

    seq_mixed = sequential(inputs.MIXED, 1e-10)
    seq_fp64 = sequential(inputs.FP64, 1e-12)
    sizes = sorted(p.nx for p in prms)
    return {"value": value, "unit": "instance-steps/s", "instances": count, "steps": steps,
            "warmup": warmup, "ms_per_step": ms / steps,
            "workload": f"{count} independent biofilm instances, sizes {sizes[0]}^2.."
                        f"{sizes[-1]}^2 (seeded draw), one CUDA graph per step",
            "nodes_total": sum(p.nx * (p.ny + 1) for p in prms),
            "node_steps_per_s": sum(p.nx * (p.ny + 1) for p in prms) * steps / (ms / 1e3),
            "gpu_launches": launches, "tile_heights": tiles,
            "sequential_mixed": {"value": seq_mixed, "unit": "instance-steps/s",
                                 "steps_per_instance": seq_steps},
            "sequential_fp64": {"value": seq_fp64, "unit": "instance-steps/s",
                                "steps_per_instance": seq_steps},
            "batched_over_sequential_mixed": value / seq_mixed,
            "batched_over_sequential_fp64": value / seq_fp64}


def paper_measure(steps, warmup, n=256):
    """The paper's own parameter set (double well Gamma2 = 1.25e6, viscosity
    ratio 4.3e5, shear u = 0.1, 256^2 over [0,1]^2, dt 0.02): device time of
    `steps` graph-mode steps, mixed and FP64, with the field error between
    the two."""
    import numpy as np
    import torch
    from paper_1811_11842_gb300 import binding, inputs
    prm, geo, _ = inputs.config_paper(n)
    state = inputs.initial_state(prm, geo)
    stream = torch.cuda.Stream()
    out = {"workload": "the paper's parameter set (Re_s 9.98e-4, Re_n 2.33e-9, Lambda 1e-10, "
                       "Gamma1 33.467, Gamma2 1.25e6, shear u 0.1) at %dx%d over [0,1]^2, "
                       "dt 0.02, S = 2 Gamma2" % (n, n)}
    finals = {}
    for name, prec, rtol in (("mixed", inputs.MIXED, 1e-10), ("fp64", inputs.FP64, 1e-12)):
        p = prm.replace(precision=prec, rtol=rtol, use_graph=1)
        sim = binding.Simulation([p], [state], stream=stream)
        for _ in range(warmup):
            sim.step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = np.zeros(binding.NSYS)
        e0.record(stream)
        _, st = sim.step(steps)
        iters += np.array(st[0]["iters"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        finals[name] = sim.numpy(0)
        sim.close()
        out[name] = {"steps_per_s": steps / (ms / 1e3), "ms_per_step": ms / steps,
                     "iters_per_step": {k: float(v) / steps
                                        for k, v in zip(("phi", "u", "v", "p"), iters)}}
    out["rel_err_mixed_vs_fp64"] = {
        k: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        for k, a, b in zip(("phi", "u", "v", "p"), finals["mixed"], finals["fp64"])}
    out["steps"], out["warmup"] = steps, warmup
    return out


def batch_bench(args):
    b = batch_measure(args.batch, args.steps, args.warmup, max(1, min(args.steps, 3)))
    line = {"metric": "aggregate instance-steps/s, batched mixed vs sequential mixed and FP64",
            "value": b["value"], "unit": "instance-steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": b["workload"], "nodes_total": b["nodes_total"],
                       "tile_heights": b["tile_heights"]},
            "gpu_launches": b["gpu_launches"],
            "sequential_mixed": b["sequential_mixed"], "sequential_fp64": b["sequential_fp64"],
            "batched_over_sequential_mixed": b["batched_over_sequential_mixed"],
            "batched_over_sequential_fp64": b["batched_over_sequential_fp64"]}
    print(json.dumps(line), flush=True)


def adjoint_bench(args):
    """Gradient of the detached-biofilm volume (rows above y = 0.25) with
    respect to phi0, chi and M through 50 FP64 steps of the 256^2 workload,
    checkpoints every 10: the time of one cahn_vjp call (forward with
    checkpoints, segment recomputation, reverse steps with transposed
    solves) beside the time of the same 50 forward steps alone."""
    import torch
    from paper_1811_11842_gb300 import autograd as AG
    from paper_1811_11842_gb300 import binding, inputs
    from paper_1811_11842_gb300 import build as B
    B.build()
    dev = torch.device("cuda", 0)
    prm, geo, _ = inputs.config_medium()
    prm = prm.replace(use_graph=1)   # forward passes replay the captured step
    nsteps, ck = 50, 10
    state = inputs.initial_state(prm, geo)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        sim = binding.Simulation([prm], [state], stream=stream)
    ins = [torch.as_tensor(a, dtype=torch.float64, device=dev).contiguous() for a in state]
    jbar = AG.detached_volume_weights(prm, device=dev)
    out = torch.empty_like(ins[0])
    ptrs = [t.data_ptr() for t in ins]
    torch.cuda.synchronize()

    def vjp():
        return binding.cahn_vjp(sim.ctx, 0, *ptrs, nsteps, ck, jbar.data_ptr(), out.data_ptr())

    for _ in range(args.warmup):
        vjp()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        _, theta, st = vjp()
        launches += binding.cahn_last_launch_count(sim.ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    # the 50 forward steps alone, from the same fresh start
    fwd = []
    for _ in range(max(1, min(args.steps, 3))):
        s1 = binding.Simulation([prm], [state], stream=stream)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s1.step(nsteps)
        f1.record(stream)
        torch.cuda.synchronize()
        fwd.append(f0.elapsed_time(f1))
        s1.close()
    sim.close()
    fwd_ms = sorted(fwd)[len(fwd) // 2]
    line = {"metric": "adjoint gradient evaluations/s (d J / d phi0, chi, M through 50 FP64 steps)",
            "value": 1e3 / ms, "unit": "gradients/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_gradient": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "one-protrusion biofilm, 256x256 intervals over [0,2]x[0,1], "
                                   "dt 2.5e-5, 50 steps, checkpoints every 10, objective: "
                                   "phi volume above y = 0.25",
                       "nx": prm.nx, "ny": prm.ny, "nsteps": nsteps, "checkpoint": ck},
            "forward_50_steps_ms": fwd_ms, "gradient_over_forward": ms / fwd_ms,
            "transposed_solve_iters_per_gradient": st["iters"],
            "dJ_dchi": theta[0], "dJ_dM": theta[1],
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP64 run beside the mixed one")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-driven convergence loops instead of CUDA-graph steps")
    ap.add_argument("--profile-kernel", nargs="?", const="ch13",
                    choices=["ch13", "nut5", "lap5", "ch13cheb", "lap5cheb", "lap5down"],
                    help="only launch one FP32 kernel three times (ncu target): the operator "
                         "of the phase field (default), the nutrient or the velocity "
                         "predictor H, a fine-level smoother step (ch13cheb, lap5cheb), or "
                         "the predictor V-cycle's first pass (lap5down)")
    ap.add_argument("--profile-n", type=int, default=1024,
                    help="grid of --profile-kernel: n x n intervals over [0,4]x[0,1]")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the discrete adjoint (gradient through 50 FP64 steps at 256^2)")
    ap.add_argument("--batch", type=int, default=0,
                    help="batched workload: N seeded instances of uneven size in one graph")
    ap.add_argument("--batch-inline", type=int, default=64,
                    help="instances of the batched workload measured beside the default run "
                         "(its 'batch' object; 0 skips it)")
    ap.add_argument("--paper-inline", type=int, default=1,
                    help="1: measure the paper's own parameter set at 256^2 beside the default "
                         "run (its 'paper_params' object); 0 skips it")
    ap.add_argument("--nutrient", action="store_true",
                    help="the 1024^2 workload with nutrient transport and network production")
    ap.add_argument("--nutrient-bc", default="flux", choices=["flux", "top"],
                    help="nutrient walls: zero flux on both (default) or c = c_bulk on the top wall")
    args = ap.parse_args()
    if args.profile_kernel:
        profile_kernel(args.profile_kernel, 1 if args.nutrient_bc == "top" else 0, args.profile_n)
        return
    if args.batch:
        batch_bench(args)
        return
    if args.adjoint:
        adjoint_bench(args)
        return
    ws, rank, local = dist_env()

    from paper_1811_11842_gb300 import inputs
    prm, geo, _ = inputs.config_large()
    prm = prm.replace(use_graph=0 if args.host_loop else 1, nutrient=1 if args.nutrient else 0,
                      nutrient_bc=1 if args.nutrient_bc == "top" else 0)
    prm64 = prm
    if args.precision == "mixed":
        # FP32 inner solves, FP64 refinement of every solve to 1e-10
        prm = prm.replace(precision=inputs.MIXED, rtol=1e-10)
    workload = {"workload": "two-protrusion biofilm step, 1024x1024 intervals over [0,4]x[0,1], "
                            "dt 1e-4, chi 2.5, M 1e-3, viscosity ratio 10:1",
                "nx": prm.nx, "ny": prm.ny, "krylov": "GMRES(%d)" % prm.restart,
                "precond": "jacobi" if prm.precond == 1 else "multigrid(%d)" % prm.mg_levels,
                "precision": args.precision, "rtol": prm.rtol,
                "launch": "host loop" if args.host_loop else "CUDA graph per step, device-side loops",
                "l2": ("step timed with warm L2: the FP32 working set of the inner solves "
                       "(4.2 MB per field) lives in the 129 MB L2 between launches; the "
                       "roofline kernels are timed with a 256 MB buffer written before each "
                       "launch (L2 flushed)" if args.precision == "mixed" else
                       "step timed with warm L2: FP64 fields of 8.4 MB; the GMRES(30) basis "
                       "(31 x 8.4 MB) exceeds the 129 MB L2; the roofline kernel is timed with "
                       "the L2 flushed before each launch")}
    if args.nutrient:
        workload["workload"] += (", nutrient transport + network production (D_s %g, mu %g, "
                                 "K_c %g, A %g, c0 %g, %s; CG + V-cycle)"
                                 % (prm.diff_s, prm.growth_mu, prm.growth_kc, prm.consume_a,
                                    prm.c_bulk, "c = c_bulk on the top wall"
                                    if prm.nutrient_bc == 1 else "zero flux on both walls"))
    names = ("phi", "u", "v", "p", "c")[:5 if args.nutrient else 4]

    if args.impl == "reference":
        if rank != 0:
            return
        w, k = min(args.warmup, 1), max(1, min(args.steps, 2))
        v, dt = oracle_sample(prm, geo, w, k)
        sample = f"{k} oracle steps of the 1024^2 workload after {w} warm-up step(s)"
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
                "steps": k, "warmup": w, "ms_per_step": 1e3 * dt / k, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload,
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": sample, "cpu": cpu_model(),
                                 "host_cores": host_cores()},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch
    from paper_1811_11842_gb300 import binding
    from paper_1811_11842_gb300 import build as B

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    # one rank per node compiles (if the library is stale); the others wait
    if local == 0:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    binding.load()

    state = inputs.initial_state(prm, geo)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        sim = binding.Simulation([prm], [state], device=str(dev), stream=stream)
    workload["tile_heights"] = binding.tile_heights(sim.ctx)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize(dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    launches = 0
    iters = np.zeros(binding.NSYS)
    barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the K steps as one call of the library (cahn_step with nsteps = K: the
    # caller's fields copied in and out once, every step's device checks
    # read back as it ends)
    ev0.record(stream)
    _, st = sim.step(args.steps)
    ev1.record(stream)
    launches = binding.cahn_last_launch_count(sim.ctx)
    iters = np.array(st[0]["iters"], dtype=float)
    torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    t_max = max_over_ranks(ms, dev)
    value = job_rate(args.steps, ws, t_max / 1e3)

    # end to end: host state in pinned memory, copies inside every step.  A
    # second context from the same input with the same warm-up times the
    # same steps as the device-timed loop above (the later steps of a run
    # need fewer iterations, so timing steps after it would flatter e2e).
    with torch.cuda.stream(stream):
        sim_e = binding.Simulation([prm], [state], device=str(dev), stream=stream)
    for _ in range(args.warmup):
        sim_e.step(1)
    host = [torch.from_numpy(a.copy()).pin_memory() for a in sim_e.numpy(0)]
    ptr = lambda k: [host[k].data_ptr()]
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        binding.cahn_step_host(sim_e.ctx, 1, ptr(0), ptr(1), ptr(2), ptr(3))
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    sim_e.close()
    nbytes = 4 * sum(h.numel() * 8 for h in host[:1])

    # roofline of the dominant kernel family, timed live with CUDA events on
    # the library's stream: the 13-point phase-field operator -- FP32 in the
    # mixed form (HBM-bound: x, a, y = 12 B/node), FP64 otherwise (FP64-ALU
    # bound: 26 flop/node)
    roofline = roofline_of(binding, sim, prm, args.precision, stream, dev)

    # FP64 form beside the mixed one: same input, same number of steps
    compare = None
    if args.precision == "mixed" and not args.no_compare:
        final_mixed = [f.cpu().numpy() for f in sim.fields[0]]
        nsteps_total = args.warmup + args.steps
        with torch.cuda.stream(stream):
            sim64 = binding.Simulation([prm64], [state], device=str(dev), stream=stream)
        for _ in range(args.warmup):
            sim64.step(1)
        torch.cuda.synchronize(dev)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.steps):
            sim64.step(1)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = c0.elapsed_time(c1)
        sim64.step(nsteps_total - args.warmup - args.steps)
        final64 = sim64.numpy(0)
        sim64.close()
        errs = {}
        for name, gm, g64 in zip(names, final_mixed, final64):
            errs[name] = float(np.linalg.norm(gm - g64) / max(np.linalg.norm(g64), 1e-300))
        ms64 = max_over_ranks(ms64, dev)
        compare = {"fp64_steps_per_s": job_rate(args.steps, ws, ms64 / 1e3),
                   "mixed_over_fp64": ms64 / t_max,
                   "rel_err_mixed_vs_fp64": errs, "steps_compared": nsteps_total,
                   "fp64_rtol": prm64.rtol, "mixed_outer_rtol": prm.rtol}

    iters_ps = {k: float(v) / args.steps for k, v in zip(names, iters)}
    nodes = prm.nx * (prm.ny + 1)
    solver = None
    if args.precision == "mixed":
        bstep, bnode = solver_bytes_model(iters_ps, nodes, names)
        gbs = bstep / (t_max / args.steps / 1e3) / 1e9
        hbm_peak = measured_peaks().get("hbm_gbs", 6793.4)
        solver = {"value": gbs, "unit": "GB/s", "frac": gbs / hbm_peak, "peak": hbm_peak,
                  "bytes_per_step": bstep, "bytes_per_node": bnode,
                  "kind": "algorithmic (modelled per-iteration bytes x measured iterations "
                          "per step / step time)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "solves_per_s": len(names) * value,   # phi, u, v, p [, c] per step
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic", "config": workload,
            "iters_per_step": iters_ps,
            "solver_gbs": solver,
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": {"value": job_rate(args.steps, ws, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "roofline": roofline}
    if compare:
        line["mixed_vs_fp64"] = compare
    sim.close()

    if rank == 0 and args.paper_inline and args.precision == "mixed":
        line["paper_params"] = paper_measure(20, 3)
    if rank == 0 and args.batch_inline > 0 and args.precision == "mixed":
        b = batch_measure(args.batch_inline, 5, 2)
        b.pop("tile_heights", None)
        line["batch"] = b
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        v, dt = oracle_sample(prm.replace(precision=0), geo, 0, 1)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "1 oracle step of the 1024^2 workload (single thread)",
                                "cpu": cpu_model(), "host_cores": host_cores()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
