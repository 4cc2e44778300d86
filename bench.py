#!/usr/bin/env python
"""Benchmark of the decomposition-method (DM) solver on one GB300 per rank.

Workload (default): the PDE-shaped block-tridiagonal system -- second-order
finite differences over N = 2048 grid points times cubic-spline collocation
with m = 256 (banded blocks, half-bandwidth 3, stored dense), one right-hand
side, float64 DM with P = 64 subsystems, DM on the supplementary system and
on its supplementary system (levels = 3: the fastest of P in {4, 16, 64} x
levels {1, 2, 3} on GB300).  A step is one factor + solve of the whole system (every stage
of the method: subsystem sweeps, supplementary assembly and solve,
back-substitution, float64 residual), inputs resident in device memory.

Printed: one JSON line (rank 0).  `value` is solved systems per second over
all ranks (each rank solves its own replica: the method has no data-path
exchange across GPUs here).  Also reported: TFLOP/s, per-step latency
percentiles, the roofline of the dominant kernel (CUDA events inside the
timed region), an end-to-end figure through the C ABI with host buffers, the
CPU oracle timed on the host cores, a sweep over P and recursion depth, and
the mixed-precision (float32 factors + float64 refinement) path on the same
workload.

`--impl reference` times the CPU oracle (oracle/dm_oracle.py, numpy float64)
on the same workload instead: the reference arm of this benchmark.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_, M_, R_, P_, LEV_ = 2048, 256, 1, 64, 3
SEED = 2
FP64_NOMINAL_TFLOPS = 1.25  # GB300 nominal float64 (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)
BF16_FALLBACK_TFLOPS = 1900.0  # recipe fallback when the measured-peaks file is absent


def measured_peaks():
    """The measured peaks (HBM copy GB/s, cuBLAS bf16 TFLOP/s) if present."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


def probe_peaks(dm, dev=0):
    """This library's own probes (dm_peak_probe): float64 and float32
    register-tile FMA loops, tcgen05 TF32 and bf16 MMA loops; best of 5
    timed launches each, with the SM clock sampled while each runs."""
    out = {}
    for name, kind in (("fp64", dm.DM_PROBE_FP64), ("fp32", dm.DM_PROBE_FP32), ("tf32", dm.DM_PROBE_TF32),
                       ("bf16", dm.DM_PROBE_BF16)):
        clk = Clocks(dev)
        clk.start()
        try:
            tf, ms = dm.dm_peak_probe(kind, 5)
            out[name] = {"tflops": tf, "ms": ms}
        except dm.DMError as e:
            out[name] = {"error": str(e)}
        c = clk.stop()
        out[name]["sm_mhz"] = c.get("sm_mhz")
        out[name]["reasons"] = c.get("reasons")
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip sweep, mixed, e2e and cpu legs")
    ap.add_argument("--N", type=int, default=2048, help="block rows (smaller cases for profiler captures)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "bf16x3"],
                    help="factor precision of the timed path (mixed ones refine in float64)")
    ap.add_argument("--workload", default="pde", choices=["pde", "precision", "batch", "serve", "paper"],
                    help="pde: the benchmark line (default); precision / batch / serve: the "
                         "conditioned-block, batched and served workloads, one JSON line each")
    ap.add_argument("--seconds", type=float, default=2.0, help="serve: length of the arrival stream")
    ap.add_argument("--budget", type=float, default=0.25,
                    help="serve: latency budget for admission in seconds (0: admit everything)")
    return ap.parse_args()


def workload():
    from paper_1505_06864_gb300 import workloads as w
    return w.pde_banded_system(N_, M_, R_, SEED)


def workload_name():
    return f"pde-banded block-tridiagonal N={N_} m={M_} hb=3 nrhs={R_} seed={SEED}"


def blas_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] or [os.cpu_count() or 1])
    except Exception:
        return os.cpu_count() or 1


def cpu_oracle_solve(s):
    from oracle import dm_oracle as o
    t0 = time.perf_counter()
    x = o.dm(s.A, s.B, s.C, s.b, P_, levels=LEV_)
    return time.perf_counter() - t0, x


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons (every 200 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev, self.proc, self.path = dev, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    global N_
    N_ = args.N
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    s = workload()
    for _ in range(args.warmup):
        cpu_oracle_solve(s)
    times = []
    for _ in range(args.steps):
        t, x = cpu_oracle_solve(s)
        times.append(t)
    total = sum(times)
    v = args.steps / total
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": "solved systems/s", "value": v, "unit": "systems/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(), "P": P_, "levels": LEV_, "precision": "fp64"},
        "cpu_baseline": {"value": v, "unit": "systems/s", "cores": cores, "kind": "oracle",
                         "sample": "the full workload, one oracle DM solve per step"},
        "e2e": {"value": v, "unit": "systems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    global N_
    args = parse()
    N_ = args.N
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "pde":
        return {"precision": run_precision, "batch": run_batch, "serve": run_serve,
                "paper": run_paper}[args.workload](args)
    import torch
    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1505_06864_gb300 import dm

    s = workload()
    dev = torch.device("cuda", local)
    A, B, C = (torch.from_numpy(v).to(dev) for v in (s.A, s.B, s.C))
    b = torch.from_numpy(s.b).to(dev)
    x = torch.empty_like(b)
    stream = torch.cuda.Stream(device=dev)
    plan = dm.dm_plan(N_, M_, R_, P_, LEV_, args.precision)
    dm.dm_set_stream(plan, stream)
    info = dm.dm_plan_query(plan)
    mixed = args.precision != "fp64"

    def step():
        dm.dm_factor(plan, A, B, C)
        return dm.dm_solve(plan, b, x, allow_notconv=mixed)

    # measured arithmetic peaks (before any timing; ~2 s)
    peaks = probe_peaks(dm, local)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # timed region: the product's path (launch sequences replayed from CUDA
    # graphs, no per-launch instrumentation)
    clocks = Clocks(local)
    clocks.start()
    launches0 = dm.dm_launch_count(plan)
    barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        relres = step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = dm.dm_launch_count(plan) - launches0
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = max_over_ranks(total_ms, ws, dev)
    xh = x.cpu().numpy()
    rel_true = rel_err(xh, s.x_true)
    flops_step = info["factor_flops"] + info["solve_flops"]
    value = job_value(args.steps, ws, total_ms)

    # per-kernel durations: the same steps again, eagerly, with CUDA events
    # around every launch on the plan's stream (a second timed region)
    dm.dm_profile(plan, True)
    ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev2[0].record(stream)
    for k in range(args.steps):
        step()
    ev2[1].record(stream)
    torch.cuda.synchronize()
    prof = dm.dm_profile(plan, False)
    prof_ms_step = ev2[0].elapsed_time(ev2[1]) / args.steps

    # roofline of the dominant kernel class (largest summed event time)
    top = max(prof.items(), key=lambda kv: kv[1]["ms"])
    kname, kd = top
    roof = class_roofline(kname, kd, prof, mixed, clk, peaks, dev)
    roof["timing"] = ("CUDA events around each launch in a second run of the same steps "
                      f"({prof_ms_step:.1f} ms/step instrumented vs {total_ms / args.steps:.1f} graph-replayed)")
    others = sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[1:4]
    roof["next"] = {k: {key: val for key, val in class_roofline(k, v, prof, mixed, clk, peaks, dev).items()
                        if key in ("bound", "achieved", "peak", "unit", "frac", "share_of_step")}
                    for k, v in others}
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps,
                   "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12) if v["ms"] > 0 else 0.0}
               for k, v in prof.items()}

    line = {
        "metric": "solved systems/s", "value": value, "unit": "systems/s", "n_gpus": ws,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if not mixed else f"{args.precision} factors + f64 refinement",
        "data": "synthetic",
        "config": {"workload": workload_name(), "P": info["P"], "levels": info["levels"], "P2": info["P2"],
                   "precision": args.precision, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (3.2 GB of blocks per step)"},
        "tflops": flops_step * value / 1e12,
        "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
        "relres": relres, "rel_err_vs_xtrue": rel_true,
        "roofline": roof, "kernels": kernels, "gpu_launches": launches, "clocks": clk,
        "peaks": {"probes": peaks, "measured_file": {k: measured_peaks().get(k) for k in
                                                      ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")}},
    }
    if rank == 0 and not args.no_extras:
        line["e2e"] = e2e_leg(dm, s, stream, ws)
        line["sweep"] = sweep_leg(dm, A, B, C, b, stream)
        line["mixed"] = mixed_leg(dm, A, B, C, b, stream, xh, peaks)
        if ws == 1:
            t, xo = cpu_oracle_solve(s)
            line["cpu_baseline"] = {"value": 1.0 / t, "unit": "systems/s", "cores": blas_threads(),
                                    "kind": "oracle",
                                    "sample": f"the full workload: one numpy float64 DM solve (P={P_}, levels={LEV_})"}
            line["rel_err_vs_oracle"] = rel_err(xh, xo)
    elif rank == 0:
        line["e2e"] = None
    dm.dm_destroy(plan)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def max_over_ranks(value, ws, device):
    """The largest of every rank's value (replicas: the job's time is the
    slowest rank's); one all_reduce of a scalar, no data-path collective."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps, ws, total_ms):
    """Whole-job throughput: every rank solved `steps` systems in total_ms."""
    return ws * steps / (total_ms / 1e3)


def rel_err(x, xref):
    """max over right-hand-side columns of ||x - xref||_2 / ||xref||_2"""
    x = x.reshape(-1, x.shape[-1])
    xref = xref.reshape(-1, xref.shape[-1])
    return float(np.max(np.linalg.norm(x - xref, axis=0) / np.maximum(np.linalg.norm(xref, axis=0), 1e-300)))


# float64 classes whose products run as digit-sliced bf16 tensor-core MMAs: per
# float64 multiply-add, 54 slice-pair products (the 53 pairs with s + t <= 11
# and one against the zero slice that initialises the accumulators)
SLICED_CLASSES = ("fwd_factor", "back_factor", "inv_update", "assemble_h")
SLICE_PRODUCTS = 54
HBM_CLASSES = ("inv", "tc_convert", "sweep_solve", "backsub", "sep_copy", "assemble_f", "axpy_norms")


def class_roofline(kname, kd, prof, mixed, clk, peaks, dev):
    """Roofline of one kernel class: algorithmic flops (or bytes) of its
    launches over their summed CUDA-event time, against the peak of what
    bounds it: the derived float64 ALU peak for float64 CUDA-core kernels, the
    measured bf16 tensor peak (in MMA flops) for the digit-sliced products,
    the measured copy bandwidth for the passes that only move data."""
    import torch
    base = kname.split("@")[0]
    secs = kd["ms"] / 1e3
    share = kd["ms"] / sum(v["ms"] for v in prof.values())
    common = {"kernel": kname, "launches": kd["launches"], "avg_launch_ms": kd["ms"] / max(kd["launches"], 1),
              "share_of_step": share, "traffic": read_traffic(kname) if not mixed else None}
    mp = measured_peaks()
    if not mixed and base in SLICED_CLASSES:
        alg = kd["flops"] / secs / 1e12
        peak = mp.get("bf16_tflops") or 1900.0
        return {**common, "bound": "tensor", "achieved": alg * SLICE_PRODUCTS, "peak": peak, "unit": "TFLOP/s",
                "frac": alg * SLICE_PRODUCTS / peak, "achieved_algorithmic": alg,
                "mma_flops_per_algorithmic": SLICE_PRODUCTS,
                "peak_source": "bf16 dense, measured cuBLAS burst (MEASURED_PEAKS.json), of measured"}
    if base in HBM_CLASSES:
        ach = kd["bytes"] / secs / 1e9
        peak = mp.get("hbm_gbs") or 6800.0
        return {**common, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json), of measured"}
    # float64 is bound by the FP64 pipe (plain ALU arithmetic): peak = SMs x 2
    # DFMA/clk (4 flop/clk) x the SM clock sampled during the timed region
    achieved = kd["flops"] / secs / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 2070.0
    peak = sms * 4.0 * mhz * 1e6 / 1e12
    src = (f"derived: {sms} SMs x 4 float64 flop/clk x {mhz:.0f} MHz (median SM clock sampled in the timed "
           f"region); the dm_peak_probe register-tile FMA loop reaches "
           f"{peaks.get('fp64', {}).get('tflops', float('nan')):.3f} TFLOP/s at "
           f"{peaks.get('fp64', {}).get('sm_mhz') or float('nan'):.0f} MHz")
    return {**common, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "peak_source": src, "nominal_peak": FP64_NOMINAL_TFLOPS,
            "probe_peak": peaks.get("fp64", {}).get("tflops")}


def read_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) >= 2 and f[0] == kernel:
            try:
                return float(f[1])
            except ValueError:
                return None
    return None


def e2e_leg(dm, s, stream, ws, steps=3):
    """Same metric through the C ABI with pinned host buffers (copies timed),
    after three warm-up steps (the first replay captures the CUDA graphs);
    beside it the pinned host-to-device bandwidth of one 1 GiB copy."""
    import torch
    pin = lambda a: torch.from_numpy(a).pin_memory()
    A, B, C, b = pin(s.A), pin(s.B), pin(s.C), pin(s.b)
    x = torch.empty_like(b).pin_memory()
    plan = dm.dm_plan(N_, M_, R_, P_, LEV_, dm.DM_FP64)
    dm.dm_set_stream(plan, stream)
    for _ in range(3):
        dm.dm_factor(plan, A, B, C)
        dm.dm_solve(plan, b, x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        dm.dm_factor(plan, A, B, C)
        dm.dm_solve(plan, b, x)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    # the same plan with device-resident inputs, and the factor / solve calls
    # of the host-input step timed apart (host clock around synchronised calls)
    dev = [t.to("cuda") for t in (A, B, C, b)]
    xd = torch.empty_like(dev[3])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        dm.dm_factor(plan, *dev[:3])
        dm.dm_solve(plan, dev[3], xd)
    torch.cuda.synchronize()
    dt_dev = (time.perf_counter() - t0) / steps
    tf = ts = 0.0
    for _ in range(steps):
        t0 = time.perf_counter()
        dm.dm_factor(plan, A, B, C)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        dm.dm_solve(plan, b, x)
        torch.cuda.synchronize()
        tf += t1 - t0
        ts += time.perf_counter() - t1
    del dev, xd
    dm.dm_destroy(plan)
    dA = torch.empty(A.shape, dtype=A.dtype, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dA.copy_(A, non_blocking=True)
    torch.cuda.synchronize()
    e0.record()
    dA.copy_(A, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    h2d_gbs = A.numel() * 8 / (e0.elapsed_time(e1) / 1e3) / 1e9
    del dA
    h2d = 8 * (3 * N_ * M_ * M_ + N_ * M_ * R_)
    return {"value": ws / dt, "unit": "systems/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * N_ * M_ * R_,
            "ms_per_step": 1e3 * dt, "pinned_h2d_gbs": h2d_gbs,
            "h2d_ms_at_that_rate": h2d / (h2d_gbs * 1e9) * 1e3,
            "same_plan_device_inputs_ms": 1e3 * dt_dev,
            "host_inputs_factor_ms": 1e3 * tf / steps, "host_inputs_solve_ms": 1e3 * ts / steps}


def timed(fn, reps=1):
    import torch
    fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        out = fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps, out


def sweep_leg(dm, A, B, C, b, stream):
    """P in {4, 16, 64} x recursion depth {1, 2, 3} (the workload's stated
    sweep), then outside it: P = 128 and 152, DM inside the subsystems
    (M subsystems of J sub-subsystems, Section 4.2.2), and P = 64 with the
    float64 products on the FP64 pipe.  One warm-up and one timed step each."""
    import torch
    out = []
    x = torch.empty_like(b)

    def run(plan, rec):
        dm.dm_set_stream(plan, stream)
        q = dm.dm_plan_query(plan)
        dt, rel = timed(lambda: (dm.dm_factor(plan, A, B, C), dm.dm_solve(plan, b, x))[1])
        rec.update({"P": q["P"], "levels": q["levels"], "P2": q["P2"], "systems_per_s": 1.0 / dt,
                    "ms": 1e3 * dt, "relres": rel})
        out.append(rec)
        dm.dm_destroy(plan)

    for P in (4, 16, 64):
        for lv in (1, 2, 3):
            run(dm.dm_plan(N_, M_, R_, P, lv, dm.DM_FP64), {})
    for P in (128, 152):
        run(dm.dm_plan(N_, M_, R_, P, 3, dm.DM_FP64), {"outside_stated_set": True})
    for M, J, outer in ((16, 4, 2), (32, 2, 2), (64, 2, 2)):
        run(dm.dm_plan_inside(N_, M_, R_, M, J, outer, dm.DM_FP64),
            {"inside": {"M": M, "J": J, "outer_levels": outer}, "outside_stated_set": True})
    run(dm.dm_plan_ex(N_, M_, R_, 64, 3, dm.DM_FP64, dm.DM_PLAN_FP64_FMA), {"products": "FP64 pipe"})
    return out


def mixed_leg(dm, A, B, C, b, stream, x64, peaks, steps=5):
    """float32 factors + float64 refinement on the same workload: systems/s
    from CUDA events over `steps` graph-replayed steps after 3 warm-ups; then
    one instrumented step for the per-kernel times and the roofline of the
    factor products (fwd_factor: tcgen05 for tf32 / bf16x3, whose MMA flops
    are 1x / 3x the algorithmic ones)."""
    import torch
    out = {}
    x = torch.empty_like(b)
    mp = measured_peaks()
    bf16_peak = mp.get("bf16_tflops") or BF16_FALLBACK_TFLOPS
    for name in ("fp32", "tf32", "bf16x3"):
        plan = dm.dm_plan(N_, M_, R_, P_, LEV_, name)
        dm.dm_set_stream(plan, stream)
        ms, rel = _timed_steps(dm, plan, A, B, C, b, x, steps, 3, stream, True)
        q = dm.dm_plan_query(plan)
        prof = dm.dm_profile(plan, True)
        dm.dm_factor(plan, A, B, C)
        dm.dm_solve(plan, b, x, allow_notconv=True)
        prof = dm.dm_profile(plan, False)
        rec = {"systems_per_s": 1e3 / ms, "ms": ms, "iters": q["last_iters"], "relres": rel,
               "rel_err_vs_fp64_dm": rel_err(x.cpu().numpy(), x64),
               "kernels_ms": {k: round(v["ms"], 3) for k, v in prof.items()}}
        ff = prof.get("fwd_factor")
        if ff and ff["ms"] > 0 and name != "fp32":
            alg = ff["flops"] / (ff["ms"] / 1e3) / 1e12
            mult = 3.0 if name == "bf16x3" else 1.0
            if name == "bf16x3":
                pk, src = bf16_peak, "bf16 dense, measured cuBLAS burst (MEASURED_PEAKS.json)" if mp.get(
                    "bf16_tflops") else "bf16 dense, recipe fallback"
            else:
                pk = peaks.get("tf32", {}).get("tflops") or bf16_peak / 2
                src = "tf32 dense, measured dm_peak_probe tcgen05 kind::tf32 loop"
            rec["roofline"] = {"kernel": "fwd_factor (k_fwd_factor_tc)", "bound": "tensor",
                               "achieved_algorithmic": alg, "mma_flops_per_algorithmic": mult,
                               "achieved": alg * mult, "peak": pk, "unit": "TFLOP/s", "frac": alg * mult / pk,
                               "peak_source": src, "launches": ff["launches"],
                               "avg_launch_ms": ff["ms"] / ff["launches"]}
        out[name] = rec
        dm.dm_destroy(plan)
    return out


# ---------------------------------------------------------------- other workloads
def _timed_steps(dm, plan, A, B, C, b, x, steps, warmup, stream, mixed):
    import torch
    for _ in range(warmup):
        dm.dm_factor(plan, A, B, C)
        dm.dm_solve(plan, b, x, allow_notconv=mixed, count=dm.dm_plan_query(plan)["count"])
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(steps):
        dm.dm_factor(plan, A, B, C)
        rel = dm.dm_solve(plan, b, x, allow_notconv=mixed, count=dm.dm_plan_query(plan)["count"])
    ev[1].record(stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / steps, rel


def _profile_pass(dm, plan, A, B, C, b, x, mixed):
    """One extra factor + solve with per-launch CUDA events (not timed above):
    per kernel class, summed ms and algorithmic TFLOP/s."""
    dm.dm_profile(plan, True)
    dm.dm_factor(plan, A, B, C)
    dm.dm_solve(plan, b, x, allow_notconv=mixed, count=dm.dm_plan_query(plan)["count"])
    return {k: {"ms": round(v["ms"], 2), "tflops": round(v["flops"] / (v["ms"] * 1e9), 3) if v["ms"] > 0 else 0.0}
            for k, v in dm.dm_profile(plan, False).items()}


def run_precision(args):
    """Conditioned dense blocks: N=4096, m=128, cond(B_i)=1e4, 8 right-hand
    sides; float64 DM against float32 / TF32 / split-bf16 factors refined in
    float64 (tolerance 1e-12 on the refinement step)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1505_06864_gb300 import dm, workloads as w
    N, m, r = 4096, 128, 8
    s = w.conditioned_system(N, m, r, 3, cond=1e4)
    dev = torch.device("cuda", 0)
    A, B, C, b = (torch.from_numpy(v).to(dev) for v in (s.A, s.B, s.C, s.b))
    x = torch.empty_like(b)
    stream = torch.cuda.Stream()
    P, lv, P2 = dm.dm_plan_tune(N, m, r)
    out, x64 = {}, None
    for prec in ("fp64", "fp32", "tf32", "bf16x3"):
        plan = dm.dm_plan(N, m, r, P, lv, prec)
        dm.dm_set_stream(plan, stream)
        mixed = prec != "fp64"
        ms, rel = _timed_steps(dm, plan, A, B, C, b, x, args.steps, max(3, args.warmup), stream, mixed)
        q = dm.dm_plan_query(plan)
        kern = _profile_pass(dm, plan, A, B, C, b, x, mixed)
        xh = x.cpu().numpy()
        if prec == "fp64":
            x64 = xh
        out[prec] = {"systems_per_s": 1e3 / ms, "ms": ms, "iters": q["last_iters"], "relres": rel,
                     "last_correction": q["last_correction"], "converged": (not mixed) or q["last_correction"] <= 1e-12,
                     "rel_err_vs_xtrue": rel_err(xh, s.x_true), "rel_err_vs_fp64_dm": rel_err(xh, x64),
                     "tflops": (q["factor_flops"] + q["solve_flops"] * q["last_iters"]) / (ms / 1e3) / 1e12,
                     "kernels_ms": kern}
        dm.dm_destroy(plan)
    ok = {k: v for k, v in out.items() if k != "fp64" and v["converged"] and v["rel_err_vs_fp64_dm"] <= 1e-10}
    best = max(ok, key=lambda k: ok[k]["systems_per_s"]) if ok else "fp64"
    line = {"metric": "solved systems/s", "workload": "precision", "value": out[best]["systems_per_s"],
            "unit": "systems/s", "best_precision": best, "n_gpus": 1, "steps": args.steps,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"conditioned dense blocks N={N} m={m} nrhs={r} cond(B_i)=1e4 seed=3",
                       "P": P, "levels": lv, "P2": P2}, "results": out}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """512 independent systems, N ~ U{32..2048}, m ~ U{32,64,96,128},
    nrhs ~ U{1..16}, dominant generator drawn in device memory; one batch plan,
    inputs borrowed in place; parity on sampled systems against the oracle."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1505_06864_gb300 import dm, workloads as w
    from oracle import dm_oracle as o
    count = args.N if args.N != 2048 else 512
    shapes = w.batch_shapes(count, 4)
    Ns, ms_, rs = zip(*shapes)
    nblk = sum(n * m * m for n, m, _ in shapes)
    nvec = sum(n * m * r for n, m, r in shapes)
    dev = torch.device("cuda", 0)
    A = torch.empty(nblk, dtype=torch.float64, device=dev)
    B = torch.empty_like(A)
    C = torch.empty_like(A)
    b = torch.empty(nvec, dtype=torch.float64, device=dev)
    ob, ov = [], []
    pb = pv = 0
    for i, (n, m, r) in enumerate(shapes):
        a_, b_, c_, rhs, _ = w.dominant_system_t(n, m, r, 4000 + i, device=dev)
        A[pb:pb + n * m * m] = a_.reshape(-1)
        B[pb:pb + n * m * m] = b_.reshape(-1)
        C[pb:pb + n * m * m] = c_.reshape(-1)
        b[pv:pv + n * m * r] = rhs.reshape(-1)
        ob.append(pb)
        ov.append(pv)
        pb += n * m * m
        pv += n * m * r
        del a_, b_, c_, rhs
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    x = torch.empty_like(b)
    stream = torch.cuda.Stream()
    out = {}
    picks = [0, count - 1, int(np.argmax(Ns)), count // 2]
    for prec in ("bf16x3", "fp64"):
        try:
            plan = dm.dm_plan_batch(Ns, ms_, rs, prec)
        except dm.DMError as e:
            out[prec] = {"skipped": str(e)}
            continue
        dm.dm_set_borrow_inputs(plan)
        dm.dm_set_stream(plan, stream)
        mixed = prec != "fp64"
        ms, rel = _timed_steps(dm, plan, A, B, C, b, x, max(1, args.steps // 3), 3, stream, mixed)
        q = dm.dm_plan_query(plan)
        kern = _profile_pass(dm, plan, A, B, C, b, x, mixed)
        errs = []
        for i in picks:
            n, m, r = shapes[i]
            sl = lambda t, o0, k: t[o0:o0 + k].cpu().numpy()
            Ai, Bi, Ci = (sl(t, ob[i], n * m * m).reshape(n, m, m) for t in (A, B, C))
            bi = sl(b, ov[i], n * m * r).reshape(n, m, r)
            xi = sl(x, ov[i], n * m * r).reshape(n, m, r)
            P, lv, P2 = dm.dm_plan_tune(n, m, r)
            errs.append(rel_err(xi, o.dm(Ai, Bi, Ci, bi, P, levels=lv, P2=P2 if P2 > 1 else None)))
        out[prec] = {"systems_per_s": count * 1e3 / ms, "ms_per_batch": ms, "iters": q["last_iters"],
                     "max_relres": max(rel) if isinstance(rel, list) else rel,
                     "tflops": (q["factor_flops"] + q["solve_flops"] * q["last_iters"]) / (ms / 1e3) / 1e12,
                     "rel_err_vs_oracle_sampled": max(errs), "sampled_systems": picks, "kernels_ms": kern,
                     "device_gb": q["device_bytes"] / 1e9}
        dm.dm_destroy(plan)
        torch.cuda.empty_cache()
    line = {"metric": "solved systems/s", "workload": "batch", "value": out.get("bf16x3", {}).get("systems_per_s"),
            "unit": "systems/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic (drawn on device)",
            "config": {"workload": f"{count} dominant systems, N~U{{32..2048}}, m~U{{32,64,96,128}}, nrhs~U{{1..16}}, "
                                   f"seed=4", "blocks_gb": 3 * nblk * 8 / 1e9}, "results": out}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson arrivals (mean 2000 requests/s) of solves on a pool of resident
    systems (the batching workload's size mix plus 5 % large N=8192, m=256);
    30 % repeat right-hand sides on resident factors (one column each,
    dm_submit_cols: queued ones on a plan share a solve), the rest factor +
    solve of the plan's nrhs columns; split-bf16 factors refined in float64.
    Admission by a latency budget (--budget).  Latency = done - submit on the
    library's clock, over admitted requests."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1505_06864_gb300 import dm, workloads as w
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    small = w.batch_shapes(48, 5)
    large = [(8192, 256, 1)] * 2
    pool = []
    for i, (n, m, r) in enumerate(small + large):
        a_, b_, c_, rhs, _ = w.dominant_system_t(n, m, r, 5000 + i, device=dev)
        P, lv, _ = dm.dm_plan_tune(n, m, r)
        plan = dm.dm_plan(n, m, r, P, lv, "bf16x3")
        dm.dm_set_borrow_inputs(plan)
        dm.dm_factor(plan, a_, b_, c_)
        rhs2 = [torch.randn(n, m, 1, dtype=torch.float64, device=dev) for _ in range(3)]
        pool.append(dict(plan=plan, A=a_, B=b_, C=c_, b=rhs, rhs=rhs2, large=i >= len(small)))
    torch.cuda.synchronize()
    # seed the admission estimates: one factor + solve and one narrow solve per plan
    seed = []
    for p in pool:
        x = torch.empty_like(p["b"])
        seed.append(dm.dm_submit_system(p["plan"], p["A"], p["B"], p["C"], p["b"], x))
        seed.append(dm.dm_submit_cols(p["plan"], p["rhs"][0], torch.empty_like(p["rhs"][0]), 1))
        p["keep"] = x
    for t in seed:
        while dm.dm_poll(t)[0] == dm.DM_PENDING:
            time.sleep(0.0005)
    dm.dm_serve_budget(args.budget)
    stats0 = dm.dm_serve_stats()
    gaps = rng.exponential(1.0 / 2000.0, size=int(args.seconds * 2000 * 1.2))
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < args.seconds]
    tickets, keep = [], []
    refused = 0
    t0 = time.perf_counter()
    for ta in arrivals:
        while time.perf_counter() - t0 < ta:
            pass
        is_large = rng.random() < 0.05
        cand = [p for p in pool if p["large"] == is_large]
        p = cand[rng.integers(len(cand))]
        x = torch.empty_like(p["b"])
        try:
            if rng.random() < 0.3:
                rhs = p["rhs"][rng.integers(3)]
                x = torch.empty_like(rhs)
                t = dm.dm_submit_cols(p["plan"], rhs, x, 1)
            else:
                t = dm.dm_submit_system(p["plan"], p["A"], p["B"], p["C"], p["b"], x)
        except dm.DMError:
            refused += 1
            continue
        tickets.append(t)
        keep.append(x)
    lat, done_t, sub_t, bad = [], [], [], 0
    for t in tickets:
        while True:
            st, rel, times = dm.dm_poll_times(t)
            if st != dm.DM_PENDING:
                break
            time.sleep(0.0005)
        if st != dm.DM_OK:
            bad += 1
        lat.append(times[2] - times[0])
        sub_t.append(times[0])
        done_t.append(times[2])
    span = max(done_t) - min(sub_t)
    stats1 = dm.dm_serve_stats()
    dm.dm_serve_budget(0.0)
    for p in pool:
        dm.dm_destroy(p["plan"])
    line = {"metric": "solved systems/s", "workload": "serve", "value": len(tickets) / span, "unit": "requests/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic (drawn on device)",
            "offered_rps": len(arrivals) / args.seconds, "completed": len(tickets), "refused": refused,
            "failed": bad, "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                          "p99": 1e3 * float(np.percentile(lat, 99))},
            "budget_ms": 1e3 * args.budget,
            "merged": stats1["merged"] - stats0["merged"], "worker_runs": stats1["runs"] - stats0["runs"],
            "config": {"workload": "Poisson 2000 req/s; pool of 48 systems of the batch mix + 2 of N=8192 m=256; "
                                   "5 % large, 30 % repeat single right-hand-side columns; bf16x3 + fp64 "
                                   "refinement; admission by latency budget",
                       "seconds": args.seconds, "slots": 8}}
    print(json.dumps(line), flush=True)


def run_paper(args):
    """The paper's validation shape (Section 6): N = 3071 blocks, n = 100 and
    400, one right-hand side, Laplace blocks with small random fill, float64.
    Measured speedup of DM over block Thomas (P = 1) on the GPU against the
    analytical speedup of Eq. (SpeedupMP) for the same P."""
    import math
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1505_06864_gb300 import dm, workloads as w
    N = 3071
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    out = {}
    for m in (100, 400):
        s = w.laplace_fill_system(N, m, 1, 6)
        A, B, C, b = (torch.from_numpy(v).to(dev) for v in (s.A, s.B, s.C, s.b))
        x = torch.empty_like(b)
        rows = []
        t1 = None
        for P in (1, 4, 16, 32, 48, 64, 85, 128):
            plan = dm.dm_plan(N, m, 1, P, 1, "fp64")
            dm.dm_set_stream(plan, stream)
            ms, rel = _timed_steps(dm, plan, A, B, C, b, x, 1, 1, stream, False)
            dm.dm_destroy(plan)
            if P == 1:
                t1 = ms
            c = 5.0 + 2.0 / (1.0 + 1.0 / m)
            s_model = (3 * N - 2) / (3 * P - 5 + c * (N - P + 1) / P) if P > 1 else 1.0
            rows.append({"P": P, "ms": ms, "speedup_vs_ta": t1 / ms, "speedup_model": s_model, "relres": rel,
                         "rel_err_vs_xtrue": rel_err(x.cpu().numpy(), s.x_true)})
        out[f"n={m}"] = rows
        del A, B, C, b, x
        torch.cuda.empty_cache()
    line = {"metric": "speedup of DM over block Thomas", "workload": "paper", "unit": "x", "n_gpus": 1,
            "data": "synthetic", "config": {"workload": "Laplace blocks with random fill (eps 1e-2), N=3071, "
                                                        "n in {100, 400}, l=1, float64, levels=1"},
            "results": out}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
