"""Benchmark of the fast Monte Carlo path on GB300.

One step = one pass of the whole path over one batch: Latin hypercube sampling
of the N x (d*K) KL coefficients, the KL increment basis, the FP64 equilibrium,
the fused tensor-core reconstruction + EM/RK4 integration + moment partials of
all N samples, and the FP64 moment combine.  Workload: the 10-machine
classical system shaped like the IEEE 39-bus case (3 OU disturbances, K = 200
per Wiener process, T = 20 s, dt = 5 ms -> 4000 steps, N = 2^16 samples).

Metric: machine-steps/s = N * Nt * n / time (higher is better).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--path fused|plain] [--precision bf16x3|bf16|f32] [--samples N]

Under torchrun each rank simulates its own contiguous block of samples of one
global design (weak scaling); the per-rank moment sums are combined with one
all-reduce.  `--impl reference` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import fmc_synth as fs  # noqa: E402

WORKLOAD = "ieee39-shaped 10-machine classical system, 3 OU disturbances, K=200, T=20s, dt=5ms, N=2^16, LHS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="fused", choices=["fused", "plain"])
    ap.add_argument("--precision", default=None, choices=[None, "bf16x3", "bf16", "f32"])
    ap.add_argument("--samples", type=int, default=1 << 16)
    ap.add_argument("--horizon", type=float, default=20.0, help="T in seconds (profiling of shorter runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload(samples: int, horizon: float = 20.0):
    return fs.multimachine_case(n=10, d=3, K=200, T=horizon, dt=0.005, N=samples, seed=0)


def algorithmic_flops_per_sample_step(n: int, d: int, integrator_stages: int = 4) -> float:
    """FP32 FMA-pipe work of one sample over one time step (FMA = 2 flop):
    per RK stage 4n^2 (network products u, v) + 2n (Pe) + n d (forcing)
    + 6n (speed/damping/RK accumulate/next-stage input); per step d (EM)."""
    per_stage = 4 * n * n + 2 * n + n * d + 6 * n
    return 2.0 * (integrator_stages * per_stage + d)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line.strip())

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def cpu_baseline(sc, target_s: float = 15.0):
    """The FP64 oracle, as it stands, on the host cores: bounded sample of the workload."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.build()
    probe = max(cores, 4)
    zeta = oracle.lhs_sample(sc.seed, sc.N, sc.M, k0=0, count=probe)
    t0 = time.perf_counter()
    oracle.simulate(sc, zeta, nthreads=cores)
    t1 = time.perf_counter()
    per_sample = (t1 - t0) / probe
    count = int(max(probe, min(sc.N, target_s / max(per_sample, 1e-9))))
    count = (count // cores) * cores or probe
    zeta = oracle.lhs_sample(sc.seed, sc.N, sc.M, k0=0, count=count)
    t0 = time.perf_counter()
    oracle.simulate(sc, zeta, nthreads=cores)
    dt = time.perf_counter() - t0
    ms = count * sc.Nt * sc.n
    return {"value": ms / dt, "unit": "machine-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"first {count} of the {sc.N} LHS samples of the workload (FP64, {cores} threads, "
                      f"{dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sc = workload(args.samples, args.horizon)
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    # size each step so that warmup + steps stay within a few minutes
    probe = max(cores, 4)
    zeta = oracle.lhs_sample(sc.seed, sc.N, sc.M, k0=0, count=probe)
    t0 = time.perf_counter()
    oracle.simulate(sc, zeta, nthreads=cores)
    per_sample = (time.perf_counter() - t0) / probe
    budget_s = 120.0 / max(1, args.steps + args.warmup)
    count = int(max(cores, min(sc.N, budget_s / max(per_sample, 1e-9))))
    count = max(cores, (count // cores) * cores)
    times = []
    for it in range(args.warmup + args.steps):
        k0 = (it * count) % max(1, sc.N - count + 1)
        zeta = oracle.lhs_sample(sc.seed, sc.N, sc.M, k0=k0, count=count)
        t0 = time.perf_counter()
        oracle.simulate(sc, zeta, nthreads=cores)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_step = sum(times) / len(times)
    value = count * sc.Nt * sc.n / per_step
    line = {
        "impl": "reference", "metric": "machine-steps/s", "value": value, "unit": "machine-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)", "config": {"workload": WORKLOAD, "samples_per_step": count},
        "cpu_baseline": {"value": value, "unit": "machine-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{count} of the {sc.N} LHS samples per step, FP64 oracle, {cores} threads"},
        "e2e": {"value": value, "unit": "machine-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_2007_03847_gb300 as fmc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    fmc.build()
    ctx = fmc.Context(local)
    sms, gpu_name = ctx.info()
    path = args.path
    precision = args.precision or ("f32" if path == "plain" else "bf16x3")
    sc = workload(args.samples, args.horizon)
    n, Nt = sc.n, sc.Nt
    units_per_step = sc.N * Nt * n

    # L2 is flushed between timed steps by writing a buffer larger than it
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        return fmc.simulate(sc, path=path, precision=precision, ctx=ctx)

    for _ in range(args.warmup):
        step()
    fmc.device_status(ctx)
    torch.cuda.synchronize()

    fmc.profile(True, max_records=64 * (args.steps + 2), ctx=ctx)
    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        step()
        stops[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, stops)]
    total_ms = sum(step_ms)
    phase = fmc.PH_FUSED if path == "fused" else fmc.PH_INTEGRATE
    k_ms, k_launches = fmc.profile_read(phase, ctx=ctx)
    launches_total = sum(fmc.profile_read(p, ctx=ctx)[1] for p in range(8))
    fmc.profile(False, ctx=ctx)
    fmc.device_status(ctx)
    t_max = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    total_ms = float(t_max.item())
    ms_per_step = total_ms / args.steps
    value = units_per_step * world / (ms_per_step / 1e3)

    # roofline of the dominant kernel: FP32 FMA pipe
    kernel_ms = k_ms / max(1, k_launches)
    flops_per_launch = algorithmic_flops_per_sample_step(n, sc.d) * sc.N * Nt
    achieved_tflops = flops_per_launch / (kernel_ms / 1e3) / 1e12
    mhz = clk.get("sm_mhz") or (measured_peaks() or {}).get("clocks_under_load", {}).get("sm_mhz_median", 1470.0)
    peak_tflops = sms * 128 * 2 * mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak_tflops, "traffic": None,
                "kernel": "simulate_fused_kernel" if path == "fused" else "simulate_plain_kernel",
                "kernel_ms": kernel_ms,
                "peak_note": f"FP32 FMA pipe: {sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz (median SM clock "
                             f"sampled during the timed region)"}

    # end to end through the public API: scenario from host memory, moments read back
    e2e = None
    if not args.no_e2e:
        h2d = sum(np.asarray(getattr(sc, k)).nbytes for k in ("G", "B", "H", "D", "E", "Pm", "theta", "sigma",
                                                                "inject"))
        host_mean = torch.empty((Nt + 1, 2 * n), dtype=torch.float64).pin_memory()
        host_var = torch.empty_like(host_mean).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            m, v = step()
            host_mean.copy_(m, non_blocking=True)
            host_var.copy_(v, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        d2h = host_mean.numel() * 8 * 2
        e2e = {"value": units_per_step * world / e2e_s, "unit": "machine-steps/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(sc)

    if rank == 0:
        line = {
            "metric": "machine-steps/s", "value": value, "unit": "machine-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == "f32" else f"f32+{precision}",
            "data": "synthetic (seeded system and LHS design)",
            "config": {"workload": WORKLOAD, "path": path, "precision": precision, "samples_per_gpu": sc.N,
                       "steps_per_sample": Nt, "machines": n, "disturbances": sc.d, "K": sc.K,
                       "l2": "flushed between timed steps (512 MB write)", "gpu": gpu_name, "sms": sms},
            "e2e": e2e, "gpu_launches": int(launches_total), "roofline": roofline, "cpu_baseline": base,
            "clocks": clk,
        }
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
