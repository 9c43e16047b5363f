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
    ap.add_argument("--machines", type=int, default=10, help="machines of the system (17..52: large-system kernel)")
    ap.add_argument("--disturbances", type=int, default=3)
    ap.add_argument("--forcing", default="increments", choices=["increments", "smooth"],
                    help="smooth: the random ODE of Eq. (eqkl) (the forcing at the RK stage times)")
    ap.add_argument("--correlation", default="none", choices=["none", "rank"],
                    help="rank: the correlation-reducing permutation of the design (Section IV-B step 2)")
    ap.add_argument("--kernel", default="auto",
                    choices=["auto", "per_sample", "split", "split_tc"],
                    help="fused-path kernel policy of the timed calls (see fmc_set_kernel_policy)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--study", default=None, choices=[None, "tol", "batch", "serve", "dn"],
                    help="tol: LHS vs SRS (and precision forms) time to a stated error on E and Var; "
                         "batch: 64 uneven scenarios in one captured graph; serve: Poisson request stream; "
                         "dn: the paper's convergence experiment (generator trip, RMS frequency deviation, D(N))")
    ap.add_argument("--dn-max", type=int, default=1000, help="largest N of the dn study")
    ap.add_argument("--max-machines", type=int, default=50,
                    help="upper end of the machine count drawn for the batch and serve studies")
    ap.add_argument("--seeds", type=int, default=32)
    ap.add_argument("--slots", type=int, default=16, help="concurrent requests of the serve study's server")
    return ap.parse_args()


def workload(samples: int, horizon: float = 20.0, machines: int = 10, disturbances: int = 3):
    return fs.multimachine_case(n=machines, d=disturbances, K=200, T=horizon, dt=0.005, N=samples, seed=0)


def workload_name(args) -> str:
    extra = ("" if getattr(args, "forcing", "increments") == "increments" else ", smooth forcing") + \
            ("" if getattr(args, "correlation", "none") == "none" else ", correlation-reducing permutation")
    if args.machines == 10 and args.disturbances == 3 and args.samples == (1 << 16) and args.horizon == 20.0:
        return WORKLOAD + extra
    return (f"classical {args.machines}-machine system (39-bus-shaped draws), {args.disturbances} OU disturbances, "
            f"K=200, T={args.horizon:g}s, dt=5ms, N={args.samples}, LHS" + extra)


def algorithmic_flops_per_machine_step(n: int, integrator_stages: int = 4) -> float:
    """The method's FP32 work per machine and time step: per RK stage and machine
    4n + 8 FMA (the network sums u = G a - B b, v = G b + B a of the product form,
    4n; the angle's cosine and sine scaled by E, the electrical power a u + b v,
    the two derivatives and the RK accumulation, 8), i.e. 16n + 32 FMA per RK4
    step, 2 flop each.  The sine and cosine themselves belong to the MUFU pipe in
    this count (4 sincos per machine-step) and are reported apart."""
    return 2.0 * integrator_stages * (4 * n + 8)


def implementation_ops_per_sample_step(n: int, d: int, integrator_stages: int = 4) -> float:
    """What the per-sample fused kernel executes on the FP32 pipe per sample and
    step, counted from its source for the smallest angle tier (every FMA, multiply
    or add = one operation; a packed FMA = two): per RK stage and machine the sin /
    cos - 1 series (5), the row's network sums 4(n-1) and their two halves (2),
    the equilibrium quadrature (1), the electrical-power deviation (3), the
    forcing over the disturbance slots (nd), the derivatives (3) and the RK
    accumulate and next-stage input (4); per stage the stage forcing (2 nd) and
    the reference speed (3); per step the state update (2n + 1).  nd is the
    kernel's slot count (1, 2, 4 or 8).  Only for the issue-level fraction
    reported beside the algorithmic one."""
    nd = next(b for b in (1, 2, 4, 8) if d <= b)
    per_stage = n * (4 * (n - 1) + 18 + nd) + 2 * nd + 3
    return float(integrator_stages * per_stage + 2 * n + 1)


def algorithmic_bytes_per_launch(N: int, n: int, d: int, K: int, Nt: int, split: bool = True) -> float:
    """HBM bytes the method must move per launch: the design zeta [N][d K] in BF16
    (hi and lo for the split form), the increment basis [Nt][K] likewise, and the
    FP64 mean and variance [Nt+1][2n] written out."""
    parts = 2 if split else 1
    return float(parts * 2 * N * d * K + parts * 2 * Nt * K + 2 * 8 * (Nt + 1) * 2 * n)


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


def profiled_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu summary, if the
    kernel sources still match the profiled ones (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "simulate_fused_kernel_ieee39_N65536.traffic.txt")
    try:
        kv = dict(line.split(None, 1) for line in open(path) if line.strip() and not line.startswith("#"))
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for f in ("simulate_fused.cuh", "swing.cuh", "tc_common.cuh", "disturb_chunk.cuh", "fmc_common.cuh", "kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2007_03847_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != kv.get("source_sha256", "").strip():
        return None
    return float(kv["dram_bytes_per_launch"])


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


def run_tol_study(args):
    """Time to a stated error on the expectation and variance trajectories.

    Reference moments: an LHS design of 2^22 samples (blocks of 2^18 combined by
    their shifted sums).  For N = 2^6 .. 2^16 and R seeds per N, the error of a
    run is max_{t,s} |E_N - E_ref| / max sqrt(Var_ref) for the expectation and
    max |Var_N - Var_ref| / max Var_ref for the variance; err(N) is the RMS over
    the seeds.  Time to tolerance tau = device time of one run at the smallest N
    with err(N) <= tau.  Forms: fused BF16x3 LHS (the chosen form), fused BF16x3
    SRS, fused BF16 LHS, plain FP32 LHS, and the paper's traditional Monte Carlo
    (a fresh normal per step, no KL expansion).  The traditional Monte Carlo
    converges to the untruncated process, so its errors are taken against a
    reference of its own (2^22 samples); the distance between the two references
    (the KL truncation at this K) is reported beside them.
    """
    import torch

    import paper_2007_03847_gb300 as fmc
    fmc.build()
    ctx = fmc.Context(0)
    base = workload(1 << 22, args.horizon)
    # references: 2^22 samples in blocks of 2^18 combined by their shifted sums
    blk = 1 << 18

    def reference(sampling):
        sc0 = base.replace(sampling=sampling)
        S1 = S2 = shift = None
        for k0 in range(0, sc0.N, blk):
            a, b, sh = fmc.simulate_sums(sc0, k0, blk, ctx=ctx)
            S1 = a if S1 is None else S1 + a
            S2 = b if S2 is None else S2 + b
            shift = sh
        m, v = fmc.moments_from_sums(S1, S2, shift, sc0.N, ctx=ctx)
        return m.cpu().numpy(), v.cpu().numpy()

    refs = {fs.LHS: reference(fs.LHS), fs.SRS_EM: reference(fs.SRS_EM)}
    mref, vref = refs[fs.LHS]
    escale = float(np.sqrt(vref.max()))
    vscale = float(vref.max())
    forms = [("fused-bf16x3-LHS", "fused", "bf16x3", fs.LHS), ("fused-bf16x3-SRS", "fused", "bf16x3", fs.SRS),
             ("fused-bf16-LHS", "fused", "bf16", fs.LHS), ("plain-f32-LHS", "plain", "f32", fs.LHS),
             ("fused-SRS_EM (traditional Monte Carlo)", "fused", "bf16x3", fs.SRS_EM)]
    Ns = [1 << e for e in range(6, 17)]
    mem, vem = refs[fs.SRS_EM]
    out = {"workload": WORKLOAD.replace("N=2^16", "N varied"), "reference_samples": base.N, "seeds": args.seeds,
           "error_definition": "E: max|E_N-E_ref|/max sqrt(Var_ref); Var: max|Var_N-Var_ref|/max Var_ref; RMS over seeds",
           "kl_truncation_between_references": {"E": float(np.max(np.abs(mem - mref)) / escale),
                                                "Var": float(np.max(np.abs(vem - vref)) / vscale)},
           "forms": {}}
    for name, path, prec, samp in forms:
        rows = []
        for N in Ns:
            errs_e, errs_v, times = [], [], []
            for r in range(args.seeds):
                sc = base.replace(N=N, seed=1000 + r, sampling=samp)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                m, v = fmc.simulate(sc, path=path, precision=prec, ctx=ctx)
                b.record()
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
                m, v = m.cpu().numpy(), v.cpu().numpy()
                mr, vr = refs[fs.SRS_EM] if samp == fs.SRS_EM else refs[fs.LHS]
                errs_e.append(np.max(np.abs(m - mr)) / escale)
                errs_v.append(np.max(np.abs(v - vr)) / vscale)
            rows.append({"N": N, "err_E": float(np.sqrt(np.mean(np.square(errs_e)))),
                         "err_Var": float(np.sqrt(np.mean(np.square(errs_v)))),
                         "ms": float(np.median(times))})
        # a single run below one wave of resident CTAs costs the same latency for
        # any N; the throughput time charges N samples at the full-GPU rate
        per_sample_ms = rows[-1]["ms"] / rows[-1]["N"]
        ttt = {}
        for tau in (1e-1, 3e-2, 1e-2, 3e-3):
            for key in ("err_E", "err_Var"):
                hit = next((r for r in rows if r[key] <= tau), None)
                ttt[f"{key}<={tau:g}"] = None if hit is None else {
                    "N": hit["N"], "latency_ms": hit["ms"], "throughput_ms": hit["N"] * per_sample_ms}
        out["forms"][name] = {"rows": rows, "time_to_tol": ttt}
    print(json.dumps(out))
    ctx.close()
    return 0


def run_batch_study(args):
    """64 seeded scenarios of uneven size (machines 3..max, disturbances 1..8,
    K 50..300, T 5..60 s at dt = 5 ms, N 1k..256k) in one captured CUDA graph,
    against the same scenarios run one after another."""
    import torch

    import paper_2007_03847_gb300 as fmc
    fmc.build()
    ctx = fmc.Context(0)
    scs = fs.batched_cases(count=64, seed=0, n_range=(3, args.max_machines))
    units = sum(sc.N * sc.Nt * sc.n for sc in scs)
    b = fmc.Batch(scs, use_graph=True, ctx=ctx)
    for _ in range(max(1, args.warmup)):
        b.launch()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(args.steps):
        b.launch()
    ev[1].record()
    torch.cuda.synchronize()
    t_batch = ev[0].elapsed_time(ev[1]) / args.steps
    fmc.device_status(ctx)
    b.close()
    ev[0].record()
    for sc in scs:
        fmc.simulate(sc, path="fused", precision="bf16x3", ctx=ctx)
    ev[1].record()
    torch.cuda.synchronize()
    t_seq = ev[0].elapsed_time(ev[1])
    out = {"study": "batch", "scenarios": len(scs), "machine_steps_per_batch": units,
           "machines": [min(sc.n for sc in scs), max(sc.n for sc in scs)],
           "samples": [min(sc.N for sc in scs), max(sc.N for sc in scs)],
           "graph_ms_per_batch": t_batch, "graph_machine_steps_per_s": units / (t_batch / 1e3),
           "sequential_ms": t_seq, "sequential_machine_steps_per_s": units / (t_seq / 1e3),
           "steps": args.steps, "warmup": args.warmup}
    print(json.dumps(out))
    ctx.close()
    return 0


def run_serve_study(args):
    """Poisson request stream at several rates.  Each request draws a scenario from
    the batch study's distribution, its own seed and a target error on E and Var
    (tol_E in {1e-2, 3e-3}, tol_Var in {3e-2, 1e-2}, the normalisation of the
    convergence study); the server grows four independent designs from 256
    samples each until the targets are met (at most 2^20 samples).  Memory
    admission under a 120 GB budget.  Reports p50/p99 latency (submit -> moments
    complete), samples/s and machine-steps/s per rate."""
    import torch

    import paper_2007_03847_gb300 as fmc
    fmc.build()
    srv = fmc.Server(slots=args.slots, mem_budget_bytes=120 << 30)
    pool = fs.batched_cases(count=256, seed=1, n_range=(3, args.max_machines))
    rng = np.random.default_rng(0)
    rows = []
    for lam in (1, 2, 5, 10, 20, 50, 100, 200):
        nreq = int(min(60, max(8, 15 * lam)))
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=nreq))
        picks = rng.integers(0, len(pool), size=nreq)
        handles = []
        t0 = time.perf_counter()
        for k in range(nreq):
            now = time.perf_counter() - t0
            if arrivals[k] > now:
                time.sleep(arrivals[k] - now)
            sc = pool[picks[k]].replace(seed=int(rng.integers(0, 2**31)), N=256)
            tol_E = float(rng.choice([1e-2, 3e-3]))
            tol_V = float(rng.choice([3e-2, 1e-2]))
            handles.append((srv.submit(sc, tol_E=tol_E, tol_Var=tol_V, max_N=1 << 20), sc))
        lat, samples, msteps, met = [], 0, 0, 0
        for h, sc in handles:
            res, _, _ = srv.wait(h, timeout_s=900)
            assert res["status"] == 0, res
            lat.append(res["latency_us"] / 1e3)
            samples += res["n_used"]
            msteps += res["n_used"] * sc.Nt * sc.n
            met += int(res["target_met"])
        t_all = time.perf_counter() - t0
        rows.append({"rate_req_s": lam, "requests": nreq, "targets_met": met,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "samples_per_s": samples / t_all, "machine_steps_per_s": msteps / t_all, "wall_s": t_all})
    srv.close()
    print(json.dumps({"study": "serve", "slots": args.slots, "budget_bytes": 120 << 30, "replicates": 4,
                      "initial_samples_per_design": 256, "max_samples": 1 << 20, "rows": rows}))
    return 0


def run_dn_study(args):
    """The paper's convergence experiment (Section V-B, Table II) on the 10-machine
    system: the generator with the largest mechanical power trips at t = 1 s (its
    mechanical power is lost; the classical model keeps it electrically connected),
    the response function is the RMS of the system (centre-of-inertia) frequency
    deviation over 60 s, and for N = 1..dn_max a fresh design of N samples gives
    E[RRF](N) and Var[RRF](N).  The degree of convergence D(N) is max - min of the
    estimate over N-4..N.  Methods: LHS with K = 6 KL terms per disturbance (the
    paper's setting) and K = 200, and the traditional Monte Carlo (a fresh normal
    per step).  Reported: D at dn_max for each method and the smallest N at which
    each KL/LHS method's D falls to the traditional Monte Carlo's D(dn_max)."""
    import paper_2007_03847_gb300 as fmc
    fmc.build()
    ctx = fmc.Context(0)
    base = fs.multimachine_case(n=10, d=3, K=6, T=60.0, dt=0.005, N=1, seed=0)
    k = int(np.argmax(base.Pm[1:])) + 1          # not the balancing machine 0
    base = base.replace(event_machine=k, event_time=1.0, event_dpm=-float(base.Pm[k]))
    methods = [("LHS, K=6", dict(K=6, sampling=fs.LHS)), ("LHS, K=200", dict(K=200, sampling=fs.LHS)),
               ("traditional Monte Carlo", dict(K=6, sampling=fs.SRS_EM))]
    Nmax = args.dn_max
    out = {"study": "dn", "system": "10-machine (39-bus-shaped draws), 3 OU disturbances, T = 60 s, dt = 5 ms",
           "event": {"machine": k, "time_s": 1.0, "dPm": -float(base.Pm[k])},
           "response": "RMS over 60 s of the centre-of-inertia speed deviation (p.u.)", "N_max": Nmax,
           "methods": {}}
    curves = {}
    t0 = time.perf_counter()
    for name, kw in methods:
        E = np.full(Nmax + 1, np.nan)
        V = np.full(Nmax + 1, np.nan)
        for N in range(1, Nmax + 1):
            sc = base.replace(N=N, seed=7919 * N + 17, **kw)
            rrf, _, _ = fmc.simulate_rrf(sc, path="fused", precision="bf16x3", ctx=ctx)
            E[N], V[N] = rrf.cpu().numpy()
        dE = np.full(Nmax + 1, np.nan)
        dV = np.full(Nmax + 1, np.nan)
        for N in range(6, Nmax + 1):
            dE[N] = np.max(E[N - 4:N + 1]) - np.min(E[N - 4:N + 1])
            dV[N] = np.max(V[N - 4:N + 1]) - np.min(V[N - 4:N + 1])
        curves[name] = (E, V, dE, dV)
    mc = curves["traditional Monte Carlo"]
    for name, (E, V, dE, dV) in curves.items():
        hitE = next((N for N in range(6, Nmax + 1) if dE[N] <= mc[2][Nmax]), None)
        hitV = next((N for N in range(6, Nmax + 1) if dV[N] <= mc[3][Nmax]), None)
        out["methods"][name] = {
            "E_RRF_at_Nmax": float(E[Nmax]), "Var_RRF_at_Nmax": float(V[Nmax]),
            "D_E_at_Nmax": float(dE[Nmax]), "D_Var_at_Nmax": float(dV[Nmax]),
            "N_to_reach_MC_D_E": hitE, "N_to_reach_MC_D_Var": hitV,
            "sample_ratio_E": None if hitE is None else Nmax / hitE,
            "sample_ratio_Var": None if hitV is None else Nmax / hitV,
            "D_E": [float(x) for x in dE[6::max(1, Nmax // 100)]],
            "D_Var": [float(x) for x in dV[6::max(1, Nmax // 100)]],
        }
    out["wall_s"] = time.perf_counter() - t0
    print(json.dumps(out))
    ctx.close()
    return 0


def main():
    args = parse()
    if args.study == "dn":
        return run_dn_study(args)
    if args.study == "batch":
        return run_batch_study(args)
    if args.study == "serve":
        return run_serve_study(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.study == "tol":
        return run_tol_study(args)
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
    fmc.set_kernel_policy(args.kernel, ctx=ctx)
    path = args.path
    precision = args.precision or ("f32" if path == "plain" else "bf16x3")
    # weak scaling: every rank simulates `samples` samples, its own block of one
    # design of samples * world samples; the moment sums meet in one all-reduce
    sc = workload(args.samples * world, args.horizon, args.machines, args.disturbances)
    sc = sc.replace(forcing=fs.FORCING_SMOOTH if args.forcing == "smooth" else fs.FORCING_INCREMENTS,
                    correlation=fs.CORR_RANK if args.correlation == "rank" else fs.CORR_NONE)
    n, Nt = sc.n, sc.Nt
    from paper_2007_03847_gb300.distributed import shard_range
    k0, count = shard_range(sc.N, world, rank)
    units_per_step = count * Nt * n

    # L2 is flushed between timed steps by writing a buffer larger than it
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        if world == 1:
            return fmc.simulate(sc, path=path, precision=precision, ctx=ctx)
        S1, S2, shift = fmc.simulate_sums(sc, k0, count, path=path, precision=precision, ctx=ctx)
        dist.all_reduce(S1)
        dist.all_reduce(S2)
        return fmc.moments_from_sums(S1, S2, shift, sc.N, ctx=ctx)

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
    value = sc.N * Nt * n / (ms_per_step / 1e3)

    # roofline of the dominant kernel: FP32 FMA pipe, on the method's own count
    kernel_ms = k_ms / max(1, k_launches)
    stages = 4
    units_per_launch = count * Nt * n
    flops_per_launch = algorithmic_flops_per_machine_step(n, stages) * units_per_launch
    achieved_tflops = flops_per_launch / (kernel_ms / 1e3) / 1e12
    mhz = clk.get("sm_mhz") or (measured_peaks() or {}).get("clocks_under_load", {}).get("sm_mhz_median", 1470.0)
    peak_tflops = sms * 128 * 2 * mhz * 1e6 / 1e12
    # MUFU: 16 lanes per SM and clock; the method's 4 sincos per machine-step as 8 MUFU operations
    mufu_ops = 8.0 * units_per_launch
    mufu_peak = sms * 16 * mhz * 1e6
    impl_ops = implementation_ops_per_sample_step(n, sc.d, stages) * count * Nt
    traffic = profiled_traffic() if (path == "fused" and precision == "bf16x3" and sc.N == (1 << 16)
                                     and Nt == 4000 and n == 10 and world == 1) else None
    roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved_tflops / peak_tflops, "traffic": traffic,
                "algorithmic_bytes": algorithmic_bytes_per_launch(count, n, sc.d, sc.K, Nt, precision == "bf16x3"),
                "kernel": ("simulate_wide_kernel" if n > 16 else "simulate_fused_kernel") if path == "fused"
                          else "simulate_plain_kernel",
                "kernel_ms": kernel_ms,
                "peak_note": f"FP32 FMA pipe, of measured clock: {sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz "
                             f"(median SM clock sampled during the timed region); achieved counts the method's "
                             f"16n+32 FMA per machine-step ({algorithmic_flops_per_machine_step(n, stages):.0f} flop "
                             f"at n={n}) x {units_per_launch} machine-steps per launch / kernel time",
                "mufu_frac": mufu_ops / (kernel_ms / 1e3) / mufu_peak,
                "implementation_frac": 2.0 * impl_ops / (kernel_ms / 1e3) / 1e12 / peak_tflops,
                "implementation_note": f"the kernel's own FP32-pipe operations "
                                       f"({implementation_ops_per_sample_step(n, sc.d, stages):.0f} per sample-step, "
                                       f"sin/cos series and bookkeeping included) against the same peak"}

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
        e2e = {"value": sc.N * Nt * n / e2e_s, "unit": "machine-steps/s", "h2d_bytes_per_step": int(h2d),
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
            "config": {"workload": workload_name(args), "path": path, "precision": precision, "samples_per_gpu": count,
                       "steps_per_sample": Nt, "machines": n, "disturbances": sc.d, "K": sc.K,
                       "l2": "flushed between timed steps (512 MB write)", "gpu": gpu_name, "sms": sms,
                       "kernel_policy": args.kernel},
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
