"""Measured launch shapes of the fused path.

For buckets of machine count, disturbance count and sample count, every
candidate shape -- the kernel (per-sample up to 16 machines; split with the
network sums on the FP32 pipes or on the tensor cores, the latter from 13
machines), the resident CTAs per SM and the time chunk -- is timed with CUDA
events on a seeded
system of the bucket's largest size, and the fastest per machine-step becomes a
launch rule (``fmc_set_launch_rules``).  The table is cached per GPU model and
SM count under ``tuning/`` and applied to every new context on that GPU.

    python -m paper_2007_03847_gb300.autotune [--quick]
"""
from __future__ import annotations

import json
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_DIR = os.path.join(HERE, "tuning")

# the large-system buckets follow the tensor-core kernel's layouts: two warps per
# sample with 10 and 13 slots (17..20, 21..26), then four with 7, 10, 13 slots
N_BUCKETS = [(1, 4), (5, 10), (11, 16), (17, 20), (21, 26), (27, 32), (33, 40), (41, 52)]
D_BUCKETS = [(1, 2), (3, 4), (5, 8)]
SAMPLE_BUCKETS = [(1, 32767), (32768, 1 << 30)]


def table_path(name: str, sms: int) -> str:
    return os.path.join(TUNING_DIR, re.sub(r"[^A-Za-z0-9]+", "_", name).strip("_") + f"_{sms}sm.json")


def candidates(n: int):
    """(kernel, max_ctas, TC) triples; 0 = the library's own choice."""
    from . import KERNEL_PER_SAMPLE, KERNEL_SPLIT, KERNEL_SPLIT_TC
    out = []
    if n <= 16:
        for mc in (0, 4, 2, 1):
            for tc in (0, 32, 16):
                out.append((KERNEL_PER_SAMPLE, mc, tc))
        out.append((KERNEL_SPLIT, 0, 0))
        out.append((KERNEL_SPLIT, 0, 32))
    else:
        out.append((KERNEL_SPLIT, 0, 0))
        out.append((KERNEL_SPLIT, 0, 64))
    if n >= 13:
        for tc in (0, 32, 16):
            out.append((KERNEL_SPLIT_TC, 0, tc))
    return out


def _time(sc, ctx, reps: int) -> float:
    import torch

    from . import simulate
    simulate(sc, ctx=ctx)  # warm-up (workspace, first launch)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        simulate(sc, ctx=ctx)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune(ctx=None, quick: bool = False, horizon: float = 2.0, reps: int = 2):
    """Measures every bucket's candidates; returns (rules, measurements)."""
    import fmc_synth as fs

    from . import Context, FastMCError, set_launch_rules
    ctx = ctx or Context(0)
    set_launch_rules([], ctx=ctx)
    rules, measured = [], []
    n_buckets = N_BUCKETS[1:2] + N_BUCKETS[3:4] + N_BUCKETS[-1:] if quick else N_BUCKETS
    for nb in n_buckets:
        for db in D_BUCKETS:
            for sb in SAMPLE_BUCKETS:
                n, d = min(nb[1], 50), db[1]
                N = 8192 if sb[1] < 32768 else 65536
                sc = fs.multimachine_case(n=n, d=d, K=100, T=horizon, dt=0.005, N=N, seed=11,
                                          system_seed=1000 + n * 10 + d)
                units = N * sc.Nt * n
                best = None
                for kernel, mc, tc in candidates(n):
                    rule = dict(n_min=nb[0], n_max=nb[1], d_min=db[0], d_max=db[1], N_min=sb[0], N_max=sb[1],
                                kernel=kernel, max_ctas=mc, TC=tc)
                    set_launch_rules([rule], ctx=ctx)
                    try:
                        ms = _time(sc, ctx, reps)
                    except FastMCError:
                        continue
                    rate = units / (ms / 1e3)
                    measured.append(dict(rule, system=dict(n=n, d=d, N=N, Nt=sc.Nt), ms=ms, machine_steps_per_s=rate))
                    if best is None or rate > best[1]:
                        best = (rule, rate)
                if best is not None:
                    rules.append(best[0])
    set_launch_rules(rules, ctx=ctx)
    return rules, measured


def save(rules, measured, name: str, sms: int) -> str:
    os.makedirs(TUNING_DIR, exist_ok=True)
    path = table_path(name, sms)
    with open(path, "w") as f:
        json.dump({"gpu": name, "sms": sms, "rules": rules, "measured": measured}, f, indent=1)
    return path


def apply_cached(ctx) -> bool:
    """Applies the cached table of the context's GPU, if there is one."""
    from . import set_launch_rules
    sms, name = ctx.info()
    path = table_path(name, sms)
    if not os.path.exists(path):
        return False
    with open(path) as f:
        rules = json.load(f).get("rules", [])
    set_launch_rules(rules, ctx=ctx)
    return True


def main():
    import argparse

    from . import Context, build
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="two machine buckets only")
    args = ap.parse_args()
    build()
    ctx = Context(0)
    sms, name = ctx.info()
    rules, measured = tune(ctx, quick=args.quick)
    print(save(rules, measured, name, sms))
    ctx.close()


if __name__ == "__main__":
    main()
