"""Host logic of the multi-GPU path with gloo ranks on the CPU (world size 2):
the sample blocks cover the design exactly once, and the all-reduced shifted
sums of the blocks give the moments of the whole design.  The per-block sums
come from the FP64 oracle (no GPU here)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2007_03847_gb300.distributed import allreduce_sums, shard_range


def test_shard_ranges_cover_design_once():
    for N in [1, 2, 3, 7, 1000, 65537]:
        for world in [1, 2, 3, 4, 8]:
            if world > N:
                continue
            seen = []
            for r in range(world):
                k0, c = shard_range(N, world, r)
                seen.extend(range(k0, k0 + c))
            assert seen == list(range(N))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import fmc_synth as fs
    import oracle
    sc = fs.multimachine_case(n=4, d=2, K=12, T=0.5, dt=0.01, N=37, seed=3)
    k0, count = shard_range(sc.N, world, rank)
    zeta = oracle.lhs_sample(sc.seed, sc.N, sc.M, k0=k0, count=count)
    r = oracle.simulate(sc, zeta, want_traj=True, want_moments=False)
    shift = np.concatenate([r["delta0"], np.zeros(sc.n)])
    x = r["traj"] - shift
    S1 = torch.from_numpy(x.sum(axis=0))
    S2 = torch.from_numpy((x * x).sum(axis=0))
    allreduce_sums(S1, S2)
    if rank == 0:
        N = sc.N
        mean = shift + S1.numpy() / N
        var = (S2.numpy() - S1.numpy() ** 2 / N) / (N - 1)
        np.save(out + ".mean.npy", mean)
        np.save(out + ".var.npy", var)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_moments_equal_single_process(tmp_path):
    import fmc_synth as fs
    import oracle
    out = str(tmp_path / "res")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    sc = fs.multimachine_case(n=4, d=2, K=12, T=0.5, dt=0.01, N=37, seed=3)
    zeta = oracle.lhs_sample(sc.seed, sc.N, sc.M)
    r = oracle.simulate(sc, zeta, want_traj=True)
    m2, v2 = oracle.moments_twopass(r["traj"])
    assert np.allclose(np.load(out + ".mean.npy"), m2, rtol=1e-12, atol=1e-15)
    assert np.allclose(np.load(out + ".var.npy"), v2, rtol=1e-9, atol=1e-20)
