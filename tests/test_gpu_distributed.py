"""The multi-rank path through the library: two gloo ranks, each a process with
its own context on the one GPU, simulate their blocks of one design with
simulate_distributed (the library's block sums, one all-reduce on the host), and
rank 0's moments match a single-process run and the oracle.  The ranks' kernels
never wait on one another: the only exchange is the host-side all-reduce."""
import os
import socket

import numpy as np
import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _case():
    import fmc_synth as fs
    return fs.multimachine_case(n=6, d=2, K=30, T=0.4, dt=0.005, N=777, seed=8)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import paper_2007_03847_gb300 as fmc
    from paper_2007_03847_gb300.distributed import simulate_distributed
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ctx = fmc.Context(0)
    mean, var = simulate_distributed(_case(), ctx=ctx)
    fmc.device_status(ctx)
    if rank == 0:
        np.save(out + ".mean.npy", mean.cpu().numpy())
        np.save(out + ".var.npy", var.cpu().numpy())
    dist.barrier()
    ctx.close()
    dist.destroy_process_group()


def test_two_ranks_equal_single_process(orc, tmp_path):
    fmc = need_gpu()
    import torch.multiprocessing as mp
    out = str(tmp_path / "res")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    sc = _case()
    m2, v2 = np.load(out + ".mean.npy"), np.load(out + ".var.npy")
    m1, v1 = fmc.simulate(sc)
    m1, v1 = m1.cpu().numpy(), v1.cpu().numpy()
    ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), nthreads=8)
    n = sc.n
    for sl in (slice(0, n), slice(n, 2 * n)):
        sd = float(np.sqrt(np.max(v1[:, sl])))
        # the same samples summed in another grouping: FP32 rounding on the spread's scale
        assert np.max(np.abs(m2[:, sl] - m1[:, sl])) <= 1e-6 * sd + 1e-15
        assert np.allclose(v2[:, sl], v1[:, sl], rtol=2e-6, atol=1e-18)
        scale = np.max(np.sqrt(ref["mean"][:, sl] ** 2 + ref["var"][:, sl]))
        assert np.max(np.abs(m2[:, sl] - ref["mean"][:, sl])) <= 1e-5 * scale
        assert np.max(np.abs(v2[:, sl] - ref["var"][:, sl])) <= 1e-5 * np.max(np.abs(ref["var"][:, sl]))
