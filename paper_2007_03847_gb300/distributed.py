"""Multi-GPU orchestration: one process per GPU, each simulating its own block
of samples of one global Latin hypercube design; the only exchange is the sum
of the per-block shifted moment sums (one all-reduce of 2 (Nt+1) 2n FP64).

The design is stateless (every sample's coefficients follow from the seed and
its index), so the blocks need no communication before the exchange.
"""
from __future__ import annotations


def shard_range(N: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block of samples of rank `rank`: (k0, count); blocks differ in
    size by at most one sample and cover [0, N) exactly once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(N, world)
    k0 = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return k0, count


def allreduce_sums(S1, S2, group=None):
    """Sum the shifted sums over all ranks in place (NCCL on CUDA tensors; with a
    gloo group CUDA tensors pass through host copies)."""
    import torch.distributed as dist
    if S1.is_cuda and dist.get_backend(group) == "gloo":
        h1, h2 = S1.cpu(), S2.cpu()
        dist.all_reduce(h1, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(h2, op=dist.ReduceOp.SUM, group=group)
        S1.copy_(h1)
        S2.copy_(h2)
        return S1, S2
    dist.all_reduce(S1, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(S2, op=dist.ReduceOp.SUM, group=group)
    return S1, S2


def simulate_distributed(scenario, path="fused", precision=None, ctx=None, group=None):
    """All ranks: Algorithm 1 over the N samples of `scenario`, split across the
    ranks of the default process group; returns (mean, var) on every rank."""
    import torch.distributed as dist

    from . import moments_from_sums, simulate_sums
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    k0, count = shard_range(scenario.N, world, rank)
    S1, S2, shift = simulate_sums(scenario, k0, count, path=path, precision=precision, ctx=ctx)
    allreduce_sums(S1, S2, group)
    return moments_from_sums(S1, S2, shift, scenario.N, ctx=ctx)
