"""Batch sharding of one system across GPUs (one process and one context per
GPU): each rank's context processes its shard of the unique occupied batches
(the library's "shard_count"/"shard_index" parameters) and one all-reduce (sum)
of the outputs gives the unsharded result, since the triples residual, the
Jacobian transformations and the multiplier transformation are sums of
per-batch terms (Sec. 3, the restricted loop over i >= j >= k)."""
from __future__ import annotations


def use_shard(ctx, rank: int, world: int):
    """Point the context at shard `rank` of `world` (batches from mlcc3_shard_batches)."""
    ctx.set_param("shard_count", world)
    ctx.set_param("shard_index", rank)


def allreduce_sum(tensors, group=None):
    """Sum the partial outputs of every rank in place (torch.distributed, one
    collective per tensor, on the tensors' own device: NCCL for CUDA tensors)."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def sharded_jacobian_right(ctx, rank, world, omega, R1, R2, rho1, rho2, group=None):
    """rho = A R of one system, sharded by batches across the ranks."""
    use_shard(ctx, rank, world)
    ctx.jacobian_right(omega, R1, R2, rho1, rho2)
    return allreduce_sum([rho1, rho2], group)
