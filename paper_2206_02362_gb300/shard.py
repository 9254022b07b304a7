"""Shot sharding across ranks (one process per GPU).

Shots are independent (Barnier et al., Computational aspects: each GPU
simulates one shot over the full domain, no domain decomposition), so a rank
owns a contiguous block of shots.  Data-space outputs stay on their rank; the
model-space outputs of the adjoint operators (B* d, B~* d, T* d, gradient) are
sums over shots and need one sum all-reduce per call -- the only exchange step.
"""
from __future__ import annotations


def shard(nshot: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of the shots owned by `rank`: contiguous blocks, sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or nshot < 0:
        raise ValueError(f"bad shard request nshot={nshot} world={world} rank={rank}")
    base, extra = divmod(nshot, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def allreduce_model(tensor, group=None):
    """Sums a model-space output (image, gradient) over all ranks in place."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor


def rank_step(apply, nshot: int, world: int, rank: int, group=None):
    """One data-parallel step of a model-space operator over `nshot` shots on `world` ranks: this rank
    applies ``apply(start, stop)`` -- the operator (B~*, B*, T*, the gradient ...) over its contiguous
    block of shots [start, stop) -- and the model-space output it returns (a torch tensor) is summed over
    all ranks in place (world = 1: no exchange, whatever process group exists).  The same function drives
    the GPU ranks (``apply`` calls libfwime on the rank's device) and the CPU tests (``apply`` calls the
    oracle, gloo all-reduce)."""
    start, stop = shard(nshot, world, rank)
    out = apply(start, stop)
    return allreduce_model(out, group) if world > 1 else out
