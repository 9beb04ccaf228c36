"""Sharding one scene's nested-SGD iteration over several devices.

The sample space of an iteration (views x pixels x samples x sets) is
embarrassingly parallel.  Each rank takes a contiguous range of the
concatenated views' pixels and traces both the residual and the derivative
samples of those pixels (so a pixel's two independent estimates, Sec. 3.3,
never cross ranks); the one exchange per iteration is a sum of the S x 10
gradient and the loss.  Every rank then applies the same Adam step to the
same summed gradient, so the parameters stay identical without a broadcast.

The compute callable is supplied by the caller: ``Tracer.loss_grad_shard``
on a GPU rank.  Both the loss and the gradient must be normalised by the
total pixel count, so the shards add up to the unsharded result.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(n_pix: int, world: int, rank: int):
    """Contiguous, balanced pixel range [begin, begin + count) of a rank."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, rem = divmod(n_pix, world)
    begin = rank * base + min(rank, rem)
    count = base + (1 if rank < rem else 0)
    return begin, count


def sharded_loss_grad(compute, n_pix: int, n_seg: int, group=None, device=None):
    """compute(begin, count, n_total) -> (loss: float, grad: (n_seg, 10)
    tensor or array).  Returns the all-reduced (loss, grad) as (float,
    float64 tensor on ``device``)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    begin, count = shard_range(n_pix, world, rank)
    if count > 0:
        loss, grad = compute(begin, count, n_pix)
        g = torch.as_tensor(grad).to(device=device, dtype=torch.float64).reshape(-1)
    else:
        loss = 0.0
        g = torch.zeros(n_seg * 10, dtype=torch.float64, device=device)
    buf = torch.cat([g, torch.tensor([float(loss)], dtype=torch.float64, device=g.device)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return float(buf[-1].item()), buf[:-1].reshape(n_seg, 10)


def sharded_step(tracer, opts, adam, iteration: int, group=None):
    """One sharded iteration on GPU ranks: local shard on this rank's
    device, NCCL sum, identical Adam step everywhere.  Returns the loss."""
    dev = tracer.device

    def compute(begin, count, n_total):
        return tracer.loss_grad_shard(opts, iteration, begin, count, n_total)

    loss, grad = sharded_loss_grad(compute, tracer.n_pix, tracer.n_seg, group, dev)
    tracer.adam_step(adam, grad.to(torch.float32).contiguous())
    return loss
