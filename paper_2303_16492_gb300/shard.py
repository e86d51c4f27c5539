"""Sample-sharded TR-BRSGD across ranks (one process per GPU).

The estimators of Eq. S_gradient and Eq. S_hessian are sums over the sampled
fibers, so an iteration shards over its samples: every rank holds X and the
cores, draws the same mode and Philox counters, computes the partial sums of
its own samples in the library's kernels (trsgd_step_partial), and the ranks
exchange them once per iteration.  The exchange is an all-gather of every
rank's FP32 partials in rank order, followed by a sum in increasing index
inside the library's update kernel (trsgd_step_apply): the reduction order is
fixed, so every rank applies the identical update, and the result equals the
single-device iteration bit for bit.

This module only moves buffers between ranks; all arithmetic of the method
runs in the CUDA library.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def gather_in_rank_order(local: torch.Tensor, world: int, group=None) -> torch.Tensor:
    """All-gather of equal-size 1-D buffers, concatenated in rank order
    (works on NCCL device tensors and on gloo CPU tensors)."""
    if world == 1:
        return local
    out = torch.empty(world * local.numel(), dtype=local.dtype, device=local.device)
    if local.device.type == "cuda":
        dist.all_gather_into_tensor(out, local, group=group)
    else:
        parts = list(out.chunk(world))
        dist.all_gather(parts, local, group=group)
    return out


def unit_ranges(total: int, unit: int, world: int, rank: int):
    """The units of a batch of `total` samples dealt in contiguous runs:
    rank r gets units [r U / world, (r + 1) U / world) of U = ceil(total /
    unit) (the rule of trsgd_shard_plan); returns (first sample, end sample,
    units, max units over ranks)."""
    U = (total + unit - 1) // unit
    u0, u1 = U * rank // world, U * (rank + 1) // world
    return min(u0 * unit, total), min(u1 * unit, total), u1 - u0, (U + world - 1) // world


class ShardedSolver:
    """One rank's view of a sample-sharded solver over an ``api.Solver``
    handle on the whole-GPU path (every rank holds identical X and cores)."""

    def __init__(self, solver, rank: int | None = None, world: int | None = None, group=None):
        self.solver = solver
        self.group = group
        self.rank = dist.get_rank(group) if rank is None else rank
        self.world = dist.get_world_size(group) if world is None else world
        self._buf = {}

    def _buffer(self, name: str, numel: int, device):
        b = self._buf.get(name)
        if b is None or b.numel() < numel:
            b = torch.empty(numel, dtype=torch.float32, device=device)
            self._buf[name] = b
        return b[:numel]

    def step(self, t: int):
        s = self.solver
        plan = s.shard_plan(t, self.rank, self.world)
        dev = s.cores[0][0].device
        g = self._buffer("g", plan.gsplits_max * plan.gelems, dev)
        h = self._buffer("h", plan.hsplits_max * plan.helems, dev) if plan.helems else None
        s.step_partial(t, plan, g, h)
        cur = torch.cuda.current_stream(dev)
        cur.wait_stream(s.stream)        # the collective runs on torch's current stream
        G = gather_in_rank_order(g, self.world, self.group)
        H = gather_in_rank_order(h, self.world, self.group) if h is not None else None
        s.stream.wait_stream(cur)
        s.step_apply(t, G, self.world * plan.gsplits_max, H, self.world * plan.hsplits_max if h is not None else 0)
        return plan
