"""Data-parallel M2M steps over particle shards (thin driver over the C-ABI).

One model's particles are split into contiguous shards, one library context
per shard (each holding the whole model's weights for its particles).  The
push, the scatter and the weight update of a particle need that particle
alone (Section 2), so each step exchanges only the observable totals and the
entropy / weight sums (and, at a prior recompute, the (E, L_z) range and the
prior-cell sums and counts): every shard scatters, the exchange buffers are
summed (the range: minimum) over shards, and every shard forms the residual
from the sums.  The totals and cell sums are integers (FP32C fixed point at
the whole model's scale), so the sums do not depend on their order and a
sharded model takes exactly the steps of the model in one context.

The collective is pluggable: ``DistReduce`` uses ``torch.distributed``
all-reduce (NCCL between GPUs, gloo on CPU), ``LocalReduce`` sums the
buffers of several shards held by one process (on one device).
"""
from dataclasses import dataclass

import numpy as np


def shard_bounds(n, world, rank):
    """[lo, hi) of shard `rank` of `world` contiguous shards of n particles
    (sizes differ by at most one)."""
    return (n * rank) // world, (n * (rank + 1)) // world


@dataclass
class ShardBuffers:
    """The exchange buffers of one shard (device tensors)."""
    totals: object        # int64[nobs]
    stats: object         # float64[2]
    rng: object           # float64[3]
    cell_sums: object     # int64[ncells]
    cell_counts: object   # int32[ncells]

    @classmethod
    def alloc(cls, nobs, ncells, device):
        import torch
        z = dict(device=device)
        return cls(torch.zeros(nobs, dtype=torch.int64, **z), torch.zeros(2, dtype=torch.float64, **z),
                   torch.zeros(3, dtype=torch.float64, **z), torch.zeros(max(1, ncells), dtype=torch.int64, **z),
                   torch.zeros(max(1, ncells), dtype=torch.int32, **z))


class DistReduce:
    """Sum / minimum over the ranks of a torch.distributed process group."""

    def __init__(self, dist, group=None):
        self.dist, self.group = dist, group

    def sum(self, ts):
        for t in ts:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)

    def min(self, ts):
        for t in ts:
            self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)


class LocalReduce:
    """Sum / minimum over several shards' buffers held by this process."""

    def sum(self, ts):
        acc = ts[0].clone()
        for t in ts[1:]:
            acc += t
        for t in ts:
            t.copy_(acc)

    def min(self, ts):
        acc = ts[0].clone()
        for t in ts[1:]:
            acc = acc.minimum(t)
        for t in ts:
            t.copy_(acc)


def ncells_of(prior):
    if prior is None or prior.kind == "flat":
        return 0
    return prior.nE * prior.nL + (1 if prior.kind == "e_lc" else 0)


def make_shard(problem, world, rank, precision="fp32c", device="cuda:0"):
    """A context over shard `rank` of the problem's particles, at the whole
    model's fixed-point scale, and its exchange buffers."""
    from . import m2m as B
    lo, hi = shard_bounds(problem.n, world, rank)
    ctx = B.m2m_init(precision, problem.pos[:, lo:hi], problem.vel[:, lo:hi], problem.w0[lo:hi],
                     problem.what0[lo:hi], problem.potential, problem.obs, B.params_of(problem), problem.prior,
                     problem.Y, problem.sigma, device)
    ctx.m2m_shard_init(problem.n, float(np.sum(problem.w0)))
    return ctx, ShardBuffers.alloc(ctx.nobs, ncells_of(problem.prior), device)


def step(shards, reduce, push=True):
    """One step of every shard held by this process (push = False: the
    initial scatter, Delta~ := Delta).  `shards`: list of (context, buffers);
    `reduce`: the collective over all shards of the model."""
    due = [ctx.m2m_shard_scatter(push, b.totals, b.stats, b.rng) for ctx, b in shards]
    reduce.sum([b.totals for _, b in shards])
    reduce.sum([b.stats for _, b in shards])
    if due[0]:
        reduce.min([b.rng for _, b in shards])
    for ctx, b in shards:
        ctx.m2m_shard_residual(b.totals, b.stats)
    if due[0]:
        for ctx, b in shards:
            ctx.m2m_shard_prior_cells(b.rng, b.cell_sums, b.cell_counts)
        reduce.sum([b.cell_sums for _, b in shards])
        reduce.sum([b.cell_counts for _, b in shards])
        for ctx, b in shards:
            ctx.m2m_shard_prior_finish(b.cell_sums, b.cell_counts)
    return due[0]


def start(shards, reduce):
    """The initial scatter of a sharded model (the smoothed residuals start
    from the whole model's observables)."""
    step(shards, reduce, push=False)
