"""Ray-sharded data-parallel training step (host logic; the compute is the library's fused training pass).

The rays of one training batch are independent units (Sec. 3.5: every ray renders and back-propagates on its
own), so a batch of M rays splits over W ranks, each holding a replica of the grid: rank r renders the contiguous
shard shard_bounds(M, r, W) with the hash ids the rays have in the whole batch and the loss normalised by M, so
the ranks' gradient channels sum to the whole batch's gradient.  One all-reduce (sum) of the FP32 gradient
channels is the only exchange; every rank then takes the same optimiser step on identical state.
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence

import torch

from . import _abi as A
from .grid import Grid
from .render import train_step_rays


def shard_bounds(n: int, rank: int, world: int) -> tuple:
    """Contiguous shard [a, b) of rank: the first n % world ranks take one ray more."""
    base, extra = divmod(n, world)
    a = rank * base + min(rank, extra)
    return a, a + base + (1 if rank < extra else 0)


def grad_tensors(grid: Grid) -> Sequence[torch.Tensor]:
    """The grid's FP32 gradient channels (zero-copy views) over its active blocks: what the all-reduce sums."""
    nb = grid.num_blocks
    if grid.rgb_dtype == "f32":
        out = [grid.channel(A.GROUP_GEO, A.KIND_GRAD)[:nb]]
    else:
        out = [grid.channel(A.GROUP_SDF, A.KIND_GRAD)[:nb], grid.channel(A.GROUP_RGB, A.KIND_GRAD)[:nb]]
    if grid.n_sem:
        out.append(grid.channel(A.GROUP_SEM, A.KIND_GRAD)[:nb])
    return out


def all_reduce_grads(grid: Grid) -> None:
    """Sums the gradient channels over the ranks of the default torch.distributed group (NCCL on GPUs)."""
    import torch.distributed as dist
    for t in grad_tensors(grid):
        dist.all_reduce(t, op=dist.ReduceOp.SUM)


def shard_train(grid: Grid, rays: torch.Tensor, t_rgb: torch.Tensor, t_depth: torch.Tensor, rank: int, world: int,
                ray_id0: int = 0, **train_kw) -> tuple:
    """This rank's shard of the batch through the fused training pass: the rays keep the hash ids they have in
    the whole batch and the loss is normalised by the whole batch, so the shards' gradients sum to the batch's.
    Returns the shard [a, b)."""
    n = rays.shape[0]
    a, b = shard_bounds(n, rank, world)
    if b > a:
        train_step_rays(grid, rays[a:b], t_rgb[a:b], t_depth[a:b], ray_id0=ray_id0 + a, norm_rays=n, **train_kw)
    return a, b


def data_parallel_step(grid: Grid, rays: torch.Tensor, t_rgb: torch.Tensor, t_depth: torch.Tensor, rank: int,
                       world: int, reduce: Optional[Callable[[Grid], None]] = None, ray_id0: int = 0,
                       lr: float = 1e-3, **train_kw) -> tuple:
    """One data-parallel training step of the batch (rays, targets), which every rank holds: shard_train,
    `reduce(grid)` (default: all_reduce_grads when world > 1), then the optimiser step.  Returns the shard."""
    a, b = shard_train(grid, rays, t_rgb, t_depth, rank, world, ray_id0=ray_id0, **train_kw)
    if world > 1:
        (reduce or all_reduce_grads)(grid)
    grid.adam_step(lr=lr)
    return a, b
