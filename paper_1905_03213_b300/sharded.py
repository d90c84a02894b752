"""Gridding one observation across several processes (one GPU each): the paper's split.

The paper spreads the visibilities over MPI ranks by rows (time ranges, Sec. 2.1; Fig. 1 and
Fig. 2), has every rank grid its share into a private uv grid, sums the grids onto the master
and runs the IFFT there. Here the ranks are torch.distributed processes:

  * `row_range(nrow, rank, world)`: the rows of one rank, a contiguous block (rows are time-major
    in a Measurement Set, so a block is a time range, as in the paper);
  * `grid_sharded`: every rank grids its block into its own grid, then the N x N complex64 grids
    and the weight sums are sum-reduced onto `root` (the only exchange of the method);
  * `degrid_sharded`: the adjoint: the grid is broadcast from `root` and every rank degrids
    its own rows (no reduction).

The gridding itself is a callable, so the same partition and exchange run with the library's
CUDA gridding on GPUs (`WProj.grid`, NCCL) and with any other gridder on CPU processes (gloo).
Only the exchange goes through torch.distributed; no kernel reads another rank's memory.
"""
from __future__ import annotations

from typing import Callable


def row_range(nrow: int, rank: int, world: int) -> tuple[int, int]:
    """[r0, r1) of rank `rank`: world nearly equal contiguous blocks (the first nrow % world
    ranks get one row more), in rank order, covering every row exactly once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(int(nrow), world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def grid_sharded(grid_fn: Callable, uvw, vis, weight=None, *, root: int = 0, group=None):
    """Grids this rank's rows and sum-reduces the result onto `root`.

    grid_fn(uvw_rows, vis_rows, weight_rows) -> (grid, sum_w, n_dropped) grids one block of rows
    (full arrays are passed in and sliced here; weight may be None). grid is an [N, N] complex
    tensor, sum_w and n_dropped one-element tensors, all on the device the process group's
    backend reduces on (CUDA for NCCL, CPU for gloo).
    Returns (grid, sum_w, n_dropped): the totals over all ranks on `root`, this rank's own
    partial results elsewhere.
    """
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    r0, r1 = row_range(uvw.shape[0], rank, world)
    g, sw, nd = grid_fn(uvw[r0:r1], vis[r0:r1], None if weight is None else weight[r0:r1])
    dst = dist.get_global_rank(group, root) if group is not None else root
    # complex tensors travel as their real view; scalars as float64 / int64
    dist.reduce(torch.view_as_real(g), dst=dst, op=dist.ReduceOp.SUM, group=group)
    dist.reduce(sw, dst=dst, op=dist.ReduceOp.SUM, group=group)
    dist.reduce(nd, dst=dst, op=dist.ReduceOp.SUM, group=group)
    return g, sw, nd


def degrid_sharded(degrid_fn: Callable, uvw, grid, *, root: int = 0, group=None):
    """Broadcasts `grid` from `root` (in place) and degrids this rank's rows:
    degrid_fn(uvw_rows, grid) -> visibilities of those rows. Returns (r0, r1, vis_rows)."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    src = dist.get_global_rank(group, root) if group is not None else root
    dist.broadcast(torch.view_as_real(grid), src=src, group=group)
    r0, r1 = row_range(uvw.shape[0], rank, world)
    return r0, r1, degrid_fn(uvw[r0:r1], grid)


def wproj_grid_fn(wp, freq, hermitian_pairs: bool = False):
    """grid_fn for `grid_sharded` that grids with the library on this rank's GPU."""
    def fn(uvw_rows, vis_rows, weight_rows):
        return wp.grid(uvw_rows.contiguous(), freq, vis_rows.contiguous(),
                       None if weight_rows is None else weight_rows.contiguous(), hermitian_pairs=hermitian_pairs)
    return fn


def wproj_degrid_fn(wp, freq):
    """degrid_fn for `degrid_sharded` that degrids with the library on this rank's GPU."""
    def fn(uvw_rows, grid):
        return wp.degrid(uvw_rows.contiguous(), freq, grid)
    return fn
