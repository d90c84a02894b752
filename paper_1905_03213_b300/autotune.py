"""Tile-shape autotuner for the gridding kernels.

The origin tile (tile_x, tile_y) sets the bin granularity of the coordinate sort: the records of
one (w-plane, tile) bin are contiguous, the gridding kernel sorts each chunk of a bin (or of up to
eight sparse bins of one tile row) by footprint origin in shared memory, and a row of a tile is a
run of footprint origins along which the warp slides its accumulators. Wider tiles give longer
runs and fewer, larger bins; taller tiles give more rows per bin. The best shape depends on the
grid size, the supports and the visibility density, so it is measured: each candidate's context
grids the job's own visibilities (or its first rows), timed with CUDA events on the current
stream, and the fastest candidate is kept in a cache keyed by the job's geometry and size class.
"""
from __future__ import annotations

import math

import torch

from ._abi import WProj

DEFAULT_TILES = ((16, 16), (32, 16), (32, 32), (64, 16), (64, 32), (64, 64))

_cache: dict = {}


def _key(params: dict, nvis: int, hermitian_pairs: bool):
    return (params["n"], params["n_w"], params["support_min"], params["support_max"], params["oversample"],
            params.get("table", "f32"), int(math.log2(max(nvis, 1))), bool(hermitian_pairs))


def tune_tile(params: dict, uvw: torch.Tensor, freq: torch.Tensor, vis: torch.Tensor, weight=None,
              hermitian_pairs: bool = False, candidates=DEFAULT_TILES, reps: int = 3, max_rows: int | None = None,
              use_cache: bool = True):
    """Returns (best_tile, {tile: median ms of one wp_grid call}) for WProj(**params, tile=...).

    `params` are WProj keyword arguments without `tile`. With `max_rows`, only the first rows are
    timed (a sample of the job). Results are cached per geometry and power-of-two size class."""
    nrow = uvw.shape[0] if max_rows is None else min(max_rows, uvw.shape[0])
    key = _key(params, nrow * freq.shape[0], hermitian_pairs)
    if use_cache and key in _cache:
        return _cache[key]
    u, v = uvw[:nrow].contiguous(), vis[:nrow].contiguous()
    w = None if weight is None else weight[:nrow].contiguous()
    timings = {}
    for tile in candidates:
        tx, ty = tile
        if tx * ty > 4096 or params["n"] % tx or params["n"] % ty:
            continue
        wp = WProj(**params, tile=tile)
        wp.make_wkernels()
        grid = torch.empty((wp.n, wp.n), dtype=torch.complex64, device=u.device)
        wp.grid(u, freq, v, w, grid=grid, hermitian_pairs=hermitian_pairs)  # warm-up (allocates scratch)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            wp.grid(u, freq, v, w, grid=grid, hermitian_pairs=hermitian_pairs)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        timings[tile] = sorted(ms)[len(ms) // 2]
        wp.close()
    best = min(timings, key=timings.get)
    _cache[key] = (best, timings)
    return best, timings
