"""Autotuner for the gridding kernels' tile shape and schedule granularity.

Two granularities decide how the work of a job is cut, and the best choice depends on the grid
size, the supports and the visibility density, so they are measured rather than modelled:

* the origin tile (tile_x, tile_y) is the sort granularity: records are binned by (w-plane,
  tile) and every bin is sorted by footprint origin, so a tile row is a run of origins along
  which a warp slides its accumulators, and the bins are the pieces the schedule hands out.
  Wider tiles give longer runs and fewer, larger bins; taller tiles more rows per bin.
* units_per_cta sets how finely the estimated work is cut into units that the persistent CTAs
  take from a counter: more units even out the CTAs' finishing times, fewer units cut fewer
  bins in two.

Each candidate's context grids the job's own visibilities (or its first rows), optionally
followed by degridding them with the same plan, timed with CUDA events on the current stream.
The search is coordinate-wise (every tile at the default granularity, then every granularity
at the best tile), and the result is cached per geometry and power-of-two size class.
"""
from __future__ import annotations

import math

import torch

from ._abi import WProj

DEFAULT_TILES = ((16, 16), (32, 16), (32, 32), (64, 16), (64, 32), (64, 64))
DEFAULT_UNITS = (3, 4, 6, 8, 12)

_cache: dict = {}


def _key(params: dict, nvis: int, hermitian_pairs: bool, with_degrid: bool, what: str):
    return (what, params["n"], params["n_w"], params["support_min"], params["support_max"], params["oversample"],
            params.get("table", "f32"), int(math.log2(max(nvis, 1))), bool(hermitian_pairs), bool(with_degrid))


def _time_config(params: dict, tile, units: int, u, f, v, w, hermitian_pairs: bool, with_degrid: bool,
                 reps: int) -> float:
    """Median ms of one wp_grid call (plus wp_degrid_last when with_degrid) for one configuration."""
    wp = WProj(**params, tile=tile, units_per_cta=units)
    try:
        wp.make_wkernels()
        grid = torch.empty((wp.n, wp.n), dtype=torch.complex64, device=u.device)
        out = torch.empty(v.shape, dtype=torch.complex64, device=u.device) if with_degrid else None

        def once():
            wp.grid(u, f, v, w, grid=grid, hermitian_pairs=hermitian_pairs, keep_binning=with_degrid)
            if with_degrid:
                wp.degrid_last(grid, vis_out=out)

        once()                                        # warm-up (allocates the context's scratch)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            once()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sorted(ms)[len(ms) // 2]
    finally:
        wp.close()


def _rows(uvw, vis, weight, max_rows):
    nrow = uvw.shape[0] if max_rows is None else min(max_rows, uvw.shape[0])
    w = None if weight is None else weight[:nrow].contiguous()
    return nrow, uvw[:nrow].contiguous(), vis[:nrow].contiguous(), w


def _valid_tile(params: dict, tile) -> bool:
    tx, ty = tile
    return tx * ty <= 4096 and params["n"] % tx == 0 and params["n"] % ty == 0


def tune(params: dict, uvw: torch.Tensor, freq: torch.Tensor, vis: torch.Tensor, weight=None,
         hermitian_pairs: bool = False, tiles=DEFAULT_TILES, units=DEFAULT_UNITS, reps: int = 3,
         max_rows: int | None = None, with_degrid: bool = False, use_cache: bool = True):
    """Returns ({"tile": (tx, ty), "units_per_cta": u}, {(tile, u): median ms}) for
    WProj(**params, tile=..., units_per_cta=...).

    `params` are WProj keyword arguments without `tile` and `units_per_cta`. With `max_rows`, only
    the first rows are timed (a sample of the job); with `with_degrid`, each timing is one
    gridding plus one degridding of the same visibilities with the gridding plan."""
    nrow, u, v, w = _rows(uvw, vis, weight, max_rows)
    key = _key(params, nrow * freq.shape[0], hermitian_pairs, with_degrid, "tile+units")
    if use_cache and key in _cache:
        return _cache[key]
    timings = {}
    u0 = 4 if 4 in units else units[0]             # the library's default
    for tile in tiles:
        if _valid_tile(params, tile):
            timings[(tuple(tile), u0)] = _time_config(params, tile, u0, u, freq, v, w, hermitian_pairs,
                                                      with_degrid, reps)
    if not timings:
        raise ValueError("no tile candidate divides the grid size with at most 4096 origins")
    best_tile = min(timings, key=timings.get)[0]
    for un in units:
        if (best_tile, un) not in timings:
            timings[(best_tile, un)] = _time_config(params, best_tile, un, u, freq, v, w, hermitian_pairs,
                                                    with_degrid, reps)
    tile, un = min(timings, key=timings.get)
    result = ({"tile": tile, "units_per_cta": un}, timings)
    _cache[key] = result
    return result


def tune_tile(params: dict, uvw: torch.Tensor, freq: torch.Tensor, vis: torch.Tensor, weight=None,
              hermitian_pairs: bool = False, candidates=DEFAULT_TILES, reps: int = 3, max_rows: int | None = None,
              use_cache: bool = True):
    """Returns (best_tile, {tile: median ms of one wp_grid call}) at the default schedule
    granularity: the tile-only search of `tune`."""
    nrow, u, v, w = _rows(uvw, vis, weight, max_rows)
    key = _key(params, nrow * freq.shape[0], hermitian_pairs, False, "tile")
    if use_cache and key in _cache:
        return _cache[key]
    timings = {tuple(t): _time_config(params, t, 0, u, freq, v, w, hermitian_pairs, False, reps)
               for t in candidates if _valid_tile(params, t)}
    best = min(timings, key=timings.get)
    _cache[key] = (best, timings)
    return best, timings
