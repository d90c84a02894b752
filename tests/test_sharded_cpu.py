"""The multi-process split of gridding (row blocks per rank, grid sum-reduced onto the root;
degridding with the grid broadcast), run as two gloo processes on CPU with the float64 oracle
as each rank's gridder, against the single-process oracle on all rows."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
from oracle import wproj
import synth

from paper_1905_03213_b300.sharded import degrid_sharded, grid_sharded, row_range


@pytest.mark.parametrize("nrow,world", [(0, 1), (1, 2), (10, 3), (21060, 2), (21061, 4), (7, 8)])
def test_row_range_partitions_rows_in_order(nrow, world):
    spans = [row_range(nrow, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == nrow
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert a1 == b0 and a0 <= a1
    sizes = [b - a for a, b in spans]
    assert max(sizes) - min(sizes) <= 1


def _case():
    cfg = synth.config("parity")
    ob = synth.observe(cfg, rows=3000)
    prm = oracle.Params(cfg.n, cfg.cell, cfg.n_w, ob.w_max, cfg.s_min, cfg.s_max, cfg.oversample)
    wt = (0.5 + np.random.default_rng(9).random(ob.weight.shape)).astype(np.float32)
    return prm, ob.uvw, ob.freqs, ob.vis, wt


def _oracle_grid_fn(prm, freqs, tabs, pairs):
    import torch

    def fn(uvw, vis, wt):
        crd = oracle.coords(uvw.numpy(), freqs, prm, hermitian_pairs=pairs)
        c = wproj.gridded_values(vis.numpy(), None if wt is None else wt.numpy(), crd)
        g = oracle.grid(crd, c, tabs, prm)
        sw = oracle.sum_weights(None if wt is None else wt.numpy(), crd)
        return (torch.from_numpy(g), torch.tensor([sw], dtype=torch.float64),
                torch.tensor([int((~crd["keep"]).sum())], dtype=torch.int64))
    return fn


def _worker(rank, world, port, out_dir, pairs):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        prm, uvw, freqs, vis, wt = _case()
        tabs, _ = oracle.wkernels(prm)
        g, sw, nd = grid_sharded(_oracle_grid_fn(prm, freqs, tabs, pairs), torch.from_numpy(uvw),
                                 torch.from_numpy(vis), torch.from_numpy(wt), root=0)
        if rank == 0:
            np.save(os.path.join(out_dir, "grid.npy"), g.numpy())
            np.save(os.path.join(out_dir, "scalars.npy"), np.array([sw.item(), nd.item()]))
        # degridding: rank 0 holds the summed grid; the others start from zeros
        G = g if rank == 0 else torch.zeros_like(g)

        def degrid_fn(uvw_rows, grid):
            crd = oracle.coords(uvw_rows.numpy(), freqs, prm)
            return oracle.degrid(crd, grid.numpy(), tabs, prm).reshape(uvw_rows.shape[0], len(freqs))

        r0, r1, v = degrid_sharded(degrid_fn, torch.from_numpy(uvw), G, root=0)
        np.save(os.path.join(out_dir, f"degrid_{rank}.npy"), np.concatenate([[r0, r1], v.ravel().view(np.float64)]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("pairs", [False, True])
def test_two_rank_split_matches_single_process(pairs):
    import torch.multiprocessing as mp
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_worker, args=(world, _free_port(), d, pairs), nprocs=world, join=True,
                           start_method="spawn")
        g = np.load(os.path.join(d, "grid.npy"))
        sw, nd = np.load(os.path.join(d, "scalars.npy"))
        parts = [np.load(os.path.join(d, f"degrid_{r}.npy")) for r in range(world)]
    prm, uvw, freqs, vis, wt = _case()
    tabs, _ = oracle.wkernels(prm)
    crd = oracle.coords(uvw, freqs, prm, hermitian_pairs=pairs)
    ref = oracle.grid(crd, wproj.gridded_values(vis, wt, crd), tabs, prm)
    # float64 sums of the two ranks' grids in another order than the single pass
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert sw == pytest.approx(oracle.sum_weights(wt, crd), rel=1e-13)
    assert nd == int((~crd["keep"]).sum())
    # degridding of the summed grid: the ranks' row blocks put together equal one pass
    crd1 = oracle.coords(uvw, freqs, prm)
    ref_v = oracle.degrid(crd1, ref, tabs, prm).reshape(vis.shape)
    got = np.zeros(vis.shape, np.complex128)
    for p in parts:
        r0, r1 = int(p[0]), int(p[1])
        got[r0:r1] = p[2:].view(np.complex128).reshape(r1 - r0, -1)
    np.testing.assert_allclose(got, ref_v, rtol=0, atol=1e-12 * np.abs(ref_v).max())
