"""Batched gridding (wp_batch_create / wp_batch_grid): many jobs of different geometries in one
persistent launch, its CUDA-graph replay, and the tile autotuner.

Every batched result is compared with the same job gridded alone by wp_grid (float32
reductions merge in another order, so grids agree to rounding; the scalars exactly), and
with the float64 oracle for one job.
"""
import numpy as np
import pytest

import oracle
from gpu_cases import make_wproj, oracle_results, peak_rel, random_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


# (grid size, planes, support range, oversampling, rows, channels, Hermitian pairs, weights, seed);
# the fifth job has supports above 16 (two row halves, global lane tables); the last job's
# supports exceed 32, so it runs the baseline kernel outside the fused launch
JOBS = [
    (64, 4, (5, 9), 8, 600, 3, False, True, 31),
    (128, 6, (6, 12), 8, 1500, 2, True, False, 32),
    (256, 8, (7, 14), 4, 2500, 2, False, True, 33),
    (128, 3, (8, 8), 8, 900, 4, True, True, 34),
    (64, 5, (12, 24), 6, 700, 2, False, False, 35),
    (128, 3, (30, 36), 4, 800, 2, False, True, 36),
]


def _make_jobs(torch, table="f32"):
    cases, wps, devs = [], [], []
    for (n, n_w, (smin, smax), os_, nrow, nchan, pairs, weights, seed) in JOBS:
        case = random_case(n=n, nrow=nrow, nchan=nchan, n_w=n_w, s_min=smin, s_max=smax, os_=os_, pairs=pairs,
                           seed=seed)
        if not weights:
            case.weight = None
        cases.append(case)
        wps.append(make_wproj(case, table=table))
        devs.append(to_dev(case))
    return cases, wps, devs


def _batch(W, cases, wps, devs):
    jobs = []
    for case, wp, (uvw, f, vis, wt) in zip(cases, wps, devs):
        jobs.append(dict(wp=wp, uvw=uvw, freq=f, vis=vis, weight=wt if case.weight is not None else None,
                         hermitian_pairs=case.pairs))
    return W.WBatch(jobs)


def test_batch_matches_single_job_calls(torch_cuda):
    torch = torch_cuda
    import paper_1905_03213_b300 as W
    cases, wps, devs = _make_jobs(torch)
    batch = _batch(W, cases, wps, devs)
    assert batch.fused_jobs == len(JOBS) - 1
    outs = batch.grid()
    torch.cuda.synchronize()
    # the same jobs one by one, on separate contexts
    for case, (g, sw, nd), (uvw, f, vis, wt) in zip(cases, outs, devs):
        ref_wp = make_wproj(case)
        g1, sw1, nd1 = ref_wp.grid(uvw, f, vis, wt if case.weight is not None else None, hermitian_pairs=case.pairs)
        e, _ = peak_rel(g.cpu().numpy(), g1.cpu().numpy())
        assert e < 1e-6, e
        assert abs(sw.item() - sw1.item()) <= 1e-12 * abs(sw1.item())
        assert nd.item() == nd1.item()
    # and one job against the float64 oracle
    _, g_ref, _ = oracle_results(cases[1])
    e, _ = peak_rel(outs[1][0].cpu().numpy(), g_ref)
    assert e < 1e-5, e


def test_batch_graph_replay_on_new_data(torch_cuda):
    """A captured batch replays on new visibilities written into the same tensors."""
    torch = torch_cuda
    import paper_1905_03213_b300 as W
    cases, wps, devs = _make_jobs(torch)
    batch = _batch(W, cases, wps, devs)
    graph = batch.capture()
    for (_, _, vis, _) in devs:
        vis.mul_(torch.tensor(0.5 - 0.25j, dtype=torch.complex64, device=vis.device))
    graph.replay()
    torch.cuda.synchronize()
    replayed = [(g.clone(), sw.clone(), nd.clone()) for (g, sw, nd) in batch.outputs]
    eager = batch.grid()
    torch.cuda.synchronize()
    for (g0, sw0, nd0), (g1, sw1, nd1) in zip(replayed, eager):
        e, _ = peak_rel(g0.cpu().numpy(), g1.cpu().numpy())
        assert e < 1e-6, e
        assert sw0.item() == sw1.item() and nd0.item() == nd1.item()


def test_batch_f16_tables(torch_cuda):
    torch = torch_cuda
    import paper_1905_03213_b300 as W
    cases, wps, devs = _make_jobs(torch, table="f16")
    batch = _batch(W, cases, wps, devs)
    outs = batch.grid()
    torch.cuda.synchronize()
    _, g_ref, _ = oracle_results(cases[2])
    e, _ = peak_rel(outs[2][0].cpu().numpy(), g_ref)
    assert e < 1e-3, e


def test_batch_rejects_a_shared_context(torch_cuda):
    torch = torch_cuda
    import paper_1905_03213_b300 as W
    cases, wps, devs = _make_jobs(torch)
    uvw, f, vis, _ = devs[0]
    with pytest.raises(W.WProjError):
        W.WBatch([dict(wp=wps[0], uvw=uvw, freq=f, vis=vis), dict(wp=wps[0], uvw=uvw, freq=f, vis=vis)])


def test_autotune_picks_a_measured_candidate(torch_cuda):
    torch = torch_cuda
    from paper_1905_03213_b300.autotune import tune_tile
    case = random_case(n=256, nrow=3000, nchan=2, n_w=6, s_min=6, s_max=12)
    uvw, f, vis, wt = to_dev(case)
    p = case.prm
    params = dict(n=p.n, cell=p.cell, n_w=p.n_w, w_max=p.w_max, support_min=p.s_min, support_max=p.s_max,
                  oversample=p.os, screen_m=p.m)
    cands = ((16, 16), (32, 32), (64, 16))
    best, timings = tune_tile(params, uvw, f, vis, wt, candidates=cands, reps=2, use_cache=False)
    assert best in cands and set(timings) == set(cands) and all(t > 0 for t in timings.values())
    g_best, _, _ = make_wproj(case, tile=best).grid(uvw, f, vis, wt)
    _, g_ref, _ = oracle_results(case)
    e, _ = peak_rel(g_best.cpu().numpy(), g_ref)
    assert e < 1e-5, e


def test_autotune_tile_and_schedule_granularity(torch_cuda):
    torch = torch_cuda
    from paper_1905_03213_b300.autotune import tune
    case = random_case(n=256, nrow=3000, nchan=2, n_w=6, s_min=6, s_max=12, pairs=True)
    uvw, f, vis, wt = to_dev(case)
    p = case.prm
    params = dict(n=p.n, cell=p.cell, n_w=p.n_w, w_max=p.w_max, support_min=p.s_min, support_max=p.s_max,
                  oversample=p.os, screen_m=p.m)
    tiles, units = ((16, 16), (32, 32)), (2, 4, 16)
    best, timings = tune(params, uvw, f, vis, wt, hermitian_pairs=True, tiles=tiles, units=units, reps=2,
                         with_degrid=True, use_cache=False)
    assert best["tile"] in tiles and best["units_per_cta"] in units
    # every tile at the default granularity, then every granularity at the best tile
    assert set(timings) >= {(t, 4) for t in tiles} | {(min(timings, key=timings.get)[0], u) for u in units}
    assert all(t > 0 for t in timings.values())
    _, g_ref, _ = oracle_results(case)
    for un in (1, best["units_per_cta"], 64):
        wp = make_wproj(case, tile=best["tile"], units_per_cta=un)
        g, _, _ = wp.grid(uvw, f, vis, wt, hermitian_pairs=True)
        e, _ = peak_rel(g.cpu().numpy(), g_ref)
        assert e < 1e-5, (un, e)
