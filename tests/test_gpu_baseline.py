"""The paper's own GPU gridding scheme (Sec. 2.2, Fig. 2), kept as a comparison variant:
wp_baseline_order (Eq. 5 baseline index, Eq. 6 start indices, rows grouped by baseline and
time-ordered) and wp_grid_baseline (one thread per support tap walking a baseline's samples).

The ordering is integer work and compared bit for bit with the oracle's; the grid is compared
with the float64 oracle's grid (peak-relative 1e-6, as the binned kernels) and with wp_grid on
the same context (the same stored tables, float32 sums in another order).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_cases import make_wproj, oracle_results, parity_case, peak_rel, random_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _order_on_gpu(torch, wp, a1, a2, n_ant):
    t1 = torch.from_numpy(np.ascontiguousarray(a1, dtype=np.int32)).cuda()
    t2 = torch.from_numpy(np.ascontiguousarray(a2, dtype=np.int32)).cuda()
    perm, start = wp.baseline_order(t1, t2, n_ant)
    return perm, start


def test_baseline_order_time_major_rows(torch_cuda):
    """27 antennas x 60 time samples in time-major order: every baseline's rows come out
    in time order at the Eq. 6 starts."""
    torch = torch_cuda
    case = parity_case()
    wp = make_wproj(case)
    cfg = synth.config("parity")
    a1, a2 = synth.row_antennas(cfg.n_ant, cfg.n_time)
    perm, start = _order_on_gpu(torch, wp, a1, a2, cfg.n_ant)
    b = oracle.baseline_index(a1, a2, cfg.n_ant)
    _, start_ref = oracle.baseline_starts(b, cfg.n_ant)
    np.testing.assert_array_equal(start.cpu().numpy().astype(np.int64), start_ref)
    np.testing.assert_array_equal(perm.cpu().numpy(), oracle.baseline_order(b, cfg.n_ant))


@pytest.mark.parametrize("n_ant,nrow,seed", [(1, 50, 1), (5, 1, 2), (40, 20000, 3), (300, 7000, 4)])
def test_baseline_order_random_pairs(torch_cuda, n_ant, nrow, seed):
    """Random antenna pairs in either order, autocorrelations included, empty baselines."""
    torch = torch_cuda
    wp = make_wproj(random_case(n=64, nrow=10))
    rng = np.random.default_rng(seed)
    a1, a2 = rng.integers(0, n_ant, nrow), rng.integers(0, n_ant, nrow)
    perm, start = _order_on_gpu(torch, wp, a1, a2, n_ant)
    b = oracle.baseline_index(a1, a2, n_ant)
    _, start_ref = oracle.baseline_starts(b, n_ant)
    np.testing.assert_array_equal(start.cpu().numpy().astype(np.int64), start_ref)
    np.testing.assert_array_equal(perm.cpu().numpy(), oracle.baseline_order(b, n_ant))


def test_baseline_order_long_baseline_and_empty(torch_cuda):
    """A baseline of more than 4096 rows stays grouped (its order within is the scatter's);
    the others are time-ordered. No rows: only the starts, all zero."""
    torch = torch_cuda
    wp = make_wproj(random_case(n=64, nrow=10))
    rng = np.random.default_rng(9)
    n_ant, nrow = 6, 9000
    a1 = np.where(rng.random(nrow) < 0.6, 2, rng.integers(0, n_ant, nrow))
    a2 = np.where(a1 == 2, 4, rng.integers(0, n_ant, nrow))
    b = oracle.baseline_index(a1, a2, n_ant)
    count, start_ref = oracle.baseline_starts(b, n_ant)
    assert count.max() > 4096
    perm, start = _order_on_gpu(torch, wp, a1, a2, n_ant)
    perm, start = perm.cpu().numpy(), start.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(start, start_ref)
    want = oracle.baseline_order(b, n_ant)
    for k in range(oracle.n_baselines(n_ant)):
        got, ref = perm[start[k]:start[k + 1]], want[start[k]:start[k + 1]]
        if count[k] > 4096:
            np.testing.assert_array_equal(np.sort(got), ref)
        else:
            np.testing.assert_array_equal(got, ref)
    e1 = torch.empty(0, dtype=torch.int32, device="cuda")
    perm0, start0 = wp.baseline_order(e1, e1, 4)
    assert perm0.numel() == 0 and torch.all(start0 == 0).item()


def test_baseline_order_rows_without_a_baseline(torch_cuda):
    """Antenna IDs outside [0, N_ant): those rows go after start[N_B], the rest as the oracle
    orders the valid rows."""
    torch = torch_cuda
    wp = make_wproj(random_case(n=64, nrow=10))
    rng = np.random.default_rng(10)
    n_ant, nrow = 7, 3000
    a1, a2 = rng.integers(-2, n_ant + 2, nrow), rng.integers(0, n_ant, nrow)
    bad = (a1 < 0) | (a1 >= n_ant)
    assert bad.any()
    perm, start = _order_on_gpu(torch, wp, a1, a2, n_ant)
    perm, start = perm.cpu().numpy(), start.cpu().numpy().astype(np.int64)
    good = np.flatnonzero(~bad)
    b = oracle.baseline_index(a1[good], a2[good], n_ant)
    _, start_ref = oracle.baseline_starts(b, n_ant)
    np.testing.assert_array_equal(start, start_ref)
    np.testing.assert_array_equal(perm[:start[-1]], good[oracle.baseline_order(b, n_ant)])
    np.testing.assert_array_equal(np.sort(perm[start[-1]:]), np.flatnonzero(bad))


def _baseline_grid(torch, wp, case, ant, n_ant, accumulate_into=None):
    uvw, f, vis, wt = to_dev(case)
    a1, a2 = ant
    perm, start = _order_on_gpu(torch, wp, a1, a2, n_ant)
    return wp.grid_baseline(uvw, f, vis, perm, start, n_ant, wt, hermitian_pairs=case.pairs,
                            grid=accumulate_into, accumulate=accumulate_into is not None)


@pytest.mark.parametrize("pairs,weights", [(False, True), (True, False), (True, True)])
def test_grid_baseline_parity_config(torch_cuda, pairs, weights):
    """The parity workload's real time-ordered baselines against the oracle and wp_grid."""
    torch = torch_cuda
    case = parity_case(pairs=pairs, weights=weights)
    cfg = synth.config("parity")
    crd, g_ref, sw_ref = oracle_results(case)
    wp = make_wproj(case)
    g, sw, nd = _baseline_grid(torch, wp, case, synth.row_antennas(cfg.n_ant, cfg.n_time), cfg.n_ant)
    e, _ = peak_rel(g.cpu().numpy(), g_ref)
    assert e < 1e-6, e
    assert abs(sw.item() - sw_ref) <= 1e-12 * sw_ref
    assert nd.item() == int((~crd["keep"]).sum())
    uvw, f, vis, wt = to_dev(case)
    g1, sw1, nd1 = wp.grid(uvw, f, vis, wt, hermitian_pairs=pairs)
    e1, _ = peak_rel(g.cpu().numpy(), g1.cpu().numpy())
    assert e1 < 1e-6, e1
    assert sw.item() == sw1.item() and nd.item() == nd1.item()


@pytest.mark.parametrize("s_min,s_max,os_,pairs,table", [
    (5, 9, 8, False, "f32"), (7, 16, 4, True, "f32"), (17, 32, 6, False, "f32"), (7, 30, 8, True, "f16"),
    (6, 12, 8, False, "bf16")])
def test_grid_baseline_random_cases(torch_cuda, s_min, s_max, os_, pairs, table):
    """Random uvw (some off the grid, w of both signs), random antenna pairs, several channels,
    supports up to 32, 16-bit tables."""
    torch = torch_cuda
    case = random_case(n=128, nrow=1500, nchan=3, n_w=7, s_min=s_min, s_max=s_max, os_=os_, pairs=pairs, seed=43)
    rng = np.random.default_rng(44)
    n_ant = 11
    ant = (rng.integers(0, n_ant, 1500), rng.integers(0, n_ant, 1500))
    wp = make_wproj(case, table=table)
    g, sw, nd = _baseline_grid(torch, wp, case, ant, n_ant)
    uvw, f, vis, wt = to_dev(case)
    g1, sw1, nd1 = wp.grid(uvw, f, vis, wt, hermitian_pairs=pairs)
    e1, _ = peak_rel(g.cpu().numpy(), g1.cpu().numpy())
    assert e1 < 1e-6, e1
    assert sw.item() == sw1.item() and nd.item() == nd1.item()
    if table == "f32":
        _, g_ref, _ = oracle_results(case)
        e, _ = peak_rel(g.cpu().numpy(), g_ref)
        assert e < 1e-6, e


def test_grid_baseline_accumulates(torch_cuda):
    torch = torch_cuda
    case = random_case(n=64, nrow=600, nchan=2, seed=45)
    rng = np.random.default_rng(46)
    ant = (rng.integers(0, 8, 600), rng.integers(0, 8, 600))
    wp = make_wproj(case)
    g, sw, _ = _baseline_grid(torch, wp, case, ant, 8)
    g0, sw0 = g.clone(), sw.clone()
    _baseline_grid(torch, wp, case, ant, 8, accumulate_into=g)
    e, _ = peak_rel(g.cpu().numpy(), 2 * g0.cpu().numpy())
    assert e < 1e-6, e


def test_grid_baseline_rejects_supports_above_32(torch_cuda):
    import paper_1905_03213_b300 as W
    torch = torch_cuda
    case = random_case(n=128, nrow=100, nchan=1, n_w=3, s_min=30, s_max=36, os_=4)
    wp = make_wproj(case)
    rng = np.random.default_rng(47)
    with pytest.raises(W.WProjError):
        _baseline_grid(torch, wp, case, (rng.integers(0, 4, 100), rng.integers(0, 4, 100)), 4)
