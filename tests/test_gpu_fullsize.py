"""GPU against the float64 oracle on the paths that the kernels only take at full size.

Small parity cases never fill a (plane, tile) bin beyond one sorted chunk, never make the
work-estimate prefix sum rescale its unit, and never reach the kernels for supports above
32. These cases do, each checked element by element against the oracle:
  * a dense bin: 60,000 visibilities whose footprints all start inside one origin tile of one
    plane, so the gridding and degridding kernels sort and walk it as 8+ chunks;
  * a geometry with 2.6M bins, whose work-estimate upper bound exceeds 2^37 tap-updates, so
    the estimate's unit doubles (shift > 0);
  * supports 33-40, which run the shared-memory baseline kernels (gridding and degridding).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import wproj
import synth
from gpu_cases import Case, make_wproj, oracle_results, peak_rel, random_case, to_dev

pytestmark = pytest.mark.gpu
ARCSEC = math.pi / (180 * 3600)


def _grid_vs_oracle(case, table="f32", tile=(0, 0), tol=1e-6):
    import torch
    wp = make_wproj(case, table=table, tile=tile)
    uvw, f, vis, wt = to_dev(case)
    g, sw, nd = wp.grid(uvw, f, vis, wt, hermitian_pairs=case.pairs)
    crd, g_ref, sw_ref = oracle_results(case)
    e, _ = peak_rel(g.cpu().numpy(), g_ref)
    assert e < tol, e
    assert abs(sw.item() - sw_ref) <= 1e-9 * max(sw_ref, 1.0)
    assert nd.item() == int((~crd["keep"]).sum())
    # degridding of a random grid through the same bins
    G = synth.random_grid(case.prm.n, 5)
    pred = wp.degrid(uvw, f, torch.from_numpy(G).cuda()).cpu().numpy().ravel()
    crd1 = oracle.coords(case.uvw, case.freqs, case.prm)
    ref = oracle.degrid(crd1, G.astype(np.complex128), case.tables, case.prm, threads=4)
    e2, _ = peak_rel(pred, ref)
    assert e2 < tol, e2
    return crd


def dense_bin_case(nvis=60_000, seed=41):
    """One 32x32 origin tile of plane 0 (and a sliver of plane 1) holds every footprint."""
    rng = np.random.default_rng(seed)
    n, cell, os_ = 256, 10 * ARCSEC, 8
    freqs = np.array([1.4e9])
    lam = oracle.C_LIGHT / freqs[0]
    du = 1.0 / (n * cell)                        # wavelengths per cell
    # origins i0 ~ N/2 + u/du - S/2 + 1 in [225, 249] for u/du in [100, 120]: tile 7 of 8
    u = rng.uniform(100.5, 119.5, nvis) * du * lam
    v = rng.uniform(100.5, 119.5, nvis) * du * lam
    w = rng.uniform(-1.0, 1.0, nvis) * 40.0 * lam        # |w| <= 40 wavelengths: planes 0 and 1
    uvw = np.stack([u, v, w], axis=1)
    vis, wt = synth.random_visibilities(nvis, 1, seed + 1)
    prm = oracle.Params(n=n, cell=cell, n_w=8, w_max=300.0, s_min=7, s_max=7, os=os_)
    tabs, nu = oracle.wkernels(prm)
    return Case(prm, uvw, freqs, vis, wt, False, tabs, nu)


# ~7,000 visibilities reach each cell of this bin, so float32 accumulation alone gives grid
# errors of a few 1e-6 of the peak: the bound is the float32 image tolerance, 1e-5
@pytest.mark.parametrize("table,tol", [("f32", 1e-5), ("f16", 1e-3)])
def test_dense_bin_spans_many_chunks(table, tol):
    case = dense_bin_case()
    crd = oracle.coords(case.uvw, case.freqs, case.prm)
    tiles = set(zip((crd["j0"][crd["keep"]] // 32).tolist(), (crd["i0"][crd["keep"]] // 32).tolist()))
    planes = np.bincount(crd["plane"][crd["keep"]])
    assert tiles == {(7, 7)} and planes.max() > 3 * 8192, (tiles, planes)
    _grid_vs_oracle(case, table=table, tol=tol)


def test_work_estimate_unit_rescaled():
    """4096^2 grid, 16x16 origin tiles and 40 planes: 2,621,440 bins. The estimate's upper bound
    (bins x 65536 fixed tap-updates, plus records x (S_max^2 + 64)) is above 2^37, so its unit
    grows from 2^6 to 2^7 tap-updates or more (the 32-bit prefix sum must not wrap)."""
    n, n_w, tile = 4096, 40, 16
    nbins = (n // tile) ** 2 * n_w
    nrow = 4000
    bound = nrow * 3 * (12 ** 2 + 64) + nbins * 65536
    shift = 0
    while (bound >> (6 + shift)) + nbins >= 1 << 31:
        shift += 1
    assert shift >= 1, shift
    case = random_case(n=n, nrow=nrow, nchan=3, n_w=n_w, s_min=6, s_max=12, seed=43, cell=2 * ARCSEC)
    _grid_vs_oracle(case, tile=(tile, tile))


# the shared-memory kernel of these supports adds up to 1,296 taps per visibility into float32
# cells with atomics, in an order that depends on the record order: the grid is held to the
# float32 image tolerance
@pytest.mark.parametrize("s_min,s_max,os_,table,tol", [(33, 36, 4, "f32", 1e-5), (34, 40, 2, "f16", 1e-3)])
def test_supports_above_32(s_min, s_max, os_, table, tol):
    case = random_case(n=160, nrow=600, nchan=2, n_w=3, s_min=s_min, s_max=s_max, os_=os_, seed=47)
    _grid_vs_oracle(case, table=table, tol=tol)


def test_compensated_accumulation_on_the_dense_bin():
    """WP_COMPENSATED: the dense bin's grid (about 7,000 visibilities per cell) with compensated
    float32 sums in the grid is no further from the float64 oracle than the plain float32 sums,
    and within 5e-7 of the peak. (What remains is the float32 accumulation inside a footprint's
    registers, over an origin's records, and the float32 rounding of the tables.)"""
    case = dense_bin_case()
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    crd, g_ref, _ = oracle_results(case)
    g_plain, _, _ = wp.grid(uvw, f, vis, wt)
    g_comp, _, _ = wp.grid(uvw, f, vis, wt, compensated=True)
    e_plain, _ = peak_rel(g_plain.cpu().numpy(), g_ref)
    e_comp, _ = peak_rel(g_comp.cpu().numpy(), g_ref)
    assert e_comp < 5e-7 and e_comp <= e_plain, (e_comp, e_plain)


def test_compensated_rejected_above_support_32():
    import paper_1905_03213_b300 as W
    case = random_case(n=160, nrow=50, nchan=1, n_w=3, s_min=33, s_max=36, os_=4, seed=48)
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    with pytest.raises(W.WProjError):
        wp.grid(uvw, f, vis, wt, compensated=True)
