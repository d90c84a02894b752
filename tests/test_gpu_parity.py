"""GPU parity: the CUDA path (through the C ABI) against the float64 oracle on the same
seeded inputs. Integer work bit-exact; floating point within the stated tolerances."""
import numpy as np
import pytest

import oracle
from oracle import wproj
import synth
from gpu_cases import (TOL_IMAGE, inner, make_wproj, oracle_results, parity_case, peak_rel, random_case,
                       to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


# ---------------------------------------------------------------- coordinates
@pytest.mark.parametrize("pairs", [False, True])
def test_coords_bit_exact(torch_cuda, pairs):
    case = random_case(nrow=2000, nchan=4, pairs=pairs, off_grid=0.2)
    wp = make_wproj(case)
    uvw, f, _, _ = to_dev(case)
    got = wp.coords(uvw, f, hermitian_pairs=pairs).cpu().numpy()
    crd = oracle.coords(case.uvw, case.freqs, case.prm, hermitian_pairs=pairs)
    keep = crd["keep"]
    np.testing.assert_array_equal(got[:, 4].astype(bool), keep)
    for col, key in ((0, "U"), (1, "V"), (2, "plane"), (3, "conj"), (5, "i0"), (6, "j0")):
        np.testing.assert_array_equal(got[keep, col], crd[key][keep].astype(np.int64), err_msg=key)
    np.testing.assert_array_equal(got[keep, 7] & 0xffff, crd["ox"][keep])
    np.testing.assert_array_equal(got[keep, 7] >> 16, crd["oy"][keep])
    assert (~keep).sum() > 0 and keep.sum() > 1000


def test_coords_edge_values(torch_cuda):
    """Half-integer ties, -0.0, beyond-w_max, NaN/inf and huge rows: identical decisions."""
    import torch
    import paper_1905_03213_b300 as W
    p = oracle.Params(n=16, cell=1.0 / (8 * 16), n_w=3, w_max=100.0, s_min=4, s_max=4, os=8)
    wp = W.WProj(n=16, cell=p.cell, n_w=3, w_max=100.0, support_min=4, support_max=4, oversample=8)
    wp.make_wkernels()
    f = np.array([oracle.C_LIGHT])
    uvw = np.array([[4.5, 5.5, 10.0], [-4.5, -5.5, -10.0], [0.0, 0.0, -0.0], [60.0, 0.0, 49.9],
                    [0.0, 0.0, 75.0], [0.0, 0.0, 1e9], [np.nan, 0.0, 0.0], [np.inf, 0, 0],
                    [0.5, -0.5, 25.0], [1.5, -1.5, -25.0], [2.5e9, 0, 0], [3.5, 2.5, 50.0]])
    got = wp.coords(torch.from_numpy(uvw).cuda(), torch.from_numpy(f).cuda(), hermitian_pairs=True).cpu().numpy()
    crd = oracle.coords(uvw, f, p, hermitian_pairs=True)
    np.testing.assert_array_equal(got[:, 4].astype(bool), crd["keep"])
    k = crd["keep"]
    np.testing.assert_array_equal(got[k, 0], crd["U"][k])
    np.testing.assert_array_equal(got[k, 1], crd["V"][k])
    np.testing.assert_array_equal(got[k, 2], crd["plane"][k])
    np.testing.assert_array_equal(got[k, 3].astype(bool), crd["conj"][k])


def test_coords_near_rounding_boundaries(torch_cuda):
    """Products within 1e-12 .. 0.05 of a half-integer, on both sides, over the whole range of a
    4096-cell grid: the float32-first evaluation must take the float64 decision in every case
    (it forms the float64 product only where its error bound leaves the rounding undecided)."""
    import torch
    import paper_1905_03213_b300 as W
    n, os_, n_w, w_max = 4096, 8, 64, 1500.0
    cell = 1.0 / (n * 3.1)
    p = oracle.Params(n=n, cell=cell, n_w=n_w, w_max=w_max, s_min=8, s_max=8, os=os_)
    wp = W.WProj(n=n, cell=cell, n_w=n_w, w_max=w_max, support_min=8, support_max=8, oversample=os_)
    wp.make_wkernels()
    f = np.array([1.0e9, 1.234567e9, 1.4e9])
    kx = f / oracle.C_LIGHT * (os_ * (n * cell))
    kw = f / oracle.C_LIGHT * ((n_w - 1) / w_max)
    rng = np.random.default_rng(31)
    offs = np.array([0.0, 1e-12, 1e-9, 1e-7, 1e-6, 1e-5, 1e-4, 3e-3, 6e-3, 1e-2, 1.4e-2, 2e-2, 5e-2])
    offs = np.concatenate([offs, -offs[1:]])
    m = rng.integers(-16000, 16000, size=(400, offs.size))
    x = (m + 0.5 + offs[None, :]).ravel()
    mw = rng.integers(0, n_w - 1, size=x.size)
    z = mw + 0.5 + rng.choice(offs, size=x.size)
    c = rng.integers(0, f.size, size=x.size)          # the channel whose factors hit the boundary
    uvw = np.stack([x / kx[c], x[::-1] / kx[c], np.where(rng.random(x.size) < 0.5, -1, 1) * z / kw[c]], axis=1)
    got = wp.coords(torch.from_numpy(uvw).cuda(), torch.from_numpy(f).cuda()).cpu().numpy()
    crd = oracle.coords(uvw, f, p)
    for col, key in ((0, "U"), (1, "V"), (2, "plane"), (3, "conj")):
        np.testing.assert_array_equal(got[:, col], crd[key].astype(np.int64), err_msg=key)
    np.testing.assert_array_equal(got[:, 4].astype(bool), crd["keep"])
    # the cases do straddle: both roundings of the nominal half-integer occur
    ux = (uvw[:, 0:1] * kx[None, :]).ravel()
    assert (np.rint(ux) > np.floor(ux)).any() and (np.rint(ux) == np.floor(ux)).any()


# ---------------------------------------------------------------- kernel tables
@pytest.mark.parametrize("which", ["parity", "range"])
def test_wkernel_tables(torch_cuda, which):
    case = parity_case() if which == "parity" else random_case(s_min=6, s_max=11, n_w=5)
    wp = make_wproj(case)
    assert abs(wp.wkernel_norm() / case.nu - 1) < 1e-13
    sup, wpl = wp.plane_info()
    np.testing.assert_array_equal(sup, oracle.plane_supports(case.prm.n_w, case.prm.s_min, case.prm.s_max))
    np.testing.assert_array_equal(wpl, oracle.plane_w(case.prm.n_w, case.prm.w_max))
    for p in range(case.prm.n_w):
        ref = case.tables[p]
        scale = np.abs(ref).max()
        k64 = wp.wkernel_export(p)
        assert np.abs(k64 - ref).max() < 1e-12 * scale, p
        k32 = wp.wkernel_export(p, stored=True)
        assert np.abs(k32 - ref).max() < 1e-7 * scale, p


@pytest.mark.parametrize("table,tol", [("f16", 1e-3), ("bf16", 8e-3)])
def test_wkernel_tables_reduced_precision(torch_cuda, table, tol):
    case = parity_case()
    wp = make_wproj(case, table=table)
    for p in (0, case.prm.n_w // 2, case.prm.n_w - 1):
        ref = case.tables[p]
        got = wp.wkernel_export(p, stored=True)
        assert np.abs(got - ref).max() < tol * np.abs(ref).max()
        if table == "bf16":
            # each component within half a bfloat16 ulp (at most 2^-8 relative) of its float64 value: the
            # real part rounded to bfloat16, the imaginary part the nearest float32 whose low 16
            # bits are the real part's bits (see the stored word format in wproj.h); the floor is
            # the float64 tables' own agreement (1e-12 of the peak), which decides components that
            # are rounding noise (the imaginary part of the w = 0 plane)
            for c in (np.real, np.imag):
                err = np.abs(c(got) - c(ref))
                bound = 2.0 ** -8 * np.abs(c(ref)) * (1 + 1e-6) + 1e-12 * np.abs(ref).max()
                assert np.all(err <= bound), (p, (err - bound).max())


# ---------------------------------------------------------------- gridding + image
def _grid_and_image(case, table="f32", tile=(0, 0)):
    """Grid, then both images: (grid, corrected image, uncorrected image, sum_w, n_dropped)."""
    import torch
    wp = make_wproj(case, table=table, tile=tile)
    uvw, f, vis, wt = to_dev(case)
    g, sw, nd = wp.grid(uvw, f, vis, wt, hermitian_pairs=case.pairs)
    gh = g.cpu().numpy()
    g2 = g.clone()
    img = wp.fft_to_image(g, sw).cpu().numpy()
    raw = wp.fft_to_image(g2, sw, taper_correct=False).cpu().numpy()
    torch.cuda.synchronize()
    return gh, img, raw, float(sw.item()), int(nd.item())


def _image_errors(case, g_ref, sw_ref, img, raw):
    """Image metric: peak-relative max error of the uncorrected image over all pixels and
    of the taper-corrected image over the inner half (the corrected image divides by
    t(x_i) t(x_j), ~1e-8 in the corners, which would amplify float32 rounding there)."""
    ref = oracle.fft_to_image(g_ref, sw_ref, case.prm)
    ref_raw = oracle.fft_to_image(g_ref, sw_ref, case.prm, taper_correct=False)
    e_raw, rms_raw = peak_rel(raw, ref_raw)
    e_cor, rms_cor = peak_rel(inner(img), inner(ref))
    return max(e_raw, e_cor), (e_raw, rms_raw, e_cor, rms_cor)


@pytest.mark.parametrize("pairs,weights", [(False, True), (True, False)])
def test_grid_and_image_parity_config(torch_cuda, pairs, weights):
    case = parity_case(pairs=pairs, weights=weights)
    crd, g_ref, sw_ref = oracle_results(case)
    g, img, raw, sw, nd = _grid_and_image(case)
    assert nd == int((~crd["keep"]).sum())
    assert abs(sw - sw_ref) <= 1e-12 * sw_ref
    eg, _ = peak_rel(g, g_ref)
    assert eg < 1e-6, eg
    emax, detail = _image_errors(case, g_ref, sw_ref, img, raw)
    assert emax < TOL_IMAGE["f32"], detail


@pytest.mark.parametrize("tile", [(8, 8), (16, 64), (64, 16), (128, 128)])
def test_grid_tile_shapes(torch_cuda, tile):
    case = random_case(n=128, nrow=1500, nchan=2, s_min=5, s_max=12, n_w=7)
    crd, g_ref, sw_ref = oracle_results(case)
    g, img, raw, sw, nd = _grid_and_image(case, tile=tile)
    eg, _ = peak_rel(g, g_ref)
    assert eg < 1e-6, (tile, eg)


@pytest.mark.parametrize("table,pairs,os_", [("f32", False, 8), ("f32", True, 4), ("f16", False, 8), ("bf16", True, 6)])
def test_grid_and_degrid_large_supports(torch_cuda, table, pairs, os_):
    """Supports 7-30: planes above 16 run with two row halves per piece and lane-order tables
    read from global memory, planes up to 16 with staged tables, in the same launch. (The taper
    follows S_min: with a larger S_min it is so small at the inner half's edge that the
    taper-corrected image magnifies f16 table rounding past 1e-3 there, table or no table.)"""
    import torch
    case = random_case(n=128, nrow=1200, nchan=2, n_w=7, s_min=7, s_max=30, os_=os_, pairs=pairs, seed=41)
    crd, g_ref, sw_ref = oracle_results(case)
    g, img, raw, sw, nd = _grid_and_image(case, table=table)
    eg, _ = peak_rel(g, g_ref)
    assert eg < (1e-6 if table == "f32" else TOL_IMAGE[table]), eg
    emax, detail = _image_errors(case, g_ref, sw_ref, img, raw)
    if table == "f32":
        assert emax < TOL_IMAGE["f32"], detail
    else:
        # 16-bit tables: the mixed-precision bound on the dirty image (uncorrected, all pixels);
        # the taper-corrected inner half magnifies the table rounding by up to 1/(t t) there
        assert detail[0] < 1e-3 and detail[2] < 5e-3, detail
    crd1 = oracle.coords(case.uvw, case.freqs, case.prm)
    gh = synth.random_grid(case.prm.n, 17)
    ref = oracle.degrid(crd1, gh.astype(np.complex128), case.tables, case.prm).reshape(case.vis.shape)
    wp = make_wproj(case, table=table)
    uvw, f, _, _ = to_dev(case)
    out = wp.degrid(uvw, f, torch.from_numpy(gh).cuda()).cpu().numpy()
    e, _ = peak_rel(out, ref)
    assert e < TOL_IMAGE[table], e


@pytest.mark.parametrize("table", ["f16", "bf16"])
def test_grid_reduced_precision_tables(torch_cuda, table):
    case = parity_case()
    crd, g_ref, sw_ref = oracle_results(case)
    g, img, raw, sw, nd = _grid_and_image(case, table=table)
    emax, detail = _image_errors(case, g_ref, sw_ref, img, raw)
    assert emax < TOL_IMAGE[table], (table, detail)


def test_uncorrected_image(torch_cuda):
    case = parity_case()
    crd, g_ref, sw_ref = oracle_results(case)
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    g, sw, nd = wp.grid(uvw, f, vis, wt)
    img = wp.fft_to_image(g, sw, taper_correct=False).cpu().numpy()
    ref = oracle.fft_to_image(g_ref, sw_ref, case.prm, taper_correct=False)
    emax, _ = peak_rel(img, ref)
    assert emax < 1e-5


def test_accumulate_two_halves(torch_cuda):
    case = parity_case()
    crd, g_ref, sw_ref = oracle_results(case)
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    h = uvw.shape[0] // 2 + 17                      # ragged split
    g, sw, nd = wp.grid(uvw[:h].contiguous(), f, vis[:h].contiguous(), wt[:h].contiguous())
    wp.grid(uvw[h:].contiguous(), f, vis[h:].contiguous(), wt[h:].contiguous(), grid=g, sum_w=sw, n_dropped=nd,
            accumulate=True)
    eg, _ = peak_rel(g.cpu().numpy(), g_ref)
    assert eg < 1e-6
    assert abs(sw.item() - sw_ref) <= 1e-12 * sw_ref
    assert nd.item() == int((~crd["keep"]).sum())


def test_empty_and_all_dropped(torch_cuda):
    import torch
    case = random_case(nrow=50, nchan=1)
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    g, sw, nd = wp.grid(uvw[:0].contiguous(), f, vis[:0].contiguous(), wt[:0].contiguous())
    assert torch.count_nonzero(g).item() == 0 and sw.item() == 0.0 and nd.item() == 0
    far = uvw * 1e6                                  # every footprint far off the grid
    g, sw, nd = wp.grid(far, f, vis, wt)
    assert torch.count_nonzero(g).item() == 0 and sw.item() == 0.0 and nd.item() == 50
    out = wp.degrid(far, f, g)
    assert torch.count_nonzero(out).item() == 0


def test_single_visibility_and_small_grid(torch_cuda):
    """N = 16 with support 8 (footprint half the grid), and one visibility alone."""
    case = random_case(n=16, nrow=40, nchan=1, n_w=2, s_min=8, s_max=8, off_grid=0.0)
    crd, g_ref, sw_ref = oracle_results(case)
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    g, sw, nd = wp.grid(uvw, f, vis, wt)
    assert crd["keep"].sum() > 0
    eg, _ = peak_rel(g.cpu().numpy(), g_ref)
    assert eg < 1e-6
    k = int(np.nonzero(crd["keep"])[0][0])
    g1, _, _ = wp.grid(uvw[k:k + 1].contiguous(), f, vis[k:k + 1].contiguous(), wt[k:k + 1].contiguous())
    one = dict(crd)
    one["keep"] = np.zeros_like(crd["keep"])
    one["keep"][k] = True
    ref1 = oracle.grid(one, wproj.gridded_values(case.vis, case.weight, crd), case.tables, case.prm)
    eg1, _ = peak_rel(g1.cpu().numpy(), ref1)
    assert eg1 < 1e-6


def test_repeat_runs_agree(torch_cuda):
    """Float32 atomics merge in any order: two runs agree to rounding."""
    case = random_case(n=128, nrow=3000, nchan=2)
    g1 = _grid_and_image(case)[0]
    g2 = _grid_and_image(case)[0]
    eg, _ = peak_rel(g1, g2)
    assert eg < 1e-6


# ---------------------------------------------------------------- degridding
@pytest.mark.parametrize("which,table", [("parity", "f32"), ("random", "f32"), ("random", "f16"), ("random", "bf16")])
def test_degrid_parity(torch_cuda, which, table):
    """Degridding against the float64 oracle; f16/bf16 tables within the mixed-precision tolerances."""
    import torch
    case = parity_case() if which == "parity" else random_case(n=128, nrow=1200, nchan=3, s_min=5, s_max=12)
    crd = oracle.coords(case.uvw, case.freqs, case.prm)
    gh = synth.random_grid(case.prm.n, 9)
    ref = oracle.degrid(crd, gh.astype(np.complex128), case.tables, case.prm).reshape(case.vis.shape)
    wp = make_wproj(case, table=table)
    uvw, f, _, _ = to_dev(case)
    out = wp.degrid(uvw, f, torch.from_numpy(gh).cuda()).cpu().numpy()
    e, _ = peak_rel(out, ref)
    assert e < TOL_IMAGE[table], e
    np.testing.assert_array_equal(out.ravel()[~crd["keep"]], 0)


@pytest.mark.parametrize("pairs,table", [(False, "f32"), (True, "f32"), (True, "f16")])
def test_degrid_last_reuses_grid_binning(torch_cuda, pairs, table):
    """wp_degrid_last after wp_grid(WP_KEEP_BINNING) equals wp_degrid on the same visibilities, element for
    element (the partners wp_grid added are skipped, dropped visibilities are 0), and against
    the oracle within the degridding tolerance."""
    import torch
    import paper_1905_03213_b300 as W
    case = random_case(n=128, nrow=1500, nchan=3, s_min=5, s_max=12, pairs=pairs, off_grid=0.1)
    wp = make_wproj(case, table=table)
    uvw, f, vis, wt = to_dev(case)
    G = torch.from_numpy(synth.random_grid(case.prm.n, 21)).cuda()
    # without WP_KEEP_BINNING the binning is not kept: degrid_last is refused
    wp.grid(uvw, f, vis, wt, hermitian_pairs=pairs)
    with pytest.raises(W.WProjError):
        wp.degrid_last(G)
    assert W.lib.wp_degrid_last(wp._h, G.data_ptr(), G.data_ptr(), None) == W.WP_ESTATE
    wp.grid(uvw, f, vis, wt, hermitian_pairs=pairs, keep_binning=True)
    last = wp.degrid_last(G)
    own = wp.degrid(uvw, f, G)
    assert torch.equal(last, own)
    crd = oracle.coords(case.uvw, case.freqs, case.prm)
    assert (~crd["keep"]).sum() > 0
    np.testing.assert_array_equal(last.cpu().numpy().ravel()[~crd["keep"]], 0)
    if table == "f32":
        ref = oracle.degrid(crd, G.cpu().numpy().astype(np.complex128), case.tables, case.prm).reshape(case.vis.shape)
        e, _ = peak_rel(last.cpu().numpy(), ref)
        assert e < 1e-5, e
    # wp_degrid replaced the binning: a second degrid_last is refused
    rc = W.lib.wp_degrid_last(wp._h, G.data_ptr(), last.data_ptr(), None)
    assert rc == W.WP_ESTATE


def test_adjoint_dot_product_gpu(torch_cuda):
    """<grid(c), G> = <c, degrid(G)> with unit weights, both on the GPU (float32)."""
    import torch
    case = random_case(n=128, nrow=2000, nchan=2, s_min=5, s_max=11)
    wp = make_wproj(case)
    uvw, f, vis, _ = to_dev(case)
    g, _, _ = wp.grid(uvw, f, vis, None)
    G = torch.from_numpy(synth.random_grid(case.prm.n, 12)).cuda()
    dv = wp.degrid(uvw, f, G)
    lhs = torch.vdot(g.ravel().to(torch.complex128), G.ravel().to(torch.complex128)).item()
    rhs = torch.vdot(vis.ravel().to(torch.complex128), dv.ravel().to(torch.complex128)).item()
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)


def test_profile_counts_phases_and_launches(torch_cuda):
    case = random_case(n=64, nrow=500, nchan=2)
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    wp.profile(True)
    wp.profile_read()
    wp.make_wkernels()
    g, sw, _ = wp.grid(uvw, f, vis, wt)
    wp.degrid(uvw, f, g)
    wp.fft_to_image(g, sw)
    ms, cnt, launches = wp.profile_read()
    assert cnt == {"wkernels": 1, "plan": 2, "grid": 1, "degrid": 1, "fft": 1, "image": 1}
    assert all(v > 0 for v in ms.values())
    # 6 kernel-table + (1 channel + 8 plan + 4 work-estimate scan + 1 grid + 1 scalars)
    # + (1 channel + 8 plan + 4 work-estimate scan + 1 degrid) + 1 image; the plan's 8 are the
    # histogram, 3 prefix-sum kernels, the bin offsets, the scatter, the bin list, the origin sort
    assert launches == 36
    # degridding the gridded visibilities again reuses wp_grid's binning: no plan phase
    g, sw, _ = wp.grid(uvw, f, vis, wt, keep_binning=True)
    wp.profile_read()
    wp.degrid_last(g)
    ms, cnt, launches = wp.profile_read()
    assert {k: v for k, v in cnt.items() if v} == {"degrid": 1} and launches == 5


def test_supports_across_16_split_into_two_launches(torch_cuda):
    """Planes of support <= 16 (a prefix of the bins) run in the 32-warp launch and the rest in
    the 16-warp launch: both halves of one grid and one degridding against the oracle, and the
    launch count shows the two launches."""
    torch = torch_cuda
    case = random_case(n=192, nrow=1500, nchan=2, n_w=9, s_min=8, s_max=24, seed=71, pairs=True)
    sup = oracle.plane_supports(case.prm.n_w, case.prm.s_min, case.prm.s_max)
    assert sup.min() <= 16 < sup.max()
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    wp.profile(True)
    wp.profile_read()
    g, _, _ = wp.grid(uvw, f, vis, wt, hermitian_pairs=True, keep_binning=True)
    _, _, launches = wp.profile_read()
    # 1 channel + 8 plan + 4 work-estimate scan + 2 gridding + 1 scalars
    assert launches == 16
    crd, g_ref, _ = oracle_results(case)
    e, _ = peak_rel(g.cpu().numpy(), g_ref)
    assert e < 1e-5, e
    G = synth.random_grid(case.prm.n, 3)
    pred = wp.degrid(uvw, f, torch.from_numpy(G).cuda()).cpu().numpy().ravel()
    ref = oracle.degrid(oracle.coords(case.uvw, case.freqs, case.prm), G.astype(np.complex128), case.tables,
                        case.prm, threads=4)
    e2, _ = peak_rel(pred, ref)
    assert e2 < 1e-5, e2
