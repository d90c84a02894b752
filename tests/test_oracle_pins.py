"""Pins for the FP64 oracle: each test checks it against something other than itself
(an integral equation, a brute-force sum, a closed form, an exact identity, or the
direct-DFT dirty image that W-projection approximates). CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import wproj
import synth

ARCMIN = math.pi / (180 * 60)


# ---------------------------------------------------------------- taper (PSWF)
@pytest.mark.parametrize("s_min", [5, 7, 8])
def test_taper_solves_prolate_integral_equation(s_min):
    """psi_0 is the eigenfunction of the finite Fourier transform on [-1, 1]:
    int exp(i c x y) psi(y) dy = lambda psi(x). Checked at interior points and x = +-1."""
    c = oracle.taper_c(s_min)
    y, wq = np.polynomial.legendre.leggauss(300)
    ty = oracle.taper(y, c)
    lam = np.sum(wq * ty)                       # x = 0, t(0) = 1
    x = np.concatenate([np.linspace(-0.98, 0.98, 23), [-1.0, 1.0]])
    lhs = (np.exp(1j * c * np.outer(x, y)) * wq * ty).sum(1) / lam
    np.testing.assert_allclose(lhs.real, oracle.taper(x, c), rtol=0, atol=1e-12)
    assert np.max(np.abs(lhs.imag)) < 1e-13


def test_taper_normalised_even_positive():
    c = oracle.taper_c(7)
    x = np.linspace(0, 1, 50)
    t = oracle.taper(x, c)
    assert t[0] == 1.0
    np.testing.assert_array_equal(oracle.taper(-x, c), t)
    assert np.all(t > 0) and np.all(np.diff(t) < 0)


# ---------------------------------------------------------------- W-kernels
def test_kernel_fft_route_equals_direct_sum():
    """The zero-padded FFT equals the defining double sum (tiny lattice, w != 0)."""
    args = dict(w=3000.0, s=4, os_=4, m=17, field=40 * ARCMIN, c=oracle.taper_c(4))
    a = oracle.wkernel_unnormalised(**args)
    b = oracle.wkernel_dft_bruteforce(**args)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())


def _mirror(k):
    """K at -d for the stored d in (-half, half): drop the last entry (d = half)."""
    return k[:-1, :-1][::-1, ::-1]


def test_kernel_even_and_conjugate_for_negative_w():
    """Odd symmetric lattice -> even screen -> K(-d) = K(d) and C_{-w} = conj(C_w)."""
    c = oracle.taper_c(6)
    kp = oracle.wkernel_unnormalised(2500.0, 6, 8, 41, 30 * ARCMIN, c)
    km = oracle.wkernel_unnormalised(-2500.0, 6, 8, 41, 30 * ARCMIN, c)
    scale = np.abs(kp).max()
    np.testing.assert_allclose(_mirror(kp), kp[:-1, :-1], rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(km, np.conj(kp), rtol=0, atol=1e-13 * scale)


def test_w0_kernel_is_separable_taper_transform():
    """w = 0: the screen is t(l) t(m), so the 2D kernel is the outer product of the 1D
    transform of the taper (computed here independently as a 1D sum)."""
    s, os_, m = 7, 8, 65
    c = oracle.taper_c(s)
    k2 = oracle.wkernel_unnormalised(0.0, s, os_, m, 1.0 * math.pi / 180, c)
    j = np.arange(m) - (m - 1) // 2
    tj = oracle.taper(2.0 * j / m, c)
    d = np.arange(-s * os_ // 2 + 1, s * os_ // 2 + 1)
    k1 = (tj[None, :] * np.cos(2 * np.pi * np.outer(d, j) / (os_ * m))).sum(1)
    np.testing.assert_allclose(k2, np.outer(k1, k1), rtol=0, atol=1e-12 * np.abs(k2).max())
    assert np.abs(k2.imag).max() < 1e-12 * np.abs(k2).max()


def test_normalisation_on_cell_w0_sums_to_one():
    prm = oracle.Params(n=128, cell=30 / 3600 * math.pi / 180, n_w=4, w_max=2000.0, s_min=7, s_max=9, os=8)
    tabs, nu = oracle.wkernels(prm)
    e = tabs[0].shape[0]
    half = e // 2
    on = np.nonzero((np.arange(e) - half + 1) % 8 == 0)[0]
    assert abs(tabs[0][np.ix_(on, on)].sum() - 1.0) < 1e-13
    # every oversampled offset's footprint sums to ~1 (the taper's transform is nearly
    # confined to the support, Sec. 2.2 "full support size"): loose, within aliasing level
    for p, t in enumerate(tabs):
        sp = t.shape[0] // 8
        sums = np.array([[t[oy::8, ox::8].sum() for ox in range(8)] for oy in range(8)])
        assert np.all(np.abs(sums - 1.0) < 0.02), (p, np.abs(sums - 1).max())


# ---------------------------------------------------------------- coordinates
def _prm(n=16, os_=8, s=4, n_w=3, w_max=100.0):
    # cell chosen so that os * N * cell = 1: uvw metres at f = c_light give U = rint(u)
    return oracle.Params(n=n, cell=1.0 / (os_ * n), n_w=n_w, w_max=w_max, s_min=s, s_max=s, os=os_)


def test_coords_closed_form():
    prm = _prm()
    f = np.array([oracle.C_LIGHT])                   # 1 wavelength per metre
    uvw = np.array([[4.5, 5.5, 10.0],                # half-to-even: U = 4, V = 6
                    [-4.5, -5.5, -10.0],             # U = -4, V = -6, conj
                    [0.0, 0.0, -0.0],                # -0.0 is not negative
                    [60.0, 0.0, 49.9],               # plane rint(49.9 * 2 / 100) = 1
                    [0.0, 0.0, 75.0],                # plane rint(1.5) = 2
                    [0.0, 0.0, 1e9],                 # beyond w_max: clamped to the last plane
                    [np.nan, 0.0, 0.0], [np.inf, 0, 0]])
    crd = oracle.coords(uvw, f, prm)
    np.testing.assert_array_equal(crd["U"][:6], [4, -4, 0, 60, 0, 0])
    np.testing.assert_array_equal(crd["V"][:6], [6, -6, 0, 0, 0, 0])
    np.testing.assert_array_equal(crd["plane"][:6], [0, 0, 0, 1, 2, 2])
    np.testing.assert_array_equal(crd["conj"][:3], [False, True, False])
    # footprint: X = U + N/2 os = 68, S os/2 = 16: i0 = floor(52 / 8) + 1 = 7, ox = 56 - 68 + 15 = 3
    assert crd["i0"][0] == 7 and crd["ox"][0] == 3
    # cells i with -16 < 8 i - 68 <= 16 are 7..10
    i = np.arange(16)
    cells = i[(8 * i - 68 > -16) & (8 * i - 68 <= 16)]
    np.testing.assert_array_equal(cells, np.arange(crd["i0"][0], crd["i0"][0] + 4))
    # tie: X - S os/2 divisible by os -> asymmetric footprint (d = +S os/2 included, -S os/2 not)
    c2 = oracle.coords(np.array([[0.0, 0.0, 0.0]]), f, prm)   # X = 64, X - 16 = 48
    assert c2["i0"][0] == 7 and c2["ox"][0] == 7             # cells 7..10: d = -8, 0, 8, 16
    assert not crd["keep"][6] and not crd["keep"][7]
    # off-grid: U = 60 -> X = 124, i0 = 14, footprint 14..17 leaves [0, 16)
    assert not crd["keep"][3]
    assert crd["keep"][0] and crd["keep"][1] and crd["keep"][2]


def test_coords_hermitian_pairs_negate():
    prm = _prm(n=64)
    rng = np.random.default_rng(5)
    uvw = rng.uniform(-100, 100, (50, 3))
    f = np.array([oracle.C_LIGHT, 1.1 * oracle.C_LIGHT])
    crd = oracle.coords(uvw, f, prm, hermitian_pairs=True)
    n = crd["nvis"]
    np.testing.assert_array_equal(crd["U"][n:], -crd["U"][:n])
    np.testing.assert_array_equal(crd["V"][n:], -crd["V"][:n])
    np.testing.assert_array_equal(crd["plane"][n:], crd["plane"][:n])
    np.testing.assert_array_equal(crd["conj"][n:], np.repeat(uvw[:, 2] > 0, 2))


# ---------------------------------------------------------------- gridding identities
@pytest.fixture(scope="module")
def parity_case():
    cfg = synth.config("parity")
    ob = synth.observe(cfg)
    prm = oracle.Params(cfg.n, cfg.cell, cfg.n_w, ob.w_max, cfg.s_min, cfg.s_max, cfg.oversample)
    tabs, _ = oracle.wkernels(prm)
    return cfg, ob, prm, tabs


def _tap_sums(crd, tabs, prm):
    """sum over a visibility's S x S taps of its (possibly conjugated) kernel."""
    out = np.zeros(len(crd["keep"]), np.complex128)
    for k in np.nonzero(crd["keep"])[0]:
        t = tabs[crd["plane"][k]]
        s = t[crd["oy"][k]::prm.os, crd["ox"][k]::prm.os].sum()
        out[k] = np.conj(s) if crd["conj"][k] else s
    return out


def test_sum_of_weights_identity(parity_case):
    """sum over cells of G = sum_k c_k * (sum of its taps), exactly; ~ sum W."""
    cfg, ob, prm, tabs = parity_case
    crd = oracle.coords(ob.uvw, ob.freqs, prm)
    c = wproj.gridded_values(np.ones_like(ob.vis), ob.weight, crd)
    g = oracle.grid(crd, c, tabs, prm)
    ts = _tap_sums(crd, tabs, prm)
    expect = np.sum(c * ts)
    assert abs(g.sum() - expect) < 1e-11 * abs(expect)
    assert abs(g.sum().real / oracle.sum_weights(ob.weight, crd) - 1) < 0.02


def test_unit_point_source_centre_pixel(parity_case):
    """V = 1, W = 1: the corrected image at the phase centre is (1/sum W) Re sum_k s_k
    (s_k its tap sum, t(0) = 1), which is ~1."""
    cfg, ob, prm, tabs = parity_case
    crd = oracle.coords(ob.uvw, ob.freqs, prm)
    ones = np.ones(ob.vis.shape, np.complex64)
    c = wproj.gridded_values(ones, None, crd)
    g = oracle.grid(crd, c, tabs, prm)
    sw = oracle.sum_weights(None, crd)
    img = oracle.fft_to_image(g, sw, prm)
    ts = _tap_sums(crd, tabs, prm)
    expect = np.sum(ts).real / sw
    assert abs(img[prm.n // 2, prm.n // 2] - expect) < 1e-12
    assert abs(expect - 1.0) < 0.02


def test_hermitian_mirror(parity_case):
    """grid(conj V, -uvw)[(N-h) % N, (N-g) % N] == conj grid(V, uvw)[h, g] for visibilities
    whose footprint is not at a tie and stays inside the grid for both signs."""
    cfg, ob, prm, tabs = parity_case
    rng = np.random.default_rng(11)
    vis, wt = synth.random_visibilities(ob.uvw.shape[0], 1, 11)
    c1 = oracle.coords(ob.uvw, ob.freqs, prm)
    c2 = oracle.coords(-ob.uvw, ob.freqs, prm)
    half = c1["support"] * prm.os // 2
    x = c1["U"] + prm.n // 2 * prm.os
    y = c1["V"] + prm.n // 2 * prm.os
    tie = ((x - half) % prm.os == 0) | ((y - half) % prm.os == 0)
    ok = c1["keep"] & c2["keep"] & ~tie & (c1["i0"] > 0) & (c1["j0"] > 0)
    assert ok.sum() > 1000
    for crd in (c1, c2):
        crd["keep"] = ok.copy()
    g1 = oracle.grid(c1, (wt * vis).ravel().astype(np.complex128), tabs, prm)
    g2 = oracle.grid(c2, (wt * np.conj(vis)).ravel().astype(np.complex128), tabs, prm)
    n = prm.n
    idx = (n - np.arange(n)) % n
    mirrored = g2[np.ix_(idx, idx)]
    np.testing.assert_allclose(mirrored, np.conj(g1), rtol=0, atol=1e-12 * np.abs(g1).max())
    del rng


def test_degrid_is_adjoint_of_grid(parity_case):
    cfg, ob, prm, tabs = parity_case
    crd = oracle.coords(ob.uvw, ob.freqs, prm)
    rng = np.random.default_rng(3)
    c = rng.standard_normal(crd["keep"].size) + 1j * rng.standard_normal(crd["keep"].size)
    c[~crd["keep"]] = 0
    g = synth.random_grid(prm.n, 4).astype(np.complex128)
    lhs = np.vdot(oracle.grid(crd, c, tabs, prm), g)
    rhs = np.vdot(c, oracle.degrid(crd, g, tabs, prm))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_threaded_grid_matches_serial(parity_case):
    cfg, ob, prm, tabs = parity_case
    crd = oracle.coords(ob.uvw, ob.freqs, prm)
    c = wproj.gridded_values(ob.vis, ob.weight, crd)
    g1 = oracle.grid(crd, c, tabs, prm, threads=1)
    g4 = oracle.grid(crd, c, tabs, prm, threads=4)
    np.testing.assert_allclose(g4, g1, rtol=0, atol=1e-12 * np.abs(g1).max())


def test_w0_reduction_against_plain_separable_gridder():
    """Nw = 1 (no w-term): W-projection reduces to plain gridding with the separable
    taper-transform kernel. Checked against a separately written numpy gridder."""
    prm = oracle.Params(n=64, cell=1.0 * ARCMIN, n_w=1, w_max=1.0, s_min=7, s_max=7, os=8)
    rng = np.random.default_rng(7)
    f = np.array([1.4e9])
    uvw = rng.uniform(-1, 1, (300, 3)) * (20 / (prm.field * f[0] / oracle.C_LIGHT))
    crd = oracle.coords(uvw, f, prm)
    c = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    tabs, nu = oracle.wkernels(prm)
    g = oracle.grid(crd, c, tabs, prm)
    # separate gridder: 1D kernel of the taper, outer product per visibility
    m, s, os_ = prm.screen_m, 7, 8
    j = np.arange(m) - (m - 1) // 2
    tj = oracle.taper(2.0 * j / m, oracle.taper_c(7))
    d = np.arange(-s * os_ // 2 + 1, s * os_ // 2 + 1)
    k1 = (tj[None, :] * np.cos(2 * np.pi * np.outer(d, j) / (os_ * m))).sum(1) / math.sqrt(nu)
    ref = np.zeros((64, 64), np.complex128)
    for k in np.nonzero(crd["keep"])[0]:
        kx = k1[crd["ox"][k]::os_]
        ky = k1[crd["oy"][k]::os_]
        ref[crd["j0"][k]:crd["j0"][k] + s, crd["i0"][k]:crd["i0"][k] + s] += c[k] * np.outer(ky, kx)
    assert crd["keep"].sum() > 200
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_image_transform_bruteforce():
    """fft_to_image equals its defining sum (small grid, no taper)."""
    n = 8
    rng = np.random.default_rng(2)
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    prm = oracle.Params(n=n, cell=1e-3, n_w=1, w_max=1.0, s_min=4, s_max=4, os=2)
    img = oracle.fft_to_image(g, 2.5, prm, taper_correct=False)
    h = np.arange(n) - n // 2
    e = np.exp(2j * np.pi * np.outer(h, h) / n)          # [j][h] = exp(2 pi i (j-N/2)(h-N/2)/N)
    ref = np.real(e @ g @ e.T) / 2.5
    np.testing.assert_allclose(img, ref, rtol=0, atol=1e-12)


def test_image_adjoint_identity():
    n = 16
    prm = oracle.Params(n=n, cell=1e-3, n_w=1, w_max=1.0, s_min=6, s_max=6, os=2)
    rng = np.random.default_rng(8)
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    x = rng.standard_normal((n, n))
    lhs = np.sum(oracle.fft_to_image(g, 3.0, prm) * x)
    rhs = np.real(np.vdot(g, oracle.image_to_grid_adjoint(x, 3.0, prm)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


# ---------------------------------------------------------------- direct DFT
def _dft_case(s, n=64, nvis=300, seed=21):
    """Visibilities on the oversampling lattice and on plane w values, from sources in the
    inner half of the field; only kernel truncation/aliasing separates W-projection from
    the direct DFT with the exact (n - 1) term."""
    os_, n_w, w_max = 8, 8, 6000.0
    cell = 1.0 * ARCMIN
    prm = oracle.Params(n=n, cell=cell, n_w=n_w, w_max=w_max, s_min=s, s_max=s, os=os_)
    rng = np.random.default_rng(seed)
    f = np.array([oracle.C_LIGHT])
    lim = (n // 2 - 6) * os_
    uu = rng.integers(-lim, lim, nvis) / (os_ * prm.field)
    vv = rng.integers(-lim, lim, nvis) / (os_ * prm.field)
    ww = rng.integers(-(n_w - 1), n_w, nvis) * (w_max / (n_w - 1))
    uvw = np.stack([uu, vv, ww], 1)
    src = np.array([[0.2, -0.15, 1.0], [-0.1, 0.22, 0.7], [0.05, 0.03, 0.4]])
    src[:, :2] *= prm.field
    vis = synth.predict_numpy(uvw, f, src)
    return prm, uvw, f, vis


def _wproj_vs_dft(s):
    prm, uvw, f, vis = _dft_case(s)
    crd = oracle.coords(uvw, f, prm)
    assert crd["keep"].all()
    tabs, _ = oracle.wkernels(prm)
    c = vis.ravel()
    g = oracle.grid(crd, c, tabs, prm)
    sw = float(len(c))
    img = oracle.fft_to_image(g, sw, prm)
    ref = oracle.dirty_image_dft(uvw, f, c, prm.n, prm.cell) / sw
    q = prm.n // 4
    inner = (slice(q, 3 * q), slice(q, 3 * q))
    return np.abs(img[inner] - ref[inner]).max() / np.abs(ref).max()


def test_wprojection_converges_to_direct_dft_with_support():
    """W-projection approximates the direct-DFT dirty image including the (n - 1) w-term;
    with coordinates on the lattice the remaining error is kernel truncation, which falls
    as the full support grows 5 -> 7 -> 9."""
    errs = [_wproj_vs_dft(s) for s in (5, 7, 9)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[1] < 2e-3, errs
    assert errs[2] < 5e-4, errs


def test_wterm_matters():
    """Control: dropping the (n - 1) term in the DFT gives a much larger difference, so the
    agreement above is due to the W-kernels, not to a negligible w-term."""
    prm, uvw, f, vis = _dft_case(9)
    crd = oracle.coords(uvw, f, prm)
    tabs, _ = oracle.wkernels(prm)
    g = oracle.grid(crd, vis.ravel(), tabs, prm)
    img = oracle.fft_to_image(g, float(vis.size), prm)
    ref2d = oracle.dirty_image_dft(uvw, f, vis.ravel(), prm.n, prm.cell, w_exact=False) / vis.size
    q = prm.n // 4
    inner = (slice(q, 3 * q), slice(q, 3 * q))
    err2d = np.abs(img[inner] - ref2d[inner]).max() / np.abs(ref2d).max()
    assert err2d > 20 * _wproj_vs_dft(9)


# ---------------------------------------------------------------- pins added for the remaining parts
@pytest.mark.parametrize("n_w,s_min,s_max,expect", [
    (1, 9, 9, [9]),                       # one plane: the paper's single full support (Sec. 3.1)
    (23, 9, 9, [9] * 23),                 # S_min == S_max: every plane the same
    (5, 8, 16, [8, 10, 12, 14, 16]),      # 8 p / 4 exact integers
    (5, 7, 9, [7, 7, 8, 9, 9]),           # 2 p / 4 = 0, .5, 1, 1.5, 2: ties go to the even integer
    (3, 8, 9, [8, 8, 9]),                 # 1 p / 2 = 0, .5, 1: the tie at p = 1 rounds down to 0
    (32, 8, 16, None),                    # checked entry by entry below
])
def test_plane_supports_hand_worked(n_w, s_min, s_max, expect):
    """S_p = S_min + rint((S_max - S_min) p / (Nw - 1)) with round-half-to-even, against
    values worked out by hand (a half-up or floor rule fails the tie rows)."""
    got = wproj.plane_supports(n_w, s_min, s_max).tolist()
    if expect is not None:
        assert got == expect
        return
    # 8 p / 31: p = 1 -> 0.258 (8), p = 2 -> 0.516 (9), p = 4 -> 1.032 (9), p = 6 -> 1.548 (10),
    # p = 29 -> 7.484 (15), p = 30 -> 7.742 (16), p = 31 -> 8 (16)
    assert len(got) == 32
    for p, s in {0: 8, 1: 8, 2: 9, 4: 9, 6: 10, 29: 15, 30: 16, 31: 16}.items():
        assert got[p] == s, (p, got[p], s)


def test_hermitian_pairs_grid_is_hermitian(parity_case):
    """A grid made with hermitian_pairs=True holds every sample and its conjugate at -uvw, so
    G[(N - h) % N, (N - g) % N] = conj G[h, g] wherever no footprint sits at a rounding tie or
    touches row/column 0 (whose mirror would be N). This pins `gridded_values` (the partner's
    W conj(V)) and the partner coordinates of `coords` together: dropping the conjugate, or
    giving the partner the original's conj flag or position, breaks the symmetry."""
    cfg, ob, prm, tabs = parity_case
    vis, wt = synth.random_visibilities(ob.uvw.shape[0], 1, 13)
    crd = oracle.coords(ob.uvw, ob.freqs, prm, hermitian_pairs=True)
    n_s = crd["nvis"]
    half = crd["support"] * prm.os // 2
    x = crd["U"] + prm.n // 2 * prm.os
    y = crd["V"] + prm.n // 2 * prm.os
    tie = ((x - half) % prm.os == 0) | ((y - half) % prm.os == 0)
    ok = crd["keep"] & ~tie & (crd["i0"] > 0) & (crd["j0"] > 0)
    both = ok[:n_s] & ok[n_s:]                 # a sample and its partner both qualify
    assert both.sum() > 1000
    crd["keep"] = np.concatenate([both, both])
    c = wproj.gridded_values(vis, wt, crd)
    g = oracle.grid(crd, c, tabs, prm)
    n = prm.n
    idx = (n - np.arange(n)) % n
    np.testing.assert_allclose(g[np.ix_(idx, idx)], np.conj(g), rtol=0, atol=1e-12 * np.abs(g).max())
    # the same grid without the partners is far from Hermitian (the check has teeth)
    crd["keep"] = np.concatenate([both, np.zeros_like(both)])
    g1 = oracle.grid(crd, c, tabs, prm)
    assert np.abs(g1[np.ix_(idx, idx)] - np.conj(g1)).max() > 0.1 * np.abs(g1).max()
