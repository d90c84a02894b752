"""The differentiable forward model V = degrid(image_to_grid(X)) behind torch.autograd.

Checks: image_to_grid against the oracle's adjoint of the imaging transform; the GPU pair
image_to_grid / fft_to_image as adjoints; the autograd vector-Jacobian product by the
dot-product test; the gradient of ||V(X) - V0||^2 against central finite differences on 100
pixels and against the float64 oracle's gradient 2 Re(A^H (A X - V0)).
"""
import numpy as np
import pytest

import oracle
from oracle import wproj
import synth
from gpu_cases import inner, make_wproj, peak_rel, random_case, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def _inner_only(torch, x):
    """Zero outside the inner half |l|, |m| < L/4: the forward model divides by t(l) t(m), which
    falls to ~1e-8 at the field edge, so a model image lives where the taper is not near zero."""
    n = x.shape[0]
    m = torch.zeros_like(x)
    m[n // 4: 3 * n // 4, n // 4: 3 * n // 4] = 1
    return x * m


def _diff_setup(torch):
    """The differentiable workload: 64 antennas, 1.0M visibilities, 2048^2, 32 planes, support 12."""
    import paper_1905_03213_b300 as W
    cfg = synth.config("diff")
    ob = synth.observe(cfg, device="cuda")
    wp = W.WProj(n=cfg.n, cell=cfg.cell, n_w=cfg.n_w, w_max=ob.w_max, support_min=cfg.s_min,
                 support_max=cfg.s_max, oversample=cfg.oversample)
    wp.make_wkernels()
    freq = torch.as_tensor(ob.freqs, dtype=torch.float64, device="cuda")
    return wp, ob.uvw.contiguous(), freq, ob.vis.contiguous(), cfg


@pytest.mark.parametrize("sum_w,taper", [(None, True), (3.5, True), (None, False)])
def test_image_to_grid_matches_oracle(torch_cuda, sum_w, taper):
    torch = torch_cuda
    case = random_case(n=128)
    wp = make_wproj(case)
    x = np.random.default_rng(3).standard_normal((128, 128)).astype(np.float32)
    sw = None if sum_w is None else torch.tensor([sum_w], dtype=torch.float64, device="cuda")
    got = wp.image_to_grid(torch.from_numpy(x).cuda(), sum_w=sw, taper_correct=taper).cpu().numpy()
    ref = oracle.image_to_grid_adjoint(x.astype(np.float64), 1.0 if sum_w is None else sum_w, case.prm,
                                       taper_correct=taper)
    e, _ = peak_rel(got, ref)
    assert e < 1e-5, e


def test_image_to_grid_is_adjoint_of_fft_to_image(torch_cuda):
    torch = torch_cuda
    case = random_case(n=128)
    wp = make_wproj(case)
    rng = np.random.default_rng(4)
    G = (rng.standard_normal((128, 128)) + 1j * rng.standard_normal((128, 128))).astype(np.complex64)
    X = rng.standard_normal((128, 128)).astype(np.float32)
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    img = wp.fft_to_image(torch.from_numpy(G).cuda(), one).cpu().numpy().astype(np.float64)
    AX = wp.image_to_grid(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.complex128)
    lhs = float(np.sum(img * X))
    rhs = float(np.real(np.vdot(AX, G.astype(np.complex128))))
    assert abs(lhs - rhs) < 1e-5 * np.sqrt(np.sum(img ** 2) * np.sum(X.astype(np.float64) ** 2))


def test_autograd_dot_product(torch_cuda):
    """Re <A X, R> = <X, backward(R)> on the differentiable workload (float32 vs float64 sums)."""
    torch = torch_cuda
    from paper_1905_03213_b300.autograd import predict
    wp, uvw, freq, _, cfg = _diff_setup(torch)
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    X = _inner_only(torch, torch.randn((cfg.n, cfg.n), generator=g, device="cuda", dtype=torch.float32) * 1e-3)
    R = torch.randn((uvw.shape[0], 1, 2), generator=g, device="cuda", dtype=torch.float32)
    R = torch.view_as_complex(R.contiguous())
    Xr = X.clone().requires_grad_(True)
    V = predict(wp, Xr, uvw, freq)
    (gx,) = torch.autograd.grad(torch.real(torch.vdot(R.ravel(), V.ravel())), Xr)
    lhs = torch.real(torch.vdot(V.ravel().to(torch.complex128), R.ravel().to(torch.complex128))).item()
    rhs = torch.sum(X.to(torch.float64) * gx.to(torch.float64)).item()
    assert abs(lhs - rhs) < 1e-5 * max(abs(lhs), 1e-30), (lhs, rhs)


def test_autograd_finite_differences_100_pixels(torch_cuda):
    """dL/dX at 100 random inner-half pixels against central differences of the float64 loss
    (the loss is quadratic in X, so the central difference is exact up to rounding)."""
    torch = torch_cuda
    from paper_1905_03213_b300.autograd import predict
    wp, uvw, freq, V0, cfg = _diff_setup(torch)
    n = cfg.n
    g = torch.Generator(device="cuda")
    g.manual_seed(12)
    X = _inner_only(torch, torch.rand((n, n), generator=g, device="cuda", dtype=torch.float32) * 1e-3)

    def loss(img):
        V = predict(wp, img, uvw, freq)
        return torch.sum(torch.abs(V.to(torch.complex128) - V0.to(torch.complex128)) ** 2)

    Xr = X.clone().requires_grad_(True)
    L = torch.sum(torch.abs(predict(wp, Xr, uvw, freq) - V0) ** 2)
    (grad,) = torch.autograd.grad(L, Xr)
    rng = np.random.default_rng(13)
    pix = rng.integers(n // 4, 3 * n // 4, size=(100, 2))
    h = 0.25
    fd = []
    with torch.no_grad():
        for j, i in pix:
            Xp = X.clone()
            Xp[j, i] += h
            Xm = X.clone()
            Xm[j, i] -= h
            fd.append(((loss(Xp) - loss(Xm)) / (2 * h)).item())
    fd = np.array(fd)
    gp = grad[pix[:, 0], pix[:, 1]].double().cpu().numpy()
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(gp - fd).max() < 1e-3 * scale, (np.abs(gp - fd).max(), scale)


def test_autograd_gradient_matches_oracle(torch_cuda):
    """x.grad of ||degrid(image_to_grid(X)) - V0||^2 against the float64 oracle's gradient."""
    torch = torch_cuda
    from paper_1905_03213_b300.autograd import predict
    case = random_case(n=128, nrow=1500, nchan=2, s_min=5, s_max=12)
    wp = make_wproj(case)
    uvw, f, vis, _ = to_dev(case)
    X = np.zeros((128, 128), np.float32)
    X[32:96, 32:96] = np.random.default_rng(21).random((64, 64)) * 0.1
    Xr = torch.from_numpy(X).cuda().requires_grad_(True)
    V = predict(wp, Xr, uvw, f)
    L = torch.sum(torch.abs(V - vis) ** 2)
    (grad,) = torch.autograd.grad(L, Xr)
    prm = case.prm
    crd = oracle.coords(case.uvw, case.freqs, prm)
    AX = oracle.degrid(crd, oracle.image_to_grid_adjoint(X.astype(np.float64), 1.0, prm), case.tables,
                       prm).reshape(case.vis.shape)
    r = 2.0 * (AX - case.vis.astype(np.complex128))
    ref = oracle.fft_to_image(oracle.grid(crd, wproj.gridded_values(r, None, crd), case.tables, prm), 1.0, prm)
    e, _ = peak_rel(inner(grad.cpu().numpy()), inner(ref))
    assert e < 1e-5, e


def test_autograd_gradient_matches_oracle_differentiable_geometry(torch_cuda):
    """The oracle gradient at the differentiable workload's own geometry (2048^2, 32 planes,
    support 12, oversampling 8) on a row subset: its first 60,000 rows (the first 30 time
    samples of all 2016 baselines), a model image over the inner half."""
    torch = torch_cuda
    import paper_1905_03213_b300 as W
    from paper_1905_03213_b300.autograd import predict
    cfg = synth.config("diff")
    enu = synth.antenna_enu(cfg.n_ant, cfg.radius_m, cfg.height_m, np.random.default_rng(cfg.seed))
    uvw_all = synth.uvw_metres(enu, synth.SITE_LAT, cfg.dec, synth.hour_angles(cfg.n_time, cfg.duration_h))
    w_max = float(np.abs(uvw_all[:, 2]).max() * np.max(cfg.freqs) / synth.C_LIGHT)   # planes of the full run
    rows = 60_000
    uvw = np.ascontiguousarray(uvw_all[:rows])
    freqs = np.asarray(cfg.freqs, dtype=np.float64)
    vis, _ = synth.random_visibilities(rows, len(freqs), 61)
    prm = oracle.Params(cfg.n, cfg.cell, cfg.n_w, w_max, cfg.s_min, cfg.s_max, cfg.oversample)
    tabs, _ = oracle.wkernels(prm)
    wp = W.WProj(n=cfg.n, cell=cfg.cell, n_w=cfg.n_w, w_max=w_max, support_min=cfg.s_min,
                 support_max=cfg.s_max, oversample=cfg.oversample)
    wp.make_wkernels()
    n = cfg.n
    X = np.zeros((n, n), np.float32)
    X[n // 4: 3 * n // 4, n // 4: 3 * n // 4] = np.random.default_rng(62).random((n // 2, n // 2)) * 1e-3
    Xr = torch.from_numpy(X).cuda().requires_grad_(True)
    d_uvw = torch.from_numpy(uvw).cuda()
    d_f = torch.from_numpy(freqs).cuda()
    d_vis = torch.from_numpy(vis).cuda()
    L = torch.sum(torch.abs(predict(wp, Xr, d_uvw, d_f) - d_vis) ** 2)
    (grad,) = torch.autograd.grad(L, Xr)
    crd = oracle.coords(uvw, freqs, prm)
    assert crd["keep"].sum() > 0.9 * rows
    AX = oracle.degrid(crd, oracle.image_to_grid_adjoint(X.astype(np.float64), 1.0, prm), tabs, prm,
                       threads=8).reshape(vis.shape)
    r = 2.0 * (AX - vis.astype(np.complex128))
    ref = oracle.fft_to_image(oracle.grid(crd, wproj.gridded_values(r, None, crd), tabs, prm, threads=8), 1.0, prm)
    e, _ = peak_rel(inner(grad.cpu().numpy()), inner(ref))
    assert e < 1e-5, e
