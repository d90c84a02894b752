"""CPU checks of the C ABI: the library loads, exports every declared function, validates
parameters on the host, and its host-side taper matches the oracle's (no device work)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "wproj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wp_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    import paper_1905_03213_b300 as W
    declared = _declared_functions()
    assert len(declared) >= 10
    raw = ctypes.CDLL(W.LIB_PATH)
    for name in declared:
        assert hasattr(raw, name), name
    assert set(declared) == set(W._abi.SYMBOLS)


def test_build_targets_sm103a():
    from paper_1905_03213_b300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


@pytest.mark.parametrize("s_min", [5, 7, 8, 12])
def test_library_taper_matches_oracle(s_min):
    import paper_1905_03213_b300 as W
    c = math.pi * s_min / 2
    x = np.concatenate([np.linspace(-1, 1, 101), [0.0, 1.0, -1.0]])
    # scipy's pro_ang1 (the oracle's route) loses digits as c grows; the library's Legendre
    # route is checked against the integral equation directly below
    tol = 5e-14 if s_min <= 8 else 2e-12
    np.testing.assert_allclose(W.taper_eval_host(c, x), oracle.taper(x, c), rtol=0, atol=tol)


@pytest.mark.parametrize("s_min", [4, 7, 12, 16, 24])
def test_library_taper_solves_prolate_integral_equation(s_min):
    import paper_1905_03213_b300 as W
    c = math.pi * s_min / 2
    y, wq = np.polynomial.legendre.leggauss(400)
    ty = W.taper_eval_host(c, y)
    lam = np.sum(wq * ty)
    x = np.linspace(-1, 1, 31)
    lhs = (np.cos(c * np.outer(x, y)) * wq * ty).sum(1) / lam
    np.testing.assert_allclose(lhs, W.taper_eval_host(c, x), rtol=0, atol=1e-13)


def test_library_taper_even_unit_and_rejects_bad_input():
    import paper_1905_03213_b300 as W
    c = math.pi * 7 / 2
    x = np.linspace(0, 1, 33)
    np.testing.assert_array_equal(W.taper_eval_host(c, -x), W.taper_eval_host(c, x))
    assert W.taper_eval_host(c, np.array([0.0]))[0] == pytest.approx(1.0, abs=1e-15)
    with pytest.raises(W.WProjError):
        W.taper_eval_host(c, np.array([1.5]))
    with pytest.raises(W.WProjError):
        W.taper_eval_host(-1.0, np.array([0.5]))


def _params(**kw):
    import paper_1905_03213_b300 as W
    base = dict(n=256, cell_rad=4.8e-5, n_w=16, w_max=4000.0, support_min=7, support_max=7, oversample=8,
                screen_m=0, table_type=0, tile_x=0, tile_y=0, device=0, units_per_cta=0)
    base.update(kw)
    return W._abi.Params(**base)


@pytest.mark.parametrize("bad", [
    dict(n=15), dict(n=8), dict(cell_rad=0.0), dict(cell_rad=float("nan")), dict(n_w=0), dict(w_max=0.0),
    dict(oversample=7), dict(oversample=0), dict(support_min=0), dict(support_min=9, support_max=8),
    dict(screen_m=64), dict(table_type=5), dict(tile_x=-1), dict(cell_rad=0.01, n=256),
    dict(units_per_cta=-1), dict(units_per_cta=65),
])
def test_create_rejects_invalid_parameters_on_host(bad):
    import paper_1905_03213_b300 as W
    h = ctypes.c_void_p()
    prm = _params(**bad)
    rc = W.lib.wp_create(ctypes.byref(h), ctypes.byref(prm))
    assert rc == W._abi.WP_EINVAL
    assert not h.value
    assert W.lib.wp_last_error(None)


def test_null_arguments_rejected():
    import paper_1905_03213_b300 as W
    lib = W.lib
    assert lib.wp_create(None, None) == W._abi.WP_EINVAL
    assert lib.wp_make_wkernels(None, None) == W._abi.WP_EINVAL
    assert lib.wp_grid(None, None, None, None, None, 0, 1, 0, None, None, None, None) == W._abi.WP_EINVAL
    assert lib.wp_profile_read(None, None, None, None) == W._abi.WP_EINVAL
    lib.wp_destroy(None)
