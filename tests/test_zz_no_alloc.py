"""The allocation-free gridding call (wp_grid_noalloc) against wp_grid, through the C ABI.

wp_grid_noalloc serves callers that must not allocate device memory while gridding (a
framework that already owns the whole device through its own memory pool, or a loop that
cannot afford an allocation's stall); its scratch is a fixed device array inside the
library. This file is collected last so that a run stopping at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""
import ctypes

import pytest

from gpu_cases import make_wproj, parity_case, peak_rel, random_case, to_dev

pytestmark = pytest.mark.gpu


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _noalloc(wp, uvw, f, vis, wt, pairs=False):
    import torch
    import paper_1905_03213_b300 as W
    n = wp.n
    g = torch.full((n, n), 7.0 + 3.0j, dtype=torch.complex64, device="cuda")   # must be overwritten
    sw = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd = torch.zeros(1, dtype=torch.int64, device="cuda")
    flags = W.WP_HERMITIAN_PAIRS if pairs else 0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = W.lib.wp_grid_noalloc(wp._h, _ptr(uvw), _ptr(f), _ptr(vis), _ptr(wt), uvw.shape[0], f.shape[0], flags,
                               _ptr(g), _ptr(sw), _ptr(nd), stream)
    assert rc == 0, W.lib.wp_last_error(wp._h).decode()
    torch.cuda.synchronize()
    return g.cpu().numpy(), sw.item(), nd.item()


def test_noalloc_matches_grid_on_two_calls_in_a_row():
    import torch
    assert torch.cuda.is_available()
    # call 1: the parity workload (21,060 visibilities, weights)
    case = parity_case(pairs=False, weights=True)
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    g_ref, sw_ref, nd_ref = wp.grid(uvw, f, vis, wt)
    g1, sw1, nd1 = _noalloc(wp, uvw, f, vis, wt)
    e1, _ = peak_rel(g1, g_ref.cpu().numpy())
    assert e1 < 1e-6, e1
    assert sw1 == pytest.approx(sw_ref.item(), rel=1e-12) and nd1 == nd_ref.item()
    # call 2, right after: different inputs (a ragged slice, Hermitian pairs, no weights), so
    # records left in the shared scratch by call 1 must not leak into the result
    k = 9_001
    uvw2, vis2 = uvw[:k].contiguous(), vis[:k].contiguous()
    g_ref2, sw_ref2, nd_ref2 = wp.grid(uvw2, f, vis2, None, hermitian_pairs=True)
    g2, sw2, nd2 = _noalloc(wp, uvw2, f, vis2, None, pairs=True)
    e2, _ = peak_rel(g2, g_ref2.cpu().numpy())
    assert e2 < 1e-6, e2
    assert sw2 == pytest.approx(sw_ref2.item(), rel=1e-12) and nd2 == nd_ref2.item()


def test_noalloc_rejects_calls_beyond_its_scratch():
    import torch
    import paper_1905_03213_b300 as W
    case = random_case(n=64, nrow=10, nchan=1)
    wp = make_wproj(case)
    uvw, f, vis, wt = to_dev(case)
    g = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 2^20 rows with pairs = 2^21 gridded visibilities: rejected before any device work
    rc = W.lib.wp_grid_noalloc(wp._h, _ptr(uvw), _ptr(f), _ptr(vis), None, 1 << 20, 1, W.WP_HERMITIAN_PAIRS,
                               _ptr(g), None, None, stream)
    assert rc == W._abi.WP_EINVAL
    assert b"1048576" in W.lib.wp_last_error(wp._h)
    assert torch.count_nonzero(g).item() == 0
