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


def _outputs(n):
    import torch
    g = torch.full((n, n), 7.0 + 3.0j, dtype=torch.complex64, device="cuda")   # must be overwritten
    sw = torch.zeros(1, dtype=torch.float64, device="cuda")
    nd = torch.zeros(1, dtype=torch.int64, device="cuda")
    return g, sw, nd


def _call(wp, uvw, f, vis, wt, out, pairs=False, accumulate=False):
    """wp_grid_noalloc through the C ABI into preallocated outputs; no host-side allocation of
    device memory happens here either."""
    import torch
    import paper_1905_03213_b300 as W
    g, sw, nd = out
    flags = (W.WP_HERMITIAN_PAIRS if pairs else 0) | (W.WP_ACCUMULATE if accumulate else 0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = W.lib.wp_grid_noalloc(wp._h, _ptr(uvw), _ptr(f), _ptr(vis), _ptr(wt), uvw.shape[0], f.shape[0], flags,
                               _ptr(g), _ptr(sw), _ptr(nd), stream)
    assert rc == 0, W.lib.wp_last_error(wp._h).decode()


def _noalloc(wp, uvw, f, vis, wt, pairs=False):
    import torch
    out = _outputs(wp.n)
    _call(wp, uvw, f, vis, wt, out, pairs=pairs)
    torch.cuda.synchronize()
    g, sw, nd = out
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


def test_noalloc_first_call_on_a_fresh_context_allocates_nothing():
    """A context that has never run wp_grid holds no coordinate scratch, so this call takes the
    path that recomputes the coordinates in the scatter pass. Across the call (after one
    warm-up call on another context has loaded the kernels), neither the device's free memory
    nor torch's reserved pool changes. Supports 6-10 (not only 7), several channels, weights,
    then an accumulating second call; the reference is wp_grid on a separate context."""
    import torch
    case = random_case(n=128, nrow=3000, nchan=3, n_w=6, s_min=6, s_max=10, seed=23)
    uvw, f, vis, wt = to_dev(case)
    warm = make_wproj(case)
    _noalloc(warm, uvw, f, vis, wt)                     # loads every kernel of the path
    ref = make_wproj(case)
    g_ref, sw_ref, nd_ref = ref.grid(uvw, f, vis, wt)
    g_ref2, sw_ref2, nd_ref2 = ref.grid(uvw[:1234].contiguous(), f, vis[:1234].contiguous(), wt[:1234].contiguous(),
                                        grid=g_ref.clone(), sum_w=sw_ref.clone(), n_dropped=nd_ref.clone(),
                                        accumulate=True)
    fresh = make_wproj(case)
    out = _outputs(fresh.n)
    uvw2, vis2, wt2 = uvw[:1234].contiguous(), vis[:1234].contiguous(), wt[:1234].contiguous()
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    _call(fresh, uvw, f, vis, wt, out)
    torch.cuda.synchronize()
    free1, reserved1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    assert (free1, reserved1) == (free0, reserved0), (free0 - free1, reserved1 - reserved0)
    g, sw, nd = out
    e1, _ = peak_rel(g.cpu().numpy(), g_ref.cpu().numpy())
    assert e1 < 1e-6, e1
    assert sw.item() == pytest.approx(sw_ref.item(), rel=1e-12) and nd.item() == nd_ref.item()
    # second call in a row, accumulating a ragged slice onto the first result
    _call(fresh, uvw2, f, vis2, wt2, out, accumulate=True)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    e2, _ = peak_rel(g.cpu().numpy(), g_ref2.cpu().numpy())
    assert e2 < 1e-6, e2
    assert sw.item() == pytest.approx(sw_ref2.item(), rel=1e-12) and nd.item() == nd_ref2.item()
