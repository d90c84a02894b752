"""W-projection gridding on one B300: thin Python binding of libwproj.so (include/wproj.h).

Every call marshals arguments (device pointers of torch tensors, the current CUDA stream)
into the C ABI; all computation runs in the library's CUDA kernels. There is no CPU
fallback: if libwproj.so is missing, importing the binding raises.

    wp = WProj(n=256, cell=..., n_w=16, w_max=..., support_min=7, support_max=7, oversample=8)
    wp.make_wkernels()
    grid, sum_w, n_dropped = wp.grid(uvw, freq, vis, weight)
    image = wp.fft_to_image(grid, sum_w)
"""
from __future__ import annotations

from ._abi import (  # noqa: F401
    LIB_PATH, PHASES, WP_ACCUMULATE, WP_COMPENSATED, WP_EINVAL, WP_ESTATE, WP_HERMITIAN_PAIRS, WP_KEEP_BINNING, WP_OK, WP_TABLE_BF16, WP_TABLE_F16,
    WP_TABLE_F32, WBatch, WProj,
    WProjError, lib, probe_fp32_fma, taper_eval_host,
)
