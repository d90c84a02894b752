"""FP64 CPU oracle for W-projection gridding -- TEST INFRASTRUCTURE, not part of the product.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import, call or link anything in this package. It shares no code with the CUDA library:
only the seeded input generators in ``synth`` serve both.

What it computes (W-projection wide-field imaging, Lao et al. 2019, and the method it
parallelises, W-projection after Cornwell et al. 2008, which the paper defers to in
Sec. 1 for the kernel): visibilities are convolved with per-w-plane kernels onto a 2D
uv grid (the gridding step of Sec. 2.1/2.2), the grid is inverse-FFT'd to the dirty
image (Fig. 1, Fig. 2 captions), and the image is divided by the taper. Degridding is
the adjoint map.

The paper never writes the W-projection formulas down, so each function states the
reading it implements; every reading is listed with its justification in the design
notes. All arithmetic is float64 except where a stored input is complex64/float32.

Pins (what ties this oracle to something other than itself) live in
tests/test_oracle_*.py: the direct DFT dirty image including the (n-1) w-term, a unit
point source, the w=0 separable reduction, the brute-force kernel DFT, Hermitian
mirror symmetry, the sum-of-weights identity, the adjoint dot-product identity, the
PSWF integral equation, and a brute-force image transform; the baseline grouping of
Sec. 2.2 (Eq. 5, Eq. 6) against the upper-triangle enumeration and brute-force sorting. No function here is
"parity unpinned".
"""
from .wproj import (  # noqa: F401
    C_LIGHT, Params, plane_supports, plane_w, default_screen_m, taper, taper_c,
    screen, wkernel_unnormalised, wkernel_dft_bruteforce, wkernels, coords, grid, degrid,
    fft_to_image, image_to_grid_adjoint, dirty_image_dft, sum_weights,
)
from .baselines import baseline_index, baseline_order, baseline_starts, n_baselines  # noqa: F401
