/*
 * FP64 gridding and degridding loops of the oracle (test infrastructure only).
 *
 * Convolutional gridding (Sec. 2.1 and Fig. 1: the gridding loop over rows, each
 * visibility convolved with its W-kernel onto the uv plane; Sec. 2.2: the kernel has
 * C_full x C_full taps per visibility):
 *     G[j0 + b][i0 + a] += c_k * K_k[b*os + oy_k][a*os + ox_k],   a, b in [0, S_p)
 * with K_k the W-kernel of the visibility's w-plane p, conjugated when w < 0.
 *
 * Degridding is the adjoint of that map (Sec. 2 cites gridding and degridding as the
 * pair of operations being accelerated):
 *     out_k = sum_{a,b} G[j0 + b][i0 + a] * conj(K_k[b*os + oy_k][a*os + ox_k])
 *
 * Multi-threaded gridding follows the paper's OpenMP scheme (Sec. 2.1, Fig. 1): each
 * thread takes an equal share of the visibilities and grids them into a private
 * sub-grid, and the private grids are summed onto the full plane at the end.
 *
 * Table layout: plane p is a dense E_p x E_p complex array (E_p = S_p * os), row index
 * ey = b*os + oy, column index ex = a*os + ox, interleaved (re, im) doubles, starting at
 * tab + 2 * tab_off[p]. Grid: n x n complex, row = v (j), column = u (i), interleaved.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void grid_range(int64_t k_begin, int64_t k_end, const int32_t* i0, const int32_t* j0,
                       const int32_t* ox, const int32_t* oy, const int32_t* plane,
                       const uint8_t* conj, const double* c, const int32_t* supp,
                       const int64_t* tab_off, const double* tab, int32_t os, int32_t n,
                       double* g) {
  for (int64_t k = k_begin; k < k_end; ++k) {
    const int32_t p = plane[k], s = supp[p], e = s * os;
    const double* t = tab + 2 * tab_off[p];
    const double cr = c[2 * k], ci = c[2 * k + 1];
    const double sgn = conj[k] ? -1.0 : 1.0;
    for (int32_t b = 0; b < s; ++b) {
      const int64_t row = (int64_t)(j0[k] + b) * n;
      const int32_t ey = b * os + oy[k];
      for (int32_t a = 0; a < s; ++a) {
        const int32_t ex = a * os + ox[k];
        const double kr = t[2 * ((int64_t)ey * e + ex)];
        const double ki = sgn * t[2 * ((int64_t)ey * e + ex) + 1];
        double* cell = g + 2 * (row + i0[k] + a);
        cell[0] += cr * kr - ci * ki;
        cell[1] += cr * ki + ci * kr;
      }
    }
  }
}

/* Returns 0 on success, 1 if a private grid could not be allocated. */
int oracle_grid(int64_t nvis, const int32_t* i0, const int32_t* j0, const int32_t* ox,
                const int32_t* oy, const int32_t* plane, const uint8_t* conj, const double* c,
                const int32_t* supp, const int64_t* tab_off, const double* tab, int32_t os,
                int32_t n, double* grid, int32_t nthreads) {
  const int64_t cells = (int64_t)n * n;
  if (nthreads <= 1) {
    grid_range(0, nvis, i0, j0, ox, oy, plane, conj, c, supp, tab_off, tab, os, n, grid);
    return 0;
  }
  double** priv = (double**)calloc((size_t)nthreads, sizeof(double*));
  if (!priv) return 1;
  int failed = 0;
  for (int t = 0; t < nthreads; ++t) {
    priv[t] = (double*)calloc((size_t)(2 * cells), sizeof(double));
    if (!priv[t]) failed = 1;
  }
  if (!failed) {
#pragma omp parallel for num_threads(nthreads) schedule(static, 1)
    for (int t = 0; t < nthreads; ++t) {
      const int64_t kb = nvis * t / nthreads, ke = nvis * (t + 1) / nthreads;
      grid_range(kb, ke, i0, j0, ox, oy, plane, conj, c, supp, tab_off, tab, os, n, priv[t]);
    }
    for (int t = 0; t < nthreads; ++t)
      for (int64_t q = 0; q < 2 * cells; ++q) grid[q] += priv[t][q];
  }
  for (int t = 0; t < nthreads; ++t) free(priv[t]);
  free(priv);
  return failed;
}

int oracle_degrid(int64_t nvis, const int32_t* i0, const int32_t* j0, const int32_t* ox,
                  const int32_t* oy, const int32_t* plane, const uint8_t* conj,
                  const int32_t* supp, const int64_t* tab_off, const double* tab, int32_t os,
                  int32_t n, const double* grid, double* out, int32_t nthreads) {
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
  for (int64_t k = 0; k < nvis; ++k) {
    const int32_t p = plane[k], s = supp[p], e = s * os;
    const double* t = tab + 2 * tab_off[p];
    /* conj(K_k): K_k is K (w >= 0) or conj(K) (w < 0) */
    const double sgn = conj[k] ? 1.0 : -1.0;
    double sr = 0.0, si = 0.0;
    for (int32_t b = 0; b < s; ++b) {
      const int64_t row = (int64_t)(j0[k] + b) * n;
      const int32_t ey = b * os + oy[k];
      for (int32_t a = 0; a < s; ++a) {
        const int32_t ex = a * os + ox[k];
        const double kr = t[2 * ((int64_t)ey * e + ex)];
        const double ki = sgn * t[2 * ((int64_t)ey * e + ex) + 1];
        const double* cell = grid + 2 * (row + i0[k] + a);
        sr += cell[0] * kr - cell[1] * ki;
        si += cell[0] * ki + cell[1] * kr;
      }
    }
    out[2 * k] = sr;
    out[2 * k + 1] = si;
  }
  (void)n;
  return 0;
}
