// The paper's own GPU gridding scheme, kept as a comparison variant of the binned kernels.
//
// Sec. 2.2 of Lao et al. 2019: the visibilities are grouped by baseline and ordered by time
// (the baseline index of Eq. 5 from the two antenna IDs, the per-baseline sample counts C and
// their prefix sum, Eq. 6, giving each baseline's start index), and the gridding kernel gives
// every (baseline, support tap) one thread: along the baseline's time samples the thread keeps
// the running sum of its tap in a register while the grid point stays the same and adds it to
// the grid with an atomic when the point moves (Fig. 2; thread blocks of 256 in the paper).
// The flush is a non-returning vector reduction (red.global.add.v2.f32).
//
// Here: k_baseline_index (Eq. 5), a count and an exclusive scan (Eq. 6), a scatter into each
// baseline's range, then a per-baseline sort by row index so that every baseline's samples are
// in time order whatever order the scatter's atomics produced. k_grid_baseline runs one CTA per
// (baseline, channel[, Hermitian partner]) with one thread per tap of the largest support, on
// the coordinates that wp_coords computes (the same float64 decisions as wp_grid).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "warp_common.cuh"

namespace wp {

namespace {

// Eq. 5: I_B = (-S^2 + 2 S N_ant + S) / 2 + |I_ant1 - I_ant2|, S = min(I_ant1, I_ant2); the
// index counts autocorrelations, so it runs over [0, N_ant (N_ant + 1) / 2).
__global__ void k_baseline_index(const int32_t* __restrict__ ant1, const int32_t* __restrict__ ant2, int64_t nrow,
                                 int32_t n_ant, int32_t* __restrict__ bidx, uint32_t* __restrict__ count) {
  const int32_t nb = n_ant * (n_ant + 1) / 2;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrow; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a1 = ant1[r], a2 = ant2[r];
    if (a1 < 0 || a2 < 0 || a1 >= n_ant || a2 >= n_ant) {  // no baseline: counted in slot nb
      bidx[r] = nb;
      atomicAdd(&count[nb], 1u);
      continue;
    }
    const int64_t s = a1 < a2 ? a1 : a2;
    const int64_t ib = (-s * s + 2 * s * n_ant + s) / 2 + (a1 > a2 ? a1 - a2 : a2 - a1);
    bidx[r] = (int32_t)ib;
    atomicAdd(&count[ib], 1u);
  }
}

// Eq. 6 for a modest number of baselines: one CTA, sequential chunks of a block-wide scan.
// start[0..nb] (start[nb] = rows with a baseline) and cursor[0..nb] (cursor[nb] = start[nb],
// where the rows without one go).
__global__ void k_baseline_start(const uint32_t* __restrict__ count, int32_t nb, uint32_t* __restrict__ start,
                                 uint32_t* __restrict__ cursor) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < nb; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < nb ? count[i] : 0u;
    uint32_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t t = lane < nw ? warp_sums[lane] : 0u;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, t, off);
        if (lane >= off) t += y;
      }
      if (lane < nw) warp_sums[lane] = t;
    }
    __syncthreads();
    const uint32_t excl = carry + (warp ? warp_sums[warp - 1] : 0u) + x - v;
    if (i < nb) {
      start[i] = excl;
      cursor[i] = excl;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) start[nb] = cursor[nb] = carry;
}

__global__ void k_baseline_scatter(const int32_t* __restrict__ bidx, int64_t nrow, uint32_t* __restrict__ cursor,
                                   int32_t* __restrict__ perm) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrow; r += (int64_t)gridDim.x * blockDim.x)
    perm[atomicAdd(&cursor[bidx[r]], 1u)] = (int32_t)r;
}

// Sorts each baseline's range of perm by row index (rows are time-ordered in the caller's
// layout) with an in-shared-memory bitonic sort; one CTA per baseline, ranges of up to
// kSortCap rows (longer ranges are left in scatter order: still correct, only less reuse).
constexpr int kSortCap = 4096;
__global__ void k_baseline_sort(const uint32_t* __restrict__ start, int32_t nb, int32_t* __restrict__ perm) {
  __shared__ int32_t v[kSortCap];
  const int b = blockIdx.x;
  if (b >= nb) return;
  const uint32_t s0 = start[b], len = start[b + 1] - s0;
  if (len < 2 || len > (uint32_t)kSortCap) return;
  int m = 1;
  while (m < (int)len) m <<= 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = i < (int)len ? perm[s0 + i] : 0x7fffffff;
  __syncthreads();
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const int a = v[i], c = v[ixj];
          if ((a > c) == up) {
            v[i] = c;
            v[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < (int)len; i += blockDim.x) perm[s0 + i] = v[i];
}

template <class T>
__device__ __forceinline__ float2 tap_f2(const T* p);
template <>
__device__ __forceinline__ float2 tap_f2<float2>(const float2* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float2 tap_f2<__half2>(const __half2* p) {
  return __half22float2(__ldg(p));
}
template <>
__device__ __forceinline__ float2 tap_f2<BfWord>(const BfWord* p) {
  const uint32_t w = __ldg((const unsigned int*)p);
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w));
}

// One CTA per (baseline b, channel ch, partner h); thread (ta, tb) = tap column ta, row tb of
// the largest support. Coordinates: coords[k][8] as written by wp_coords (U, V, plane, conj,
// keep, i0, j0, ox | oy << 16), k = row * nchan + ch, partners at + nrow * nchan.
template <class T>
__global__ void __launch_bounds__(1024) k_grid_baseline(const int32_t* __restrict__ coords,
                                                        const uint32_t* __restrict__ start,
                                                        const int32_t* __restrict__ perm, int32_t nb,
                                                        int32_t nchan, int64_t nvis, int32_t smax,
                                                        const float2* __restrict__ vis,
                                                        const float* __restrict__ weight, Geometry g,
                                                        const T* __restrict__ tab,
                                                        const int64_t* __restrict__ tab_off,
                                                        float2* __restrict__ grid) {
  const int b = blockIdx.x % nb;
  const int rest = blockIdx.x / nb;
  const int ch = rest % nchan, h = rest / nchan;
  const int ta = threadIdx.x % smax, tb = threadIdx.x / smax;
  if (tb >= smax) return;
  float ar = 0.f, ai = 0.f;
  int64_t cell = -1;
  const uint32_t nrow = (uint32_t)(nvis / nchan);
  const uint32_t s0 = start[b], s1 = min(start[b + 1], nrow);
  for (uint32_t q = s0; q < s1; ++q) {
    const uint32_t row = (uint32_t)perm[q];
    if (row >= nrow) continue;                              // not a row index: skipped
    const int64_t kv = (int64_t)row * nchan + ch;
    const int32_t* c = coords + 8 * (kv + h * nvis);
    if (!c[4]) continue;                                    // dropped
    const int p = c[2], s = g.supp[p];
    const int64_t here = ta < s && tb < s ? (int64_t)(c[6] + tb) * g.n + (c[5] + ta) : -2;  // keep: inside
    if (here != cell) {                                     // the grid point moved: flush the register
      if (cell >= 0 && (ar != 0.f || ai != 0.f)) red_add2(&grid[cell], ar, ai);
      ar = ai = 0.f;
      cell = here;
    }
    if (here < 0) continue;
    const float wt = weight ? weight[kv] : 1.f;
    const float2 v = vis[kv];
    const float cr = wt * v.x, cim = wt * (h ? -v.y : v.y);
    const int ox = c[7] & 0xffff, oy = c[7] >> 16;
    const float2 k = tap_f2<T>(tab + tab_off[p] + ((int64_t)(oy * g.os + ox) * s + ta) * s + tb);
    const float ki = c[3] ? -k.y : k.y;                     // conj(K) for w < 0
    ar = fmaf(cr, k.x, fmaf(-cim, ki, ar));
    ai = fmaf(cim, k.x, fmaf(cr, ki, ai));
  }
  if (cell >= 0 && (ar != 0.f || ai != 0.f)) red_add2(&grid[cell], ar, ai);
}

// Kept-weight sum and dropped count of wp_coords' output (gridded visibility k has weight
// weight[k mod nvis], 1 without weights).
__global__ void k_kept_sums(const int32_t* __restrict__ coords, int64_t ng, int64_t nvis,
                            const float* __restrict__ weight, double* __restrict__ wsum,
                            unsigned long long* __restrict__ dropped) {
  double w = 0.0;
  unsigned long long d = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ng; k += (int64_t)gridDim.x * blockDim.x) {
    if (coords[8 * k + 4]) w += weight ? (double)weight[k % nvis] : 1.0;
    else ++d;
  }
  for (int off = 16; off > 0; off >>= 1) {
    w += __shfl_xor_sync(0xffffffffu, w, off);
    d += __shfl_xor_sync(0xffffffffu, d, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (w != 0.0) atomicAdd(wsum, w);
    if (d) atomicAdd(dropped, d);
  }
}

}  // namespace

cudaError_t launch_kept_sums(wp_ctx* ctx, const int32_t* coords, int64_t ng, int64_t nvis, const float* weight,
                             cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ctx->d_wsum, 0, sizeof(double), s);
  if (!e) e = cudaMemsetAsync(ctx->d_dropped, 0, sizeof(unsigned long long), s);
  if (e || ng == 0) return e;
  const int blocks = (int)std::min<int64_t>((ng + 255) / 256, (int64_t)ctx->nsm * 8);
  k_kept_sums<<<blocks, 256, 0, s>>>(coords, ng, nvis, weight, ctx->d_wsum, ctx->d_dropped);
  ++ctx->launches;
  return cudaGetLastError();
}

cudaError_t launch_baseline_order(wp_ctx* ctx, const int32_t* ant1, const int32_t* ant2, int64_t nrow,
                                  int32_t n_ant, int32_t* bidx, uint32_t* count, uint32_t* start,
                                  uint32_t* cursor, int32_t* perm, cudaStream_t s) {
  const int32_t nb = n_ant * (n_ant + 1) / 2;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint32_t) * (nb + 1), s);
  if (e) return e;
  const int blocks = (int)std::min<int64_t>((nrow + 255) / 256, (int64_t)ctx->nsm * 16);
  if (nrow > 0) {
    k_baseline_index<<<blocks, 256, 0, s>>>(ant1, ant2, nrow, n_ant, bidx, count);
    if ((e = cudaGetLastError())) return e;
  }
  k_baseline_start<<<1, 1024, 0, s>>>(count, nb, start, cursor);
  if ((e = cudaGetLastError())) return e;
  if (nrow > 0) {
    k_baseline_scatter<<<blocks, 256, 0, s>>>(bidx, nrow, cursor, perm);
    if ((e = cudaGetLastError())) return e;
    k_baseline_sort<<<nb, 512, 0, s>>>(start, nb, perm);
    if ((e = cudaGetLastError())) return e;
  }
  ctx->launches += nrow > 0 ? 4 : 1;
  return cudaSuccess;
}

cudaError_t launch_grid_baseline(wp_ctx* ctx, const int32_t* coords, const uint32_t* start, const int32_t* perm,
                                 int32_t n_ant, int32_t nchan, int64_t nrow, bool pairs, const float2* vis,
                                 const float* weight, float2* grid, cudaStream_t s) {
  const int32_t nb = n_ant * (n_ant + 1) / 2;
  int smax = 0;
  for (int sp : ctx->supp) smax = std::max(smax, sp);
  const int64_t nblocks = (int64_t)nb * nchan * (pairs ? 2 : 1);
  if (nblocks == 0) return cudaSuccess;
  const int threads = ((smax * smax + 31) / 32) * 32;
  const int64_t nvis = nrow * nchan;
  ++ctx->launches;
  switch (ctx->prm.table_type) {
    case WP_TABLE_F16:
      k_grid_baseline<__half2><<<(unsigned)nblocks, threads, 0, s>>>(coords, start, perm, nb, nchan, nvis, smax, vis,
                                                                     weight, ctx->geo, (const __half2*)ctx->d_tab,
                                                                     ctx->d_tab_off, grid);
      break;
    case WP_TABLE_BF16:
      k_grid_baseline<BfWord><<<(unsigned)nblocks, threads, 0, s>>>(
          coords, start, perm, nb, nchan, nvis, smax, vis, weight, ctx->geo, (const BfWord*)ctx->d_tab,
          ctx->d_tab_off, grid);
      break;
    default:
      k_grid_baseline<float2><<<(unsigned)nblocks, threads, 0, s>>>(coords, start, perm, nb, nchan, nvis, smax, vis,
                                                                    weight, ctx->geo, (const float2*)ctx->d_tab,
                                                                    ctx->d_tab_off, grid);
  }
  return cudaGetLastError();
}

}  // namespace wp
