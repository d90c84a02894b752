// Gridding and degridding over the binned records (baseline kernels). Gridding with float32
// tables and supports up to 32 runs the register-accumulating kernel of grid2.cu instead;
// this one covers the other cases.
//
// Gridding (Sec. 2.1/2.2 of Lao et al. 2019): every visibility adds c_k K_k(a, b) to the
// S_p x S_p cells of its footprint. Degridding is the adjoint gather.
//
// Work split: the sorted record array is cut into gridDim.x equal contiguous ranges, one
// per CTA, so every CTA gets the same number of visibilities however uneven the bins are
// (the load imbalance the paper reports for its OpenMP split, Sec. 3.2, does not arise).
// A CTA walks the bins its range touches; each bin segment is gridded into a shared-memory
// sub-grid covering the bin's origin tile plus the (S_p - 1)-cell halo, one warp per
// visibility and the warp's lanes over the taps, and the sub-grid is then merged into the
// HBM grid with one vector atomic per non-zero cell.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace wp {

namespace {

template <class T>
__device__ __forceinline__ float2 load_tap(const T* p);
template <>
__device__ __forceinline__ float2 load_tap<float2>(const float2* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float2 load_tap<__half2>(const __half2* p) {
  return __half22float2(__ldg(p));
}
template <>
__device__ __forceinline__ float2 load_tap<BfWord>(const BfWord* p) {
  const uint32_t w = __ldg((const unsigned int*)p);
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w));
}

struct TableRef {
  const void* tab;
  const int64_t* tab_off;
};

// The bin containing record index `pos`: the largest b with offsets[b] <= pos.
__device__ __forceinline__ int64_t find_bin(const uint32_t* __restrict__ offsets, int64_t nbins, uint32_t pos) {
  int64_t lo = 0, hi = nbins;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= pos) lo = mid;
    else hi = mid;
  }
  return lo;
}

// From `b` (offsets[b] <= pos) forward to the bin containing `pos`: galloping steps then
// bisection, so runs of empty bins cost O(log) loads.
__device__ __forceinline__ int64_t advance_bin(const uint32_t* __restrict__ offsets, int64_t b, int64_t nbins,
                                               uint32_t pos) {
  if (offsets[b + 1] > pos) return b;
  int64_t lo = b + 1, step = 1;
  while (lo + step < nbins && offsets[lo + step] <= pos) {
    lo += step;
    step <<= 1;
  }
  int64_t hi = min(lo + step, nbins);
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= pos) lo = mid;
    else hi = mid;
  }
  return lo;
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <class T>
__global__ void __launch_bounds__(kThreads) k_grid_v1(const Record* __restrict__ recs,
                                                      const uint32_t* __restrict__ offsets, int64_t nbins, Geometry g,
                                                      TableRef tr, float2* __restrict__ grid) {
  extern __shared__ float2 sub[];
  const uint32_t total = offsets[nbins];
  const uint32_t beg = (uint32_t)((uint64_t)total * blockIdx.x / gridDim.x);
  const uint32_t end = (uint32_t)((uint64_t)total * (blockIdx.x + 1) / gridDim.x);
  if (beg >= end) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t b = find_bin(offsets, nbins, beg);
  uint32_t pos = beg;
  while (pos < end) {
    b = advance_bin(offsets, b, nbins, pos);
    const uint32_t seg_end = min(end, offsets[b + 1]);
    const int p = (int)(b / g.ntiles);
    const int64_t tile = b - (int64_t)p * g.ntiles;
    const int ty = (int)(tile / g.ntx), tx = (int)(tile - (int64_t)ty * g.ntx);
    const int s = g.supp[p];
    const int pitch = g.tile_x + s - 1, rows = g.tile_y + s - 1;
    const int x0 = tx * g.tile_x, y0 = ty * g.tile_y;
    for (int q = threadIdx.x; q < pitch * rows; q += kThreads) sub[q] = make_float2(0.f, 0.f);
    __syncthreads();
    const T* tab = (const T*)tr.tab + tr.tab_off[p];
    const int taps = s * s;
    for (uint32_t r = pos + warp; r < seg_end; r += kWarps) {
      const Record rec = recs[r];
      const float cr = __uint_as_float(rec.x), ci = __uint_as_float(rec.y);
      const int i0 = rec.z & 0xffff, j0 = rec.z >> 16;
      const int ox = rec.w & 0xff, oy = (rec.w >> 8) & 0xff;
      const float sg = (rec.w >> 31) ? -1.f : 1.f;
      const int li = i0 - x0, lj = j0 - y0;
      const T* kb = tab + (int64_t)(oy * g.os + ox) * taps;
      for (int t = lane; t < taps; t += 32) {
        const int bb = t / s, aa = t - bb * s;
        const float2 k = load_tap<T>(kb + aa * s + bb);
        const float ki = sg * k.y;
        float2* cell = &sub[(lj + bb) * pitch + li + aa];
        atomicAdd(&cell->x, cr * k.x - ci * ki);
        atomicAdd(&cell->y, cr * ki + ci * k.x);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < pitch * rows; q += kThreads) {
      const float2 v = sub[q];
      const int gy = y0 + q / pitch, gx = x0 + q % pitch;
      if ((v.x != 0.f || v.y != 0.f) && gy < g.n && gx < g.n) atomicAdd(&grid[(int64_t)gy * g.n + gx], v);
    }
    __syncthreads();
    pos = seg_end;
  }
}

template <class T>
__global__ void __launch_bounds__(kThreads) k_degrid_v1(const Record* __restrict__ recs,
                                                        const uint32_t* __restrict__ offsets, int64_t nbins,
                                                        Geometry g, TableRef tr, const float2* __restrict__ grid,
                                                        float2* __restrict__ out,
                                                        const uint32_t* __restrict__ index) {
  const uint32_t total = offsets[nbins];
  const uint32_t beg = (uint32_t)((uint64_t)total * blockIdx.x / gridDim.x);
  const uint32_t end = (uint32_t)((uint64_t)total * (blockIdx.x + 1) / gridDim.x);
  if (beg >= end) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t b = find_bin(offsets, nbins, beg);
  uint32_t pos = beg;
  while (pos < end) {
    b = advance_bin(offsets, b, nbins, pos);
    const uint32_t seg_end = min(end, offsets[b + 1]);
    const int p = (int)(b / g.ntiles);
    const int s = g.supp[p];
    const int taps = s * s;
    const T* tab = (const T*)tr.tab + tr.tab_off[p];
    for (uint32_t r = pos + warp; r < seg_end; r += kWarps) {
      const Record rec = recs[r];
      const uint32_t idx = index ? index[r] : rec.x;
      if (idx >> 31) continue;                     // a gridding plan's Hermitian partner
      const int i0 = rec.z & 0xffff, j0 = rec.z >> 16;
      const int ox = rec.w & 0xff, oy = (rec.w >> 8) & 0xff;
      // conj(K_k): K_k = K (w >= 0) or conj(K) (w < 0)
      const float sg = (rec.w >> 31) ? 1.f : -1.f;
      const T* kb = tab + (int64_t)(oy * g.os + ox) * taps;
      float sr = 0.f, si = 0.f;
      for (int t = lane; t < taps; t += 32) {
        const int bb = t / s, aa = t - bb * s;
        const float2 k = load_tap<T>(kb + aa * s + bb);
        const float ki = sg * k.y;
        const float2 v = __ldg(&grid[(int64_t)(j0 + bb) * g.n + i0 + aa]);
        sr += v.x * k.x - v.y * ki;
        si += v.x * ki + v.y * k.x;
      }
      for (int off = 16; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, off);
        si += __shfl_xor_sync(0xffffffffu, si, off);
      }
      if (lane == 0) out[idx] = make_float2(sr, si);
    }
    pos = seg_end;
  }
}

template <class T>
cudaError_t grid_typed(wp_ctx* ctx, float2* grid, cudaStream_t s) {
  const int smax = *std::max_element(ctx->supp.begin(), ctx->supp.end());
  const size_t smem = sizeof(float2) * (size_t)(ctx->geo.tile_x + smax - 1) * (ctx->geo.tile_y + smax - 1);
  cudaError_t e = cudaFuncSetAttribute(k_grid_v1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  TableRef tr{ctx->d_tab, ctx->d_tab_off};
  k_grid_v1<T><<<ctx->nsm * 4, kThreads, smem, s>>>((const Record*)ctx->records.ptr, ctx->d_offsets, ctx->nbins,
                                                    ctx->geo, tr, grid);
  return cudaGetLastError();
}

template <class T>
cudaError_t degrid_typed(wp_ctx* ctx, const float2* grid, float2* out, const uint32_t* index, cudaStream_t s) {
  TableRef tr{ctx->d_tab, ctx->d_tab_off};
  k_degrid_v1<T><<<ctx->nsm * 4, kThreads, 0, s>>>((const Record*)ctx->records.ptr, ctx->d_offsets, ctx->nbins,
                                                   ctx->geo, tr, grid, out, index);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grid(wp_ctx* ctx, float2* grid, cudaStream_t s) {
  bool used = false;                       // the warp kernels count their own launches (one or two)
  const cudaError_t e = launch_grid_v2(ctx, grid, s, &used);
  if (e != cudaSuccess || used) return e;
  ++ctx->launches;
  switch (ctx->prm.table_type) {
    case WP_TABLE_F16: return grid_typed<__half2>(ctx, grid, s);
    case WP_TABLE_BF16: return grid_typed<BfWord>(ctx, grid, s);
    default: return grid_typed<float2>(ctx, grid, s);
  }
}

cudaError_t launch_degrid(wp_ctx* ctx, const float2* grid, float2* out, const uint32_t* index, cudaStream_t s) {
  bool used = false;                       // the warp kernels count their own launches (one or two)
  const cudaError_t e = launch_degrid_v2(ctx, grid, out, index, s, &used);
  if (e != cudaSuccess || used) return e;
  ++ctx->launches;
  switch (ctx->prm.table_type) {
    case WP_TABLE_F16: return degrid_typed<__half2>(ctx, grid, out, index, s);
    case WP_TABLE_BF16: return degrid_typed<BfWord>(ctx, grid, out, index, s);
    default: return degrid_typed<float2>(ctx, grid, out, index, s);
  }
}

}  // namespace wp
