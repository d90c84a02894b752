// Coordinates (float64) and binning of visibilities by (w-plane, footprint-origin tile).
//
// Coordinates follow the W-projection gridding step (Sec. 2.1/2.2 of Lao et al. 2019: each
// visibility lands on the uv grid through a C_full x C_full kernel); the arithmetic is
// float64 and round-half-to-even, in the order written in wproj.h, so that the integer
// decisions (oversampled position, plane, footprint) are the same on every platform that
// evaluates the same IEEE float64 operations.
//
// Binning is a counting sort: a histogram of bin keys, an exclusive prefix sum giving each
// bin's start index (the construction of Eq. 6, there applied to baselines), and a scatter
// that writes each visibility's 16-byte record into its bin. Records within a bin are in
// no particular order.
#include <cuda_runtime.h>

#include "internal.h"

namespace wp {

namespace {

struct Coord {
  int32_t u, v, plane, i0, j0, ox, oy;
  bool conj, keep;
};

__device__ __forceinline__ int32_t floor_div(int32_t a, int32_t b) {
  // b > 0
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// Coordinates of one gridded visibility. (ux, vy, wz) are the float64 products
// u*kx, v*kx, |w|*kw; `neg` selects the Hermitian partner at -uvw.
__device__ __forceinline__ Coord make_coord(double ux, double vy, double wz, double w_m, bool neg,
                                           const Geometry& g) {
  Coord c;
  const bool fin = isfinite(ux) && isfinite(vy) && isfinite(wz) && fabs(ux) < kCoordLimit &&
                   fabs(vy) < kCoordLimit;
  int32_t u = fin ? (int32_t)rint(ux) : 0;
  int32_t v = fin ? (int32_t)rint(vy) : 0;
  const int32_t p = fin ? (int32_t)fmin((double)(g.n_w - 1), rint(fmin(wz, kCoordLimit))) : 0;
  if (neg) {
    u = -u;
    v = -v;
  }
  c.u = u;
  c.v = v;
  c.plane = p;
  c.conj = neg ? (w_m > 0.0) : (w_m < 0.0);
  const int32_t s = g.supp[p];
  const int32_t half = s * g.os / 2;
  const int32_t x = u + (g.n / 2) * g.os;
  const int32_t y = v + (g.n / 2) * g.os;
  c.i0 = floor_div(x - half, g.os) + 1;
  c.j0 = floor_div(y - half, g.os) + 1;
  c.ox = c.i0 * g.os - x + half - 1;
  c.oy = c.j0 * g.os - y + half - 1;
  c.keep = fin && c.i0 >= 0 && c.i0 + s <= g.n && c.j0 >= 0 && c.j0 + s <= g.n;
  return c;
}

__device__ __forceinline__ uint32_t bin_of(const Coord& c, const Geometry& g) {
  return (uint32_t)((int64_t)c.plane * g.ntiles + (int64_t)(c.j0 / g.tile_y) * g.ntx + c.i0 / g.tile_x);
}

// Per-(row, channel) products, shared by the visibility and its Hermitian partner.
struct Products {
  double ux, vy, wz, w;
};

__device__ __forceinline__ Products products(const double* __restrict__ uvw, const double* __restrict__ chan,
                                             int64_t k, int32_t nchan) {
  const int64_t r = k / nchan;
  const int32_t ch = (int32_t)(k - r * nchan);
  const double u = uvw[3 * r], v = uvw[3 * r + 1], w = uvw[3 * r + 2];
  const double kx = chan[2 * ch], kw = chan[2 * ch + 1];
  Products p;
  p.ux = __dmul_rn(u, kx);
  p.vy = __dmul_rn(v, kx);
  p.wz = __dmul_rn(fabs(w), kw);
  p.w = w;
  return p;
}

// Warp-aggregated atomicAdd of 1 on counter[key] for the active lanes with key != ~0u.
// Returns the per-lane slot (old value + rank among lanes with the same key).
__device__ __forceinline__ uint32_t aggregated_increment(uint32_t* counter, uint32_t key) {
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  const unsigned rank = __popc(peers & ((1u << lane) - 1));
  uint32_t base = 0;
  if (lane == leader && key != 0xffffffffu) base = atomicAdd(&counter[key], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + rank;
}

__global__ void k_channel_factors(const double* __restrict__ freq, int32_t nchan, double os_l,
                                  double wscale, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nchan) {
    const double s = freq[c] / kCLight;
    out[2 * c] = __dmul_rn(s, os_l);
    out[2 * c + 1] = __dmul_rn(s, wscale);
  }
}

// Pass 1: bin histogram, dropped count and kept-weight sum.
__global__ void __launch_bounds__(256) k_histogram(const double* __restrict__ uvw, const double* __restrict__ chan,
                                                   const float* __restrict__ weight, int64_t nvis, int32_t nchan,
                                                   int32_t pairs, Geometry g, uint32_t* __restrict__ counts,
                                                   unsigned long long* __restrict__ dropped,
                                                   double* __restrict__ wsum) {
  double my_w = 0.0;
  unsigned long long my_drop = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nvis; k += (int64_t)gridDim.x * blockDim.x) {
    const Products pr = products(uvw, chan, k, nchan);
    const double wt = weight ? (double)weight[k] : 1.0;
    for (int h = 0; h <= pairs; ++h) {
      const Coord c = make_coord(pr.ux, pr.vy, pr.wz, pr.w, h == 1, g);
      const uint32_t key = c.keep ? bin_of(c, g) : 0xffffffffu;
      aggregated_increment(counts, key);
      if (c.keep) my_w += wt;
      else ++my_drop;
    }
  }
  // block reduction of the two scalars
  __shared__ double sw[8];
  __shared__ unsigned long long sd[8];
  for (int off = 16; off > 0; off >>= 1) {
    my_w += __shfl_xor_sync(0xffffffffu, my_w, off);
    my_drop += __shfl_xor_sync(0xffffffffu, my_drop, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sw[warp] = my_w;
    sd[warp] = my_drop;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tw = 0.0;
    unsigned long long td = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      tw += sw[i];
      td += sd[i];
    }
    if (tw != 0.0) atomicAdd(wsum, tw);
    if (td) atomicAdd(dropped, td);
  }
}

// Pass 3: scatter records into their bins.
__global__ void __launch_bounds__(256) k_scatter(const double* __restrict__ uvw, const double* __restrict__ chan,
                                                 const float2* __restrict__ vis, const float* __restrict__ weight,
                                                 int64_t nvis, int32_t nchan, int32_t pairs, int32_t for_degrid,
                                                 Geometry g, uint32_t* __restrict__ cursor,
                                                 Record* __restrict__ records) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nvis; k += (int64_t)gridDim.x * blockDim.x) {
    const Products pr = products(uvw, chan, k, nchan);
    float2 val = make_float2(0.f, 0.f);
    if (!for_degrid) {
      const float2 v = vis[k];
      const float wt = weight ? weight[k] : 1.0f;
      val = make_float2(wt * v.x, wt * v.y);
    }
    for (int h = 0; h <= pairs; ++h) {
      const Coord c = make_coord(pr.ux, pr.vy, pr.wz, pr.w, h == 1, g);
      const uint32_t key = c.keep ? bin_of(c, g) : 0xffffffffu;
      const uint32_t slot = aggregated_increment(cursor, key);
      if (c.keep) {
        Record rec;
        if (for_degrid) {
          rec.x = (uint32_t)k;
          rec.y = 0u;
        } else {
          rec.x = __float_as_uint(val.x);
          rec.y = __float_as_uint(h ? -val.y : val.y);
        }
        rec.z = (uint32_t)c.i0 | ((uint32_t)c.j0 << 16);
        rec.w = (uint32_t)c.ox | ((uint32_t)c.oy << 8) | (c.conj ? 0x80000000u : 0u);
        records[slot] = rec;
      }
    }
  }
}

// Exclusive prefix sum over nbins counts in three kernels (4096 elements per block).
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t s = lane < nw ? warp_sums[lane] : 0u;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  const uint32_t before = warp ? warp_sums[warp - 1] : 0u;
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t* __restrict__ in, int64_t n,
                                                             uint32_t* __restrict__ out,
                                                             uint32_t* __restrict__ partials) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPerThread;
  uint32_t v[kScanPerThread];
  uint32_t sum = 0;
  for (int i = 0; i < kScanPerThread; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    sum += v[i];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(sum, &total);
  for (int i = 0; i < kScanPerThread; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials(uint32_t* __restrict__ partials, int64_t nparts) {
  // single block; nparts <= kScanTile
  const int64_t base = (int64_t)threadIdx.x * kScanPerThread;
  uint32_t v[kScanPerThread];
  uint32_t sum = 0;
  for (int i = 0; i < kScanPerThread; ++i) {
    v[i] = (base + i < nparts) ? partials[base + i] : 0u;
    sum += v[i];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(sum, &total);
  for (int i = 0; i < kScanPerThread; ++i) {
    if (base + i < nparts) partials[base + i] = run;
    run += v[i];
  }
  if (threadIdx.x == 0) partials[nparts] = total;
}

__global__ void k_scan_finish(uint32_t* __restrict__ offsets, uint32_t* __restrict__ cursor, int64_t n,
                              const uint32_t* __restrict__ partials, int64_t nparts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint32_t o = offsets[i] + partials[i / kScanTile];
    offsets[i] = o;
    cursor[i] = o;
  }
  if (i == 0) offsets[n] = partials[nparts];
}

// Work estimate of bin b in units of 64 tap-updates: a fixed part for every non-empty bin
// (segment set-up, local sort, barriers) plus, per record, its S_p^2 taps and a record cost.
constexpr uint32_t kBinFixedTaps = 2048;
constexpr uint32_t kRecordTaps = 32;

__global__ void k_bin_costs(const uint32_t* __restrict__ offsets, int64_t nbins, Geometry g,
                            uint32_t* __restrict__ cost) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const uint32_t cnt = offsets[b + 1] - offsets[b];
  const int s = g.supp[b / g.ntiles];
  const uint64_t taps = cnt ? (uint64_t)kBinFixedTaps + (uint64_t)cnt * (uint64_t)(s * s + kRecordTaps) : 0;
  cost[b] = (uint32_t)((taps + 63) / 64);
}

__global__ void k_coords_out(const double* __restrict__ uvw, const double* __restrict__ chan, int64_t nvis,
                             int32_t nchan, int32_t pairs, Geometry g, int32_t* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nvis; k += (int64_t)gridDim.x * blockDim.x) {
    const Products pr = products(uvw, chan, k, nchan);
    for (int h = 0; h <= pairs; ++h) {
      const Coord c = make_coord(pr.ux, pr.vy, pr.wz, pr.w, h == 1, g);
      int32_t* o = out + 8 * (k + h * nvis);
      o[0] = c.u;
      o[1] = c.v;
      o[2] = c.plane;
      o[3] = c.conj ? 1 : 0;
      o[4] = c.keep ? 1 : 0;
      o[5] = c.i0;
      o[6] = c.j0;
      o[7] = (c.ox & 0xffff) | (c.oy << 16);
    }
  }
}

int grid_blocks(int64_t work, int nsm) {
  const int64_t want = (work + 255) / 256;
  const int64_t cap = (int64_t)nsm * 16;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_channel_factors(const double* freq, int32_t nchan, double os_l, double wscale, double* d_chan,
                                   cudaStream_t s) {
  k_channel_factors<<<(nchan + 127) / 128, 128, 0, s>>>(freq, nchan, os_l, wscale, d_chan);
  return cudaGetLastError();
}

cudaError_t launch_plan(wp_ctx* ctx, const double* uvw, const float2* vis, const float* weight, int64_t nrow,
                        int32_t nchan, bool pairs, bool for_degrid, cudaStream_t s) {
  const int64_t nvis = nrow * nchan;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ctx->d_counts, 0, sizeof(uint32_t) * ctx->nbins, s))) return e;
  if ((e = cudaMemsetAsync(ctx->d_dropped, 0, sizeof(unsigned long long), s))) return e;
  if ((e = cudaMemsetAsync(ctx->d_wsum, 0, sizeof(double), s))) return e;
  const int blocks = grid_blocks(nvis, ctx->nsm);
  ctx->launches += 3 + (nvis > 0 ? 2 : 0);  // prefix sum (3), histogram and scatter
  if (nvis > 0) {
    k_histogram<<<blocks, 256, 0, s>>>(uvw, ctx->d_chan, for_degrid ? nullptr : weight, nvis, nchan, pairs ? 1 : 0,
                                       ctx->geo, ctx->d_counts, ctx->d_dropped, ctx->d_wsum);
    if ((e = cudaGetLastError())) return e;
  }
  const int64_t tiles = (ctx->nbins + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(ctx->d_counts, ctx->nbins, ctx->d_offsets, ctx->d_partials);
  if ((e = cudaGetLastError())) return e;
  k_scan_partials<<<1, kScanThreads, 0, s>>>(ctx->d_partials, tiles);
  if ((e = cudaGetLastError())) return e;
  k_scan_finish<<<(unsigned)((ctx->nbins + 255) / 256), 256, 0, s>>>(ctx->d_offsets, ctx->d_cursor, ctx->nbins,
                                                                     ctx->d_partials, tiles);
  if ((e = cudaGetLastError())) return e;
  if (nvis > 0) {
    k_scatter<<<blocks, 256, 0, s>>>(uvw, ctx->d_chan, vis, weight, nvis, nchan, pairs ? 1 : 0, for_degrid ? 1 : 0,
                                     ctx->geo, ctx->d_cursor, (Record*)ctx->records.ptr);
    if ((e = cudaGetLastError())) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_bin_costs(wp_ctx* ctx, cudaStream_t s) {
  cudaError_t e;
  ctx->launches += 4;
  const unsigned blocks = (unsigned)((ctx->nbins + 255) / 256);
  k_bin_costs<<<blocks, 256, 0, s>>>(ctx->d_offsets, ctx->nbins, ctx->geo, ctx->d_counts);
  if ((e = cudaGetLastError())) return e;
  const int64_t tiles = (ctx->nbins + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(ctx->d_counts, ctx->nbins, ctx->d_costoff, ctx->d_partials2);
  if ((e = cudaGetLastError())) return e;
  k_scan_partials<<<1, kScanThreads, 0, s>>>(ctx->d_partials2, tiles);
  if ((e = cudaGetLastError())) return e;
  // finish into d_costoff; d_counts (holding the costs) serves as the unused cursor output
  k_scan_finish<<<blocks, 256, 0, s>>>(ctx->d_costoff, ctx->d_counts, ctx->nbins, ctx->d_partials2, tiles);
  return cudaGetLastError();
}

cudaError_t launch_coords(wp_ctx* ctx, const double* uvw, int64_t nrow, int32_t nchan, bool pairs, int32_t* out,
                          cudaStream_t s) {
  const int64_t nvis = nrow * nchan;
  if (nvis == 0) return cudaSuccess;
  ++ctx->launches;
  k_coords_out<<<grid_blocks(nvis, ctx->nsm), 256, 0, s>>>(uvw, ctx->d_chan, nvis, nchan, pairs ? 1 : 0, ctx->geo,
                                                            out);
  return cudaGetLastError();
}

}  // namespace wp
