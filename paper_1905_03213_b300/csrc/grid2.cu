// Register-accumulating gridding kernel (the hot path of wp_grid).
//
// Gridding (Sec. 2.1/2.2 of Lao et al. 2019): visibility k adds c_k K_k(a, b) to the cell
// (i0 + a, j0 + b) of its S x S footprint. The paper's GPU scheme (Fig. 2, after Romein)
// gives each thread one support tap and keeps that tap's sum in a register while the
// grid point stays the same; here the same idea is organised around sorted bins:
//
//   * A CTA takes a contiguous share of the (plane, tile)-sorted records, of equal estimated
//     work, and sorts each chunk of them by footprint origin (row j0, then column i0) in
//     shared memory, the chunk as large as the shared memory left beside the plane's table.
//   * A "stream" of S threads walks a contiguous piece of the sorted chunk. Thread x owns
//     the cells whose column is congruent to x modulo S: every footprint covers exactly one
//     such cell per row, in tap column a = (x - i0) mod S. Its S accumulators (row pairs,
//     packed for f32x2 FMAs) hold rows j0 .. j0 + S - 1 of that column while consecutive
//     records keep the origin row and the column; when i0 passes the column, or the row
//     changes, the thread adds its S cells to the HBM grid with vector reductions (a
//     "flush") and restarts.
//   * Per tap a thread does a quarter of a 16-byte shared-memory load (the staged table holds
//     row pairs, padded to an odd stride so the S threads of a stream hit distinct banks) and
//     two packed FMAs.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace wp {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxS = 32;
constexpr int kMaxKeys = 4096;                                  // origins of one segment
constexpr int kCountsBytes = ((kMaxKeys + 1) * 4 + 15) & ~15;  // shared-memory counters
constexpr int kMinChunk = 512;

struct G2Args {
  const Record* recs;
  const uint32_t* offsets;
  const uint32_t* costoff;  // [nbins + 1] prefix sums of per-bin work estimates
  int64_t nbins;
  Geometry g;
  const float2* tab;        // stored tables (f32), layout [plane][oy*os+ox][a][b]
  const int64_t* tab_off;
  float2* grid;
  int smem_bytes;           // dynamic shared memory of the launch
  int group_tiles;          // origin tiles of one tile row gridded as one segment, at most
};

__device__ __forceinline__ unsigned char* dyn_smem() {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return smem_raw;
}

__host__ __device__ __forceinline__ int row_pairs(int s) { return (s + 1) / 2; }
// float4 entries per staged table column: the row pairs, padded to an odd count
__host__ __device__ __forceinline__ int column_stride(int s) { return row_pairs(s) | 1; }
__host__ __device__ __forceinline__ int table_bytes(int os, int s) { return os * os * s * column_stride(s) * 16; }

__device__ __forceinline__ int64_t find_bin(const uint32_t* __restrict__ offsets, int64_t nbins, uint32_t pos) {
  int64_t lo = 0, hi = nbins;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= pos) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The bin containing record `pos`, searching forward from `bin` (offsets[bin] <= pos):
// galloping steps of 1, 2, 4, ... then bisection, so long runs of empty bins cost O(log).
__device__ __forceinline__ int64_t advance_bin(const uint32_t* __restrict__ offsets, int64_t bin, int64_t nbins,
                                               uint32_t pos) {
  if (offsets[bin + 1] > pos) return bin;
  int64_t lo = bin + 1, step = 1;                 // offsets[lo] <= pos; offsets[nbins] > pos
  while (lo + step < nbins && offsets[lo + step] <= pos) {
    lo += step;
    step <<= 1;
  }
  int64_t hi = min(lo + step, nbins);             // offsets[hi] > pos
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= pos) lo = mid;
    else hi = mid;
  }
  return lo;
}

// In-place exclusive scan of the shared counters counts[0..n) by the whole block.
__device__ void block_exclusive_scan(int n) {
  __shared__ uint32_t warp_sums[kWarps];
  uint32_t* counts = (uint32_t*)dyn_smem();
  const int per = (n + kThreads - 1) / kThreads;
  const int beg = threadIdx.x * per;
  uint32_t local = 0;
  for (int i = 0; i < per; ++i)
    if (beg + i < n) local += counts[beg + i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = local;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < kWarps ? warp_sums[lane] : 0u;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += y;
    }
    if (lane < kWarps) warp_sums[lane] = s;
  }
  __syncthreads();
  uint32_t run = (warp ? warp_sums[warp - 1] : 0u) + x - local;
  for (int i = 0; i < per; ++i) {
    if (beg + i < n) {
      const uint32_t v = counts[beg + i];
      counts[beg + i] = run;
      run += v;
    }
  }
  __syncthreads();
}

// Packed pair of floats (two footprint rows) as one 64-bit register for fma.rn.f32x2.
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  return (unsigned long long)__float_as_uint(a) | ((unsigned long long)__float_as_uint(b) << 32);
}
__device__ __forceinline__ float lo_of(unsigned long long v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_of(unsigned long long v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Adds a thread's S accumulated cells (column `col`, rows row0 .. row0 + S - 1) to the grid
// with vector reductions and clears the accumulators.
template <int S, int H>
__device__ __forceinline__ void flush_column(unsigned long long (&re)[H], unsigned long long (&im)[H],
                                             float2* __restrict__ grid, int n, int row0, int col) {
  float2* cell = grid + (int64_t)row0 * n + col;
#pragma unroll
  for (int q = 0; q < H; ++q) {
    atomicAdd(cell + (int64_t)(2 * q) * n, make_float2(lo_of(re[q]), lo_of(im[q])));
    if (2 * q + 1 < S) atomicAdd(cell + (int64_t)(2 * q + 1) * n, make_float2(hi_of(re[q]), hi_of(im[q])));
    re[q] = 0ull;
    im[q] = 0ull;
  }
}

// One stream grids the decoded, sorted records [beg, end) of the chunk at byte offset
// rec_off; thread x of the stream owns the cell columns congruent to x modulo S.
// Staged table (byte offset tab_off): [cls][a][q < ST] = {re(2q), re(2q+1), im(2q), im(2q+1)}.
// Decoded record: x, y = c (float bits); z = i0 | j0 << 16; w = cls*S*ST | (i0 mod S) << 20 | conj << 31.
template <int S>
__device__ void stream_grid(int tab_off, int rec_off, int beg, int end, int x, float2* __restrict__ grid, int n) {
  constexpr int H = (S + 1) / 2, ST = H | 1;
  unsigned long long re[H], im[H];
#pragma unroll
  for (int q = 0; q < H; ++q) re[q] = im[q] = 0ull;
  const float4* tab = (const float4*)(dyn_smem() + tab_off);
  const uint4* drec = (const uint4*)(dyn_smem() + rec_off);
  int cj = -1, ci = 0, col = -1;                   // run row, last origin column, this thread's cell column
  uint4 nxt = beg < end ? drec[beg] : make_uint4(0u, 0u, 0u, 0u);
  for (int q = beg; q < end; ++q) {
    const uint4 rec = nxt;
    if (q + 1 < end) nxt = drec[q + 1];
    const int i0 = rec.z & 0xffff, j0 = rec.z >> 16;
    if (j0 != cj || i0 < ci) {                     // new run (row): every thread flushes its column
      if (col >= 0) flush_column<S, H>(re, im, grid, n, cj, col);
      cj = j0;
      col = -1;
    }
    ci = i0;
    const int r0x = (rec.w >> 20) & 0x1f;
    const int a = x - r0x + (x < r0x ? S : 0);
    const int cx = i0 + a;
    if (cx != col) {                               // this thread's class moved to a new cell column
      if (col >= 0) flush_column<S, H>(re, im, grid, n, cj, col);
      col = cx;
    }
    // acc.re += cr kr + be ki, acc.im += ci kr + de ki: c K, or c conj(K) for w < 0
    const uint32_t flip = (rec.w & 0x80000000u) ^ 0x80000000u;
    const float cr = __uint_as_float(rec.x), cim = __uint_as_float(rec.y);
    const float be = __uint_as_float(rec.y ^ flip), de = __uint_as_float(rec.x ^ flip ^ 0x80000000u);
    const unsigned long long CR = pack2(cr, cr), CI = pack2(cim, cim);
    const unsigned long long BE = pack2(be, be), DE = pack2(de, de);
    const float4* t = tab + (int)(rec.w & 0xfffff) + a * ST;
#pragma unroll
    for (int qq = 0; qq < H; ++qq) {
      const float4 v = t[qq];
      const unsigned long long kr = pack2(v.x, v.y), ki = pack2(v.z, v.w);
      re[qq] = fma2(CR, kr, re[qq]);
      re[qq] = fma2(BE, ki, re[qq]);
      im[qq] = fma2(CI, kr, im[qq]);
      im[qq] = fma2(DE, ki, im[qq]);
    }
  }
  if (col >= 0) flush_column<S, H>(re, im, grid, n, cj, col);
}

// Grids records [s0, s1) of one segment (plane p, support S; origin tiles of one tile row,
// columns x0 .. x0 + width) in chunks of at most `cap` records.
template <int S>
__device__ void grid_segment(const G2Args& a, int x0, int y0, int width, uint32_t s0, uint32_t s1, int cap,
                             int tab_off, int rec_off) {
  constexpr int H = (S + 1) / 2, ST = H | 1;
  const int keys = width * a.g.tile_y;
  const int nst = kThreads / S;                    // streams of S threads over the whole block
  const int stream = threadIdx.x / S, x = threadIdx.x - stream * S;
  const int os = a.g.os;
  uint32_t* counts = (uint32_t*)dyn_smem();
  uint4* drec = (uint4*)(dyn_smem() + rec_off);
  const uint4* grecs = (const uint4*)a.recs;
  for (uint32_t c0 = s0; c0 < s1; c0 += (uint32_t)cap) {
    const int m = (int)min((uint32_t)cap, s1 - c0);
    for (int k = threadIdx.x; k < keys; k += kThreads) counts[k] = 0u;
    __syncthreads();
    // pass 1: histogram of the origin keys (row-major within the segment)
    for (int r = threadIdx.x; r < m; r += kThreads) {
      const uint32_t z = __ldcg(&grecs[c0 + r].z);
      atomicAdd(&counts[((int)(z >> 16) - y0) * width + ((int)(z & 0xffff) - x0)], 1u);
    }
    __syncthreads();
    block_exclusive_scan(keys);
    // pass 2: decode each record into its sorted slot
    for (int r = threadIdx.x; r < m; r += kThreads) {
      const uint4 rec = __ldcs(grecs + c0 + r);
      const int i0 = rec.z & 0xffff;
      const int key = ((int)(rec.z >> 16) - y0) * width + (i0 - x0);
      const int cls = (int)((rec.w >> 8) & 0xff) * os + (int)(rec.w & 0xff);
      const uint32_t w = (uint32_t)(cls * S * ST) | ((uint32_t)(i0 % S) << 20) | (rec.w & 0x80000000u);
      drec[atomicAdd(&counts[key], 1u)] = make_uint4(rec.x, rec.y, rec.z, w);
    }
    __syncthreads();
    if (stream < nst) {
      const int beg = (int)((int64_t)m * stream / nst), end = (int)((int64_t)m * (stream + 1) / nst);
      stream_grid<S>(tab_off, rec_off, beg, end, x, a.grid, a.g.n);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_grid_v2(G2Args a) {
  // Equal shares of the estimated work: cost position x maps to bin b (costoff[b] <= x <
  // costoff[b+1]) and to the record offsets[b] + (x - costoff[b]) / cost_b * count_b, a
  // monotone map, so consecutive CTAs partition the records exactly.
  const uint32_t total = a.offsets[a.nbins];
  const uint32_t ctotal = a.costoff[a.nbins];
  auto split = [&](uint64_t x) -> uint32_t {
    if (x >= ctotal) return total;
    const int64_t b = find_bin(a.costoff, a.nbins, (uint32_t)x);
    const uint32_t c0 = a.costoff[b], cb = a.costoff[b + 1] - c0;
    const uint32_t n = a.offsets[b + 1] - a.offsets[b];
    return a.offsets[b] + (uint32_t)(((uint64_t)(x - c0) * n) / cb);
  };
  const uint32_t beg = split((uint64_t)ctotal * blockIdx.x / gridDim.x);
  const uint32_t end = split((uint64_t)ctotal * (blockIdx.x + 1) / gridDim.x);
  if (beg >= end) return;
  int64_t bin = find_bin(a.offsets, a.nbins, beg);
  uint32_t pos = beg;
  int cur_plane = -1;
  const int tab_off = kCountsBytes;
  while (pos < end) {
    bin = advance_bin(a.offsets, bin, a.nbins, pos);
    const int p = (int)(bin / a.g.ntiles);
    const int64_t tile = bin - (int64_t)p * a.g.ntiles;
    const int ty = (int)(tile / a.g.ntx), tx = (int)(tile - (int64_t)ty * a.g.ntx);
    const int s = a.g.supp[p];
    const int rec_off = tab_off + table_bytes(a.g.os, s);
    const int cap = (a.smem_bytes - rec_off) / (int)sizeof(Record);
    // a segment: this bin, plus the following bins of the same tile row while the records
    // still fit one chunk (sparse tiles are sorted together, dense ones alone)
    uint32_t bound[8];                            // ends of this bin and the next 7 (independent loads)
#pragma unroll
    for (int k = 0; k < 8; ++k) bound[k] = a.offsets[min(bin + k + 1, a.nbins)];
    uint32_t seg_end = min(end, bound[0]);
    int ntiles = 1;
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      if (ntiles == k && k < a.group_tiles && tx + k < a.g.ntx && seg_end < end) {
        const uint32_t nxt = min(end, bound[k]);
        if (nxt - pos <= (uint32_t)cap) {
          seg_end = nxt;
          ntiles = k + 1;
        }
      }
    }
    if (p != cur_plane) {
      // stage the plane's table: [cls][a][q] = {re(2q), re(2q+1), im(2q), im(2q+1)}, ST per column
      const int half = row_pairs(s), st = column_stride(s);
      const int ncols = a.g.os * a.g.os * s;
      const float2* src = a.tab + a.tab_off[p];
      float4* dst = (float4*)(dyn_smem() + tab_off);
      for (int i = threadIdx.x; i < ncols * half; i += kThreads) {
        const int ca = i / half, q = i - ca * half;
        const float2 v0 = __ldg(&src[ca * s + 2 * q]);
        const float2 v1 = (2 * q + 1 < s) ? __ldg(&src[ca * s + 2 * q + 1]) : make_float2(0.f, 0.f);
        dst[ca * st + q] = make_float4(v0.x, v1.x, v0.y, v1.y);
      }
      cur_plane = p;
    }
    const int x0 = tx * a.g.tile_x, y0 = ty * a.g.tile_y;
    const int width = ntiles * a.g.tile_x;
    switch (s) {
#define WP_SEG_CASE(N)                                                              \
  case N:                                                                           \
    grid_segment<N>(a, x0, y0, width, pos, seg_end, cap, tab_off, rec_off);         \
    break;
      WP_SEG_CASE(1) WP_SEG_CASE(2) WP_SEG_CASE(3) WP_SEG_CASE(4) WP_SEG_CASE(5) WP_SEG_CASE(6) WP_SEG_CASE(7)
      WP_SEG_CASE(8) WP_SEG_CASE(9) WP_SEG_CASE(10) WP_SEG_CASE(11) WP_SEG_CASE(12) WP_SEG_CASE(13)
      WP_SEG_CASE(14) WP_SEG_CASE(15) WP_SEG_CASE(16) WP_SEG_CASE(17) WP_SEG_CASE(18) WP_SEG_CASE(19)
      WP_SEG_CASE(20) WP_SEG_CASE(21) WP_SEG_CASE(22) WP_SEG_CASE(23) WP_SEG_CASE(24) WP_SEG_CASE(25)
      WP_SEG_CASE(26) WP_SEG_CASE(27) WP_SEG_CASE(28) WP_SEG_CASE(29) WP_SEG_CASE(30) WP_SEG_CASE(31)
      WP_SEG_CASE(32)
#undef WP_SEG_CASE
      default:
        break;
    }
    pos = seg_end;
  }
}

}  // namespace

// Dynamic shared memory of the launch (the device's opt-in maximum), or 0 when the geometry
// is outside the kernel's limits (then the baseline kernel of grid.cu runs).
size_t grid_v2_smem(const wp_ctx* ctx, int* group_tiles) {
  const int smax = *std::max_element(ctx->supp.begin(), ctx->supp.end());
  if (smax > kMaxS || ctx->prm.table_type != WP_TABLE_F32) return 0;
  const int os = ctx->prm.oversample;
  if ((int64_t)os * os * smax * column_stride(smax) >= (1 << 20)) return 0;   // packed in 20 bits
  const int tx = ctx->geo.tile_x, ty = ctx->geo.tile_y;
  if ((int64_t)tx * ty > kMaxKeys) return 0;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->prm.device) != cudaSuccess)
    return 0;
  const size_t bytes = (size_t)optin - 1024;        // room for the static scan scratch
  if ((size_t)kCountsBytes + (size_t)table_bytes(os, smax) + (size_t)kMinChunk * sizeof(Record) > bytes) return 0;
  *group_tiles = std::max(1, std::min(8, kMaxKeys / (tx * ty)));
  return bytes;
}

cudaError_t launch_grid_v2(wp_ctx* ctx, float2* grid, cudaStream_t s, bool* used) {
  int group = 1;
  const size_t smem = grid_v2_smem(ctx, &group);
  *used = smem != 0;
  if (!smem) return cudaSuccess;
  G2Args a;
  a.recs = (const Record*)ctx->records.ptr;
  a.offsets = ctx->d_offsets;
  a.costoff = ctx->d_costoff;
  a.nbins = ctx->nbins;
  a.g = ctx->geo;
  a.tab = (const float2*)ctx->d_tab;
  a.tab_off = ctx->d_tab_off;
  a.grid = grid;
  a.smem_bytes = (int)smem;
  a.group_tiles = group;
  cudaError_t e;
  if ((e = launch_bin_costs(ctx, s))) return e;
  if ((e = cudaFuncSetAttribute(k_grid_v2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
  k_grid_v2<<<ctx->nsm, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wp
