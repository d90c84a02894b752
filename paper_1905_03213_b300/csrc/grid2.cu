// Register-accumulating gridding kernel (the hot path of wp_grid).
//
// Gridding (Sec. 2.1/2.2 of Lao et al. 2019): visibility k adds c_k K_k(a, b) to the cell
// (i0 + a, j0 + b) of its S x S footprint. The paper's GPU scheme (Fig. 2, after Romein)
// keeps each support tap's running sum in a register while the grid point it maps to stays
// the same; here that idea is organised around sorted bins and whole warps:
//
//   * A CTA takes a contiguous share of the (plane, tile)-sorted records, of equal estimated
//     work, and counting-sorts each chunk of them by footprint origin (row j0, then column
//     i0) in shared memory; the chunk is as large as the shared memory left beside the
//     plane's staged table.
//   * Each warp walks one contiguous piece of the sorted chunk, all 32 lanes on the same
//     record, so every branch is warp-uniform. Lane (g, a) holds rows g R .. g R + R - 1 of
//     footprint column a in registers (row pairs packed for f32x2 FMAs): the warp's
//     registers are the S x S cells under the current origin.
//   * Consecutive records with the same origin accumulate in place. When the origin moves
//     right by d < S columns on the same row, the lanes of the d leaving columns add their
//     cells to the HBM grid (vector reductions) and the accumulators slide d lanes with one
//     shuffle per register; any other move flushes all S x S cells. Per record and row pair a
//     lane does two 8-byte table loads (the kr and ki pairs, each a 256-byte conflict-free
//     block per warp) and four packed FMAs.
//   * CTAs take work units (equal shares of the estimated work) from a global counter, the
//     most expensive end of the record order first, so no CTA is left with a long tail.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace wp {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxS = 16;                                     // larger supports: baseline kernel
constexpr int kMaxKeys = 4096;                                  // origins of one segment
constexpr int kCountsBytes = ((kMaxKeys + 1) * 4 + 15) & ~15;  // shared-memory counters
constexpr int kMinChunk = 512;
constexpr uint32_t kNoOrigin = 0xffffffffu;
constexpr int kUnitsPerCta = 8;                              // work units per CTA, on average

// Lane layout for support S: G row groups of S lanes; lane g*S + a holds rows g*R ..
// g*R + R - 1 of footprint column a, as RP row pairs and RT (0/1) single tail row. The staged
// table of one oversampling class holds, per row pair k, a block of 32 float2 {kr(2k), kr(2k+1)}
// then a block of 32 float2 {ki(2k), ki(2k+1)} (one entry per lane), then for the tail row a
// block of 32 float2 {kr, ki}.
__host__ __device__ constexpr int lay_rows(int s) { return (s + 32 / s - 1) / (32 / s); }
__host__ __device__ constexpr int lay_groups(int s) { return (s + lay_rows(s) - 1) / lay_rows(s); }
// staged bytes per oversampling class: 2 RP blocks of 32 x float2, then one more if RT
__host__ __device__ constexpr int lay_class_bytes(int s) { return (lay_rows(s) / 2) * 512 + (lay_rows(s) & 1) * 256; }

template <int S>
struct Lay {
  static constexpr int R = lay_rows(S), G = lay_groups(S), NL = G * S;
  static constexpr int RP = R / 2, RT = R & 1, RPA = RP > 0 ? RP : 1;
  static constexpr int CB = lay_class_bytes(S);
};

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
  int group_tiles;          // origin tiles of one tile row sorted as one segment, at most
  int nunits;               // work units (equal shares of the estimated work)
  uint32_t* work;           // [2]: next unit, finished CTAs (both zero between launches)
};

__device__ __forceinline__ unsigned char* dyn_smem() {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return smem_raw;
}

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
__device__ __forceinline__ unsigned long long shfl_down2(unsigned long long v, int d) {
  const uint32_t lo = __shfl_down_sync(0xffffffffu, (uint32_t)v, d);
  const uint32_t hi = __shfl_down_sync(0xffffffffu, (uint32_t)(v >> 32), d);
  return (unsigned long long)lo | ((unsigned long long)hi << 32);
}

// The S x S cells under one footprint origin, distributed over a warp (see Lay).
template <int S>
struct Footprint {
  using L = Lay<S>;
  unsigned long long re[L::RPA], im[L::RPA];   // row pairs (2k, 2k + 1) of this lane's rows
  float tre, tim;                              // tail row 2 RP
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < L::RPA; ++k) re[k] = im[k] = 0ull;
    tre = tim = 0.f;
  }
  // Adds this lane's cells (column col0 + a, rows j0 + row0 + r) to the grid when `pred`.
  __device__ __forceinline__ void flush(bool pred, float2* __restrict__ grid, int n, int j0, int col0, int a,
                                        int row0) const {
    if (!pred) return;
    float2* p = grid + (int64_t)(j0 + row0) * n + col0 + a;
#pragma unroll
    for (int k = 0; k < L::RP; ++k) {
      if (row0 + 2 * k < S) atomicAdd(p + (int64_t)(2 * k) * n, make_float2(lo_of(re[k]), lo_of(im[k])));
      if (row0 + 2 * k + 1 < S) atomicAdd(p + (int64_t)(2 * k + 1) * n, make_float2(hi_of(re[k]), hi_of(im[k])));
    }
    if (L::RT && row0 + 2 * L::RP < S) atomicAdd(p + (int64_t)(2 * L::RP) * n, make_float2(tre, tim));
  }
  // acc(a) <- acc(a + d); columns a + d >= S start at zero.
  __device__ __forceinline__ void slide(int d, int a) {
    const bool keep = a + d < S;
#pragma unroll
    for (int k = 0; k < L::RP; ++k) {
      const unsigned long long r = shfl_down2(re[k], d), i = shfl_down2(im[k], d);
      re[k] = keep ? r : 0ull;
      im[k] = keep ? i : 0ull;
    }
    if (L::RT) {
      const float r = __shfl_down_sync(0xffffffffu, tre, d), i = __shfl_down_sync(0xffffffffu, tim, d);
      tre = keep ? r : 0.f;
      tim = keep ? i : 0.f;
    }
  }
};

// This lane's taps of one record: RP row pairs as {kr(2k), kr(2k+1)} and {ki(2k), ki(2k+1)}, and the tail.
template <int S>
struct Taps {
  float2 r[Lay<S>::RPA], i[Lay<S>::RPA];
  float2 t;
  // Lanes beyond the layout (lane >= NL) read their all-zero table entries.
  __device__ __forceinline__ void load(const unsigned char* cls_base, int lane) {
    using L = Lay<S>;
#pragma unroll
    for (int k = 0; k < L::RP; ++k) {
      r[k] = *(const float2*)(cls_base + k * 512 + lane * 8);
      i[k] = *(const float2*)(cls_base + k * 512 + 256 + lane * 8);
    }
    if (L::RT) t = *(const float2*)(cls_base + L::RP * 512 + lane * 8);
  }
};

// One warp grids the decoded, sorted records [beg, end) of the chunk at byte offset rec_off.
// Staged table (byte offset tab_off): per class, Lay<S>::CB bytes as described at Lay.
// Decoded record: x, y = c (float bits); z = i0 | j0 << 16; w = class byte offset | conj << 31.
template <int S>
__device__ __forceinline__ void warp_grid(int tab_off, int rec_off, int beg, int end, float2* __restrict__ grid, int n) {
  using L = Lay<S>;
  const int lane = threadIdx.x & 31;
  const int g = lane / S, a = lane - g * S;
  const bool active = lane < L::NL;
  const int row0 = g * L::R;
  const unsigned char* tab = dyn_smem() + tab_off;
  const uint4* drec = (const uint4*)(dyn_smem() + rec_off);
  Footprint<S> fp;
  fp.zero();
  uint32_t cz = kNoOrigin;
  int col0 = 0, cj = 0;
#pragma unroll(L::RP > 1 ? 2 : 4)
  for (int q = beg; q < end; ++q) {
    const uint4 rec = drec[q];
    Taps<S> tv;
    tv.load(tab + (rec.w & 0x7fffffffu), lane);
    if (rec.z != cz) {                             // warp-uniform: a new footprint origin
      const int i0 = rec.z & 0xffff, j0 = rec.z >> 16;
      if (cz != kNoOrigin) {
        const int d = i0 - col0;
        if (j0 == cj && d > 0 && d < S) {
          fp.flush(active && a < d, grid, n, cj, col0, a, row0);
          fp.slide(d, a);
        } else {
          fp.flush(active, grid, n, cj, col0, a, row0);
          fp.zero();
        }
      }
      cz = rec.z;
      col0 = i0;
      cj = j0;
    }
    // acc.re += cr kr + be ki, acc.im += ci kr + de ki: c K, or c conj(K) for w < 0
    const uint32_t flip = (rec.w & 0x80000000u) ^ 0x80000000u;
    const float cr = __uint_as_float(rec.x), cim = __uint_as_float(rec.y);
    const float be = __uint_as_float(rec.y ^ flip), de = __uint_as_float(rec.x ^ flip ^ 0x80000000u);
    const unsigned long long CR = pack2(cr, cr), CI = pack2(cim, cim);
    const unsigned long long BE = pack2(be, be), DE = pack2(de, de);
#pragma unroll
    for (int k = 0; k < L::RP; ++k) {
      const unsigned long long kr = pack2(tv.r[k].x, tv.r[k].y), ki = pack2(tv.i[k].x, tv.i[k].y);
      fp.re[k] = fma2(CR, kr, fp.re[k]);
      fp.re[k] = fma2(BE, ki, fp.re[k]);
      fp.im[k] = fma2(CI, kr, fp.im[k]);
      fp.im[k] = fma2(DE, ki, fp.im[k]);
    }
    if (L::RT) {
      fp.tre = fmaf(cr, tv.t.x, fp.tre);
      fp.tre = fmaf(be, tv.t.y, fp.tre);
      fp.tim = fmaf(cim, tv.t.x, fp.tim);
      fp.tim = fmaf(de, tv.t.y, fp.tim);
    }
  }
  if (cz == kNoOrigin) return;
  fp.flush(active, grid, n, cj, col0, a, row0);
}

// Stages plane p's table in the lane layout of Lay<S> at byte offset tab_off.
template <int S>
__device__ __forceinline__ void stage_table(const G2Args& a, int p, int tab_off) {
  using L = Lay<S>;
  constexpr int kPer = L::RP + L::RT;           // entries per lane and class
  const int ncls = a.g.os * a.g.os;
  const float2* src = a.tab + a.tab_off[p];
  unsigned char* dst = dyn_smem() + tab_off;
  for (int i = threadIdx.x; i < ncls * 32 * kPer; i += kThreads) {
    const int cls = i / (32 * kPer), rem = i - cls * (32 * kPer);
    const int k = rem >> 5, lane = rem & 31;
    const int g = lane / S, col = lane - g * S;
    const bool active = lane < L::NL;
    const int b0 = g * L::R + 2 * k;
    const float2* s = src + ((int64_t)cls * S + col) * S;
    const float2 v0 = (active && b0 < S) ? __ldg(s + b0) : make_float2(0.f, 0.f);
    unsigned char* d = dst + cls * L::CB + k * 512 + lane * 8;
    if (k < L::RP) {
      const float2 v1 = (active && b0 + 1 < S) ? __ldg(s + b0 + 1) : make_float2(0.f, 0.f);
      *(float2*)d = make_float2(v0.x, v1.x);
      *(float2*)(d + 256) = make_float2(v0.y, v1.y);
    } else {
      *(float2*)d = v0;
    }
  }
}

// Grids records [s0, s1) of one segment (plane p, support S; origin tiles of one tile row,
// columns x0 .. x0 + width) in chunks of at most `cap` records.
template <int S>
__device__ __noinline__ void grid_segment(const G2Args& a, int p, bool stage, int x0, int y0, int width, uint32_t s0,
                             uint32_t s1, int cap, int tab_off, int rec_off) {
  using L = Lay<S>;
  if (stage) stage_table<S>(a, p, tab_off);
  const int keys = width * a.g.tile_y;
  const int warp = threadIdx.x >> 5;
  const int os = a.g.os;
  uint32_t* counts = (uint32_t*)dyn_smem();
  uint4* drec = (uint4*)(dyn_smem() + rec_off);
  const uint4* grecs = (const uint4*)a.recs;
  for (uint32_t c0 = s0; c0 < s1; c0 += (uint32_t)cap) {
    const int m = (int)min((uint32_t)cap, s1 - c0);
    for (int k = threadIdx.x; k < keys; k += kThreads) counts[k] = 0u;
    __syncthreads();
    // pass 1: histogram of the origin keys (row-major within the segment), 4 loads in flight
    for (int r0 = threadIdx.x; r0 < m; r0 += 4 * kThreads) {
      uint32_t z[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) z[u] = r0 + u * kThreads < m ? __ldcg(&grecs[c0 + r0 + u * kThreads].z) : kNoOrigin;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (z[u] != kNoOrigin) atomicAdd(&counts[((int)(z[u] >> 16) - y0) * width + ((int)(z[u] & 0xffff) - x0)], 1u);
    }
    __syncthreads();
    block_exclusive_scan(keys);
    // pass 2: decode each record into its sorted slot
    for (int r0 = threadIdx.x; r0 < m; r0 += 4 * kThreads) {
      uint4 rec[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r0 + u * kThreads < m) rec[u] = __ldcs(grecs + c0 + r0 + u * kThreads);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (r0 + u * kThreads < m) {
          const int key = ((int)(rec[u].z >> 16) - y0) * width + ((int)(rec[u].z & 0xffff) - x0);
          const int cls = (int)((rec[u].w >> 8) & 0xff) * os + (int)(rec[u].w & 0xff);
          const uint32_t w = (uint32_t)(cls * L::CB) | (rec[u].w & 0x80000000u);
          drec[atomicAdd(&counts[key], 1u)] = make_uint4(rec[u].x, rec[u].y, rec[u].z, w);
        }
      }
    }
    __syncthreads();
    const int beg = (int)((int64_t)m * warp / kWarps), end = (int)((int64_t)m * (warp + 1) / kWarps);
    warp_grid<S>(tab_off, rec_off, beg, end, a.grid, a.g.n);
    __syncthreads();
  }
}

// Grids the records [beg, end) of the (plane, tile)-sorted array, segment by segment.
__device__ void grid_range(const G2Args& a, uint32_t beg, uint32_t end) {
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
    const int rec_off = tab_off + a.g.os * a.g.os * lay_class_bytes(s);
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
    const bool stage = p != cur_plane;
    cur_plane = p;
    const int x0 = tx * a.g.tile_x, y0 = ty * a.g.tile_y;
    const int width = ntiles * a.g.tile_x;
    switch (s) {
#define WP_SEG_CASE(N)                                                                   \
  case N:                                                                                \
    grid_segment<N>(a, p, stage, x0, y0, width, pos, seg_end, cap, tab_off, rec_off);    \
    break;
      WP_SEG_CASE(1) WP_SEG_CASE(2) WP_SEG_CASE(3) WP_SEG_CASE(4) WP_SEG_CASE(5) WP_SEG_CASE(6) WP_SEG_CASE(7)
      WP_SEG_CASE(8) WP_SEG_CASE(9) WP_SEG_CASE(10) WP_SEG_CASE(11) WP_SEG_CASE(12) WP_SEG_CASE(13)
      WP_SEG_CASE(14) WP_SEG_CASE(15) WP_SEG_CASE(16)
#undef WP_SEG_CASE
      default:
        break;
    }
    pos = seg_end;
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_grid_v2(G2Args a) {
  // Work unit u covers the estimated-work range [ctotal u / nunits, ctotal (u + 1) / nunits):
  // cost position x maps to bin b (costoff[b] <= x < costoff[b+1]) and to the record
  // offsets[b] + (x - costoff[b]) / cost_b * count_b, a monotone map, so the units partition
  // the records exactly. Units are taken from the counter from the last one down.
  __shared__ int unit;
  const uint32_t total = a.offsets[a.nbins];
  const uint32_t ctotal = a.costoff[a.nbins];
  auto split = [&](uint64_t x) -> uint32_t {
    if (x >= ctotal) return total;
    const int64_t b = find_bin(a.costoff, a.nbins, (uint32_t)x);
    const uint32_t c0 = a.costoff[b], cb = a.costoff[b + 1] - c0;
    const uint32_t n = a.offsets[b + 1] - a.offsets[b];
    return a.offsets[b] + (uint32_t)(((uint64_t)(x - c0) * n) / cb);
  };
  for (;;) {
    if (threadIdx.x == 0) unit = a.nunits - 1 - (int)atomicAdd(&a.work[0], 1u);
    __syncthreads();
    const int u = unit;
    __syncthreads();
    if (u < 0) break;
    const uint32_t beg = split((uint64_t)ctotal * u / a.nunits);
    const uint32_t end = split((uint64_t)ctotal * (u + 1) / a.nunits);
    if (beg < end) grid_range(a, beg, end);
  }
  // the last CTA to finish leaves both counters zero for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.work[1], 1u) == gridDim.x - 1) {
      a.work[0] = 0u;
      a.work[1] = 0u;
      __threadfence();
    }
  }
}

}  // namespace

// Dynamic shared memory of the launch (the device's opt-in maximum), or 0 when the geometry
// is outside the kernel's limits (then the baseline kernel of grid.cu runs).
size_t grid_v2_smem(const wp_ctx* ctx, int* group_tiles) {
  const int smax = *std::max_element(ctx->supp.begin(), ctx->supp.end());
  if (smax > kMaxS || ctx->prm.table_type != WP_TABLE_F32) return 0;
  const int os = ctx->prm.oversample;
  const int tx = ctx->geo.tile_x, ty = ctx->geo.tile_y;
  if ((int64_t)tx * ty > kMaxKeys) return 0;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->prm.device) != cudaSuccess)
    return 0;
  const size_t bytes = (size_t)optin - 1024;        // room for the static scan scratch
  size_t tab = 0;
  for (int sp : ctx->supp) tab = std::max(tab, (size_t)os * os * lay_class_bytes(sp));
  if ((size_t)kCountsBytes + tab + (size_t)kMinChunk * sizeof(Record) > bytes) return 0;
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
  a.nunits = ctx->nsm * kUnitsPerCta;
  a.work = ctx->d_work;
  cudaError_t e;
  if ((e = launch_bin_costs(ctx, s))) return e;
  if ((e = cudaFuncSetAttribute(k_grid_v2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
  k_grid_v2<<<ctx->nsm, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wp
