// Register-accumulating gridding kernel (the hot path of wp_grid).
//
// Gridding (Sec. 2.1/2.2 of Lao et al. 2019): visibility k adds c_k K_k(a, b) to the cell
// (i0 + a, j0 + b) of its S x S footprint. The paper's GPU scheme (Fig. 2, after Romein)
// gives each thread one support tap and keeps that tap's sum in a register while the
// grid point stays the same; here the same idea is organised around sorted bins:
//
//   * A CTA takes an equal contiguous share of the (plane, tile)-sorted records and sorts
//     each chunk of them by footprint origin (row j0, then column i0) in shared memory.
//   * A "stream" of S lanes walks its part of the sorted chunk. Lane b owns footprint row
//     b, so for a run of records with the same j0 its cells are on grid row j0 + b.
//   * Register x of a lane accumulates the cells whose column is congruent to x modulo S.
//     Every footprint covers exactly one such cell per class: a = (x - i0) mod S is the
//     tap column, i0 + a the cell. While the records' i0 grows by less than S, a class
//     keeps its cell and its register keeps accumulating; when i0 passes it, that one
//     register is added to the shared-memory sub-grid (a "flush") and restarts.
//   * Per tap a lane does one shared-memory (or L1) load and four FMAs; the tap address
//     for class x is one of two base pointers plus a compile-time offset.
//   * The sub-grid (tile + (S-1)-cell halo) is merged into the HBM grid with one vector
//     atomic per non-zero cell when the CTA leaves the bin.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace wp {

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 2048;  // records sorted per pass (u16 indices)
constexpr int kMaxS = 32;

struct G2Args {
  const Record* recs;
  const uint32_t* offsets;
  const uint32_t* costoff;  // [nbins + 1] prefix sums of per-bin work estimates
  int64_t nbins;
  Geometry g;
  const float2* tab;        // stored tables (f32), layout [plane][oy*os+ox][a][b]
  const int64_t* tab_off;
  float2* grid;
  int table_in_smem;        // stage each plane's table in shared memory
  int table_capacity;       // float2 entries reserved for it
  int sub_capacity;         // float2 entries of the sub-grid
  int group_tiles;          // origin tiles of one tile row gridded as one segment, at most
};

__device__ __forceinline__ unsigned char* dyn_smem() {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return smem_raw;
}

// Shared-memory map (dynamic, byte offsets): table | sub-grid | records | counts | sorted indices.
// Pointers are rebuilt from the __shared__ base where they are used, so that loads through
// them are shared-memory loads.
struct Smem {
  int table, sub, recs, counts, sidx;
  __device__ __forceinline__ float2* table_p() const { return (float2*)(dyn_smem() + table); }
  __device__ __forceinline__ float2* sub_p() const { return (float2*)(dyn_smem() + sub); }
  __device__ __forceinline__ Record* recs_p() const { return (Record*)(dyn_smem() + recs); }
  __device__ __forceinline__ uint32_t* counts_p() const { return (uint32_t*)(dyn_smem() + counts); }
  __device__ __forceinline__ uint16_t* sidx_p() const { return (uint16_t*)(dyn_smem() + sidx); }
};

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

// In-place exclusive scan of counts[0..n) by the whole block (n <= 4 * kThreads * 2).
__device__ void block_exclusive_scan(uint32_t* counts, int n) {
  __shared__ uint32_t warp_sums[kWarps];
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

// Adds a lane's S row accumulators (column col, rows row0 .. row0 + S - 1 of the sub-grid)
// into the sub-grid and clears them. P = S rounded up to even: accumulators hold row pairs.
template <int S, int P>
__device__ __forceinline__ void flush_column(unsigned long long (&re)[P / 2], unsigned long long (&im)[P / 2],
                                             float2* sub, int pitch, int row0, int col) {
  float2* cell = sub + row0 * pitch + col;
#pragma unroll
  for (int q = 0; q < P / 2; ++q) {
    const float r0 = lo_of(re[q]), r1 = hi_of(re[q]), i0 = lo_of(im[q]), i1 = hi_of(im[q]);
    if (r0 != 0.f || i0 != 0.f) {
      atomicAdd(&cell[(2 * q) * pitch].x, r0);
      atomicAdd(&cell[(2 * q) * pitch].y, i0);
    }
    if (2 * q + 1 < S && (r1 != 0.f || i1 != 0.f)) {
      atomicAdd(&cell[(2 * q + 1) * pitch].x, r1);
      atomicAdd(&cell[(2 * q + 1) * pitch].y, i1);
    }
    re[q] = 0ull;
    im[q] = 0ull;
  }
}

// One stream of S lanes grids the decoded, sorted records drec[beg..end) of a chunk.
// Lane x owns the cells whose column is congruent to x modulo S; for a run of records with
// the same origin row j0 its S registers (row pairs) accumulate rows j0 .. j0 + S - 1 of its
// current column. For a record with origin i0 the lane's tap column is a = (x - i0) mod S and
// its cell column i0 + a; when that column moves on (i0 passed x), the lane flushes.
// Shared table layout (staged per plane): [cls][a][row pair q] = {re(2q), re(2q+1), im(2q), im(2q+1)}.
// Decoded record: x, y = c (float bits); z = i0 | j0 << 16; w = cls * S | r0x << 20 | conj << 31.
template <int S>
__device__ void stream_grid(const Smem& sm, int x0, int y0, int pitch, int beg, int end, int x) {
  constexpr int P = S + (S & 1);
  unsigned long long re[P / 2], im[P / 2];
#pragma unroll
  for (int q = 0; q < P / 2; ++q) re[q] = im[q] = 0ull;
  const float4* tab = (const float4*)sm.table_p();
  float2* sub = sm.sub_p();
  const uint4* drec = (const uint4*)sm.recs_p();
  int cj = -1, ci = 0, col = -1;                   // run row, last origin column, this lane's cell column
  uint4 nxt = beg < end ? drec[beg] : make_uint4(0u, 0u, 0u, 0u);
  for (int q = beg; q < end; ++q) {
    const uint4 rec = nxt;
    if (q + 1 < end) nxt = drec[q + 1];
    const int i0 = rec.z & 0xffff, j0 = rec.z >> 16;
    if (j0 != cj || i0 < ci) {                     // new run (row): every lane flushes its column
      if (col >= 0) flush_column<S, P>(re, im, sub, pitch, cj - y0, col - x0);
      cj = j0;
      col = -1;
    }
    ci = i0;
    const int r0x = (rec.w >> 20) & 0x1f;
    const int a = x - r0x + (x < r0x ? S : 0);
    const int cx = i0 + a;
    if (cx != col) {                               // this lane's class moved to a new cell column
      if (col >= 0) flush_column<S, P>(re, im, sub, pitch, cj - y0, col - x0);
      col = cx;
    }
    const float cr = __uint_as_float(rec.x), cim = __uint_as_float(rec.y);
    const bool conj = (rec.w >> 31) != 0;
    // acc.re += cr kr + be ki, acc.im += cim kr + de ki (c * K, or c * conj(K) for w < 0)
    const unsigned long long CR = pack2(cr, cr), CI = pack2(cim, cim);
    const float be = conj ? cim : -cim, de = conj ? -cr : cr;
    const unsigned long long BE = pack2(be, be), DE = pack2(de, de);
    const float4* t = tab + ((int)(rec.w & 0xfffff) + a) * (P / 2);
#pragma unroll
    for (int qq = 0; qq < P / 2; ++qq) {
      const float4 v = t[qq];
      const unsigned long long kr = pack2(v.x, v.y), ki = pack2(v.z, v.w);
      re[qq] = fma2(CR, kr, re[qq]);
      re[qq] = fma2(BE, ki, re[qq]);
      im[qq] = fma2(CI, kr, im[qq]);
      im[qq] = fma2(DE, ki, im[qq]);
    }
  }
  if (col >= 0) flush_column<S, P>(re, im, sub, pitch, cj - y0, col - x0);
}

// Grids records [s0, s1) of one segment (plane p; origin tiles of one tile row, columns
// x0 .. x0 + width) into the sub-grid (all zero on entry); widens [*jlo, *jhi] to the
// footprint-origin rows it saw.
template <int S>
__device__ void grid_segment(const G2Args& a, const Smem& sm, int p, int x0, int y0, int width, uint32_t s0,
                             uint32_t s1, int* jlo, int* jhi) {
  const int pitch = (width + S - 1) | 1;
  const int keys = width * a.g.tile_y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kSpw = 32 / S;                     // streams per warp
  const int stream = lane / S, x = lane - stream * S;
  const int os = a.g.os;
  uint4* drec = (uint4*)sm.recs_p();
  uint32_t* counts = sm.counts_p();
  uint16_t* rkey = sm.sidx_p();
  const uint4* grecs = (const uint4*)a.recs;
  for (uint32_t c0 = s0; c0 < s1; c0 += kChunk) {
    const int m = (int)min((uint32_t)kChunk, s1 - c0);
    for (int k = threadIdx.x; k < keys; k += kThreads) counts[k] = 0u;
    __syncthreads();
    // pass 1: origin key of every record (row-major within the segment) and its histogram
    for (int r = threadIdx.x; r < m; r += kThreads) {
      const uint4 rec = __ldcg(grecs + c0 + r);
      const int key = ((int)(rec.z >> 16) - y0) * width + ((int)(rec.z & 0xffff) - x0);
      rkey[r] = (uint16_t)key;
      atomicAdd(&counts[key], 1u);
    }
    __syncthreads();
    block_exclusive_scan(counts, keys);
    // pass 2: decode each record into its sorted slot
    for (int r = threadIdx.x; r < m; r += kThreads) {
      const uint4 rec = __ldcs(grecs + c0 + r);
      const int i0 = rec.z & 0xffff;
      const int cls = (int)((rec.w >> 8) & 0xff) * os + (int)(rec.w & 0xff);
      const uint32_t w = (uint32_t)(cls * S) | ((uint32_t)(i0 % S) << 20) | (rec.w & 0x80000000u);
      drec[atomicAdd(&counts[rkey[r]], 1u)] = make_uint4(rec.x, rec.y, rec.z, w);
    }
    __syncthreads();
    *jlo = min(*jlo, (int)(drec[0].z >> 16));          // sorted: first and last rows
    *jhi = max(*jhi, (int)(drec[m - 1].z >> 16));
    if (stream < kSpw) {
      const int gs = warp * kSpw + stream, nst = kWarps * kSpw;
      const int beg = (int)((int64_t)m * gs / nst), end = (int)((int64_t)m * (gs + 1) / nst);
      stream_grid<S>(sm, x0, y0, pitch, beg, end, x);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_grid_v2(G2Args a) {
  Smem sm;
  sm.table = 0;
  sm.sub = sm.table + a.table_capacity * (int)sizeof(float2);
  sm.recs = sm.sub + a.sub_capacity * (int)sizeof(float2);          // sub_capacity is even: 16-byte aligned
  sm.counts = sm.recs + kChunk * (int)sizeof(Record);
  sm.sidx = sm.counts + (a.group_tiles * a.g.tile_x * a.g.tile_y + 1) * (int)sizeof(uint32_t);
  float2* sub = sm.sub_p();

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
  for (int q = threadIdx.x; q < a.sub_capacity; q += kThreads) sub[q] = make_float2(0.f, 0.f);
  int64_t bin = find_bin(a.offsets, a.nbins, beg);
  uint32_t pos = beg;
  int cur_plane = -1;
  while (pos < end) {
    bin = advance_bin(a.offsets, bin, a.nbins, pos);
    const int p = (int)(bin / a.g.ntiles);
    const int64_t tile = bin - (int64_t)p * a.g.ntiles;
    const int ty = (int)(tile / a.g.ntx), tx = (int)(tile - (int64_t)ty * a.g.ntx);
    // a segment: this bin, plus the following bins of the same tile row while the records
    // still fit one chunk (sparse tiles are gridded together, dense ones alone)
    uint32_t bound[8];                            // ends of this bin and the next 7 (independent loads)
#pragma unroll
    for (int k = 0; k < 8; ++k) bound[k] = a.offsets[min(bin + k + 1, a.nbins)];
    uint32_t seg_end = min(end, bound[0]);
    int ntiles = 1;
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      if (ntiles == k && k < a.group_tiles && tx + k < a.g.ntx && seg_end < end) {
        const uint32_t nxt = min(end, bound[k]);
        if (nxt - pos <= (uint32_t)kChunk) {
          seg_end = nxt;
          ntiles = k + 1;
        }
      }
    }
    const int x0 = tx * a.g.tile_x, y0 = ty * a.g.tile_y;
    const int width = ntiles * a.g.tile_x;
    const int s = a.g.supp[p];
    const int pitch = (width + s - 1) | 1, rows = a.g.tile_y + s - 1;
    if (p != cur_plane) {
      // stage the plane's table as row pairs: [cls][a][q] = {re(2q), re(2q+1), im(2q), im(2q+1)}
      const int half = (s + 1) / 2;
      const int n = a.g.os * a.g.os * s * half;
      const float2* src = a.tab + a.tab_off[p];
      float4* dst = (float4*)sm.table_p();
      for (int i = threadIdx.x; i < n; i += kThreads) {
        const int ca = i / half, q = i - ca * half;
        const float2 v0 = __ldg(&src[ca * s + 2 * q]);
        const float2 v1 = (2 * q + 1 < s) ? __ldg(&src[ca * s + 2 * q + 1]) : make_float2(0.f, 0.f);
        dst[i] = make_float4(v0.x, v1.x, v0.y, v1.y);
      }
      cur_plane = p;
    }
    __syncthreads();
    int jlo = 1 << 30, jhi = -1;
    switch (s) {
#define WP_SEG_CASE(N)                                                                  \
  case N:                                                                               \
    grid_segment<N>(a, sm, p, x0, y0, width, pos, seg_end, &jlo, &jhi);                 \
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
    // Merge the rows the segment touched (origin rows jlo..jhi plus the S-1 halo rows) into
    // the HBM grid, one vector atomic per non-zero cell, and leave the sub-grid zero again.
    const int cols = width + s - 1;
    const int r_end = min(rows, jhi - y0 + s);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = jlo - y0 + warp; r < r_end; r += kWarps) {
      const int gy = y0 + r;
      for (int c = lane; c < cols; c += 32) {
        float2* cell = &sub[r * pitch + c];
        const float2 v = *cell;
        if (v.x != 0.f || v.y != 0.f) {
          if (gy < a.g.n && x0 + c < a.g.n) atomicAdd(&a.grid[(int64_t)gy * a.g.n + x0 + c], v);
          *cell = make_float2(0.f, 0.f);
        }
      }
    }
    __syncthreads();
    pos = seg_end;
  }
}

}  // namespace

// Shared memory the kernel needs, or 0 when the geometry is outside its limits (then the
// baseline kernel of grid.cu runs).
size_t grid_v2_smem(const wp_ctx* ctx, int* table_capacity, int* sub_capacity, int* group_tiles) {
  const int smax = *std::max_element(ctx->supp.begin(), ctx->supp.end());
  if (smax > kMaxS || ctx->prm.table_type != WP_TABLE_F32) return 0;
  const int os = ctx->prm.oversample;
  if ((int64_t)os * os * smax >= (1 << 20)) return 0;   // cls * S packed in 20 bits
  const int tx = ctx->geo.tile_x, ty = ctx->geo.tile_y;
  if ((int64_t)tx * ty > 4096) return 0;
  *group_tiles = std::max(1, std::min(8, 4096 / (tx * ty)));
  const int gw = *group_tiles * tx;
  const int sub = ((((gw + smax - 1) | 1) * (ty + smax - 1)) + 1) & ~1;   // even: records stay 16-byte aligned
  const int pmax = smax + (smax & 1);
  int cap = 0;                                      // float2 entries of the largest staged table
  for (int sp : ctx->supp) cap = std::max(cap, os * os * sp * (sp + (sp & 1)));
  const size_t bytes = sizeof(float2) * ((size_t)cap + sub) + sizeof(Record) * kChunk +
                       sizeof(uint32_t) * ((size_t)gw * ty + 1) + sizeof(uint16_t) * kChunk + 64;
  (void)pmax;
  if (bytes > 227 * 1024) return 0;
  *table_capacity = cap;
  *sub_capacity = sub;
  return bytes;
}

cudaError_t launch_grid_v2(wp_ctx* ctx, float2* grid, cudaStream_t s, bool* used) {
  int tab_cap = 0, sub_cap = 0, group = 1;
  const size_t smem = grid_v2_smem(ctx, &tab_cap, &sub_cap, &group);
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
  a.table_in_smem = 1;
  a.table_capacity = tab_cap;
  a.sub_capacity = sub_cap;
  a.group_tiles = group;
  cudaError_t e;
  if ((e = launch_bin_costs(ctx, s))) return e;
  if ((e = cudaFuncSetAttribute(k_grid_v2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
  k_grid_v2<<<ctx->nsm, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace wp
