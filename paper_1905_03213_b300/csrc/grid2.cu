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
#include <cstring>

#include "internal.h"
#include "warp_common.cuh"

namespace wp {

namespace {

struct G2Args {
  const Record* recs;
  const uint32_t* offsets;
  const uint32_t* costoff;  // [nbins + 1] prefix sums of per-bin work estimates
  int64_t nbins;
  Geometry g;
  const void* tab;          // stored tables (f32, f16 or bf16 taps), layout [plane][oy*os+ox][a][b]
  const int64_t* tab_off;
  const unsigned char* lanetab;   // lane-order tables of the planes with S > 16 (global)
  const int64_t* lanetab_off;     // [Nw] byte offset of each plane in lanetab (-1: none)
  float2* grid;
  int smem_bytes;           // dynamic shared memory of the launch
  int group_tiles;          // origin tiles of one tile row sorted as one segment, at most
  int nunits;               // work units (equal shares of the estimated work)
  uint32_t* work;           // [2]: next unit, finished CTAs (both zero between launches)
};

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
  // Adds this lane's cells to the grid where `pred`: rows r < nrow of its column, the first at
  // cell index idx (32-bit: n <= 32768), the next ones n cells apart. Predicated, no branch.
  __device__ __forceinline__ void flush(bool pred, float2* __restrict__ grid, uint32_t idx, uint32_t n, int nrow) const {
#pragma unroll
    for (int k = 0; k < L::RP; ++k) {
      red_add2_if(pred && 2 * k < nrow, grid + idx, lo_of(re[k]), lo_of(im[k]));
      idx += n;
      red_add2_if(pred && 2 * k + 1 < nrow, grid + idx, hi_of(re[k]), hi_of(im[k]));
      idx += n;
    }
    if (L::RT) red_add2_if(pred && 2 * L::RP < nrow, grid + idx, tre, tim);
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

// One warp grids the decoded, sorted records [beg, end) of the chunk at byte offset rec_off.
// Table: staged in shared memory at byte offset tab_off, or (kGlobal: S > 16 and too large to
// stage beside a chunk) the plane's lane-order copy at gtab; per class Lay<S, T>::CB bytes as
// described at Lay. Row half h (S > 16).
// Decoded record: x, y = c (float bits); z = i0 | j0 << 16; w = class byte offset | conj << 31.
// Taps are widened to float32; every product and sum is float32.
template <int S, class T, bool kGlobal>
__device__ __forceinline__ void warp_grid(int tab_off, const unsigned char* gtab, int h, int rec_off, int beg,
                                          int end, float2* __restrict__ grid, int n) {
  using L = Lay<S, T>;
  const int lane = threadIdx.x & 31;
  const int g = lane / S, a = lane - g * S;
  const bool active = lane < L::NL;
  const int row0 = L::H > 1 ? h * L::R : g * L::R;
  const unsigned char* tab = (kGlobal ? gtab : dyn_smem() + tab_off) + h * L::HB;
  const uint4* drec = (const uint4*)(dyn_smem() + rec_off);
  Footprint<S> fp;
  fp.zero();
  uint32_t cz = kNoOrigin;
  int col0 = 0, cj = 0;
  // this lane's rows inside the footprint, and its offset from the origin's cell index
  const int nrow = active ? min(L::R, S - row0) : 0;
  const uint32_t lane_off = (uint32_t)row0 * (uint32_t)n + (uint32_t)a;
  uint32_t cidx = 0;                               // cell index of this lane's first cell
#pragma unroll(L::RP > 1 ? 2 : 4)
  for (int q = beg; q < end; ++q) {
    const uint4 rec = drec[q];
    Taps<S, T, kGlobal> tv;
    tv.load(tab + (rec.w & 0x7fffffffu), lane);
    if (rec.z != cz) {                             // warp-uniform: a new footprint origin
      const int i0 = rec.z & 0xffff, j0 = rec.z >> 16;
      const int d = i0 - col0;
      const bool slide = j0 == cj && (unsigned)(d - 1) < (unsigned)(S - 1);   // 0 < d < S on the same row
      // a slide adds the d leaving columns to the grid, any other move every cell
      fp.flush(cz != kNoOrigin && (!slide || a < d), grid, cidx, (uint32_t)n, nrow);
      if (slide) fp.slide(d, a);
      else fp.zero();
      cz = rec.z;
      col0 = i0;
      cj = j0;
      cidx = (uint32_t)j0 * (uint32_t)n + (uint32_t)i0 + lane_off;
    }
    // acc.re += cr kr + be ki, acc.im += ci kr + de ki: c K, or c conj(K) for w < 0
    const uint32_t flip = (rec.w & 0x80000000u) ^ 0x80000000u;
    const float cr = __uint_as_float(rec.x), cim = __uint_as_float(rec.y);
    const float be = __uint_as_float(rec.y ^ flip), de = __uint_as_float(rec.x ^ flip ^ 0x80000000u);
    const unsigned long long CR = pack2(cr, cr), CI = pack2(cim, cim);
    const unsigned long long BE = pack2(be, be), DE = pack2(de, de);
#pragma unroll
    for (int k = 0; k < L::RP; ++k) {
      const unsigned long long kr = tv.r[k], ki = tv.i[k];
      fp.re[k] = fma2(CR, kr, fp.re[k]);
      fp.re[k] = fma2(BE, ki, fp.re[k]);
      fp.im[k] = fma2(CI, kr, fp.im[k]);
      fp.im[k] = fma2(DE, ki, fp.im[k]);
    }
    if (L::RT) {
      fp.tre = fmaf(cr, tv.tr, fp.tre);
      fp.tre = fmaf(be, tv.ti, fp.tre);
      fp.tim = fmaf(cim, tv.tr, fp.tim);
      fp.tim = fmaf(de, tv.ti, fp.tim);
    }
  }
  fp.flush(cz != kNoOrigin, grid, cidx, (uint32_t)n, nrow);
}

template <int S, class T>
__device__ __noinline__ void grid_segment(const G2Args& a, int p, bool stage, bool staged, int x0, int y0, int width,
                                          uint32_t s0, uint32_t s1, int cap, int tab_off, int rec_off) {
  using L = Lay<S, T>;
  if (staged && stage) stage_table<S, T>((const T*)a.tab + a.tab_off[p], a.g.os, tab_off);
  const unsigned char* gtab = staged ? nullptr : a.lanetab + a.lanetab_off[p];
  const int keys = width * a.g.tile_y;
  const int warp = threadIdx.x >> 5;
  constexpr int kPieces = kWarps / L::H;            // warps of a row-half pair share a piece
  const int piece = warp / L::H, h = warp % L::H;
  for (uint32_t c0 = s0; c0 < s1; c0 += (uint32_t)cap) {
    const int m = (int)min((uint32_t)cap, s1 - c0);
    sort_chunk<S, T>((const uint4*)a.recs, nullptr, c0, m, x0, y0, width, keys, a.g.os, rec_off);
    const int beg = (int)((int64_t)m * piece / kPieces), end = (int)((int64_t)m * (piece + 1) / kPieces);
    if (L::H == 1 || staged) warp_grid<S, T, false>(tab_off, nullptr, h, rec_off, beg, end, a.grid, a.g.n);
    else warp_grid<S, T, true>(tab_off, gtab, h, rec_off, beg, end, a.grid, a.g.n);
    __syncthreads();
  }
}

// Grids the records [beg, end) of the (plane, tile)-sorted array, segment by segment.
template <class T>
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
    // tables of S > 16 are staged too when they leave room for a chunk of kStagedChunk records
    const int tbytes = a.g.os * a.g.os * lay_class_bytes(s, TabElem<T>::E);
    const bool staged = s <= kMaxStagedS || tab_off + tbytes + kStagedChunk * (int)sizeof(Record) <= a.smem_bytes;
    const int rec_off = tab_off + (staged ? tbytes : 0);
    const int cap = min(kMaxChunk, (a.smem_bytes - rec_off) / (int)sizeof(Record));
    int ntiles = 1;
    const uint32_t seg_end = segment_end(a.offsets, a.nbins, bin, tx, a.g.ntx, pos, end, cap, a.group_tiles, &ntiles);
    const bool stage = staged && p != cur_plane;
    cur_plane = staged ? p : -1;                  // an unstaged segment's records overwrite the table
    const int x0 = tx * a.g.tile_x, y0 = ty * a.g.tile_y;
    const int width = ntiles * a.g.tile_x;
    switch (s) {
#define WP_SEG_CASE(N)                                                                   \
  case N:                                                                                \
    grid_segment<N, T>(a, p, stage, staged, x0, y0, width, pos, seg_end, cap, tab_off, rec_off);   \
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

template <class T>
__global__ void __launch_bounds__(kThreads, 1) k_grid_v2(G2Args a) {
  for_each_unit<true>(a.offsets, a.costoff, a.nbins, a.nunits, a.work,
                [&](uint32_t beg, uint32_t end) { grid_range<T>(a, beg, end); });
}

// ---- lane-order tables in global memory for the planes with S > 16 ----

// Writes plane tables (stored layout [oy*os+ox][a][b] of T) in the lane order of Lay<S> with
// two row halves, for a runtime support s (17 .. 32); grid-stride over the table's entries.
template <class T>
__global__ void k_lane_table(const T* __restrict__ src, int s, int os, unsigned char* __restrict__ dst) {
  const int n = half_entries(os, s);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) write_half_entry<T>(src, s, dst, i);
}

// ---- many jobs in one persistent launch (wp_batch_grid) ----

// Finer units than a single job uses: the units running at one time then cover a small slice of
// the concatenated work, so the CTAs of a moment mostly share one job's grid and tables in L2.
constexpr int kBatchUnitsPerCta = 64;

struct BatchArgs {
  const G2Args* jobs;        // [njobs] per-job arguments (device), smem_bytes shared
  const uint64_t* jobcost;   // [njobs + 1] prefix sums of each job's total estimated work
  int njobs;
  int nunits;
  uint32_t* work;            // [2]: next unit, finished CTAs (both zero between launches)
};

// jobcost[j + 1] = jobcost[j] + (total estimated work of job j), one thread.
__global__ void k_job_costs(const G2Args* __restrict__ jobs, int njobs, uint64_t* __restrict__ jobcost) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint64_t c = 0;
  jobcost[0] = 0;
  for (int j = 0; j < njobs; ++j) {
    c += jobs[j].costoff[jobs[j].nbins];
    jobcost[j + 1] = c;
  }
}

// Record position of cost position x (0 <= x <= ctotal) of one job: the monotone map of the
// single-job schedule.
__device__ __forceinline__ uint32_t job_split(const G2Args& a, uint64_t x) {
  const uint32_t total = a.offsets[a.nbins];
  const uint32_t ctotal = a.costoff[a.nbins];
  if (x >= ctotal) return total;
  const int64_t b = find_bin(a.costoff, a.nbins, (uint32_t)x);
  const uint32_t c0 = a.costoff[b], cb = a.costoff[b + 1] - c0;
  const uint32_t n = a.offsets[b + 1] - a.offsets[b];
  return a.offsets[b] + (uint32_t)(((uint64_t)(x - c0) * n) / cb);
}

// Work unit u covers [C u / nunits, C (u + 1) / nunits) of the concatenated work of all jobs
// (C = jobcost[njobs]); the part inside job j is gridded with job j's arguments. Units are
// taken from the counter from the last one down.
template <class T>
__global__ void __launch_bounds__(kThreads, 1) k_grid_batch(BatchArgs b) {
  __shared__ int unit;
  const uint64_t ctot = b.jobcost[b.njobs];
  for (;;) {
    if (threadIdx.x == 0) unit = b.nunits - 1 - (int)atomicAdd(&b.work[0], 1u);
    __syncthreads();
    const int u = unit;
    __syncthreads();
    if (u < 0) break;
    const uint64_t x0 = ctot * (uint64_t)u / (uint64_t)b.nunits, x1 = ctot * (uint64_t)(u + 1) / (uint64_t)b.nunits;
    int j = 0;
    while (j + 1 < b.njobs && b.jobcost[j + 1] <= x0) ++j;
    for (; j < b.njobs && b.jobcost[j] < x1; ++j) {
      const G2Args a = b.jobs[j];
      const uint64_t lo = max(x0, b.jobcost[j]) - b.jobcost[j], hi = min(x1, b.jobcost[j + 1]) - b.jobcost[j];
      const uint32_t beg = job_split(a, lo), end = job_split(a, hi);
      if (beg < end) grid_range<T>(a, beg, end);
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&b.work[1], 1u) == gridDim.x - 1) {
      b.work[0] = 0u;
      b.work[1] = 0u;
      __threadfence();
    }
  }
}

}  // namespace

// Dynamic shared memory of the launch (the device's opt-in maximum), or 0 when the geometry
// is outside the kernel's limits (then the baseline kernel of grid.cu runs).
size_t grid_v2_smem(const wp_ctx* ctx, int* group_tiles) {
  const int smax = *std::max_element(ctx->supp.begin(), ctx->supp.end());
  if (smax > kMaxS) return 0;
  const int e = ctx->prm.table_type == WP_TABLE_F32 ? 4 : 2;
  const int os = ctx->prm.oversample;
  const int tx = ctx->geo.tile_x, ty = ctx->geo.tile_y;
  if ((int64_t)tx * ty > kMaxKeys) return 0;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->prm.device) != cudaSuccess)
    return 0;
  const size_t bytes = (size_t)optin - 1024;        // room for the static scan scratch
  size_t tab = 0;
  for (int sp : ctx->supp) tab = std::max(tab, (size_t)lay_staged_bytes(os, sp, e));
  if (smax > kMaxStagedS && !ctx->d_lanetab) return 0;
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
  a.tab = ctx->d_tab;
  a.tab_off = ctx->d_tab_off;
  a.lanetab = (const unsigned char*)ctx->d_lanetab;
  a.lanetab_off = ctx->d_lanetab_off;
  a.grid = grid;
  a.smem_bytes = (int)smem;
  a.group_tiles = group;
  a.nunits = ctx->nsm * kUnitsPerCta;
  a.work = ctx->d_work;
  cudaError_t e;
  if ((e = launch_bin_costs(ctx, s))) return e;
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err) return err;
    kern<<<ctx->nsm, kThreads, smem, s>>>(a);
    return cudaGetLastError();
  };
  switch (ctx->prm.table_type) {
    case WP_TABLE_F16: return run(k_grid_v2<__half2>);
    case WP_TABLE_BF16: return run(k_grid_v2<__nv_bfloat162>);
    default: return run(k_grid_v2<float2>);
  }
}

}  // namespace wp

namespace wp {

size_t grid_job_desc_bytes() { return sizeof(G2Args); }

// Host-side arguments of one job for the multi-job launch (job's context, grid and the launch's
// shared-memory size); the job's own work-estimate scan must have run before the launch.
void grid_job_desc(wp_ctx* ctx, float2* grid, size_t smem, void* out) {
  int group = 1;
  grid_v2_smem(ctx, &group);
  G2Args a;
  a.recs = (const Record*)ctx->records.ptr;
  a.offsets = ctx->d_offsets;
  a.costoff = ctx->d_costoff;
  a.nbins = ctx->nbins;
  a.g = ctx->geo;
  a.tab = ctx->d_tab;
  a.tab_off = ctx->d_tab_off;
  a.lanetab = (const unsigned char*)ctx->d_lanetab;
  a.lanetab_off = ctx->d_lanetab_off;
  a.grid = grid;
  a.smem_bytes = (int)smem;
  a.group_tiles = group;
  a.nunits = 0;
  a.work = nullptr;
  memcpy(out, &a, sizeof(a));
}

cudaError_t prepare_grid_batch(int table_type, size_t smem) {
  switch (table_type) {
    case WP_TABLE_F16: return cudaFuncSetAttribute(k_grid_batch<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case WP_TABLE_BF16: return cudaFuncSetAttribute(k_grid_batch<__nv_bfloat162>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    default: return cudaFuncSetAttribute(k_grid_batch<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
}

cudaError_t launch_grid_batch(const void* d_jobs, int njobs, uint64_t* d_jobcost, uint32_t* d_work, int table_type,
                              size_t smem, int nsm, cudaStream_t s) {
  k_job_costs<<<1, 32, 0, s>>>((const G2Args*)d_jobs, njobs, d_jobcost);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  BatchArgs b;
  b.jobs = (const G2Args*)d_jobs;
  b.jobcost = d_jobcost;
  b.njobs = njobs;
  b.nunits = nsm * kBatchUnitsPerCta;
  b.work = d_work;
  switch (table_type) {
    case WP_TABLE_F16: k_grid_batch<__half2><<<nsm, kThreads, smem, s>>>(b); break;
    case WP_TABLE_BF16: k_grid_batch<__nv_bfloat162><<<nsm, kThreads, smem, s>>>(b); break;
    default: k_grid_batch<float2><<<nsm, kThreads, smem, s>>>(b); break;
  }
  return cudaGetLastError();
}

}  // namespace wp

namespace wp {

// Bytes of the lane-order table of one plane with support s (0 when it is staged instead).
size_t lane_table_bytes(int s, int os, int table_type) {
  const int e = table_type == WP_TABLE_F32 ? 4 : 2;
  return s > kMaxStagedS && s <= kMaxS ? (size_t)os * os * lay_class_bytes(s, e) : 0;
}

cudaError_t launch_lane_tables(wp_ctx* ctx, cudaStream_t s) {
  if (!ctx->d_lanetab) return cudaSuccess;
  const int os = ctx->prm.oversample;
  for (int p = 0; p < ctx->prm.n_w; ++p) {
    if (ctx->lanetab_off[p] < 0) continue;
    const int sp = ctx->supp[p];
    unsigned char* dst = (unsigned char*)ctx->d_lanetab + ctx->lanetab_off[p];
    const int blocks = std::min(1024, (os * os * 2 * 32 * 16 + 255) / 256);
    switch (ctx->prm.table_type) {
      case WP_TABLE_F16:
        k_lane_table<__half2><<<blocks, 256, 0, s>>>((const __half2*)ctx->d_tab + ctx->tab_off[p], sp, os, dst);
        break;
      case WP_TABLE_BF16:
        k_lane_table<__nv_bfloat162><<<blocks, 256, 0, s>>>((const __nv_bfloat162*)ctx->d_tab + ctx->tab_off[p], sp,
                                                            os, dst);
        break;
      default:
        k_lane_table<float2><<<blocks, 256, 0, s>>>((const float2*)ctx->d_tab + ctx->tab_off[p], sp, os, dst);
        break;
    }
    ++ctx->launches;
    const cudaError_t e = cudaGetLastError();
    if (e) return e;
  }
  return cudaSuccess;
}

}  // namespace wp
