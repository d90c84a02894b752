// Register-accumulating gridding kernel (the hot path of wp_grid).
//
// Gridding (Sec. 2.1/2.2 of Lao et al. 2019): visibility k adds c_k K_k(a, b) to the cell
// (i0 + a, j0 + b) of its S x S footprint. The paper's GPU scheme (Fig. 2, after Romein)
// keeps each support tap's running sum in a register while the grid point it maps to stays
// the same; here that idea is organised around records sorted by (w-plane, origin tile,
// footprint origin) and whole warps:
//
//   * The plan sorts each (plane, tile) bin's records by footprint origin (row j0, then column
//     i0), so the records of one origin are contiguous. A CTA takes work units (shares of the
//     estimated work) from a global counter, the most expensive end first; per plane inside a
//     unit it stages the plane's table in shared memory, and its warps (warp pairs for S > 16)
//     take the plane's records in guided batches from a shared-memory counter. There is no
//     other CTA-wide step.
//   * A warp streams its batch 64 records at a time: each lane loads two records (coalesced),
//     decodes them into the warp's shared-memory ring (FMA operands, origin, class offset), and
//     loads its records of the next group while the warp walks this one.
//   * The walk: all 32 lanes on the same record, so every branch is warp-uniform. Lane (g, a)
//     holds rows g R .. g R + R - 1 of one footprint column in registers: the warp's registers
//     are the S x S cells under the current origin. Records of the same origin accumulate in
//     place; footprint moves are described at warp_grid.
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
  float2* comp;             // compensated accumulation: the rounding errors of the grid's sums, or nullptr
  int smem_bytes;           // dynamic shared memory of the launch
  int group_tiles;          // origin tiles of one tile row sorted as one segment, at most
  int nunits;               // work units (equal shares of the estimated work)
  int64_t bin_lo, bin_hi;   // the bins this launch grids (a prefix or suffix of the planes)
  uint32_t* work;           // [2]: next unit, finished CTAs (both zero between launches)
};

// The warp's ring in shared memory: 32 decoded records, the FMA operands (cr, be, ci, de) and
// the header (origin i0 | j0 << 16, byte offset of the record's class in the plane's table).
// Two launch shapes: 32 warps (eight per scheduler, at most 64 registers a thread) when every
// plane's support is at most 16, 16 warps (128 registers) when larger supports need them.
// Measured on the float32 workload: 1.65 ms with 24 warps against 1.88 ms with 16, and 32 warps
// 2% faster than 24.
constexpr int kGridThreadsSmall = 1024;
constexpr int kGridThreadsLarge = 512;
constexpr int kRingRecs = 64;                  // a group: two records per lane
// ... followed by the batch slots of a warp pair (S > 16: two [start, size] slots, used by the
// pair's first warp's ring)
constexpr int kPairSlot = kRingRecs * (16 + 8);
constexpr int kRingBytes = kPairSlot + 16;
__host__ __device__ constexpr int rings_bytes(int threads) { return threads / 32 * kRingBytes; }
// Records a warp takes at a time (S <= 16): a guided size, the plane's remaining records over
// twice the CTA's warps, rounded up to 32 and kept within [32, 256], so that batches shrink as the
// plane runs out and the warps reach the next plane's barrier close together (1.70 -> 1.59 ms on
// the float32 workload against fixed batches of 256).
constexpr uint32_t kBatchMin = 32, kBatchMax = 256;

// The S x S cells under one footprint origin, distributed over a warp (see Lay): lane row r
// of this lane's footprint column, as two float32 pairs whose lane sums are the cell's real
// and imaginary parts.
template <int S>
struct Footprint {
  using L = Lay<S>;
  unsigned long long p1[L::R], p2[L::R];     // (cr kr, be ki) and (ci kr, de ki) summed over records
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < L::R; ++r) p1[r] = p2[r] = 0ull;
  }
  // keep == false: zero (a select, so that a non-finite sum does not outlive its cell)
  __device__ __forceinline__ void keep_if(bool keep) {
#pragma unroll
    for (int r = 0; r < L::R; ++r) {
      p1[r] = keep ? p1[r] : 0ull;
      p2[r] = keep ? p2[r] : 0ull;
    }
  }
  // Adds this lane's cells to the grid where `pred`: rows r < nrow of its column, the first at
  // cell index idx (32-bit: n <= 32768), the next ones n cells apart. Predicated, no branch.
  __device__ __forceinline__ void flush(bool pred, float2* __restrict__ grid, float2* __restrict__ comp, uint32_t idx,
                                        uint32_t n, int nrow) const {
    if (!comp) {
#pragma unroll
      for (int r = 0; r < L::R; ++r) {
        red_add2_if(pred && r < nrow, grid + idx, lo_of(p1[r]) + hi_of(p1[r]), lo_of(p2[r]) + hi_of(p2[r]));
        idx += n;
      }
      return;
    }
    // compensated: each addition returns the cell's previous value, and the exact rounding error
    // of old + x (TwoSum) goes to the compensation grid
#pragma unroll
    for (int r = 0; r < L::R; ++r) {
      if (pred && r < nrow) {
        const float x = lo_of(p1[r]) + hi_of(p1[r]), y = lo_of(p2[r]) + hi_of(p2[r]);
        const float2 old = atom_add2(grid + idx, x, y);
        red_add2(comp + idx, two_sum_err(old.x, x), two_sum_err(old.y, y));
      }
      idx += n;
    }
  }
};

// One warp grids the records [beg, end) of one plane (support S, table type T). Table: the
// plane's tap layout in shared memory at tab_off, or (kGlobal: too large to stage) its global
// copy gtab; row half h (S > 16). The records stream through the warp's ring at ring_off.
//
// Per record and tap, with the tap's pair (kr, ki):
//   p1 += (cr, be) * (kr, ki),  p2 += (ci, de) * (kr, ki)    (two fma.rn.f32x2)
// and the cell receives (p1.x + p1.y, p2.x + p2.y): c K with be = -ci, de = cr, or
// c conj(K) (w < 0) with be = ci, de = -cr. Every product and sum is float32.
//
// Footprint moves (the paper's register reuse, Fig. 2, after Romein): lane slot a owns the
// cells whose column is congruent to a modulo S. When the origin moves right by 0 < d < S on
// the same row, a lane whose current tap column ac is >= d keeps its cells (now tap column
// ac - d); the others add their cells to the grid and start on the column S cells further
// right (tap column ac - d + S). So a slide moves no data between lanes; any other move
// flushes every cell and resets ac to the lane's slot.
// Loads this lane's two records of the group at q (records q + lane and q + 32 + lane below e).
__device__ __forceinline__ void load_group(const uint4* __restrict__ grecs, uint32_t q, uint32_t e, int lane,
                                           uint4& r0, uint4& r1) {
  if (q + lane < e) r0 = __ldcs(grecs + q + lane);
  if (q + 32 + lane < e) r1 = __ldcs(grecs + q + 32 + lane);
}

// The record's FMA operands and header in the ring: be = -ci, de = cr (K) or be = ci, de = -cr
// (conj K), and the byte offset of its class in the plane's table.
template <int CB>
__device__ __forceinline__ void decode_record(const uint4& r, int os, ulonglong2* ops, uint2* hdr, int i) {
  const uint32_t flip = (r.w & 0x80000000u) ^ 0x80000000u;      // sign bit set unless conj
  ops[i] = make_ulonglong2((unsigned long long)r.x | ((unsigned long long)(r.y ^ flip) << 32),
                           (unsigned long long)r.y | ((unsigned long long)(r.x ^ flip ^ 0x80000000u) << 32));
  const uint32_t cls = ((r.w >> 8) & 0xffu) * (uint32_t)os + (r.w & 0xffu);
  hdr[i] = make_uint2(r.z, cls * (uint32_t)CB);
}

template <int S, class T, bool kGlobal>
__device__ __forceinline__ void warp_grid(const G2Args& a, int tab_off, const unsigned char* gtab, int h, int ring_off,
                                          uint32_t pe, uint32_t* next) {
  using L = Lay<S, T>;
  const int lane = threadIdx.x & 31;
  const int g = lane / S, slot = lane - g * S;
  const bool active = lane < L::NL;
  const int row0 = L::H > 1 ? h * L::R : g * L::R;
  const unsigned char* tab = (kGlobal ? gtab : dyn_smem() + tab_off) + h * L::HB;
  ulonglong2* ops = (ulonglong2*)(dyn_smem() + ring_off);
  uint2* hdr = (uint2*)(dyn_smem() + ring_off + 16 * kRingRecs);
  const uint4* grecs = (const uint4*)a.recs;
  float2* __restrict__ grid = a.grid;
  float2* __restrict__ comp = a.comp;
  const uint32_t n = (uint32_t)a.g.n;
  const int os = a.g.os;
  // Batches from the CTA's counter, of a guided size: the plane's remaining records over twice
  // the CTA's walkers (warps, or warp pairs for S > 16), rounded up to 32 and kept within
  // [32, 256]. For S > 16 the two warps of a pair (row halves) walk the same batches: the first
  // takes each from the counter into one of two slots, alternately, and both read it after the
  // pair's named barrier (one barrier per batch: a slot is rewritten only after the other warp
  // has passed the next barrier, so after it has read the slot). Both warps take the same
  // batches in the same order, so they reach every barrier together.
  uint32_t grabs = 0;
  auto grab = [&](uint32_t& b, uint32_t& e) {
    uint32_t v = 0, want = 0;
    if (lane == 0 && h == 0) {
      const uint32_t walkers = (blockDim.x / 32u) / L::H;  // warps, or warp pairs
      const uint32_t cur = *(volatile uint32_t*)next;     // a lower bound of the next record
      const uint32_t rem = cur < pe ? pe - cur : 0u;
      want = min(kBatchMax, max(kBatchMin, (rem / (2u * walkers) + 31u) & ~31u));
      v = atomicAdd(next, want);
    }
    if constexpr (L::H > 1) {
      const int pair = (int)(threadIdx.x >> 5) / L::H;
      uint32_t* slot = (uint32_t*)(dyn_smem() + pair * L::H * kRingBytes + kPairSlot) + 2 * (grabs & 1u);
      if (lane == 0 && h == 0) {
        slot[0] = v;
        slot[1] = want;
      }
      asm volatile("bar.sync %0, %1;" ::"r"(1 + pair), "r"(32 * L::H) : "memory");
      v = slot[0];
      want = slot[1];
      ++grabs;
    } else {
      v = __shfl_sync(0xffffffffu, v, 0);
      want = __shfl_sync(0xffffffffu, want, 0);
    }
    b = v;
    e = b < pe ? min(b + want, pe) : b;
  };
  uint32_t cb, ce, nb, ne;
  grab(cb, ce);
  if (cb >= ce) return;
  grab(nb, ne);
  Footprint<S> fp;
  fp.zero();
  uint32_t cz = kNoOrigin;
  int ci0 = 0, cj0 = -1;                                   // no row: the first origin never slides
  const int nrow = active ? min(L::R, S - row0) : 0;       // this lane's rows inside the footprint
  int ac = active ? slot : 0;                              // current tap column
  const unsigned char* lt = tab + lane * L::SB;            // this lane's slot in each block
  uint32_t cidx = 0;                                       // cell index of this lane's first cell
  uint4 r0 = make_uint4(0u, 0u, 0u, 0u), r1 = r0;
  uint32_t q = cb;
  load_group(grecs, q, ce, lane, r0, r1);
  for (;;) {
    const int m = (int)min((uint32_t)kRingRecs, ce - q);
    __syncwarp();
    if (lane < m) decode_record<L::CB>(r0, os, ops, hdr, lane);
    if (lane + 32 < m) decode_record<L::CB>(r1, os, ops, hdr, lane + 32);
    __syncwarp();
    // the next group (of this batch or of the next one) loads while the warp walks this one
    const bool last = q + kRingRecs >= ce;
    if (!last) load_group(grecs, q + kRingRecs, ce, lane, r0, r1);
    else if (nb < ne) load_group(grecs, nb, ne, lane, r0, r1);
#pragma unroll 2
    for (int j = 0; j < m; ++j) {
      const uint2 hd = hdr[j];
      const ulonglong2 op = ops[j];
      if (hd.x != cz) {                                    // warp-uniform: a new footprint origin
        const int i0 = hd.x & 0xffff, j0 = hd.x >> 16;
        const int d = i0 - ci0;
        const bool slide = j0 == cj0 && (unsigned)(d - 1) < (unsigned)(S - 1);   // 0 < d < S on the same row
        const bool keep = slide && ac >= d;
        fp.flush(cz != kNoOrigin && !keep, grid, comp, cidx, n, nrow);
        if (slide) {
          fp.keep_if(keep);
          ac = keep ? ac - d : ac - d + S;
          cidx = keep ? cidx : cidx + S;
        } else {
          fp.zero();
          ac = active ? slot : 0;
          cidx = (uint32_t)(j0 + row0) * n + (uint32_t)(i0 + ac);
        }
        lt = tab + (active ? g * S + ac : lane) * L::SB;
        cz = hd.x;
        ci0 = i0;
        cj0 = j0;
      }
      const unsigned char* p = lt + hd.y;
#pragma unroll
      for (int r = 0; r < L::R; ++r) {
        const unsigned long long t = tap_pair<T, kGlobal>(p + r * L::BB);
        fp.p1[r] = fma2(op.x, t, fp.p1[r]);
        fp.p2[r] = fma2(op.y, t, fp.p2[r]);
      }
    }
    if (!last) {
      q += kRingRecs;
      continue;
    }
    if (nb >= ne) break;
    if (nb != ce) {                                        // not the continuation of this batch
      fp.flush(cz != kNoOrigin, grid, comp, cidx, n, nrow);
      fp.zero();
      cz = kNoOrigin;
      cj0 = -1;
    }
    cb = nb;
    ce = ne;
    q = cb;
    grab(nb, ne);
  }
  fp.flush(cz != kNoOrigin, grid, comp, cidx, n, nrow);
}

// The records [pb, pe) of plane p (support S) with the whole CTA: stage the plane's table
// unless it is staged already (or too large: then its global copy is read), and walk the
// records: each warp (for S > 16 each pair of warps, one per row half) takes guided batches
// from a counter, so that dense and sparse regions even out.
template <int S, class T, int NT>
__device__ __noinline__ void grid_plane(const G2Args& a, int p, bool stage, bool staged, uint32_t pb, uint32_t pe) {
  using L = Lay<S, T>;
  __shared__ uint32_t next;
  const int tab_off = rings_bytes(NT);
  __syncthreads();                                 // every warp is done with the previous plane
  if (threadIdx.x == 0) next = pb;
  if (stage) stage_table<S, T>((const T*)a.tab + a.tab_off[p], a.g.os, tab_off);
  __syncthreads();
  const unsigned char* gtab = staged ? nullptr : a.lanetab + a.lanetab_off[p];
  const int warp = threadIdx.x >> 5;
  const int ring_off = warp * kRingBytes;
  const int h = warp % L::H;
  if (staged) warp_grid<S, T, false>(a, tab_off, nullptr, h, ring_off, pe, &next);
  else warp_grid<S, T, true>(a, tab_off, gtab, h, ring_off, pe, &next);
}

// cur_plane: the plane whose table is staged (-1: none), the same in every thread of the CTA.
template <class T, int NT>
__device__ void grid_range(const G2Args& a, uint32_t beg, uint32_t end, int& cur_plane) {
  constexpr int kMaxSupp = NT == kGridThreadsSmall ? kSmallMaxS : kMaxS;
  int64_t bin = find_bin(a.offsets, a.nbins, beg);
  uint32_t pos = beg;
  const int tab_off = rings_bytes(NT);
  while (pos < end) {
    bin = advance_bin(a.offsets, bin, a.nbins, pos);
    const int p = (int)a.g.div_ntiles.div((uint32_t)bin);   // bins < 2^24
    const uint32_t pe = min(end, a.offsets[(int64_t)(p + 1) * a.g.ntiles]);
    const int s = a.g.supp[p];
    const int tbytes = a.g.os * a.g.os * lay_class_bytes(s, TabElem<T>::E);
    const bool staged = s <= kMaxStagedS || tab_off + tbytes <= a.smem_bytes;
    const bool stage = staged && p != cur_plane;
    if (staged) cur_plane = p;
    switch (s) {
#define WP_SEG_CASE(N)                                                           \
  case N:                                                                        \
    if constexpr (N <= kMaxSupp) grid_plane<N, T, NT>(a, p, stage, staged, pos, pe); \
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
    pos = pe;
  }
}

template <class T, int NT>
__global__ void __launch_bounds__(NT, 1) k_grid_v2(G2Args a) {
  int cur_plane = -1;
  for_each_unit<true>(a.offsets, a.costoff, a.nbins, a.bin_lo, a.bin_hi, a.nunits, a.work,
                      [&](uint32_t beg, uint32_t end) { grid_range<T, NT>(a, beg, end, cur_plane); });
}

// ---- tap-layout tables in global memory for the planes with S > 16 ----

// Writes a plane's table (stored layout [oy*os+ox][a][b] of T) in the tap layout for a runtime
// support s (17 .. 32); grid-stride over the table's entries.
template <class T>
__global__ void k_lane_table(const T* __restrict__ src, int s, int os, unsigned char* __restrict__ dst) {
  const int n = tap_entries(os, s);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) write_tap_entry<T>(src, s, dst, i);
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
__global__ void __launch_bounds__(kGridThreadsLarge, 1) k_grid_batch(BatchArgs b) {
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
      int cur_plane = -1;                          // another job's tables
      if (beg < end) grid_range<T, kGridThreadsLarge>(a, beg, end, cur_plane);
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
// is outside the kernel's limits (then the baseline kernel of grid.cu runs): supports up to 32,
// and the warps' rings plus the largest table of S <= 16 within the device's shared memory
// (larger supports read a global copy of their table when it does not fit).
size_t grid_v2_smem(const wp_ctx* ctx, int* group_tiles) {
  const int smax = *std::max_element(ctx->supp.begin(), ctx->supp.end());
  if (smax > kMaxS) return 0;
  const int e = ctx->prm.table_type == WP_TABLE_F32 ? 4 : 2;
  const int os = ctx->prm.oversample;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->prm.device) != cudaSuccess)
    return 0;
  const size_t bytes = (size_t)optin - 1024;        // room for the static scratch
  size_t tab = 0;
  for (int sp : ctx->supp) tab = std::max(tab, (size_t)lay_staged_bytes(os, sp, e));
  if (smax > kMaxStagedS && !ctx->d_lanetab) return 0;
  if ((size_t)rings_bytes(kGridThreadsSmall) + tab > bytes) return 0;
  *group_tiles = 1;
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
  a.comp = ctx->comp_active;
  a.smem_bytes = (int)smem;
  a.group_tiles = group;
  a.nunits = ctx->nsm * ctx->prm.units_per_cta;
  a.work = ctx->d_work;
  cudaError_t e;
  if ((e = launch_bin_costs(ctx, s))) return e;
  // Supports grow with the plane, so the planes of support <= 16 are a prefix of the bins: they
  // run in the 32-warp shape, the planes of larger support in a second, 16-warp launch.
  const int64_t split = small_planes_end(ctx) * ctx->geo.ntiles;
  auto run = [&](auto kern, int threads, int64_t lo, int64_t hi) -> cudaError_t {
    if (lo >= hi) return cudaSuccess;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err) return err;
    a.bin_lo = lo;
    a.bin_hi = hi;
    ++ctx->launches;
    kern<<<ctx->nsm, threads, smem, s>>>(a);
    return cudaGetLastError();
  };
  auto both = [&](auto small_kern, auto large_kern) -> cudaError_t {
    cudaError_t err = run(small_kern, kGridThreadsSmall, 0, split);
    if (err) return err;
    return run(large_kern, kGridThreadsLarge, split, ctx->nbins);
  };
  switch (ctx->prm.table_type) {
    case WP_TABLE_F16: return both(k_grid_v2<__half2, kGridThreadsSmall>, k_grid_v2<__half2, kGridThreadsLarge>);
    case WP_TABLE_BF16: return both(k_grid_v2<BfWord, kGridThreadsSmall>, k_grid_v2<BfWord, kGridThreadsLarge>);
    default: return both(k_grid_v2<float2, kGridThreadsSmall>, k_grid_v2<float2, kGridThreadsLarge>);
  }
}

}  // namespace wp

namespace wp {

size_t grid_job_desc_bytes() { return sizeof(G2Args); }

namespace {
// grid += comp, elementwise (the compensated accumulation's last step).
__global__ void k_add_comp(float2* __restrict__ grid, const float2* __restrict__ comp, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 c = comp[i];
    float2 g = grid[i];
    g.x += c.x;
    g.y += c.y;
    grid[i] = g;
  }
}
}  // namespace

cudaError_t launch_add_comp(float2* grid, const float2* comp, int64_t n, int nsm, cudaStream_t s) {
  k_add_comp<<<nsm * 8, 256, 0, s>>>(grid, comp, n);
  return cudaGetLastError();
}

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
  a.comp = nullptr;
  a.smem_bytes = (int)smem;
  a.group_tiles = group;
  a.nunits = 0;
  a.bin_lo = 0;
  a.bin_hi = ctx->nbins;
  a.work = nullptr;
  memcpy(out, &a, sizeof(a));
}

cudaError_t prepare_grid_batch(int table_type, size_t smem) {
  switch (table_type) {
    case WP_TABLE_F16: return cudaFuncSetAttribute(k_grid_batch<__half2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    case WP_TABLE_BF16: return cudaFuncSetAttribute(k_grid_batch<BfWord>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
    case WP_TABLE_F16: k_grid_batch<__half2><<<nsm, kGridThreadsLarge, smem, s>>>(b); break;
    case WP_TABLE_BF16: k_grid_batch<BfWord><<<nsm, kGridThreadsLarge, smem, s>>>(b); break;
    default: k_grid_batch<float2><<<nsm, kGridThreadsLarge, smem, s>>>(b); break;
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
    const int blocks = std::min(1024, (tap_entries(os, sp) + 255) / 256);
    switch (ctx->prm.table_type) {
      case WP_TABLE_F16:
        k_lane_table<__half2><<<blocks, 256, 0, s>>>((const __half2*)ctx->d_tab + ctx->tab_off[p], sp, os, dst);
        break;
      case WP_TABLE_BF16:
        k_lane_table<BfWord><<<blocks, 256, 0, s>>>((const BfWord*)ctx->d_tab + ctx->tab_off[p], sp,
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
