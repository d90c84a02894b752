// Coordinates (float64 definition) and binning of visibilities by (w-plane, footprint-origin
// tile).
//
// Coordinates follow the W-projection gridding step (Sec. 2.1/2.2 of Lao et al. 2019: each
// visibility lands on the uv grid through a C_full x C_full kernel); they are defined by float64
// products and round-half-to-even, in the order written in wproj.h, so that the integer
// decisions (oversampled position, plane, footprint) are the same on every platform that
// evaluates the same IEEE float64 operations. The kernels reach that definition through a
// float32 evaluation with a proven error bound and form the float64 products only where the
// bound leaves the rounding undecided.
//
// Binning is a counting sort: a histogram of bin keys, an exclusive prefix sum giving each
// bin's start index (the construction of Eq. 6, there applied to baselines), and a scatter
// that writes each visibility's 16-byte record into its bin; a last pass sorts each bin's
// records by footprint origin.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "internal.h"

namespace wp {

namespace {

struct Coord {
  int32_t u, v, plane, i0, j0, ox, oy;
  bool conj, keep;
};

// Round-half-to-even of a float64 with |x| < 2^30 (the caller checks), as an integer, from
// its bit pattern with integer operations only: x = m 2^(e - 1075) with the 53-bit
// significand m, so the integer part is m >> (1075 - e) and the dropped bits decide the
// rounding (above half: up; exactly half: up when the integer part is odd).
__device__ __forceinline__ int32_t rint_small(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  const int sh = 1075 - e;                             // >= 23 for |x| < 2^30
  if (sh > 53) return 0;                               // |x| < 1/2
  const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;
  const unsigned long long q = m >> sh;
  const unsigned long long rem = m & ((1ull << sh) - 1ull);
  const unsigned long long half = 1ull << (sh - 1);
  const int32_t n = (int32_t)q + ((rem > half || (rem == half && (q & 1ull))) ? 1 : 0);
  return (b >> 63) ? -n : n;
}

// |x| as float64 bits (sign cleared); finite values compare below 0x7ff0000000000000.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
constexpr unsigned long long kBitsCoordLimit = 0x41D0000000000000ull;   // 2^30
constexpr unsigned long long kBitsInf = 0x7ff0000000000000ull;

// The rounded coordinates of one visibility, shared by it and its Hermitian partner:
// U = rint(u kx), V = rint(v kx), plane = min(Nw - 1, rint(min(|w| kw, 2^30))), valid when
// all three products are finite and |u kx|, |v kx| < 2^30.
struct Rounded {
  int32_t u, v, plane;
  bool fin, wpos, wneg;
};

__device__ __forceinline__ Rounded round_coords(double ux, double vy, double wz, double w_m, const Geometry& g) {
  Rounded r;
  const unsigned long long bx = abs_bits(ux), by = abs_bits(vy), bz = abs_bits(wz);
  r.fin = bx < kBitsCoordLimit && by < kBitsCoordLimit && bz < kBitsInf;
  r.u = r.fin ? rint_small(ux) : 0;
  r.v = r.fin ? rint_small(vy) : 0;
  r.plane = !r.fin ? 0 : (bz >= kBitsCoordLimit ? g.n_w - 1 : min(g.n_w - 1, rint_small(wz)));
  const unsigned long long bw = (unsigned long long)__double_as_longlong(w_m);
  r.wpos = (bw >> 63) == 0 && (bw << 1) != 0;        // w > 0
  r.wneg = (bw >> 63) != 0 && (bw << 1) != 0;        // w < 0
  return r;
}

// Coordinates of one gridded visibility from its rounded coordinates; `neg` selects the
// Hermitian partner at -uvw.
__device__ __forceinline__ Coord make_coord(const Rounded& r, bool neg, const Geometry& g) {
  Coord c;
  const int32_t u = neg ? -r.u : r.u;
  const int32_t v = neg ? -r.v : r.v;
  const int32_t p = r.plane;
  c.u = u;
  c.v = v;
  c.plane = p;
  c.conj = neg ? r.wpos : r.wneg;
  const int32_t s = g.supp[p];
  const int32_t half = s * g.os / 2;
  const int32_t x = u + (g.n / 2) * g.os;
  const int32_t y = v + (g.n / 2) * g.os;
  // floor((x - half) / os) + 1 = floor((x - half + os) / os) when x - half + os >= 0; below
  // that the footprint starts left of cell 0 and the visibility is dropped (i0 = -1)
  const int32_t ax = x - half + g.os, ay = y - half + g.os;
  c.i0 = ax >= 0 ? (int32_t)g.div_os.div((uint32_t)ax) : -1;
  c.j0 = ay >= 0 ? (int32_t)g.div_os.div((uint32_t)ay) : -1;
  c.ox = c.i0 * g.os - x + half - 1;
  c.oy = c.j0 * g.os - y + half - 1;
  c.keep = r.fin && c.i0 >= 0 && c.i0 + s <= g.n && c.j0 >= 0 && c.j0 + s <= g.n;
  return c;
}

// The (plane, origin tile) bin of a kept visibility (i0, j0 >= 0).
__device__ __forceinline__ uint32_t bin_of(const Coord& c, const Geometry& g) {
  return (uint32_t)((int64_t)c.plane * g.ntiles + (int64_t)g.div_ty.div((uint32_t)c.j0) * g.ntx +
                    g.div_tx.div((uint32_t)c.i0));
}

// ---- the rounded coordinates of one visibility, float32 first ----
//
// B300 issues float64 arithmetic at a small fraction of its float32 rate (a few operations per
// SM and clock), and three float64 products per visibility made the histogram pass bound by
// that pipe. The products are therefore first formed in float32 from truncated operands, whose
// distance to the float64 product is bounded; where that bound cannot carry the product across
// a rounding boundary (a half-integer), the rint of the float32 value is the rint of the
// float64 product. Only the remaining visibilities (within about 1e-6 |x| of a boundary, and
// any operand out of range, infinite or NaN) form the float64 products. Either way the result
// is the float64 definition above, bit for bit.

// float32 of a float64 with its significand truncated, from the bit pattern (no float64
// instruction): |f - x| < 2^-23 |x| for 2^-126 <= |x| < 2^128, and +-0 for |x| < 2^-126. The
// callers take it only for biased exponents <= 1086 (|x| < 2^64).
__device__ __forceinline__ float trunc_float(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t e = (hi >> 20) & 0x7ffu;
  const uint32_t sign = hi & 0x80000000u;
  return __uint_as_float(e < 897u ? sign : sign | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
__device__ __forceinline__ uint32_t exp_of(double x) {
  return (uint32_t)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu;
}

// n = rint(p) for the float64 product p of two operands whose truncated float32 product is X,
// when that is decided: |X - p| < 3e-7 |X| + 2^-62 (two truncations below 2^-23 each, the
// float32 product's rounding 2^-24 and the float64 product's 2^-53, relative; an operand
// flushed to zero contributes below 2^-62), so p lies within `margin` of X, and when the
// half-integers nearest X are farther than that, p rounds to the same integer as X.
__device__ __forceinline__ bool rint_decided(float X, int32_t& n) {
  const float ax = fabsf(X);
  const float r = rintf(X);
  const float margin = fmaf(ax, 0x1p-20f, 0x1p-40f);
  n = (int32_t)r;
  return ax < 0x1p28f && 0.5f - fabsf(X - r) > margin;
}

// The rounded coordinates of visibility k (row k / nchan, channel k % nchan).
__device__ __forceinline__ Rounded rounded_coords(const double* __restrict__ uvw, const double* __restrict__ chan,
                                                  int64_t k, const FastDiv& nchan, const Geometry& g) {
  const uint32_t row = nchan.div((uint32_t)k);         // nvis < 2^32 (32-bit record offsets)
  const int32_t ch = (int32_t)((uint32_t)k - row * nchan.d);
  const double u = uvw[3 * (size_t)row], v = uvw[3 * (size_t)row + 1], w = uvw[3 * (size_t)row + 2];
  const double kx = chan[2 * ch], kw = chan[2 * ch + 1];
  const double aw = __longlong_as_double(__double_as_longlong(w) & 0x7fffffffffffffffll);
  const uint32_t ekx = exp_of(kx), ekw = exp_of(kw);
  bool done = exp_of(u) <= 1086u && exp_of(v) <= 1086u && exp_of(aw) <= 1086u && ekx >= 897u && ekx <= 1086u &&
              ekw >= 897u && ekw <= 1086u;
  Rounded r;
  if (done) {
    const float fkx = trunc_float(kx);
    int32_t nu, nv, np;
    done = rint_decided(trunc_float(u) * fkx, nu) && rint_decided(trunc_float(v) * fkx, nv) &&
           rint_decided(trunc_float(aw) * trunc_float(kw), np);
    r.u = nu;
    r.v = nv;
    r.plane = min(g.n_w - 1, np);
    r.fin = true;
    const unsigned long long bw = (unsigned long long)__double_as_longlong(w);
    r.wpos = (bw >> 63) == 0 && (bw << 1) != 0;
    r.wneg = (bw >> 63) != 0 && (bw << 1) != 0;
  }
  if (!done) r = round_coords(__dmul_rn(u, kx), __dmul_rn(v, kx), __dmul_rn(aw, kw), w, g);
  return r;
}

// Adds x to the float32 pair (hi, lo) whose sum carries a running total: TwoSum (Knuth) puts
// the exact rounding error of hi + x into lo, so the pair stays within a few 2^-48 of the exact
// sum over a thread's handful of terms.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
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

// Passes 1 and 3 give each CTA kPlanVis consecutive visibilities and count its records per bin
// in a shared-memory hash table first, so that a bin costs one global atomic per CTA rather
// than one per record (the records of a dense bin otherwise serialise on its counter).
// 2048 visibilities per CTA measured 2% faster than 1024 and 4096 on the float32 workload (more
// records of a bin per CTA, so fewer cursor reservations, against fewer CTAs per SM).
constexpr int kPlanThreads = 512;
constexpr int kPlanPer = 4;                              // visibilities per thread
constexpr int kPlanVis = kPlanThreads * kPlanPer;        // per CTA
constexpr int kHashBits = 13;
constexpr int kHashSlots = 1 << kHashBits;               // >= twice the records of a CTA (with partners)
constexpr int kHashBytes = 2 * kHashSlots * 4;           // keys and counts, dynamic shared memory
constexpr uint32_t kHashEmpty = 0xffffffffu;

// The slot of `key` in the table (inserted if absent), or -1 if the table is full (it cannot
// be: a CTA has at most 2 kPlanVis keys; the bound keeps the loop finite regardless).
__device__ __forceinline__ int hash_slot(uint32_t* keys, uint32_t key) {
  uint32_t s = (key * 2654435761u) >> (32 - kHashBits);
  for (int i = 0; i < kHashSlots; ++i) {
    const uint32_t prev = atomicCAS(&keys[s], kHashEmpty, key);
    if (prev == kHashEmpty || prev == key) return (int)s;
    s = (s + 1) & (kHashSlots - 1);
  }
  return -1;
}

__device__ __forceinline__ void hash_clear(uint32_t* keys, uint32_t* cnt) {
  for (int i = threadIdx.x; i < kHashSlots; i += kPlanThreads) {
    keys[i] = kHashEmpty;
    cnt[i] = 0u;
  }
}

// Pass 1: bin histogram, dropped count and kept-weight sum.
__global__ void __launch_bounds__(kPlanThreads) k_histogram(const double* __restrict__ uvw,
                                                            const double* __restrict__ chan,
                                                            const float* __restrict__ weight, int64_t nvis,
                                                            FastDiv nchan, int32_t pairs, Geometry g,
                                                            uint32_t* __restrict__ counts,
                                                            unsigned long long* __restrict__ dropped,
                                                            double* __restrict__ wsum) {
  extern __shared__ uint32_t hash_smem[];
  uint32_t* keys = hash_smem;
  uint32_t* cnt = hash_smem + kHashSlots;
  hash_clear(keys, cnt);
  __syncthreads();
  float w_hi = 0.f, w_lo = 0.f;                             // kept-weight sum as a float32 pair
  uint32_t my_drop = 0;
  const int64_t base = (int64_t)blockIdx.x * kPlanVis;
#pragma unroll
  for (int u = 0; u < kPlanPer; ++u) {
    const int64_t k = base + u * kPlanThreads + threadIdx.x;
    if (k >= nvis) break;
    const Rounded rd = rounded_coords(uvw, chan, k, nchan, g);
    int nkept = 0;
    for (int h = 0; h <= pairs; ++h) {
      const Coord c = make_coord(rd, h == 1, g);
      if (c.keep) {
        const uint32_t b = bin_of(c, g);
        const int sl = hash_slot(keys, b);
        if (sl >= 0) atomicAdd(&cnt[sl], 1u);
        else atomicAdd(&counts[b], 1u);
      }
      nkept += c.keep ? 1 : 0;
    }
    my_drop += (uint32_t)(pairs + 1 - nkept);
    // weight x 1 or x 2 is exact in float32
    if (nkept) pair_add(w_hi, w_lo, (weight ? weight[k] : 1.0f) * (float)nkept);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kHashSlots; i += kPlanThreads)
    if (keys[i] != kHashEmpty) atomicAdd(&counts[keys[i]], cnt[i]);
  // block reduction of the two scalars: float32 pairs within a warp, float64 across warps
  __shared__ double sw[kPlanThreads / 32];
  __shared__ unsigned long long sd[kPlanThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, w_hi, off), ol = __shfl_xor_sync(0xffffffffu, w_lo, off);
    pair_add(w_hi, w_lo, oh);
    w_lo += ol;
    my_drop += __shfl_xor_sync(0xffffffffu, my_drop, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sw[warp] = (double)w_hi + (double)w_lo;
    sd[warp] = my_drop;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tw = 0.0;
    unsigned long long td = 0;
    for (int i = 0; i < kPlanThreads / 32; ++i) {
      tw += sw[i];
      td += sd[i];
    }
    if (tw != 0.0) atomicAdd(wsum, tw);
    if (td) atomicAdd(dropped, td);
  }
}

// Pass 3: scatter records into their bins (coordinates recomputed as in pass 1): each
// record's rank among the CTA's records of its bin comes from the hash table's counter, then one
// global atomic per bin reserves the CTA's run of slots, and the records go to run start + rank.
__global__ void __launch_bounds__(kPlanThreads) k_scatter(const double* __restrict__ uvw, const double* __restrict__ chan,
                                                          const float2* __restrict__ vis, const float* __restrict__ weight,
                                                          int64_t nvis, FastDiv nchan, int32_t pairs, int32_t for_degrid,
                                                          Geometry g, uint32_t* __restrict__ cursor,
                                                          Record* __restrict__ records, uint32_t* __restrict__ index) {
  extern __shared__ uint32_t hash_smem[];
  uint32_t* keys = hash_smem;
  uint32_t* cnt = hash_smem + kHashSlots;
  hash_clear(keys, cnt);
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kPlanVis;
  Rounded rd[kPlanPer];
  uint32_t code[kPlanPer][2];                             // slot << 16 | rank, or 0xffffffff
  float2 v[kPlanPer];                                     // loaded here, used after the barriers
  float wt[kPlanPer];
#pragma unroll
  for (int u = 0; u < kPlanPer; ++u) {
    const int64_t k = base + u * kPlanThreads + threadIdx.x;
    code[u][0] = code[u][1] = 0xffffffffu;
    if (k >= nvis) continue;
    if (!for_degrid) {
      v[u] = __ldcs(vis + k);
      wt[u] = weight ? __ldcs(weight + k) : 1.0f;
    }
    rd[u] = rounded_coords(uvw, chan, k, nchan, g);
    for (int h = 0; h <= pairs; ++h) {
      const Coord c = make_coord(rd[u], h == 1, g);
      if (c.keep) {
        const uint32_t b = bin_of(c, g);
        const int sl = hash_slot(keys, b);
        // a full table (impossible by its size) would fall back to a per-record global cursor
        code[u][h] = sl >= 0 ? ((uint32_t)sl << 16) | atomicAdd(&cnt[sl], 1u) : 0xfffffffeu;
      }
    }
  }
  __syncthreads();
  {
    // every reservation of this thread in flight before the first result is used
    constexpr int kSlotsPer = kHashSlots / kPlanThreads;
    uint32_t start[kSlotsPer];
#pragma unroll
    for (int j = 0; j < kSlotsPer; ++j) {
      const int i = threadIdx.x + j * kPlanThreads;
      const uint32_t key = keys[i];
      start[j] = key != kHashEmpty ? atomicAdd(&cursor[key], cnt[i]) : 0u;
    }
#pragma unroll
    for (int j = 0; j < kSlotsPer; ++j) cnt[threadIdx.x + j * kPlanThreads] = start[j];
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kPlanPer; ++u) {
    const int64_t k = base + u * kPlanThreads + threadIdx.x;
    if (k >= nvis) continue;
    float2 val = make_float2(0.f, 0.f);
    if (!for_degrid) val = make_float2(wt[u] * v[u].x, wt[u] * v[u].y);
    for (int h = 0; h <= pairs; ++h) {
      if (code[u][h] == 0xffffffffu) continue;
      const Coord c = make_coord(rd[u], h == 1, g);
      const uint32_t slot = code[u][h] == 0xfffffffeu ? atomicAdd(&cursor[bin_of(c, g)], 1u)
                                                      : cnt[code[u][h] >> 16] + (code[u][h] & 0xffffu);
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
      if (index) index[slot] = (uint32_t)k | (h ? 0x80000000u : 0u);
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

// Work estimate of bin b in units of 2^(6 + shift) tap-updates: a fixed part for every non-empty
// bin (segment set-up, table and grid-region staging, local sort, barriers) plus, per record,
// its S_p^2 taps and a record cost. The two constants are measured: on the float32 workload
// 65536 and 64 beat 2048 and 32 by 0.08 ms in gridding and 0.2 ms in degridding (the CTAs
// finish closer together). `shift` keeps the 32-bit prefix sum of the costs from overflowing.
constexpr uint32_t kBinFixedTaps = 65536;
constexpr uint32_t kRecordTaps = 64;

__global__ void k_bin_costs(const uint32_t* __restrict__ offsets, int64_t nbins, Geometry g, int shift,
                            uint32_t* __restrict__ cost) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const uint32_t cnt = offsets[b + 1] - offsets[b];
  const int s = g.supp[b / g.ntiles];
  const uint64_t taps = cnt ? (uint64_t)kBinFixedTaps + (uint64_t)cnt * (uint64_t)(s * s + kRecordTaps) : 0;
  const int sh = 6 + shift;
  cost[b] = (uint32_t)((taps + (1ull << sh) - 1) >> sh);
}

__global__ void k_coords_out(const double* __restrict__ uvw, const double* __restrict__ chan, int64_t nvis,
                             FastDiv nchan, int32_t pairs, Geometry g, int32_t* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nvis; k += (int64_t)gridDim.x * blockDim.x) {
    const Rounded rd = rounded_coords(uvw, chan, k, nchan, g);
    for (int h = 0; h <= pairs; ++h) {
      const Coord c = make_coord(rd, h == 1, g);
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

// offsets[b] = suboff[b << nsub_log2] for b <= nbins (the first sub-counter of each bin).
__global__ void k_gather_offsets(const uint32_t* __restrict__ suboff, int64_t nbins, int32_t nsub_log2,
                                 uint32_t* __restrict__ offsets) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b <= nbins) offsets[b] = suboff[b << nsub_log2];
}

// ---- pass 4: the records of every bin sorted by footprint origin ----

// The non-empty bins as a work list: bins of at least kBigBin records from the front
// (list[0 .. count[0])), the others from the back (list[nbins - count[1] .. nbins)), so that the
// largest bins are taken first. count[0..1] start at zero.
constexpr uint32_t kBigBin = 8192;

__global__ void k_list_bins(const uint32_t* __restrict__ offsets, int64_t nbins, uint32_t* __restrict__ list,
                            uint32_t* __restrict__ count) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const uint32_t n = offsets[b + 1] - offsets[b];
  if (n >= kBigBin) list[atomicAdd(&count[0], 1u)] = (uint32_t)b;
  else if (n > 0) list[nbins - 1 - atomicAdd(&count[1], 1u)] = (uint32_t)b;
}

// Work item i of the bin list (i < count[0] + count[1]).
__device__ __forceinline__ uint32_t listed_bin(const uint32_t* __restrict__ list, const uint32_t* count, int64_t nbins,
                                               uint32_t i) {
  return i < count[0] ? list[i] : list[nbins - 1 - (i - count[0])];
}

constexpr int kBinSortThreads = 512;
constexpr int kBinSortPer = 8;                                   // records per thread in one chunk
constexpr int kBinSortChunk = kBinSortThreads * kBinSortPer;     // 4096
constexpr int kBinSortHistPer = 16;                              // keys per thread in flight (pass 1)

// Exclusive scan of a[0 .. n) in place by the whole CTA (n <= 8 kBinSortThreads).
__device__ __forceinline__ void cta_exclusive_scan(uint32_t* a, int n, uint32_t* warp_sums) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (n + kBinSortThreads - 1) / kBinSortThreads;
  const int beg = tid * per;
  uint32_t local = 0;
  for (int i = 0; i < per; ++i)
    if (beg + i < n) local += a[beg + i];
  uint32_t x = local;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    constexpr int kSortWarps = kBinSortThreads / 32;
    uint32_t v = lane < kSortWarps ? warp_sums[lane] : 0u;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, off);
      if (lane >= off) v += y;
    }
    if (lane < kSortWarps) warp_sums[lane] = v;
  }
  __syncthreads();
  uint32_t run = (warp ? warp_sums[warp - 1] : 0u) + x - local;
  for (int i = 0; i < per; ++i) {
    if (beg + i < n) {
      const uint32_t v = a[beg + i];
      a[beg + i] = run;
      run += v;
    }
  }
  __syncthreads();
}

// One CTA per non-empty bin (taken from a counter): the bin's records (and visibility indices,
// when given) from `in` to the same range of `out`, sorted by the origin key
// (j0 - y0) tile_x + (i0 - x0) of its tile (row-major). A chunk of up to kBinSortChunk records
// is loaded into registers (all loads in flight together), counted per key in shared memory,
// placed in key order in a shared-memory stage, and written out from the stage, so that the
// global stores run along each key's records. A bin of one chunk is sorted by that alone; a
// larger bin first counts its keys (pass 1) so that each chunk's run of a key lands after the
// earlier chunks' runs of it. Shared memory: start[keys + 1], loc[keys + 1], the stage
// (kBinSortChunk records and indices). work[0] is the bin counter, work[1] the finished CTAs;
// the last CTA resets both.
__global__ void __launch_bounds__(kBinSortThreads) k_bin_sort(const uint4* __restrict__ in,
                                                              const uint32_t* __restrict__ in_idx,
                                                              uint4* __restrict__ out, uint32_t* __restrict__ out_idx,
                                                              const uint32_t* __restrict__ offsets, int64_t nbins,
                                                              const uint32_t* __restrict__ list,
                                                              const uint32_t* __restrict__ nlist, Geometry g,
                                                              uint32_t* __restrict__ work) {
  extern __shared__ __align__(16) uint32_t sort_smem[];
  __shared__ uint32_t item;
  __shared__ uint32_t warp_sums[kBinSortThreads / 32];
  const int keys = g.tile_x * g.tile_y;
  const int kpad = (keys + 1 + 3) & ~3;
  uint32_t* start = sort_smem;                          // [keys + 1]
  uint32_t* loc = sort_smem + kpad;                     // [keys + 1]
  uint4* stage = (uint4*)(sort_smem + 2 * kpad);        // [kBinSortChunk]
  uint32_t* stage_idx = (uint32_t*)(stage + kBinSortChunk);
  const uint32_t total = nlist[0] + nlist[1];
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) item = atomicAdd(&work[0], 1u);
    __syncthreads();
    const uint32_t it = item;
    __syncthreads();
    if (it >= total) break;
    const uint32_t b = listed_bin(list, nlist, nbins, it);
    const uint32_t s0 = offsets[b], s1 = offsets[b + 1], nrec = s1 - s0;
    const int64_t tile = (int64_t)b % g.ntiles;
    const int y0 = (int)(tile / g.ntx) * g.tile_y, x0 = (int)(tile % g.ntx) * g.tile_x;
    auto key_of = [&](uint32_t z) { return ((int)(z >> 16) - y0) * g.tile_x + ((int)(z & 0xffff) - x0); };
    const bool multi = nrec > (uint32_t)kBinSortChunk;
    if (multi) {                                        // pass 1: key counts of the whole bin
      for (int k = tid; k <= keys; k += kBinSortThreads) start[k] = 0u;
      __syncthreads();
      for (uint32_t r0 = s0 + tid; r0 < s1; r0 += kBinSortHistPer * kBinSortThreads) {
        uint32_t z[kBinSortHistPer];
#pragma unroll
        for (int u = 0; u < kBinSortHistPer; ++u) {
          const uint32_t r = r0 + u * kBinSortThreads;
          z[u] = r < s1 ? __ldg(&in[r].z) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kBinSortHistPer; ++u)
          if (r0 + u * kBinSortThreads < s1) atomicAdd(&start[key_of(z[u])], 1u);
      }
      __syncthreads();
      cta_exclusive_scan(start, keys + 1, warp_sums);
    }
    for (uint32_t c0 = s0; c0 < s1; c0 += kBinSortChunk) {
      const int m = (int)min((uint32_t)kBinSortChunk, s1 - c0);
      uint4 rec[kBinSortPer];
      uint32_t idx[kBinSortPer], rank[kBinSortPer];
#pragma unroll
      for (int u = 0; u < kBinSortPer; ++u) {
        const int i = tid + u * kBinSortThreads;
        const uint32_t r = c0 + (uint32_t)min(i, m - 1);
        rec[u] = __ldcs(&in[r]);
        idx[u] = in_idx ? in_idx[r] : 0u;
        rank[u] = 0u;
      }
      for (int k = tid; k <= keys; k += kBinSortThreads) loc[k] = 0u;
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kBinSortPer; ++u)
        if (tid + u * kBinSortThreads < m) rank[u] = atomicAdd(&loc[key_of(rec[u].z)], 1u);
      __syncthreads();
      cta_exclusive_scan(loc, keys + 1, warp_sums);
#pragma unroll
      for (int u = 0; u < kBinSortPer; ++u) {
        if (tid + u * kBinSortThreads < m) {
          const uint32_t pos = loc[key_of(rec[u].z)] + rank[u];
          stage[pos] = rec[u];
          stage_idx[pos] = idx[u];
        }
      }
      __syncthreads();
      for (int i = tid; i < m; i += kBinSortThreads) {
        const uint4 v = stage[i];
        uint32_t pos = (uint32_t)i;
        if (multi) {
          const int k = key_of(v.z);
          pos = start[k] + ((uint32_t)i - loc[k]);
        }
        out[s0 + pos] = v;
        if (in_idx) out_idx[s0 + pos] = stage_idx[i];
      }
      __syncthreads();
      if (multi) {                                      // this chunk's runs come before the next chunk's
        for (int k = tid; k < keys; k += kBinSortThreads) start[k] += loc[k + 1] - loc[k];
        __syncthreads();
      }
    }
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&work[1], 1u) == gridDim.x - 1) {
      work[0] = 0u;
      work[1] = 0u;
      __threadfence();
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
                        int32_t nchan, bool pairs, bool for_degrid, bool keep_index,
                        cudaStream_t s) {
  const int64_t nvis = nrow * nchan;
  cudaError_t e;
  const int64_t nsub = ctx->nbins << ctx->nsub_log2;
  if ((e = cudaMemsetAsync(ctx->d_counts, 0, sizeof(uint32_t) * nsub, s))) return e;
  if ((e = cudaMemsetAsync(ctx->d_dropped, 0, sizeof(unsigned long long), s))) return e;
  if ((e = cudaMemsetAsync(ctx->d_wsum, 0, sizeof(double), s))) return e;
  const unsigned plan_blocks = (unsigned)((nvis + kPlanVis - 1) / kPlanVis);
  const FastDiv fdiv = FastDiv::make((uint32_t)std::max<int32_t>(nchan, 1));
  // a gridding plan asked to keep its binning also records each record's visibility index, for
  // wp_degrid_last
  const size_t nrec = (size_t)nvis * (pairs ? 2 : 1);
  uint32_t* index = (keep_index && !for_degrid && ctx->rec_index.bytes >= nrec * 4) ? (uint32_t*)ctx->rec_index.ptr : nullptr;
  ctx->launches += 4 + (nvis > 0 ? 2 : 0);  // prefix sum (3), bin offsets, histogram and scatter
  if (nvis > 0) {
    if ((e = cudaFuncSetAttribute(k_histogram, cudaFuncAttributeMaxDynamicSharedMemorySize, kHashBytes))) return e;
    k_histogram<<<plan_blocks, kPlanThreads, kHashBytes, s>>>(uvw, ctx->d_chan, for_degrid ? nullptr : weight, nvis, fdiv,
                                                       pairs ? 1 : 0, ctx->geo, ctx->d_counts, ctx->d_dropped,
                                                       ctx->d_wsum);
    if ((e = cudaGetLastError())) return e;
  }
  const int64_t tiles = (nsub + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(ctx->d_counts, nsub, ctx->d_suboff, ctx->d_partials);
  if ((e = cudaGetLastError())) return e;
  k_scan_partials<<<1, kScanThreads, 0, s>>>(ctx->d_partials, tiles);
  if ((e = cudaGetLastError())) return e;
  k_scan_finish<<<(unsigned)((nsub + 255) / 256), 256, 0, s>>>(ctx->d_suboff, ctx->d_cursor, nsub, ctx->d_partials,
                                                               tiles);
  if ((e = cudaGetLastError())) return e;
  k_gather_offsets<<<(unsigned)((ctx->nbins + 256) / 256), 256, 0, s>>>(ctx->d_suboff, ctx->nbins, ctx->nsub_log2,
                                                                          ctx->d_offsets);
  if ((e = cudaGetLastError())) return e;
  if (nvis > 0) {
    if ((e = cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, kHashBytes))) return e;
    k_scatter<<<plan_blocks, kPlanThreads, kHashBytes, s>>>(uvw, ctx->d_chan, vis, weight, nvis, fdiv, pairs ? 1 : 0,
                                                     for_degrid ? 1 : 0, ctx->geo, ctx->d_cursor,
                                                     (Record*)ctx->records.ptr, index);
    if ((e = cudaGetLastError())) return e;
  }
  // pass 4: every bin's records sorted by footprint origin, into the second record buffer, which
  // then becomes the context's record buffer (skipped when the buffers or the origin keys of a
  // tile do not fit: the kernels are correct for any order within a bin, only slower)
  const int keys = ctx->geo.tile_x * ctx->geo.tile_y;
  const bool index_ok = !index || ctx->rec_index2.bytes >= nrec * 4;
  if (nvis > 0 && keys <= kBinSortMaxKeys && ctx->records2.bytes >= nrec * sizeof(Record) && index_ok) {
    if ((e = cudaMemsetAsync(ctx->d_binwork, 0, 2 * sizeof(uint32_t), s))) return e;
    k_list_bins<<<(unsigned)((ctx->nbins + 255) / 256), 256, 0, s>>>(ctx->d_offsets, ctx->nbins, ctx->d_binlist,
                                                                      ctx->d_binwork);
    if ((e = cudaGetLastError())) return e;
    const size_t smem = 2 * sizeof(uint32_t) * (size_t)((keys + 1 + 3) & ~3) + (size_t)kBinSortChunk * 20;
    if ((e = cudaFuncSetAttribute(k_bin_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    k_bin_sort<<<ctx->nsm * 2, kBinSortThreads, smem, s>>>(
        (const uint4*)ctx->records.ptr, index, (uint4*)ctx->records2.ptr,
        index ? (uint32_t*)ctx->rec_index2.ptr : nullptr, ctx->d_offsets, ctx->nbins, ctx->d_binlist, ctx->d_binwork,
        ctx->geo, ctx->d_binwork + 2);
    if ((e = cudaGetLastError())) return e;
    ctx->launches += 2;
    std::swap(ctx->records, ctx->records2);
    if (index) std::swap(ctx->rec_index, ctx->rec_index2);
  }
  return cudaSuccess;
}

cudaError_t launch_bin_costs(wp_ctx* ctx, cudaStream_t s) {
  cudaError_t e;
  ctx->launches += 4;
  const unsigned blocks = (unsigned)((ctx->nbins + 255) / 256);
  // an upper bound of the total cost (the record buffer's capacity, the largest support, every
  // bin non-empty and rounded up) must stay below 2^31 units
  int smax = 0;
  for (int sp : ctx->supp) smax = std::max(smax, sp);
  const uint64_t nrec = ctx->records.bytes / sizeof(Record);
  const uint64_t bound = nrec * (uint64_t)(smax * smax + kRecordTaps) + (uint64_t)ctx->nbins * kBinFixedTaps;
  int shift = 0;
  while ((bound >> (6 + shift)) + (uint64_t)ctx->nbins >= (1ull << 31)) ++shift;
  k_bin_costs<<<blocks, 256, 0, s>>>(ctx->d_offsets, ctx->nbins, ctx->geo, shift, ctx->d_counts);
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
  k_coords_out<<<grid_blocks(nvis, ctx->nsm), 256, 0, s>>>(uvw, ctx->d_chan, nvis, FastDiv::make((uint32_t)nchan),
                                                            pairs ? 1 : 0, ctx->geo,
                                                            out);
  return cudaGetLastError();
}

}  // namespace wp
