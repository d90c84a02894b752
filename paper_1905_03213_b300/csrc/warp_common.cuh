// Device code shared by the warp-synchronous gridding (grid2.cu) and degridding (degrid2.cu)
// kernels: the lane layout of a footprint over a warp, the staged kernel-table layout, the
// in-order decode of a chunk of sorted records, the segment walk over the (plane, tile) bins
// and the work-unit schedule. Included by exactly those two files; every
// definition has internal linkage.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace wp {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxS = 32;                                     // larger supports: baseline kernel
constexpr int kMaxStagedS = 16;                               // larger: staged if it fits, else global
constexpr int kSmallMaxS = 16;                                // supports of the 32-warp launch shape
constexpr int kStagedChunk = 2048;                            // records left room for beside a large table
constexpr int kMaxKeys = 4096;                                  // origins of one segment
constexpr int kCountsBytes = ((kMaxKeys + 1) * 4 + 15) & ~15;  // shared-memory counters
constexpr int kMinChunk = 512;
constexpr int kSortPer = 16;                                  // records per thread in one sort
constexpr uint32_t kNoOrigin = 0xffffffffu;

// Lane layout. For support S <= 16 the warp's lanes form G row groups of S lanes; lane
// g*S + e holds rows g*R .. g*R + R - 1 of one footprint column. For 16 < S <= 32 (H = 2 row
// halves) two warps share the records of one piece: lane e < S of warp half h holds rows
// h*R .. h*R + R - 1 (R = ceil(S/2)). NL lanes hold a column; the others hold nothing.
__host__ __device__ constexpr int lay_halves(int s) { return s > kMaxStagedS ? 2 : 1; }
__host__ __device__ constexpr int lay_rows(int s) { return s > kMaxStagedS ? (s + 1) / 2 : (s + 32 / s - 1) / (32 / s); }
__host__ __device__ constexpr int lay_groups(int s) { return s > kMaxStagedS ? 1 : (s + lay_rows(s) - 1) / lay_rows(s); }
// rows spanned by the lanes of all groups or halves (>= s)
__host__ __device__ constexpr int lay_span(int s) { return lay_rows(s) * (lay_groups(s) > lay_halves(s) ? lay_groups(s) : lay_halves(s)); }

// Tap layout of one plane's table, per oversampling class: for each row half h and lane row
// r < R, a block of 32 slots, slot g*S + a holding tap (column a, row h*R + r or g*R + r) of
// the class; slots of rows >= S or beyond NL are zero. A slot is 4 bytes wide: with 16-bit
// tables it holds the stored element (__half2 or BfWord), and with float32 tables the block
// is two 128-byte halves, the real parts of the 32 slots and then their imaginary parts. A
// lane reads its current column's slot of each block with 4-byte loads, so any permutation of
// the slots (the gridding kernel rotates each group's columns as the footprint slides) keeps
// the 32 reads of one load on 32 distinct banks.
__host__ __device__ constexpr int tap_entry_bytes(int e) { return e == 4 ? 8 : 4; }
__host__ __device__ constexpr int lay_half_bytes(int s, int e) { return lay_rows(s) * 32 * tap_entry_bytes(e); }
__host__ __device__ constexpr int lay_class_bytes(int s, int e) { return lay_halves(s) * lay_half_bytes(s, e); }
// bytes of one plane's table that must fit shared memory (S <= 16; larger tables are staged
// only when they fit beside a chunk, else read from their global copy)
__host__ __device__ constexpr int lay_staged_bytes(int os, int s, int e) {
  return s > kMaxStagedS ? 0 : os * os * lay_class_bytes(s, e);
}

template <class T>
struct TabElem;  // component size of a stored table element (a complex tap)
template <>
struct TabElem<float2> {
  static constexpr int E = 4;
};
template <>
struct TabElem<__half2> {
  static constexpr int E = 2;
};
template <>
struct TabElem<BfWord> {
  static constexpr int E = 2;
};

template <int S, class T = float2>
struct Lay {
  static constexpr int R = lay_rows(S), G = lay_groups(S), H = lay_halves(S), NL = G * S;
  static constexpr int E = TabElem<T>::E;
  static constexpr int SB = 4;                   // bytes between slots (float32: per component half)
  static constexpr int BB = 32 * tap_entry_bytes(E);   // bytes of one row block
  static constexpr int HB = lay_half_bytes(S, E);
  static constexpr int CB = lay_class_bytes(S, E);
};

// The number of leading planes whose support is at most kSmallMaxS: their bins are the prefix
// [0, end * ntiles) of the bin order, run in the 32-warp shape; the others in the 16-warp shape.
inline int64_t small_planes_end(const wp_ctx* ctx) {
  int64_t p = 0;
  while (p < (int64_t)ctx->supp.size() && ctx->supp[(size_t)p] <= kSmallMaxS) ++p;
  return p;
}

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

// Packed pair of floats as one 64-bit register for fma.rn.f32x2.
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
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// Vector reduction (no return value) of two floats into global memory: *p += (x, y).
__device__ __forceinline__ void red_add2(float2* p, float x, float y) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(x), "f"(y) : "memory");
}

// Atomic addition of two floats into global memory returning the previous values (one vector
// atomic, rounded to nearest like the reduction).
__device__ __forceinline__ float2 atom_add2(float2* p, float x, float y) {
  float2 old;
  asm volatile("atom.global.v2.f32.add {%0, %1}, [%2], {%3, %4};" : "=f"(old.x), "=f"(old.y) : "l"(p), "f"(x), "f"(y)
               : "memory");
  return old;
}

// The rounding error e of s = fl(a + b), so that a + b = s + e exactly (Knuth's TwoSum: six
// additions in round-to-nearest, no ordering of |a| and |b| needed).
__device__ __forceinline__ float two_sum_err(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  return __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// red_add2 where p is true: one predicated instruction, no branch.
__device__ __forceinline__ void red_add2_if(bool pred, float2* p, float x, float y) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q red.global.add.v2.f32 [%0], {%1, %2};\n\t}"
      ::"l"(p), "f"(x), "f"(y), "r"((uint32_t)pred) : "memory");
}

// One tap of the tap layout as the float32 pair (kr, ki) in a 64-bit register, from its slot
// at p: in shared memory, or (kGlobal) in the global copy, read through the read-only path.
template <class T, bool kGlobal>
__device__ __forceinline__ unsigned long long tap_pair(const unsigned char* p);
template <>
__device__ __forceinline__ unsigned long long tap_pair<float2, false>(const unsigned char* p) {
  return (unsigned long long)*(const uint32_t*)p | ((unsigned long long)*(const uint32_t*)(p + 128) << 32);
}
template <>
__device__ __forceinline__ unsigned long long tap_pair<float2, true>(const unsigned char* p) {
  return (unsigned long long)__ldg((const uint32_t*)p) | ((unsigned long long)__ldg((const uint32_t*)(p + 128)) << 32);
}
template <bool kGlobal>
__device__ __forceinline__ unsigned long long half_pair(const unsigned char* p) {
  const __half2 h = kGlobal ? __ldg((const __half2*)p) : *(const __half2*)p;
  const float2 f = __half22float2(h);
  return pack2(f.x, f.y);
}
template <>
__device__ __forceinline__ unsigned long long tap_pair<__half2, false>(const unsigned char* p) {
  return half_pair<false>(p);
}
template <>
__device__ __forceinline__ unsigned long long tap_pair<__half2, true>(const unsigned char* p) {
  return half_pair<true>(p);
}
// BfWord: kr = word << 16, ki = word (see BfWord)
template <>
__device__ __forceinline__ unsigned long long tap_pair<BfWord, false>(const unsigned char* p) {
  const uint32_t w = *(const uint32_t*)p;
  return (unsigned long long)(w << 16) | ((unsigned long long)w << 32);
}
template <>
__device__ __forceinline__ unsigned long long tap_pair<BfWord, true>(const unsigned char* p) {
  const uint32_t w = __ldg((const uint32_t*)p);
  return (unsigned long long)(w << 16) | ((unsigned long long)w << 32);
}

// Entry i of one plane's tap-layout table (classes x halves x R blocks x 32 slots, in that
// order), copied from the stored layout src[(cls * S + a) * S + b] of T; written at dst.
template <class T>
__device__ __forceinline__ void write_tap_entry(const T* __restrict__ src, int s, unsigned char* dst, int i) {
  const int r_rows = lay_rows(s), g_rows = lay_groups(s), halves = lay_halves(s);
  const int per_class = halves * r_rows * 32;
  const int cls = i / per_class, rem = i - cls * per_class;
  const int h = rem / (r_rows * 32), rem2 = rem - h * (r_rows * 32);
  const int r = rem2 >> 5, slot = rem2 & 31;
  const int g = slot / s, a = slot - g * s;
  const int b = (halves > 1 ? h : g) * r_rows + r;
  const bool valid = slot < g_rows * s && b < s;
  T v;
  if (valid) v = src[((int64_t)cls * s + a) * s + b];
  else memset(&v, 0, sizeof(T));
  if constexpr (sizeof(T) == 8) {               // float32: real parts, then imaginary parts
    unsigned char* blk = dst + (int64_t)(i >> 5) * 256;
    uint32_t c[2];
    memcpy(c, &v, 8);
    *(uint32_t*)(blk + slot * 4) = c[0];
    *(uint32_t*)(blk + 128 + slot * 4) = c[1];
  } else {
    *(T*)(dst + (int64_t)i * sizeof(T)) = v;
  }
}
__host__ __device__ constexpr int tap_entries(int os, int s) { return os * os * lay_halves(s) * lay_rows(s) * 32; }

// Stages one plane's table (stored layout) in the tap layout at byte offset tab_off of the
// dynamic shared memory: a plain copy of each element into its slot.
template <int S, class T = float2>
__device__ __forceinline__ void stage_table(const T* __restrict__ src, int os, int tab_off) {
  unsigned char* dst = dyn_smem() + tab_off;
  const int n = tap_entries(os, S);
  for (int i = threadIdx.x; i < n; i += blockDim.x) write_tap_entry<T>(src, S, dst, i);
}

// Decodes the records grecs[c0, c0 + m) of one segment into the shared array the caller's
// `emit(slot, rec, idx)` writes, in their order (the plan has sorted every bin by footprint
// origin, and a segment's bins follow one another). Each thread takes PER consecutive
// records, all loads in flight together. With `index` (a gridding plan's visibility index per
// record, partner flag in bit 31) the Hermitian partners are left out and the others close up.
// Returns the number of records decoded.
// NT threads (the CTA); warp_sums: NT / 32 words of shared memory for the prefix sum.
template <int NT, int PER, class Emit>
__device__ __forceinline__ int decode_chunk(const uint4* __restrict__ grecs, const uint32_t* __restrict__ index,
                                            uint32_t c0, int m, uint32_t* warp_sums, Emit emit) {
  constexpr int kW = NT / 32;
  uint4 rec[PER];
  uint32_t idx[PER];
  const int first = threadIdx.x * PER;
  int count = 0;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int i = min(first + u, m - 1);            // m >= 1: loads past the chunk repeat its last record
    rec[u] = __ldcs(grecs + c0 + i);
    idx[u] = index ? index[c0 + i] : 0u;
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) count += (first + u < m && !(idx[u] >> 31)) ? 1 : 0;
  // exclusive prefix of the threads' counts
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = (uint32_t)count;
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < kW ? warp_sums[lane] : 0u;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, off);
      if (lane >= off) v += y;
    }
    if (lane < kW) warp_sums[lane] = v;
  }
  __syncthreads();
  int pos = (int)((warp ? warp_sums[warp - 1] : 0u) + x) - count;
  const int kept = (int)warp_sums[kW - 1];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    if (first + u < m && !(idx[u] >> 31)) {
      emit(pos, rec[u], idx[u]);
      ++pos;
    }
  }
  __syncthreads();
  return kept;
}

// Work units: unit u covers the estimated-work range [ctotal u / nunits, ctotal (u + 1) /
// nunits). Cost position x maps to bin b (costoff[b] <= x < costoff[b+1]) and to the record
// offsets[b] + (x - costoff[b]) / cost_b * count_b, a monotone map, so the units partition
// the records exactly. CTAs take units from work[0], the last one first; the last CTA to
// finish leaves work[0] and work[1] zero for the next launch. body(beg, end) runs with the
// whole CTA.
//
// kTapered: unit u covers [C (u / N)^2, C ((u + 1) / N)^2) instead, so the units taken first (the
// highest u) are the largest, about twice the mean, and the last ones taken are small: the CTAs
// finish within a small unit of each other.
// Only the bins [bin_lo, bin_hi) are cut into units (a launch that grids part of the planes).
template <bool kTapered = false, class Body>
__device__ __forceinline__ void for_each_unit(const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ costoff,
                                              int64_t nbins, int64_t bin_lo, int64_t bin_hi, int nunits,
                                              uint32_t* work, Body body) {
  __shared__ int unit;
  const uint32_t total = offsets[bin_hi];
  const uint32_t clo = costoff[bin_lo], chi = costoff[bin_hi];
  const uint32_t ctotal = chi - clo;
  auto split = [&](uint64_t x) -> uint32_t {        // x: cost position relative to clo
    if (x >= ctotal) return total;
    const int64_t b = find_bin(costoff, nbins, clo + (uint32_t)x);
    const uint32_t c0 = costoff[b], cb = costoff[b + 1] - c0;
    const uint32_t n = offsets[b + 1] - offsets[b];
    return offsets[b] + (uint32_t)(((uint64_t)(clo + x - c0) * n) / cb);
  };
  for (;;) {
    if (threadIdx.x == 0) unit = nunits - 1 - (int)atomicAdd(&work[0], 1u);
    __syncthreads();
    const int u = unit;
    __syncthreads();
    if (u < 0) break;
    // ctotal < 2^32 and nunits < 2^16 keep the products below 2^64
    const uint64_t nn = kTapered ? (uint64_t)nunits * nunits : (uint64_t)nunits;
    const uint64_t u0 = kTapered ? (uint64_t)u * u : (uint64_t)u;
    const uint64_t u1 = kTapered ? (uint64_t)(u + 1) * (u + 1) : (uint64_t)(u + 1);
    const uint32_t beg = split((uint64_t)ctotal * u0 / nn);
    const uint32_t end = split((uint64_t)ctotal * u1 / nn);
    if (beg < end) body(beg, end);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&work[1], 1u) == gridDim.x - 1) {
      work[0] = 0u;
      work[1] = 0u;
      __threadfence();
    }
  }
}

}  // namespace
}  // namespace wp
