// Device code shared by the warp-synchronous gridding (grid2.cu) and degridding (degrid2.cu)
// kernels: the lane layout of a footprint over a warp, the staged kernel-table layout, the
// in-CTA counting sort of binned records by footprint origin, the segment walk over the
// (plane, tile) bins and the work-unit schedule. Included by exactly those two files; every
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
constexpr int kStagedChunk = 2048;                            // records left room for beside a large table
constexpr int kMaxKeys = 4096;                                  // origins of one segment
constexpr int kCountsBytes = ((kMaxKeys + 1) * 4 + 15) & ~15;  // shared-memory counters
constexpr int kMinChunk = 512;
constexpr int kSortPer = 16;                                  // records per thread in one sort
constexpr int kMaxChunk = kThreads * kSortPer;                 // records of one sorted chunk, at most
constexpr uint32_t kNoOrigin = 0xffffffffu;
constexpr int kUnitsPerCta = 6;                              // work units per CTA, on average


// Lane layout for support S <= 16: G row groups of S lanes; lane g*S + a holds rows g*R ..
// g*R + R - 1 of footprint column a, as RP row pairs and RT (0/1) single tail row. For
// 16 < S <= 32 (H = 2 row halves) two warps share the records of one piece: lane a of warp
// half h holds rows h*R .. h*R + R - 1 (R = ceil(S/2)) of column a.
//
// Table of one oversampling class in lane order, for tap components of E bytes (4: f32, 2:
// f16/bf16), one entry per lane in 32-lane blocks (lanes and rows outside the footprint hold
// zeros), per row half:
//   f32:     per row pair k a block of float2 {kr(2k), kr(2k+1)} then a block of float2
//            {ki(2k), ki(2k+1)}; then for the tail row a block of float2 {kr, ki}.
//   f16/bf16: per row pair k one block of 8-byte entries {kr(2k), kr(2k+1), ki(2k), ki(2k+1)};
//            then for the tail row a block of 4-byte entries {kr, ki}.
// Either way a lane reads 8 bytes per row pair and load instruction. Tables of S <= 16 are
// staged in shared memory per plane; for S > 16 a copy in this layout is built in global memory
// once (it does not fit shared memory at oversampling 8) and read through the L1/L2 path.
__host__ __device__ constexpr int lay_halves(int s) { return s > kMaxStagedS ? 2 : 1; }
__host__ __device__ constexpr int lay_rows(int s) { return s > kMaxStagedS ? (s + 1) / 2 : (s + 32 / s - 1) / (32 / s); }
__host__ __device__ constexpr int lay_groups(int s) { return s > kMaxStagedS ? 1 : (s + lay_rows(s) - 1) / lay_rows(s); }
// rows spanned by the lanes of all groups or halves (>= s)
__host__ __device__ constexpr int lay_span(int s) { return lay_rows(s) * (lay_groups(s) > lay_halves(s) ? lay_groups(s) : lay_halves(s)); }
// bytes of one row half of a class, and of a class
__host__ __device__ constexpr int lay_half_bytes(int s, int e) {
  return ((lay_rows(s) / 2) * 128 + (lay_rows(s) & 1) * 64) * e;
}
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
struct TabElem<__nv_bfloat162> {
  static constexpr int E = 2;
};

template <int S, class T = float2>
struct Lay {
  static constexpr int R = lay_rows(S), G = lay_groups(S), H = lay_halves(S), NL = G * S;
  static constexpr int RP = R / 2, RT = R & 1, RPA = RP > 0 ? RP : 1;
  static constexpr int E = TabElem<T>::E;
  static constexpr int PB = 128 * E;           // bytes of one row pair's blocks
  static constexpr int HB = lay_half_bytes(S, E);
  static constexpr int CB = lay_class_bytes(S, E);
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
__device__ __forceinline__ void block_exclusive_scan(int n) {
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
// Vector reduction (no return value) of two floats into global memory: *p += (x, y).
__device__ __forceinline__ void red_add2(float2* p, float x, float y) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(x), "f"(y) : "memory");
}

// red_add2 where p is true: one predicated instruction, no branch.
__device__ __forceinline__ void red_add2_if(bool pred, float2* p, float x, float y) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\t@q red.global.add.v2.f32 [%0], {%1, %2};\n\t}"
      ::"l"(p), "f"(x), "f"(y), "r"((uint32_t)pred) : "memory");
}

__device__ __forceinline__ unsigned long long shfl_down2(unsigned long long v, int d) {
  const uint32_t lo = __shfl_down_sync(0xffffffffu, (uint32_t)v, d);
  const uint32_t hi = __shfl_down_sync(0xffffffffu, (uint32_t)(v >> 32), d);
  return (unsigned long long)lo | ((unsigned long long)hi << 32);
}

__device__ __forceinline__ float2 to_float2(__half2 h) { return __half22float2(h); }
__device__ __forceinline__ float2 to_float2(__nv_bfloat162 h) { return __bfloat1622float2(h); }
template <class T>
__device__ __forceinline__ T bits_as(uint32_t u) {
  T t;
  memcpy(&t, &u, 4);
  return t;
}

// This lane's taps of one record as float32: RP row pairs packed {kr(2k), kr(2k+1)} and
// {ki(2k), ki(2k+1)} for f32x2 FMAs, and the tail row.
template <int S, class T = float2, bool kGlobal = false>
struct Taps {
  unsigned long long r[Lay<S, T>::RPA], i[Lay<S, T>::RPA];
  float tr, ti;
  // Lanes beyond the layout (lane >= NL) read their all-zero table entries. cls_base points into
  // shared memory, or (kGlobal) into the global lane-order copy, read through the read-only path.
  template <class U>
  static __device__ __forceinline__ U rd(const unsigned char* p) {
    if constexpr (kGlobal) return __ldg((const U*)p);
    else return *(const U*)p;
  }
  __device__ __forceinline__ void load(const unsigned char* cls_base, int lane) {
    using L = Lay<S, T>;
    if constexpr (L::E == 4) {
#pragma unroll
      for (int k = 0; k < L::RP; ++k) {
        r[k] = rd<unsigned long long>(cls_base + k * L::PB + lane * 8);
        i[k] = rd<unsigned long long>(cls_base + k * L::PB + 256 + lane * 8);
      }
      if (L::RT) {
        const float2 t = rd<float2>(cls_base + L::RP * L::PB + lane * 8);
        tr = t.x;
        ti = t.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < L::RP; ++k) {
        const uint2 v = rd<uint2>(cls_base + k * L::PB + lane * 8);
        const float2 a = to_float2(bits_as<T>(v.x)), b = to_float2(bits_as<T>(v.y));
        r[k] = pack2(a.x, a.y);
        i[k] = pack2(b.x, b.y);
      }
      if (L::RT) {
        const float2 t = to_float2(bits_as<T>(rd<uint32_t>(cls_base + L::RP * L::PB + lane * 4)));
        tr = t.x;
        ti = t.y;
      }
    }
  }
};

__device__ __forceinline__ float2 tap_float2(float2 v) { return v; }
__device__ __forceinline__ float2 tap_float2(__half2 v) { return __half22float2(v); }
__device__ __forceinline__ float2 tap_float2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
__device__ __forceinline__ uint32_t pack_pair(__half2, float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}
__device__ __forceinline__ uint32_t pack_pair(__nv_bfloat162, float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

// Entry i of the two-row-half lane layout (16 < s <= 32) of one plane's table: the table's
// classes x halves x (row pairs + tail) x 32 lanes entries in order; writes it below dst.
template <class T>
__device__ __forceinline__ void write_half_entry(const T* __restrict__ src, int s, unsigned char* dst, int i) {
  constexpr int E = TabElem<T>::E, PB = 128 * E;
  const int r = (s + 1) / 2, rp = r / 2, per = rp + (r & 1);
  const int hb = lay_half_bytes(s, E), cb = 2 * hb;
  const int cls = i / (2 * 32 * per), rem = i - cls * (2 * 32 * per);
  const int h = rem / (32 * per), rem2 = rem - h * (32 * per);
  const int k = rem2 >> 5, lane = rem2 & 31;
  const bool active = lane < s;
  const int b0 = h * r + 2 * k;
  const T* col = src + ((int64_t)cls * s + lane) * s;
  const float2 v0 = (active && b0 < s) ? tap_float2(col[b0]) : make_float2(0.f, 0.f);
  unsigned char* base = dst + (int64_t)cls * cb + h * hb + k * PB;
  if (k < rp) {
    const float2 v1 = (active && b0 + 1 < s) ? tap_float2(col[b0 + 1]) : make_float2(0.f, 0.f);
    if constexpr (E == 4) {
      *(float2*)(base + lane * 8) = make_float2(v0.x, v1.x);
      *(float2*)(base + 256 + lane * 8) = make_float2(v0.y, v1.y);
    } else {
      *(uint2*)(base + lane * 8) = make_uint2(pack_pair(T{}, v0.x, v1.x), pack_pair(T{}, v0.y, v1.y));
    }
  } else {
    if constexpr (E == 4) *(float2*)(base + lane * 8) = v0;
    else *(uint32_t*)(base + lane * 4) = pack_pair(T{}, v0.x, v0.y);
  }
}
__host__ __device__ constexpr int half_entries(int os, int s) {
  return os * os * 2 * 32 * ((s + 1) / 2 / 2 + ((s + 1) / 2 & 1));
}

// Stages one plane's table (src: stored layout [oy*os+ox][a][b] of T) in the lane layout of
// Lay<S, T> at byte offset tab_off of the dynamic shared memory. 16-bit components are copied
// exactly (each is representable after the round trip through float32).
template <int S, class T = float2>
__device__ __forceinline__ void stage_table(const T* __restrict__ src, int os, int tab_off) {
  using L = Lay<S, T>;
  if constexpr (L::H > 1) {
    for (int i = threadIdx.x; i < half_entries(os, S); i += kThreads) write_half_entry<T>(src, S, dyn_smem() + tab_off, i);
    return;
  }
  constexpr int kPer = L::RP + L::RT;           // entries per lane and class
  const int ncls = os * os;
  unsigned char* dst = dyn_smem() + tab_off;
  for (int i = threadIdx.x; i < ncls * 32 * kPer; i += kThreads) {
    const int cls = i / (32 * kPer), rem = i - cls * (32 * kPer);
    const int k = rem >> 5, lane = rem & 31;
    const int g = lane / S, col = lane - g * S;
    const bool active = lane < L::NL;
    const int b0 = g * L::R + 2 * k;
    const T* s = src + ((int64_t)cls * S + col) * S;
    const float2 v0 = (active && b0 < S) ? tap_float2(s[b0]) : make_float2(0.f, 0.f);
    unsigned char* base = dst + cls * L::CB + k * L::PB;
    if (k < L::RP) {
      const float2 v1 = (active && b0 + 1 < S) ? tap_float2(s[b0 + 1]) : make_float2(0.f, 0.f);
      if constexpr (L::E == 4) {
        *(float2*)(base + lane * 8) = make_float2(v0.x, v1.x);
        *(float2*)(base + 256 + lane * 8) = make_float2(v0.y, v1.y);
      } else {
        *(uint2*)(base + lane * 8) = make_uint2(pack_pair(T{}, v0.x, v1.x), pack_pair(T{}, v0.y, v1.y));
      }
    } else {
      if constexpr (L::E == 4) *(float2*)(base + lane * 8) = v0;
      else *(uint32_t*)(base + lane * 4) = pack_pair(T{}, v0.x, v0.y);
    }
  }
}

// Counting-sorts the binned records grecs[c0, c0 + m) of one segment (origin tiles of one
// tile row, columns x0 .. x0 + width, rows y0 .. y0 + tile_y) by origin key (row-major within
// the segment) into the shared array at byte offset rec_off, decoding each into
//   x, y : as binned;  z : i0 | j0 << 16;  w : class byte offset in the staged table | conj << 31.
// With `index` (a gridding plan's visibility index per record, partner flag in bit 31) the
// Hermitian partners are left out and x becomes the visibility index. Returns the number of
// records sorted; counts[key] (the shared counters at offset 0) is then the end of each key.
template <int S, class T = float2>
__device__ __forceinline__ int sort_chunk(const uint4* __restrict__ grecs, const uint32_t* __restrict__ index,
                                          uint32_t c0, int m, int x0, int y0, int width, int keys, int os,
                                          int rec_off) {
  using L = Lay<S, T>;
  uint32_t* counts = (uint32_t*)dyn_smem();
  uint4* drec = (uint4*)(dyn_smem() + rec_off);
  // the whole chunk is read in one round of independent loads (kSortPer per thread), so the
  // sort waits for global memory once; the counters are cleared while the loads are in flight
  uint4 rec[kSortPer];
  uint32_t idx[kSortPer];
#pragma unroll
  for (int u = 0; u < kSortPer; ++u) {
    const int r = threadIdx.x + u * kThreads;
    const int rr = min(r, m - 1);                 // m >= 1: loads past the chunk repeat its last record
    idx[u] = index ? index[c0 + rr] : 0u;
    rec[u] = __ldcs(grecs + c0 + rr);
  }
  for (int k = threadIdx.x; k <= keys; k += kThreads) counts[k] = 0u;
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kSortPer; ++u)
    if (threadIdx.x + u * kThreads < m && !(idx[u] >> 31))
      atomicAdd(&counts[((int)(rec[u].z >> 16) - y0) * width + ((int)(rec[u].z & 0xffff) - x0)], 1u);
  __syncthreads();
  block_exclusive_scan(keys + 1);
  const int kept = (int)counts[keys];
  // decode each record into its sorted slot
#pragma unroll
  for (int u = 0; u < kSortPer; ++u) {
    if (threadIdx.x + u * kThreads < m && !(idx[u] >> 31)) {
      const int key = ((int)(rec[u].z >> 16) - y0) * width + ((int)(rec[u].z & 0xffff) - x0);
      const int cls = (int)((rec[u].w >> 8) & 0xff) * os + (int)(rec[u].w & 0xff);
      const uint32_t w = (uint32_t)(cls * L::CB) | (rec[u].w & 0x80000000u);
      drec[atomicAdd(&counts[key], 1u)] = make_uint4(index ? idx[u] : rec[u].x, rec[u].y, rec[u].z, w);
    }
  }
  __syncthreads();
  return kept;
}

// The segment starting at record `pos` of bin `bin` (tile column tx): the bin, plus the
// following bins of the same tile row while all their records still fit one chunk of `cap`
// (sparse tiles are sorted together, dense ones alone), never beyond `end`.
__device__ __forceinline__ uint32_t segment_end(const uint32_t* __restrict__ offsets, int64_t nbins, int64_t bin,
                                                int tx, int ntx, uint32_t pos, uint32_t end, int cap,
                                                int group_tiles, int* ntiles) {
  uint32_t bound[8];                            // ends of this bin and the next 7 (independent loads)
#pragma unroll
  for (int k = 0; k < 8; ++k) bound[k] = offsets[min(bin + k + 1, nbins)];
  uint32_t seg_end = min(end, bound[0]);
  int nt = 1;
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    if (nt == k && k < group_tiles && tx + k < ntx && seg_end < end) {
      const uint32_t nxt = min(end, bound[k]);
      if (nxt - pos <= (uint32_t)cap) {
        seg_end = nxt;
        nt = k + 1;
      }
    }
  }
  *ntiles = nt;
  return seg_end;
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
template <bool kTapered = false, class Body>
__device__ __forceinline__ void for_each_unit(const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ costoff,
                                              int64_t nbins, int nunits, uint32_t* work, Body body) {
  __shared__ int unit;
  const uint32_t total = offsets[nbins];
  const uint32_t ctotal = costoff[nbins];
  auto split = [&](uint64_t x) -> uint32_t {
    if (x >= ctotal) return total;
    const int64_t b = find_bin(costoff, nbins, (uint32_t)x);
    const uint32_t c0 = costoff[b], cb = costoff[b + 1] - c0;
    const uint32_t n = offsets[b + 1] - offsets[b];
    return offsets[b] + (uint32_t)(((uint64_t)(x - c0) * n) / cb);
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
