// Register-holding degridding kernel (the hot path of wp_degrid).
//
// Degridding (Sec. 2.1 of Lao et al. 2019; the adjoint of gridding): visibility k is
//   V_k = sum_{a,b} conj(K_k(a, b)) G(i0 + a, j0 + b),
// with K_k = K_p for w >= 0 and conj(K_p) for w < 0. The organisation mirrors the gridding
// kernel (grid2.cu): CTAs take work units of equal estimated work and decode each chunk of the
// records, which the plan has sorted by footprint origin within every (plane, tile) bin, into
// shared memory; each warp walks a contiguous piece of the chunk with all 32 lanes on the same
// record.
//
//   * The grid region under the segment's footprints is staged in shared memory once per
//     segment; lane (g, a) keeps the cells of its rows of footprint column a in registers
//     (row pairs packed for f32x2 FMAs) and reloads them only when the origin changes.
//   * Per record a lane multiplies its taps (the same tap layout as gridding, 4-byte loads)
//     with its cells into a partial sum; the partials of a batch of records are then reduced
//     across the warp with a halving butterfly (about one shuffle per record and component),
//     after which each record's total sits in the lanes batch_record names and one of them
//     stores it.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "warp_common.cuh"

namespace wp {

namespace {

constexpr int kDecodeScratch = 128;            // bytes of dynamic shared memory before the table
// Two launch shapes, as for gridding: 32 warps (64 registers a thread) when every support is at
// most 16, else 16. The 32-warp shape decodes 4 records per thread per chunk and reduces batches
// of 8 records, which keeps it within its registers: 1.69 -> 1.61 ms on the float32 workload
// against 24 warps with 8 records per thread and batches of 16.
constexpr int kDegridThreadsSmall = 1024;
constexpr int kDegridThreadsLarge = 512;
// records per thread in one decoded chunk
__host__ __device__ constexpr int decode_per(int threads) { return threads == kDegridThreadsSmall ? 4 : 16; }

struct D2Args {
  const Record* recs;
  const uint32_t* offsets;
  const uint32_t* costoff;  // [nbins + 1] prefix sums of per-bin work estimates
  int64_t nbins;
  Geometry g;
  const void* tab;          // stored tables (f32, f16 or bf16 taps), layout [plane][oy*os+ox][a][b]
  const int64_t* tab_off;
  const unsigned char* lanetab;   // lane-order tables of the planes with S > 16 (global)
  const int64_t* lanetab_off;     // [Nw] byte offset of each plane in lanetab (-1: none)
  const float2* grid;
  float2* out;              // visibilities in caller order (record x = caller index)
  const uint32_t* index;    // gridding plan's visibility index per record (partners flagged), or nullptr
  int smem_bytes;
  int group_tiles;
  int nunits;
  int64_t bin_lo, bin_hi;   // the bins this launch degrids (a prefix or suffix of the planes)
  uint32_t* work;           // [2]: next unit, finished CTAs (both zero between launches)
};

// Row pitch (float2 entries) of the staged grid region: the smallest p >= cols with p = 4
// mod 8, so rows two apart fall in opposite halves of the 32 banks.
__host__ __device__ constexpr int sub_pitch(int cols) { return cols + ((12 - cols % 8) % 8); }
// Rows staged for support s: the tile rows plus every row a lane of the layout can address.
__host__ __device__ constexpr int sub_rows(int tile_y, int s) { return tile_y + lay_span(s) - 1; }
__host__ __device__ constexpr int sub_bytes(int tile_x, int tile_y, int group, int s) {
  return sub_rows(tile_y, s) * sub_pitch(group * tile_x + s - 1) * 8;
}

// Butterfly over the warp: on entry every lane holds partials v[0..NB) of the batch's NB
// records; on return v[0] of lane l is the warp total of record l mod NB.
// Sums each of NB per-lane partials over the warp's 32 lanes. Halving levels first, at lane
// bits 16, 8, ...: at each, a lane sends the half of its values that the lane across the bit
// keeps, and adds the other half's partner values, so the values held halve per level; then
// full sums over the remaining low lane bits. Lane l ends with the total of record
// batch_record<NB>(l) in v[0] (the same in the lanes that differ only in the low bits).
// NB = 8: 9 shuffles and 9 additions per component and batch (23 and 23 summing first).
template <int NB>
__device__ __forceinline__ void batch_reduce(float (&v)[NB], int lane) {
  static_assert(NB == 8 || NB == 16 || NB == 32, "batch of 8, 16 or 32 records");
#pragma unroll
  for (int half = NB / 2, bit = 16; half >= 1; half >>= 1, bit >>= 1) {
    const bool upper = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = upper ? v[i] : v[i + half];
      const float keep = upper ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
  }
#pragma unroll
  for (int bit = 16 / (NB / 2) / 2; bit >= 1; bit >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], bit);
}
// The batch record whose total lane l holds after batch_reduce<NB>, and whether l is the lane
// that stores it (its bits below the halving levels are zero).
template <int NB>
__device__ __forceinline__ int batch_record(int lane) {
  int r = 0;
#pragma unroll
  for (int half = NB / 2, bit = 16; half >= 1; half >>= 1, bit >>= 1) r += (lane & bit) ? half : 0;
  return r;
}
template <int NB>
__device__ __forceinline__ bool batch_writer(int lane) {
  return (lane & (32 / NB - 1)) == 0;
}

// One warp degrids the decoded, sorted records [beg, end) of the chunk at byte offset rec_off
// from the grid region staged at sub_off (pitch entries per row, origin (sx0, sy0)). Table as
// in the gridding kernel (tap layout staged at tab_off, or the global copy gtab for S > 16,
// row half h); with two row halves each warp adds its half of every visibility to the
// (zeroed) output. Decoded record: x = output index, y = s as float bits (+1 for K_k = K_p,
// -1 for K_k = conj K_p), z = origin i0 | j0 << 16, w = class byte offset in the table.
//
// Per record a lane forms, over its rows, with the tap pair (kr, ki) and its cell (gr, gi)
// (held as the pairs (gr, gi) and (gi, gr)):
//   P1 += (kr, ki) * (gr, gi),  P2 += (kr, ki) * (gi, gr)
// and its part of conj(K_k) G is (P1.x + s P1.y) + i (P2.x - s P2.y).
template <int S, class T, bool kGlobal, int NT>
__device__ __forceinline__ void warp_degrid(int tab_off, const unsigned char* gtab, int h, int sub_off, int pitch,
                                            int sx0, int sy0, int rec_off, int beg, int end,
                                            float2* __restrict__ out) {
  using L = Lay<S, T>;
  constexpr int NB = NT == kDegridThreadsSmall ? 8 : (L::R <= 5 ? 32 : 16);
  const int lane = threadIdx.x & 31;
  const int g = lane / S, slot = lane - g * S;
  // lanes beyond the layout read (zero-tap) cells of the half's first row
  const int row0 = L::H > 1 ? h * L::R : (lane < L::NL ? g * L::R : 0);
  const unsigned char* lt = (kGlobal ? gtab : dyn_smem() + tab_off) + h * L::HB + lane * L::SB;
  const float2* sub = (const float2*)(dyn_smem() + sub_off);
  const uint4* drec = (const uint4*)(dyn_smem() + rec_off);
  unsigned long long GA[L::R], GB[L::R];      // cells (gr, gi) and (gi, gr) of this lane's rows
#pragma unroll
  for (int k = 0; k < L::R; ++k) GA[k] = GB[k] = 0ull;
  uint32_t cz = kNoOrigin;
  for (int b0 = beg; b0 < end; b0 += NB) {
    float pre[NB], pim[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      pre[r] = pim[r] = 0.f;
      if (b0 + r < end) {                          // warp-uniform
        const uint4 rec = drec[b0 + r];
        if (rec.z != cz) {                         // warp-uniform: load the cells under the new origin
          cz = rec.z;
          const float2* c = sub + ((int)(rec.z >> 16) - sy0 + row0) * pitch + ((int)(rec.z & 0xffff) - sx0) + slot;
#pragma unroll
          for (int k = 0; k < L::R; ++k) {
            const float2 v = c[k * pitch];
            GA[k] = pack2(v.x, v.y);
            GB[k] = pack2(v.y, v.x);
          }
        }
        const unsigned char* p = lt + rec.w;
        unsigned long long P1 = 0ull, P2 = 0ull;
#pragma unroll
        for (int k = 0; k < L::R; ++k) {
          const unsigned long long t = tap_pair<T, kGlobal>(p + k * L::BB);
          P1 = fma2(t, GA[k], P1);
          P2 = fma2(t, GB[k], P2);
        }
        const float sg = __uint_as_float(rec.y);
        pre[r] = fmaf(sg, hi_of(P1), lo_of(P1));
        pim[r] = fmaf(-sg, hi_of(P2), lo_of(P2));
      }
    }
    batch_reduce<NB>(pre, lane);
    batch_reduce<NB>(pim, lane);
    const int rb = b0 + batch_record<NB>(lane);
    if (batch_writer<NB>(lane) && rb < end) {
      if constexpr (L::H > 1) red_add2(&out[drec[rb].x], pre[0], pim[0]);
      else out[drec[rb].x] = make_float2(pre[0], pim[0]);
    }
  }
}

template <int S, class T, int NT>
__device__ __noinline__ void degrid_segment(const D2Args& a, int p, bool stage, bool staged, int x0, int y0, int width,
                                            uint32_t s0, uint32_t s1, int cap, int tab_off, int sub_off,
                                            int rec_off) {
  using L = Lay<S, T>;
  if (staged && stage) stage_table<S, T>((const T*)a.tab + a.tab_off[p], a.g.os, tab_off);
  const unsigned char* gtab = staged ? nullptr : a.lanetab + a.lanetab_off[p];
  constexpr int kPieces = NT / 32 / L::H;          // warps of a row-half pair share a piece
  // the grid region under the segment's footprints (cells outside the grid read as zero)
  const int cols = width + S - 1, rows = sub_rows(a.g.tile_y, S), pitch = sub_pitch(cols);
  float2* sub = (float2*)(dyn_smem() + sub_off);
  for (int i = threadIdx.x; i < rows * cols; i += NT) {
    const int r = i / cols, c = i - r * cols;
    const int gy = y0 + r, gx = x0 + c;
    sub[r * pitch + c] = (gy < a.g.n && gx < a.g.n) ? __ldg(&a.grid[(int64_t)gy * a.g.n + gx]) : make_float2(0.f, 0.f);
  }
  const int warp = threadIdx.x >> 5;
  const int os = a.g.os;
  uint4* drec = (uint4*)(dyn_smem() + rec_off);
  const bool indexed = a.index != nullptr;
  for (uint32_t c0 = s0; c0 < s1; c0 += (uint32_t)cap) {
    const int m = (int)min((uint32_t)cap, s1 - c0);
    const int kept = decode_chunk<NT, decode_per(NT)>((const uint4*)a.recs, a.index, c0, m, (uint32_t*)dyn_smem(),
                                  [&](int slot, const uint4& rec, uint32_t idx) {
      const int cls = (int)((rec.w >> 8) & 0xff) * os + (int)(rec.w & 0xff);
      const uint32_t sg = (rec.w & 0x80000000u) ? 0xbf800000u : 0x3f800000u;     // -1.0f or +1.0f
      drec[slot] = make_uint4(indexed ? idx : rec.x, sg, rec.z, (uint32_t)(cls * L::CB));
    });
    const int piece = warp / L::H, h = warp % L::H;
    const int beg = (int)((int64_t)kept * piece / kPieces), end = (int)((int64_t)kept * (piece + 1) / kPieces);
    if (L::H == 1 || staged) warp_degrid<S, T, false, NT>(tab_off, nullptr, h, sub_off, pitch, x0, y0, rec_off, beg, end, a.out);
    else warp_degrid<S, T, true, NT>(tab_off, gtab, h, sub_off, pitch, x0, y0, rec_off, beg, end, a.out);
    __syncthreads();
  }
}

template <class T, int NT>
__device__ void degrid_range(const D2Args& a, uint32_t beg, uint32_t end) {
  constexpr int kMaxSupp = NT == kDegridThreadsSmall ? kSmallMaxS : kMaxS;
  const int lane = threadIdx.x & 31;
  int64_t bin = find_bin(a.offsets, a.nbins, beg);
  uint32_t pos = beg;
  int cur_plane = -1;
  const int tab_off = kDecodeScratch;          // the decode's prefix-sum scratch comes first
  // Every warp runs this loop redundantly, once per segment, so its loads are taken off the
  // segment's critical path: lane l holds the end offsets[wb + 1 + l] of bin wb + l for a window
  // of 32 bins starting at wb (offsets[wb] <= pos), loaded before the previous segment's work.
  int64_t wb = bin;
  uint32_t wend = a.offsets[min(wb + 1 + lane, a.nbins)];
  // the values that depend only on the plane, recomputed when it changes
  int pl = -1, s = 0, sub_off = 0, rec_off = 0, cap = 0;
  bool staged = false;
  while (pos < end) {
    // the bin containing pos: the first window bin whose end exceeds pos (offsets[nbins] > pos)
    const unsigned past = __ballot_sync(0xffffffffu, wend > pos);
    if (past) {
      bin = wb + __ffs(past) - 1;
    } else {
      bin = advance_bin(a.offsets, wb + 32, a.nbins, pos);      // offsets[wb + 32] <= pos
      wb = bin;
      wend = a.offsets[min(wb + 1 + lane, a.nbins)];
    }
    // 32-bit multiply-high divisions (bins < 2^24)
    const uint32_t b32 = (uint32_t)bin;
    const int p = (int)a.g.div_ntiles.div(b32);
    const uint32_t tile = b32 - (uint32_t)p * (uint32_t)a.g.ntiles;
    const int ty = (int)a.g.div_ntx.div(tile), tx = (int)(tile - (uint32_t)ty * (uint32_t)a.g.ntx);
    if (p != pl) {
      pl = p;
      s = a.g.supp[p];
      // tables of S > 16 are staged too when they leave room for the grid region and a chunk
      const int tbytes = a.g.os * a.g.os * lay_class_bytes(s, TabElem<T>::E);
      const int sbytes = sub_bytes(a.g.tile_x, a.g.tile_y, a.group_tiles, s);
      staged = s <= kMaxStagedS || tab_off + tbytes + sbytes + kStagedChunk * (int)sizeof(Record) <= a.smem_bytes;
      sub_off = tab_off + (staged ? tbytes : 0);
      rec_off = sub_off + sbytes;
      cap = min(NT * decode_per(NT), (a.smem_bytes - rec_off) / (int)sizeof(Record));
    }
    // the segment: this bin, plus the following bins of the tile row while all their records
    // fit one chunk (ends from the window when it holds them)
    const int wo = (int)(bin - wb);
    uint32_t bound[8];
    if (wo + 8 <= 32) {
#pragma unroll
      for (int k = 0; k < 8; ++k) bound[k] = __shfl_sync(0xffffffffu, wend, wo + k);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) bound[k] = a.offsets[min(bin + k + 1, a.nbins)];
    }
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
    // the next window, loaded now and used after this segment's work (the next segment starts
    // at bin + ntiles or later when seg_end is a bin end)
    if (seg_end < end) {
      wb = bin + ntiles;
      wend = a.offsets[min(wb + 1 + lane, a.nbins)];
    }
    const bool stage = staged && p != cur_plane;
    cur_plane = staged ? p : -1;                  // an unstaged segment's grid region overwrites the table
    const int x0 = tx * a.g.tile_x, y0 = ty * a.g.tile_y;
    const int width = ntiles * a.g.tile_x;
    switch (s) {
#define WP_SEG_CASE(N)                                                                    \
  case N:                                                                                 \
    if constexpr (N <= kMaxSupp)                                                          \
      degrid_segment<N, T, NT>(a, p, stage, staged, x0, y0, width, pos, seg_end, cap, tab_off, sub_off, rec_off); \
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

template <class T, int NT>
__global__ void __launch_bounds__(NT, 1) k_degrid_v2(D2Args a) {
  for_each_unit<true>(a.offsets, a.costoff, a.nbins, a.bin_lo, a.bin_hi, a.nunits, a.work,
                      [&](uint32_t beg, uint32_t end) { degrid_range<T, NT>(a, beg, end); });
}

}  // namespace

// Dynamic shared memory of the launch, or 0 when the geometry is outside the kernel's limits
// (then the baseline kernel of grid.cu runs).
size_t degrid_v2_smem(const wp_ctx* ctx, int* group_tiles) {
  const int smax = *std::max_element(ctx->supp.begin(), ctx->supp.end());
  if (smax > kMaxS) return 0;
  if (smax > kMaxStagedS && !ctx->d_lanetab) return 0;
  const int e = ctx->prm.table_type == WP_TABLE_F32 ? 4 : 2;
  const int os = ctx->prm.oversample;
  const int tx = ctx->geo.tile_x, ty = ctx->geo.tile_y;
  if ((int64_t)tx * ty > kMaxKeys) return 0;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->prm.device) != cudaSuccess)
    return 0;
  const size_t bytes = (size_t)optin - 1024;
  int group = std::max(1, std::min(8, kMaxKeys / (tx * ty)));
  // narrow the segment groups until every plane's table, grid region and a minimal chunk fit
  for (; group >= 1; --group) {
    bool fits = true;
    for (int sp : ctx->supp) {
      const size_t need = (size_t)kDecodeScratch + (size_t)lay_staged_bytes(os, sp, e) +
                          (size_t)sub_bytes(tx, ty, group, sp) + (size_t)kMinChunk * sizeof(Record);
      if (need > bytes) fits = false;
    }
    if (fits) break;
  }
  if (group < 1) return 0;
  *group_tiles = group;
  return bytes;
}

cudaError_t launch_degrid_v2(wp_ctx* ctx, const float2* grid, float2* out, const uint32_t* index,
                             cudaStream_t s, bool* used) {
  int group = 1;
  const size_t smem = degrid_v2_smem(ctx, &group);
  *used = smem != 0;
  if (!smem) return cudaSuccess;
  D2Args a;
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
  a.out = out;
  a.index = index;
  a.smem_bytes = (int)smem;
  a.group_tiles = group;
  a.nunits = ctx->nsm * ctx->prm.units_per_cta;
  a.work = ctx->d_work + 2;
  cudaError_t e;
  if ((e = launch_bin_costs(ctx, s))) return e;
  // the planes of support <= 16 (a prefix of the bins) in the 32-warp shape, the rest in 16 warps
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
    cudaError_t err = run(small_kern, kDegridThreadsSmall, 0, split);
    if (err) return err;
    return run(large_kern, kDegridThreadsLarge, split, ctx->nbins);
  };
  switch (ctx->prm.table_type) {
    case WP_TABLE_F16: return both(k_degrid_v2<__half2, kDegridThreadsSmall>, k_degrid_v2<__half2, kDegridThreadsLarge>);
    case WP_TABLE_BF16: return both(k_degrid_v2<BfWord, kDegridThreadsSmall>, k_degrid_v2<BfWord, kDegridThreadsLarge>);
    default: return both(k_degrid_v2<float2, kDegridThreadsSmall>, k_degrid_v2<float2, kDegridThreadsLarge>);
  }
}

}  // namespace wp
