// Internal declarations of libwproj (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/wproj.h"

namespace wp {

constexpr double kCLight = 299792458.0;
constexpr double kCoordLimit = 1073741824.0;  // 2^30: |U|, |V| bound for the int32 path
constexpr int kBinSortMaxKeys = 4096;          // origins of one tile the plan's origin sort handles

// Unsigned 32-bit division by an invariant divisor d >= 1 with one multiply-high, after
// Granlund and Montgomery, "Division by invariant integers using multiplication" (PLDI 1994,
// Fig. 4.1): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
//   q = (t + ((n - t) >> s1)) >> s2,  t = umulhi(m, n),  s1 = min(l, 1), s2 = max(l - 1, 0),
// which equals floor(n / d) for every 32-bit n.
struct FastDiv {
  uint32_t d, m;
  int32_t s1, s2;
  static FastDiv make(uint32_t div) {
    FastDiv f;
    f.d = div;
    int l = 0;
    while (l < 32 && (1ull << l) < div) ++l;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - div)) / div + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
  }
#ifdef __CUDACC__
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
#endif
};

// Imaging geometry used by the coordinate and binning kernels (passed by value).
struct Geometry {
  int32_t n;            // N
  int32_t os;           // oversampling
  int32_t n_w;          // planes
  int32_t tile_x, tile_y, ntx, nty;
  int64_t ntiles;       // ntx * nty
  double os_l;          // os * (N * cell)
  double wscale;        // (Nw - 1) / w_max, 0 if Nw == 1
  const int32_t* supp;  // [Nw] device
  FastDiv div_os, div_tx, div_ty;   // divisions by os, tile_x, tile_y
  FastDiv div_ntiles, div_ntx;      // divisions of a bin index (< 2^24) by ntiles, of a tile by ntx
};

// Stored element of a WP_TABLE_BF16 kernel table: one 32-bit word per complex tap, read as
//   kr = the word shifted left by 16, as float32 (exactly kr rounded to bfloat16), and
//   ki = the whole word as float32 (its high 16 bits chosen so that, with kr's 16 bits below
//        them, the float32 value is the nearest such value to ki: within half a bfloat16 ulp).
// Both components thus carry bfloat16 precision, and a kernel widens a tap to the float32 pair
// (kr, ki) with one shift instead of two conversions.
struct __align__(4) BfWord {
  uint32_t w;
};

// One gridded (or degridded) visibility after binning: 16 bytes.
//   x, y : W*V as float bits (gridding) or the caller-order index in x (degridding)
//   z    : i0 | (j0 << 16)                      footprint origin
//   w    : ox | (oy << 8) | (conj << 31)        oversample offsets, conjugate flag
struct __align__(16) Record {
  uint32_t x, y, z, w;
};

// Host-side PSWF: Legendre coefficients gamma_k (even k) of
// t(x) = psi_0(c, x) / psi_0(c, 0) = sum_k gamma_k P_k(x).
std::vector<double> pswf_legendre_coefficients(double c);

// sum_i g[i] P_{2i}(x) for i < ncoef.
__host__ __device__ inline double legendre_even_series(const double* g, int ncoef, double x) {
  // Bonnet recurrence: P_{k+1} = ((2k+1) x P_k - k P_{k-1}) / (k+1)
  double p_prev = 1.0, p = x, sum = g[0];
  for (int k = 1; k < 2 * ncoef - 1; ++k) {
    const double p_next = ((2.0 * k + 1.0) * x * p - k * p_prev) / (k + 1.0);
    p_prev = p;
    p = p_next;
    if ((k + 1) % 2 == 0) sum += g[(k + 1) / 2] * p;
  }
  return sum;
}

struct DeviceBuffer {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace wp

struct wp_ctx {
  wp_params prm{};
  int32_t m = 0;                       // screen lattice (odd)
  int32_t nsm = 0;                     // SM count of the device
  double taper_c = 0.0;
  std::vector<int32_t> supp;           // S_p
  std::vector<double> wplane;          // w_p
  std::vector<int64_t> tab_off;        // element offset of plane p in the stored (grid-layout) table
  std::vector<int64_t> tab64_off;      // element offset of plane p in the canonical float64 table
  std::vector<int64_t> quad_off;       // element offset of plane p's quadrant table
  int64_t tab_elems = 0, tab64_elems = 0, quad_elems = 0;
  std::vector<double> legendre;        // taper coefficients (even degrees)

  // device state owned by the context
  double* d_legendre = nullptr;
  double* d_taper_img = nullptr;       // [N] t(x_i), x_i = 2 (i - N/2) / N
  float* d_taper_inv = nullptr;        // [N] 1 / t(x_i)
  double* d_taper_lat = nullptr;       // [(M+1)/2] t(x_j), j = 0 .. (M-1)/2
  double* d_cos = nullptr;             // [os M] cos(2 pi r / (os M))
  double2* d_screen = nullptr;         // [Nw][H][H] screen quadrant (j, j' >= 0)
  double2* d_stage = nullptr;          // [Nw][H][Dmax] first-axis sums
  double2* d_quad = nullptr;           // quadrant kernels, per plane [D_p][D_p], d >= 0
  double2* d_tab64 = nullptr;          // canonical float64 tables
  void* d_tab = nullptr;               // stored tables (grid layout)
  int32_t* d_supp = nullptr;
  double* d_wplane = nullptr;
  int64_t* d_tab_off = nullptr;
  void* d_lanetab = nullptr;           // lane-order tables of the planes with S > 16 (warp kernels)
  std::vector<int64_t> lanetab_off;    // byte offset per plane, -1 when the plane is staged
  int64_t* d_lanetab_off = nullptr;
  int64_t* d_tab64_off = nullptr;
  int64_t* d_quad_off = nullptr;
  double* d_nu = nullptr;
  bool have_kernels = false;

  // binning
  wp::Geometry geo{};
  int64_t nbins = 0;
  // Sub-counters per bin (2^nsub_log2; now always 1: the plan aggregates per CTA instead).
  int32_t nsub_log2 = 0;
  uint32_t* d_counts = nullptr;        // [nbins * nsub] histogram (also scratch for the work estimates)
  uint32_t* d_suboff = nullptr;        // [nbins * nsub + 1] exclusive prefix sums of the sub-counters
  uint32_t* d_offsets = nullptr;       // [nbins + 1], exclusive prefix sums, total at the end
  uint32_t* d_cursor = nullptr;        // [nbins * nsub]
  uint32_t* d_partials = nullptr;      // scan partials
  uint32_t* d_costoff = nullptr;       // [nbins + 1] exclusive prefix sums of per-bin work estimates
  uint32_t* d_partials2 = nullptr;     // scan partials of the work estimates
  uint32_t* d_work = nullptr;          // [4] work-unit counters: gridding [0..1], degridding [2..3] (zero at rest)
  double* d_chan = nullptr;            // [max_chan][2]: kx_c, kw_c
  int32_t max_chan = 0;
  wp::DeviceBuffer records;
  wp::DeviceBuffer records2;           // the origin sort's output; swapped with records after it
  wp::DeviceBuffer coord_scratch;      // wp_grid_baseline: [ngridded][8] int32 coordinates
  wp::DeviceBuffer bl_scratch;         // wp_baseline_order: row baseline indices, counts, cursors
  wp::DeviceBuffer rec_index;          // [records] uint32: visibility index | partner << 31 (wp_grid)
  wp::DeviceBuffer rec_index2;         // the origin sort's output for rec_index
  uint32_t* d_binlist = nullptr;       // [nbins] the non-empty bins (origin sort work list)
  uint32_t* d_binwork = nullptr;       // [4]: list lengths (large, other bins), next entry, finished CTAs
  wp::DeviceBuffer comp;               // [N][N] float2: rounding errors of a compensated wp_grid
  float2* comp_active = nullptr;       // set for the duration of a compensated wp_grid call
  bool have_grid_plan = false;         // records/rec_index hold the last wp_grid's binning
  int64_t plan_nrow = 0;
  int32_t plan_nchan = 0;
  unsigned long long* d_dropped = nullptr;
  double* d_wsum = nullptr;

  cufftHandle fft = 0;
  bool have_fft = false;
  std::string err;

  // tracing
  bool profiling = false;
  std::vector<cudaEvent_t> event_pool;  // free events
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> intervals;
  int64_t launches = 0;                 // own kernel launches since the last read
};

namespace wp {
// kernel tables (wkernels.cu)
cudaError_t launch_make_wkernels(wp_ctx* ctx, cudaStream_t s);
cudaError_t launch_taper_eval(const double* d_leg, int ncoef, double* out, int64_t n, int mode,
                              int32_t param, cudaStream_t s);
// coordinates and binning (plan.cu)
cudaError_t launch_channel_factors(const double* freq, int32_t nchan, double os_l, double wscale,
                                   double* d_chan, cudaStream_t s);
cudaError_t launch_plan(wp_ctx* ctx, const double* uvw, const float2* vis, const float* weight,
                        int64_t nrow, int32_t nchan, bool pairs, bool for_degrid, bool keep_index, cudaStream_t s);
// per-bin work estimate (fixed cost per non-empty bin + records x (S_p^2 + per-record cost)), scanned
cudaError_t launch_bin_costs(wp_ctx* ctx, cudaStream_t s);
cudaError_t launch_coords(wp_ctx* ctx, const double* uvw, int64_t nrow, int32_t nchan, bool pairs,
                          int32_t* out, cudaStream_t s);
// gridding / degridding (grid.cu)
cudaError_t launch_grid(wp_ctx* ctx, float2* grid, cudaStream_t s);
// register-accumulating gridding kernel (grid2.cu); *used = false when the geometry is outside its limits
cudaError_t launch_grid_v2(wp_ctx* ctx, float2* grid, cudaStream_t s, bool* used);
// shared memory the warp gridding kernel needs for ctx (0: outside its limits)
size_t grid_v2_smem(const wp_ctx* ctx, int* group_tiles);
// grid += comp (the last step of a compensated gridding call; grid2.cu)
cudaError_t launch_add_comp(float2* grid, const float2* comp, int64_t n, int nsm, cudaStream_t s);
// lane-order global tables of the planes with S > 16 (grid2.cu)
size_t lane_table_bytes(int s, int os, int table_type);
cudaError_t launch_lane_tables(wp_ctx* ctx, cudaStream_t s);
// multi-job persistent gridding (grid2.cu): per-job descriptors, then one launch over all jobs
size_t grid_job_desc_bytes();
void grid_job_desc(wp_ctx* ctx, float2* grid, size_t smem, void* out);
cudaError_t prepare_grid_batch(int table_type, size_t smem);
cudaError_t launch_grid_batch(const void* d_jobs, int njobs, uint64_t* d_jobcost, uint32_t* d_work, int table_type,
                              size_t smem, int nsm, cudaStream_t s);
// index: the gridding plan's visibility indices (degrid that plan's records), or nullptr
cudaError_t launch_degrid(wp_ctx* ctx, const float2* grid, float2* vis_out, const uint32_t* index,
                          cudaStream_t s);
// register-holding degridding kernel (degrid2.cu); *used = false when the geometry is outside its limits
cudaError_t launch_degrid_v2(wp_ctx* ctx, const float2* grid, float2* vis_out, const uint32_t* index,
                             cudaStream_t s, bool* used);
// the paper's baseline-ordered gridding, a comparison variant (baseline.cu)
cudaError_t launch_baseline_order(wp_ctx* ctx, const int32_t* ant1, const int32_t* ant2, int64_t nrow,
                                  int32_t n_ant, int32_t* bidx, uint32_t* count, uint32_t* start,
                                  uint32_t* cursor, int32_t* perm, cudaStream_t s);
cudaError_t launch_grid_baseline(wp_ctx* ctx, const int32_t* coords, const uint32_t* start, const int32_t* perm,
                                 int32_t n_ant, int32_t nchan, int64_t nrow, bool pairs, const float2* vis,
                                 const float* weight, float2* grid, cudaStream_t s);
cudaError_t launch_kept_sums(wp_ctx* ctx, const int32_t* coords, int64_t ng, int64_t nvis, const float* weight,
                             cudaStream_t s);
// the fixed scratch of wp_grid_noalloc (noalloc.cu): resolve its address on `dev` (current)
cudaError_t noalloc_prepare(int dev);
// imaging (image.cu)
cudaError_t launch_taper_inverse(const double* taper_img, float* inv, int32_t n, cudaStream_t s);
cudaError_t launch_image_pre(const float* image, const double* sum_w, const float* inv_taper, int32_t taper_correct,
                             float2* z, int32_t n, cudaStream_t s);
cudaError_t launch_checker_sign(float2* g, int32_t n, cudaStream_t s);
cudaError_t launch_image_post(const float2* spectrum, const double* sum_w, const float* inv_taper,
                              int32_t taper_correct, float* image, int32_t n, cudaStream_t s);
}  // namespace wp
