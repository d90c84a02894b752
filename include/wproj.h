/*
 * wproj.h -- C ABI of libwproj.so: W-projection gridding, degridding and imaging on one
 * NVIDIA B300 (sm_103a). After Lao et al. 2019, "Parallel Implementation of W-projection
 * Wide-Field Imaging" (the gridding step of Sec. 2.1/2.2, the IFFT to the image in the
 * Fig. 1 and Fig. 2 captions), with the W-projection kernel of the method that paper
 * parallelises (Cornwell et al. 2008, cited in Sec. 1).
 *
 * Conventions (all calls):
 *   - Every pointer documented "device" is CUDA device memory owned by the caller and must
 *     stay valid until the work on `stream` completes. The context owns its kernel tables
 *     and scratch. `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - Calls are asynchronous on `stream` unless documented otherwise; they return a
 *     WP_* status and never throw. On failure wp_last_error() describes the cause. After
 *     WP_ECUDA the context may hold partial results; other failures leave outputs untouched.
 *   - A context is not thread-safe and its scratch is shared by its calls: issue calls on
 *     one context from one host thread, on one stream at a time.
 *   - Calls that take a context make the context's device current (cudaSetDevice) and leave
 *     it current on return; they do not restore the caller's previous device.
 *   - Complex values are interleaved (re, im) float32 pairs ("float2"); arrays are C order.
 *   - Units: uvw in metres, frequencies in Hz, cell size in radians, w in wavelengths.
 *
 * Notation: N grid size, delta cell, L = N delta, du = 1/L, Nw planes, S_p full support of
 * plane p, os oversampling, M screen lattice, c = 299792458 m/s.
 */
#ifndef WPROJ_H
#define WPROJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define WP_OK        0
#define WP_EINVAL    1   /* bad argument or parameter (message says which) */
#define WP_ENOMEM    2   /* device or host allocation failed */
#define WP_ECUDA     3   /* a CUDA runtime or cuFFT call failed */
#define WP_EOVERFLOW 4   /* a size exceeds a 32-bit index the kernels use */
#define WP_ESTATE    5   /* call order: e.g. gridding before wp_make_wkernels */

/* Kernel-table precision (stored precision; generation is always float64). The gridding
 * arithmetic is float32 for every table type; only the stored taps are rounded.
 *   WP_TABLE_F32  float32 (re, im) pairs, 8 bytes per tap.
 *   WP_TABLE_F16  float16 (re, im) pairs, 4 bytes per tap.
 *   WP_TABLE_BF16 one 32-bit word w per tap, 4 bytes: re = (w << 16) read as float32 (re rounded
 *                 to bfloat16), im = w read as float32 (the float32 nearest to im among those whose
 *                 low 16 bits are re's bits). Both within half a bfloat16 ulp; a kernel widens a
 *                 tap to float32 with one shift. */
#define WP_TABLE_F32  0
#define WP_TABLE_F16  1
#define WP_TABLE_BF16 2

/* wp_grid flags. */
#define WP_ACCUMULATE      1  /* add into `grid` (and *sum_w, *n_dropped) instead of overwriting */
#define WP_HERMITIAN_PAIRS 2  /* also grid each sample as W*conj(V) at -uvw */
#define WP_KEEP_BINNING    4  /* wp_grid: keep this call's binning for wp_degrid_last (one more
                                 4-byte store per gridded visibility: its visibility index) */
#define WP_COMPENSATED     8  /* wp_grid: compensated float32 accumulation of the grid. Every
                                 addition of a footprint's partial sums into a cell returns the
                                 cell's previous value, and the exact rounding error of that
                                 float32 addition (TwoSum) is summed into a context-owned
                                 compensation grid, added to the grid at the end: the cell then
                                 carries the float32 rounding of its sum rather than the rounding
                                 errors of all its additions. Slower (the atomics return); supports
                                 up to 32 only (WP_EINVAL otherwise). */

typedef struct wp_ctx wp_ctx;

typedef struct wp_params {
  int32_t n;            /* grid and image size N (even, 16 <= N <= 32768) */
  double  cell_rad;     /* image cell size delta (rad); the field L = N*delta needs L/sqrt(2) < 1 */
  int32_t n_w;          /* number of w-planes, >= 1 (Sec. 3.1 uses 23) */
  double  w_max;        /* |w| of the last plane (wavelengths), > 0 when n_w > 1 */
  int32_t support_min;  /* full support of plane 0, taps per axis (Sec. 3.1 uses 9) */
  int32_t support_max;  /* full support of plane Nw-1; S_p = S_min + rint((S_max-S_min) p/(Nw-1)) */
  int32_t oversample;   /* os, even, 2..64 */
  int32_t screen_m;     /* odd screen lattice size M; 0 selects max(65, 4*support_max + 1) */
  int32_t table_type;   /* WP_TABLE_* */
  int32_t tile_x;       /* origin-tile width for binning (cells); 0 = default */
  int32_t tile_y;       /* origin-tile height (cells); 0 = default */
  int32_t device;       /* CUDA device ordinal */
  int32_t units_per_cta; /* schedule granularity of the gridding and degridding kernels: their
                            estimated work is cut into units_per_cta x (SM count) work units that
                            persistent CTAs take from a counter; 1..64, 0 = default (4) */
} wp_params;

/* Creates a context: validates `p`, derives the per-plane supports and w values, computes
 * the taper's Legendre coefficients on the host and its image-plane correction on the
 * device, and allocates the tables. Synchronous. *out is NULL on failure. */
int wp_create(wp_ctx** out, const wp_params* p);

/* Frees everything the context owns (synchronises its device first). NULL is a no-op. */
void wp_destroy(wp_ctx* ctx);

/* Message of the last failure on this context ("" if none). Valid until the next call.
 * With ctx == NULL: the last wp_create failure of the calling thread. */
const char* wp_last_error(const wp_ctx* ctx);

/* Builds the oversampled W-kernel of every plane, in float64, then stores it in the
 * table precision (W-projection kernel: the method of Cornwell et al. 2008, Sec. 1):
 *   screen  s_p(l_k, m_q) = t(x_k) t(x_q) exp(2 pi i w_p (n - 1)),  n = sqrt(1 - l^2 - m^2)
 *           j = k - (M-1)/2, l_k = j L/M, x_k = 2 j/M, t = PSWF psi_0(c = pi S_min/2) / psi_0(0)
 *   kernel  K_p(dx, dy) = (1/nu) sum_{k,q} s_p exp(-2 pi i (dx j_k + dy j_q)/(os M)),
 *           dx, dy in (-S_p os/2, S_p os/2], w_p = p w_max/(Nw-1),
 *           nu = Re sum of plane 0's taps at whole-cell offsets (dx, dy = 0 mod os).
 * Must precede wp_grid / wp_degrid. Errors: WP_ECUDA. */
int wp_make_wkernels(wp_ctx* ctx, void* stream);

/* Convolutional gridding (Sec. 2.1 gridding loop; Sec. 2.2: C_full^2 taps per visibility):
 * for every kept visibility k of row r, channel c (and its Hermitian partner if flagged):
 *   U = rint(u * kx_c), V = rint(v * kx_c), kx_c = (f_c/c) * (os * (N*delta))   [float64]
 *   p = min(Nw-1, rint(|w| * kw_c)), kw_c = (f_c/c) * ((Nw-1)/w_max), conj = (w < 0)
 *   X = U + (N/2) os, i0 = floor((X - S_p os/2)/os) + 1, ox = i0 os - X + S_p os/2 - 1
 *   grid[j0+b][i0+a] += W V * K_p[b os + oy - S_p os/2 + 1][a os + ox - S_p os/2 + 1]
 *     (K_p conjugated when conj), a, b in [0, S_p).
 * A visibility is dropped (and counted) if its footprint leaves [0, N)^2 or its
 * coordinates are not finite or |U|, |V| >= 2^30. The Hermitian partner uses -uvw and
 * W conj(V). The visibilities are binned by (plane, footprint-origin tile) with a counting
 * sort (histogram, exclusive prefix sum, scatter: the start-index construction of Eq. 6).
 *   uvw      device [nrow][3] float64 metres        freq   device [nchan] float64 Hz
 *   vis      device [nrow][nchan] float2            weight device [nrow][nchan] float32, or NULL (all 1)
 *   grid     device [N][N] float2 (row = v, column = u); zeroed first unless WP_ACCUMULATE
 *   sum_w    device float64, or NULL: receives (adds, with WP_ACCUMULATE) sum of kept weights
 *   n_dropped device int64, or NULL: receives (adds) the number of dropped gridded visibilities
 * Errors: WP_EINVAL (sizes, NULL pointers), WP_ESTATE (no kernels), WP_ENOMEM (scratch),
 * WP_EOVERFLOW (more than 2^31 - 1 gridded visibilities), WP_ECUDA. */
int wp_grid(wp_ctx* ctx, const double* uvw, const double* freq, const void* vis,
            const float* weight, int64_t nrow, int32_t nchan, int32_t flags, void* grid,
            double* sum_w, int64_t* n_dropped, void* stream);

/* Gridding without any device allocation during the call. The paper has no counterpart;
 * this is a service for callers that cannot allocate device memory while they grid: for
 * example a host program whose framework has already reserved the whole device for its own
 * memory pool (a cudaMalloc from inside the library would fail or fragment that pool), or a
 * latency-bound ingest loop in which a device allocation, which may synchronise the device
 * and take milliseconds, is not acceptable. Such a caller creates the context and builds the
 * kernels once beforehand (wp_create and wp_make_wkernels do allocate) and then calls this.
 *
 * Same arguments, flags, results and errors as wp_grid, computed by the same kernels. The
 * per-call scratch that wp_grid keeps in growable context buffers (two 16-byte records per
 * gridded visibility: binned, then sorted by footprint origin; plus per-channel factors) is
 * instead a fixed file-scope device array of 32 MiB + 64 KiB, which every GPU that loads this
 * library holds until the process exits.
 * Limits: at most 2^20 = 1048576 gridded visibilities per call (nrow * nchan, doubled with
 * WP_HERMITIAN_PAIRS) and at most 4096 channels; larger calls return WP_EINVAL with a
 * message and touch nothing. The call allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.
 *
 * wp_create looks up the array's device address (cudaGetSymbolAddress, with the context's
 * device current), which also loads the array on that device, and caches it per device, so
 * this call itself neither loads nor looks up anything on a device that has a context. The
 * cache does not survive cudaDeviceReset: contexts made before a reset are unusable after it,
 * and the next wp_create on that device resolves the address again. All calls, from every context on the device, share the one array, and it keeps the last
 * call's contents (each call writes every record it reads, so nothing in it needs to start
 * at zero): calls that overlap on the GPU (different streams, or different contexts on the
 * same device, in flight at the same time) race on it and must be serialised by the caller.
 * The context's own bin counters are also shared with its other calls, as for wp_grid. */
int wp_grid_noalloc(wp_ctx* ctx, const double* uvw, const double* freq, const void* vis,
                    const float* weight, int64_t nrow, int32_t nchan, int32_t flags, void* grid,
                    double* sum_w, int64_t* n_dropped, void* stream);

/* ---- the paper's baseline-ordered GPU gridding (a comparison variant) ---- */

/* Rows grouped by baseline and time-ordered within each (Sec. 2.2): the baseline index of Eq. 5,
 *   I_B = (-S^2 + 2 S N_ant + S)/2 + |I_ant1 - I_ant2|,  S = min(I_ant1, I_ant2)
 * (autocorrelations counted, so I_B < N_ant (N_ant + 1)/2), the sample count C of every baseline
 * and the start indices of Eq. 6 (exclusive prefix sums of C).
 *   ant1, ant2 device [nrow] int32 antenna IDs in [0, n_ant); rows in time order (row index).
 *   perm_out  device [nrow] int32: row indices, baseline after baseline, rising within one.
 *   start_out device [N_ant (N_ant + 1)/2 + 1] uint32: Eq. 6, the row total at the end.
 * Baselines of more than 4096 rows keep the order of an atomic scatter (still grouped).
 * A row with an antenna ID outside [0, n_ant) belongs to no baseline: such rows fill
 * perm_out after start_out[N_B] (in any order), so start_out[N_B] < nrow shows them.
 * Errors: WP_EINVAL, WP_ENOMEM, WP_ECUDA. */
int wp_baseline_order(wp_ctx* ctx, const int32_t* ant1, const int32_t* ant2, int64_t nrow, int32_t n_ant,
                      int32_t* perm_out, uint32_t* start_out, void* stream);

/* Gridding in the paper's GPU scheme (Sec. 2.2, Fig. 2): one thread block per (baseline, channel
 * [, Hermitian partner]) and one thread per support tap; along the baseline's time samples a
 * thread keeps its tap's sum in a register while the grid point stays the same and adds it to
 * the grid atomically when the point moves. Same arguments and results as wp_grid (same float64
 * coordinates), plus perm and start from wp_baseline_order; rows outside every baseline's
 * range are not gridded (their weights still enter sum_w), entries of perm outside [0, nrow)
 * are skipped. Supports up to 32. A comparison variant: wp_grid is the fast path. Errors as
 * wp_grid, and WP_EINVAL for a support above 32. */
int wp_grid_baseline(wp_ctx* ctx, const double* uvw, const double* freq, const void* vis, const float* weight,
                     const int32_t* perm, const uint32_t* start, int32_t n_ant, int64_t nrow, int32_t nchan,
                     int32_t flags, void* grid, double* sum_w, int64_t* n_dropped, void* stream);

/* ---- many gridding jobs in one launch ---- */

/* One gridding job: the arguments of one wp_grid call. Each job has its own context (its own
 * geometry, kernel tables and binning); all contexts on one device, no context twice. */
typedef struct wp_job {
  wp_ctx* ctx;
  const double* uvw;     /* device [nrow][3] */
  const double* freq;    /* device [nchan] */
  const void* vis;       /* device [nrow][nchan] float2 */
  const float* weight;   /* device [nrow][nchan] or NULL */
  int64_t nrow;
  int32_t nchan;
  int32_t flags;         /* WP_ACCUMULATE | WP_HERMITIAN_PAIRS */
  void* grid;            /* device [N][N] float2 of the job's context */
  double* sum_w;         /* device, or NULL */
  int64_t* n_dropped;    /* device, or NULL */
} wp_job;

typedef struct wp_batch wp_batch;

/* A batch of gridding jobs (imaging jobs of different visibility counts, grid sizes, supports,
 * oversampling and plane counts). Creation validates the jobs, allocates every per-job scratch
 * buffer and the batch's descriptors, and fixes the job table: the pointers and sizes are read
 * once, the data behind them is read at every wp_batch_grid. Each job's context must have its
 * kernel tables (wp_make_wkernels). Synchronous. Errors: WP_EINVAL (bad job, shared context,
 * mixed devices), WP_ESTATE, WP_ENOMEM, WP_ECUDA; the message is in the failing job's context. */
int wp_batch_create(const wp_job* jobs, int32_t njobs, wp_batch** out);

/* Grids every job of the batch, with the results of calling wp_grid on each: the jobs'
 * coordinates and binning (per-job launches), then ONE persistent launch of the warp gridding
 * kernel over the work of all jobs whose geometry it takes and whose table type is that of the
 * first such job (the other jobs run the baseline kernel one by one). Makes no allocation and
 * no host synchronisation, so a stream capture of it replays as a CUDA graph. Errors: WP_ECUDA. */
int wp_batch_grid(wp_batch* batch, void* stream);

/* Number of jobs in the batch's persistent launch. */
int32_t wp_batch_fused_jobs(const wp_batch* batch);

/* Frees the batch (not the jobs' contexts or buffers). */
void wp_batch_destroy(wp_batch* batch);

/* Degridding, the adjoint of wp_grid with unit weights (Sec. 2 names gridding and
 * degridding as the pair being accelerated):
 *   vis_out[r][c] = sum_{a,b} grid[j0+b][i0+a] * conj(K_k[...])   (same coordinates and taps;
 *   K_k = K_p or conj(K_p) for w < 0); dropped visibilities get 0.
 *   grid device [N][N] float2 (read only); vis_out device [nrow][nchan] float2 (overwritten).
 * Errors as wp_grid. */
int wp_degrid(wp_ctx* ctx, const double* uvw, const double* freq, const void* grid,
              int64_t nrow, int32_t nchan, void* vis_out, void* stream);

/* Degridding of the visibilities of this context's most recent wp_grid call, reusing that
 * call's coordinates and binning instead of computing them again (in an imaging loop the same
 * visibilities are gridded and degridded every cycle). The result is the one wp_degrid gives
 * for that call's uvw, freq, nrow and nchan, element for element: the Hermitian partners that
 * wp_grid added are skipped, dropped visibilities get 0.
 *   grid device [N][N] float2 (read only); vis_out device [nrow][nchan] float2 (overwritten),
 *   nrow and nchan those of the wp_grid call.
 * That wp_grid call must pass WP_KEEP_BINNING. The binning stays valid until the context's next
 * wp_grid, wp_grid_noalloc or wp_degrid.
 * Errors: WP_ESTATE when there is no such wp_grid call (none yet, one without WP_KEEP_BINNING,
 * or a later wp_degrid or wp_grid_noalloc replaced its binning); WP_EINVAL, WP_ECUDA. */
int wp_degrid_last(wp_ctx* ctx, const void* grid, void* vis_out, void* stream);

/* Dirty image from the grid (the IFFT of Fig. 1 / Fig. 2) with the taper correction:
 *   I[j][i] = Re sum_{h,g} G[h][g] exp(+2 pi i ((g-N/2)(i-N/2) + (h-N/2)(j-N/2))/N)
 *             / (sum_w * t(x_i) t(x_j)),  x_i = 2 (i - N/2)/N   (no t factor if !taper_correct)
 *   grid  device [N][N] float2, CLOBBERED (used as the in-place FFT buffer)
 *   sum_w device float64 (e.g. as written by wp_grid)
 *   image device [N][N] float32 (row = m, column = l)
 * Uses one cuFFT C2C plan owned by the context. Errors: WP_EINVAL, WP_ECUDA. */
int wp_fft_to_image(wp_ctx* ctx, void* grid, const double* sum_w, int32_t taper_correct,
                    float* image, void* stream);

/* The adjoint of wp_fft_to_image (image -> grid), the first half of the forward model
 * image -> grid -> visibilities whose second half is wp_degrid:
 *   grid[h][g] = sum_{j,i} X[j][i] exp(-2 pi i ((g-N/2)(i-N/2) + (h-N/2)(j-N/2))/N),
 *   X[j][i] = image[j][i] / (sum_w * t(x_i) t(x_j))   (no t factor if !taper_correct),
 * so that <wp_fft_to_image(G), image> = Re <G, wp_image_to_grid(image)> for real images.
 *   image device [N][N] float32 (read only); sum_w device float64, or NULL for 1;
 *   grid  device [N][N] float2 (overwritten; the in-place FFT buffer).
 * Uses the context's cuFFT plan. Errors: WP_EINVAL, WP_ECUDA. */
int wp_image_to_grid(wp_ctx* ctx, const float* image, const double* sum_w, int32_t taper_correct,
                     void* grid, void* stream);

/* ---- inspection and tracing ---- */

/* Per-plane full support S_p and w_p (host memory, Nw entries each). Synchronous. */
int wp_plane_info(const wp_ctx* ctx, int32_t* support_out, double* w_out);

/* The float64 coordinate step of wp_grid alone. For each gridded visibility
 * (k = r*nchan + c, then the Hermitian partners at k + nrow*nchan if flagged) writes 8
 * int32: U, V, plane, conj, keep, i0, j0, ox | (oy << 16); i0, j0, ox and oy are defined for
 * kept visibilities only.
 *   out device [ngridded][8] int32. Errors: WP_EINVAL, WP_ECUDA. */
int wp_coords(wp_ctx* ctx, const double* uvw, const double* freq, int64_t nrow, int32_t nchan,
              int32_t flags, int32_t* out, void* stream);

/* Copies plane p's kernel to HOST memory in the canonical layout [ey][ex], ey, ex in
 * [0, S_p os), offset d = e - S_p os/2 + 1: as float64 pairs (which = 0: the float64
 * table before storage) or as float32 pairs of the stored values (which = 1).
 * cap = capacity of out in complex elements (>= (S_p os)^2). Synchronous. */
int wp_wkernel_export(wp_ctx* ctx, int32_t plane, int32_t which, void* out_host, int64_t cap);

/* Normalisation nu of the last wp_make_wkernels (host double). Synchronous. */
int wp_wkernel_norm(wp_ctx* ctx, double* nu_out);

/* Phases reported by wp_profile_read (index into its output arrays). */
#define WP_PHASE_WKERNELS 0  /* wp_make_wkernels */
#define WP_PHASE_PLAN     1  /* coordinates, histogram, prefix sum, scatter (wp_grid / wp_degrid) */
#define WP_PHASE_GRID     2  /* the gridding kernel */
#define WP_PHASE_DEGRID   3  /* the degridding kernel */
#define WP_PHASE_FFT      4  /* cuFFT inverse transform */
#define WP_PHASE_IMAGE    5  /* image epilogue (shift, sign, weight and taper division) */
#define WP_NPHASES        6

/* Tracing: with enable != 0 the context records a CUDA event pair on the call's stream
 * around each phase of every later call, and counts its own kernel launches. Events are
 * only recorded, never waited on, so enabling adds no synchronisation. */
int wp_profile(wp_ctx* ctx, int32_t enable);

/* Waits for the recorded events, then writes per phase (WP_NPHASES entries, host arrays)
 * the summed elapsed milliseconds and the number of timed intervals since the last read,
 * and the number of this library's kernel launches since the last read; resets all three.
 * Any output pointer may be NULL. Synchronous. */
int wp_profile_read(wp_ctx* ctx, double* ms_out, int32_t* count_out, int64_t* launches_out);

/* Measurement aid (no counterpart in the paper): the device's FP32 FMA throughput, the
 * compute bound of the gridding roofline (8 flop per kernel tap). Runs `reps` timed launches
 * (after one warm-up launch) of a kernel whose threads each run 16 independent FMA chains of
 * `iters` steps, as scalar fma.rn.f32 (packed == 0) or packed fma.rn.f32x2 (packed != 0, the
 * form the gridding kernels issue), on every SM at full occupancy, on the legacy default
 * stream. Writes TFLOP/s (2 flop per FMA) to *tflops_out and the mean launch time in ms to
 * *ms_out (may be NULL). Synchronous; allocates 8 bytes of device memory for the duration.
 * Errors: WP_EINVAL (iters or reps < 1, NULL tflops_out, no such device), WP_ECUDA. */
int wp_probe_fp32_fma(int32_t device, int32_t packed, int64_t iters, int32_t reps, double* tflops_out,
                      double* ms_out);

/* Host only (no device needed): the taper t(x) = psi_0(c, x) / psi_0(c, 0) that
 * wp_make_wkernels and wp_fft_to_image use, at n points |x| <= 1 (host arrays).
 * psi_0 from its Legendre expansion (eigenvector of the prolate operator in the Legendre
 * basis, Xiao, Rokhlin & Yarvin 2001). Errors: WP_EINVAL (c <= 0, |x| > 1, NULL). */
int wp_taper_eval_host(double c, const double* x, int64_t n, double* out);

#ifdef __cplusplus
}
#endif

#endif /* WPROJ_H */
