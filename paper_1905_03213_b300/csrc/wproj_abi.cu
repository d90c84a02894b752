// C ABI of libwproj (declared in include/wproj.h): argument checking, context state,
// scratch management, tracing and the order of launches. No arithmetic of the method
// lives here except the host-side parameter derivations (per-plane support and w, the
// channel factors' inputs, the taper's Legendre coefficients).
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <memory>
#include <string>

#include "internal.h"

using wp::DeviceBuffer;

namespace {

thread_local std::string g_create_error;

int fail(wp_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(wp_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, WP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define WP_CUDA(ctx, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * count);
}

int ensure_buffer(wp_ctx* ctx, DeviceBuffer& b, size_t bytes, const char* what) {
  if (b.bytes >= bytes) return WP_OK;
  if (b.ptr) {
    cudaError_t e = cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    if (e) return cuda_fail(ctx, e, "cudaFree");
  }
  if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.ptr = nullptr;
    return fail(ctx, WP_ENOMEM, std::string("cannot allocate ") + std::to_string(bytes) + " bytes of " + what);
  }
  b.bytes = bytes;
  return WP_OK;
}

int ensure_channels(wp_ctx* ctx, int32_t nchan) {
  if (nchan <= ctx->max_chan) return WP_OK;
  if (ctx->d_chan) cudaFree(ctx->d_chan);
  ctx->d_chan = nullptr;
  ctx->max_chan = 0;
  if (dalloc(&ctx->d_chan, 2 * (size_t)nchan) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, WP_ENOMEM, "cannot allocate channel factors");
  }
  ctx->max_chan = nchan;
  return WP_OK;
}

int check_vis_args(wp_ctx* ctx, const double* uvw, const double* freq, int64_t nrow, int32_t nchan, int pairs) {
  if (!ctx) return WP_EINVAL;
  if (nrow < 0 || nchan < 1) return fail(ctx, WP_EINVAL, "nrow must be >= 0 and nchan >= 1");
  if (nrow > 0 && (!uvw || !freq)) return fail(ctx, WP_EINVAL, "uvw and freq must not be NULL");
  const int64_t lim = (int64_t)0x7fffffff;
  if (nrow > lim / nchan || nrow * nchan * (pairs ? 2 : 1) > lim)
    return fail(ctx, WP_EOVERFLOW, "more than 2^31 - 1 gridded visibilities in one call");
  return WP_OK;
}

cudaEvent_t take_event(wp_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Records a CUDA event pair around one phase of a call when tracing is on.
struct Phase {
  wp_ctx* ctx;
  int id;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Phase(wp_ctx* c, int phase, cudaStream_t st) : ctx(c), id(phase), s(st) {
    if (ctx->profiling && (a = take_event(ctx))) cudaEventRecord(a, s);
  }
  ~Phase() {
    if (!a) return;
    cudaEvent_t b = take_event(ctx);
    if (!b) {
      ctx->event_pool.push_back(a);
      return;
    }
    cudaEventRecord(b, s);
    ctx->intervals.push_back({id, {a, b}});
  }
};

__global__ void k_store_scalars(const double* wsum, const unsigned long long* dropped, double* sum_w,
                                long long* n_dropped, int accumulate) {
  if (sum_w) *sum_w = accumulate ? *sum_w + *wsum : *wsum;
  if (n_dropped) *n_dropped = accumulate ? *n_dropped + (long long)*dropped : (long long)*dropped;
}

int prepare_vis_call(wp_ctx* ctx, const double* uvw, const double* freq, int64_t nrow, int32_t nchan, int pairs,
                     bool want_index, cudaStream_t s) {
  int rc = check_vis_args(ctx, uvw, freq, nrow, nchan, pairs);
  if (rc) return rc;
  if (!ctx->have_kernels) return fail(ctx, WP_ESTATE, "wp_make_wkernels has not been called");
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  if ((rc = ensure_channels(ctx, nchan))) return rc;
  const size_t ng = (size_t)nrow * nchan * (pairs ? 2 : 1);
  if ((rc = ensure_buffer(ctx, ctx->records, std::max<size_t>(ng, 1) * sizeof(wp::Record), "records"))) return rc;
  if ((rc = ensure_buffer(ctx, ctx->records2, std::max<size_t>(ng, 1) * sizeof(wp::Record), "sorted records"))) return rc;
  if (want_index && (rc = ensure_buffer(ctx, ctx->rec_index, std::max<size_t>(ng, 1) * 4, "record indices"))) return rc;
  if (want_index && (rc = ensure_buffer(ctx, ctx->rec_index2, std::max<size_t>(ng, 1) * 4, "sorted record indices"))) return rc;
  ctx->have_grid_plan = false;          // the records are about to be replaced
  if (nrow > 0) {
    WP_CUDA(ctx, wp::launch_channel_factors(freq, nchan, ctx->geo.os_l, ctx->geo.wscale, ctx->d_chan, s));
    ++ctx->launches;
  }
  return WP_OK;
}

float half_to_float(uint16_t h) {
  const uint32_t sign = (uint32_t)(h & 0x8000) << 16;
  int exp = (h >> 10) & 0x1f;
  uint32_t man = h & 0x3ff, bits;
  if (exp == 0) {
    if (man == 0) {
      bits = sign;
    } else {  // subnormal: normalise
      exp = 1;
      while (!(man & 0x400)) {
        man <<= 1;
        --exp;
      }
      man &= 0x3ff;
      bits = sign | ((uint32_t)(exp + 112) << 23) | (man << 13);
    }
  } else if (exp == 31) {
    bits = sign | 0x7f800000u | (man << 13);
  } else {
    bits = sign | ((uint32_t)(exp + 112) << 23) | (man << 13);
  }
  float f;
  std::memcpy(&f, &bits, 4);
  return f;
}

}  // namespace

extern "C" {

const char* wp_last_error(const wp_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void wp_destroy(wp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->prm.device);
  cudaDeviceSynchronize();
  if (ctx->have_fft) cufftDestroy(ctx->fft);
  for (auto& it : ctx->intervals) {
    cudaEventDestroy(it.second.first);
    cudaEventDestroy(it.second.second);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  void* ptrs[] = {ctx->d_legendre, ctx->d_taper_img, ctx->d_taper_inv, ctx->d_taper_lat, ctx->d_cos,      ctx->d_screen,
                  ctx->d_stage,    ctx->d_quad,      ctx->d_tab64,     ctx->d_tab,      ctx->d_supp,
                  ctx->d_wplane,   ctx->d_tab_off,   ctx->d_tab64_off, ctx->d_quad_off, ctx->d_nu,
                  ctx->d_counts,   ctx->d_offsets,   ctx->d_cursor,    ctx->d_partials, ctx->d_chan,
                  ctx->records.ptr, ctx->d_dropped,  ctx->d_wsum,     ctx->d_costoff,  ctx->d_partials2, ctx->d_work, ctx->rec_index.ptr, ctx->d_suboff, ctx->d_lanetab, ctx->d_lanetab_off,
                  ctx->coord_scratch.ptr, ctx->bl_scratch.ptr, ctx->records2.ptr, ctx->rec_index2.ptr, ctx->comp.ptr,
                  ctx->d_binlist, ctx->d_binwork};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete ctx;
}

int wp_create(wp_ctx** out, const wp_params* p) {
  if (!out) return fail(nullptr, WP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p) return fail(nullptr, WP_EINVAL, "params is NULL");
  const wp_params& q = *p;
  if (q.n < 16 || q.n > 32768 || (q.n & 1)) return fail(nullptr, WP_EINVAL, "n must be even, 16..32768");
  if (!(q.cell_rad > 0.0) || !std::isfinite(q.cell_rad)) return fail(nullptr, WP_EINVAL, "cell_rad must be > 0");
  const double field = (double)q.n * q.cell_rad;
  if (!(0.5 * field * std::sqrt(2.0) < 1.0)) return fail(nullptr, WP_EINVAL, "field too wide (L/sqrt(2) >= 1)");
  if (q.n_w < 1 || q.n_w > 4096) return fail(nullptr, WP_EINVAL, "n_w must be 1..4096");
  if (q.n_w > 1 && !(q.w_max > 0.0 && std::isfinite(q.w_max)))
    return fail(nullptr, WP_EINVAL, "w_max must be finite and > 0 when n_w > 1");
  if (q.oversample < 2 || q.oversample > 64 || (q.oversample & 1))
    return fail(nullptr, WP_EINVAL, "oversample must be even, 2..64");
  if (q.support_min < 1 || q.support_max < q.support_min || q.support_max > 64)
    return fail(nullptr, WP_EINVAL, "need 1 <= support_min <= support_max <= 64");
  if (q.support_max >= q.n) return fail(nullptr, WP_EINVAL, "support_max must be < n");
  if (q.screen_m != 0 && (q.screen_m < 3 || !(q.screen_m & 1) || q.screen_m > 4097))
    return fail(nullptr, WP_EINVAL, "screen_m must be 0 or odd in 3..4097");
  if (q.table_type < WP_TABLE_F32 || q.table_type > WP_TABLE_BF16)
    return fail(nullptr, WP_EINVAL, "table_type must be WP_TABLE_F32, _F16 or _BF16");
  if (q.tile_x < 0 || q.tile_y < 0 || q.tile_x > 1024 || q.tile_y > 1024)
    return fail(nullptr, WP_EINVAL, "tile sizes must be 0 (default) or 1..1024");
  if (q.units_per_cta < 0 || q.units_per_cta > 64)
    return fail(nullptr, WP_EINVAL, "units_per_cta must be 0 (default) or 1..64");

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || q.device < 0 || q.device >= ndev) {
    cudaGetLastError();
    return fail(nullptr, WP_EINVAL, "no such CUDA device");
  }
  wp_ctx* ctx = new (std::nothrow) wp_ctx();
  if (!ctx) return fail(nullptr, WP_ENOMEM, "host allocation failed");
  ctx->prm = q;
  if (ctx->prm.tile_x == 0) ctx->prm.tile_x = 32;
  if (ctx->prm.tile_y == 0) ctx->prm.tile_y = 32;
  if (ctx->prm.units_per_cta == 0) ctx->prm.units_per_cta = 4;
  ctx->m = q.screen_m ? q.screen_m : std::max(65, 4 * q.support_max + 1);
  auto bail = [&](int code, const std::string& msg) {
    g_create_error = msg;
    wp_destroy(ctx);
    return code;
  };
  if (cudaSetDevice(q.device) != cudaSuccess) return bail(WP_ECUDA, "cudaSetDevice failed");
  // the fixed scratch of wp_grid_noalloc is taken here, not inside that call
  if (wp::noalloc_prepare(q.device) != cudaSuccess) return bail(WP_ECUDA, "wp_grid_noalloc scratch set-up failed");
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, q.device) != cudaSuccess) return bail(WP_ECUDA, "cudaGetDeviceProperties failed");
  ctx->nsm = prop.multiProcessorCount;

  // per-plane support and w (the float64 expressions documented in wproj.h)
  ctx->supp.resize(q.n_w);
  ctx->wplane.resize(q.n_w);
  for (int i = 0; i < q.n_w; ++i) {
    if (q.n_w == 1) {
      ctx->supp[i] = q.support_min;
      ctx->wplane[i] = 0.0;
    } else {
      ctx->supp[i] = q.support_min + (int32_t)std::nearbyint((double)(q.support_max - q.support_min) * i / (q.n_w - 1));
      ctx->wplane[i] = (double)i * (q.w_max / (q.n_w - 1));
    }
    if ((ctx->supp[i] * q.oversample) % 2) return bail(WP_EINVAL, "support * oversample must be even");
  }
  int64_t acc = 0, accq = 0;
  for (int i = 0; i < q.n_w; ++i) {
    const int64_t e = (int64_t)ctx->supp[i] * q.oversample;
    const int64_t dp = e / 2 + 1;
    ctx->tab_off.push_back(acc);
    ctx->tab64_off.push_back(acc);
    ctx->quad_off.push_back(accq);
    acc += e * e;
    accq += dp * dp;
  }
  ctx->tab_elems = acc;
  ctx->tab64_elems = acc;
  int64_t lane_bytes = 0;                 // lane-order tables of the planes with S > 16
  for (int i = 0; i < q.n_w; ++i) {
    const size_t b = wp::lane_table_bytes(ctx->supp[i], q.oversample, q.table_type);
    ctx->lanetab_off.push_back(b ? lane_bytes : -1);
    lane_bytes += (int64_t)((b + 255) & ~(size_t)255);
  }
  ctx->quad_elems = accq;
  ctx->taper_c = M_PI * q.support_min / 2.0;
  ctx->legendre = wp::pswf_legendre_coefficients(ctx->taper_c);

  // geometry for binning
  wp::Geometry& g = ctx->geo;
  g.n = q.n;
  g.os = q.oversample;
  g.n_w = q.n_w;
  g.tile_x = ctx->prm.tile_x;
  g.tile_y = ctx->prm.tile_y;
  g.ntx = (q.n + g.tile_x - 1) / g.tile_x;
  g.nty = (q.n + g.tile_y - 1) / g.tile_y;
  g.ntiles = (int64_t)g.ntx * g.nty;
  g.div_os = wp::FastDiv::make((uint32_t)g.os);
  g.div_tx = wp::FastDiv::make((uint32_t)g.tile_x);
  g.div_ty = wp::FastDiv::make((uint32_t)g.tile_y);
  g.div_ntiles = wp::FastDiv::make((uint32_t)g.ntiles);
  g.div_ntx = wp::FastDiv::make((uint32_t)g.ntx);
  g.os_l = (double)q.oversample * ((double)q.n * q.cell_rad);
  g.wscale = q.n_w > 1 ? (double)(q.n_w - 1) / q.w_max : 0.0;
  ctx->nbins = g.ntiles * q.n_w;
  if (ctx->nbins > (int64_t)4096 * 4096) return bail(WP_EINVAL, "too many bins (n_w * tiles > 2^24): use larger tiles");
  // one counter per bin: the plan's histogram and scatter aggregate each CTA's records per bin in
  // shared memory before their global atomics, so a dense bin's counter sees one atomic per CTA
  ctx->nsub_log2 = 0;
  const int64_t nsubbins = ctx->nbins << ctx->nsub_log2;
  const int64_t scan_tiles = (nsubbins + 4095) / 4096;

  const int h = (ctx->m + 1) / 2;
  int dmax = 0;
  for (int i = 0; i < q.n_w; ++i) dmax = std::max(dmax, ctx->supp[i] * q.oversample / 2 + 1);
  const size_t tab_bytes = (q.table_type == WP_TABLE_F32 ? 8 : 4) * (size_t)ctx->tab_elems;
  bool ok = (lane_bytes == 0 || (cudaMalloc(&ctx->d_lanetab, (size_t)lane_bytes) == cudaSuccess &&
                                  dalloc(&ctx->d_lanetab_off, (size_t)q.n_w) == cudaSuccess &&
                                  cudaMemcpy(ctx->d_lanetab_off, ctx->lanetab_off.data(), sizeof(int64_t) * q.n_w,
                                             cudaMemcpyHostToDevice) == cudaSuccess)) &&
            dalloc(&ctx->d_legendre, ctx->legendre.size()) == cudaSuccess &&
            dalloc(&ctx->d_taper_img, (size_t)q.n) == cudaSuccess && dalloc(&ctx->d_taper_inv, (size_t)q.n) == cudaSuccess && dalloc(&ctx->d_taper_lat, (size_t)h) == cudaSuccess &&
            dalloc(&ctx->d_cos, (size_t)q.oversample * ctx->m) == cudaSuccess &&
            dalloc(&ctx->d_screen, (size_t)q.n_w * h * h) == cudaSuccess &&
            dalloc(&ctx->d_stage, (size_t)q.n_w * h * dmax) == cudaSuccess &&
            dalloc(&ctx->d_quad, (size_t)ctx->quad_elems) == cudaSuccess &&
            dalloc(&ctx->d_tab64, (size_t)ctx->tab64_elems) == cudaSuccess &&
            cudaMalloc(&ctx->d_tab, tab_bytes) == cudaSuccess && dalloc(&ctx->d_supp, (size_t)q.n_w) == cudaSuccess &&
            dalloc(&ctx->d_wplane, (size_t)q.n_w) == cudaSuccess &&
            dalloc(&ctx->d_tab_off, (size_t)q.n_w) == cudaSuccess &&
            dalloc(&ctx->d_tab64_off, (size_t)q.n_w) == cudaSuccess &&
            dalloc(&ctx->d_quad_off, (size_t)q.n_w) == cudaSuccess && dalloc(&ctx->d_nu, 1) == cudaSuccess &&
            dalloc(&ctx->d_counts, (size_t)nsubbins) == cudaSuccess &&
            dalloc(&ctx->d_suboff, (size_t)nsubbins + 1) == cudaSuccess &&
            dalloc(&ctx->d_offsets, (size_t)ctx->nbins + 1) == cudaSuccess &&
            dalloc(&ctx->d_cursor, (size_t)nsubbins) == cudaSuccess &&
            dalloc(&ctx->d_partials, (size_t)scan_tiles + 1) == cudaSuccess &&
            dalloc(&ctx->d_costoff, (size_t)ctx->nbins + 1) == cudaSuccess &&
            dalloc(&ctx->d_partials2, (size_t)scan_tiles + 1) == cudaSuccess &&
            dalloc(&ctx->d_work, 4) == cudaSuccess && cudaMemset(ctx->d_work, 0, 4 * sizeof(uint32_t)) == cudaSuccess &&
            dalloc(&ctx->d_binlist, (size_t)ctx->nbins) == cudaSuccess && dalloc(&ctx->d_binwork, 4) == cudaSuccess &&
            cudaMemset(ctx->d_binwork, 0, 4 * sizeof(uint32_t)) == cudaSuccess &&
            dalloc(&ctx->d_dropped, 1) == cudaSuccess && dalloc(&ctx->d_wsum, 1) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return bail(WP_ENOMEM, "device allocation failed in wp_create");
  }
  g.supp = ctx->d_supp;
  ok = cudaMemcpy(ctx->d_legendre, ctx->legendre.data(), sizeof(double) * ctx->legendre.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(ctx->d_supp, ctx->supp.data(), sizeof(int32_t) * q.n_w, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(ctx->d_wplane, ctx->wplane.data(), sizeof(double) * q.n_w, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(ctx->d_tab_off, ctx->tab_off.data(), sizeof(int64_t) * q.n_w, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(ctx->d_tab64_off, ctx->tab64_off.data(), sizeof(int64_t) * q.n_w, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(ctx->d_quad_off, ctx->quad_off.data(), sizeof(int64_t) * q.n_w, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) return bail(WP_ECUDA, "upload of context tables failed");
  const int ncoef = (int)ctx->legendre.size();
  if (wp::launch_taper_eval(ctx->d_legendre, ncoef, ctx->d_taper_img, q.n, 1, q.n, 0) != cudaSuccess ||
      wp::launch_taper_eval(ctx->d_legendre, ncoef, ctx->d_taper_lat, h, 0, ctx->m, 0) != cudaSuccess ||
      wp::launch_taper_inverse(ctx->d_taper_img, ctx->d_taper_inv, q.n, 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    return bail(WP_ECUDA, std::string("taper evaluation failed: ") + cudaGetErrorString(cudaGetLastError()));
  }
  *out = ctx;
  return WP_OK;
}

int wp_make_wkernels(wp_ctx* ctx, void* stream) {
  if (!ctx) return WP_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  {
    Phase ph(ctx, WP_PHASE_WKERNELS, s);
    WP_CUDA(ctx, wp::launch_make_wkernels(ctx, s));
  }
  ctx->have_kernels = true;
  return WP_OK;
}

int wp_grid(wp_ctx* ctx, const double* uvw, const double* freq, const void* vis, const float* weight, int64_t nrow,
            int32_t nchan, int32_t flags, void* grid, double* sum_w, int64_t* n_dropped, void* stream) {
  if (!ctx) return WP_EINVAL;
  if (flags & ~(WP_ACCUMULATE | WP_HERMITIAN_PAIRS | WP_KEEP_BINNING | WP_COMPENSATED))
    return fail(ctx, WP_EINVAL, "unknown flag bits");
  const bool keep = (flags & WP_KEEP_BINNING) != 0;
  const bool compensated = (flags & WP_COMPENSATED) != 0;
  if (compensated) {
    int group = 1;
    if (!wp::grid_v2_smem(ctx, &group))
      return fail(ctx, WP_EINVAL, "WP_COMPENSATED needs the register-accumulating kernel (supports up to 32)");
  }
  if (!grid) return fail(ctx, WP_EINVAL, "grid must not be NULL");
  if (nrow > 0 && !vis) return fail(ctx, WP_EINVAL, "vis must not be NULL");
  const int pairs = (flags & WP_HERMITIAN_PAIRS) ? 1 : 0;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = prepare_vis_call(ctx, uvw, freq, nrow, nchan, pairs, keep, s);
  if (rc) return rc;
  const int32_t n = ctx->prm.n;
  if (!(flags & WP_ACCUMULATE)) WP_CUDA(ctx, cudaMemsetAsync(grid, 0, sizeof(float2) * (size_t)n * n, s));
  if (compensated) {
    if ((rc = ensure_buffer(ctx, ctx->comp, sizeof(float2) * (size_t)n * n, "compensation grid"))) return rc;
    WP_CUDA(ctx, cudaMemsetAsync(ctx->comp.ptr, 0, sizeof(float2) * (size_t)n * n, s));
  }
  {
    Phase ph(ctx, WP_PHASE_PLAN, s);
    WP_CUDA(ctx, wp::launch_plan(ctx, uvw, (const float2*)vis, weight, nrow, nchan, pairs != 0, false, keep, s));
  }
  ctx->have_grid_plan = keep;
  ctx->plan_nrow = nrow;
  ctx->plan_nchan = nchan;
  {
    Phase ph(ctx, WP_PHASE_GRID, s);
    ctx->comp_active = compensated ? (float2*)ctx->comp.ptr : nullptr;
    const cudaError_t eg = wp::launch_grid(ctx, (float2*)grid, s);
    ctx->comp_active = nullptr;
    WP_CUDA(ctx, eg);
    if (compensated) {
      WP_CUDA(ctx, wp::launch_add_comp((float2*)grid, (const float2*)ctx->comp.ptr, (int64_t)n * n, ctx->nsm, s));
      ++ctx->launches;
    }
  }
  if (sum_w || n_dropped) {
    k_store_scalars<<<1, 1, 0, s>>>(ctx->d_wsum, ctx->d_dropped, sum_w, (long long*)n_dropped,
                                    (flags & WP_ACCUMULATE) ? 1 : 0);
    WP_CUDA(ctx, cudaGetLastError());
    ++ctx->launches;
  }
  return WP_OK;
}

int wp_degrid(wp_ctx* ctx, const double* uvw, const double* freq, const void* grid, int64_t nrow, int32_t nchan,
              void* vis_out, void* stream) {
  if (!ctx) return WP_EINVAL;
  if (!grid) return fail(ctx, WP_EINVAL, "grid must not be NULL");
  if (nrow > 0 && !vis_out) return fail(ctx, WP_EINVAL, "vis_out must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = prepare_vis_call(ctx, uvw, freq, nrow, nchan, 0, false, s);
  if (rc) return rc;
  if (nrow == 0) return WP_OK;
  WP_CUDA(ctx, cudaMemsetAsync(vis_out, 0, sizeof(float2) * (size_t)nrow * nchan, s));
  {
    Phase ph(ctx, WP_PHASE_PLAN, s);
    WP_CUDA(ctx, wp::launch_plan(ctx, uvw, nullptr, nullptr, nrow, nchan, false, true, false, s));
  }
  {
    Phase ph(ctx, WP_PHASE_DEGRID, s);
    WP_CUDA(ctx, wp::launch_degrid(ctx, (const float2*)grid, (float2*)vis_out, nullptr, s));
  }
  return WP_OK;
}

int wp_degrid_last(wp_ctx* ctx, const void* grid, void* vis_out, void* stream) {
  if (!ctx) return WP_EINVAL;
  if (!ctx->have_grid_plan) return fail(ctx, WP_ESTATE, "no wp_grid binning to reuse (none yet, none kept with WP_KEEP_BINNING, or replaced since)");
  if (!grid) return fail(ctx, WP_EINVAL, "grid must not be NULL");
  const int64_t nvis = ctx->plan_nrow * ctx->plan_nchan;
  if (nvis > 0 && !vis_out) return fail(ctx, WP_EINVAL, "vis_out must not be NULL");
  if (nvis == 0) return WP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  WP_CUDA(ctx, cudaMemsetAsync(vis_out, 0, sizeof(float2) * (size_t)nvis, s));
  {
    Phase ph(ctx, WP_PHASE_DEGRID, s);
    WP_CUDA(ctx, wp::launch_degrid(ctx, (const float2*)grid, (float2*)vis_out, (const uint32_t*)ctx->rec_index.ptr, s));
  }
  return WP_OK;
}

namespace {
// The context's N x N C2C plan, created on first use, bound to stream s.
int ensure_fft(wp_ctx* ctx, cudaStream_t s) {
  if (!ctx->have_fft) {
    if (cufftPlan2d(&ctx->fft, ctx->prm.n, ctx->prm.n, CUFFT_C2C) != CUFFT_SUCCESS)
      return fail(ctx, WP_ECUDA, "cufftPlan2d failed");
    ctx->have_fft = true;
  }
  if (cufftSetStream(ctx->fft, s) != CUFFT_SUCCESS) return fail(ctx, WP_ECUDA, "cufftSetStream failed");
  return WP_OK;
}
}  // namespace

int wp_fft_to_image(wp_ctx* ctx, void* grid, const double* sum_w, int32_t taper_correct, float* image, void* stream) {
  if (!ctx) return WP_EINVAL;
  if (!grid || !sum_w || !image) return fail(ctx, WP_EINVAL, "grid, sum_w and image must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  int rc = ensure_fft(ctx, s);
  if (rc) return rc;
  {
    Phase ph(ctx, WP_PHASE_FFT, s);
    if (cufftExecC2C(ctx->fft, (cufftComplex*)grid, (cufftComplex*)grid, CUFFT_INVERSE) != CUFFT_SUCCESS)
      return fail(ctx, WP_ECUDA, "cufftExecC2C failed");
  }
  {
    Phase ph(ctx, WP_PHASE_IMAGE, s);
    WP_CUDA(ctx, wp::launch_image_post((const float2*)grid, sum_w, ctx->d_taper_inv, taper_correct, image,
                                       ctx->prm.n, s));
    ++ctx->launches;
  }
  return WP_OK;
}

int wp_image_to_grid(wp_ctx* ctx, const float* image, const double* sum_w, int32_t taper_correct, void* grid,
                     void* stream) {
  if (!ctx) return WP_EINVAL;
  if (!grid || !image) return fail(ctx, WP_EINVAL, "image and grid must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  int rc = ensure_fft(ctx, s);
  if (rc) return rc;
  Phase ph(ctx, WP_PHASE_FFT, s);
  WP_CUDA(ctx, wp::launch_image_pre(image, sum_w, ctx->d_taper_inv, taper_correct, (float2*)grid, ctx->prm.n, s));
  if (cufftExecC2C(ctx->fft, (cufftComplex*)grid, (cufftComplex*)grid, CUFFT_FORWARD) != CUFFT_SUCCESS)
    return fail(ctx, WP_ECUDA, "cufftExecC2C failed");
  WP_CUDA(ctx, wp::launch_checker_sign((float2*)grid, ctx->prm.n, s));
  ctx->launches += 2;
  return WP_OK;
}

int wp_plane_info(const wp_ctx* ctx, int32_t* support_out, double* w_out) {
  if (!ctx) return WP_EINVAL;
  for (int i = 0; i < ctx->prm.n_w; ++i) {
    if (support_out) support_out[i] = ctx->supp[i];
    if (w_out) w_out[i] = ctx->wplane[i];
  }
  return WP_OK;
}

int wp_coords(wp_ctx* ctx, const double* uvw, const double* freq, int64_t nrow, int32_t nchan, int32_t flags,
              int32_t* out, void* stream) {
  if (!ctx) return WP_EINVAL;
  if (nrow > 0 && !out) return fail(ctx, WP_EINVAL, "out must not be NULL");
  const int pairs = (flags & WP_HERMITIAN_PAIRS) ? 1 : 0;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_vis_args(ctx, uvw, freq, nrow, nchan, pairs);
  if (rc) return rc;
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  if ((rc = ensure_channels(ctx, nchan))) return rc;
  if (nrow == 0) return WP_OK;
  WP_CUDA(ctx, wp::launch_channel_factors(freq, nchan, ctx->geo.os_l, ctx->geo.wscale, ctx->d_chan, s));
  ++ctx->launches;
  WP_CUDA(ctx, wp::launch_coords(ctx, uvw, nrow, nchan, pairs != 0, out, s));
  return WP_OK;
}

int wp_baseline_order(wp_ctx* ctx, const int32_t* ant1, const int32_t* ant2, int64_t nrow, int32_t n_ant,
                      int32_t* perm_out, uint32_t* start_out, void* stream) {
  if (!ctx) return WP_EINVAL;
  if (nrow < 0 || nrow > 0x7fffffff || n_ant < 1 || n_ant > 46000)
    return fail(ctx, WP_EINVAL, "nrow must be in [0, 2^31) and n_ant in [1, 46000]");
  if (!start_out || (nrow > 0 && (!ant1 || !ant2 || !perm_out)))
    return fail(ctx, WP_EINVAL, "ant1, ant2, perm_out and start_out must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  const int64_t nb = (int64_t)n_ant * (n_ant + 1) / 2;
  int rc = ensure_buffer(ctx, ctx->bl_scratch, sizeof(int32_t) * (size_t)std::max<int64_t>(nrow, 1) +
                                                   2 * sizeof(uint32_t) * (size_t)(nb + 1), "baseline scratch");
  if (rc) return rc;
  int32_t* bidx = (int32_t*)ctx->bl_scratch.ptr;
  uint32_t* count = (uint32_t*)(bidx + std::max<int64_t>(nrow, 1));
  uint32_t* cursor = count + nb + 1;
  WP_CUDA(ctx, wp::launch_baseline_order(ctx, ant1, ant2, nrow, n_ant, bidx, count, start_out, cursor, perm_out, s));
  return WP_OK;
}

int wp_grid_baseline(wp_ctx* ctx, const double* uvw, const double* freq, const void* vis, const float* weight,
                     const int32_t* perm, const uint32_t* start, int32_t n_ant, int64_t nrow, int32_t nchan,
                     int32_t flags, void* grid, double* sum_w, int64_t* n_dropped, void* stream) {
  if (!ctx) return WP_EINVAL;
  if (flags & ~(WP_ACCUMULATE | WP_HERMITIAN_PAIRS)) return fail(ctx, WP_EINVAL, "unknown flag bits");
  if (!grid) return fail(ctx, WP_EINVAL, "grid must not be NULL");
  if (nrow > 0 && (!vis || !perm || !start)) return fail(ctx, WP_EINVAL, "vis, perm and start must not be NULL");
  if (n_ant < 1 || n_ant > 46000) return fail(ctx, WP_EINVAL, "n_ant must be in [1, 46000]");
  if (*std::max_element(ctx->supp.begin(), ctx->supp.end()) > 32)
    return fail(ctx, WP_EINVAL, "wp_grid_baseline takes supports up to 32");
  const int pairs = (flags & WP_HERMITIAN_PAIRS) ? 1 : 0;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = check_vis_args(ctx, uvw, freq, nrow, nchan, pairs);
  if (rc) return rc;
  if (!ctx->have_kernels) return fail(ctx, WP_ESTATE, "wp_make_wkernels has not been called");
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  if ((rc = ensure_channels(ctx, nchan))) return rc;
  if (nrow > 0) {
    WP_CUDA(ctx, wp::launch_channel_factors(freq, nchan, ctx->geo.os_l, ctx->geo.wscale, ctx->d_chan, s));
    ++ctx->launches;
  }
  const int64_t nvis = nrow * nchan, ng = nvis * (pairs ? 2 : 1);
  if ((rc = ensure_buffer(ctx, ctx->coord_scratch, sizeof(int32_t) * 8 * (size_t)std::max<int64_t>(ng, 1),
                          "coordinate scratch")))
    return rc;
  const int32_t n = ctx->prm.n;
  if (!(flags & WP_ACCUMULATE)) WP_CUDA(ctx, cudaMemsetAsync(grid, 0, sizeof(float2) * (size_t)n * n, s));
  int32_t* coords = (int32_t*)ctx->coord_scratch.ptr;
  {
    Phase ph(ctx, WP_PHASE_PLAN, s);
    if (nrow > 0) WP_CUDA(ctx, wp::launch_coords(ctx, uvw, nrow, nchan, pairs != 0, coords, s));
    WP_CUDA(ctx, wp::launch_kept_sums(ctx, coords, ng, nvis, weight, s));
  }
  {
    Phase ph(ctx, WP_PHASE_GRID, s);
    if (nrow > 0)
      WP_CUDA(ctx, wp::launch_grid_baseline(ctx, coords, start, perm, n_ant, nchan, nrow, pairs != 0,
                                            (const float2*)vis, weight, (float2*)grid, s));
  }
  if (sum_w || n_dropped) {
    k_store_scalars<<<1, 1, 0, s>>>(ctx->d_wsum, ctx->d_dropped, sum_w, (long long*)n_dropped,
                                    (flags & WP_ACCUMULATE) ? 1 : 0);
    WP_CUDA(ctx, cudaGetLastError());
    ++ctx->launches;
  }
  return WP_OK;
}

int wp_wkernel_export(wp_ctx* ctx, int32_t plane, int32_t which, void* out_host, int64_t cap) {
  if (!ctx) return WP_EINVAL;
  if (!ctx->have_kernels) return fail(ctx, WP_ESTATE, "wp_make_wkernels has not been called");
  if (plane < 0 || plane >= ctx->prm.n_w) return fail(ctx, WP_EINVAL, "plane out of range");
  if (which != 0 && which != 1) return fail(ctx, WP_EINVAL, "which must be 0 or 1");
  const int s = ctx->supp[plane], os = ctx->prm.oversample, e = s * os;
  if (!out_host || cap < (int64_t)e * e) return fail(ctx, WP_EINVAL, "output too small");
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  WP_CUDA(ctx, cudaDeviceSynchronize());
  if (which == 0) {
    WP_CUDA(ctx, cudaMemcpy(out_host, ctx->d_tab64 + ctx->tab64_off[plane], sizeof(double2) * (size_t)e * e,
                            cudaMemcpyDeviceToHost));
    return WP_OK;
  }
  const size_t esz = ctx->prm.table_type == WP_TABLE_F32 ? 8 : 4;
  std::vector<unsigned char> raw(esz * (size_t)e * e);
  WP_CUDA(ctx, cudaMemcpy(raw.data(), (const unsigned char*)ctx->d_tab + esz * ctx->tab_off[plane], raw.size(),
                          cudaMemcpyDeviceToHost));
  float* o = (float*)out_host;
  for (int ey = 0; ey < e; ++ey) {
    for (int ex = 0; ex < e; ++ex) {
      const int a = ex / os, ox = ex % os, b = ey / os, oy = ey % os;
      const size_t src = ((size_t)(oy * os + ox) * s + a) * s + b;
      float re, im;
      if (esz == 8) {
        std::memcpy(&re, &raw[8 * src], 4);
        std::memcpy(&im, &raw[8 * src + 4], 4);
      } else {
        uint16_t hr, hi;
        std::memcpy(&hr, &raw[4 * src], 2);
        std::memcpy(&hi, &raw[4 * src + 2], 2);
        if (ctx->prm.table_type == WP_TABLE_BF16) {   // BfWord: re = word << 16, im = word
          uint32_t w;
          std::memcpy(&w, &raw[4 * src], 4);
          const uint32_t ur = w << 16;
          std::memcpy(&re, &ur, 4);
          std::memcpy(&im, &w, 4);
        } else {
          re = half_to_float(hr);
          im = half_to_float(hi);
        }
      }
      o[2 * ((size_t)ey * e + ex)] = re;
      o[2 * ((size_t)ey * e + ex) + 1] = im;
    }
  }
  return WP_OK;
}

int wp_wkernel_norm(wp_ctx* ctx, double* nu_out) {
  if (!ctx || !nu_out) return WP_EINVAL;
  if (!ctx->have_kernels) return fail(ctx, WP_ESTATE, "wp_make_wkernels has not been called");
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  WP_CUDA(ctx, cudaMemcpy(nu_out, ctx->d_nu, sizeof(double), cudaMemcpyDeviceToHost));
  return WP_OK;
}

int wp_profile(wp_ctx* ctx, int32_t enable) {
  if (!ctx) return WP_EINVAL;
  ctx->profiling = enable != 0;
  return WP_OK;
}

int wp_profile_read(wp_ctx* ctx, double* ms_out, int32_t* count_out, int64_t* launches_out) {
  if (!ctx) return WP_EINVAL;
  double ms[WP_NPHASES] = {0};
  int32_t cnt[WP_NPHASES] = {0};
  WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
  cudaError_t first = cudaSuccess;
  for (auto& it : ctx->intervals) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(it.second.second);
    if (!e) e = cudaEventElapsedTime(&t, it.second.first, it.second.second);
    if (e && !first) first = e;
    if (!e && it.first >= 0 && it.first < WP_NPHASES) {
      ms[it.first] += t;
      ++cnt[it.first];
    }
    ctx->event_pool.push_back(it.second.first);
    ctx->event_pool.push_back(it.second.second);
  }
  ctx->intervals.clear();
  for (int i = 0; i < WP_NPHASES; ++i) {
    if (ms_out) ms_out[i] = ms[i];
    if (count_out) count_out[i] = cnt[i];
  }
  if (launches_out) *launches_out = ctx->launches;
  ctx->launches = 0;
  if (first) return cuda_fail(ctx, first, "cudaEventElapsedTime");
  return WP_OK;
}

int wp_taper_eval_host(double c, const double* x, int64_t n, double* out) {
  if (!(c > 0.0) || n < 0 || (n > 0 && (!x || !out))) return WP_EINVAL;
  const std::vector<double> g = wp::pswf_legendre_coefficients(c);
  for (int64_t i = 0; i < n; ++i) {
    if (!(std::fabs(x[i]) <= 1.0)) return WP_EINVAL;
    out[i] = wp::legendre_even_series(g.data(), (int)g.size(), x[i]);
  }
  return WP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batches of gridding jobs

struct wp_batch {
  std::vector<wp_job> jobs;
  std::vector<int> fused;               // jobs in the persistent launch
  int table_type = WP_TABLE_F32;
  size_t smem = 0;
  int device = 0;
  int nsm = 0;
  void* d_desc = nullptr;               // [fused] per-job kernel arguments
  uint64_t* d_jobcost = nullptr;        // [fused + 1]
  uint32_t* d_work = nullptr;           // [2]
};

void wp_batch_destroy(wp_batch* b) {
  if (!b) return;
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->d_jobcost) cudaFree(b->d_jobcost);
  if (b->d_work) cudaFree(b->d_work);
  delete b;
}

int32_t wp_batch_fused_jobs(const wp_batch* b) { return b ? (int32_t)b->fused.size() : 0; }

int wp_batch_create(const wp_job* jobs, int32_t njobs, wp_batch** out) {
  if (!out) return WP_EINVAL;
  *out = nullptr;
  if (njobs < 1 || !jobs) return WP_EINVAL;
  std::unique_ptr<wp_batch, void (*)(wp_batch*)> b(new wp_batch, wp_batch_destroy);
  for (int32_t i = 0; i < njobs; ++i) {
    const wp_job& j = jobs[i];
    if (!j.ctx) return WP_EINVAL;
    wp_ctx* ctx = j.ctx;
    for (int32_t k = 0; k < i; ++k)
      if (jobs[k].ctx == ctx) return fail(ctx, WP_EINVAL, "wp_batch_create: a context appears in two jobs");
    if (ctx->prm.device != jobs[0].ctx->prm.device)
      return fail(ctx, WP_EINVAL, "wp_batch_create: all jobs must be on one device");
    if (j.flags & ~(WP_ACCUMULATE | WP_HERMITIAN_PAIRS)) return fail(ctx, WP_EINVAL, "unknown flag bits");
    if (!j.grid) return fail(ctx, WP_EINVAL, "grid must not be NULL");
    if (j.nrow > 0 && !j.vis) return fail(ctx, WP_EINVAL, "vis must not be NULL");
    const int pairs = (j.flags & WP_HERMITIAN_PAIRS) ? 1 : 0;
    int rc = check_vis_args(ctx, j.uvw, j.freq, j.nrow, j.nchan, pairs);
    if (rc) return rc;
    if (!ctx->have_kernels) return fail(ctx, WP_ESTATE, "wp_make_wkernels has not been called");
    WP_CUDA(ctx, cudaSetDevice(ctx->prm.device));
    if ((rc = ensure_channels(ctx, j.nchan))) return rc;
    const size_t nv = (size_t)j.nrow * j.nchan, ng = nv * (pairs ? 2 : 1);
    if ((rc = ensure_buffer(ctx, ctx->records, std::max<size_t>(ng, 1) * sizeof(wp::Record), "records"))) return rc;
    if ((rc = ensure_buffer(ctx, ctx->records2, std::max<size_t>(ng, 1) * sizeof(wp::Record), "sorted records"))) return rc;
    b->jobs.push_back(j);
  }
  wp_ctx* c0 = jobs[0].ctx;
  b->device = c0->prm.device;
  b->nsm = c0->nsm;
  // the persistent launch takes the jobs the warp kernel takes, of the first such job's table type
  for (int32_t i = 0; i < njobs; ++i) {
    int group = 1;
    const size_t sm = wp::grid_v2_smem(jobs[i].ctx, &group);
    if (!sm) continue;
    if (b->fused.empty()) b->table_type = jobs[i].ctx->prm.table_type;
    if (jobs[i].ctx->prm.table_type != b->table_type) continue;
    b->fused.push_back(i);
    b->smem = std::max(b->smem, sm);
  }
  if (!b->fused.empty()) {
    const size_t db = wp::grid_job_desc_bytes();
    std::vector<unsigned char> host(db * b->fused.size());
    for (size_t f = 0; f < b->fused.size(); ++f) {
      const wp_job& j = jobs[b->fused[f]];
      wp::grid_job_desc(j.ctx, (float2*)j.grid, b->smem, host.data() + f * db);
    }
    if (cudaMalloc(&b->d_desc, host.size()) != cudaSuccess ||
        cudaMalloc((void**)&b->d_jobcost, sizeof(uint64_t) * (b->fused.size() + 1)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_work, 2 * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c0, WP_ENOMEM, "wp_batch_create: device allocation failed");
    }
    if (cudaMemcpy(b->d_desc, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_work, 0, 2 * sizeof(uint32_t)) != cudaSuccess ||
        wp::prepare_grid_batch(b->table_type, b->smem) != cudaSuccess) {
      const cudaError_t e = cudaGetLastError();
      return fail(c0, WP_ECUDA, std::string("wp_batch_create: ") + cudaGetErrorString(e));
    }
  }
  *out = b.release();
  return WP_OK;
}

int wp_batch_grid(wp_batch* b, void* stream) {
  if (!b) return WP_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  WP_CUDA(b->jobs[0].ctx, cudaSetDevice(b->device));
  std::vector<char> is_fused(b->jobs.size(), 0);
  for (int f : b->fused) is_fused[f] = 1;
  // coordinates and binning of every job; the baseline kernel for jobs outside the launch
  for (size_t i = 0; i < b->jobs.size(); ++i) {
    const wp_job& j = b->jobs[i];
    wp_ctx* ctx = j.ctx;
    const int pairs = (j.flags & WP_HERMITIAN_PAIRS) ? 1 : 0;
    ctx->have_grid_plan = false;
    const int32_t n = ctx->prm.n;
    if (!(j.flags & WP_ACCUMULATE)) WP_CUDA(ctx, cudaMemsetAsync(j.grid, 0, sizeof(float2) * (size_t)n * n, s));
    if (j.nrow > 0) {
      WP_CUDA(ctx, wp::launch_channel_factors(j.freq, j.nchan, ctx->geo.os_l, ctx->geo.wscale, ctx->d_chan, s));
      ++ctx->launches;
    }
    {
      Phase ph(ctx, WP_PHASE_PLAN, s);
      WP_CUDA(ctx, wp::launch_plan(ctx, j.uvw, (const float2*)j.vis, j.weight, j.nrow, j.nchan, pairs != 0, false, false, s));
    }
    if (is_fused[i]) {
      WP_CUDA(ctx, wp::launch_bin_costs(ctx, s));
    } else {
      Phase ph(ctx, WP_PHASE_GRID, s);
      WP_CUDA(ctx, wp::launch_grid(ctx, (float2*)j.grid, s));
    }
  }
  if (!b->fused.empty()) {
    wp_ctx* c0 = b->jobs[b->fused[0]].ctx;
    Phase ph(c0, WP_PHASE_GRID, s);
    WP_CUDA(c0, wp::launch_grid_batch(b->d_desc, (int)b->fused.size(), b->d_jobcost, b->d_work, b->table_type,
                                      b->smem, b->nsm, s));
    c0->launches += 2;
  }
  for (const wp_job& j : b->jobs) {
    if (j.sum_w || j.n_dropped) {
      k_store_scalars<<<1, 1, 0, s>>>(j.ctx->d_wsum, j.ctx->d_dropped, j.sum_w, (long long*)j.n_dropped,
                                      (j.flags & WP_ACCUMULATE) ? 1 : 0);
      WP_CUDA(j.ctx, cudaGetLastError());
      ++j.ctx->launches;
    }
  }
  return WP_OK;
}
