// W-kernel generation in float64 on the device.
//
// The W-projection kernel of plane p is the Fourier transform of the tapered w-screen
//     s_p(l, m) = t(l) t(m) exp(2 pi i w_p (n - 1)),   n = sqrt(1 - l^2 - m^2)
// sampled on an odd M x M lattice (j = -(M-1)/2 .. (M-1)/2, l = j L / M) and evaluated at
// 1/os-cell offsets (the oversampled kernel of the method of Cornwell et al. 2008, which
// Lao et al. 2019 defer to in Sec. 1; full support S_p as in Sec. 2.2 / 3.1):
//     K_p(dx, dy) = sum_{j,j'} s_p(j, j') exp(-2 pi i (dx j + dy j') / (os M)).
// The screen is even in l and in m (n depends on l^2 + m^2; the lattice is symmetric), so
// the transform folds into a real cosine transform over the j, j' >= 0 quadrant with
// weights mu_0 = 1, mu_{j>0} = 2, applied one axis at a time, and K_p is even in dx and
// dy: only dx, dy >= 0 is computed, the rest follows by symmetry. This computes only the
// (S_p os/2 + 1)^2 outputs that gridding reads instead of a full os*M-point 2D FFT.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace wp {

namespace {

__global__ void k_cos_table(double* __restrict__ out, int32_t period) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < period) out[r] = cospi(2.0 * r / period);
}

// mode 0: x = 2 j / param (screen lattice, j = 0 .. n-1); mode 1: x = 2 (i - param/2) / param (pixels)
__global__ void k_taper_eval(const double* __restrict__ leg, int ncoef, double* __restrict__ out, int64_t n,
                             int mode, int32_t param) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = mode == 0 ? 2.0 * (double)i / param : 2.0 * (double)(i - param / 2) / param;
  out[i] = legendre_even_series(leg, ncoef, x);
}

struct KernelGeo {
  int32_t n_w, m, h, os, period, dmax;
  double field;
  const double* wplane;   // [Nw]
  const int32_t* supp;    // [Nw]
  const int64_t* quad_off;
  const int64_t* tab_off;
};

// Screen quadrant: scr[p][jq][jk] for jq, jk in [0, H), H = (M+1)/2.
__global__ void k_screen(KernelGeo kg, const double* __restrict__ taper_lat, double2* __restrict__ scr) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t hh = (int64_t)kg.h * kg.h;
  if (idx >= hh * kg.n_w) return;
  const int p = (int)(idx / hh);
  const int jq = (int)((idx - (int64_t)p * hh) / kg.h);
  const int jk = (int)(idx - (int64_t)p * hh - (int64_t)jq * kg.h);
  const double l = (double)jk * kg.field / kg.m;
  const double mm = (double)jq * kg.field / kg.m;
  const double r2 = l * l + mm * mm;
  const double nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
  double sn, cs;
  sincospi(2.0 * kg.wplane[p] * nm1, &sn, &cs);
  const double t = taper_lat[jk] * taper_lat[jq];
  scr[idx] = make_double2(t * cs, t * sn);
}

// First axis: stage[p][jq][dx] = sum_jk mu_k scr[p][jq][jk] cos(2 pi dx jk / (os M)).
__global__ void k_stage1(KernelGeo kg, const double2* __restrict__ scr, const double* __restrict__ cosv,
                         double2* __restrict__ stage) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)kg.h * kg.dmax;
  if (idx >= per * kg.n_w) return;
  const int p = (int)(idx / per);
  const int jq = (int)((idx - (int64_t)p * per) / kg.dmax);
  const int dx = (int)(idx - (int64_t)p * per - (int64_t)jq * kg.dmax);
  const int dp = kg.supp[p] * kg.os / 2 + 1;
  if (dx >= dp) return;
  const double2* row = scr + ((int64_t)p * kg.h + jq) * kg.h;
  double re = 0.0, im = 0.0;
  for (int jk = 0; jk < kg.h; ++jk) {
    const double c = (jk ? 2.0 : 1.0) * cosv[(dx * jk) % kg.period];
    re = fma(c, row[jk].x, re);
    im = fma(c, row[jk].y, im);
  }
  stage[idx] = make_double2(re, im);
}

// Second axis: quad[p][dy][dx] = sum_jq mu_q stage[p][jq][dx] cos(2 pi dy jq / (os M)).
__global__ void k_stage2(KernelGeo kg, const double2* __restrict__ stage, const double* __restrict__ cosv,
                         double2* __restrict__ quad) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)kg.dmax * kg.dmax;
  if (idx >= per * kg.n_w) return;
  const int p = (int)(idx / per);
  const int dy = (int)((idx - (int64_t)p * per) / kg.dmax);
  const int dx = (int)(idx - (int64_t)p * per - (int64_t)dy * kg.dmax);
  const int dp = kg.supp[p] * kg.os / 2 + 1;
  if (dx >= dp || dy >= dp) return;
  const double2* col = stage + (int64_t)p * kg.h * kg.dmax + dx;
  double re = 0.0, im = 0.0;
  for (int jq = 0; jq < kg.h; ++jq) {
    const double c = (jq ? 2.0 : 1.0) * cosv[(dy * jq) % kg.period];
    const double2 v = col[(int64_t)jq * kg.dmax];
    re = fma(c, v.x, re);
    im = fma(c, v.y, im);
  }
  quad[kg.quad_off[p] + (int64_t)dy * dp + dx] = make_double2(re, im);
}

// nu = Re sum of plane 0's taps at whole-cell offsets d = os e in (-S0 os/2, S0 os/2].
__global__ void k_norm(KernelGeo kg, const double2* __restrict__ quad, double* __restrict__ nu) {
  const int s0 = kg.supp[0];
  const int half = s0 * kg.os / 2;
  const int dp = half + 1;
  const int emin = -((half - 1) / kg.os);  // smallest e with os e > -half; S0 values e .. e + S0 - 1
  double acc = 0.0;
  for (int q = threadIdx.x; q < s0 * s0; q += blockDim.x) {
    const int a = q % s0, b = q / s0;
    const int dx = abs((emin + a) * kg.os), dy = abs((emin + b) * kg.os);
    acc += quad[kg.quad_off[0] + (int64_t)dy * dp + dx].x;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *nu = red[0];
}

template <class T>
__device__ __forceinline__ T store_tap(double re, double im);
template <>
__device__ __forceinline__ float2 store_tap<float2>(double re, double im) {
  return make_float2(__double2float_rn(re), __double2float_rn(im));
}
template <>
__device__ __forceinline__ __half2 store_tap<__half2>(double re, double im) {
  return __halves2half2(__double2half(re), __double2half(im));
}
// BfWord: low 16 bits = re rounded to bfloat16; high 16 bits chosen so that the whole word, as
// float32, is the nearest such value to im (candidates: the float32 of im truncated to its high
// half and its two neighbours; non-finite candidates are skipped).
template <>
__device__ __forceinline__ BfWord store_tap<BfWord>(double re, double im) {
  const __nv_bfloat16 rb = __double2bfloat16(re);
  uint16_t lo;
  memcpy(&lo, &rb, 2);
  const uint32_t hi0 = __float_as_uint(__double2float_rn(im)) >> 16;
  uint32_t best = (hi0 << 16) | lo;
  double err = fabs((double)__uint_as_float(best) - im);
  if (!isfinite(__uint_as_float(best))) err = INFINITY;
  for (int dlt = -1; dlt <= 1; dlt += 2) {
    const uint32_t w = (((hi0 + (uint32_t)dlt) & 0xffffu) << 16) | lo;
    const float v = __uint_as_float(w);
    if (isfinite(v) && fabs((double)v - im) < err) {
      err = fabs((double)v - im);
      best = w;
    }
  }
  return BfWord{best};
}

// Full tables: canonical float64 [ey][ex] and the stored grid layout
// tab[p] + ((oy*os + ox)*S + a)*S + b with ex = a os + ox, ey = b os + oy (footprint row b
// fastest: the lanes that hold consecutive rows read consecutive taps).
template <class T>
__global__ void k_tables(KernelGeo kg, const double2* __restrict__ quad, const double* __restrict__ nu,
                         const int64_t* __restrict__ tab64_off, double2* __restrict__ tab64, T* __restrict__ tab,
                         int64_t total) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int p = 0;  // tab64_off is increasing; plane p holds [tab64_off[p], tab64_off[p+1])
  while (p + 1 < kg.n_w && tab64_off[p + 1] <= idx) ++p;
  const int s = kg.supp[p];
  const int e = s * kg.os;
  const int half = e / 2;
  const int64_t local = idx - tab64_off[p];
  const int ey = (int)(local / e), ex = (int)(local - (int64_t)ey * e);
  const int dx = abs(ex - half + 1), dy = abs(ey - half + 1);
  const int dp = half + 1;
  const double2 k = quad[kg.quad_off[p] + (int64_t)dy * dp + dx];
  const double norm = *nu;
  const double re = k.x / norm, im = k.y / norm;
  tab64[idx] = make_double2(re, im);
  const int a = ex / kg.os, ox = ex - a * kg.os;
  const int b = ey / kg.os, oy = ey - b * kg.os;
  tab[kg.tab_off[p] + ((int64_t)(oy * kg.os + ox) * s + a) * s + b] = store_tap<T>(re, im);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_taper_eval(const double* d_leg, int ncoef, double* out, int64_t n, int mode, int32_t param,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_taper_eval<<<nblk(n, 128), 128, 0, s>>>(d_leg, ncoef, out, n, mode, param);
  return cudaGetLastError();
}

cudaError_t launch_make_wkernels(wp_ctx* ctx, cudaStream_t s) {
  const wp_params& prm = ctx->prm;
  KernelGeo kg;
  kg.n_w = prm.n_w;
  kg.m = ctx->m;
  kg.h = (ctx->m + 1) / 2;
  kg.os = prm.oversample;
  kg.period = prm.oversample * ctx->m;
  kg.dmax = 0;
  for (int p = 0; p < prm.n_w; ++p) kg.dmax = std::max(kg.dmax, ctx->supp[p] * prm.oversample / 2 + 1);
  kg.field = (double)prm.n * prm.cell_rad;
  kg.wplane = ctx->d_wplane;
  kg.supp = ctx->d_supp;
  kg.quad_off = ctx->d_quad_off;
  kg.tab_off = ctx->d_tab_off;
  cudaError_t e;
  ctx->launches += 6;
  k_cos_table<<<nblk(kg.period, 256), 256, 0, s>>>(ctx->d_cos, kg.period);
  if ((e = cudaGetLastError())) return e;
  k_screen<<<nblk((int64_t)kg.h * kg.h * kg.n_w, 256), 256, 0, s>>>(kg, ctx->d_taper_lat, ctx->d_screen);
  if ((e = cudaGetLastError())) return e;
  k_stage1<<<nblk((int64_t)kg.h * kg.dmax * kg.n_w, 128), 128, 0, s>>>(kg, ctx->d_screen, ctx->d_cos, ctx->d_stage);
  if ((e = cudaGetLastError())) return e;
  k_stage2<<<nblk((int64_t)kg.dmax * kg.dmax * kg.n_w, 128), 128, 0, s>>>(kg, ctx->d_stage, ctx->d_cos, ctx->d_quad);
  if ((e = cudaGetLastError())) return e;
  k_norm<<<1, 256, 0, s>>>(kg, ctx->d_quad, ctx->d_nu);
  if ((e = cudaGetLastError())) return e;
  const int64_t total = ctx->tab64_elems;
  switch (prm.table_type) {
    case WP_TABLE_F16:
      k_tables<__half2><<<nblk(total, 256), 256, 0, s>>>(kg, ctx->d_quad, ctx->d_nu, ctx->d_tab64_off, ctx->d_tab64,
                                                         (__half2*)ctx->d_tab, total);
      break;
    case WP_TABLE_BF16:
      k_tables<BfWord><<<nblk(total, 256), 256, 0, s>>>(kg, ctx->d_quad, ctx->d_nu, ctx->d_tab64_off,
                                                                ctx->d_tab64, (BfWord*)ctx->d_tab, total);
      break;
    default:
      k_tables<float2><<<nblk(total, 256), 256, 0, s>>>(kg, ctx->d_quad, ctx->d_nu, ctx->d_tab64_off, ctx->d_tab64,
                                                        (float2*)ctx->d_tab, total);
  }
  const cudaError_t et = cudaGetLastError();
  if (et) return et;
  // lane-order copies of the planes with S > 16 for the warp kernels
  return launch_lane_tables(ctx, s);
}

}  // namespace wp
