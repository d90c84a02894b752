// Image formation after the inverse FFT (the IFFT step of the Fig. 1 / Fig. 2 captions of
// Lao et al. 2019) and the taper correction.
//
// With F = unnormalised inverse DFT of the grid (cuFFT C2C, CUFFT_INVERSE, in place),
// the centred transform of wproj.h is
//     I[j][i] = (-1)^(i + j) Re F[(j + N/2) mod N][(i + N/2) mod N]
// (for even N the (g - N/2)(i - N/2) phase splits into e^{2 pi i g i / N} (-1)^(g + i)
// times a factor (-1)^(N/2) per axis, which cancels over two axes, and (-1)^g on the
// input is a shift of the output by N/2). The epilogue also divides by the weight sum
// and by t(x_i) t(x_j), as float32 products of reciprocals computed once per context.
#include <cuda_runtime.h>

#include "internal.h"

namespace wp {

namespace {

// inv[i] = 1 / t(x_i) in float32 (once per context).
__global__ void k_taper_inverse(const double* __restrict__ taper, float* __restrict__ inv, int32_t n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) inv[i] = (float)(1.0 / taper[i]);
}

// The image in float32: sign * Re F * (1 / sum_w) * (1 / t(x_i)) * (1 / t(x_j)).
__global__ void k_image_post(const float2* __restrict__ f, const double* __restrict__ sum_w,
                             const float* __restrict__ inv_taper, int32_t taper_correct, float* __restrict__ image,
                             int32_t n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  const int h = n / 2;
  const float v = f[(int64_t)((j + h) % n) * n + (i + h) % n].x;
  float scale = 1.0f / (float)*sum_w;
  if (taper_correct) scale *= inv_taper[i] * inv_taper[j];
  const float sgn = ((i + j) & 1) ? -1.f : 1.f;
  image[(int64_t)j * n + i] = sgn * v * scale;
}

// The adjoint direction (wp_image_to_grid): with z[j][i] = (-1)^(i + j) X[j][i], the centred
// forward transform is G[h][g] = (-1)^(g + h) DFT2(z)[h][g] (same parity argument as above), so
// the pre-kernel forms z, cuFFT runs forward in place and the post-kernel flips the signs.
__global__ void k_image_pre(const float* __restrict__ image, const double* __restrict__ sum_w,
                            const float* __restrict__ inv_taper, int32_t taper_correct, float2* __restrict__ z,
                            int32_t n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  float scale = sum_w ? 1.0f / (float)*sum_w : 1.0f;
  if (taper_correct) scale *= inv_taper[i] * inv_taper[j];
  const float sgn = ((i + j) & 1) ? -1.f : 1.f;
  z[(int64_t)j * n + i] = make_float2(sgn * scale * image[(int64_t)j * n + i], 0.f);
}

__global__ void k_checker_sign(float2* __restrict__ g, int32_t n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n || !((i + j) & 1)) return;
  float2* p = &g[(int64_t)j * n + i];
  const float2 v = *p;
  *p = make_float2(-v.x, -v.y);
}

}  // namespace

cudaError_t launch_image_pre(const float* image, const double* sum_w, const float* inv_taper, int32_t taper_correct,
                             float2* z, int32_t n, cudaStream_t s) {
  dim3 grid((n + 255) / 256, n);
  k_image_pre<<<grid, 256, 0, s>>>(image, sum_w, inv_taper, taper_correct, z, n);
  return cudaGetLastError();
}

cudaError_t launch_checker_sign(float2* g, int32_t n, cudaStream_t s) {
  dim3 grid((n + 255) / 256, n);
  k_checker_sign<<<grid, 256, 0, s>>>(g, n);
  return cudaGetLastError();
}

cudaError_t launch_taper_inverse(const double* taper_img, float* inv, int32_t n, cudaStream_t s) {
  k_taper_inverse<<<(n + 255) / 256, 256, 0, s>>>(taper_img, inv, n);
  return cudaGetLastError();
}

cudaError_t launch_image_post(const float2* spectrum, const double* sum_w, const float* inv_taper,
                              int32_t taper_correct, float* image, int32_t n, cudaStream_t s) {
  dim3 grid((n + 255) / 256, n);
  k_image_post<<<grid, 256, 0, s>>>(spectrum, sum_w, inv_taper, taper_correct, image, n);
  return cudaGetLastError();
}

}  // namespace wp
