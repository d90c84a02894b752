// wp_grid_noalloc: the gridding call of wp_grid for callers that must not allocate device
// memory during the call. The per-call scratch that wp_grid sizes to the call and keeps in
// a context-owned, growable buffer (the binned 16-byte records and the per-channel
// factors) lives here in one fixed file-scope device array instead. Everything else is the
// wp_grid pipeline unchanged: the same coordinate, binning and gridding kernels, and the
// context's bin counters, which wp_create sized once.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr int64_t kMaxRecords = int64_t(1) << 20;  // gridded visibilities per call (pairs count twice)
constexpr int32_t kMaxChannels = 4096;
constexpr size_t kRecordBytes = sizeof(wp::Record) * (size_t)kMaxRecords;
// the binned records, the same records sorted by footprint origin, the channel factors
constexpr size_t kScratchBytes = 2 * kRecordBytes + sizeof(double) * 2 * (size_t)kMaxChannels;
constexpr int kMaxDevices = 64;

// 32 MiB + 64 KiB on every GPU that loads this library, held until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Looks up the device address of g_scratch on `dev` (which must be current) and caches it.
// The lookup also loads this file's module on that device, which is when the array's memory
// is taken: wp_create does it, so that a wp_grid_noalloc call never loads the module itself.
cudaError_t lookup_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_mutex);
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_addr[dev] = p;
  return cudaSuccess;
}

// The cached address for `dev`, looked up now if no context has done it yet.
cudaError_t scratch_address(int dev, void** out) {
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_addr[dev]) {
      *out = g_scratch_addr[dev];
      return cudaSuccess;
    }
  }
  const cudaError_t e = lookup_scratch(dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mutex);
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void k_noalloc_scalars(const double* wsum, const unsigned long long* dropped, double* sum_w,
                                  long long* n_dropped, int accumulate) {
  if (sum_w) *sum_w = accumulate ? *sum_w + *wsum : *wsum;
  if (n_dropped) *n_dropped = accumulate ? *n_dropped + (long long)*dropped : (long long)*dropped;
}

int reject(wp_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

// Points the context's per-call scratch at g_scratch for the duration of one call.
struct ScratchView {
  wp_ctx* ctx;
  wp::DeviceBuffer records, records2;
  double* chan;
  int32_t max_chan;
  ScratchView(wp_ctx* c, void* base)
      : ctx(c), records(c->records), records2(c->records2), chan(c->d_chan), max_chan(c->max_chan) {
    ctx->records.ptr = base;
    ctx->records.bytes = kRecordBytes;
    ctx->records2.ptr = (unsigned char*)base + kRecordBytes;
    ctx->records2.bytes = kRecordBytes;
    ctx->d_chan = (double*)((unsigned char*)base + 2 * kRecordBytes);
    ctx->max_chan = kMaxChannels;
  }
  ~ScratchView() {
    ctx->records = records;
    ctx->records2 = records2;
    ctx->d_chan = chan;
    ctx->max_chan = max_chan;
  }
};

}  // namespace

namespace wp {
// Called by wp_create with the context's device current: resolves (again) the scratch array's
// address on that device. Re-resolving at every context creation keeps the cache valid after a
// cudaDeviceReset, since contexts made before a reset cannot be used after it anyway.
cudaError_t noalloc_prepare(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return cudaSuccess;     // wp_grid_noalloc rejects such devices
  return lookup_scratch(dev);
}
}  // namespace wp

extern "C" int wp_grid_noalloc(wp_ctx* ctx, const double* uvw, const double* freq, const void* vis,
                               const float* weight, int64_t nrow, int32_t nchan, int32_t flags, void* grid,
                               double* sum_w, int64_t* n_dropped, void* stream) {
  if (!ctx) return WP_EINVAL;
  if (flags & ~(WP_ACCUMULATE | WP_HERMITIAN_PAIRS)) return reject(ctx, WP_EINVAL, "unknown flag bits");
  if (nrow < 0 || nchan < 1) return reject(ctx, WP_EINVAL, "nrow must be >= 0 and nchan >= 1");
  const int pairs = (flags & WP_HERMITIAN_PAIRS) ? 1 : 0;
  if (nchan > kMaxChannels)
    return reject(ctx, WP_EINVAL, "wp_grid_noalloc: nchan exceeds its fixed scratch (at most 4096 channels)");
  if (nrow > kMaxRecords / nchan || nrow * nchan * (pairs ? 2 : 1) > kMaxRecords)
    return reject(ctx, WP_EINVAL,
                  "wp_grid_noalloc: more than 1048576 gridded visibilities (nrow * nchan, x2 with Hermitian "
                  "pairs) in one call; split the call or use wp_grid");
  if (!grid) return reject(ctx, WP_EINVAL, "grid must not be NULL");
  if (nrow > 0 && (!uvw || !freq || !vis)) return reject(ctx, WP_EINVAL, "uvw, freq and vis must not be NULL");
  if (!ctx->have_kernels) return reject(ctx, WP_ESTATE, "wp_make_wkernels has not been called");
  const int dev = ctx->prm.device;
  if (dev < 0 || dev >= kMaxDevices) return reject(ctx, WP_EINVAL, "device ordinal beyond 63");
  cudaError_t e = cudaSetDevice(dev);
  void* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  if (e != cudaSuccess) return reject(ctx, WP_ECUDA, std::string("wp_grid_noalloc set-up: ") + cudaGetErrorString(e));

  cudaStream_t s = (cudaStream_t)stream;
  ctx->have_grid_plan = false;          // the context's binning is not kept by this call
  ScratchView view(ctx, base);
  const int32_t n = ctx->prm.n;
  if (!(flags & WP_ACCUMULATE)) e = cudaMemsetAsync(grid, 0, sizeof(float2) * (size_t)n * n, s);
  if (e == cudaSuccess && nrow > 0)
    e = wp::launch_channel_factors(freq, nchan, ctx->geo.os_l, ctx->geo.wscale, ctx->d_chan, s);
  if (e == cudaSuccess)
    e = wp::launch_plan(ctx, uvw, (const float2*)vis, weight, nrow, nchan, pairs != 0, false, false, s);
  if (e == cudaSuccess) e = wp::launch_grid(ctx, (float2*)grid, s);
  if (e == cudaSuccess && (sum_w || n_dropped)) {
    k_noalloc_scalars<<<1, 1, 0, s>>>(ctx->d_wsum, ctx->d_dropped, sum_w, (long long*)n_dropped,
                                      (flags & WP_ACCUMULATE) ? 1 : 0);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return reject(ctx, WP_ECUDA, std::string("wp_grid_noalloc: ") + cudaGetErrorString(e));
  return WP_OK;
}
