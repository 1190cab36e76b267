// Allocation-free inner products for callers that cannot allocate device
// memory (for example code running inside a host framework that owns every
// allocation, or a process that must not grow its device footprint after
// start-up).  Same reduction as the library's fused inner-product kernel, but
// its per-block partial sums live in a file-scope device array instead of a
// plan-owned buffer, so no plan is needed.
#include <cuda_runtime.h>

#include <mutex>

#include "atkm_internal.cuh"

namespace atkm {

namespace {

constexpr int kNaPairs = ATKM_NOALLOC_MAX_PAIRS;  // pairs per call
constexpr int kNaBlocks = 1216;                    // most reduction CTAs of a call (scratch capacity)
constexpr int kNaThreads = 256;
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: kNaPairs x kNaBlocks partial sums
// (77,824 bytes).  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) double g_noalloc_partials[kNaPairs * kNaBlocks];

// Device address of the scratch per device ordinal, set up on first use.
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

struct NaPairs {
  const double2* u[kNaPairs];
  const double2* v[kNaPairs];
  int n;
};

__global__ void __launch_bounds__(kNaThreads) k_na_dots(NaPairs dp, size_t N, double* __restrict__ part) {
  double acc[kNaPairs];
#pragma unroll
  for (int i = 0; i < kNaPairs; ++i) acc[i] = 0.0;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < N; j += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int i = 0; i < kNaPairs; ++i) {
      if (i < dp.n) {
        const double2 a = dp.u[i][j], b = dp.v[i][j];
        acc[i] += a.x * b.x + a.y * b.y;
      }
    }
  }
  // every block writes all kNaPairs slots (zeros beyond dp.n), so nothing
  // from an earlier call is ever read
  block_reduce_store<kNaPairs>(acc, part, gridDim.x, blockIdx.x);
}

__global__ void k_na_finalize(const double* __restrict__ part, int nblocks, double scale, double* __restrict__ out) {
  __shared__ double sh[kNaThreads];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kNaThreads) acc += part[(size_t)s * nblocks + i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kNaThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[s] = scale * sh[0];
}

// Returns the scratch's device address on the current device, looking it up
// (cudaGetSymbolAddress) the first time this device is seen.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace atkm

using namespace atkm;

extern "C" int atkm_inner_products_noalloc(const double* const* u, const double* const* v, int npairs,
                                           unsigned long long n, double hvol, double* out, void* stream) {
  if (!u || !v || !out) return fail(nullptr, ATKM_ERR_ARG, "atkm_inner_products_noalloc: NULL argument");
  if (npairs < 1 || npairs > kNaPairs)
    return fail(nullptr, ATKM_ERR_ARG,
                "atkm_inner_products_noalloc: npairs must be in [1, ATKM_NOALLOC_MAX_PAIRS = 8]");
  if (n == 0) return fail(nullptr, ATKM_ERR_ARG, "atkm_inner_products_noalloc: n must be positive");
  NaPairs dp;
  for (int i = 0; i < kNaPairs; ++i) { dp.u[i] = nullptr; dp.v[i] = nullptr; }
  dp.n = npairs;
  for (int i = 0; i < npairs; ++i) {
    if (!u[i] || !v[i]) return fail(nullptr, ATKM_ERR_ARG, "atkm_inner_products_noalloc: NULL vector");
    dp.u[i] = reinterpret_cast<const double2*>(u[i]);
    dp.v[i] = reinterpret_cast<const double2*>(v[i]);
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "atkm_inner_products_noalloc: scratch set-up");
  cudaStream_t st = (cudaStream_t)stream;
  size_t G = (n + (size_t)kNaThreads * 4 - 1) / ((size_t)kNaThreads * 4);
  if (G > (size_t)kNaBlocks) G = kNaBlocks;
  if (G < 1) G = 1;
  k_na_dots<<<(int)G, kNaThreads, 0, st>>>(dp, (size_t)n, scratch);
  k_na_finalize<<<npairs, kNaThreads, 0, st>>>(scratch, (int)G, hvol, out);
  count_launches(2);
  e = cudaGetLastError();
  return e == cudaSuccess ? ATKM_OK : cuda_fail(nullptr, e, "atkm_inner_products_noalloc");
}
