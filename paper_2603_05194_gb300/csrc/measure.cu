// Peak-rate measurement of the binary64 FMA pipe, the denominator of the
// roofline of the binary64 FFT passes (which are bound by that pipe on this
// GPU).  Every thread runs kChains independent FMA chains a = a * b + c with
// |b| < 1, so each chain stays bounded and no chain waits on another; the
// sums are stored so the compiler keeps every FMA.  Measurement support of
// the library; the paper has no counterpart.
#include <cuda_runtime.h>

#include "atkm_internal.cuh"

namespace atkm {
namespace {

constexpr int kChains = 8;
constexpr int kFmaThreads = 256;

__global__ void __launch_bounds__(kFmaThreads) k_fma_chains(double* __restrict__ out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (double)(threadIdx.x + i) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace atkm

using namespace atkm;

extern "C" int atkm_measure_fp64_fma(int blocks_per_sm, int iters, int repeats, double* gflops, void* stream) {
  if (!gflops || blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || repeats < 1)
    return fail(nullptr, ATKM_ERR_ARG, "atkm_measure_fp64_fma: bad argument");
  const int nsm = device_sm_count();
  if (nsm <= 0) return fail(nullptr, ATKM_ERR_CUDA, "atkm_measure_fp64_fma: no device");
  const int blocks = nsm * blocks_per_sm;
  cudaStream_t st = (cudaStream_t)stream;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void**)&out, (size_t)blocks * kFmaThreads * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  for (int r = 0; r <= repeats && e == cudaSuccess; ++r) {  // r = 0 warms up
    e = cudaEventRecord(e0, st);
    k_fma_chains<<<blocks, kFmaThreads, 0, st>>>(out, iters, 0.999999, 1e-7);
    count_launches(1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms > 0.0f) {
      const double flops = 2.0 * kChains * (double)iters * blocks * kFmaThreads;
      const double g = flops / (ms * 1e-3) / 1e9;
      if (g > best) best = g;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "atkm_measure_fp64_fma");
  *gflops = best;
  return ATKM_OK;
}
