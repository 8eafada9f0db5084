// Measured FMA rate of the device's FP32 and FP64 pipes (the paper has no
// counterpart: it is the denominator of the pipe fractions that the
// benchmark reports beside the HBM fraction).
//
// Every thread runs NCHAIN independent fused multiply-add chains of `iters`
// steps each (a = a * b + c with b, c runtime values, so nothing folds), in
// enough resident blocks to fill every SM.  One untimed launch, then one
// launch timed with CUDA events on a private stream; flops = 2 per FMA.
#include <cuda_runtime.h>

#include "../../include/cweno.h"
#include "api_internal.h"

namespace cw {
namespace {

constexpr int kNChain = 16;
constexpr int kThreads = 256;

// never written for finite sums; naming it keeps the chains live
template <typename T>
__device__ T g_fma_sink;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T b, T c) {
  T a[kNChain];
#pragma unroll
  for (int k = 0; k < kNChain; ++k) a[k] = T(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kNChain; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kNChain; ++k) s += a[k];
  // b = 1 - 2^-20 and c = 1/2 keep every chain finite (it tends to 2^19)
  if (!(s < T(1e30))) g_fma_sink<T> = s;
}

template <typename T>
int measure(double* tflops, double* ms_out) {
  int dev = 0, nsm = 0, nb = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fma_chains<T>, kThreads, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const int blocks = nsm * (nb > 0 ? nb : 1);
  // about 10 ms per timed launch: FP64 runs at a small fraction of FP32
  const int iters = sizeof(T) == 4 ? 16384 : 512;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = CWENO_OK;
  const T b = T(1) - T(1.0 / 1048576.0), c = T(0.5);
  float ms = 0.f;
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    rc = cuda_fail(e, "stream/event create");
    goto done;
  }
  k_fma_chains<T><<<blocks, kThreads, 0, st>>>(iters, b, c);
  cudaEventRecord(e0, st);
  k_fma_chains<T><<<blocks, kThreads, 0, st>>>(iters, b, c);
  cudaEventRecord(e1, st);
  if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
      (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
    rc = cuda_fail(e, "k_fma_chains");
    goto done;
  }
  *tflops = 2.0 * kNChain * (double)iters * (double)blocks * kThreads / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return rc;
}

}  // namespace
}  // namespace cw

extern "C" int cweno_measure_fma_peak(int fp64, double* tflops, double* ms) {
  if (!tflops) return cw::fail(CWENO_EINVAL, "null pointer");
  return fp64 ? cw::measure<double>(tflops, ms) : cw::measure<float>(tflops, ms);
}
