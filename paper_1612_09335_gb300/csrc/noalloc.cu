// Time-step bound for callers that cannot allocate device memory.
//
// Some callers own a CUDA context in which they may not call cudaMalloc:
// code running inside another framework's memory pool or allocator, or in a
// process whose device memory is fully reserved up front.  cweno_stable_dt_noalloc gives them the CFL bound of a
// state that lives in their own buffers without allocating anything: the
// per-block partial minima live in a file-scope device array that every GPU
// loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/cweno.h"
#include "api_internal.h"
#include "kernels.cuh"

namespace cw {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = CWENO_NOALLOC_MAX_CELLS / kThreads;

// Scratch: one partial minimum (of h_i / |lambda_max,i|) per block of 256
// cells.  In host code this name is only a stand-in; kernels receive the
// address returned by cudaGetSymbolAddress for the current device.
static __device__ __align__(256) double g_dt_partial[kMaxBlocks];

std::mutex g_mu;
void* g_scratch[64] = {nullptr};

__device__ __forceinline__ double block_min(double v) {
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = lane < kThreads / 32 ? red[lane] : __longlong_as_double(0x7ff0000000000000ll);
  if (warp == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w < v ? w : v;
    }
  }
  return v;  // valid in thread 0
}

// one thread per cell; every block writes its own slot, so no slot has to be
// cleared before a call
template <int D, int PDE>
__global__ void __launch_bounds__(kThreads)
    k_dt_partial(const double* __restrict__ Q, const double* __restrict__ h, int64_t n, double gamma, double ch,
                 double* __restrict__ partial) {
  constexpr int NV = PDE == 0 ? D + 2 : 9;
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  double r = __longlong_as_double(0x7ff0000000000000ll);
  if (i < n) {
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = Q[i * NV + v];
    r = h[i] / Phys<D, PDE, double>::speed(q, gamma, ch);
  }
  r = block_min(r);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kThreads)
    k_dt_final(const double* __restrict__ partial, int nb, double cfl, double* __restrict__ dt) {
  double r = __longlong_as_double(0x7ff0000000000000ll);
  for (int b = threadIdx.x; b < nb; b += kThreads) r = partial[b] < r ? partial[b] : r;
  r = block_min(r);
  if (threadIdx.x == 0) *dt = cfl * r;
}

}  // namespace
}  // namespace cw

extern "C" int cweno_stable_dt_noalloc(int dim, int pde, int64_t ncells, const double* Q, const double* h,
                                       double gamma, double c_h, double cfl, double* dt, void* stream) {
  using namespace cw;
  if (dim != 2 && dim != 3) return fail(CWENO_EINVAL, "dim must be 2 or 3");
  if (pde != CWENO_EULER && pde != CWENO_MHD_GLM) return fail(CWENO_EINVAL, "unknown pde");
  if (dim == 3 && pde == CWENO_MHD_GLM) return fail(CWENO_EINVAL, "MHD-GLM is built for 2D meshes only");
  if (!Q || !h || !dt) return fail(CWENO_EINVAL, "null pointer");
  if (!(gamma > 1.0) || !(cfl > 0.0)) return fail(CWENO_EINVAL, "bad gamma or cfl");
  if (ncells <= 0) return fail(CWENO_EINVAL, "no cells");
  if (ncells > CWENO_NOALLOC_MAX_CELLS)
    return fail(CWENO_EINVAL, "ncells exceeds CWENO_NOALLOC_MAX_CELLS (16777216): the static scratch holds one "
                              "partial minimum per 256 cells");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(CWENO_EINVAL, "device ordinal out of range");
  void* scratch = nullptr;
  {
    // set-up once per device, with that device current: the device address
    // of the file-scope scratch array
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
      e = cudaGetSymbolAddress(&g_scratch[dev], g_dt_partial);
      if (e != cudaSuccess) {
        g_scratch[dev] = nullptr;
        return cuda_fail(e, "cudaGetSymbolAddress(g_dt_partial)");
      }
    }
    scratch = g_scratch[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)((ncells + kThreads - 1) / kThreads);
  double* part = (double*)scratch;
  if (dim == 2 && pde == CWENO_EULER) k_dt_partial<2, 0><<<nb, kThreads, 0, st>>>(Q, h, ncells, gamma, c_h, part);
  else if (dim == 3 && pde == CWENO_EULER) k_dt_partial<3, 0><<<nb, kThreads, 0, st>>>(Q, h, ncells, gamma, c_h, part);
  else k_dt_partial<2, 1><<<nb, kThreads, 0, st>>>(Q, h, ncells, gamma, c_h, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_dt_partial launch");
  k_dt_final<<<1, kThreads, 0, st>>>(part, nb, cfl, dt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_dt_final launch");
  return CWENO_OK;
}
