// Least-squares reconstruction matrices of a fixed mesh on the device, once
// at setup (Sec. 2.1: precomputed for fixed meshes), with the kernels of
// lsq_kernels.cuh.  This unit is compiled without FMA contraction, the same
// arithmetic as the host setup.  The stencils themselves (ranked breadth-first
// search) and the sectors stay on the host.
#include "lsq_kernels.cuh"

namespace cw {

int lsq_setup_device(const MeshHost& m, const RefElem& re, const int32_t* d_sten, void* d_R, int fp32,
                     void* stream, std::string& err) {
  cudaStream_t st = (cudaStream_t)stream;
  const int d = m.d, M = re.M;
  const int64_t N = m.nc;
  LsqTab tab;
  if (!make_tab(m, re, tab, err)) return CWENO_EINVAL;
  double* dX = nullptr;
  double* dB = nullptr;
  int* dbad = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&dX, sizeof(double) * m.X.size(), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dB, sizeof(double) * m.bary.size(), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dbad, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dX, m.X.data(), sizeof(double) * m.X.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dB, m.bary.data(), sizeof(double) * m.bary.size(), cudaMemcpyHostToDevice, st);
  const int big = INT_MAX;
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbad, &big, sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = fp32 ? dispatch<float>(d, M, dX, dB, d_sten, N, tab, d_R, dbad, st)
             : dispatch<double>(d, M, dX, dB, d_sten, N, tab, d_R, dbad, st);
  int hbad = INT_MAX;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dX) cudaFreeAsync(dX, st);
  if (dB) cudaFreeAsync(dB, st);
  if (dbad) cudaFreeAsync(dbad, st);
  if (e != cudaSuccess) {
    err = std::string("device least-squares setup: ") + cudaGetErrorString(e);
    return CWENO_ECUDA;
  }
  if (hbad != INT_MAX) {
    err = "rank-deficient least-squares system at cell " + std::to_string(m.perm[hbad]);
    return CWENO_EDEGENERATE;
  }
  return CWENO_OK;
}

}  // namespace cw
