// Least-squares pseudo-inverses R_i of fixed meshes on the device (Sec. 2.1,
// Eq. CWENO:Popt, precomputed once per mesh), with the kernel of
// lsq_kernels.cuh.  Unlike the stencil search this unit compiles with FMA
// contraction: no integer decision depends on the rounding of R_i, and the
// least squares is bound by the FP64 pipe.
#include "lsq_kernels.cuh"

namespace cw {

int lsq_launch_device(const MeshHost& m, const RefElem& re, const double* d_X, const double* d_bary,
                      const int32_t* d_sten, void* d_R, int fp32, int* d_bad, void* stream, std::string& err) {
  LsqTab tab;
  if (!make_tab(m, re, tab, err)) return CWENO_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const cudaError_t e = fp32 ? dispatch<float>(m.d, re.M, d_X, d_bary, d_sten, m.nc, tab, d_R, d_bad, st)
                             : dispatch<double>(m.d, re.M, d_X, d_bary, d_sten, m.nc, tab, d_R, d_bad, st);
  if (e != cudaSuccess) {
    err = std::string("device least-squares setup: ") + cudaGetErrorString(e);
    return CWENO_ECUDA;
  }
  return CWENO_OK;
}

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
