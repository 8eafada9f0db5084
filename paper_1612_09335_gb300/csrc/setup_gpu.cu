// Per-cell reconstruction data of a fixed mesh on the device, once at setup
// (Sec. 2.1: precomputed for fixed meshes): the ranked stencil search, the
// sectors and their inverses and the inverse Jacobians; the least-squares
// matrices follow with the kernel of lsq_gpu.cu.  This unit is compiled
// without FMA contraction, the same arithmetic as the host setup (which
// remains for cweno_mesh_stencils and for searches beyond the device
// kernel's per-thread capacity), so that the quantised distance keys and the
// cone tests pick the host's cells.
#include "lsq_kernels.cuh"

namespace cw {

// ------------------------------------------------------------------ stencils
// The per-cell stencil setup of a fixed mesh on the device, one thread per
// cell, with the host setup's rule and arithmetic (this unit compiles
// without FMA contraction): the central stencil S_i^0 as the first n_e - 1
// cells of the ranked breadth-first sequence over face neighbours (inside a
// layer by the quantised squared distance of the minimum-image barycentre to
// b_i, then its coordinates, then the caller's cell index), continued two
// layers further; sector s as the first d cells of that sequence whose
// barycentre has barycentric coordinates > 1e-9 w.r.t. every vertex of T_i
// but s (Sec. 2.1, readings c2/c3), dropped when its barycentres are
// collinear / coplanar or its matrix singular; the inverse Jacobian and the
// sector inverses B_s^-1 of Eq. (CWENO:Ps).  Written in the layouts the
// reconstruction kernel reads (layout.h, SoA).  A breadth-first search that
// outgrows the fixed per-thread capacity (SEQ cells, LAY per layer) is
// reported in *cap, and the caller runs the host search instead.
namespace {

template <int D, int M, typename T, int SEQ, int LAY>
__global__ void __launch_bounds__(128) k_stencils(const double* __restrict__ X, const double* __restrict__ bary,
                                                  const int32_t* __restrict__ nbr, const int32_t* __restrict__ perm,
                                                  int64_t N, const LsqTab tab, double qscale, int32_t* sten,
                                                  int32_t* sten4, int32_t* sec, T* Binv, uint8_t* nsec, T* Jinv,
                                                  int* small, int* cap) {
  constexpr int NVX = D + 1, MC = cmc(M, D), NE = D * MC, NE1 = NE - 1, NX = NVX * 3;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  auto shift = [&](int64_t j, double* s) {
    for (int a = 0; a < 3; ++a) {
      s[a] = 0.0;
      if (a < D && tab.per[a]) s[a] = tab.Lper[a] * nearbyint((bary[i * 3 + a] - bary[j * 3 + a]) / tab.Lper[a]);
    }
  };
  // ---- ranked breadth-first sequence (cell i excluded)
  int32_t seq[SEQ];
  long long key[LAY][4];
  int32_t usr[LAY];
  int nseq = 0;
  int p0 = 0;   // first index of layer L-2 (the oldest layer a new neighbour can lie in)
  int f0 = 0, f1 = 0;  // the front (layer L-1); layer 1 grows from i itself
  const double tol = 1e-9 * qscale;
  int done_layer = -1;
  bool ok = false;
  for (int layer = 1;; ++layer) {
    const int n0 = nseq;
    const int nfront = layer == 1 ? 1 : f1 - f0;
    for (int q = 0; q < nfront; ++q) {
      const int64_t c = layer == 1 ? i : seq[f0 + q];
      for (int k = 0; k < NVX; ++k) {
        const int32_t j = nbr[c * NVX + k];
        if (j < 0 || j == i) continue;
        bool seen = false;
        for (int r = p0; r < nseq && !seen; ++r) seen = seq[r] == j;
        if (seen) continue;
        if (nseq >= SEQ || nseq - n0 >= LAY) {
          atomicMax(cap, 1);
          return;
        }
        seq[nseq++] = j;
      }
    }
    const int nn = nseq - n0;
    if (nn == 0) break;
    for (int q = 0; q < nn; ++q) {
      const int32_t j = seq[n0 + q];
      double s[3];
      shift(j, s);
      double b[3] = {0, 0, 0}, d2 = 0.0;
      for (int a = 0; a < D; ++a) {
        b[a] = bary[j * 3 + a] + s[a];
        const double df = b[a] - bary[i * 3 + a];
        d2 += df * df;
      }
      key[q][0] = llround(d2 / (tol * qscale));
      for (int a = 0; a < 3; ++a) key[q][1 + a] = llround(b[a] / tol);
      usr[q] = perm[j];
    }
    // insertion sort of the layer by (key, caller index)
    for (int q = 1; q < nn; ++q) {
      long long kq[4] = {key[q][0], key[q][1], key[q][2], key[q][3]};
      const int32_t uq = usr[q], cq = seq[n0 + q];
      int r = q - 1;
      for (; r >= 0; --r) {
        bool greater = false;  // entry r > entry q
        bool decided = false;
        for (int t = 0; t < 4 && !decided; ++t)
          if (key[r][t] != kq[t]) {
            greater = key[r][t] > kq[t];
            decided = true;
          }
        if (!decided) greater = usr[r] > uq;
        if (!greater) break;
        for (int t = 0; t < 4; ++t) key[r + 1][t] = key[r][t];
        usr[r + 1] = usr[r];
        seq[n0 + r + 1] = seq[n0 + r];
      }
      for (int t = 0; t < 4; ++t) key[r + 1][t] = kq[t];
      usr[r + 1] = uq;
      seq[n0 + r + 1] = cq;
    }
    if (done_layer < 0 && nseq + 1 >= NE) done_layer = layer;
    if (done_layer >= 0 && layer >= done_layer + 2) {
      ok = true;
      break;
    }
    p0 = layer == 1 ? 0 : f0;
    f0 = n0;
    f1 = nseq;
  }
  if (!ok && nseq + 1 >= NE) ok = true;  // the mesh ran out of layers after S_i^0 was complete
  if (!ok) {
    atomicMin(small, (int)i);
    return;
  }
  for (int r = 0; r < NE1; ++r) sten[(int64_t)r * N + i] = seq[r];
  for (int r = 0; r < (NE1 + 3) / 4 * 4; ++r) sten4[((int64_t)(r / 4) * N + i) * 4 + r % 4] = r < NE1 ? seq[r] : (int32_t)i;
  // ---- inverse Jacobian
  const double* Xi = X + i * NX;
  double Ji[3][3];
  jac_inv<D>(Xi, Ji);
  for (int a = 0; a < D; ++a)
    for (int b = 0; b < D; ++b) Jinv[(int64_t)(a * D + b) * N + i] = (T)Ji[a][b];
  // ---- sectors
  auto ref_coords = [&](int32_t j, double* xi) {
    double s[3];
    shift(j, s);
    double x[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) x[a] = bary[j * 3 + a] + s[a];
    for (int a = 0; a < 3; ++a) xi[a] = 0.0;
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) xi[a] += Ji[a][b] * (x[b] - Xi[b]);
  };
  int kept = 0;
  double psi[MC];
  for (int sct = 0; sct < NVX; ++sct) {
    int32_t chosen[3];
    double xib[3][3];
    int nch = 0;
    for (int q = 0; q < nseq && nch < D; ++q) {
      double xi[3];
      ref_coords(seq[q], xi);
      double lam[4];
      lam[0] = 1.0;
      for (int a = 0; a < D; ++a) {
        lam[a + 1] = xi[a];
        lam[0] -= xi[a];
      }
      bool in = true;
      for (int v = 0; v < NVX; ++v)
        if (v != sct && !(lam[v] > 1e-9)) in = false;
      if (!in) continue;
      for (int a = 0; a < 3; ++a) xib[nch][a] = xi[a];
      chosen[nch++] = seq[q];
    }
    if (nch < D) continue;
    double G[9];
    for (int k = 0; k < D; ++k)
      for (int a = 0; a < D; ++a) G[k * D + a] = xib[k][a] - 1.0 / NVX;
    const double dG = D == 2 ? G[0] * G[3] - G[1] * G[2]
                             : G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                                   G[2] * (G[3] * G[7] - G[4] * G[6]);
    if (fabs(dG) < 1e-8) continue;
    double B[9], Bi[9];
    for (int k = 0; k < D; ++k) {
      dubiner<D, M>(tab, xib[k], psi);
      for (int l = 0; l < D; ++l) B[k * D + l] = psi[1 + l];
    }
    if (D == 2) {
      const double det = B[0] * B[3] - B[1] * B[2];
      if (det == 0.0) continue;
      Bi[0] = B[3] / det;
      Bi[1] = -B[1] / det;
      Bi[2] = -B[2] / det;
      Bi[3] = B[0] / det;
    } else {
      const double c00 = B[4] * B[8] - B[5] * B[7], c01 = B[5] * B[6] - B[3] * B[8],
                   c02 = B[3] * B[7] - B[4] * B[6];
      const double det = B[0] * c00 + B[1] * c01 + B[2] * c02;
      if (det == 0.0) continue;
      Bi[0] = c00 / det;
      Bi[3] = c01 / det;
      Bi[6] = c02 / det;
      Bi[1] = (B[2] * B[7] - B[1] * B[8]) / det;
      Bi[4] = (B[0] * B[8] - B[2] * B[6]) / det;
      Bi[7] = (B[1] * B[6] - B[0] * B[7]) / det;
      Bi[2] = (B[1] * B[5] - B[2] * B[4]) / det;
      Bi[5] = (B[2] * B[3] - B[0] * B[5]) / det;
      Bi[8] = (B[0] * B[4] - B[1] * B[3]) / det;
    }
    for (int k = 0; k < D; ++k) sec[(int64_t)(sct * D + k) * N + i] = chosen[k];
    for (int q = 0; q < D * D; ++q) Binv[(int64_t)(sct * D * D + q) * N + i] = (T)Bi[q];
    ++kept;
  }
  nsec[i] = (uint8_t)kept;
}

template <int D, int M, typename T>
cudaError_t launch_stencils(const double* X, const double* bary, const int32_t* nbr, const int32_t* perm, int64_t N,
                            const LsqTab& tab, double qscale, int32_t* sten, int32_t* sten4, int32_t* sec, void* Binv,
                            uint8_t* nsec, void* Jinv, int* small, int* cap, cudaStream_t st) {
  // fifth order on the Kuhn tetrahedra: at most 294 cells in the sequence
  // and 100 in one layer (measured on jittered meshes)
  constexpr int SEQ = D == 2 ? 128 : M >= 4 ? 384 : 320, LAY = D == 2 ? 48 : 128;
  k_stencils<D, M, T, SEQ, LAY><<<(unsigned)((N + 127) / 128), 128, 0, st>>>(
      X, bary, nbr, perm, N, tab, qscale, sten, sten4, sec, (T*)Binv, nsec, (T*)Jinv, small, cap);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_stencils(int d, int M, const double* X, const double* bary, const int32_t* nbr,
                              const int32_t* perm, int64_t N, const LsqTab& tab, double qscale, int32_t* sten,
                              int32_t* sten4, int32_t* sec, void* Binv, uint8_t* nsec, void* Jinv, int* small,
                              int* cap, cudaStream_t st) {
#define CW_ST(DD, MM) \
  return launch_stencils<DD, MM, T>(X, bary, nbr, perm, N, tab, qscale, sten, sten4, sec, Binv, nsec, Jinv, small, cap, st)
  if (d == 2) {
    switch (M) {
      case 1: CW_ST(2, 1);
      case 2: CW_ST(2, 2);
      case 3: CW_ST(2, 3);
      case 4: CW_ST(2, 4);
    }
  } else {
    switch (M) {
      case 1: CW_ST(3, 1);
      case 2: CW_ST(3, 2);
      case 3: CW_ST(3, 3);
      case 4: CW_ST(3, 4);
    }
  }
#undef CW_ST
  return cudaErrorInvalidValue;
}

}  // namespace

int cell_setup_device(const MeshHost& m, const RefElem& re, int fp32, void* stream, int32_t* d_sten, int32_t* d_sten4,
                      int32_t* d_sec, void* d_Binv, uint8_t* d_nsec, void* d_Jinv, void* d_R, std::string& err) {
  cudaStream_t st = (cudaStream_t)stream;
  const int d = m.d, M = re.M;
  const int64_t N = m.nc;
  LsqTab tab;
  if (!make_tab(m, re, tab, err)) return CWENO_EINVAL;
  double *dX = nullptr, *dB = nullptr;
  int32_t *dN = nullptr, *dP = nullptr;
  int* flags = nullptr;  // [0] smallest cell too small for S_i^0, [1] capacity, [2] rank-deficient R
  int hflags[3] = {INT_MAX, 0, INT_MAX};
  cudaError_t e = cudaMallocAsync((void**)&dX, sizeof(double) * m.X.size(), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dB, sizeof(double) * m.bary.size(), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dN, sizeof(int32_t) * m.nbr.size(), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dP, sizeof(int32_t) * m.perm.size(), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&flags, sizeof(hflags), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dX, m.X.data(), sizeof(double) * m.X.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dB, m.bary.data(), sizeof(double) * m.bary.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dN, m.nbr.data(), sizeof(int32_t) * m.nbr.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dP, m.perm.data(), sizeof(int32_t) * m.perm.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags, hflags, sizeof(hflags), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = fp32 ? dispatch_stencils<float>(d, M, dX, dB, dN, dP, N, tab, m.qscale, d_sten, d_sten4, d_sec, d_Binv,
                                        d_nsec, d_Jinv, flags, flags + 1, st)
             : dispatch_stencils<double>(d, M, dX, dB, dN, dP, N, tab, m.qscale, d_sten, d_sten4, d_sec, d_Binv,
                                         d_nsec, d_Jinv, flags, flags + 1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const bool search_ok = e == cudaSuccess && hflags[0] == INT_MAX && hflags[1] == 0;
  if (search_ok) {
    const int rc = lsq_launch_device(m, re, dX, dB, d_sten, d_R, fp32, flags + 2, st, err);
    if (rc != CWENO_OK) {
      cudaFreeAsync(dX, st);
      cudaFreeAsync(dB, st);
      cudaFreeAsync(dN, st);
      cudaFreeAsync(dP, st);
      cudaFreeAsync(flags, st);
      return rc;
    }
  }
  if (search_ok && e == cudaSuccess) e = cudaMemcpyAsync(hflags + 2, flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (search_ok && e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dX) cudaFreeAsync(dX, st);
  if (dB) cudaFreeAsync(dB, st);
  if (dN) cudaFreeAsync(dN, st);
  if (dP) cudaFreeAsync(dP, st);
  if (flags) cudaFreeAsync(flags, st);
  if (e != cudaSuccess) {
    err = std::string("device cell setup: ") + cudaGetErrorString(e);
    return CWENO_ECUDA;
  }
  if (hflags[1]) return kCellSetupOnHost;
  if (hflags[0] != INT_MAX) {
    err = "mesh too small for the central stencil at cell " + std::to_string(m.perm[hflags[0]]);
    return CWENO_EDEGENERATE;
  }
  if (hflags[2] != INT_MAX) {
    err = "rank-deficient least-squares system at cell " + std::to_string(m.perm[hflags[2]]);
    return CWENO_EDEGENERATE;
  }
  return CWENO_OK;
}

}  // namespace cw
