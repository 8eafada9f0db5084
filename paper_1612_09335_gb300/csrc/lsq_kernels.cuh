// Least-squares reconstruction matrices on the device (Sec. 2.1, Eq.
// CWENO:Popt), shared by the fixed-mesh setup (lsq_gpu.cu; setup_gpu.cu uses
// the tables and the Dubiner evaluation for its sector inverses) and the
// per-step rebuild on moving meshes (ale.cu): for every cell, the averages of the Dubiner basis
// functions psi_1..psi_{Mc-1} of its reference frame over the cells of its
// central stencil (the constrained problem with the constant part removed),
// the pseudo-inverse R_i of that (n_e - 1) x (Mc - 1) matrix by modified
// Gram-Schmidt with one reorthogonalisation pass (FMA, reciprocals instead of
// per-entry divisions), written in the vector layout
// the reconstruction kernel reads (layout.h); and the sector inverses of Eq. (CWENO:Ps).
// FP64 throughout, one thread per cell.  Each including translation unit gets
// its own copy (unnamed namespace).
#pragma once
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/cweno.h"
#include "host.h"
#include "layout.h"

namespace cw {

namespace {

constexpr int kMaxQ = 27, kMaxB = 35, kMaxRec = 11 * 5;

// reference data of one (d, M) as a kernel parameter
struct LsqTab {
  int nq;
  double qx[kMaxQ][3];
  double qw[kMaxQ];
  double wsum;
  int nb;
  int pqr[kMaxB][3];
  double norm[kMaxB];
  double rec[kMaxRec][3];  // [(alpha * (M + 1) + k)]
  double Lper[3];
  int per[3];
};

__host__ __device__ constexpr int cmc(int M, int d) {
  return d == 2 ? (M + 1) * (M + 2) / 2 : (M + 1) * (M + 2) * (M + 3) / 6;
}

template <int M>
__device__ __forceinline__ void jacobi_seq(const LsqTab& t, int alpha, int nmax, double u, double s, double* p) {
  p[0] = 1.0;
  if (nmax < 1) return;
  p[1] = 0.5 * ((alpha + 2.0) * u + alpha * s);
#pragma unroll
  for (int k = 2; k <= nmax; ++k) {
    const double* r = t.rec[alpha * (M + 1) + k];
    p[k] = (r[0] * s + r[1] * u) * p[k - 1] - r[2] * s * s * p[k - 2];
  }
}

// all Dubiner basis functions at xi (psi_0 = 1), shared Jacobi sequences.
// The basis order is the reference element's (by total degree k, then r,
// then q; make_tab checks it), unrolled at compile time so that every index
// is static and the sequences stay in registers.  The third-direction
// sequence depends on (p + q, r) only: one per p + q, a prefix of which
// serves every r.
template <int D, int M>
__device__ __forceinline__ void dubiner(const LsqTab& t, const double* xi, double* out) {
  double f1[M + 1], f2[M + 1][M + 1];
  out[0] = 1.0;
  if (D == 2) {
    const double s1 = 1.0 - xi[1], u1 = 2.0 * xi[0] - s1;
    jacobi_seq<M>(t, 0, M, u1, s1, f1);
#pragma unroll
    for (int p = 0; p <= M; ++p) jacobi_seq<M>(t, 2 * p + 1, M - p, 2.0 * xi[1] - 1.0, 1.0, f2[p]);
    int l = 0;
#pragma unroll
    for (int k = 0; k <= M; ++k)
#pragma unroll
      for (int q = 0; q <= k; ++q, ++l)
        if (l > 0) out[l] = t.norm[l] * (f1[k - q] * f2[k - q][q]);
    return;
  }
  double f3[M + 1][M + 1];
  const double s1 = 1.0 - xi[1] - xi[2], u1 = 2.0 * xi[0] - s1;
  const double s2 = 1.0 - xi[2], u2 = 2.0 * xi[1] - s2;
  jacobi_seq<M>(t, 0, M, u1, s1, f1);
#pragma unroll
  for (int p = 0; p <= M; ++p) jacobi_seq<M>(t, 2 * p + 1, M - p, u2, s2, f2[p]);
#pragma unroll
  for (int pq = 0; pq <= M; ++pq) jacobi_seq<M>(t, 2 * pq + 2, M - pq, 2.0 * xi[2] - 1.0, 1.0, f3[pq]);
  int l = 0;
#pragma unroll
  for (int k = 0; k <= M; ++k)
#pragma unroll
    for (int r = 0; r <= k; ++r)
#pragma unroll
      for (int q = 0; q <= k - r; ++q, ++l)
        if (l > 0) out[l] = t.norm[l] * (f1[k - q - r] * f2[k - q - r][q] * f3[k - r][r]);
}

template <int D>
__device__ void jac_inv(const double* X, double Ji[3][3]) {
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int a = 0; a < D; ++a)
    for (int k = 0; k < D; ++k) J[a][k] = X[(k + 1) * 3 + a] - X[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Ji[a][b] = 0.0;
  if (D == 2) {
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det;
    Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det;
    Ji[1][1] = J[0][0] / det;
    return;
  }
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  Ji[0][0] = c00 / det;
  Ji[1][0] = c01 / det;
  Ji[2][0] = c02 / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

// X: nc x (D+1) x 3 unwrapped vertices, bary: nc x 3, sten: SoA [k N + i].
// bad: smallest internal index of a cell whose system is rank deficient.
template <int D, int M, typename T>
__global__ void __launch_bounds__(128) k_lsq(const double* __restrict__ X, const double* __restrict__ bary,
                                             const int32_t* __restrict__ sten, int64_t N, const LsqTab tab,
                                             T* __restrict__ R, int* bad) {
  constexpr int MC = cmc(M, D), NE1 = D * MC - 1, MC1 = MC - 1, NX = (D + 1) * 3;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* Xi = X + i * NX;
  double Ji[3][3];
  jac_inv<D>(Xi, Ji);
  // FP64 divisions are long instruction sequences: reciprocals once, then
  // products; explicit fma() in the inner loops
  const double iwsum = 1.0 / tab.wsum;
  double Qc[MC1][NE1];  // A by columns, then Q
  double psi[MC];
  for (int r = 0; r < NE1; ++r) {
    const int64_t j = sten[(int64_t)r * N + i];
    const double* Xj = X + j * NX;
    double s[3];
    for (int a = 0; a < 3; ++a) {
      s[a] = 0.0;
      if (a < D && tab.per[a])
        s[a] = tab.Lper[a] * nearbyint((bary[i * 3 + a] - bary[j * 3 + a]) / tab.Lper[a]);
    }
    double acc[MC];
    for (int l = 0; l < MC; ++l) acc[l] = 0.0;
    for (int g = 0; g < tab.nq; ++g) {
      double x[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) {
        x[a] = Xj[a] + s[a];
        for (int k = 0; k < D; ++k) x[a] = fma(tab.qx[g][k], Xj[(k + 1) * 3 + a] - Xj[a], x[a]);
      }
      double xi[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) xi[a] = fma(Ji[a][b], x[b] - Xi[b], xi[a]);
      dubiner<D, M>(tab, xi, psi);
#pragma unroll
      for (int l = 1; l < MC; ++l) acc[l] = fma(tab.qw[g], psi[l], acc[l]);
    }
#pragma unroll
    for (int l = 1; l < MC; ++l) Qc[l - 1][r] = acc[l] * iwsum;
  }
  // modified Gram-Schmidt with one reorthogonalisation pass: A = Q Rm
  double Rm[MC1][MC1];
  for (int a = 0; a < MC1; ++a)
    for (int b = 0; b < MC1; ++b) Rm[a][b] = 0.0;
  bool ok = true;
  // column k in registers while the earlier columns are projected out, where
  // a column fits (n_e - 1 <= 64: up to 3D P3, whose 59-row column in
  // registers measured 36 % less setup time than in local memory); longer
  // columns stay in local memory
  constexpr int UR = NE1 <= 64 ? NE1 : 1;
  for (int k = 0; k < MC1; ++k) {
    double v[NE1];
#pragma unroll UR
    for (int r = 0; r < NE1; ++r) v[r] = Qc[k][r];
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < k; ++j) {
        double sdot = 0.0;
#pragma unroll UR
        for (int r = 0; r < NE1; ++r) sdot = fma(Qc[j][r], v[r], sdot);
        Rm[j][k] += sdot;
#pragma unroll UR
        for (int r = 0; r < NE1; ++r) v[r] = fma(-sdot, Qc[j][r], v[r]);
      }
    double nn = 0.0;
#pragma unroll UR
    for (int r = 0; r < NE1; ++r) nn = fma(v[r], v[r], nn);
    nn = sqrt(nn);
    Rm[k][k] = nn;
    if (nn == 0.0) {
      ok = false;
      break;
    }
    const double inn = 1.0 / nn;
#pragma unroll UR
    for (int r = 0; r < NE1; ++r) Qc[k][r] = v[r] * inn;
  }
  if (ok) {
    double dmax = 0.0;
    for (int k = 0; k < MC1; ++k) dmax = fmax(dmax, fabs(Rm[k][k]));
    for (int k = 0; k < MC1; ++k)
      if (fabs(Rm[k][k]) <= 1e-13 * dmax) ok = false;
  }
  if (!ok) {
    atomicMin(bad, (int)i);
    return;
  }
  // pinv = Rm^{-1} Q^T, column by column of Q^T, in the vector layout of
  // layout.h (r_index)
  double iR[MC1];
  for (int k = 0; k < MC1; ++k) iR[k] = 1.0 / Rm[k][k];
  for (int r = 0; r < NE1; ++r) {
    double col[MC1];
#pragma unroll
    for (int k = MC1 - 1; k >= 0; --k) {
      double sv = Qc[k][r];
#pragma unroll
      for (int j = k + 1; j < MC1; ++j) sv = fma(-Rm[k][j], col[j], sv);
      col[k] = sv * iR[k];
    }
#pragma unroll
    for (int k = 0; k < MC1; ++k) R[r_index<T>(r, k, MC1, i, N)] = (T)col[k];
  }
}

// Moving meshes: the sector inverses of Eq. (CWENO:Ps) for the fixed sector
// cells on the current geometry, B[k][l] = psi_{1+l}(xi_i(b_jk)) (b_jk the
// minimum-image barycentre of the k-th cell of sector s, xi_i the reference
// coordinates of cell i) and Binv[((s D + e) D + k) N + i] = (B^-1)[e][k],
// the layout the reconstruction kernel reads.  Dropped sectors (first id
// < 0) are skipped.  bad: smallest cell index with a singular B.
template <int D, int M, typename T>
__global__ void __launch_bounds__(128) k_sectors(const double* __restrict__ X, const double* __restrict__ bary,
                                                 const int32_t* __restrict__ sec, int64_t N, const LsqTab tab,
                                                 T* __restrict__ Binv, int* bad) {
  constexpr int MC = cmc(M, D), NX = (D + 1) * 3;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* Xi = X + i * NX;
  double Ji[3][3];
  jac_inv<D>(Xi, Ji);
  double psi[MC];
  for (int s = 0; s <= D; ++s) {
    if (sec[(int64_t)(s * D) * N + i] < 0) continue;
    double B[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < D; ++k) {
      const int64_t j = sec[(int64_t)(s * D + k) * N + i];
      double xi[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) {
        double sh = 0.0;
        if (tab.per[a]) sh = tab.Lper[a] * nearbyint((bary[i * 3 + a] - bary[j * 3 + a]) / tab.Lper[a]);
        const double db = bary[j * 3 + a] + sh - Xi[a];
        for (int b = 0; b < D; ++b) xi[b] += Ji[b][a] * db;
      }
      dubiner<D, M>(tab, xi, psi);
      for (int l = 0; l < D; ++l) B[k][l] = psi[1 + l];
    }
    double Bi[3][3];
    double det;
    if (D == 2) {
      det = B[0][0] * B[1][1] - B[0][1] * B[1][0];
      Bi[0][0] = B[1][1] / det;
      Bi[0][1] = -B[0][1] / det;
      Bi[1][0] = -B[1][0] / det;
      Bi[1][1] = B[0][0] / det;
    } else {
      const double c00 = B[1][1] * B[2][2] - B[1][2] * B[2][1];
      const double c01 = B[1][2] * B[2][0] - B[1][0] * B[2][2];
      const double c02 = B[1][0] * B[2][1] - B[1][1] * B[2][0];
      det = B[0][0] * c00 + B[0][1] * c01 + B[0][2] * c02;
      Bi[0][0] = c00 / det;
      Bi[1][0] = c01 / det;
      Bi[2][0] = c02 / det;
      Bi[0][1] = (B[0][2] * B[2][1] - B[0][1] * B[2][2]) / det;
      Bi[1][1] = (B[0][0] * B[2][2] - B[0][2] * B[2][0]) / det;
      Bi[2][1] = (B[0][1] * B[2][0] - B[0][0] * B[2][1]) / det;
      Bi[0][2] = (B[0][1] * B[1][2] - B[0][2] * B[1][1]) / det;
      Bi[1][2] = (B[0][2] * B[1][0] - B[0][0] * B[1][2]) / det;
      Bi[2][2] = (B[0][0] * B[1][1] - B[0][1] * B[1][0]) / det;
    }
    if (!(det != 0.0) || !isfinite(det)) {
      atomicMin(bad, (int)i);
      continue;
    }
    for (int e = 0; e < D; ++e)
      for (int k = 0; k < D; ++k) Binv[(int64_t)((s * D + e) * D + k) * N + i] = (T)Bi[e][k];
  }
}

template <int D, int M, typename T>
cudaError_t launch(const double* X, const double* bary, const int32_t* sten, int64_t N, const LsqTab& tab, void* R,
                   int* bad, cudaStream_t st) {
  const unsigned nb = (unsigned)((N + 127) / 128);
  k_lsq<D, M, T><<<nb, 128, 0, st>>>(X, bary, sten, N, tab, (T*)R, bad);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(int d, int M, const double* X, const double* bary, const int32_t* sten, int64_t N,
                     const LsqTab& tab, void* R, int* bad, cudaStream_t st) {
  if (d == 2) {
    switch (M) {
      case 1: return launch<2, 1, T>(X, bary, sten, N, tab, R, bad, st);
      case 2: return launch<2, 2, T>(X, bary, sten, N, tab, R, bad, st);
      case 3: return launch<2, 3, T>(X, bary, sten, N, tab, R, bad, st);
      case 4: return launch<2, 4, T>(X, bary, sten, N, tab, R, bad, st);
    }
  } else {
    switch (M) {
      case 1: return launch<3, 1, T>(X, bary, sten, N, tab, R, bad, st);
      case 2: return launch<3, 2, T>(X, bary, sten, N, tab, R, bad, st);
      case 3: return launch<3, 3, T>(X, bary, sten, N, tab, R, bad, st);
      case 4: return launch<3, 4, T>(X, bary, sten, N, tab, R, bad, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

namespace {

bool make_tab(const MeshHost& m, const RefElem& re, LsqTab& tab, std::string& err) {
  const int d = m.d, M = re.M;
  // averages of degree-M polynomials: a rule exact to degree M.  The
  // collapsed Gauss rule with (M + 2) / 2 points per direction is; with fewer
  // points: on triangles at M = 2 the three-point degree-2 rule (barycentric
  // permutations of (2/3, 1/6, 1/6), equal weights); on tetrahedra at M = 2
  // the four-point degree-2 rule of Hammer, Marlowe and Stroud (barycentric
  // permutations of (a, b, b, b), a = (5 + 3 sqrt 5) / 20, b = (5 - sqrt 5) /
  // 20, equal weights) and at M = 3 the five-point degree-3 rule (centroid
  // weight -4/5, permutations of (1/2, 1/6, 1/6, 1/6) weight 9/20; the
  // integrands are polynomials of degree M, so the negative weight costs no
  // accuracy).  The weights are normalised by their sum in k_lsq.
  SimplexQuad Q = simplex_quad(d, (M + 2) / 2);
  if (d == 2 && M == 2) {
    const double a = 2.0 / 3.0, b = 1.0 / 6.0;
    Q.x = {{b, b, 0.0}, {a, b, 0.0}, {b, a, 0.0}};
    Q.w = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};
  } else if (d == 3 && M == 2) {
    const double a = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, b = (5.0 - std::sqrt(5.0)) / 20.0;
    Q.x = {{b, b, b}, {a, b, b}, {b, a, b}, {b, b, a}};
    Q.w = {0.25, 0.25, 0.25, 0.25};
  } else if (d == 3 && M == 3) {
    const double a = 0.5, b = 1.0 / 6.0, c = 0.25;
    Q.x = {{c, c, c}, {b, b, b}, {a, b, b}, {b, a, b}, {b, b, a}};
    Q.w = {-0.8, 0.45, 0.45, 0.45, 0.45};
  }
  if ((int)Q.w.size() > kMaxQ || re.psi.n > kMaxB || (2 * M + 3) * (M + 1) > kMaxRec) {
    err = "least-squares tables exceed the device setup limits";
    return false;
  }
  tab.nq = (int)Q.w.size();
  tab.wsum = 0.0;
  for (int g = 0; g < tab.nq; ++g) {
    for (int a = 0; a < 3; ++a) tab.qx[g][a] = Q.x[g][a];
    tab.qw[g] = Q.w[g];
    tab.wsum += Q.w[g];
  }
  tab.nb = re.psi.n;
  // the device Dubiner evaluation unrolls this order (total degree, then r, then q)
  {
    int l = 0;
    bool same = true;
    for (int k = 0; k <= M; ++k)
      for (int r = 0; r <= (d == 3 ? k : 0); ++r)
        for (int q = 0; q <= k - r; ++q, ++l)
          if (l >= tab.nb || re.psi.pqr[l][0] != k - q - r || re.psi.pqr[l][1] != q || re.psi.pqr[l][2] != r)
            same = false;
    if (!same || l != tab.nb) {
      err = "Dubiner basis order differs from the device evaluation";
      return false;
    }
  }
  for (int l = 0; l < tab.nb; ++l) {
    for (int a = 0; a < 3; ++a) tab.pqr[l][a] = re.psi.pqr[l][a];
    tab.norm[l] = re.psi.norm[l];
  }
  for (size_t k = 0; k < re.psi.rec.size(); ++k)
    for (int a = 0; a < 3; ++a) tab.rec[k][a] = re.psi.rec[k][a];
  for (int a = 0; a < 3; ++a) {
    tab.per[a] = m.per[a] ? 1 : 0;
    tab.Lper[a] = m.Lper[a];
  }
  return true;
}

template <int D, int M, typename T>
cudaError_t launch_sectors(const double* X, const double* bary, const int32_t* sec, int64_t N, const LsqTab& tab,
                           T* Binv, int* bad, cudaStream_t st) {
  k_sectors<D, M, T><<<(unsigned)((N + 127) / 128), 128, 0, st>>>(X, bary, sec, N, tab, Binv, bad);
  return cudaGetLastError();
}

}  // namespace

}  // namespace cw
