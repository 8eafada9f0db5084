// Moving meshes: the direct ALE ADER-CWENO step (Secs. 2.2-2.4) on 2D
// triangle meshes (tetrahedra: ale3.cuh), Euler equations, FP64 or FP32-mixed (k_ale_pred32,
// k_ale_flux32: FP32 deviations, FP64 least squares, averages' face part,
// nodal solver and update), Rusanov flux with the ALE Jacobian.  Mesh velocity V = v (the local fluid velocity, the choice of the
// paper's moving-mesh tests) or V = 0 (the same machinery on a mesh that does
// not move).  One step:
//   k_ale_geom      cell geometry of the current vertices (unwrapped
//                   vertices, |T|, barycentre, h, 1/|T|);
//   matrices        least-squares pseudo-inverses and sector inverses for
//                   the fixed stencils, rebuilt on the device every step
//                   (Sec. 2.1: on moving meshes they change with the mesh);
//   reconstruction  the fixed-mesh CWENO kernel (gather, P_opt, sectors,
//                   indicators, weights), values at the
//                   lattice nodes;
//   k_ale_pred      space-time predictor on the moving element: state and
//                   geometry DOFs iterated together (Eqs. CGfinal, ODEfinal)
//                   with H of Eq. (Hterm) from the nodal derivatives;
//   k_ale_nodes     nodal solver, Eqs. (NScs)-(newX), one thread per vertex
//                   over a fixed incidence list (increasing cell order, so
//                   the sums are deterministic);
//   k_ale_flux      lateral space-time faces, normals of Eq. (detChi),
//                   Rusanov flux of Eq. (rusanov) with s_max of A_n^V;
//   k_ale_update    Eq. (PDEfinal): |T^{n+1}| Q^{n+1} = |T^n| Q^n - sum.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/cweno.h"
#include "ale.h"
#include "lsq_kernels.cuh"

namespace cw {

constexpr int kLmax = 20, kL0max = 10, kL1max = 10, kNQ = 4;

// Reference tables of one M (2D) in the arithmetic type T, passed as a
// kernel parameter.
template <typename T>
struct AleTabT {
  // d theta_l / d xi_e at node n, nonzero entries only (about a third of
  // them are nonzero): for (e, n) the first nnz[e][n] pairs (col, val)
  T val[2][kLmax][kLmax];
  uint8_t col[2][kLmax][kLmax];
  int nnz[2][kLmax];
  int nnz0[2][kLmax];  // of which on tau = 0 nodes (listed first)
  T Gal[kL1max][kLmax];    // (K_tau^1)^-1 M^1
  T C0[kL1max][kL0max];    // theta_n(xi_k, 0): constant extension in time
  T Wv[3][kLmax];          // int_0^1 theta_l(vertex v, tau) dtau
  T node[kLmax][3];        // xi, eta, tau
  T chi[kNQ], wq[kNQ], wt[kNQ], tq[kNQ];
  T gamma;
  int mode;  // CWENO_MOTION_LAGRANGE or CWENO_MOTION_STILL
  int pos;   // positivity switch (fallbacks as on fixed meshes)
};
using AleTab = AleTabT<double>;
using AleTab32 = AleTabT<float>;

template <typename T>
AleTabT<T> ale_tab_cast(const AleTab& t) {
  AleTabT<T> o;
  std::memset(&o, 0, sizeof(o));
  for (int e = 0; e < 2; ++e)
    for (int n = 0; n < kLmax; ++n) {
      for (int l = 0; l < kLmax; ++l) {
        o.val[e][n][l] = (T)t.val[e][n][l];
        o.col[e][n][l] = t.col[e][n][l];
      }
      o.nnz[e][n] = t.nnz[e][n];
      o.nnz0[e][n] = t.nnz0[e][n];
    }
  for (int k = 0; k < kL1max; ++k) {
    for (int l = 0; l < kLmax; ++l) o.Gal[k][l] = (T)t.Gal[k][l];
    for (int n = 0; n < kL0max; ++n) o.C0[k][n] = (T)t.C0[k][n];
  }
  for (int v = 0; v < 3; ++v)
    for (int l = 0; l < kLmax; ++l) o.Wv[v][l] = (T)t.Wv[v][l];
  for (int l = 0; l < kLmax; ++l)
    for (int a = 0; a < 3; ++a) o.node[l][a] = (T)t.node[l][a];
  for (int q = 0; q < kNQ; ++q) {
    o.chi[q] = (T)t.chi[q];
    o.wq[q] = (T)t.wq[q];
    o.wt[q] = (T)t.wt[q];
    o.tq[q] = (T)t.tq[q];
  }
  o.gamma = (T)t.gamma;
  o.mode = t.mode;
  o.pos = t.pos;
  return o;
}

namespace {

__host__ __device__ constexpr int lcal2(int M) { return (M + 1) * (M + 2) * (M + 3) / 6; }
__host__ __device__ constexpr int mcal2(int M) { return (M + 1) * (M + 2) / 2; }

__device__ __forceinline__ double step_dt(double dt_fixed, double cfl, const unsigned long long* dtmin) {
  return dt_fixed > 0.0 ? dt_fixed : cfl * __longlong_as_double((long long)dtmin[0]);
}

__device__ __forceinline__ double pressure(const double* q, double g) {
  return (g - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
}

__device__ __forceinline__ bool admissible(const double* q, double g) {
  bool fin = isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]);
  return fin && q[0] > 0.0 && pressure(q, g) > 0.0;
}

// ---------------------------------------------------------------- geometry
// Per cell: vertices Xv[g] + the cell's periodic image shift, |T|, the
// barycentre, h = 4|T| / perimeter (incircle diameter, Eq. timestep), 1/|T|.
__global__ void __launch_bounds__(256) k_ale_geom(const double* __restrict__ Xv, const int32_t* __restrict__ gv,
                                                  const double* __restrict__ shift, int64_t N, double* __restrict__ X,
                                                  double* __restrict__ bary, double* __restrict__ vol,
                                                  double* __restrict__ hsize, double* __restrict__ invvol) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double P[3][2];
  for (int k = 0; k < 3; ++k) {
    const int64_t g = gv[k * N + i];
    for (int a = 0; a < 2; ++a) {
      P[k][a] = Xv[g * 2 + a] + shift[(k * 2 + a) * N + i];
      X[i * 9 + k * 3 + a] = P[k][a];
    }
    X[i * 9 + k * 3 + 2] = 0.0;
  }
  const double det = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]);
  const double v = det / 2.0;
  double per = 0.0;
  for (int k = 0; k < 3; ++k) {
    const int a = k == 0 ? 1 : 0, b = k == 2 ? 1 : 2;
    per += hypot(P[b][0] - P[a][0], P[b][1] - P[a][1]);
  }
  vol[i] = v;
  hsize[i] = 4.0 * v / per;
  invvol[i] = 1.0 / v;
  for (int a = 0; a < 2; ++a) bary[i * 3 + a] = (P[0][a] + P[1][a] + P[2][a]) / 3.0;
  bary[i * 3 + 2] = 0.0;
}

// Reset of the time-step bound of slot 0 before it is recomputed.
__global__ void k_ale_dt_reset(unsigned long long* dtmin) { dtmin[0] = 0x7ff0000000000000ull; }

// ---------------------------------------------------------------- predictor
// Euler fluxes (x and y) and the mesh velocity of one nodal state.
__device__ __forceinline__ void ale_flux(const double* q, double gamma, int mode, double F[2][4], double V[2]) {
  const double ir = 1.0 / q[0], u = q[1] * ir, vv = q[2] * ir;
  const double p = (gamma - 1.0) * (q[3] - 0.5 * (q[1] * u + q[2] * vv));
  F[0][0] = q[1];
  F[0][1] = q[1] * u + p;
  F[0][2] = q[2] * u;
  F[0][3] = u * (q[3] + p);
  F[1][0] = q[2];
  F[1][1] = q[1] * vv;
  F[1][2] = q[2] * vv + p;
  F[1][3] = vv * (q[3] + p);
  V[0] = mode == CWENO_MOTION_LAGRANGE ? u : 0.0;
  V[1] = mode == CWENO_MOTION_LAGRANGE ? vv : 0.0;
}

// One thread per cell.  w: reconstruction values at the lattice nodes
// (N x L0 x 4); X: unwrapped vertices of T_i^n.  Writes q_hat (N x L x 4) and,
// per vertex k of the cell, (mu V_kj, mu) with mu = rho_j |T_j| and V_kj the
// time integral of the predictor's mesh velocity at that vertex.
template <int M>
__global__ void __launch_bounds__(128) k_ale_pred(const __grid_constant__ AleTab t, const double* __restrict__ w,
                                                  const double* __restrict__ Q, const double* __restrict__ X,
                                                  const double* __restrict__ vol, int64_t N, int niter,
                                                  double dt_fixed, double cfl, const unsigned long long* dtmin,
                                                  double* __restrict__ qhat, double* __restrict__ vcon) {
  constexpr int L = lcal2(M), L0 = mcal2(M), L1 = L - L0;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double dt = step_dt(dt_fixed, cfl, dtmin);
  double q[L][4], x[L][2];
  for (int n = 0; n < L0; ++n)
    for (int v = 0; v < 4; ++v) q[n][v] = w[(i * L0 + n) * 4 + v];
  for (int k = 0; k < L1; ++k)
    for (int v = 0; v < 4; ++v) {
      double s = 0.0;
      for (int n = 0; n < L0; ++n) s += t.C0[k][n] * q[n][v];
      q[L0 + k][v] = s;
    }
  const double* Xi = X + i * 9;
  for (int l = 0; l < L; ++l)
    for (int a = 0; a < 2; ++a)
      x[l][a] = Xi[a] + (Xi[3 + a] - Xi[a]) * t.node[l][0] + (Xi[6 + a] - Xi[a]) * t.node[l][1];
  // The tau = 0 nodes never change: their fluxes and mesh velocities, their
  // part of every xi-derivative (200 of the 284 nonzero entries at M = 3)
  // and the constant extensions C0 q^0, C0 x^0 (the initial tau > 0 values)
  // are formed once.
  double qe[L1][4], xe[L1][2], V[L][2];
  for (int k = 0; k < L1; ++k) {
    for (int v = 0; v < 4; ++v) qe[k][v] = q[L0 + k][v];
    for (int a = 0; a < 2; ++a) xe[k][a] = x[L0 + k][a];
  }
  double c0[L][2][14];  // per node and direction: d x (2), d q (4), d F (2 x 4) over tau = 0 nodes
  {
    double F0[L0][2][4];
    for (int l = 0; l < L0; ++l) ale_flux(q[l], t.gamma, t.mode, F0[l], V[l]);
    for (int n = 0; n < L; ++n)
      for (int e = 0; e < 2; ++e) {
        double* c = c0[n][e];
        for (int m = 0; m < 14; ++m) c[m] = 0.0;
        for (int j = 0; j < t.nnz0[e][n]; ++j) {
          const int l = t.col[e][n][j];
          const double dd = t.val[e][n][j];
          for (int a2 = 0; a2 < 2; ++a2) c[a2] += dd * x[l][a2];
          for (int v = 0; v < 4; ++v) {
            c[2 + v] += dd * q[l][v];
            c[6 + v] += dd * F0[l][0][v];
            c[10 + v] += dd * F0[l][1][v];
          }
        }
      }
  }
  for (int it = 0; it < niter; ++it) {
    double F[L1][2][4];
    for (int l = L0; l < L; ++l) ale_flux(q[l], t.gamma, t.mode, F[l - L0], V[l]);
    double H[L][4];
    for (int n = 0; n < L; ++n) {
      // xi-derivatives at node n of the interpolants of x, q and F: the cached
      // tau = 0 part plus one pass over the remaining nonzero entries
      double dx[2][2], dq[2][4], df[2][2][4];
      for (int e = 0; e < 2; ++e) {
        const double* c = c0[n][e];
        for (int a2 = 0; a2 < 2; ++a2) dx[e][a2] = c[a2];
        for (int v = 0; v < 4; ++v) {
          dq[e][v] = c[2 + v];
          df[e][0][v] = c[6 + v];
          df[e][1][v] = c[10 + v];
        }
        const int cnt = t.nnz[e][n];
        for (int j = t.nnz0[e][n]; j < cnt; ++j) {
          const int l = t.col[e][n][j];
          const double dd = t.val[e][n][j];
          for (int a2 = 0; a2 < 2; ++a2) dx[e][a2] += dd * x[l][a2];
          for (int v = 0; v < 4; ++v) {
            dq[e][v] += dd * q[l][v];
            df[e][0][v] += dd * F[l - L0][0][v];
            df[e][1][v] += dd * F[l - L0][1][v];
          }
        }
      }
      // d x / d xi of the isoparametric map at node n (J[a][e] = dx[e][a]) and its inverse
      const double idet = 1.0 / (dx[0][0] * dx[1][1] - dx[1][0] * dx[0][1]);
      const double Ji[2][2] = {{dx[1][1] * idet, -dx[1][0] * idet}, {-dx[0][1] * idet, dx[0][0] * idet}};
      double dxidt[2];
      for (int e = 0; e < 2; ++e) dxidt[e] = -(Ji[e][0] * V[n][0] + Ji[e][1] * V[n][1]);
      for (int v = 0; v < 4; ++v) {
        double h = 0.0;
        for (int e = 0; e < 2; ++e) h += dq[e][v] * dxidt[e] + Ji[e][0] * df[e][0][v] + Ji[e][1] * df[e][1][v];
        H[n][v] = h;
      }
    }
    for (int k = 0; k < L1; ++k) {
      for (int v = 0; v < 4; ++v) {
        double g = 0.0;
        for (int l = 0; l < L; ++l) g += t.Gal[k][l] * H[l][v];
        q[L0 + k][v] = qe[k][v] - dt * g;
      }
      for (int a2 = 0; a2 < 2; ++a2) {
        double g = 0.0;
        for (int l = 0; l < L; ++l) g += t.Gal[k][l] * V[l][a2];
        x[L0 + k][a2] = xe[k][a2] + dt * g;
      }
    }
  }
  double qb[4];
  for (int v = 0; v < 4; ++v) qb[v] = Q[v * N + i];
  if (t.pos) {
    // fallback: a tau > 0 node inadmissible or outside [1/2 min, 2 max] of
    // the tau = 0 nodes' density and pressure (a Picard iteration with V = v
    // can stop on large positive oscillations in a cell cut by a shock)
    double r0 = 1e300, r1 = -1e300, p0 = 1e300, p1 = -1e300;
    for (int l = 0; l < L0; ++l) {
      const double pl = pressure(q[l], t.gamma);
      r0 = fmin(r0, q[l][0]);
      r1 = fmax(r1, q[l][0]);
      p0 = fmin(p0, pl);
      p1 = fmax(p1, pl);
    }
    bool ok = true;
    for (int l = L0; l < L; ++l) {
      const double pl = pressure(q[l], t.gamma);
      ok = ok && admissible(q[l], t.gamma) && q[l][0] >= 0.5 * r0 && q[l][0] <= 2.0 * r1 && pl >= 0.5 * p0 &&
           pl <= 2.0 * p1;
    }
    if (!ok)
      for (int l = 0; l < L; ++l)
        for (int v = 0; v < 4; ++v) q[l][v] = qb[v];
  }
  for (int l = 0; l < L; ++l) {
    for (int v = 0; v < 4; ++v) qhat[(i * L + l) * 4 + v] = q[l][v];
    const double ir = 1.0 / q[l][0];
    V[l][0] = t.mode == CWENO_MOTION_LAGRANGE ? q[l][1] * ir : 0.0;
    V[l][1] = t.mode == CWENO_MOTION_LAGRANGE ? q[l][2] * ir : 0.0;
  }
  const double mu = qb[0] * vol[i];
  for (int k = 0; k < 3; ++k) {
    for (int a = 0; a < 2; ++a) {
      double s = 0.0;
      for (int l = 0; l < L; ++l) s += t.Wv[k][l] * V[l][a];
      vcon[(i * 3 + k) * 3 + a] = mu * s;
    }
    vcon[(i * 3 + k) * 3 + 2] = mu;
  }
}

// FP32-mixed form of k_ale_pred: the same iteration in single precision on
// deviations — of the state from the cell average Q_i, of the node positions
// from the cell's first vertex, of the nodal fluxes from the flux of the
// cell average (rounded once to FP32) — so that the xi-derivatives of a
// constant state are exactly zero and positions keep FP32 accuracy relative
// to the cell.  The mesh velocity uses the absolute nodal state.  Writes the
// state deviations q_hat - Q_i (N x L x 4, FP32) and, per vertex of the
// cell, (mu V_kj, mu) in FP64.
__device__ __forceinline__ void ale_flux32(const float* q, float gamma, int mode, float F[2][4], float V[2]) {
  const float ir = 1.0f / q[0], u = q[1] * ir, vv = q[2] * ir;
  const float p = (gamma - 1.0f) * (q[3] - 0.5f * (q[1] * u + q[2] * vv));
  F[0][0] = q[1];
  F[0][1] = q[1] * u + p;
  F[0][2] = q[2] * u;
  F[0][3] = u * (q[3] + p);
  F[1][0] = q[2];
  F[1][1] = q[1] * vv;
  F[1][2] = q[2] * vv + p;
  F[1][3] = vv * (q[3] + p);
  V[0] = mode == CWENO_MOTION_LAGRANGE ? u : 0.0f;
  V[1] = mode == CWENO_MOTION_LAGRANGE ? vv : 0.0f;
}

__device__ __forceinline__ bool admissible32(const float* q, float g) {
  bool fin = isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]);
  return fin && q[0] > 0.0f && (g - 1.0f) * (q[3] - 0.5f * (q[1] * q[1] + q[2] * q[2]) / q[0]) > 0.0f;
}

template <int M>
__global__ void __launch_bounds__(128) k_ale_pred32(const __grid_constant__ AleTab32 t, const double* __restrict__ w,
                                                    const double* __restrict__ Q, const double* __restrict__ X,
                                                    const double* __restrict__ vol, int64_t N, int niter,
                                                    double dt_fixed, double cfl, const unsigned long long* dtmin,
                                                    float* __restrict__ qhat, double* __restrict__ vcon) {
  constexpr int L = lcal2(M), L0 = mcal2(M), L1 = L - L0;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float dt = (float)step_dt(dt_fixed, cfl, dtmin);
  double Qd[4];
  float qb[4];
  for (int v = 0; v < 4; ++v) {
    Qd[v] = Q[v * N + i];
    qb[v] = (float)Qd[v];
  }
  float q[L][4], x[L][2];
  for (int n = 0; n < L0; ++n)
    for (int v = 0; v < 4; ++v) q[n][v] = (float)(w[(i * L0 + n) * 4 + v] - Qd[v]);
  for (int k = 0; k < L1; ++k)
    for (int v = 0; v < 4; ++v) {
      float s = 0.0f;
      for (int n = 0; n < L0; ++n) s += t.C0[k][n] * q[n][v];
      q[L0 + k][v] = s;
    }
  const double* Xi = X + i * 9;
  float E[2][2];  // edge vectors X1 - X0, X2 - X0
  for (int a = 0; a < 2; ++a) {
    E[0][a] = (float)(Xi[3 + a] - Xi[a]);
    E[1][a] = (float)(Xi[6 + a] - Xi[a]);
  }
  for (int l = 0; l < L; ++l)
    for (int a = 0; a < 2; ++a) x[l][a] = E[0][a] * t.node[l][0] + E[1][a] * t.node[l][1];
  float Fb[2][4], Vb[2];
  ale_flux32(qb, t.gamma, t.mode, Fb, Vb);
  float qe[L1][4], xe[L1][2], V[L][2];
  for (int k = 0; k < L1; ++k) {
    for (int v = 0; v < 4; ++v) qe[k][v] = q[L0 + k][v];
    for (int a = 0; a < 2; ++a) xe[k][a] = x[L0 + k][a];
  }
  auto nodal_flux = [&](const float* dq, float F[2][4], float* Vn) {
    float qa[4];
    for (int v = 0; v < 4; ++v) qa[v] = qb[v] + dq[v];
    ale_flux32(qa, t.gamma, t.mode, F, Vn);
    for (int e = 0; e < 2; ++e)
      for (int v = 0; v < 4; ++v) F[e][v] -= Fb[e][v];
  };
  float c0[L][2][14];  // per node and direction: d x (2), d q (4), d F (2 x 4) over tau = 0 nodes
  {
    float F0[L0][2][4];
    for (int l = 0; l < L0; ++l) nodal_flux(q[l], F0[l], V[l]);
    for (int n = 0; n < L; ++n)
      for (int e = 0; e < 2; ++e) {
        float* c = c0[n][e];
        for (int m = 0; m < 14; ++m) c[m] = 0.0f;
        for (int j = 0; j < t.nnz0[e][n]; ++j) {
          const int l = t.col[e][n][j];
          const float dd = t.val[e][n][j];
          for (int a2 = 0; a2 < 2; ++a2) c[a2] += dd * x[l][a2];
          for (int v = 0; v < 4; ++v) {
            c[2 + v] += dd * q[l][v];
            c[6 + v] += dd * F0[l][0][v];
            c[10 + v] += dd * F0[l][1][v];
          }
        }
      }
  }
  for (int it = 0; it < niter; ++it) {
    float F[L1][2][4];
    for (int l = L0; l < L; ++l) nodal_flux(q[l], F[l - L0], V[l]);
    float H[L][4];
    for (int n = 0; n < L; ++n) {
      float dx[2][2], dq[2][4], df[2][2][4];
      for (int e = 0; e < 2; ++e) {
        const float* c = c0[n][e];
        for (int a2 = 0; a2 < 2; ++a2) dx[e][a2] = c[a2];
        for (int v = 0; v < 4; ++v) {
          dq[e][v] = c[2 + v];
          df[e][0][v] = c[6 + v];
          df[e][1][v] = c[10 + v];
        }
        const int cnt = t.nnz[e][n];
        for (int j = t.nnz0[e][n]; j < cnt; ++j) {
          const int l = t.col[e][n][j];
          const float dd = t.val[e][n][j];
          for (int a2 = 0; a2 < 2; ++a2) dx[e][a2] += dd * x[l][a2];
          for (int v = 0; v < 4; ++v) {
            dq[e][v] += dd * q[l][v];
            df[e][0][v] += dd * F[l - L0][0][v];
            df[e][1][v] += dd * F[l - L0][1][v];
          }
        }
      }
      const float idet = 1.0f / (dx[0][0] * dx[1][1] - dx[1][0] * dx[0][1]);
      const float Ji[2][2] = {{dx[1][1] * idet, -dx[1][0] * idet}, {-dx[0][1] * idet, dx[0][0] * idet}};
      float dxidt[2];
      for (int e = 0; e < 2; ++e) dxidt[e] = -(Ji[e][0] * V[n][0] + Ji[e][1] * V[n][1]);
      for (int v = 0; v < 4; ++v) {
        float h = 0.0f;
        for (int e = 0; e < 2; ++e) h += dq[e][v] * dxidt[e] + Ji[e][0] * df[e][0][v] + Ji[e][1] * df[e][1][v];
        H[n][v] = h;
      }
    }
    for (int k = 0; k < L1; ++k) {
      for (int v = 0; v < 4; ++v) {
        float g = 0.0f;
        for (int l = 0; l < L; ++l) g += t.Gal[k][l] * H[l][v];
        q[L0 + k][v] = qe[k][v] - dt * g;
      }
      for (int a2 = 0; a2 < 2; ++a2) {
        float g = 0.0f;
        for (int l = 0; l < L; ++l) g += t.Gal[k][l] * V[l][a2];
        x[L0 + k][a2] = xe[k][a2] + dt * g;
      }
    }
  }
  if (t.pos) {  // the fallback rule of k_ale_pred, on absolute states
    auto pres = [&](const float* qa) {
      return (t.gamma - 1.0f) * (qa[3] - 0.5f * (qa[1] * qa[1] + qa[2] * qa[2]) / qa[0]);
    };
    float r0 = 3e38f, r1 = -3e38f, p0 = 3e38f, p1 = -3e38f;
    for (int l = 0; l < L0; ++l) {
      float qa[4];
      for (int v = 0; v < 4; ++v) qa[v] = qb[v] + q[l][v];
      const float pl = pres(qa);
      r0 = fminf(r0, qa[0]);
      r1 = fmaxf(r1, qa[0]);
      p0 = fminf(p0, pl);
      p1 = fmaxf(p1, pl);
    }
    bool ok = true;
    for (int l = L0; l < L; ++l) {
      float qa[4];
      for (int v = 0; v < 4; ++v) qa[v] = qb[v] + q[l][v];
      const float pl = pres(qa);
      ok = ok && admissible32(qa, t.gamma) && qa[0] >= 0.5f * r0 && qa[0] <= 2.0f * r1 && pl >= 0.5f * p0 &&
           pl <= 2.0f * p1;
    }
    if (!ok)
      for (int l = 0; l < L; ++l)
        for (int v = 0; v < 4; ++v) q[l][v] = 0.0f;
  }
  for (int l = 0; l < L; ++l) {
    for (int v = 0; v < 4; ++v) qhat[(i * L + l) * 4 + v] = q[l][v];
    const float ir = 1.0f / (qb[0] + q[l][0]);
    V[l][0] = t.mode == CWENO_MOTION_LAGRANGE ? (qb[1] + q[l][1]) * ir : 0.0f;
    V[l][1] = t.mode == CWENO_MOTION_LAGRANGE ? (qb[2] + q[l][2]) * ir : 0.0f;
  }
  const double mu = Qd[0] * vol[i];
  for (int k = 0; k < 3; ++k) {
    for (int a = 0; a < 2; ++a) {
      float s = 0.0f;
      for (int l = 0; l < L; ++l) s += t.Wv[k][l] * V[l][a];
      vcon[(i * 3 + k) * 3 + a] = mu * (double)s;
    }
    vcon[(i * 3 + k) * 3 + 2] = mu;
  }
}

// ------------------------------------------------------------- nodal solver
// One thread per vertex: V_k = sum mu V_kj / sum mu over the incident cells
// (entries ent[start[g] .. start[g+1]) = cell * 3 + local vertex, in
// increasing caller cell order), X^{n+1} = X^n + dt V_k.
__global__ void __launch_bounds__(256) k_ale_nodes(const int32_t* __restrict__ start, const int32_t* __restrict__ ent,
                                                   const double* __restrict__ vcon, const double* __restrict__ Xv,
                                                   int64_t nvert, double dt_fixed, double cfl,
                                                   const unsigned long long* dtmin, double* __restrict__ Xv1) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nvert) return;
  const double dt = step_dt(dt_fixed, cfl, dtmin);
  double ax = 0.0, ay = 0.0, mu = 0.0;
  for (int32_t e = start[g]; e < start[g + 1]; ++e) {
    const double* c = vcon + (int64_t)ent[e] * 3;
    ax += c[0];
    ay += c[1];
    mu += c[2];
  }
  Xv1[g * 2] = mu > 0.0 ? Xv[g * 2] + dt * (ax / mu) : Xv[g * 2];
  Xv1[g * 2 + 1] = mu > 0.0 ? Xv[g * 2 + 1] + dt * (ay / mu) : Xv[g * 2 + 1];
}

// -------------------------------------------------------------------- faces
struct FaceGeo {
  double A0[2], B0[2], A1[2], B1[2];
};

// Space-time normal (x, y, t) at (chi, tau) of the face moving on straight
// lines from A0-B0 to A1-B1 over dt: cross product of d x/d chi = (e, 0) and
// d x/d tau = (w, dt), the cofactor expansion of Eq. (detChi).
__device__ __forceinline__ void st_normal(const FaceGeo& f, double chi, double tau, double dt, double* n) {
  double e[2], w[2];
  for (int a = 0; a < 2; ++a) {
    e[a] = (1.0 - tau) * (f.B0[a] - f.A0[a]) + tau * (f.B1[a] - f.A1[a]);
    w[a] = (1.0 - chi) * (f.A1[a] - f.A0[a]) + chi * (f.B1[a] - f.B0[a]);
  }
  n[0] = e[1] * dt;
  n[1] = -(e[0] * dt);
  n[2] = e[0] * w[1] - e[1] * w[0];
}

// One thread per face: the integral over the lateral space-time face of the
// Rusanov flux, (F~(q+) + F~(q-)).n~/2 - s_max (q+ - q-)/2 with F~ = (f, g, Q)
// and s_max = |n~_x| max(|v.n - V.n| + c) over both sides, V.n = -n~_t/|n~_x|;
// Gauss-Legendre in chi and tau.  Traces from the face basis table of each
// side's face code (points ordered from the lower to the higher global
// vertex id).  Transmissive boundary: q+ = q-.  Positivity switch: an
// inadmissible trace is replaced by that side's cell average.
template <int M>
__global__ void __launch_bounds__(128) k_ale_flux(const __grid_constant__ AleTab t, const double* __restrict__ ftab,
                                                  const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
                                                  const uint8_t* __restrict__ codeL, const uint8_t* __restrict__ codeR,
                                                  const int32_t* __restrict__ gv, const double* __restrict__ shift,
                                                  const double* __restrict__ Xv, const double* __restrict__ Xv1,
                                                  const double* __restrict__ bary, const double* __restrict__ qhat,
                                                  const double* __restrict__ Q, int64_t N, int64_t F,
                                                  double dt_fixed, double cfl, const unsigned long long* dtmin,
                                                  double* __restrict__ G) {
  constexpr int L = lcal2(M), NQ = M + 1;
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double dt = step_dt(dt_fixed, cfl, dtmin);
  const int64_t cl = fL[f], cr = fR[f];
  const int kL = codeL[f], kR = cr >= 0 ? codeR[f] : 0;
  const int lf = kL / 2;
  int la = (lf + 1) % 3, lb = (lf + 2) % 3;
  int64_t ga = gv[la * N + cl], gb = gv[lb * N + cl];
  if (ga > gb) {
    const int64_t tg = ga;
    ga = gb;
    gb = tg;
    const int tl = la;
    la = lb;
    lb = tl;
  }
  FaceGeo fg;
  for (int a = 0; a < 2; ++a) {
    const double sa = shift[(la * 2 + a) * N + cl], sb = shift[(lb * 2 + a) * N + cl];
    fg.A0[a] = Xv[ga * 2 + a] + sa;
    fg.B0[a] = Xv[gb * 2 + a] + sb;
    fg.A1[a] = Xv1[ga * 2 + a] + sa;
    fg.B1[a] = Xv1[gb * 2 + a] + sb;
  }
  double n0[3];
  st_normal(fg, 0.0, 0.0, dt, n0);
  const double sgn =
      n0[0] * (fg.A0[0] - bary[cl * 3]) + n0[1] * (fg.A0[1] - bary[cl * 3 + 1]) > 0.0 ? 1.0 : -1.0;
  double qbL[4], qbR[4];
  for (int v = 0; v < 4; ++v) {
    qbL[v] = Q[v * N + cl];
    qbR[v] = cr >= 0 ? Q[v * N + cr] : qbL[v];
  }
  const double* qL = qhat + cl * L * 4;
  const double* qR = qhat + (cr >= 0 ? cr : cl) * L * 4;
  double acc[4] = {0, 0, 0, 0};
  for (int qp = 0; qp < NQ; ++qp)
    for (int tt = 0; tt < NQ; ++tt) {
      const double* bL = ftab + ((int64_t)(kL * NQ + tt) * NQ + qp) * L;
      const double* bR = ftab + ((int64_t)(kR * NQ + tt) * NQ + qp) * L;
      double qm[4] = {0, 0, 0, 0}, qq[4] = {0, 0, 0, 0};
      for (int l = 0; l < L; ++l)
        for (int v = 0; v < 4; ++v) {
          qm[v] += bL[l] * qL[l * 4 + v];
          qq[v] += bR[l] * qR[l * 4 + v];
        }
      if (cr < 0)
        for (int v = 0; v < 4; ++v) qq[v] = qm[v];
      if (t.pos) {
        if (!admissible(qm, t.gamma))
          for (int v = 0; v < 4; ++v) qm[v] = qbL[v];
        if (!admissible(qq, t.gamma))
          for (int v = 0; v < 4; ++v) qq[v] = qbR[v];
      }
      double n[3];
      st_normal(fg, t.chi[qp], t.tq[tt], dt, n);
      for (int a = 0; a < 3; ++a) n[a] *= sgn;
      const double nx = sqrt(n[0] * n[0] + n[1] * n[1]), inx = 1.0 / nx;
      const double un[2] = {n[0] * inx, n[1] * inx};
      const double Vn = -n[2] * inx;
      double sm = 0.0, fsum[4];
      const double* sides[2] = {qm, qq};
      for (int v = 0; v < 4; ++v) fsum[v] = 0.0;
      for (int s = 0; s < 2; ++s) {
        const double* z = sides[s];
        const double ir = 1.0 / z[0], u = z[1] * ir, vv = z[2] * ir;
        const double p = (t.gamma - 1.0) * (z[3] - 0.5 * (z[1] * u + z[2] * vv));
        const double c = sqrt(fmax(0.0, t.gamma * p * ir));
        const double vn = u * un[0] + vv * un[1];
        sm = fmax(sm, fabs(vn - Vn) + c);
        fsum[0] += z[1] * n[0] + z[2] * n[1];
        fsum[1] += (z[1] * u + p) * n[0] + z[1] * vv * n[1];
        fsum[2] += z[2] * u * n[0] + (z[2] * vv + p) * n[1];
        fsum[3] += u * (z[3] + p) * n[0] + vv * (z[3] + p) * n[1];
      }
      sm *= nx;
      const double wgt = t.wq[qp] * t.wt[tt];
      for (int v = 0; v < 4; ++v)
        acc[v] += wgt * (0.5 * fsum[v] + 0.5 * (qm[v] + qq[v]) * n[2] - 0.5 * sm * (qq[v] - qm[v]));
    }
  for (int v = 0; v < 4; ++v) G[v * F + f] = acc[v];
}

// FP32-mixed form of k_ale_flux.  Each side's trace is a deviation from its
// cell average (q_hat in deviations, FP32); the flux, the mesh-motion term
// and the dissipation of the deviations are integrated in FP32 with the
// point normals in FP32.  The cell averages' part, 1/2 (F(Q-) + F(Q+)) . n +
// 1/2 (Q- + Q+) n_t, is integrated exactly in FP64 once per face: the
// space-time normal is bilinear in (chi, tau), so its integral over the
// tensor Gauss rule is its value at (1/2, 1/2).  A constant state therefore
// gives the FP64 face integrals of the FP64 path's geometry, and the
// geometric conservation law closes to FP64 rounding.
__device__ __forceinline__ void euler_xy64(const double* z, double g, double F[2][4]) {
  const double ir = 1.0 / z[0], u = z[1] * ir, vv = z[2] * ir;
  const double p = (g - 1.0) * (z[3] - 0.5 * (z[1] * u + z[2] * vv));
  F[0][0] = z[1];
  F[0][1] = z[1] * u + p;
  F[0][2] = z[2] * u;
  F[0][3] = u * (z[3] + p);
  F[1][0] = z[2];
  F[1][1] = z[1] * vv;
  F[1][2] = z[2] * vv + p;
  F[1][3] = vv * (z[3] + p);
}

template <int M>
__global__ void __launch_bounds__(128) k_ale_flux32(const __grid_constant__ AleTab32 t, double gamma64,
                                                    const float* __restrict__ ftab, const int32_t* __restrict__ fL,
                                                    const int32_t* __restrict__ fR, const uint8_t* __restrict__ codeL,
                                                    const uint8_t* __restrict__ codeR, const int32_t* __restrict__ gv,
                                                    const double* __restrict__ shift, const double* __restrict__ Xv,
                                                    const double* __restrict__ Xv1, const double* __restrict__ bary,
                                                    const float* __restrict__ qhat, const double* __restrict__ Q,
                                                    int64_t N, int64_t F, double dt_fixed, double cfl,
                                                    const unsigned long long* dtmin, double* __restrict__ G) {
  constexpr int L = lcal2(M), NQ = M + 1;
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double dt = step_dt(dt_fixed, cfl, dtmin);
  const int64_t cl = fL[f], cr = fR[f];
  const int kL = codeL[f], kR = cr >= 0 ? codeR[f] : 0;
  const int lf = kL / 2;
  int la = (lf + 1) % 3, lb = (lf + 2) % 3;
  int64_t ga = gv[la * N + cl], gb = gv[lb * N + cl];
  if (ga > gb) {
    const int64_t tg = ga;
    ga = gb;
    gb = tg;
    const int tl = la;
    la = lb;
    lb = tl;
  }
  FaceGeo fg;
  for (int a = 0; a < 2; ++a) {
    const double sa = shift[(la * 2 + a) * N + cl], sb = shift[(lb * 2 + a) * N + cl];
    fg.A0[a] = Xv[ga * 2 + a] + sa;
    fg.B0[a] = Xv[gb * 2 + a] + sb;
    fg.A1[a] = Xv1[ga * 2 + a] + sa;
    fg.B1[a] = Xv1[gb * 2 + a] + sb;
  }
  double n0[3], nbar[3];
  st_normal(fg, 0.0, 0.0, dt, n0);
  const double sgn =
      n0[0] * (fg.A0[0] - bary[cl * 3]) + n0[1] * (fg.A0[1] - bary[cl * 3 + 1]) > 0.0 ? 1.0 : -1.0;
  st_normal(fg, 0.5, 0.5, dt, nbar);
  // edge and displacement vectors of the moving face in FP32 (differences in FP64)
  float eA[2], eB[2], wA[2], wB[2];
  for (int a = 0; a < 2; ++a) {
    eA[a] = (float)(fg.B0[a] - fg.A0[a]);
    eB[a] = (float)(fg.B1[a] - fg.A1[a]);
    wA[a] = (float)(fg.A1[a] - fg.A0[a]);
    wB[a] = (float)(fg.B1[a] - fg.B0[a]);
  }
  const float sg = (float)sgn, dt32 = (float)dt;
  double QL[4], QR[4];
  float qbL[4], qbR[4], dQ[4];
  for (int v = 0; v < 4; ++v) {
    QL[v] = Q[v * N + cl];
    QR[v] = cr >= 0 ? Q[v * N + cr] : QL[v];
    qbL[v] = (float)QL[v];
    qbR[v] = (float)QR[v];
    dQ[v] = (float)(QR[v] - QL[v]);
  }
  float FbL[2][4], FbR[2][4], Vd[2];
  ale_flux32(qbL, t.gamma, CWENO_MOTION_FIXED, FbL, Vd);
  ale_flux32(qbR, t.gamma, CWENO_MOTION_FIXED, FbR, Vd);
  const float* qL = qhat + cl * L * 4;
  const float* qR = qhat + (cr >= 0 ? cr : cl) * L * 4;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int qp = 0; qp < NQ; ++qp)
    for (int tt = 0; tt < NQ; ++tt) {
      const float* bL = ftab + ((int64_t)(kL * NQ + tt) * NQ + qp) * L;
      const float* bR = ftab + ((int64_t)(kR * NQ + tt) * NQ + qp) * L;
      float dm[4] = {0.f, 0.f, 0.f, 0.f}, dp[4] = {0.f, 0.f, 0.f, 0.f};
      for (int l = 0; l < L; ++l)
        for (int v = 0; v < 4; ++v) {
          dm[v] += bL[l] * qL[l * 4 + v];
          dp[v] += bR[l] * qR[l * 4 + v];
        }
      if (cr < 0)
        for (int v = 0; v < 4; ++v) dp[v] = dm[v];
      float qm[4], qq[4];
      for (int v = 0; v < 4; ++v) {
        qm[v] = qbL[v] + dm[v];
        qq[v] = qbR[v] + dp[v];
      }
      if (t.pos) {
        if (!admissible32(qm, t.gamma))
          for (int v = 0; v < 4; ++v) {
            qm[v] = qbL[v];
            dm[v] = 0.f;
          }
        if (!admissible32(qq, t.gamma))
          for (int v = 0; v < 4; ++v) {
            qq[v] = qbR[v];
            dp[v] = 0.f;
          }
      }
      // space-time normal at (chi, tau), Eq. (detChi), in FP32
      const float chi = t.chi[qp], tau = t.tq[tt];
      float e[2], wv[2];
      for (int a = 0; a < 2; ++a) {
        e[a] = (1.0f - tau) * eA[a] + tau * eB[a];
        wv[a] = (1.0f - chi) * wA[a] + chi * wB[a];
      }
      const float n[3] = {sg * e[1] * dt32, -sg * e[0] * dt32, sg * (e[0] * wv[1] - e[1] * wv[0])};
      const float nx = sqrtf(n[0] * n[0] + n[1] * n[1]), inx = 1.0f / nx;
      const float un[2] = {n[0] * inx, n[1] * inx};
      const float Vn = -n[2] * inx;
      float sm = 0.0f, dfs[4] = {0.f, 0.f, 0.f, 0.f};
      const float* sides[2] = {qm, qq};
      for (int s = 0; s < 2; ++s) {
        const float* z = sides[s];
        float Fz[2][4], Vz[2];
        ale_flux32(z, t.gamma, CWENO_MOTION_FIXED, Fz, Vz);
        const float ir = 1.0f / z[0], u = z[1] * ir, vv = z[2] * ir;
        const float p = (t.gamma - 1.0f) * (z[3] - 0.5f * (z[1] * u + z[2] * vv));
        const float c = sqrtf(fmaxf(0.0f, t.gamma * p * ir));
        sm = fmaxf(sm, fabsf(u * un[0] + vv * un[1] - Vn) + c);
        const float(*Fb)[4] = s == 0 ? FbL : FbR;
        for (int v = 0; v < 4; ++v) dfs[v] += (Fz[0][v] - Fb[0][v]) * n[0] + (Fz[1][v] - Fb[1][v]) * n[1];
      }
      sm *= nx;
      const float wgt = t.wq[qp] * t.wt[tt];
      for (int v = 0; v < 4; ++v)
        acc[v] += wgt * (0.5f * dfs[v] + 0.5f * (dm[v] + dp[v]) * n[2] - 0.5f * sm * (dQ[v] + dp[v] - dm[v]));
    }
  // the cell averages' part, in FP64 with the integrated normal
  double FL[2][4], FR[2][4];
  euler_xy64(QL, gamma64, FL);
  euler_xy64(QR, gamma64, FR);
  for (int a = 0; a < 3; ++a) nbar[a] *= sgn;
  for (int v = 0; v < 4; ++v)
    G[v * F + f] = (double)acc[v] + 0.5 * ((FL[0][v] + FR[0][v]) * nbar[0] + (FL[1][v] + FR[1][v]) * nbar[1]) +
                   0.5 * (QL[v] + QR[v]) * nbar[2];
}

// ------------------------------------------------------------------- update
// Eq. (PDEfinal) with the face integrals (outward from fL), new volume from
// the new vertices; status bit on an inadmissible result or a tangled cell.
__global__ void __launch_bounds__(256) k_ale_update(const int32_t* __restrict__ cellface, const double* __restrict__ G,
                                                    const int32_t* __restrict__ gv, const double* __restrict__ shift,
                                                    const double* __restrict__ Xv1, const double* __restrict__ vol0,
                                                    int64_t N, int64_t F, double gamma, double dt_fixed, double cfl,
                                                    const unsigned long long* dtmin, double* __restrict__ Q,
                                                    float* __restrict__ Qp, double* time, int* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *time += step_dt(dt_fixed, cfl, dtmin);
  if (i >= N) return;
  double acc[4] = {0, 0, 0, 0};
  for (int k = 0; k < 3; ++k) {
    const int32_t cf = cellface[k * N + i];
    const int64_t f = cf >> 1;
    const double s = (cf & 1) ? -1.0 : 1.0;
    for (int v = 0; v < 4; ++v) acc[v] += s * G[v * F + f];
  }
  double P[3][2];
  for (int k = 0; k < 3; ++k) {
    const int64_t g = gv[k * N + i];
    for (int a = 0; a < 2; ++a) P[k][a] = Xv1[g * 2 + a] + shift[(k * 2 + a) * N + i];
  }
  const double det = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]);
  const double v1 = det / 2.0, v0 = vol0[i];
  double q[4];
  for (int v = 0; v < 4; ++v) {
    q[v] = (v0 * Q[v * N + i] - acc[v]) / v1;
    Q[v * N + i] = q[v];
  }
  if (Qp) {  // FP32-mixed: the state's FP32 pairs for the reconstruction (layout.h)
    float pr[8];
    for (int v = 0; v < 4; ++v) split_hilo(q[v], pr[2 * v], pr[2 * v + 1]);
    float4* dst = reinterpret_cast<float4*>(Qp) + i * 2;
    dst[0] = make_float4(pr[0], pr[1], pr[2], pr[3]);
    dst[1] = make_float4(pr[4], pr[5], pr[6], pr[7]);
  }
  if (!(v1 > 0.0) || !admissible(q, gamma)) atomicOr(status, 1);
}

}  // namespace

#include "ale3.cuh"

// ---------------------------------------------------------------- host side
struct Ale {
  int d = 2;
  int M = 1;
  MeshHost slim;  // d, nc, periodicity: what the device matrices refresh reads
  int64_t nvert = 0;
  AleTab tab;
  AleTab3 tab3;  // tetrahedra
  AleTab3f tab3f;
  AleDer3* der3 = nullptr;  // device copies of the nodal derivative tables
  AleDer3f* der3f = nullptr;
  double *Xv = nullptr, *Xv1 = nullptr, *shift = nullptr, *X = nullptr, *bary = nullptr, *vol = nullptr;
  double *w = nullptr, *qhat = nullptr, *vcon = nullptr, *G = nullptr, *ftab = nullptr;
  // FP32-mixed: tables, face basis and predictor deviations in FP32
  bool fp32 = false;
  AleTab32 tab32;
  float *ftab32 = nullptr, *qhat32 = nullptr;
  int32_t *gv = nullptr, *start = nullptr, *ent = nullptr, *ident = nullptr;
  int* bad = nullptr;
  bool fresh = false;
  std::vector<void*> allocs;
  size_t bytes = 0;
  ~Ale() {
    for (void* p : allocs) cudaFree(p);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t n, cudaStream_t st) {
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, sizeof(T) * std::max<size_t>(n, 1), st);
    if (e != cudaSuccess) return e;
    allocs.push_back(q);
    bytes += sizeof(T) * n;
    *p = (T*)q;
    return cudaSuccess;
  }
  template <typename T>
  cudaError_t put(T** p, const std::vector<T>& h, cudaStream_t st) {
    cudaError_t e = alloc(p, h.size(), st);
    if (e != cudaSuccess || h.empty()) return e;
    e = cudaMemcpyAsync(*p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);  // h is a host temporary
  }
};

namespace {

#define ACK(x)                                               \
  do {                                                       \
    cudaError_t e_ = (x);                                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x);         \
  } while (0)

unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <int M>
cudaError_t launch_pred(Ale& A, cweno_solver* s, double dtf, cudaStream_t st) {
  const DevState& ds = s->ds;
  if (A.fp32)
    k_ale_pred32<M><<<nblk(ds.N, 128), 128, 0, st>>>(A.tab32, A.w, ds.Q, A.X, A.vol, ds.N, s->ph.niter, dtf,
                                                      s->prm.cfl, ds.dtmin, A.qhat32, A.vcon);
  else
    k_ale_pred<M><<<nblk(ds.N, 128), 128, 0, st>>>(A.tab, A.w, ds.Q, A.X, A.vol, ds.N, s->ph.niter, dtf,
                                                    s->prm.cfl, ds.dtmin, A.qhat, A.vcon);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_flux(Ale& A, cweno_solver* s, double dtf, cudaStream_t st) {
  const DevState& ds = s->ds;
  if (A.fp32) {
    k_ale_flux32<M><<<nblk(ds.F, 128), 128, 0, st>>>(A.tab32, s->prm.gamma, A.ftab32, ds.fL, ds.fR, ds.codeL,
                                                      ds.codeR, A.gv, A.shift, A.Xv, A.Xv1, A.bary, A.qhat32, ds.Q,
                                                      ds.N, ds.F, dtf, s->prm.cfl, ds.dtmin, A.G);
    return cudaGetLastError();
  }
  k_ale_flux<M><<<nblk(ds.F, 128), 128, 0, st>>>(A.tab, A.ftab, ds.fL, ds.fR, ds.codeL, ds.codeR, A.gv, A.shift,
                                                  A.Xv, A.Xv1, A.bary, A.qhat, ds.Q, ds.N, ds.F, dtf, s->prm.cfl,
                                                  ds.dtmin, A.G);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_pred3(Ale& A, cweno_solver* s, double dtf, cudaStream_t st) {
  const DevState& ds = s->ds;
  if (A.fp32)
    k_ale_pred3_32<M><<<nblk(ds.N, 128), 128, 0, st>>>(A.tab3f, A.der3f, A.w, ds.Q, A.X, A.vol, ds.N, s->ph.niter,
                                                        dtf, s->prm.cfl, ds.dtmin, A.qhat32, A.vcon);
  else
    k_ale_pred3<M><<<nblk(ds.N, 128), 128, 0, st>>>(A.tab3, A.der3, A.w, ds.Q, A.X, A.vol, ds.N, s->ph.niter, dtf,
                                                     s->prm.cfl, ds.dtmin, A.qhat, A.vcon);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_flux3(Ale& A, cweno_solver* s, double dtf, cudaStream_t st) {
  const DevState& ds = s->ds;
  if (A.fp32)
    k_ale_flux3_32<M><<<nblk(ds.F, 128), 128, 0, st>>>(A.tab3f, s->prm.gamma, A.ftab32, ds.fL, ds.fR, ds.codeL,
                                                        ds.codeR, A.gv, A.shift, A.Xv, A.Xv1, A.bary, A.qhat32, ds.Q,
                                                        ds.N, ds.F, dtf, s->prm.cfl, ds.dtmin, A.G);
  else
    k_ale_flux3<M><<<nblk(ds.F, 128), 128, 0, st>>>(A.tab3, A.ftab, ds.fL, ds.fR, ds.codeL, ds.codeR, A.gv, A.shift,
                                                     A.Xv, A.Xv1, A.bary, A.qhat, ds.Q, ds.N, ds.F, dtf, s->prm.cfl,
                                                     ds.dtmin, A.G);
  return cudaGetLastError();
}

}  // namespace

// Per-step rebuild for a moving mesh: this unit keeps FMA contraction (the
// matrices change every step; the host setup's exact arithmetic is not needed).
int ale_matrices_device(const MeshHost& m, const RefElem& re, const double* d_X, const double* d_bary,
                        const int32_t* d_sten, const int32_t* d_sec, void* d_R, void* d_Binv, int fp32, int* d_bad,
                        void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  LsqTab tab;
  std::string err;
  if (!make_tab(m, re, tab, err)) return CWENO_EINVAL;
  cudaError_t e = fp32 ? dispatch<float>(m.d, re.M, d_X, d_bary, d_sten, m.nc, tab, d_R, d_bad, st)
                       : dispatch<double>(m.d, re.M, d_X, d_bary, d_sten, m.nc, tab, d_R, d_bad, st);
  if (e == cudaSuccess && m.d == 2) {
    switch (re.M) {
      case 1: e = fp32 ? launch_sectors<2, 1, float>(d_X, d_bary, d_sec, m.nc, tab, (float*)d_Binv, d_bad, st)
                       : launch_sectors<2, 1, double>(d_X, d_bary, d_sec, m.nc, tab, (double*)d_Binv, d_bad, st);
        break;
      case 2: e = fp32 ? launch_sectors<2, 2, float>(d_X, d_bary, d_sec, m.nc, tab, (float*)d_Binv, d_bad, st)
                       : launch_sectors<2, 2, double>(d_X, d_bary, d_sec, m.nc, tab, (double*)d_Binv, d_bad, st);
        break;
      case 3: e = fp32 ? launch_sectors<2, 3, float>(d_X, d_bary, d_sec, m.nc, tab, (float*)d_Binv, d_bad, st)
                       : launch_sectors<2, 3, double>(d_X, d_bary, d_sec, m.nc, tab, (double*)d_Binv, d_bad, st);
        break;
      default: e = cudaErrorInvalidValue;
    }
  } else if (e == cudaSuccess && m.d == 3) {
    switch (re.M) {
      case 1: e = fp32 ? launch_sectors<3, 1, float>(d_X, d_bary, d_sec, m.nc, tab, (float*)d_Binv, d_bad, st)
                       : launch_sectors<3, 1, double>(d_X, d_bary, d_sec, m.nc, tab, (double*)d_Binv, d_bad, st);
        break;
      case 2: e = fp32 ? launch_sectors<3, 2, float>(d_X, d_bary, d_sec, m.nc, tab, (float*)d_Binv, d_bad, st)
                       : launch_sectors<3, 2, double>(d_X, d_bary, d_sec, m.nc, tab, (double*)d_Binv, d_bad, st);
        break;
      case 3: e = fp32 ? launch_sectors<3, 3, float>(d_X, d_bary, d_sec, m.nc, tab, (float*)d_Binv, d_bad, st)
                       : launch_sectors<3, 3, double>(d_X, d_bary, d_sec, m.nc, tab, (double*)d_Binv, d_bad, st);
        break;
      default: e = cudaErrorInvalidValue;
    }
  } else if (e == cudaSuccess) {
    e = cudaErrorInvalidValue;
  }
  return e == cudaSuccess ? CWENO_OK : CWENO_ECUDA;
}

int ale_create3(cweno_solver* s, const MeshHost& m, std::string& err);

int ale_create(cweno_solver* s, const MeshHost& m, std::string& err) {
  if (m.d == 3) return ale_create3(s, m, err);
  const RefElem& re = *s->re;
  if (m.d != 2 || s->pde != CWENO_EULER || re.M > 3 || s->prm.flux != CWENO_FLUX_RUSANOV) {
    err = "moving meshes are built for 2D Euler, order 2..4, Rusanov flux";
    return CWENO_EINVAL;
  }
  auto A = std::make_shared<Ale>();
  cudaStream_t st = s->stream;
  const int64_t N = m.nc, nv = m.nv;
  const int L = re.L, L0 = re.L0, L1 = re.L1;
  A->M = re.M;
  A->nvert = nv;
  A->slim.d = 2;
  A->slim.nc = N;
  for (int a = 0; a < 3; ++a) {
    A->slim.per[a] = m.per[a];
    A->slim.Lper[a] = m.Lper[a];
  }
  // reference tables
  AleTab& t = A->tab;
  std::memset(&t, 0, sizeof(t));
  {
    double dmax = 0.0;
    for (double v : re.Dxi) dmax = std::max(dmax, std::fabs(v));
    for (int e = 0; e < 2; ++e)
      for (int n = 0; n < L; ++n) {
        int c = 0;
        for (int l = 0; l < L; ++l) {
          const double v = re.Dxi[((size_t)e * L + n) * L + l];
          if (std::fabs(v) <= 1e-12 * dmax) continue;  // exact zeros, rounded in extended precision
          t.val[e][n][c] = v;
          t.col[e][n][c] = (uint8_t)l;
          ++c;
          if (l < L0) t.nnz0[e][n] = c;  // columns ascend: tau = 0 nodes first
        }
        t.nnz[e][n] = c;
      }
  }
  for (int k = 0; k < L1; ++k) {
    for (int l = 0; l < L; ++l) t.Gal[k][l] = re.Gal[(size_t)k * L + l];
    for (int n = 0; n < L0; ++n) t.C0[k][n] = re.C0[(size_t)k * L0 + n];
  }
  for (int v = 0; v < 3; ++v)
    for (int l = 0; l < L; ++l) t.Wv[v][l] = re.Wv[(size_t)v * L + l];
  for (int l = 0; l < L; ++l) {
    t.node[l][0] = re.stnode[l][0];
    t.node[l][1] = re.stnode[l][1];
    t.node[l][2] = re.stnode[l][3];
  }
  for (int q = 0; q <= re.M; ++q) {
    t.chi[q] = re.chi[q];
    t.wq[q] = re.wq[q];
    t.wt[q] = re.wt[q];
    t.tq[q] = re.tq[q];
  }
  t.gamma = s->prm.gamma;
  t.mode = s->prm.mesh_motion;
  t.pos = s->prm.positivity;
  // per-cell global vertices and periodic image shifts (the unwrapping of
  // the mesh: image nearest the cell's first vertex), SoA
  std::vector<int32_t> gv((size_t)3 * N);
  std::vector<double> sh((size_t)6 * N, 0.0);
  for (int64_t i = 0; i < N; ++i) {
    const int64_t g0 = m.gv[i * 3];
    for (int k = 0; k < 3; ++k) {
      const int64_t g = m.gv[i * 3 + k];
      gv[(size_t)k * N + i] = (int32_t)g;
      for (int a = 0; a < 2; ++a)
        if (m.per[a] && k > 0)
          sh[(size_t)(k * 2 + a) * N + i] = m.Lper[a] * std::nearbyint((m.xyz[g0 * 2 + a] - m.xyz[g * 2 + a]) / m.Lper[a]);
    }
  }
  // vertex -> (cell, local vertex) incidence, cells in increasing caller order
  std::vector<int32_t> start(nv + 1, 0), ent((size_t)3 * N);
  for (int64_t i = 0; i < N; ++i)
    for (int k = 0; k < 3; ++k) ++start[m.gv[i * 3 + k] + 1];
  for (int64_t g = 0; g < nv; ++g) start[g + 1] += start[g];
  {
    std::vector<int32_t> fill(start.begin(), start.end() - 1);
    for (int64_t u = 0; u < N; ++u) {
      const int64_t i = m.iperm[u];
      for (int k = 0; k < 3; ++k) ent[fill[m.gv[i * 3 + k]]++] = (int32_t)(i * 3 + k);
    }
  }
  std::vector<int32_t> ident(N);
  std::iota(ident.begin(), ident.end(), 0);
  ACK(A->put(&A->gv, gv, st));
  ACK(A->put(&A->shift, sh, st));
  ACK(A->put(&A->start, start, st));
  ACK(A->put(&A->ent, ent, st));
  ACK(A->put(&A->ident, ident, st));
  ACK(A->put(&A->Xv, m.xyz, st));
  ACK(A->put(&A->ftab, re.ftab, st));
  ACK(A->alloc(&A->Xv1, (size_t)nv * 2, st));
  ACK(A->alloc(&A->X, (size_t)N * 9, st));
  ACK(A->alloc(&A->bary, (size_t)N * 3, st));
  ACK(A->alloc(&A->vol, (size_t)N, st));
  ACK(A->alloc(&A->w, (size_t)N * L0 * 4, st));
  ACK(A->alloc(&A->qhat, (size_t)N * L * 4, st));
  ACK(A->alloc(&A->vcon, (size_t)N * 9, st));
  ACK(A->alloc(&A->G, (size_t)4 * m.nf, st));
  ACK(A->alloc(&A->bad, 1, st));
  if (s->prec == CWENO_FP32_MIXED) {
    A->fp32 = true;
    A->tab32 = ale_tab_cast<float>(t);
    std::vector<float> f32(re.ftab.begin(), re.ftab.end());
    ACK(A->put(&A->ftab32, f32, st));
    ACK(A->alloc(&A->qhat32, (size_t)N * L * 4, st));
  }
  const int big = 0x7fffffff;
  ACK(cudaMemcpyAsync(A->bad, &big, sizeof(int), cudaMemcpyHostToDevice, st));
  ACK(cudaStreamSynchronize(st));
  s->bytes += A->bytes;
  s->ale = A;
  return CWENO_OK;
}

// Tetrahedra (M = 1, 2; FP64 or FP32-mixed): tables, vertex incidence,
// periodic shifts and scratch of the moving mesh.
int ale_create3(cweno_solver* s, const MeshHost& m, std::string& err) {
  const RefElem& re = *s->re;
  if (s->pde != CWENO_EULER || re.M < 1 || re.M > 3 || s->prm.flux != CWENO_FLUX_RUSANOV) {
    err = "moving tetrahedral meshes are built for Euler, order 2..4, Rusanov flux";
    return CWENO_EINVAL;
  }
  auto A = std::make_shared<Ale>();
  cudaStream_t st = s->stream;
  const int64_t N = m.nc, nv = m.nv;
  const int L = re.L, L0 = re.L0, L1 = re.L1;
  if (L > kL3 || L0 > kL03 || L1 > kL13 || re.nqs > kNQS3 || re.nqt > kNQT3) {
    err = "moving tetrahedral mesh tables exceed their fixed sizes";
    return CWENO_EINVAL;
  }
  A->d = 3;
  A->M = re.M;
  A->nvert = nv;
  A->slim.d = 3;
  A->slim.nc = N;
  for (int a = 0; a < 3; ++a) {
    A->slim.per[a] = m.per[a];
    A->slim.Lper[a] = m.Lper[a];
  }
  AleTab3& t = A->tab3;
  std::memset(&t, 0, sizeof(t));
  std::vector<AleDer3> hd(1);
  {
    AleDer3& dd = hd[0];
    std::memset(&dd, 0, sizeof(dd));
    double dmax = 0.0;
    for (double v : re.Dxi) dmax = std::max(dmax, std::fabs(v));
    for (int e = 0; e < 3; ++e)
      for (int n = 0; n < L; ++n) {
        int c = 0;
        for (int l = 0; l < L; ++l) {
          const double v = re.Dxi[((size_t)e * L + n) * L + l];
          if (std::fabs(v) <= 1e-12 * dmax) continue;  // exact zeros, rounded in extended precision
          dd.val[e][n][c] = v;
          dd.col[e][n][c] = (uint8_t)l;
          ++c;
          if (l < L0) dd.nnz0[e][n] = c;  // columns ascend: tau = 0 nodes first
        }
        dd.nnz[e][n] = c;
      }
  }
  for (int k = 0; k < L1; ++k) {
    for (int l = 0; l < L; ++l) t.Gal[k][l] = re.Gal[(size_t)k * L + l];
    for (int n = 0; n < L0; ++n) t.C0[k][n] = re.C0[(size_t)k * L0 + n];
  }
  for (int v = 0; v < 4; ++v)
    for (int l = 0; l < L; ++l) t.Wv[v][l] = re.Wv[(size_t)v * L + l];
  for (int l = 0; l < L; ++l)
    for (int a = 0; a < 4; ++a) t.node[l][a] = re.stnode[l][a];
  for (int q = 0; q < re.nqs; ++q) {
    t.chi[q][0] = re.chi3[2 * q];
    t.chi[q][1] = re.chi3[2 * q + 1];
    t.wq[q] = re.wq[q];
  }
  for (int q = 0; q < re.nqt; ++q) {
    t.wt[q] = re.wt[q];
    t.tq[q] = re.tq[q];
  }
  t.gamma = s->prm.gamma;
  t.mode = s->prm.mesh_motion;
  t.pos = s->prm.positivity;
  // per-cell global vertices and periodic image shifts (image nearest the
  // cell's first vertex), SoA
  std::vector<int32_t> gv((size_t)4 * N);
  std::vector<double> sh((size_t)12 * N, 0.0);
  for (int64_t i = 0; i < N; ++i) {
    const int64_t g0 = m.gv[i * 4];
    for (int k = 0; k < 4; ++k) {
      const int64_t g = m.gv[i * 4 + k];
      gv[(size_t)k * N + i] = (int32_t)g;
      for (int a = 0; a < 3; ++a)
        if (m.per[a] && k > 0)
          sh[(size_t)(k * 3 + a) * N + i] = m.Lper[a] * std::nearbyint((m.xyz[g0 * 3 + a] - m.xyz[g * 3 + a]) / m.Lper[a]);
    }
  }
  // vertex -> (cell, local vertex) incidence, cells in increasing caller order
  std::vector<int32_t> start(nv + 1, 0), ent((size_t)4 * N);
  for (int64_t i = 0; i < N; ++i)
    for (int k = 0; k < 4; ++k) ++start[m.gv[i * 4 + k] + 1];
  for (int64_t g = 0; g < nv; ++g) start[g + 1] += start[g];
  {
    std::vector<int32_t> fill(start.begin(), start.end() - 1);
    for (int64_t u = 0; u < N; ++u) {
      const int64_t i = m.iperm[u];
      for (int k = 0; k < 4; ++k) ent[fill[m.gv[i * 4 + k]]++] = (int32_t)(i * 4 + k);
    }
  }
  std::vector<int32_t> ident(N);
  std::iota(ident.begin(), ident.end(), 0);
  ACK(A->put(&A->gv, gv, st));
  ACK(A->put(&A->shift, sh, st));
  ACK(A->put(&A->start, start, st));
  ACK(A->put(&A->ent, ent, st));
  ACK(A->put(&A->ident, ident, st));
  ACK(A->put(&A->Xv, m.xyz, st));
  ACK(A->put(&A->ftab, re.ftab, st));
  ACK(A->put(&A->der3, hd, st));
  ACK(A->alloc(&A->Xv1, (size_t)nv * 3, st));
  ACK(A->alloc(&A->X, (size_t)N * 12, st));
  ACK(A->alloc(&A->bary, (size_t)N * 3, st));
  ACK(A->alloc(&A->vol, (size_t)N, st));
  ACK(A->alloc(&A->w, (size_t)N * L0 * 5, st));
  ACK(A->alloc(&A->qhat, (size_t)N * L * 5, st));
  ACK(A->alloc(&A->vcon, (size_t)N * 16, st));
  ACK(A->alloc(&A->G, (size_t)5 * m.nf, st));
  ACK(A->alloc(&A->bad, 1, st));
  if (s->prec == CWENO_FP32_MIXED) {
    A->fp32 = true;
    A->tab3f = ale_tab3_float(t);
    std::vector<AleDer3f> hdf(1);
    ale_der3_float(hd[0], hdf[0]);
    ACK(A->put(&A->der3f, hdf, st));
    std::vector<float> f32(re.ftab.begin(), re.ftab.end());
    ACK(A->put(&A->ftab32, f32, st));
    ACK(A->alloc(&A->qhat32, (size_t)N * L * 5, st));
  }
  const int big = 0x7fffffff;
  ACK(cudaMemcpyAsync(A->bad, &big, sizeof(int), cudaMemcpyHostToDevice, st));
  ACK(cudaStreamSynchronize(st));
  s->bytes += A->bytes;
  s->ale = A;
  return CWENO_OK;
}

int ale_refresh(cweno_solver* s) {
  Ale& A = *s->ale;
  if (A.fresh) return CWENO_OK;
  DevState& ds = s->ds;
  cudaStream_t st = s->stream;
  if (A.d == 3)
    k_ale_geom3<<<nblk(ds.N, 256), 256, 0, st>>>(A.Xv, A.gv, A.shift, ds.N, A.X, A.bary, A.vol,
                                                  const_cast<double*>(ds.hsize), const_cast<double*>(ds.invvol));
  else
    k_ale_geom<<<nblk(ds.N, 256), 256, 0, st>>>(A.Xv, A.gv, A.shift, ds.N, A.X, A.bary, A.vol,
                                                 const_cast<double*>(ds.hsize), const_cast<double*>(ds.invvol));
  ACK(cudaGetLastError());
  int rc = ale_matrices_device(A.slim, *s->re, A.X, A.bary, ds.sten, ds.sec, const_cast<void*>(ds.R),
                               const_cast<void*>(ds.Binv), A.fp32, A.bad, st);
  if (rc) return fail(rc, "moving-mesh matrices");
  A.fresh = true;
  return CWENO_OK;
}

int ale_step(cweno_solver* s, double dt) {
  Ale& A = *s->ale;
  // stages timed when profiling is on (cweno_profile_read_stages)
  cudaEvent_t ev = nullptr;
  ACK(prof_begin(s, &ev));
  int rc = ale_refresh(s);
  if (rc) return rc;
  ACK(prof_end(s, ev, 0));
  DevState& ds = s->ds;
  cudaStream_t st = s->stream;
  const double dtf = dt > 0 ? dt : 0.0;
  if (dtf == 0.0) {  // CFL bound of the current state on the current mesh
    ACK(prof_begin(s, &ev));
    k_ale_dt_reset<<<1, 1, 0, st>>>(ds.dtmin);
    ACK(cudaGetLastError());
    ACK(s->ops->stable_dt(ds, s->ph, 0, st));
    ACK(prof_end(s, ev, 6));
  }
  DevState d2 = ds;
  d2.perm = A.ident;  // reconstruction values in internal cell order
  ACK(prof_begin(s, &ev));
  ACK(s->ops->reconstruct(d2, s->ph, A.w, st));
  ACK(prof_end(s, ev, 1));
  ACK(prof_begin(s, &ev));
  if (A.d == 3) {
    switch (A.M) {
      case 1: ACK(launch_pred3<1>(A, s, dtf, st)); break;
      case 2: ACK(launch_pred3<2>(A, s, dtf, st)); break;
      default: ACK(launch_pred3<3>(A, s, dtf, st)); break;
    }
    ACK(prof_end(s, ev, 2));
    ACK(prof_begin(s, &ev));
    k_ale_nodes3<<<nblk(A.nvert, 256), 256, 0, st>>>(A.start, A.ent, A.vcon, A.Xv, A.nvert, dtf, s->prm.cfl,
                                                      ds.dtmin, A.Xv1);
    ACK(cudaGetLastError());
    ACK(prof_end(s, ev, 3));
    ACK(prof_begin(s, &ev));
    switch (A.M) {
      case 1: ACK(launch_flux3<1>(A, s, dtf, st)); break;
      case 2: ACK(launch_flux3<2>(A, s, dtf, st)); break;
      default: ACK(launch_flux3<3>(A, s, dtf, st)); break;
    }
    ACK(prof_end(s, ev, 4));
    ACK(prof_begin(s, &ev));
    k_ale_update3<<<nblk(ds.N, 256), 256, 0, st>>>(ds.cellface, A.G, A.gv, A.shift, A.Xv1, A.vol, ds.N, ds.F,
                                                    s->prm.gamma, dtf, s->prm.cfl, ds.dtmin, ds.Q, ds.Qp, ds.time,
                                                    ds.status);
    ACK(cudaGetLastError());
    ACK(prof_end(s, ev, 5));
    std::swap(A.Xv, A.Xv1);
    A.fresh = false;
    return CWENO_OK;
  }
  switch (A.M) {
    case 1: ACK(launch_pred<1>(A, s, dtf, st)); break;
    case 2: ACK(launch_pred<2>(A, s, dtf, st)); break;
    default: ACK(launch_pred<3>(A, s, dtf, st)); break;
  }
  ACK(prof_end(s, ev, 2));
  ACK(prof_begin(s, &ev));
  k_ale_nodes<<<nblk(A.nvert, 256), 256, 0, st>>>(A.start, A.ent, A.vcon, A.Xv, A.nvert, dtf, s->prm.cfl, ds.dtmin,
                                                   A.Xv1);
  ACK(cudaGetLastError());
  ACK(prof_end(s, ev, 3));
  ACK(prof_begin(s, &ev));
  switch (A.M) {
    case 1: ACK(launch_flux<1>(A, s, dtf, st)); break;
    case 2: ACK(launch_flux<2>(A, s, dtf, st)); break;
    default: ACK(launch_flux<3>(A, s, dtf, st)); break;
  }
  ACK(prof_end(s, ev, 4));
  ACK(prof_begin(s, &ev));
  k_ale_update<<<nblk(ds.N, 256), 256, 0, st>>>(ds.cellface, A.G, A.gv, A.shift, A.Xv1, A.vol, ds.N, ds.F,
                                                 s->prm.gamma, dtf, s->prm.cfl, ds.dtmin, ds.Q, ds.Qp, ds.time,
                                                 ds.status);
  ACK(cudaGetLastError());
  ACK(prof_end(s, ev, 5));
  std::swap(A.Xv, A.Xv1);
  A.fresh = false;
  return CWENO_OK;
}

int ale_vertices(cweno_solver* s, double* xyz, int on_device) {
  Ale& A = *s->ale;
  ACK(cudaMemcpyAsync(xyz, A.Xv, sizeof(double) * A.nvert * A.d,
                      on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
  ACK(cudaStreamSynchronize(s->stream));
  return CWENO_OK;
}

int ale_degenerate(cweno_solver* s, int* cell) {
  Ale& A = *s->ale;
  int b = 0;
  ACK(cudaMemcpyAsync(&b, A.bad, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  ACK(cudaStreamSynchronize(s->stream));
  *cell = b == 0x7fffffff ? -1 : b;  // internal cell index
  return CWENO_OK;
}

}  // namespace cw
