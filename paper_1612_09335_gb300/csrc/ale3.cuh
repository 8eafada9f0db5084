// Moving meshes in three space dimensions: the direct ALE step (Secs.
// 2.2-2.4) on tetrahedra, Euler equations, FP64 or FP32-mixed, orders 2 to 4
// (M = 1..3),
// Rusanov flux with the ALE Jacobian.  The same step as the triangle path of
// ale.cu, kernel for kernel:
//   k_ale_geom3    unwrapped vertices, |T|, barycentre, h = 6|T| / surface
//                  (insphere diameter, Eq. timestep), 1/|T|;
//   k_ale_pred3    space-time predictor of the moving tetrahedron: state and
//                  geometry DOFs iterated together (Eqs. CGfinal, ODEfinal),
//                  H of Eq. (Hterm) from the nodal xi-derivatives with the
//                  3 x 3 inverse of d x / d xi at every node;
//   k_ale_nodes3   nodal solver, Eqs. (NScs)-(newX);
//   k_ale_flux3    lateral space-time faces: a triangle (A, B, C) moving on
//                  straight lines, x(chi1, chi2, tau) of Eq. (SurfPar) with
//                  the bilinear basis of Eq. (BetaBaseFunc), its normal the
//                  cofactors of the 4 x 4 matrix of Eq. (ChiTransf) (Eq.
//                  detChi); the face rule of the fixed-mesh kernels (collapsed
//                  Gauss on the triangle, weights normalised to 1, times the
//                  reference area 1/2) and Gauss-Legendre in tau;
//   k_ale_update3  Eq. (PDEfinal) with the new volume of the moved vertices.
// Included by ale.cu (shares its unnamed-namespace helpers).

constexpr int kL3 = 35, kL03 = 20, kL13 = 15, kNQS3 = 16, kNQT3 = 4;

// Nodal derivative tables of one M (tetrahedra) in the arithmetic type T, in
// device memory (at M = 3 they outgrow the kernel-parameter space): d theta_l
// / d xi_e at node n, nonzero entries only, tau = 0 columns first.
template <typename T>
struct AleDer3T {
  T val[3][kL3][kL3];
  uint8_t col[3][kL3][kL3];
  int nnz[3][kL3];
  int nnz0[3][kL3];
};
using AleDer3 = AleDer3T<double>;
using AleDer3f = AleDer3T<float>;

// The other reference tables of one M, a kernel parameter.
template <typename T>
struct AleTab3T {
  T Gal[kL13][kL3];  // (K_tau^1)^-1 M^1
  T C0[kL13][kL03];  // constant extension in time
  T Wv[4][kL3];      // int_0^1 theta_l(vertex v, tau) dtau
  T node[kL3][4];    // xi, eta, zeta, tau
  T chi[kNQS3][2], wq[kNQS3], wt[kNQT3], tq[kNQT3];
  T gamma;
  int mode;
  int pos;
};
using AleTab3 = AleTab3T<double>;
using AleTab3f = AleTab3T<float>;

inline void ale_der3_float(const AleDer3& t, AleDer3f& o) {
  std::memset(&o, 0, sizeof(o));
  for (int e = 0; e < 3; ++e)
    for (int n = 0; n < kL3; ++n) {
      for (int l = 0; l < kL3; ++l) {
        o.val[e][n][l] = (float)t.val[e][n][l];
        o.col[e][n][l] = t.col[e][n][l];
      }
      o.nnz[e][n] = t.nnz[e][n];
      o.nnz0[e][n] = t.nnz0[e][n];
    }
}

inline AleTab3f ale_tab3_float(const AleTab3& t) {
  AleTab3f o;
  std::memset(&o, 0, sizeof(o));
  for (int k = 0; k < kL13; ++k) {
    for (int l = 0; l < kL3; ++l) o.Gal[k][l] = (float)t.Gal[k][l];
    for (int n = 0; n < kL03; ++n) o.C0[k][n] = (float)t.C0[k][n];
  }
  for (int v = 0; v < 4; ++v)
    for (int l = 0; l < kL3; ++l) o.Wv[v][l] = (float)t.Wv[v][l];
  for (int l = 0; l < kL3; ++l)
    for (int a = 0; a < 4; ++a) o.node[l][a] = (float)t.node[l][a];
  for (int q = 0; q < kNQS3; ++q) {
    o.chi[q][0] = (float)t.chi[q][0];
    o.chi[q][1] = (float)t.chi[q][1];
    o.wq[q] = (float)t.wq[q];
  }
  for (int q = 0; q < kNQT3; ++q) {
    o.wt[q] = (float)t.wt[q];
    o.tq[q] = (float)t.tq[q];
  }
  o.gamma = (float)t.gamma;
  o.mode = t.mode;
  o.pos = t.pos;
  return o;
}

namespace {

__host__ __device__ constexpr int lcal3(int M) { return (M + 1) * (M + 2) * (M + 3) * (M + 4) / 24; }
__host__ __device__ constexpr int mcal3(int M) { return (M + 1) * (M + 2) * (M + 3) / 6; }

__device__ __forceinline__ double pressure3(const double* q, double g) {
  return (g - 1.0) * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
}

__device__ __forceinline__ bool admissible3(const double* q, double g) {
  bool fin = true;
  for (int v = 0; v < 5; ++v) fin = fin && isfinite(q[v]);
  return fin && q[0] > 0.0 && pressure3(q, g) > 0.0;
}

// Face points per chunk of the face kernels: the largest divisor of np not
// above cap.  The traces of a chunk's points are formed in one pass over
// both sides' q_hat (read once per chunk instead of once per point).
__host__ __device__ constexpr int point_chunk(int np, int cap) {
  int c = cap;
  while (c > 1 && np % c != 0) --c;
  return c;
}

__device__ __forceinline__ double det3(const double* a, const double* b, const double* c) {
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
}

// ---------------------------------------------------------------- geometry
__global__ void __launch_bounds__(256) k_ale_geom3(const double* __restrict__ Xv, const int32_t* __restrict__ gv,
                                                   const double* __restrict__ shift, int64_t N, double* __restrict__ X,
                                                   double* __restrict__ bary, double* __restrict__ vol,
                                                   double* __restrict__ hsize, double* __restrict__ invvol) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double P[4][3];
  for (int k = 0; k < 4; ++k) {
    const int64_t g = gv[k * N + i];
    for (int a = 0; a < 3; ++a) {
      P[k][a] = Xv[g * 3 + a] + shift[(k * 3 + a) * N + i];
      X[i * 12 + k * 3 + a] = P[k][a];
    }
  }
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) e[k][a] = P[k + 1][a] - P[0][a];
  const double v = det3(e[0], e[1], e[2]) / 6.0;
  double surf = 0.0;
  for (int k = 0; k < 4; ++k) {
    int o[3], n = 0;
    for (int q = 0; q < 4; ++q)
      if (q != k) o[n++] = q;
    double u[3], w[3];
    for (int a = 0; a < 3; ++a) {
      u[a] = P[o[1]][a] - P[o[0]][a];
      w[a] = P[o[2]][a] - P[o[0]][a];
    }
    const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
    surf += 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
  }
  vol[i] = v;
  hsize[i] = 6.0 * v / surf;
  invvol[i] = 1.0 / v;
  for (int a = 0; a < 3; ++a) bary[i * 3 + a] = (P[0][a] + P[1][a] + P[2][a] + P[3][a]) / 4.0;
}

// ---------------------------------------------------------------- predictor
// Euler fluxes (x, y, z) and the mesh velocity of one nodal state.
__device__ __forceinline__ void ale_flux3(const double* q, double gamma, int mode, double F[3][5], double V[3]) {
  const double ir = 1.0 / q[0];
  const double u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const double p = (gamma - 1.0) * (q[4] - 0.5 * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
  for (int m = 0; m < 3; ++m) {
    F[m][0] = q[1 + m];
    for (int b = 0; b < 3; ++b) F[m][1 + b] = q[1 + b] * u[m] + (b == m ? p : 0.0);
    F[m][4] = u[m] * (q[4] + p);
    V[m] = mode == CWENO_MOTION_LAGRANGE ? u[m] : 0.0;
  }
}

// One thread per cell.  w: reconstruction values at the lattice nodes
// (N x L0 x 5); X: unwrapped vertices of T_i^n (N x 4 x 3).  Writes q_hat
// (N x L x 5) and, per vertex k of the cell, (mu V_kj, mu) with mu =
// rho_j |T_j| (N x 4 x 4).
template <int M>
__global__ void __launch_bounds__(128) k_ale_pred3(const __grid_constant__ AleTab3 t,
                                                   const AleDer3* __restrict__ dr, const double* __restrict__ w,
                                                   const double* __restrict__ Q, const double* __restrict__ X,
                                                   const double* __restrict__ vol, int64_t N, int niter,
                                                   double dt_fixed, double cfl, const unsigned long long* dtmin,
                                                   double* __restrict__ qhat, double* __restrict__ vcon) {
  constexpr int L = lcal3(M), L0 = mcal3(M), L1 = L - L0, NC = 3 + 5 + 15;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double dt = step_dt(dt_fixed, cfl, dtmin);
  double q[L][5], x[L][3], V[L][3];
  for (int n = 0; n < L0; ++n)
    for (int v = 0; v < 5; ++v) q[n][v] = w[(i * L0 + n) * 5 + v];
  for (int k = 0; k < L1; ++k)
    for (int v = 0; v < 5; ++v) {
      double s = 0.0;
      for (int n = 0; n < L0; ++n) s += t.C0[k][n] * q[n][v];
      q[L0 + k][v] = s;
    }
  const double* Xi = X + i * 12;
  for (int l = 0; l < L; ++l)
    for (int a = 0; a < 3; ++a)
      x[l][a] = Xi[a] + (Xi[3 + a] - Xi[a]) * t.node[l][0] + (Xi[6 + a] - Xi[a]) * t.node[l][1] +
                (Xi[9 + a] - Xi[a]) * t.node[l][2];
  double qe[L1][5], xe[L1][3];
  for (int k = 0; k < L1; ++k) {
    for (int v = 0; v < 5; ++v) qe[k][v] = q[L0 + k][v];
    for (int a = 0; a < 3; ++a) xe[k][a] = x[L0 + k][a];
  }
  // the tau = 0 nodes never change: their part of every xi-derivative of x,
  // q and F is formed once (per node and direction: 3 + 5 + 3 x 5 sums)
  double c0[L][3][NC];
  {
    double F0[L0][3][5];
    for (int l = 0; l < L0; ++l) ale_flux3(q[l], t.gamma, t.mode, F0[l], V[l]);
    for (int n = 0; n < L; ++n)
      for (int e = 0; e < 3; ++e) {
        double* c = c0[n][e];
        for (int m = 0; m < NC; ++m) c[m] = 0.0;
        for (int j = 0; j < dr->nnz0[e][n]; ++j) {
          const int l = dr->col[e][n][j];
          const double dd = dr->val[e][n][j];
          for (int a = 0; a < 3; ++a) c[a] += dd * x[l][a];
          for (int v = 0; v < 5; ++v) {
            c[3 + v] += dd * q[l][v];
            for (int m = 0; m < 3; ++m) c[8 + m * 5 + v] += dd * F0[l][m][v];
          }
        }
      }
  }
  for (int it = 0; it < niter; ++it) {
    double F[L1][3][5];
    for (int l = L0; l < L; ++l) ale_flux3(q[l], t.gamma, t.mode, F[l - L0], V[l]);
    double H[L][5];
    for (int n = 0; n < L; ++n) {
      double dx[3][3], dq[3][5], df[3][3][5];
      for (int e = 0; e < 3; ++e) {
        const double* c = c0[n][e];
        for (int a = 0; a < 3; ++a) dx[e][a] = c[a];
        for (int v = 0; v < 5; ++v) {
          dq[e][v] = c[3 + v];
          for (int m = 0; m < 3; ++m) df[e][m][v] = c[8 + m * 5 + v];
        }
        const int cnt = dr->nnz[e][n];
        for (int j = dr->nnz0[e][n]; j < cnt; ++j) {
          const int l = dr->col[e][n][j];
          const double dd = dr->val[e][n][j];
          for (int a = 0; a < 3; ++a) dx[e][a] += dd * x[l][a];
          for (int v = 0; v < 5; ++v) {
            dq[e][v] += dd * q[l][v];
            for (int m = 0; m < 3; ++m) df[e][m][v] += dd * F[l - L0][m][v];
          }
        }
      }
      // J[a][e] = d x_a / d xi_e = dx[e][a]; Ji[e][a] = d xi_e / d x_a by
      // cofactors: row e of J^-1 is (dx[e+1] x dx[e+2]) / det
      const double det = det3(dx[0], dx[1], dx[2]), idet = 1.0 / det;
      double Ji[3][3];
      for (int e = 0; e < 3; ++e) {
        const double* p = dx[(e + 1) % 3];
        const double* r = dx[(e + 2) % 3];
        Ji[e][0] = (p[1] * r[2] - p[2] * r[1]) * idet;
        Ji[e][1] = (p[2] * r[0] - p[0] * r[2]) * idet;
        Ji[e][2] = (p[0] * r[1] - p[1] * r[0]) * idet;
      }
      double dxidt[3];
      for (int e = 0; e < 3; ++e) dxidt[e] = -(Ji[e][0] * V[n][0] + Ji[e][1] * V[n][1] + Ji[e][2] * V[n][2]);
      for (int v = 0; v < 5; ++v) {
        double h = 0.0;
        for (int e = 0; e < 3; ++e)
          h += dq[e][v] * dxidt[e] + Ji[e][0] * df[e][0][v] + Ji[e][1] * df[e][1][v] + Ji[e][2] * df[e][2][v];
        H[n][v] = h;
      }
    }
    for (int k = 0; k < L1; ++k) {
      for (int v = 0; v < 5; ++v) {
        double g = 0.0;
        for (int l = 0; l < L; ++l) g += t.Gal[k][l] * H[l][v];
        q[L0 + k][v] = qe[k][v] - dt * g;
      }
      for (int a = 0; a < 3; ++a) {
        double g = 0.0;
        for (int l = 0; l < L; ++l) g += t.Gal[k][l] * V[l][a];
        x[L0 + k][a] = xe[k][a] + dt * g;
      }
    }
  }
  double qb[5];
  for (int v = 0; v < 5; ++v) qb[v] = Q[v * N + i];
  if (t.pos) {
    // fallback: a tau > 0 node inadmissible or outside [1/2 min, 2 max] of
    // the tau = 0 nodes' density and pressure (the triangle path's rule)
    double r0 = 1e300, r1 = -1e300, p0 = 1e300, p1 = -1e300;
    for (int l = 0; l < L0; ++l) {
      const double pl = pressure3(q[l], t.gamma);
      r0 = fmin(r0, q[l][0]);
      r1 = fmax(r1, q[l][0]);
      p0 = fmin(p0, pl);
      p1 = fmax(p1, pl);
    }
    bool ok = true;
    for (int l = L0; l < L; ++l) {
      const double pl = pressure3(q[l], t.gamma);
      ok = ok && admissible3(q[l], t.gamma) && q[l][0] >= 0.5 * r0 && q[l][0] <= 2.0 * r1 && pl >= 0.5 * p0 &&
           pl <= 2.0 * p1;
    }
    if (!ok)
      for (int l = 0; l < L; ++l)
        for (int v = 0; v < 5; ++v) q[l][v] = qb[v];
  }
  for (int l = 0; l < L; ++l) {
    for (int v = 0; v < 5; ++v) qhat[(i * L + l) * 5 + v] = q[l][v];
    const double ir = 1.0 / q[l][0];
    for (int a = 0; a < 3; ++a) V[l][a] = t.mode == CWENO_MOTION_LAGRANGE ? q[l][1 + a] * ir : 0.0;
  }
  const double mu = qb[0] * vol[i];
  for (int k = 0; k < 4; ++k) {
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int l = 0; l < L; ++l) s += t.Wv[k][l] * V[l][a];
      vcon[(i * 4 + k) * 4 + a] = mu * s;
    }
    vcon[(i * 4 + k) * 4 + 3] = mu;
  }
}

// ------------------------------------------------------------- nodal solver
// One thread per vertex over the incidence list (cell * 4 + local vertex, in
// increasing caller cell order): V_k = sum mu V_kj / sum mu, X^{n+1} = X^n +
// dt V_k.
__global__ void __launch_bounds__(256) k_ale_nodes3(const int32_t* __restrict__ start, const int32_t* __restrict__ ent,
                                                    const double* __restrict__ vcon, const double* __restrict__ Xv,
                                                    int64_t nvert, double dt_fixed, double cfl,
                                                    const unsigned long long* dtmin, double* __restrict__ Xv1) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nvert) return;
  const double dt = step_dt(dt_fixed, cfl, dtmin);
  double ax = 0.0, ay = 0.0, az = 0.0, mu = 0.0;
  for (int32_t e = start[g]; e < start[g + 1]; ++e) {
    const double* c = vcon + (int64_t)ent[e] * 4;
    ax += c[0];
    ay += c[1];
    az += c[2];
    mu += c[3];
  }
  Xv1[g * 3] = mu > 0.0 ? Xv[g * 3] + dt * (ax / mu) : Xv[g * 3];
  Xv1[g * 3 + 1] = mu > 0.0 ? Xv[g * 3 + 1] + dt * (ay / mu) : Xv[g * 3 + 1];
  Xv1[g * 3 + 2] = mu > 0.0 ? Xv[g * 3 + 2] + dt * (az / mu) : Xv[g * 3 + 2];
}

// -------------------------------------------------------------------- faces
struct FaceGeo3 {
  double A0[3], B0[3], C0[3], A1[3], B1[3], C1[3];
};

// Space-time normal (x, y, z, t) at (chi1, chi2, tau): component p is
// (-1)^(1+p) times the minor of the rows (dx/dchi1, 0), (dx/dchi2, 0),
// (dx/dtau, dt) that deletes column p (Eq. detChi).
__device__ __forceinline__ void st_normal3(const FaceGeo3& f, double c1, double c2, double tau, double dt, double* n) {
  double r1[3], r2[3], r3[3];
  for (int a = 0; a < 3; ++a) {
    r1[a] = (1.0 - tau) * (f.B0[a] - f.A0[a]) + tau * (f.B1[a] - f.A1[a]);
    r2[a] = (1.0 - tau) * (f.C0[a] - f.A0[a]) + tau * (f.C1[a] - f.A1[a]);
    r3[a] = (1.0 - c1 - c2) * (f.A1[a] - f.A0[a]) + c1 * (f.B1[a] - f.B0[a]) + c2 * (f.C1[a] - f.C0[a]);
  }
  // the t-column is (0, 0, dt): the spatial components expand along it
  n[0] = dt * (r1[1] * r2[2] - r1[2] * r2[1]);
  n[1] = dt * (r1[2] * r2[0] - r1[0] * r2[2]);
  n[2] = dt * (r1[0] * r2[1] - r1[1] * r2[0]);
  n[3] = -det3(r1, r2, r3);
}

// One thread per face: the integral over the lateral space-time face of the
// Rusanov flux (F~(q+) + F~(q-)).n~/2 - s_max (q+ - q-)/2, F~ = (f, g, h, Q),
// s_max = |n~_x| max(|v.n - V.n| + c) over both sides, V.n = -n~_t/|n~_x|.
// Face vertices in ascending global id (the order of the face tables of
// both sides' codes).  Transmissive boundary: q+ = q-.  Positivity switch:
// an inadmissible trace is replaced by that side's cell average.
template <int M>
__global__ void __launch_bounds__(128) k_ale_flux3(const __grid_constant__ AleTab3 t, const double* __restrict__ ftab,
                                                   const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
                                                   const uint8_t* __restrict__ codeL, const uint8_t* __restrict__ codeR,
                                                   const int32_t* __restrict__ gv, const double* __restrict__ shift,
                                                   const double* __restrict__ Xv, const double* __restrict__ Xv1,
                                                   const double* __restrict__ bary, const double* __restrict__ qhat,
                                                   const double* __restrict__ Q, int64_t N, int64_t F,
                                                   double dt_fixed, double cfl, const unsigned long long* dtmin,
                                                   double* __restrict__ G) {
  constexpr int L = lcal3(M), NQT = M + 1, NQS = (M + 1) * (M + 1);
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double dt = step_dt(dt_fixed, cfl, dtmin);
  const int64_t cl = fL[f], cr = fR[f];
  const int kL = codeL[f], kR = cr >= 0 ? codeR[f] : 0;
  const int lf = kL / 6;
  int lv[3], n3 = 0;
  for (int q = 0; q < 4; ++q)
    if (q != lf) lv[n3++] = q;
  int64_t gg[3];
  for (int r = 0; r < 3; ++r) gg[r] = gv[lv[r] * N + cl];
  // ascending global id (insertion sort of three)
  for (int r = 1; r < 3; ++r)
    for (int s = r; s > 0 && gg[s] < gg[s - 1]; --s) {
      const int64_t tg = gg[s];
      gg[s] = gg[s - 1];
      gg[s - 1] = tg;
      const int tl = lv[s];
      lv[s] = lv[s - 1];
      lv[s - 1] = tl;
    }
  FaceGeo3 fg;
  for (int a = 0; a < 3; ++a) {
    const double sa = shift[(lv[0] * 3 + a) * N + cl], sb = shift[(lv[1] * 3 + a) * N + cl],
                 sc = shift[(lv[2] * 3 + a) * N + cl];
    fg.A0[a] = Xv[gg[0] * 3 + a] + sa;
    fg.B0[a] = Xv[gg[1] * 3 + a] + sb;
    fg.C0[a] = Xv[gg[2] * 3 + a] + sc;
    fg.A1[a] = Xv1[gg[0] * 3 + a] + sa;
    fg.B1[a] = Xv1[gg[1] * 3 + a] + sb;
    fg.C1[a] = Xv1[gg[2] * 3 + a] + sc;
  }
  double n0[4];
  st_normal3(fg, 0.0, 0.0, 0.0, dt, n0);
  const double sgn = n0[0] * (fg.A0[0] - bary[cl * 3]) + n0[1] * (fg.A0[1] - bary[cl * 3 + 1]) +
                             n0[2] * (fg.A0[2] - bary[cl * 3 + 2]) >
                             0.0
                         ? 1.0
                         : -1.0;
  double qbL[5], qbR[5];
  for (int v = 0; v < 5; ++v) {
    qbL[v] = Q[v * N + cl];
    qbR[v] = cr >= 0 ? Q[v * N + cr] : qbL[v];
  }
  const double* qL = qhat + cl * L * 5;
  const double* qR = qhat + (cr >= 0 ? cr : cl) * L * 5;
  double acc[5] = {0, 0, 0, 0, 0};
  constexpr int NP = NQS * NQT, PC = point_chunk(NP, 4);
  for (int p0 = 0; p0 < NP; p0 += PC) {
    // traces of the chunk's points (point p = qp NQT + tt), q_hat read once
    double qmc[PC][5], qqc[PC][5];
#pragma unroll
    for (int j = 0; j < PC; ++j)
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        qmc[j][v] = 0.0;
        qqc[j][v] = 0.0;
      }
    for (int l = 0; l < L; ++l) {
      double xa[5], xb[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        xa[v] = qL[l * 5 + v];
        xb[v] = qR[l * 5 + v];
      }
#pragma unroll
      for (int j = 0; j < PC; ++j) {
        const int pj = p0 + j, qj = pj / NQT, tj = pj % NQT;
        const double wl = ftab[((int64_t)(kL * NQT + tj) * NQS + qj) * L + l];
        const double wr = ftab[((int64_t)(kR * NQT + tj) * NQS + qj) * L + l];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          qmc[j][v] += wl * xa[v];
          qqc[j][v] += wr * xb[v];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < PC; ++j) {
      const int qp = (p0 + j) / NQT, tt = (p0 + j) % NQT;
      double qm[5], qq[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        qm[v] = qmc[j][v];
        qq[v] = qqc[j][v];
      }
      if (cr < 0)
        for (int v = 0; v < 5; ++v) qq[v] = qm[v];
      if (t.pos) {
        if (!admissible3(qm, t.gamma))
          for (int v = 0; v < 5; ++v) qm[v] = qbL[v];
        if (!admissible3(qq, t.gamma))
          for (int v = 0; v < 5; ++v) qq[v] = qbR[v];
      }
      double n[4];
      st_normal3(fg, t.chi[qp][0], t.chi[qp][1], t.tq[tt], dt, n);
      for (int a = 0; a < 4; ++a) n[a] *= sgn;
      const double nx = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]), inx = 1.0 / nx;
      const double un[3] = {n[0] * inx, n[1] * inx, n[2] * inx};
      const double Vn = -n[3] * inx;
      double sm = 0.0, fsum[5] = {0, 0, 0, 0, 0};
      const double* sides[2] = {qm, qq};
      for (int s = 0; s < 2; ++s) {
        const double* z = sides[s];
        const double ir = 1.0 / z[0];
        const double u[3] = {z[1] * ir, z[2] * ir, z[3] * ir};
        const double p = (t.gamma - 1.0) * (z[4] - 0.5 * (z[1] * u[0] + z[2] * u[1] + z[3] * u[2]));
        const double c = sqrt(fmax(0.0, t.gamma * p * ir));
        const double vn = u[0] * un[0] + u[1] * un[1] + u[2] * un[2];
        sm = fmax(sm, fabs(vn - Vn) + c);
        const double un_n = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];  // v . n~_x
        fsum[0] += z[1] * n[0] + z[2] * n[1] + z[3] * n[2];
        for (int b = 0; b < 3; ++b) fsum[1 + b] += z[1 + b] * un_n + p * n[b];
        fsum[4] += (z[4] + p) * un_n;
      }
      sm *= nx;
      const double wgt = 0.5 * t.wq[qp] * t.wt[tt];  // reference triangle area 1/2
      for (int v = 0; v < 5; ++v)
        acc[v] += wgt * (0.5 * fsum[v] + 0.5 * (qm[v] + qq[v]) * n[3] - 0.5 * sm * (qq[v] - qm[v]));
    }
  }
  for (int v = 0; v < 5; ++v) G[v * F + f] = acc[v];
}

// ------------------------------------------------------------ FP32-mixed
// The same predictor and face integrals in single precision on deviations
// (the design of the triangle path's k_ale_pred32 / k_ale_flux32): the state
// from the cell average, node positions from the cell's first vertex, nodal
// fluxes from the flux of the FP32-rounded average, so that a constant state
// has exactly zero xi-derivatives; the least squares, the nodal solver, the
// update and the face integral of the cell averages stay FP64.
__device__ __forceinline__ void ale_flux3f(const float* q, float gamma, int mode, float F[3][5], float V[3]) {
  const float ir = 1.0f / q[0];
  const float u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const float p = (gamma - 1.0f) * (q[4] - 0.5f * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
  for (int m = 0; m < 3; ++m) {
    F[m][0] = q[1 + m];
    for (int b = 0; b < 3; ++b) F[m][1 + b] = q[1 + b] * u[m] + (b == m ? p : 0.0f);
    F[m][4] = u[m] * (q[4] + p);
    V[m] = mode == CWENO_MOTION_LAGRANGE ? u[m] : 0.0f;
  }
}

__device__ __forceinline__ bool admissible3f(const float* q, float g) {
  bool fin = true;
  for (int v = 0; v < 5; ++v) fin = fin && isfinite(q[v]);
  return fin && q[0] > 0.0f && (g - 1.0f) * (q[4] - 0.5f * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]) > 0.0f;
}

// Writes the state deviations q_hat - Q_i (N x L x 5, FP32) and (mu V_kj, mu)
// per vertex of the cell in FP64.
template <int M>
__global__ void __launch_bounds__(128) k_ale_pred3_32(const __grid_constant__ AleTab3f t,
                                                      const AleDer3f* __restrict__ dr, const double* __restrict__ w,
                                                      const double* __restrict__ Q, const double* __restrict__ X,
                                                      const double* __restrict__ vol, int64_t N, int niter,
                                                      double dt_fixed, double cfl, const unsigned long long* dtmin,
                                                      float* __restrict__ qhat, double* __restrict__ vcon) {
  constexpr int L = lcal3(M), L0 = mcal3(M), L1 = L - L0, NC = 3 + 5 + 15;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float dt = (float)step_dt(dt_fixed, cfl, dtmin);
  double Qd[5];
  float qb[5];
  for (int v = 0; v < 5; ++v) {
    Qd[v] = Q[v * N + i];
    qb[v] = (float)Qd[v];
  }
  float q[L][5], x[L][3], V[L][3];
  for (int n = 0; n < L0; ++n)
    for (int v = 0; v < 5; ++v) q[n][v] = (float)(w[(i * L0 + n) * 5 + v] - Qd[v]);
  for (int k = 0; k < L1; ++k)
    for (int v = 0; v < 5; ++v) {
      float s = 0.0f;
      for (int n = 0; n < L0; ++n) s += t.C0[k][n] * q[n][v];
      q[L0 + k][v] = s;
    }
  const double* Xi = X + i * 12;
  float E[3][3];  // edge vectors X_k - X_0
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) E[k][a] = (float)(Xi[3 * (k + 1) + a] - Xi[a]);
  for (int l = 0; l < L; ++l)
    for (int a = 0; a < 3; ++a) x[l][a] = E[0][a] * t.node[l][0] + E[1][a] * t.node[l][1] + E[2][a] * t.node[l][2];
  float Fb[3][5], Vb[3];
  ale_flux3f(qb, t.gamma, t.mode, Fb, Vb);
  float qe[L1][5], xe[L1][3];
  for (int k = 0; k < L1; ++k) {
    for (int v = 0; v < 5; ++v) qe[k][v] = q[L0 + k][v];
    for (int a = 0; a < 3; ++a) xe[k][a] = x[L0 + k][a];
  }
  auto nodal_flux = [&](const float* dq, float F[3][5], float* Vn) {
    float qa[5];
    for (int v = 0; v < 5; ++v) qa[v] = qb[v] + dq[v];
    ale_flux3f(qa, t.gamma, t.mode, F, Vn);
    for (int m = 0; m < 3; ++m)
      for (int v = 0; v < 5; ++v) F[m][v] -= Fb[m][v];
  };
  float c0[L][3][NC];
  {
    float F0[L0][3][5];
    for (int l = 0; l < L0; ++l) nodal_flux(q[l], F0[l], V[l]);
    for (int n = 0; n < L; ++n)
      for (int e = 0; e < 3; ++e) {
        float* c = c0[n][e];
        for (int m = 0; m < NC; ++m) c[m] = 0.0f;
        for (int j = 0; j < dr->nnz0[e][n]; ++j) {
          const int l = dr->col[e][n][j];
          const float dd = dr->val[e][n][j];
          for (int a = 0; a < 3; ++a) c[a] += dd * x[l][a];
          for (int v = 0; v < 5; ++v) {
            c[3 + v] += dd * q[l][v];
            for (int m = 0; m < 3; ++m) c[8 + m * 5 + v] += dd * F0[l][m][v];
          }
        }
      }
  }
  for (int it = 0; it < niter; ++it) {
    float F[L1][3][5];
    for (int l = L0; l < L; ++l) nodal_flux(q[l], F[l - L0], V[l]);
    float H[L][5];
    for (int n = 0; n < L; ++n) {
      float dx[3][3], dq[3][5], df[3][3][5];
      for (int e = 0; e < 3; ++e) {
        const float* c = c0[n][e];
        for (int a = 0; a < 3; ++a) dx[e][a] = c[a];
        for (int v = 0; v < 5; ++v) {
          dq[e][v] = c[3 + v];
          for (int m = 0; m < 3; ++m) df[e][m][v] = c[8 + m * 5 + v];
        }
        const int cnt = dr->nnz[e][n];
        for (int j = dr->nnz0[e][n]; j < cnt; ++j) {
          const int l = dr->col[e][n][j];
          const float dd = dr->val[e][n][j];
          for (int a = 0; a < 3; ++a) dx[e][a] += dd * x[l][a];
          for (int v = 0; v < 5; ++v) {
            dq[e][v] += dd * q[l][v];
            for (int m = 0; m < 3; ++m) df[e][m][v] += dd * F[l - L0][m][v];
          }
        }
      }
      float Ji[3][3];
      {
        const float det = dx[0][0] * (dx[1][1] * dx[2][2] - dx[1][2] * dx[2][1]) -
                          dx[0][1] * (dx[1][0] * dx[2][2] - dx[1][2] * dx[2][0]) +
                          dx[0][2] * (dx[1][0] * dx[2][1] - dx[1][1] * dx[2][0]);
        const float idet = 1.0f / det;
        for (int e = 0; e < 3; ++e) {
          const float* p = dx[(e + 1) % 3];
          const float* r = dx[(e + 2) % 3];
          Ji[e][0] = (p[1] * r[2] - p[2] * r[1]) * idet;
          Ji[e][1] = (p[2] * r[0] - p[0] * r[2]) * idet;
          Ji[e][2] = (p[0] * r[1] - p[1] * r[0]) * idet;
        }
      }
      float dxidt[3];
      for (int e = 0; e < 3; ++e) dxidt[e] = -(Ji[e][0] * V[n][0] + Ji[e][1] * V[n][1] + Ji[e][2] * V[n][2]);
      for (int v = 0; v < 5; ++v) {
        float h = 0.0f;
        for (int e = 0; e < 3; ++e)
          h += dq[e][v] * dxidt[e] + Ji[e][0] * df[e][0][v] + Ji[e][1] * df[e][1][v] + Ji[e][2] * df[e][2][v];
        H[n][v] = h;
      }
    }
    for (int k = 0; k < L1; ++k) {
      for (int v = 0; v < 5; ++v) {
        float g = 0.0f;
        for (int l = 0; l < L; ++l) g += t.Gal[k][l] * H[l][v];
        q[L0 + k][v] = qe[k][v] - dt * g;
      }
      for (int a = 0; a < 3; ++a) {
        float g = 0.0f;
        for (int l = 0; l < L; ++l) g += t.Gal[k][l] * V[l][a];
        x[L0 + k][a] = xe[k][a] + dt * g;
      }
    }
  }
  if (t.pos) {  // the fallback rule of k_ale_pred3, on absolute states
    auto pres = [&](const float* qa) {
      return (t.gamma - 1.0f) * (qa[4] - 0.5f * (qa[1] * qa[1] + qa[2] * qa[2] + qa[3] * qa[3]) / qa[0]);
    };
    float r0 = 3e38f, r1 = -3e38f, p0 = 3e38f, p1 = -3e38f;
    for (int l = 0; l < L0; ++l) {
      float qa[5];
      for (int v = 0; v < 5; ++v) qa[v] = qb[v] + q[l][v];
      const float pl = pres(qa);
      r0 = fminf(r0, qa[0]);
      r1 = fmaxf(r1, qa[0]);
      p0 = fminf(p0, pl);
      p1 = fmaxf(p1, pl);
    }
    bool ok = true;
    for (int l = L0; l < L; ++l) {
      float qa[5];
      for (int v = 0; v < 5; ++v) qa[v] = qb[v] + q[l][v];
      const float pl = pres(qa);
      ok = ok && admissible3f(qa, t.gamma) && qa[0] >= 0.5f * r0 && qa[0] <= 2.0f * r1 && pl >= 0.5f * p0 &&
           pl <= 2.0f * p1;
    }
    if (!ok)
      for (int l = 0; l < L; ++l)
        for (int v = 0; v < 5; ++v) q[l][v] = 0.0f;
  }
  for (int l = 0; l < L; ++l) {
    for (int v = 0; v < 5; ++v) qhat[(i * L + l) * 5 + v] = q[l][v];
    const float ir = 1.0f / (qb[0] + q[l][0]);
    for (int a = 0; a < 3; ++a) V[l][a] = t.mode == CWENO_MOTION_LAGRANGE ? (qb[1 + a] + q[l][1 + a]) * ir : 0.0f;
  }
  const double mu = Qd[0] * vol[i];
  for (int k = 0; k < 4; ++k) {
    for (int a = 0; a < 3; ++a) {
      float s = 0.0f;
      for (int l = 0; l < L; ++l) s += t.Wv[k][l] * V[l][a];
      vcon[(i * 4 + k) * 4 + a] = mu * (double)s;
    }
    vcon[(i * 4 + k) * 4 + 3] = mu;
  }
}

__device__ __forceinline__ void euler_xyz64(const double* z, double g, double F[3][5]) {
  const double ir = 1.0 / z[0];
  const double u[3] = {z[1] * ir, z[2] * ir, z[3] * ir};
  const double p = (g - 1.0) * (z[4] - 0.5 * (z[1] * u[0] + z[2] * u[1] + z[3] * u[2]));
  for (int m = 0; m < 3; ++m) {
    F[m][0] = z[1 + m];
    for (int b = 0; b < 3; ++b) F[m][1 + b] = z[1 + b] * u[m] + (b == m ? p : 0.0);
    F[m][4] = u[m] * (z[4] + p);
  }
}

// Face integrals with FP32 deviations.  The cell averages' part,
// 1/2 (F(Q-) + F(Q+)) . n + 1/2 (Q- + Q+) n_t, is integrated in FP64 with the
// face's integrated normal: n_x is quadratic in tau and constant in chi, n_t
// quadratic in tau and linear in chi, so the integral over the reference
// triangle x [0, 1] is 1/2 times Simpson's rule in tau at the triangle's
// centroid (exact).  A constant state therefore sees the FP64 geometry.
template <int M>
__global__ void __launch_bounds__(128) k_ale_flux3_32(const __grid_constant__ AleTab3f t, double gamma64,
                                                      const float* __restrict__ ftab, const int32_t* __restrict__ fL,
                                                      const int32_t* __restrict__ fR,
                                                      const uint8_t* __restrict__ codeL,
                                                      const uint8_t* __restrict__ codeR, const int32_t* __restrict__ gv,
                                                      const double* __restrict__ shift, const double* __restrict__ Xv,
                                                      const double* __restrict__ Xv1, const double* __restrict__ bary,
                                                      const float* __restrict__ qhat, const double* __restrict__ Q,
                                                      int64_t N, int64_t F, double dt_fixed, double cfl,
                                                      const unsigned long long* dtmin, double* __restrict__ G) {
  constexpr int L = lcal3(M), NQT = M + 1, NQS = (M + 1) * (M + 1);
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double dt = step_dt(dt_fixed, cfl, dtmin);
  const int64_t cl = fL[f], cr = fR[f];
  const int kL = codeL[f], kR = cr >= 0 ? codeR[f] : 0;
  const int lf = kL / 6;
  int lv[3], n3 = 0;
  for (int q = 0; q < 4; ++q)
    if (q != lf) lv[n3++] = q;
  int64_t gg[3];
  for (int r = 0; r < 3; ++r) gg[r] = gv[lv[r] * N + cl];
  for (int r = 1; r < 3; ++r)
    for (int s = r; s > 0 && gg[s] < gg[s - 1]; --s) {
      const int64_t tg = gg[s];
      gg[s] = gg[s - 1];
      gg[s - 1] = tg;
      const int tl = lv[s];
      lv[s] = lv[s - 1];
      lv[s - 1] = tl;
    }
  FaceGeo3 fg;
  for (int a = 0; a < 3; ++a) {
    const double sa = shift[(lv[0] * 3 + a) * N + cl], sb = shift[(lv[1] * 3 + a) * N + cl],
                 sc = shift[(lv[2] * 3 + a) * N + cl];
    fg.A0[a] = Xv[gg[0] * 3 + a] + sa;
    fg.B0[a] = Xv[gg[1] * 3 + a] + sb;
    fg.C0[a] = Xv[gg[2] * 3 + a] + sc;
    fg.A1[a] = Xv1[gg[0] * 3 + a] + sa;
    fg.B1[a] = Xv1[gg[1] * 3 + a] + sb;
    fg.C1[a] = Xv1[gg[2] * 3 + a] + sc;
  }
  double n0[4];
  st_normal3(fg, 0.0, 0.0, 0.0, dt, n0);
  const double sgn = n0[0] * (fg.A0[0] - bary[cl * 3]) + n0[1] * (fg.A0[1] - bary[cl * 3 + 1]) +
                             n0[2] * (fg.A0[2] - bary[cl * 3 + 2]) >
                             0.0
                         ? 1.0
                         : -1.0;
  double nbar[4];
  {
    double na[4], nm[4], nb[4];
    const double c = 1.0 / 3.0;
    st_normal3(fg, c, c, 0.0, dt, na);
    st_normal3(fg, c, c, 0.5, dt, nm);
    st_normal3(fg, c, c, 1.0, dt, nb);
    for (int a = 0; a < 4; ++a) nbar[a] = sgn * (0.5 / 6.0) * (na[a] + 4.0 * nm[a] + nb[a]);
  }
  // edge and displacement vectors of the moving face in FP32 (differences in FP64)
  float eB0[3], eB1[3], eC0[3], eC1[3], wA[3], wB[3], wC[3];
  for (int a = 0; a < 3; ++a) {
    eB0[a] = (float)(fg.B0[a] - fg.A0[a]);
    eB1[a] = (float)(fg.B1[a] - fg.A1[a]);
    eC0[a] = (float)(fg.C0[a] - fg.A0[a]);
    eC1[a] = (float)(fg.C1[a] - fg.A1[a]);
    wA[a] = (float)(fg.A1[a] - fg.A0[a]);
    wB[a] = (float)(fg.B1[a] - fg.B0[a]);
    wC[a] = (float)(fg.C1[a] - fg.C0[a]);
  }
  const float sg = (float)sgn, dt32 = (float)dt;
  double QL[5], QR[5];
  float qbL[5], qbR[5], dQ[5];
  for (int v = 0; v < 5; ++v) {
    QL[v] = Q[v * N + cl];
    QR[v] = cr >= 0 ? Q[v * N + cr] : QL[v];
    qbL[v] = (float)QL[v];
    qbR[v] = (float)QR[v];
    dQ[v] = (float)(QR[v] - QL[v]);
  }
  float FbL[3][5], FbR[3][5], Vd[3];
  ale_flux3f(qbL, t.gamma, CWENO_MOTION_FIXED, FbL, Vd);
  ale_flux3f(qbR, t.gamma, CWENO_MOTION_FIXED, FbR, Vd);
  const float* qL = qhat + cl * L * 5;
  const float* qR = qhat + (cr >= 0 ? cr : cl) * L * 5;
  float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  constexpr int NP = NQS * NQT, PC = point_chunk(NP, 9);
  for (int p0 = 0; p0 < NP; p0 += PC) {
    float dmc[PC][5], dpc[PC][5];
#pragma unroll
    for (int j = 0; j < PC; ++j)
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        dmc[j][v] = 0.f;
        dpc[j][v] = 0.f;
      }
    for (int l = 0; l < L; ++l) {
      float xa[5], xb[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        xa[v] = qL[l * 5 + v];
        xb[v] = qR[l * 5 + v];
      }
#pragma unroll
      for (int j = 0; j < PC; ++j) {
        const int pj = p0 + j, qj = pj / NQT, tj = pj % NQT;
        const float wl = ftab[((int64_t)(kL * NQT + tj) * NQS + qj) * L + l];
        const float wr = ftab[((int64_t)(kR * NQT + tj) * NQS + qj) * L + l];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          dmc[j][v] += wl * xa[v];
          dpc[j][v] += wr * xb[v];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < PC; ++j) {
      const int qp = (p0 + j) / NQT, tt = (p0 + j) % NQT;
      float dm[5], dp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        dm[v] = dmc[j][v];
        dp[v] = dpc[j][v];
      }
      if (cr < 0)
        for (int v = 0; v < 5; ++v) dp[v] = dm[v];
      float qm[5], qq[5];
      for (int v = 0; v < 5; ++v) {
        qm[v] = qbL[v] + dm[v];
        qq[v] = qbR[v] + dp[v];
      }
      if (t.pos) {
        if (!admissible3f(qm, t.gamma))
          for (int v = 0; v < 5; ++v) {
            qm[v] = qbL[v];
            dm[v] = 0.f;
          }
        if (!admissible3f(qq, t.gamma))
          for (int v = 0; v < 5; ++v) {
            qq[v] = qbR[v];
            dp[v] = 0.f;
          }
      }
      // space-time normal at (chi1, chi2, tau), Eq. (detChi), in FP32
      const float c1 = t.chi[qp][0], c2 = t.chi[qp][1], tau = t.tq[tt];
      float r1[3], r2[3], r3[3];
      for (int a = 0; a < 3; ++a) {
        r1[a] = (1.0f - tau) * eB0[a] + tau * eB1[a];
        r2[a] = (1.0f - tau) * eC0[a] + tau * eC1[a];
        r3[a] = (1.0f - c1 - c2) * wA[a] + c1 * wB[a] + c2 * wC[a];
      }
      float n[4];
      n[0] = sg * dt32 * (r1[1] * r2[2] - r1[2] * r2[1]);
      n[1] = sg * dt32 * (r1[2] * r2[0] - r1[0] * r2[2]);
      n[2] = sg * dt32 * (r1[0] * r2[1] - r1[1] * r2[0]);
      n[3] = -sg * (r1[0] * (r2[1] * r3[2] - r2[2] * r3[1]) - r1[1] * (r2[0] * r3[2] - r2[2] * r3[0]) +
                    r1[2] * (r2[0] * r3[1] - r2[1] * r3[0]));
      const float nx = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]), inx = 1.0f / nx;
      const float un[3] = {n[0] * inx, n[1] * inx, n[2] * inx};
      const float Vn = -n[3] * inx;
      float sm = 0.0f, dfs[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      const float* sides[2] = {qm, qq};
      for (int s = 0; s < 2; ++s) {
        const float* z = sides[s];
        float Fz[3][5], Vz[3];
        ale_flux3f(z, t.gamma, CWENO_MOTION_FIXED, Fz, Vz);
        const float ir = 1.0f / z[0];
        const float u[3] = {z[1] * ir, z[2] * ir, z[3] * ir};
        const float p = (t.gamma - 1.0f) * (z[4] - 0.5f * (z[1] * u[0] + z[2] * u[1] + z[3] * u[2]));
        const float c = sqrtf(fmaxf(0.0f, t.gamma * p * ir));
        sm = fmaxf(sm, fabsf(u[0] * un[0] + u[1] * un[1] + u[2] * un[2] - Vn) + c);
        const float(*Fb)[5] = s == 0 ? FbL : FbR;
        for (int v = 0; v < 5; ++v)
          dfs[v] += (Fz[0][v] - Fb[0][v]) * n[0] + (Fz[1][v] - Fb[1][v]) * n[1] + (Fz[2][v] - Fb[2][v]) * n[2];
      }
      sm *= nx;
      const float wgt = 0.5f * t.wq[qp] * t.wt[tt];  // reference triangle area 1/2
      for (int v = 0; v < 5; ++v)
        acc[v] += wgt * (0.5f * dfs[v] + 0.5f * (dm[v] + dp[v]) * n[3] - 0.5f * sm * (dQ[v] + dp[v] - dm[v]));
    }
  }
  double FL[3][5], FR[3][5];
  euler_xyz64(QL, gamma64, FL);
  euler_xyz64(QR, gamma64, FR);
  for (int v = 0; v < 5; ++v)
    G[v * F + f] = (double)acc[v] +
                   0.5 * ((FL[0][v] + FR[0][v]) * nbar[0] + (FL[1][v] + FR[1][v]) * nbar[1] +
                          (FL[2][v] + FR[2][v]) * nbar[2]) +
                   0.5 * (QL[v] + QR[v]) * nbar[3];
}

// ------------------------------------------------------------------- update
__global__ void __launch_bounds__(256) k_ale_update3(const int32_t* __restrict__ cellface, const double* __restrict__ G,
                                                     const int32_t* __restrict__ gv, const double* __restrict__ shift,
                                                     const double* __restrict__ Xv1, const double* __restrict__ vol0,
                                                     int64_t N, int64_t F, double gamma, double dt_fixed, double cfl,
                                                     const unsigned long long* dtmin, double* __restrict__ Q,
                                                     float* __restrict__ Qp, double* time, int* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *time += step_dt(dt_fixed, cfl, dtmin);
  if (i >= N) return;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int k = 0; k < 4; ++k) {
    const int32_t cf = cellface[k * N + i];
    const int64_t f = cf >> 1;
    const double s = (cf & 1) ? -1.0 : 1.0;
    for (int v = 0; v < 5; ++v) acc[v] += s * G[v * F + f];
  }
  double P[4][3];
  for (int k = 0; k < 4; ++k) {
    const int64_t g = gv[k * N + i];
    for (int a = 0; a < 3; ++a) P[k][a] = Xv1[g * 3 + a] + shift[(k * 3 + a) * N + i];
  }
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 3; ++a) e[k][a] = P[k + 1][a] - P[0][a];
  const double v1 = det3(e[0], e[1], e[2]) / 6.0, v0 = vol0[i];
  double q[5];
  for (int v = 0; v < 5; ++v) {
    q[v] = (v0 * Q[v * N + i] - acc[v]) / v1;
    Q[v * N + i] = q[v];
  }
  if (Qp) {  // FP32-mixed: the state's FP32 pairs, six variables (one padding)
    float pr[12];
    for (int v = 0; v < 6; ++v) {
      float hi = 0.f, lo = 0.f;
      if (v < 5) split_hilo(q[v], hi, lo);
      pr[2 * v] = hi;
      pr[2 * v + 1] = lo;
    }
    float4* dst = reinterpret_cast<float4*>(Qp) + i * 3;
    for (int m = 0; m < 3; ++m) dst[m] = make_float4(pr[4 * m], pr[4 * m + 1], pr[4 * m + 2], pr[4 * m + 3]);
  }
  if (!(v1 > 0.0) || !admissible3(q, gamma)) atomicOr(status, 1);
}

}  // namespace
