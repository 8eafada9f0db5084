#include "refelem.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace cw {

int mcal(int M, int d) {
  // (1/d!) prod_{l=1..d} (M+l), Eq. (cwenoM)
  long num = 1, den = 1;
  for (int l = 1; l <= d; ++l) {
    num *= (M + l);
    den *= l;
  }
  return (int)(num / den);
}

// ---------------------------------------------------------- Golub-Welsch
// Symmetric eigenproblem of the Jacobi (three-term recurrence) matrix by
// cyclic Jacobi rotations; eigenvalues are the nodes, the squared first
// components of the eigenvectors times mu_0 the weights.
static void sym_eig(int n, std::vector<double>& A, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-32) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A R
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- R^T A
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> J((size_t)n * n, 0.0), V;
  for (int k = 0; k < n; ++k) {
    double s = 2.0 * k + a + b;
    double diag = (s == 0.0 || (s + 2.0) == 0.0) ? (b - a) / (a + b + 2.0) : (b * b - a * a) / (s * (s + 2.0));
    if (k == 0) diag = (b - a) / (a + b + 2.0);
    J[k * n + k] = diag;
    if (k + 1 < n) {
      double m = k + 1.0;
      double sm = 2.0 * m + a + b;
      double num = 4.0 * m * (m + a) * (m + b) * (m + a + b);
      double den = sm * sm * (sm + 1.0) * (sm - 1.0);
      double off = std::sqrt(num / den);
      J[k * n + k + 1] = off;
      J[(k + 1) * n + k] = off;
    }
  }
  sym_eig(n, J, V);
  double mu0 = std::pow(2.0, a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) / std::tgamma(a + b + 2.0);
  std::vector<std::pair<double, double>> nw(n);
  for (int i = 0; i < n; ++i) nw[i] = {J[i * n + i], mu0 * V[0 * n + i] * V[0 * n + i]};
  std::sort(nw.begin(), nw.end());
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    x[i] = nw[i].first;
    w[i] = nw[i].second;
  }
}

SimplexQuad simplex_quad(int d, int n) {
  SimplexQuad Q;
  Q.d = d;
  std::vector<double> x1, w1, x2, w2, x3, w3;
  gauss_jacobi(n, 0.0, 0.0, x1, w1);
  gauss_jacobi(n, 1.0, 0.0, x2, w2);
  if (d == 2) {
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        double s = 0.5 * (1.0 + x1[a]), t = 0.5 * (1.0 + x2[b]);
        Q.x.push_back({s * (1.0 - t), t, 0.0});
        Q.w.push_back(w1[a] * w2[b] / 8.0);
      }
  } else {
    gauss_jacobi(n, 2.0, 0.0, x3, w3);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b)
        for (int c = 0; c < n; ++c) {
          double s = 0.5 * (1.0 + x1[a]), t = 0.5 * (1.0 + x2[b]), u = 0.5 * (1.0 + x3[c]);
          Q.x.push_back({s * (1.0 - t) * (1.0 - u), t * (1.0 - u), u});
          Q.w.push_back(w1[a] * w2[b] * w3[c] / 64.0);
        }
  }
  return Q;
}

// ---------------------------------------------------------- power form
std::vector<std::array<int, 4>> graded_monomials(int nvar, int deg) {
  std::vector<std::array<int, 4>> out;
  for (int k = 0; k <= deg; ++k) {
    // all exponent tuples of total degree k, last variable outermost
    std::array<int, 4> e = {0, 0, 0, 0};
    std::vector<std::array<int, 4>> lvl;
    if (nvar == 1) lvl.push_back({k, 0, 0, 0});
    else if (nvar == 2)
      for (int b = 0; b <= k; ++b) lvl.push_back({k - b, b, 0, 0});
    else if (nvar == 3)
      for (int c = 0; c <= k; ++c)
        for (int b = 0; b <= k - c; ++b) lvl.push_back({k - b - c, b, c, 0});
    else
      for (int t = 0; t <= k; ++t)
        for (int c = 0; c <= k - t; ++c)
          for (int b = 0; b <= k - t - c; ++b) lvl.push_back({k - b - c - t, b, c, t});
    (void)e;
    out.insert(out.end(), lvl.begin(), lvl.end());
  }
  return out;
}

double PPoly::eval(const double* x) const {
  double s = 0.0;
  for (size_t k = 0; k < c.size(); ++k) {
    if (c[k] == 0.0) continue;
    double m = c[k];
    for (int a = 0; a < nvar; ++a) {
      int p = e[k][a];
      double xa = x[a];
      while (p-- > 0) m *= xa;
    }
    s += m;
  }
  return s;
}

PPoly PPoly::deriv(int var) const {
  PPoly r;
  r.nvar = nvar;
  for (size_t k = 0; k < c.size(); ++k) {
    if (e[k][var] == 0 || c[k] == 0.0) continue;
    std::array<int, 4> ee = e[k];
    double cc = c[k] * ee[var];
    ee[var] -= 1;
    r.e.push_back(ee);
    r.c.push_back(cc);
  }
  return r;
}

template <typename R>
static bool lu_solve_t(int n, std::vector<R> A, std::vector<R>& B, int nrhs) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    R best = std::fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > best) {
        best = std::fabs(A[i * n + k]);
        p = i;
      }
    if (best == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      for (int j = 0; j < nrhs; ++j) std::swap(B[k * nrhs + j], B[p * nrhs + j]);
    }
    R inv = R(1) / A[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      R f = A[i * n + k] * inv;
      A[i * n + k] = f;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      for (int j = 0; j < nrhs; ++j) B[i * nrhs + j] -= f * B[k * nrhs + j];
    }
  }
  for (int j = 0; j < nrhs; ++j)
    for (int k = n - 1; k >= 0; --k) {
      R s = B[k * nrhs + j];
      for (int i = k + 1; i < n; ++i) s -= A[k * n + i] * B[i * nrhs + j];
      B[k * nrhs + j] = s / A[k * n + k];
    }
  return true;
}

bool lu_solve(int n, std::vector<double> A, std::vector<double>& B, int nrhs) {
  return lu_solve_t<double>(n, std::move(A), B, nrhs);
}

// Homogenised Jacobi polynomial s^n P_n^{(alpha,0)}(u/s) by the three-term
// recurrence multiplied through by s^n (no division by s).
static double jacobi_h(int n, double alpha, double u, double s) {
  if (n == 0) return 1.0;
  double b = 0.0;
  double p0 = 1.0;
  double p1 = 0.5 * ((alpha + b + 2.0) * u + (alpha - b) * s);
  for (int k = 2; k <= n; ++k) {
    double kk = k;
    double c = 2.0 * kk + alpha + b;
    double a1 = 2.0 * kk * (kk + alpha + b) * (c - 2.0);
    double a2 = (c - 1.0) * (alpha * alpha - b * b);
    double a3 = (c - 2.0) * (c - 1.0) * c;
    double a4 = 2.0 * (kk + alpha - 1.0) * (kk + b - 1.0) * c;
    double p2 = ((a2 * s + a3 * u) * p1 - a4 * s * s * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

static double dubiner_raw(int d, const std::array<int, 3>& id, const double* xi) {
  if (d == 2) {
    double s1 = 1.0 - xi[1];
    double u1 = 2.0 * xi[0] - s1;
    return jacobi_h(id[0], 0.0, u1, s1) * jacobi_h(id[1], 2.0 * id[0] + 1.0, 2.0 * xi[1] - 1.0, 1.0);
  }
  double s1 = 1.0 - xi[1] - xi[2], u1 = 2.0 * xi[0] - s1;
  double s2 = 1.0 - xi[2], u2 = 2.0 * xi[1] - s2;
  return jacobi_h(id[0], 0.0, u1, s1) * jacobi_h(id[1], 2.0 * id[0] + 1.0, u2, s2) *
         jacobi_h(id[2], 2.0 * id[0] + 2.0 * id[1] + 2.0, 2.0 * xi[2] - 1.0, 1.0);
}

void Dubiner::init(int d_, int M_) {
  d = d_;
  M = M_;
  // recurrence coefficients for alpha = 0 .. 2M + 2 (the Jacobi weights the
  // collapsed directions need), the same three-term recurrence as jacobi_h
  rec.assign((size_t)(2 * M + 3) * (M + 1), {0.0, 0.0, 0.0});
  for (int al = 0; al <= 2 * M + 2; ++al)
    for (int k = 2; k <= M; ++k) {
      const double alpha = al, kk = k, c = 2.0 * kk + alpha;
      const double a1 = 2.0 * kk * (kk + alpha) * (c - 2.0);
      const double a2 = (c - 1.0) * (alpha * alpha);
      const double a3 = (c - 2.0) * (c - 1.0) * c;
      const double a4 = 2.0 * (kk + alpha - 1.0) * (kk - 1.0) * c;
      rec[(size_t)al * (M + 1) + k] = {a2 / a1, a3 / a1, a4 / a1};
    }
  pqr.clear();
  for (int k = 0; k <= M; ++k) {
    if (d == 2) {
      for (int q = 0; q <= k; ++q) pqr.push_back({k - q, q, 0});
    } else {
      for (int r = 0; r <= k; ++r)
        for (int q = 0; q <= k - r; ++q) pqr.push_back({k - q - r, q, r});
    }
  }
  n = (int)pqr.size();
  norm.assign(n, 1.0);
  SimplexQuad Q = simplex_quad(d, M + 2);
  for (int l = 1; l < n; ++l) {
    double s = 0.0;
    for (size_t g = 0; g < Q.w.size(); ++g) {
      double v = dubiner_raw(d, pqr[l], Q.x[g].data());
      s += Q.w[g] * v * v;
    }
    norm[l] = 1.0 / std::sqrt(s);
  }
  // power form by interpolation on the degree-M lattice (unisolvent)
  std::vector<std::array<int, 4>> mono = graded_monomials(d, M);
  std::vector<std::array<double, 3>> pts;
  if (d == 2) {
    for (int j = 0; j <= M; ++j)
      for (int i = 0; i <= M - j; ++i) pts.push_back({(double)i / M, (double)j / M, 0.0});
  } else {
    for (int k = 0; k <= M; ++k)
      for (int j = 0; j <= M - k; ++j)
        for (int i = 0; i <= M - j - k; ++i) pts.push_back({(double)i / M, (double)j / M, (double)k / M});
  }
  std::vector<double> V((size_t)n * n), B((size_t)n * n);
  for (int r = 0; r < n; ++r) {
    for (int k = 0; k < n; ++k) {
      double m = 1.0;
      for (int a = 0; a < d; ++a) m *= std::pow(pts[r][a], mono[k][a]);
      V[r * n + k] = m;
    }
    double vals[64];
    eval(pts[r].data(), vals);
    for (int l = 0; l < n; ++l) B[r * n + l] = vals[l];
  }
  if (!lu_solve(n, V, B, n)) throw std::runtime_error("singular lattice Vandermonde");
  power.assign(n, PPoly());
  for (int l = 0; l < n; ++l) {
    power[l].nvar = d;
    power[l].e = mono;
    power[l].c.resize(n);
    for (int k = 0; k < n; ++k) power[l].c[k] = B[k * n + l];
  }
}

// p[k] = s^k P_k^(alpha,0)(u/s), k = 0..nmax, by the precomputed recurrence
void Dubiner::jacobi_seq(int alpha, int nmax, double u, double s, double* p) const {
  p[0] = 1.0;
  if (nmax < 1) return;
  p[1] = 0.5 * ((alpha + 2.0) * u + alpha * s);
  for (int k = 2; k <= nmax; ++k) {
    const std::array<double, 3>& r = rec[(size_t)alpha * (M + 1) + k];
    p[k] = (r[0] * s + r[1] * u) * p[k - 1] - r[2] * s * s * p[k - 2];
  }
}

// All basis functions at one point, sharing the Jacobi sequences of the
// collapsed directions (one recurrence per direction and outer index).
void Dubiner::eval(const double* xi, double* out) const {
  double f1[16], f2[16][16], f3[16];
  if (d == 2) {
    const double s1 = 1.0 - xi[1], u1 = 2.0 * xi[0] - s1;
    jacobi_seq(0, M, u1, s1, f1);
    for (int p = 0; p <= M; ++p) jacobi_seq(2 * p + 1, M - p, 2.0 * xi[1] - 1.0, 1.0, f2[p]);
    out[0] = 1.0;
    for (int l = 1; l < n; ++l) out[l] = norm[l] * (f1[pqr[l][0]] * f2[pqr[l][0]][pqr[l][1]]);
    return;
  }
  const double s1 = 1.0 - xi[1] - xi[2], u1 = 2.0 * xi[0] - s1;
  const double s2 = 1.0 - xi[2], u2 = 2.0 * xi[1] - s2;
  jacobi_seq(0, M, u1, s1, f1);
  for (int p = 0; p <= M; ++p) jacobi_seq(2 * p + 1, M - p, u2, s2, f2[p]);
  out[0] = 1.0;
  for (int l = 1; l < n; ++l) {
    const int p = pqr[l][0], q = pqr[l][1], r = pqr[l][2];
    jacobi_seq(2 * p + 2 * q + 2, r, 2.0 * xi[2] - 1.0, 1.0, f3);
    out[l] = norm[l] * (f1[p] * f2[p][q] * f3[r]);
  }
}

// ---------------------------------------------------------- face codes
static const int PERM3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

int face_code(int d, const int* ol, int* local_face) {
  int present[4] = {0, 0, 0, 0};
  for (int k = 0; k < d; ++k) present[ol[k]] = 1;
  int lf = -1;
  for (int k = 0; k <= d; ++k)
    if (!present[k]) lf = k;
  *local_face = lf;
  int asc[3], n = 0;
  for (int k = 0; k <= d; ++k)
    if (k != lf) asc[n++] = k;
  if (d == 2) return lf * 2 + (ol[0] == asc[0] ? 0 : 1);
  for (int p = 0; p < 6; ++p)
    if (ol[0] == asc[PERM3[p][0]] && ol[1] == asc[PERM3[p][1]] && ol[2] == asc[PERM3[p][2]]) return lf * 6 + p;
  return -1;
}

static void ref_vertex(int d, int k, double* v) {
  for (int a = 0; a < 3; ++a) v[a] = 0.0;
  if (k > 0) v[k - 1] = 1.0;
  (void)d;
}

// ---------------------------------------------------------- RefElem
void RefElem::init(int d_, int M_) {
  d = d_;
  M = M_;
  Mc = mcal(M, d);
  ne = d * Mc;
  L = mcal(M, d + 1);
  L0 = Mc;
  L1 = L - L0;
  psi.init(d, M);
  // lattice nodes (zeta outermost, then eta, then xi)
  lattice.clear();
  if (d == 2) {
    for (int j = 0; j <= M; ++j)
      for (int i = 0; i <= M - j; ++i) lattice.push_back({(double)i / M, (double)j / M, 0.0});
  } else {
    for (int k = 0; k <= M; ++k)
      for (int j = 0; j <= M - k; ++j)
        for (int i = 0; i <= M - j - k; ++i) lattice.push_back({(double)i / M, (double)j / M, (double)k / M});
  }
  // space-time nodes: principal lattice of the (d+1)-simplex, tau level outermost
  stnode.clear();
  for (int t = 0; t <= M; ++t) {
    int K = M - t;
    if (d == 2) {
      for (int j = 0; j <= K; ++j)
        for (int i = 0; i <= K - j; ++i) stnode.push_back({(double)i / M, (double)j / M, 0.0, (double)t / M});
    } else {
      for (int k = 0; k <= K; ++k)
        for (int j = 0; j <= K - k; ++j)
          for (int i = 0; i <= K - j - k; ++i)
            stnode.push_back({(double)i / M, (double)j / M, (double)k / M, (double)t / M});
    }
  }
  if ((int)stnode.size() != L) throw std::runtime_error("space-time node count");
  // E: basis at the lattice
  E.assign((size_t)Mc * (Mc - 1), 0.0);
  for (int n = 0; n < Mc; ++n) {
    double v[64];
    psi.eval(lattice[n].data(), v);
    for (int l = 1; l < Mc; ++l) E[n * (Mc - 1) + (l - 1)] = v[l];
  }
  // Sigma_lm = sum_{1<=|alpha|<=M} int d^alpha psi_l d^alpha psi_m
  {
    SimplexQuad Q = simplex_quad(d, M + 1);
    std::vector<std::array<int, 4>> alphas = graded_monomials(d, M);
    Sigma.assign((size_t)(Mc - 1) * (Mc - 1), 0.0);
    for (const auto& al : alphas) {
      int tot = al[0] + al[1] + al[2];
      if (tot < 1) continue;
      std::vector<PPoly> dp(Mc);
      for (int l = 0; l < Mc; ++l) {
        PPoly p = psi.power[l];
        for (int a = 0; a < d; ++a)
          for (int r = 0; r < al[a]; ++r) p = p.deriv(a);
        dp[l] = p;
      }
      for (size_t g = 0; g < Q.w.size(); ++g) {
        std::vector<double> vals(Mc);
        for (int l = 1; l < Mc; ++l) vals[l] = dp[l].eval(Q.x[g].data());
        for (int l = 1; l < Mc; ++l)
          for (int m = 1; m < Mc; ++m) Sigma[(l - 1) * (Mc - 1) + (m - 1)] += Q.w[g] * vals[l] * vals[m];
      }
    }
  }
  // Space-time nodal basis theta_l = sum_k Cb[k][l] m_k(xi, tau) in
  // monomials of (xi_0..xi_{d-1}, tau), built and evaluated in extended
  // precision (long double): the coefficients reach 2.6e2 at M = 4, so
  // double evaluation would lose about 1e-13.
  using LD = long double;
  std::vector<std::array<int, 4>> stm = graded_monomials(d + 1, M);
  std::vector<LD> V((size_t)L * L), Cb((size_t)L * L, 0.0L);
  auto ipow = [](LD x, int n) {
    LD r = 1.0L;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
  };
  for (int n = 0; n < L; ++n) {
    LD x[4];
    for (int a = 0; a < d; ++a) x[a] = (LD)stnode[n][a];
    x[d] = (LD)stnode[n][3];
    for (int k = 0; k < L; ++k) {
      LD m = 1.0L;
      for (int a = 0; a <= d; ++a) m *= ipow(x[a], stm[k][a]);
      V[n * L + k] = m;
    }
  }
  for (int k = 0; k < L; ++k) Cb[k * L + k] = 1.0L;
  if (!lu_solve_t<LD>(L, V, Cb, L)) throw std::runtime_error("singular space-time Vandermonde");
  // theta_l at (xi, tau), variables x[0..d-1] = xi, x[d] = tau
  auto theta = [&](int l, const LD* x) {
    LD s = 0.0L;
    for (int k = 0; k < L; ++k) {
      LD m = Cb[k * L + l];
      for (int a = 0; a <= d; ++a) m *= ipow(x[a], stm[k][a]);
      s += m;
    }
    return s;
  };
  // Predictor matrices in closed form.  With the nodal flux interpolant in
  // P_M, q(xi, tau) = q(xi, 0) - dt int_0^tau H(xi, s) ds is a degree-M
  // polynomial with d_tau q + dt H = 0 pointwise, so the residual of Eq.
  // (CGfinal) vanishes for every test function and (K_tau^1 being
  // invertible) it is the Galerkin solution.  At the unknown node k:
  //   C0[k][n]   = theta_n(xi_k, 0)  (the tau = 0 data extended in time),
  //   P_e[k][l]  = int_0^{tau_k} d theta_l / d xi_e (xi_k, s) ds,
  // the latter integrated exactly monomial by monomial.  This never forms
  // (K_tau^1)^-1, whose condition number is 1.5e4 at M = 3 and 1.4e6 at M = 4.
  C0.assign((size_t)L1 * L0, 0.0);
  P.assign((size_t)d * L1 * L, 0.0);
  for (int k = 0; k < L1; ++k) {
    const std::array<double, 4>& nk = stnode[L0 + k];
    LD x0[4];
    for (int a = 0; a < d; ++a) x0[a] = (LD)nk[a];
    x0[d] = 0.0L;
    for (int n = 0; n < L0; ++n) C0[k * L0 + n] = (double)theta(n, x0);
    const LD tk = (LD)nk[3];
    for (int e = 0; e < d; ++e)
      for (int l = 0; l < L; ++l) {
        LD s = 0.0L;
        for (int j = 0; j < L; ++j) {
          const int pe = stm[j][e];
          if (pe == 0) continue;
          LD m = Cb[j * L + l] * pe;
          for (int a = 0; a < d; ++a) m *= ipow((LD)nk[a], a == e ? stm[j][a] - 1 : stm[j][a]);
          const int pt = stm[j][d];
          m *= ipow(tk, pt + 1) / (LD)(pt + 1);
          s += m;
        }
        P[((size_t)e * L1 + k) * L + l] = (double)s;
      }
  }
  // Moving-mesh predictor tables.  K_tau and M (rows: test functions of the
  // tau > 0 nodes) by the collapsed Gauss rule on T_E times Gauss-Legendre
  // on [0, 1], exact for their degree 2M; Gal = (K_tau^1)^-1 M^1 solved in
  // extended precision (K_tau^1 has condition number 1.5e4 at M = 3).  In
  // exact arithmetic -(K_tau^1)^-1 K_tau^0 is the constant extension C0 above,
  // so only Gal is new.
  {
    auto dtheta = [&](int l, int e, const LD* x) {
      LD s = 0.0L;
      for (int k = 0; k < L; ++k) {
        const int pe = stm[k][e];
        if (pe == 0) continue;
        LD m = Cb[k * L + l] * (LD)pe;
        for (int a = 0; a <= d; ++a) m *= ipow(x[a], a == e ? stm[k][a] - 1 : stm[k][a]);
        s += m;
      }
      return s;
    };
    Dxi.assign((size_t)d * L * L, 0.0);
    for (int e = 0; e < d; ++e)
      for (int n = 0; n < L; ++n) {
        LD x[4];
        for (int a = 0; a < d; ++a) x[a] = (LD)stnode[n][a];
        x[d] = (LD)stnode[n][3];
        for (int l = 0; l < L; ++l) Dxi[((size_t)e * L + n) * L + l] = (double)dtheta(l, e, x);
      }
    SimplexQuad Qs = simplex_quad(d, M + 1);
    std::vector<double> gx, gw;
    gauss_jacobi(M + 1, 0.0, 0.0, gx, gw);
    std::vector<LD> Kt((size_t)L1 * L, 0.0L), Mm((size_t)L1 * L, 0.0L);
    std::vector<LD> th(L), dtt(L);
    for (size_t g = 0; g < Qs.w.size(); ++g)
      for (int t = 0; t <= M; ++t) {
        LD x[4];
        for (int a = 0; a < d; ++a) x[a] = (LD)Qs.x[g][a];
        x[d] = 0.5L * (1.0L + (LD)gx[t]);
        const LD w = (LD)Qs.w[g] * 0.5L * (LD)gw[t];
        for (int l = 0; l < L; ++l) {
          th[l] = theta(l, x);
          dtt[l] = dtheta(l, d, x);
        }
        for (int k = 0; k < L1; ++k)
          for (int l = 0; l < L; ++l) {
            Kt[(size_t)k * L + l] += w * th[L0 + k] * dtt[l];
            Mm[(size_t)k * L + l] += w * th[L0 + k] * th[l];
          }
      }
    std::vector<LD> K1((size_t)L1 * L1);
    for (int k = 0; k < L1; ++k)
      for (int l = 0; l < L1; ++l) K1[(size_t)k * L1 + l] = Kt[(size_t)k * L + L0 + l];
    if (!lu_solve_t<LD>(L1, K1, Mm, L)) throw std::runtime_error("singular K_tau^1");
    Gal.assign((size_t)L1 * L, 0.0);
    for (size_t k = 0; k < Mm.size(); ++k) Gal[k] = (double)Mm[k];
    Wv.assign((size_t)(d + 1) * L, 0.0);
    for (int v = 0; v <= d; ++v)
      for (int t = 0; t <= M; ++t) {
        LD x[4] = {0.0L, 0.0L, 0.0L, 0.0L};
        if (v > 0) x[v - 1] = 1.0L;
        x[d] = 0.5L * (1.0L + (LD)gx[t]);
        for (int l = 0; l < L; ++l) Wv[(size_t)v * L + l] += (double)(0.5L * (LD)gw[t] * theta(l, x));
      }
  }
  // face quadrature tables
  {
    std::vector<double> gx, gw, jx, jw;
    gauss_jacobi(M + 1, 0.0, 0.0, gx, gw);
    gauss_jacobi(M + 1, 1.0, 0.0, jx, jw);
    nqt = M + 1;
    tq.assign(nqt, 0.0);
    wt.assign(nqt, 0.0);
    for (int t = 0; t < nqt; ++t) {
      tq[t] = 0.5 * (1.0 + gx[t]);
      wt[t] = 0.5 * gw[t];
    }
    std::vector<std::array<double, 2>> chi;
    wq.clear();
    if (d == 2) {
      for (int a = 0; a <= M; ++a) {
        chi.push_back({0.5 * (1.0 + gx[a]), 0.0});
        wq.push_back(0.5 * gw[a]);
      }
    } else {
      double sw = 0.0;
      for (int a = 0; a <= M; ++a)
        for (int b = 0; b <= M; ++b) {
          double s = 0.5 * (1.0 + gx[a]), t = 0.5 * (1.0 + jx[b]);
          chi.push_back({s * (1.0 - t), t});
          wq.push_back(gw[a] * jw[b]);
          sw += gw[a] * jw[b];
        }
      for (double& w : wq) w /= sw;
    }
    nqs = (int)chi.size();
    this->chi.clear();
    if (d == 2)
      for (const auto& c : chi) this->chi.push_back(c[0]);
    chi3.clear();
    if (d == 3)
      for (const auto& c : chi) {
        chi3.push_back(c[0]);
        chi3.push_back(c[1]);
      }
    ncode = (d == 2) ? 6 : 24;
    ftab.assign((size_t)ncode * nqt * nqs * L, 0.0);
    std::vector<LD> fi((size_t)ncode * L, 0.0L);
    for (int code = 0; code < ncode; ++code) {
      int lf = (d == 2) ? code / 2 : code / 6;
      int asc[3], n = 0;
      for (int k = 0; k <= d; ++k)
        if (k != lf) asc[n++] = k;
      int ol[3];
      if (d == 2) {
        int o = code % 2;
        ol[0] = o ? asc[1] : asc[0];
        ol[1] = o ? asc[0] : asc[1];
      } else {
        int p = code % 6;
        for (int r = 0; r < 3; ++r) ol[r] = asc[PERM3[p][r]];
      }
      double vA[3], vB[3], vC[3];
      ref_vertex(d, ol[0], vA);
      ref_vertex(d, ol[1], vB);
      if (d == 3) ref_vertex(d, ol[2], vC);
      for (int t = 0; t < nqt; ++t)
        for (int q = 0; q < nqs; ++q) {
          LD x[4];
          for (int a = 0; a < d; ++a) {
            double xa = vA[a] + chi[q][0] * (vB[a] - vA[a]);
            if (d == 3) xa += chi[q][1] * (vC[a] - vA[a]);
            x[a] = (LD)xa;
          }
          x[d] = (LD)tq[t];
          for (int l = 0; l < L; ++l) {
            const LD th = theta(l, x);
            ftab[(((size_t)code * nqt + t) * nqs + q) * L + l] = (double)th;
            fi[(size_t)code * L + l] += (LD)wt[t] * (LD)wq[q] * th;
          }
        }
    }
    fint.assign((size_t)ncode * L, 0.0);
    for (size_t k = 0; k < fi.size(); ++k) fint[k] = (double)fi[k];
  }
}

}  // namespace cw
