// ============================================================================
// ORACLE -- test infrastructure only.
//
// A plain, slow, FP64 CPU implementation of the fixed-mesh (Eulerian) and
// the moving-mesh (direct ALE, triangles and tetrahedra, Euler, Rusanov)
// ADER-CWENO finite-volume steps of Dumbser, Boscheri, Semplice & Russo,
// "Central WENO schemes on unstructured meshes" (arXiv 1612.09335).
// It is used only by tests/, by the smoke check and by the CPU-baseline /
// reference arm of bench.py.  The product (the CUDA path) never calls it,
// links it or includes it, and it shares no code with the product.
//
// Representation: polynomials are kept as sparse lists of monomials in the
// reference coordinates (xi, eta, zeta, tau) and integrated exactly with the
// closed form  int_{T_E} xi^a eta^b zeta^c = a! b! c! / (a+b+c+d)!.
// The product path uses an orthonormal Dubiner basis and numerical
// quadrature instead; every quantity compared between the two is a value
// (basis independent), never a coefficient.
//
// Paper passages followed (section / equation labels of the paper):
//   affine map                           Sec. 2, Eq. (xietaTransf)
//   cell averages                        Eq. (cellaverage)
//   central stencil, recursive fill      Sec. 2.1, Eq. (stencil)
//   constrained least squares P_opt      Eq. (CWENO:Popt), (recpolydef)
//   sectorial stencils and P_s           Sec. 2.1 (cone rule), Eq. (CWENO:Ps)
//   P_0 and linear weights               Eq. (CWENO:P0), lambda_0=1e5, lambda_s=1
//   nonlinear weights, indicators        Eq. (CWENO:Prec), (weights), (weights2),
//                                        oscillation matrix Sigma_lm
//   time step                            Eq. (timestep)
//   space-time Galerkin predictor        Sec. 2.2, Eqs. (PDExi2)-(CGfinal)
//   one-step finite volume update        Sec. 2.4, Eq. (PDEfinal), Eulerian case
//   Rusanov flux                         Eq. (rusanov)
//   Osher-type flux (Euler, switchable)  Eq. (osher), |A| = R|Lambda|R^-1
//   quadrature-free Rusanov (switchable) fixed-mesh form described after Eq. (osher)
//   Euler equations / EOS                Eqs. (eulerTerms), (eos)
//   ideal MHD with GLM cleaning          Eqs. (MHDTerms), (MHDeos)
//   moving meshes: predictor on a moving Sec. 2.2, Eqs. (PDExi2), (Hterm),
//     element with the trajectory eq.    (CGfinal), (ODEfinal), (xh_vh)
//   nodal solver and new vertices        Sec. 2.3, Eqs. (NScs)-(newX)
//   space-time control volumes, normals  Sec. 2.4, Eqs. (dCi)-(detChi)
//   ALE update and Rusanov flux          Eqs. (PDEfinal), (rusanov) with A_n^V
//
// Readings where the paper is silent (documented in the design notes):
//   * stencil fill = face-neighbour BFS by layers, candidates of a layer ranked
//     by distance of the (minimum-image) barycentre, then by its coordinates;
//   * sector s = first d cells of that ranked BFS sequence (extended by two
//     layers beyond the central stencil) whose barycentre has strictly positive
//     barycentric coordinates for every vertex except s; else the sector is
//     dropped and the linear weights are renormalised over the kept ones;
//   * lambda_0 = 1e5, lambda_s = 1 normalised to sum 1;
//   * predictor nodes = equispaced principal lattice of the (d+1)-simplex
//     {xi >= 0, sum(xi) + tau <= 1} with step 1/M; test functions = nodal
//     functions of the tau > 0 nodes; M+1 Picard iterations from w(xi);
//   * Rusanov s_max per quadrature point, max over both sides;
//   * Osher-type flux: the path integral of |A_n| by 3-point Gauss-Legendre;
//   * MHD EOS p = (gamma-1)(rho E - rho|v|^2/2 - |B|^2/(8 pi)).
//   * moving meshes: mesh velocity V = v (Sec. 3) or V = 0; stencils and
//     sectors fixed on the initial mesh, their matrices rebuilt each step;
//     M+1 coupled Picard iterations; a lateral face point (chi, tau) is
//     evaluated at the reference point at parameter chi on the cell's own
//     reference edge; Gauss-Legendre with M+1 points in chi and tau; the
//     vertex velocity uses the mesh velocity of the final predictor states.
//   * s_max and the time-step speed take sqrt(max(0, .)) of the sound speed.
// Addition not in the paper (switchable, on by default): a positivity
// preserving scaling of the reconstruction toward the cell average at the
// lattice nodes, first for the density, then for the pressure, with floors
// of 1e-3 of their cell-average values (the scaling
// limiter of Zhang & Shu, J. Comput. Phys. 229 (2010) 3091), and, at a face
// quadrature point where one side's predictor is not an admissible state,
// that side's cell average in place of its trace, and, where the space-time
// predictor of a cell leaves the admissible set at any node, that cell's
// average as its predictor.  Where everything is admissible none of these
// changes anything.
// ============================================================================
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

namespace {

// ---------------------------------------------------------------- polynomials
struct Term {
  int e[4];
  double c;
};
typedef std::vector<Term> Poly;

double factorial(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= k;
  return f;
}

bool exp_less(const Term& a, const Term& b) {
  for (int k = 0; k < 4; ++k)
    if (a.e[k] != b.e[k]) return a.e[k] < b.e[k];
  return false;
}

bool exp_equal(const Term& a, const Term& b) {
  for (int k = 0; k < 4; ++k)
    if (a.e[k] != b.e[k]) return false;
  return true;
}

// Merge equal monomials, drop exact zeros.
Poly normalise(Poly p) {
  std::sort(p.begin(), p.end(), exp_less);
  Poly out;
  for (const Term& t : p) {
    if (!out.empty() && exp_equal(out.back(), t))
      out.back().c += t.c;
    else
      out.push_back(t);
  }
  Poly res;
  for (const Term& t : out)
    if (t.c != 0.0) res.push_back(t);
  return res;
}

Term monomial(int a, int b, int c, int t, double coef) {
  Term x;
  x.e[0] = a;
  x.e[1] = b;
  x.e[2] = c;
  x.e[3] = t;
  x.c = coef;
  return x;
}

Poly poly_mul(const Poly& a, const Poly& b) {
  Poly r;
  r.reserve(a.size() * b.size());
  for (const Term& x : a)
    for (const Term& y : b) {
      Term z;
      for (int k = 0; k < 4; ++k) z.e[k] = x.e[k] + y.e[k];
      z.c = x.c * y.c;
      r.push_back(z);
    }
  return normalise(r);
}

Poly poly_axpy(double alpha, const Poly& a, double beta, const Poly& b) {
  Poly r;
  for (const Term& x : a) {
    Term z = x;
    z.c *= alpha;
    r.push_back(z);
  }
  for (const Term& x : b) {
    Term z = x;
    z.c *= beta;
    r.push_back(z);
  }
  return normalise(r);
}

Poly poly_deriv(const Poly& p, int var) {
  Poly r;
  for (const Term& x : p) {
    if (x.e[var] == 0) continue;
    Term z = x;
    z.c *= x.e[var];
    z.e[var] -= 1;
    r.push_back(z);
  }
  return normalise(r);
}

double poly_eval(const Poly& p, const double* x /* 4 coordinates */) {
  double s = 0.0;
  for (const Term& t : p) {
    double v = t.c;
    for (int k = 0; k < 4; ++k)
      for (int q = 0; q < t.e[k]; ++q) v *= x[k];
    s += v;
  }
  return s;
}

// Exact integral over the unit d-simplex of xi^a eta^b (zeta^c).
double simplex_integral(int d, const int* e) {
  double num = 1.0;
  int tot = 0;
  for (int k = 0; k < d; ++k) {
    num *= factorial(e[k]);
    tot += e[k];
  }
  return num / factorial(tot + d);
}

// Exact integral of a polynomial over T_E (spatial variables 0..d-1, no tau).
double integrate_simplex(const Poly& p, int d) {
  double s = 0.0;
  for (const Term& t : p) s += t.c * simplex_integral(d, t.e);
  return s;
}

// Exact integral over the space-time element T_E x [0,1]; tau is variable 3.
double integrate_prism(const Poly& p, int d) {
  double s = 0.0;
  for (const Term& t : p) s += t.c * simplex_integral(d, t.e) / (t.e[3] + 1.0);
  return s;
}

// p(A + B u): substitute xi_k = A[k] + sum_m B[k][m] u_m for the d spatial
// variables (tau untouched).
Poly poly_compose_affine(const Poly& p, int d, const double* A, const double B[3][3]) {
  std::vector<Poly> lin(d);
  for (int k = 0; k < d; ++k) {
    Poly l;
    l.push_back(monomial(0, 0, 0, 0, A[k]));
    for (int m = 0; m < d; ++m) {
      int e[4] = {0, 0, 0, 0};
      e[m] = 1;
      l.push_back(monomial(e[0], e[1], e[2], e[3], B[k][m]));
    }
    lin[k] = normalise(l);
  }
  Poly r;
  for (const Term& t : p) {
    Poly prod;
    prod.push_back(monomial(0, 0, 0, t.e[3], t.c));
    for (int k = 0; k < d; ++k)
      for (int q = 0; q < t.e[k]; ++q) prod = poly_mul(prod, lin[k]);
    r.insert(r.end(), prod.begin(), prod.end());
  }
  return normalise(r);
}

// Monomial exponents of total degree <= M in nvar variables (graded order).
std::vector<std::array<int, 4>> monomial_list(int nvar, int M) {
  std::vector<std::array<int, 4>> out;
  for (int deg = 0; deg <= M; ++deg) {
    if (nvar == 2) {
      for (int b = 0; b <= deg; ++b) out.push_back({deg - b, b, 0, 0});
    } else if (nvar == 3) {
      for (int c = 0; c <= deg; ++c)
        for (int b = 0; b <= deg - c; ++b) out.push_back({deg - b - c, b, c, 0});
    } else {
      for (int t = 0; t <= deg; ++t)
        for (int c = 0; c <= deg - t; ++c)
          for (int b = 0; b <= deg - t - c; ++b) out.push_back({deg - b - c - t, b, c, t});
    }
  }
  return out;
}

// Number of coefficients of P_M in d variables, Eq. (cwenoM).
int Mcal(int M, int d) {
  double p = 1.0;
  for (int l = 1; l <= d; ++l) p *= (M + l);
  return (int)std::lround(p / factorial(d));
}

// ------------------------------------------------------------ linear algebra
// Gaussian elimination with partial pivoting; solves A X = B in place
// (A n x n row-major, B n x nrhs row-major).  Returns false if singular.
bool gauss_solve(int n, std::vector<double> A, std::vector<double>& B, int nrhs) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      for (int j = 0; j < nrhs; ++j) std::swap(B[k * nrhs + j], B[p * nrhs + j]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      for (int j = 0; j < nrhs; ++j) B[i * nrhs + j] -= f * B[k * nrhs + j];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    for (int j = 0; j < nrhs; ++j) {
      double s = B[k * nrhs + j];
      for (int i = k + 1; i < n; ++i) s -= A[k * n + i] * B[i * nrhs + j];
      B[k * nrhs + j] = s / A[k * n + k];
    }
  return true;
}

// Least squares min ||A x - b|| (A m x n, m >= n, row-major) for nrhs right
// hand sides by Householder QR.  Returns false if rank deficient.
bool householder_lsq(int m, int n, std::vector<double> A, std::vector<double> B, int nrhs,
                     std::vector<double>& X) {
  for (int k = 0; k < n; ++k) {
    double norm = 0.0;
    for (int i = k; i < m; ++i) norm += A[i * n + k] * A[i * n + k];
    norm = std::sqrt(norm);
    if (norm == 0.0) return false;
    double alpha = A[k * n + k] > 0 ? -norm : norm;
    std::vector<double> v(m, 0.0);
    for (int i = k; i < m; ++i) v[i] = A[i * n + k];
    v[k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int j = k; j < n; ++j) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += v[i] * A[i * n + j];
      s = 2.0 * s / vv;
      for (int i = k; i < m; ++i) A[i * n + j] -= s * v[i];
    }
    for (int j = 0; j < nrhs; ++j) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += v[i] * B[i * nrhs + j];
      s = 2.0 * s / vv;
      for (int i = k; i < m; ++i) B[i * nrhs + j] -= s * v[i];
    }
  }
  double dmax = 0.0;
  for (int k = 0; k < n; ++k) dmax = std::max(dmax, std::fabs(A[k * n + k]));
  for (int k = 0; k < n; ++k)
    if (std::fabs(A[k * n + k]) <= 1e-13 * dmax) return false;
  X.assign((size_t)n * nrhs, 0.0);
  for (int k = n - 1; k >= 0; --k)
    for (int j = 0; j < nrhs; ++j) {
      double s = B[k * nrhs + j];
      for (int i = k + 1; i < n; ++i) s -= A[k * n + i] * X[i * nrhs + j];
      X[k * nrhs + j] = s / A[k * n + k];
    }
  return true;
}

double det3(const double J[3][3], int d) {
  if (d == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

void inv3(const double J[3][3], int d, double Ji[3][3]) {
  double det = det3(J, d);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Ji[a][b] = 0.0;
  if (d == 2) {
    Ji[0][0] = J[1][1] / det;
    Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det;
    Ji[1][1] = J[0][0] / det;
    return;
  }
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

// ------------------------------------------------------------ Gauss rules
// Legendre polynomial P_n and derivative at x by the three-term recurrence.
void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    p = 1.0;
    dp = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// n-point Gauss-Legendre rule on [0,1], weights summing to 1.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, z, p, dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(n, z, p, dp);
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/(..)/2
  }
}

// Nodes of the degree-n polynomial orthogonal on [0,1] w.r.t. weight (1-t)
// (Gauss-Jacobi alpha=1, beta=0), found as roots by bisection of the
// recurrence-generated orthogonal polynomial; weights from the moment
// equations int_0^1 (1-t) t^k dt = 1/((k+1)(k+2)), normalised to sum 1.
void gauss_jacobi10_01(int n, std::vector<double>& x, std::vector<double>& w) {
  // Orthogonal polynomials for weight (1-t) on [0,1] via Stieltjes with exact
  // moments: build monic p_k by Gram-Schmidt on monomials using moment matrix.
  auto moment = [](int k) { return 1.0 / ((k + 1.0) * (k + 2.0)); };
  // coefficients of monic orthogonal polys in the monomial basis
  std::vector<std::vector<double>> P;
  P.push_back({1.0});
  for (int k = 1; k <= n; ++k) {
    std::vector<double> q(k + 1, 0.0);
    q[k] = 1.0;
    for (int j = 0; j < k; ++j) {
      // <t^k, P_j> / <P_j, P_j>
      double num = 0.0, den = 0.0;
      for (size_t a = 0; a < P[j].size(); ++a) num += P[j][a] * moment(k + (int)a);
      for (size_t a = 0; a < P[j].size(); ++a)
        for (size_t b = 0; b < P[j].size(); ++b) den += P[j][a] * P[j][b] * moment((int)(a + b));
      for (size_t a = 0; a < P[j].size(); ++a) q[a] -= num / den * P[j][a];
    }
    P.push_back(q);
  }
  auto evalp = [&](double t) {
    double s = 0.0;
    for (int a = n; a >= 0; --a) s = s * t + P[n][a];
    return s;
  };
  // bracket roots on a fine grid, then bisect
  std::vector<double> roots;
  const int NG = 20000;
  double t0 = 0.0, f0 = evalp(0.0);
  for (int g = 1; g <= NG; ++g) {
    double t1 = (double)g / NG, f1 = evalp(t1);
    if (f0 == 0.0) roots.push_back(t0);
    else if (f0 * f1 < 0.0) {
      double a = t0, b = t1, fa = f0;
      for (int it = 0; it < 200; ++it) {
        double m = 0.5 * (a + b), fm = evalp(m);
        if (fa * fm <= 0.0) b = m;
        else {
          a = m;
          fa = fm;
        }
      }
      roots.push_back(0.5 * (a + b));
    }
    t0 = t1;
    f0 = f1;
  }
  x = roots;
  std::vector<double> V((size_t)n * n), b(n);
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < n; ++i) V[k * n + i] = std::pow(x[i], k);
    b[k] = moment(k);
  }
  gauss_solve(n, V, b, 1);
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += b[i];
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) w[i] = b[i] / s;
}

// ------------------------------------------------------------------ physics
enum { PDE_EULER = 0, PDE_MHD = 1 };

struct Params {
  double eps, r, lam0, lams, gamma, ch, cfl;
  int niter, linear_weights, positivity;
  int flux = 0;  // 0 Rusanov, Eq. (rusanov); 1 Osher-type, Eq. (osher) (Euler);
                 // 2 quadrature-free Rusanov (fixed-mesh form, after Eq. osher)
};

const double PI = 3.14159265358979323846;

int nvars(int pde, int d) { return pde == PDE_EULER ? d + 2 : 9; }

// Physical flux in direction m (0..d-1) for state q, Eq. (eulerTerms) or
// Eq. (MHDTerms).  f has nvars entries.
void flux(int pde, int d, const Params& P, const double* q, int m, double* f) {
  if (pde == PDE_EULER) {
    double rho = q[0];
    double v[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) v[k] = q[1 + k] / rho;
    double rhoE = q[d + 1];
    double v2 = 0.0;
    for (int k = 0; k < d; ++k) v2 += v[k] * v[k];
    double p = (P.gamma - 1.0) * (rhoE - 0.5 * rho * v2);  // Eq. (eos)
    f[0] = rho * v[m];
    for (int k = 0; k < d; ++k) f[1 + k] = rho * v[k] * v[m] + (k == m ? p : 0.0);
    f[d + 1] = v[m] * (rhoE + p);
    return;
  }
  // MHD-GLM: (rho, rho v(3), rho E, B(3), psi), Gaussian units
  double rho = q[0];
  double v[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
  double rhoE = q[4];
  double B[3] = {q[5], q[6], q[7]};
  double psi = q[8];
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  double p = (P.gamma - 1.0) * (rhoE - 0.5 * rho * v2 - B2 / (8.0 * PI));  // Eq. (MHDeos)
  double pm = B2 / (8.0 * PI);
  double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  f[0] = rho * v[m];
  for (int k = 0; k < 3; ++k) f[1 + k] = rho * v[k] * v[m] + (k == m ? p + pm : 0.0) - B[k] * B[m] / (4.0 * PI);
  f[4] = v[m] * (rhoE + p + pm) - B[m] * vB / (4.0 * PI);
  for (int k = 0; k < 3; ++k) f[5 + k] = v[m] * B[k] - B[m] * v[k] + (k == m ? psi : 0.0);
  f[8] = P.ch * P.ch * B[m];
}

// Largest |eigenvalue| of the flux Jacobian in unit direction n.
double max_speed_normal(int pde, int d, const Params& P, const double* q, const double* n) {
  if (pde == PDE_EULER) {
    double rho = q[0];
    double vn = 0.0, v2 = 0.0;
    for (int k = 0; k < d; ++k) {
      double vk = q[1 + k] / rho;
      vn += vk * n[k];
      v2 += vk * vk;
    }
    double p = (P.gamma - 1.0) * (q[d + 1] - 0.5 * rho * v2);
    double c = std::sqrt(std::max(0.0, P.gamma * p / rho));
    return std::fabs(vn) + c;
  }
  double rho = q[0];
  double v[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
  double B[3] = {q[5], q[6], q[7]};
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  double p = (P.gamma - 1.0) * (q[4] - 0.5 * rho * v2 - B2 / (8.0 * PI));
  double vn = 0.0, Bn = 0.0;
  for (int k = 0; k < d; ++k) {
    vn += v[k] * n[k];
    Bn += B[k] * n[k];
  }
  double a2 = P.gamma * p / rho;
  double b2 = B2 / (4.0 * PI * rho);
  double bn2 = Bn * Bn / (4.0 * PI * rho);
  double cf2 = 0.5 * (a2 + b2 + std::sqrt(std::max(0.0, (a2 + b2) * (a2 + b2) - 4.0 * a2 * bn2)));
  return std::max(std::fabs(vn) + std::sqrt(std::max(0.0, cf2)), P.ch);
}

// |A_n(q)| = R |Lambda| R^{-1} for the Euler normal flux Jacobian
// dF/dq . n at state q (unit normal n): R holds the right eigenvectors
// (columns) for the eigenvalues vn - c, vn (entropy), vn (shear, d-1
// tangents), vn + c; R^{-1} is formed numerically.  Out: nu x nu row-major.
void euler_abs_jacobian(int d, double gamma, const double* q, const double* n, double* out) {
  const int nu = d + 2;
  double rho = q[0], v[3] = {0, 0, 0}, v2 = 0.0, vn = 0.0;
  for (int k = 0; k < d; ++k) {
    v[k] = q[1 + k] / rho;
    v2 += v[k] * v[k];
    vn += v[k] * n[k];
  }
  double p = (gamma - 1.0) * (q[d + 1] - 0.5 * rho * v2);
  double c = std::sqrt(gamma * p / rho);
  double H = (q[d + 1] + p) / rho;
  // tangents: 2D (-n_y, n_x); 3D two unit vectors orthogonal to n
  double t[2][3] = {{0, 0, 0}, {0, 0, 0}};
  if (d == 2) {
    t[0][0] = -n[1];
    t[0][1] = n[0];
  } else {
    int a = 0;
    for (int k = 1; k < 3; ++k)
      if (std::fabs(n[k]) < std::fabs(n[a])) a = k;
    double e[3] = {0, 0, 0};
    e[a] = 1.0;
    double t0[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
    double l0 = std::sqrt(t0[0] * t0[0] + t0[1] * t0[1] + t0[2] * t0[2]);
    for (int k = 0; k < 3; ++k) t[0][k] = t0[k] / l0;
    double t1[3] = {n[1] * t[0][2] - n[2] * t[0][1], n[2] * t[0][0] - n[0] * t[0][2], n[0] * t[0][1] - n[1] * t[0][0]};
    for (int k = 0; k < 3; ++k) t[1][k] = t1[k];
  }
  std::vector<double> R((size_t)nu * nu, 0.0), lam(nu);
  auto col = [&](int j, const std::vector<double>& r) {
    for (int i = 0; i < nu; ++i) R[i * nu + j] = r[i];
  };
  std::vector<double> r(nu);
  r[0] = 1.0;
  for (int k = 0; k < d; ++k) r[1 + k] = v[k] - c * n[k];
  r[d + 1] = H - c * vn;
  col(0, r);
  lam[0] = vn - c;
  r[0] = 1.0;
  for (int k = 0; k < d; ++k) r[1 + k] = v[k];
  r[d + 1] = 0.5 * v2;
  col(1, r);
  lam[1] = vn;
  for (int a = 0; a < d - 1; ++a) {
    r[0] = 0.0;
    double vt = 0.0;
    for (int k = 0; k < d; ++k) {
      r[1 + k] = t[a][k];
      vt += v[k] * t[a][k];
    }
    r[d + 1] = vt;
    col(2 + a, r);
    lam[2 + a] = vn;
  }
  r[0] = 1.0;
  for (int k = 0; k < d; ++k) r[1 + k] = v[k] + c * n[k];
  r[d + 1] = H + c * vn;
  col(nu - 1, r);
  lam[nu - 1] = vn + c;
  // R^{-1} by elimination on the identity
  std::vector<double> Rinv((size_t)nu * nu, 0.0);
  for (int i = 0; i < nu; ++i) Rinv[i * nu + i] = 1.0;
  gauss_solve(nu, R, Rinv, nu);
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nu; ++j) {
      double sum = 0.0;
      for (int k = 0; k < nu; ++k) sum += R[i * nu + k] * std::fabs(lam[k]) * Rinv[k * nu + j];
      out[i * nu + j] = sum;
    }
}

// Numerical normal flux at a face point (unit normal n): Rusanov, Eq.
// (rusanov), or Osher-type, Eq. (osher), whose dissipation integrates
// |A_n| along the straight path psi(s) = q- + s (q+ - q-) with 3-point
// Gauss-Legendre (the paper leaves the rule open).
void numerical_flux(int pde, int d, const Params& P, const double* qm, const double* qp, const double* n,
                    double* G) {
  const int nu = nvars(pde, d);
  std::vector<double> fm(nu, 0.0), fp(nu, 0.0), fd(nu);
  for (int mm = 0; mm < d; ++mm) {
    flux(pde, d, P, qm, mm, fd.data());
    for (int v = 0; v < nu; ++v) fm[v] += fd[v] * n[mm];
    flux(pde, d, P, qp, mm, fd.data());
    for (int v = 0; v < nu; ++v) fp[v] += fd[v] * n[mm];
  }
  if (P.flux == 1 && pde == PDE_EULER) {
    std::vector<double> sx, sw;
    gauss_legendre01(3, sx, sw);
    std::vector<double> absA((size_t)nu * nu), psi(nu), dis(nu, 0.0);
    for (int j = 0; j < 3; ++j) {
      for (int v = 0; v < nu; ++v) psi[v] = qm[v] + sx[j] * (qp[v] - qm[v]);
      euler_abs_jacobian(d, P.gamma, psi.data(), n, absA.data());
      for (int a = 0; a < nu; ++a)
        for (int b = 0; b < nu; ++b) dis[a] += sw[j] * absA[a * nu + b] * (qp[b] - qm[b]);
    }
    for (int v = 0; v < nu; ++v) G[v] = 0.5 * (fm[v] + fp[v]) - 0.5 * dis[v];
    return;
  }
  double smax = std::max(max_speed_normal(pde, d, P, qm, n), max_speed_normal(pde, d, P, qp, n));
  for (int v = 0; v < nu; ++v) G[v] = 0.5 * (fm[v] + fp[v]) - 0.5 * smax * (qp[v] - qm[v]);
}

// Largest |eigenvalue| over all directions (for the time step).
double max_speed(int pde, int d, const Params& P, const double* q) {
  double rho = q[0];
  if (pde == PDE_EULER) {
    double v2 = 0.0;
    for (int k = 0; k < d; ++k) v2 += (q[1 + k] / rho) * (q[1 + k] / rho);
    double p = (P.gamma - 1.0) * (q[d + 1] - 0.5 * rho * v2);
    return std::sqrt(v2) + std::sqrt(std::max(0.0, P.gamma * p / rho));
  }
  double v[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
  double B[3] = {q[5], q[6], q[7]};
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  double p = (P.gamma - 1.0) * (q[4] - 0.5 * rho * v2 - B2 / (8.0 * PI));
  double a2 = P.gamma * p / rho;
  double b2 = B2 / (4.0 * PI * rho);
  return std::max(std::sqrt(v2) + std::sqrt(std::max(0.0, a2 + b2)), P.ch);
}

// Pressure from the conserved state, Eq. (eos) / Eq. (MHDeos).
double pressure(int pde, int d, const Params& P, const double* q) {
  double rho = q[0];
  if (pde == PDE_EULER) {
    double m2 = 0.0;
    for (int k = 0; k < d; ++k) m2 += q[1 + k] * q[1 + k];
    return (P.gamma - 1.0) * (q[d + 1] - 0.5 * m2 / rho);
  }
  double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
  return (P.gamma - 1.0) * (q[4] - 0.5 * m2 / rho - B2 / (8.0 * PI));
}

// --------------------------------------------------------------------- mesh
struct OMesh {
  int d = 2;
  long nv = 0, nc = 0;
  std::vector<double> xyz;
  std::vector<long> cells;
  bool per[3] = {false, false, false};
  double L[3] = {0, 0, 0};
  std::vector<double> X;     // nc x (d+1) x 3 unwrapped vertex coordinates
  std::vector<double> vol;   // |T_i|
  std::vector<double> bary;  // nc x 3
  std::vector<long> nbr;     // nc x (d+1): neighbour across face k (opposite vertex k)
  double qscale = 1.0;       // length scale for ranking tolerances
};

double vx(const OMesh& m, long c, int k, int a) { return m.X[((size_t)c * (m.d + 1) + k) * 3 + a]; }

// Shift to add to cell j's coordinates to bring it next to cell i
// (minimum image of the barycentre difference).
void min_image_shift(const OMesh& m, long i, long j, double* s) {
  for (int a = 0; a < 3; ++a) {
    s[a] = 0.0;
    if (a < m.d && m.per[a]) {
      double diff = m.bary[i * 3 + a] - m.bary[j * 3 + a];
      s[a] = m.L[a] * std::nearbyint(diff / m.L[a]);
    }
  }
}

// Jacobian J[a][k] = X_{k+1,a} - X_{0,a} of the map (xietaTransf) of cell c.
void cell_jacobian(const OMesh& m, long c, double J[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) J[a][k] = 0.0;
  for (int a = 0; a < m.d; ++a)
    for (int k = 0; k < m.d; ++k) J[a][k] = vx(m, c, k + 1, a) - vx(m, c, 0, a);
}

// Reference coordinates in cell c of a physical point x (already in c's frame).
void to_ref(const OMesh& m, long c, const double* x, double* xi) {
  double J[3][3], Ji[3][3];
  cell_jacobian(m, c, J);
  inv3(J, m.d, Ji);
  for (int a = 0; a < 3; ++a) xi[a] = 0.0;
  for (int a = 0; a < m.d; ++a)
    for (int b = 0; b < m.d; ++b) xi[a] += Ji[a][b] * (x[b] - vx(m, c, 0, b));
}

// Geometry of every cell from the vertex coordinates m.xyz: unwrapped vertex
// coordinates (periodic images nearest the cell's first vertex), |T_i| and the
// barycentre.  Called at construction and again after every mesh motion.
bool mesh_geometry(OMesh& m, std::string& err) {
  int d = m.d;
  m.X.assign((size_t)m.nc * (d + 1) * 3, 0.0);
  m.vol.assign(m.nc, 0.0);
  m.bary.assign((size_t)m.nc * 3, 0.0);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (long v = 0; v < m.nv; ++v)
    for (int a = 0; a < d; ++a) {
      lo[a] = std::min(lo[a], m.xyz[v * d + a]);
      hi[a] = std::max(hi[a], m.xyz[v * d + a]);
    }
  m.qscale = 0.0;
  for (int a = 0; a < d; ++a) m.qscale = std::max(m.qscale, hi[a] - lo[a]);
  for (long c = 0; c < m.nc; ++c) {
    for (int k = 0; k <= d; ++k) {
      long v = m.cells[c * (d + 1) + k];
      if (v < 0 || v >= m.nv) {
        err = "vertex index out of range";
        return false;
      }
      for (int a = 0; a < d; ++a) {
        double x = m.xyz[v * d + a];
        if (m.per[a] && k > 0) {
          double x0 = m.xyz[m.cells[c * (d + 1)] * d + a];
          x += m.L[a] * std::nearbyint((x0 - x) / m.L[a]);
        }
        m.X[((size_t)c * (d + 1) + k) * 3 + a] = x;
      }
    }
    double J[3][3];
    cell_jacobian(m, c, J);
    double det = det3(J, d);
    m.vol[c] = det / factorial(d);
    if (!(m.vol[c] > 0.0)) {
      err = "cell with non-positive volume";
      return false;
    }
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int k = 0; k <= d; ++k) s += vx(m, c, k, a);
      m.bary[c * 3 + a] = s / (d + 1);
    }
  }
  return true;
}

bool build_mesh(OMesh& m, std::string& err) {
  int d = m.d;
  if (!mesh_geometry(m, err)) return false;
  // face matching by sorted global vertex ids
  struct FaceKey {
    long v[3];
    long cell;
    int face;
  };
  std::vector<FaceKey> keys;
  keys.reserve((size_t)m.nc * (d + 1));
  for (long c = 0; c < m.nc; ++c)
    for (int k = 0; k <= d; ++k) {
      FaceKey f;
      int n = 0;
      for (int q = 0; q <= d; ++q)
        if (q != k) f.v[n++] = m.cells[c * (d + 1) + q];
      if (d == 2) f.v[2] = -1;
      std::sort(f.v, f.v + d);
      f.cell = c;
      f.face = k;
      keys.push_back(f);
    }
  std::sort(keys.begin(), keys.end(), [](const FaceKey& a, const FaceKey& b) {
    for (int q = 0; q < 3; ++q)
      if (a.v[q] != b.v[q]) return a.v[q] < b.v[q];
    return a.cell < b.cell;
  });
  m.nbr.assign((size_t)m.nc * (d + 1), -1);
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j].v[0] == keys[i].v[0] && keys[j].v[1] == keys[i].v[1] &&
           keys[j].v[2] == keys[i].v[2])
      ++j;
    if (j - i > 2) {
      err = "face shared by more than two cells";
      return false;
    }
    if (j - i == 2) {
      m.nbr[keys[i].cell * (d + 1) + keys[i].face] = keys[i + 1].cell;
      m.nbr[keys[i + 1].cell * (d + 1) + keys[i + 1].face] = keys[i].cell;
    }
    i = j;
  }
  return true;
}

// Characteristic size h_i: incircle (2D) / insphere (3D) diameter, Eq. (timestep).
double cell_h(const OMesh& m, long c) {
  int d = m.d;
  double surf = 0.0;
  for (int k = 0; k <= d; ++k) {
    double P[3][3];
    int n = 0;
    for (int q = 0; q <= d; ++q)
      if (q != k) {
        for (int a = 0; a < 3; ++a) P[n][a] = vx(m, c, q, a);
        ++n;
      }
    if (d == 2) {
      surf += std::hypot(P[1][0] - P[0][0], P[1][1] - P[0][1]);
    } else {
      double u[3], w[3];
      for (int a = 0; a < 3; ++a) {
        u[a] = P[1][a] - P[0][a];
        w[a] = P[2][a] - P[0][a];
      }
      double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
      surf += 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }
  }
  return 2.0 * d * m.vol[c] / surf;
}

// ------------------------------------------------------------------ solver
struct Stencil {
  std::vector<long> S0;                  // n_e cells, S0[0] = i
  std::vector<std::vector<long>> sector;  // d+1 sectors, each d cells or empty (dropped)
};

struct CellRec {
  bool ready = false;
  Stencil st;
  // reduced LSQ matrix (rows j in S0\{i}, columns monomials e != 0): a_j[e] - a_i[e]
  std::vector<double> Ared;
  std::vector<double> ai;  // constraint row avg_{T_E} xi^e
  // sectors: d x d matrix rows (xi(b_j) - xi_bary) for the chosen cells
  std::vector<std::vector<double>> Bsec;
};

struct OSolver {
  OMesh* mesh = nullptr;
  int M = 2, pde = 0, nu = 4, d = 2;
  Params P;
  int Mc = 0, ne = 0, Lc = 0, L0 = 0;
  std::vector<std::array<int, 4>> mono;  // spatial monomials of P_M
  // predictor
  std::vector<std::array<double, 4>> st_nodes;  // space-time nodes (xi..., tau in slot 3)
  std::vector<std::array<int, 5>> alpha;        // lattice indices of the space-time nodes
  std::vector<double> Pint;                     // d x (L-L0) x L: int_0^tau_k d theta_l / d xi_e
  std::vector<Poly> theta;                      // nodal basis as polynomials (Galerkin form)
  std::vector<double> Ktau, Mmat;               // rows: unknown nodes (L-L0) x L columns
  std::vector<std::array<double, 4>> lat;       // spatial lattice (M), same as tau=0 nodes
  std::map<long, CellRec> cache;
};

// Spatial principal lattice of degree K on T_E with step 1/M.  Enumeration:
// outer loop over zeta index, then eta index, then xi index.
std::vector<std::array<double, 4>> spatial_lattice(int d, int K, int M) {
  std::vector<std::array<double, 4>> out;
  if (d == 2) {
    for (int j = 0; j <= K; ++j)
      for (int i = 0; i <= K - j; ++i) out.push_back({(double)i / M, (double)j / M, 0.0, 0.0});
  } else {
    for (int k = 0; k <= K; ++k)
      for (int j = 0; j <= K - k; ++j)
        for (int i = 0; i <= K - j - k; ++i) out.push_back({(double)i / M, (double)j / M, (double)k / M, 0.0});
  }
  if (K == 0 && M == 0) out.assign(1, {0, 0, 0, 0});
  return out;
}

// Ranked, layer-by-layer breadth-first sequence of face neighbours of cell i
// (cell i itself excluded), continued `extra` layers beyond the layer in which
// `need` cells (i included) are first reached.
std::vector<long> ranked_bfs(const OMesh& m, long i, int need, int extra, std::string& err) {
  int d = m.d;
  std::vector<long> seq;
  std::vector<long> frontier(1, i);
  std::map<long, bool> seen;
  seen[i] = true;
  int complete_layer = -1;
  for (int layer = 1;; ++layer) {
    std::vector<long> next;
    for (long c : frontier)
      for (int k = 0; k <= d; ++k) {
        long j = m.nbr[c * (d + 1) + k];
        if (j < 0 || seen.count(j)) continue;
        seen[j] = true;
        next.push_back(j);
      }
    if (next.empty()) break;
    // rank: quantised squared distance of the minimum-image barycentre, then
    // its coordinates (x, y, z), then the cell index
    struct Key {
      long long q[4];
      long cell;
    };
    std::vector<Key> keys;
    double tol = 1e-9 * m.qscale;
    for (long j : next) {
      double s[3];
      min_image_shift(m, i, j, s);
      double b[3], d2 = 0.0;
      for (int a = 0; a < 3; ++a) b[a] = 0.0;
      for (int a = 0; a < d; ++a) {
        b[a] = m.bary[j * 3 + a] + s[a];
        double diff = b[a] - m.bary[i * 3 + a];
        d2 += diff * diff;
      }
      Key key;
      key.q[0] = std::llround(d2 / (tol * m.qscale));
      for (int a = 0; a < 3; ++a) key.q[1 + a] = std::llround(b[a] / tol);
      key.cell = j;
      keys.push_back(key);
    }
    std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
      for (int q = 0; q < 4; ++q)
        if (a.q[q] != b.q[q]) return a.q[q] < b.q[q];
      return a.cell < b.cell;
    });
    for (const Key& k : keys) seq.push_back(k.cell);
    if (complete_layer < 0 && (long)seq.size() + 1 >= need) complete_layer = layer;
    if (complete_layer >= 0 && layer >= complete_layer + extra) break;
    frontier = next;
  }
  if ((long)seq.size() + 1 < need) err = "mesh too small for the central stencil";
  return seq;
}

// Reference coordinates (in cell i) of the minimum-image barycentre of cell j.
void bary_in_ref(const OMesh& m, long i, long j, double* xi) {
  double s[3];
  min_image_shift(m, i, j, s);
  double b[3] = {0, 0, 0};
  for (int a = 0; a < m.d; ++a) b[a] = m.bary[j * 3 + a] + s[a];
  to_ref(m, i, b, xi);
}

void cell_matrices(OSolver& S, long i, CellRec& R);

bool prepare_cell(OSolver& S, long i, std::string& err) {
  CellRec& R = S.cache[i];
  if (R.ready) return true;
  const OMesh& m = *S.mesh;
  int d = m.d;
  // --- stencils, Eq. (stencil) and the sector rule
  std::vector<long> seq = ranked_bfs(m, i, S.ne, 2, err);
  if (!err.empty()) return false;
  R.st.S0.assign(1, i);
  for (int k = 0; k < S.ne - 1; ++k) R.st.S0.push_back(seq[k]);
  R.st.sector.assign(d + 1, std::vector<long>());
  R.Bsec.assign(d + 1, std::vector<double>());
  double xb = 1.0 / (d + 1);
  for (int s = 0; s <= d; ++s) {
    std::vector<long> chosen;
    for (long j : seq) {
      double xi[3];
      bary_in_ref(m, i, j, xi);
      double lam[4];
      lam[0] = 1.0;
      for (int a = 0; a < d; ++a) {
        lam[a + 1] = xi[a];
        lam[0] -= xi[a];
      }
      bool inside = true;
      for (int q = 0; q <= d; ++q)
        if (q != s && !(lam[q] > 1e-9)) inside = false;
      if (inside) chosen.push_back(j);
      if ((int)chosen.size() == d) break;
    }
    if ((int)chosen.size() < d) continue;  // dropped sector
    std::vector<double> B((size_t)d * d);
    for (int k = 0; k < d; ++k) {
      double xi[3];
      bary_in_ref(m, i, chosen[k], xi);
      for (int a = 0; a < d; ++a) B[k * d + a] = xi[a] - xb;
    }
    double Bm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < d; ++k)
      for (int a = 0; a < d; ++a) Bm[k][a] = B[k * d + a];
    if (std::fabs(det3(Bm, d)) < 1e-8) continue;  // degenerate sector: dropped
    R.st.sector[s] = chosen;
  }
  cell_matrices(S, i, R);
  R.ready = true;
  return true;
}

// Geometry-dependent data of cell i for its (fixed) stencils, from the current
// vertex positions: the sector rows xi(b_j) - xi_bary of Eq. (CWENO:Ps) and
// the least-squares rows of Eq. (CWENO:Popt).  On a moving mesh the stencils
// stay those chosen on the initial mesh (the topology never changes) and
// only these matrices are rebuilt every step (Sec. 2.1).
void cell_matrices(OSolver& S, long i, CellRec& R) {
  const OMesh& m = *S.mesh;
  int d = m.d;
  double xb = 1.0 / (d + 1);
  R.Bsec.assign(d + 1, std::vector<double>());
  for (int s = 0; s <= d; ++s) {
    if (R.st.sector[s].empty()) continue;
    std::vector<double> B((size_t)d * d);
    for (int k = 0; k < d; ++k) {
      double xi[3];
      bary_in_ref(m, i, R.st.sector[s][k], xi);
      for (int a = 0; a < d; ++a) B[k * d + a] = xi[a] - xb;
    }
    R.Bsec[s] = B;
  }
  // --- least-squares rows, Eq. (CWENO:Popt): averages of the monomials over
  // each stencil cell, in the reference frame of cell i
  int nmono = S.Mc;
  R.ai.assign(nmono, 0.0);
  for (int e = 0; e < nmono; ++e) {
    int ex[4] = {S.mono[e][0], S.mono[e][1], S.mono[e][2], 0};
    R.ai[e] = simplex_integral(d, ex) * factorial(d);  // average over T_E (|T_E| = 1/d!)
  }
  int nrow = S.ne - 1;
  R.Ared.assign((size_t)nrow * (nmono - 1), 0.0);
  for (int r = 0; r < nrow; ++r) {
    long j = R.st.S0[r + 1];
    double s[3];
    min_image_shift(m, i, j, s);
    // vertices of T_j (shifted) in the reference coordinates of T_i
    double V[4][3];
    for (int k = 0; k <= d; ++k) {
      double x[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) x[a] = vx(m, j, k, a) + s[a];
      to_ref(m, i, x, V[k]);
    }
    double A[3] = {0, 0, 0}, B[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < d; ++a) {
      A[a] = V[0][a];
      for (int q = 0; q < d; ++q) B[a][q] = V[q + 1][a] - V[0][a];
    }
    for (int e = 1; e < nmono; ++e) {
      Poly p;
      p.push_back(monomial(S.mono[e][0], S.mono[e][1], S.mono[e][2], 0, 1.0));
      Poly pc = poly_compose_affine(p, d, A, B);
      double avg = integrate_simplex(pc, d) * factorial(d);
      R.Ared[(size_t)r * (nmono - 1) + (e - 1)] = avg - R.ai[e];
    }
  }
}

// Polynomial in the spatial monomials from coefficients (index = mono order).
Poly poly_from_coef(const OSolver& S, const double* c) {
  Poly p;
  for (int e = 0; e < S.Mc; ++e) p.push_back(monomial(S.mono[e][0], S.mono[e][1], S.mono[e][2], 0, c[e]));
  return normalise(p);
}

// Oscillation indicator: sum over multi-indices 1 <= |alpha| <= M of the
// integral over T_E of (d^alpha p)^2.
double sigma_of(const OSolver& S, const Poly& p) {
  int d = S.d;
  double s = 0.0;
  std::vector<std::array<int, 4>> alphas = monomial_list(d, S.M);
  for (const auto& a : alphas) {
    int tot = a[0] + a[1] + a[2];
    if (tot < 1) continue;
    Poly q = p;
    for (int k = 0; k < d; ++k)
      for (int r = 0; r < a[k]; ++r) q = poly_deriv(q, k);
    s += integrate_simplex(poly_mul(q, q), d);
  }
  return s;
}

struct RecOut {
  std::vector<Poly> w;              // per variable
  std::vector<Poly> popt;           // per variable
  std::vector<double> omega;        // (d+2) x nu, dropped sectors get 0
  std::vector<double> sigma;        // (d+2) x nu
};

bool reconstruct_cell(OSolver& S, const double* Q, long i, RecOut& out, std::string& err) {
  if (!prepare_cell(S, i, err)) return false;
  const CellRec& R = S.cache[i];
  int d = S.d, nu = S.nu, nm = S.Mc;
  int nrow = S.ne - 1;
  out.w.assign(nu, Poly());
  out.popt.assign(nu, Poly());
  out.omega.assign((size_t)(d + 2) * nu, 0.0);
  out.sigma.assign((size_t)(d + 2) * nu, 0.0);
  // --- P_opt, Eq. (CWENO:Popt): the constraint fixes the constant coefficient,
  // the remaining ones solve the reduced least-squares problem
  std::vector<double> rhs((size_t)nrow * nu);
  for (int r = 0; r < nrow; ++r)
    for (int v = 0; v < nu; ++v) rhs[r * nu + v] = Q[R.st.S0[r + 1] * nu + v] - Q[i * nu + v];
  std::vector<double> X;
  if (!householder_lsq(nrow, nm - 1, R.Ared, rhs, nu, X)) {
    err = "rank-deficient least-squares system";
    return false;
  }
  std::vector<Poly> Popt(nu);
  for (int v = 0; v < nu; ++v) {
    std::vector<double> c(nm, 0.0);
    double c0 = Q[i * nu + v];
    for (int e = 1; e < nm; ++e) {
      c[e] = X[(e - 1) * nu + v];
      c0 -= R.ai[e] * c[e];
    }
    c[0] = c0;
    Popt[v] = poly_from_coef(S, c.data());
  }
  out.popt = Popt;
  // --- sectorial polynomials, Eq. (CWENO:Ps): P_s(xi) = Q_i + g.(xi - xi_b)
  double xb = 1.0 / (d + 1);
  std::vector<std::vector<Poly>> Ps(d + 1, std::vector<Poly>(nu));
  std::vector<bool> kept(d + 1, false);
  int Ns = 0;
  for (int s = 0; s <= d; ++s) {
    if (R.st.sector[s].empty()) continue;
    kept[s] = true;
    ++Ns;
    std::vector<double> g((size_t)d * nu);
    for (int k = 0; k < d; ++k)
      for (int v = 0; v < nu; ++v) g[k * nu + v] = Q[R.st.sector[s][k] * nu + v] - Q[i * nu + v];
    if (!gauss_solve(d, R.Bsec[s], g, nu)) {
      err = "singular sector system";
      return false;
    }
    for (int v = 0; v < nu; ++v) {
      Poly p;
      double c0 = Q[i * nu + v];
      for (int a = 0; a < d; ++a) {
        int e[3] = {0, 0, 0};
        e[a] = 1;
        p.push_back(monomial(e[0], e[1], e[2], 0, g[a * nu + v]));
        c0 -= g[a * nu + v] * xb;
      }
      p.push_back(monomial(0, 0, 0, 0, c0));
      Ps[s][v] = normalise(p);
    }
  }
  // --- linear weights (normalised), Eq. (CWENO:P0)
  double lam0 = S.P.lam0 / (S.P.lam0 + Ns * S.P.lams);
  double lams = S.P.lams / (S.P.lam0 + Ns * S.P.lams);
  for (int v = 0; v < nu; ++v) {
    Poly P0 = Popt[v];
    for (int s = 0; s <= d; ++s)
      if (kept[s]) P0 = poly_axpy(1.0, P0, -lams, Ps[s][v]);
    P0 = poly_axpy(1.0 / lam0, P0, 0.0, Poly());
    // --- indicators and nonlinear weights, Eqs. (weights), (weights2)
    std::vector<double> wt(d + 2, 0.0), sig(d + 2, 0.0);
    sig[0] = sigma_of(S, P0);
    wt[0] = lam0 / std::pow(sig[0] + S.P.eps, S.P.r);
    for (int s = 0; s <= d; ++s) {
      if (!kept[s]) continue;
      sig[s + 1] = sigma_of(S, Ps[s][v]);
      wt[s + 1] = lams / std::pow(sig[s + 1] + S.P.eps, S.P.r);
    }
    if (S.P.linear_weights) {
      wt[0] = lam0;
      for (int s = 0; s <= d; ++s) wt[s + 1] = kept[s] ? lams : 0.0;
    }
    double tot = 0.0;
    for (double x : wt) tot += x;
    for (double& x : wt) x /= tot;
    // --- reconstruction polynomial, Eq. (CWENO:Prec)
    Poly w = poly_axpy(wt[0], P0, 0.0, Poly());
    for (int s = 0; s <= d; ++s)
      if (kept[s]) w = poly_axpy(1.0, w, wt[s + 1], Ps[s][v]);
    out.w[v] = w;
    for (int s = 0; s < d + 2; ++s) {
      out.omega[s * nu + v] = wt[s];
      out.sigma[s * nu + v] = sig[s];
    }
  }
  if (S.P.positivity) {
    // Positivity scaling (addition, see the header): w <- Qbar + theta (w - Qbar)
    // with theta the largest value in [0,1] keeping density, then pressure,
    // above 1e-3 times their cell-average values at every lattice node (a
    // floor above single-precision rounding, so both precisions of the
    // product take the same decisions).  Density and pressure are concave in
    // the conserved variables, so the linear interpolation bound below is
    // sufficient; a node whose scaled density is not positive gives theta 0.
    const double floor_rel = 1e-3;
    const double* qb = &Q[i * nu];
    double rb = qb[0], pb = pressure(S.pde, d, S.P, qb);
    std::vector<std::vector<double>> node(S.Mc, std::vector<double>(nu));
    for (int n = 0; n < S.Mc; ++n) {
      double x[4] = {S.lat[n][0], S.lat[n][1], S.lat[n][2], 0.0};
      for (int v = 0; v < nu; ++v) node[n][v] = poly_eval(out.w[v], x);
    }
    double th_rho = 1.0;
    for (int n = 0; n < S.Mc; ++n)
      if (node[n][0] < floor_rel * rb) th_rho = std::min(th_rho, (rb - floor_rel * rb) / (rb - node[n][0]));
    double th_p = 1.0;
    if (pb > 0.0)
      for (int n = 0; n < S.Mc; ++n) {
        std::vector<double> q(nu);
        for (int v = 0; v < nu; ++v) q[v] = qb[v] + th_rho * (node[n][v] - qb[v]);
        if (!(q[0] > 0.0)) {
          th_p = 0.0;
          continue;
        }
        double pk = pressure(S.pde, d, S.P, q.data());
        if (pk < floor_rel * pb) th_p = std::min(th_p, (pb - floor_rel * pb) / (pb - pk));
      }
    double theta = th_rho * th_p;
    if (theta < 1.0)
      for (int v = 0; v < nu; ++v) {
        Poly c;
        c.push_back(monomial(0, 0, 0, 0, qb[v]));
        out.w[v] = poly_axpy(theta, out.w[v], 1.0 - theta, c);
      }
  }
  return true;
}

// --------------------------------------------------------------- predictor
// Nodal basis of the space-time nodes, evaluated in closed form.  The nodes
// are the principal lattice of the (d+1)-simplex with barycentric
// coordinates lambda_0 = 1 - sum(xi) - tau, lambda_{1..d} = xi, lambda_{d+1}
// = tau; node l has lattice indices alpha_l (summing to M), and its Lagrange
// polynomial is the product over c and j < alpha_c of (M lambda_c - j)/(j+1):
// one at node l, zero at every other node of the lattice.  x holds
// (xi_0, xi_1, xi_2, tau) with tau in slot 3.  th[l]; dth (optional) holds
// d theta_l / d xi_e at dth[e * L + l] for e < d and d/d tau at e = d.
void st_basis(const OSolver& S, const double* x, double* th, double* dth) {
  const int d = S.d, M = S.M, L = S.Lc;
  double lam[5];
  lam[0] = 1.0 - x[3];
  for (int a = 0; a < d; ++a) {
    lam[1 + a] = x[a];
    lam[0] -= x[a];
  }
  lam[d + 1] = x[3];
  for (int l = 0; l < L; ++l) {
    // the M linear factors of theta_l and their barycentric variable
    double f[8];
    int var[8], jj[8], nf = 0;
    for (int c = 0; c <= d + 1; ++c)
      for (int j = 0; j < S.alpha[l][c]; ++j) {
        f[nf] = (M * lam[c] - j) / (j + 1);
        var[nf] = c;
        jj[nf] = j;
        ++nf;
      }
    double v = 1.0;
    for (int q = 0; q < nf; ++q) v *= f[q];
    th[l] = v;
    if (!dth) continue;
    // product rule; d lambda_0 / d x_a = -1, d lambda_{1+a} / d xi_a = 1,
    // d lambda_{d+1} / d tau = 1
    for (int e = 0; e <= d; ++e) {
      double g = 0.0;
      for (int q = 0; q < nf; ++q) {
        double dl = var[q] == 0 ? -1.0 : (var[q] == e + 1 ? 1.0 : 0.0);
        if (dl == 0.0) continue;
        // factor q is (M lambda - j)/(j+1): its derivative is M/(j+1) dlambda
        double t = dl * M / (jj[q] + 1);
        for (int r = 0; r < nf; ++r)
          if (r != q) t *= f[r];
        g += t;
      }
      dth[e * L + l] = g;
    }
  }
}

// Space-time predictor in closed form.  With the nodal flux interpolant
// F_h in P_M (Eq. PDEterm), q_h(xi, tau) = w(xi) - dt int_0^tau H_h(xi, s) ds
// is a polynomial of degree M that satisfies d q_h / d tau + dt H_h = 0
// pointwise and takes the known values at tau = 0, so it makes the residual
// of Eq. (CGfinal) vanish for every test function: it is the Galerkin
// solution (K_tau^1 is invertible, reading c6).  Its value at the unknown
// node k is w(xi_k) - dt sum_e sum_l Pint[e][k][l] G_e,l with
//   Pint[e][k][l] = int_0^{tau_k} d theta_l / d xi_e (xi_k, s) ds,
// integrated by Gauss-Legendre (exact: the integrand has degree M-1 in s).
// This avoids forming (K_tau^1)^-1, whose condition number reaches 1.4e6 at
// M = 4; the Galerkin form is kept for comparison (predictor_cell_galerkin).
void init_predictor_integrals(OSolver& S) {
  const int d = S.d, M = S.M, L = S.Lc, L0 = S.L0, L1 = L - L0;
  std::vector<double> gx, gw;
  gauss_legendre01(M + 1, gx, gw);
  S.Pint.assign((size_t)d * L1 * L, 0.0);
  std::vector<double> th(L), dth((size_t)(d + 1) * L);
  for (int k = 0; k < L1; ++k) {
    const std::array<double, 4>& nk = S.st_nodes[L0 + k];
    for (size_t q = 0; q < gx.size(); ++q) {
      double x[4] = {nk[0], nk[1], nk[2], nk[3] * gx[q]};
      st_basis(S, x, th.data(), dth.data());
      for (int e = 0; e < d; ++e)
        for (int l = 0; l < L; ++l) S.Pint[((size_t)e * L1 + k) * L + l] += nk[3] * gw[q] * dth[e * L + l];
    }
  }
}

void init_predictor(OSolver& S) {
  int d = S.d, M = S.M;
  // space-time nodes: time level t (tau = t/M) carries the spatial lattice of
  // degree M - t with step 1/M, i.e. the principal lattice of the (d+1)-simplex
  S.st_nodes.clear();
  for (int t = 0; t <= M; ++t) {
    std::vector<std::array<double, 4>> sl = spatial_lattice(d, M - t, M);
    for (auto x : sl) {
      x[3] = (double)t / M;
      S.st_nodes.push_back(x);
    }
  }
  S.Lc = (int)S.st_nodes.size();
  S.L0 = S.Mc;
  S.lat = spatial_lattice(d, M, M);
  S.alpha.clear();
  for (const auto& nd : S.st_nodes) {
    std::array<int, 5> al = {0, 0, 0, 0, 0};
    int sum = 0;
    for (int a = 0; a < d; ++a) {
      al[1 + a] = (int)std::lround(nd[a] * M);
      sum += al[1 + a];
    }
    al[d + 1] = (int)std::lround(nd[3] * M);
    sum += al[d + 1];
    al[0] = M - sum;
    S.alpha.push_back(al);
  }
  // nodal basis: theta_l = sum_k C[k][l] m_k with V[n][k] = m_k(node_n), C = V^{-1}
  std::vector<std::array<int, 4>> stm = monomial_list(d + 1, M);
  for (auto& e : stm)
    if (d == 2) {  // variables (xi, eta, tau): move the 3rd exponent into the tau slot
      e[3] = e[2];
      e[2] = 0;
    }
  int L = S.Lc;
  std::vector<double> V((size_t)L * L), C((size_t)L * L, 0.0);
  for (int n = 0; n < L; ++n)
    for (int k = 0; k < L; ++k) {
      double v = 1.0;
      for (int a = 0; a < 4; ++a) v *= std::pow(S.st_nodes[n][a], stm[k][a]);
      V[n * L + k] = v;
    }
  for (int k = 0; k < L; ++k) C[k * L + k] = 1.0;
  gauss_solve(L, V, C, L);
  S.theta.assign(L, Poly());
  for (int l = 0; l < L; ++l) {
    Poly p;
    for (int k = 0; k < L; ++k) p.push_back(monomial(stm[k][0], stm[k][1], stm[k][2], stm[k][3], C[k * L + l]));
    S.theta[l] = normalise(p);
  }
  // Galerkin matrices, Eq. (cgPDE), test functions = unknown (tau > 0) nodes
  int L1 = L - S.L0;
  S.Ktau.assign((size_t)L1 * L, 0.0);
  S.Mmat.assign((size_t)L1 * L, 0.0);
  for (int k = 0; k < L1; ++k)
    for (int l = 0; l < L; ++l) {
      const Poly& tk = S.theta[S.L0 + k];
      S.Ktau[k * L + l] = integrate_prism(poly_mul(tk, poly_deriv(S.theta[l], 3)), d);
      S.Mmat[k * L + l] = integrate_prism(poly_mul(tk, S.theta[l]), d);
    }
  init_predictor_integrals(S);
}

// Space-time predictor of cell i from its reconstruction w (per variable),
// Eq. (CGfinal), in the closed form of init_predictor_integrals: M+1 Picard
// iterations q_k <- w(xi_k) - dt sum_e sum_l Pint[e][k][l] G_e(q_l), with
// G_e = sum_m (d xi_e / d x_m) F_m (Eq. Hterm, Eulerian), from the initial
// guess w(xi) at every node.  qhat: L x nu nodal values.
void predictor_cell(const OSolver& S, long i, const std::vector<Poly>& w, double dt, std::vector<double>& qhat,
                    const double* qbar) {
  int d = S.d, nu = S.nu, L = S.Lc, L0 = S.L0, L1 = L - L0;
  const OMesh& m = *S.mesh;
  double J[3][3], Ji[3][3];
  cell_jacobian(m, i, J);
  inv3(J, d, Ji);  // Ji[e][m] = d xi_e / d x_m
  qhat.assign((size_t)L * nu, 0.0);
  std::vector<double> wk((size_t)L * nu);
  for (int l = 0; l < L; ++l) {
    double x[4] = {S.st_nodes[l][0], S.st_nodes[l][1], S.st_nodes[l][2], 0.0};
    for (int v = 0; v < nu; ++v) wk[l * nu + v] = poly_eval(w[v], x);
  }
  qhat = wk;
  std::vector<double> F((size_t)d * nu), G((size_t)L * d * nu);
  for (int it = 0; it < S.P.niter; ++it) {
    for (int l = 0; l < L; ++l) {
      for (int mm = 0; mm < d; ++mm) flux(S.pde, d, S.P, &qhat[l * nu], mm, &F[mm * nu]);
      for (int e = 0; e < d; ++e)
        for (int v = 0; v < nu; ++v) {
          double g = 0.0;
          for (int mm = 0; mm < d; ++mm) g += Ji[e][mm] * F[mm * nu + v];
          G[((size_t)l * d + e) * nu + v] = g;
        }
    }
    std::vector<double> q1((size_t)L1 * nu);
    for (int k = 0; k < L1; ++k)
      for (int v = 0; v < nu; ++v) {
        double s = 0.0;
        for (int e = 0; e < d; ++e)
          for (int l = 0; l < L; ++l) s += S.Pint[((size_t)e * L1 + k) * L + l] * G[((size_t)l * d + e) * nu + v];
        q1[k * nu + v] = wk[(L0 + k) * nu + v] - dt * s;
      }
    for (int k = 0; k < L1; ++k)
      for (int v = 0; v < nu; ++v) qhat[(L0 + k) * nu + v] = q1[k * nu + v];
  }
  // Predictor fallback (addition, with the positivity switch): if a
  // space-time node left the admissible set (density or pressure <= 0, or
  // not finite), the cell's predictor is its cell average at every node.
  // A lattice node scaled close to vacuum can carry a wave speed far above
  // the cell average's, which the time step of Eq. (timestep) does not see.
  if (qbar && S.P.positivity) {
    bool ok = true;
    for (int l = L0; l < L; ++l) {
      const double* q = &qhat[(size_t)l * nu];
      bool fin = true;
      for (int v = 0; v < nu; ++v) fin = fin && std::isfinite(q[v]);
      if (!(fin && q[0] > 0.0 && pressure(S.pde, d, S.P, q) > 0.0)) ok = false;
    }
    if (!ok)
      for (int l = 0; l < L; ++l)
        for (int v = 0; v < nu; ++v) qhat[(size_t)l * nu + v] = qbar[v];
  }
}

// The same predictor through the Galerkin system of Eq. (CGfinal) as
// written: K_tau^1 q^1 = -dt M H - K_tau^0 q^0 solved every iteration, with
// the matrices integrated exactly from the nodal basis in monomial form.
// Used only to check the closed form (their difference is the rounding of
// the Galerkin solve, which grows with the condition number of K_tau^1).
void predictor_cell_galerkin(const OSolver& S, long i, const std::vector<Poly>& w, double dt,
                             std::vector<double>& qhat) {
  int d = S.d, nu = S.nu, L = S.Lc, L0 = S.L0, L1 = L - L0;
  const OMesh& m = *S.mesh;
  double J[3][3], Ji[3][3];
  cell_jacobian(m, i, J);
  inv3(J, d, Ji);  // Ji[e][m] = d xi_e / d x_m
  qhat.assign((size_t)L * nu, 0.0);
  // known DOFs (tau = 0) and initial guess (w extended constantly in time)
  for (int l = 0; l < L; ++l) {
    double x[4] = {S.st_nodes[l][0], S.st_nodes[l][1], S.st_nodes[l][2], 0.0};
    for (int v = 0; v < nu; ++v) qhat[l * nu + v] = poly_eval(w[v], x);
  }
  // derivatives of the nodal basis at the nodes: dtheta[e][n][l]
  std::vector<double> dth((size_t)d * L * L);
  for (int e = 0; e < d; ++e)
    for (int l = 0; l < L; ++l) {
      Poly dp = poly_deriv(S.theta[l], e);
      for (int n = 0; n < L; ++n) {
        double x[4] = {S.st_nodes[n][0], S.st_nodes[n][1], S.st_nodes[n][2], S.st_nodes[n][3]};
        dth[((size_t)e * L + n) * L + l] = poly_eval(dp, x);
      }
    }
  std::vector<double> K1((size_t)L1 * L1);
  for (int k = 0; k < L1; ++k)
    for (int l = 0; l < L1; ++l) K1[k * L1 + l] = S.Ktau[k * L + L0 + l];
  std::vector<double> F((size_t)L * d * nu), H((size_t)L * nu);
  for (int it = 0; it < S.P.niter; ++it) {
    // nodal fluxes F_hat, Eq. (PDEterm)
    for (int l = 0; l < L; ++l)
      for (int mm = 0; mm < d; ++mm) flux(S.pde, d, S.P, &qhat[l * nu], mm, &F[((size_t)l * d + mm) * nu]);
    // H at the nodes: sum_m sum_e (d xi_e/d x_m) d F_m / d xi_e, Eq. (Hterm), Eulerian
    for (int n = 0; n < L; ++n)
      for (int v = 0; v < nu; ++v) {
        double h = 0.0;
        for (int mm = 0; mm < d; ++mm)
          for (int e = 0; e < d; ++e) {
            double dF = 0.0;
            for (int l = 0; l < L; ++l) dF += dth[((size_t)e * L + n) * L + l] * F[((size_t)l * d + mm) * nu + v];
            h += Ji[e][mm] * dF;
          }
        H[n * nu + v] = h;
      }
    // K_tau^1 q^1 = -dt M H - K_tau^0 q^0, Eq. (CGfinal)
    std::vector<double> rhs((size_t)L1 * nu, 0.0);
    for (int k = 0; k < L1; ++k)
      for (int v = 0; v < nu; ++v) {
        double s = 0.0;
        for (int l = 0; l < L; ++l) s -= dt * S.Mmat[k * L + l] * H[l * nu + v];
        for (int l = 0; l < L0; ++l) s -= S.Ktau[k * L + l] * qhat[l * nu + v];
        rhs[k * nu + v] = s;
      }
    gauss_solve(L1, K1, rhs, nu);
    for (int k = 0; k < L1; ++k)
      for (int v = 0; v < nu; ++v) qhat[(L0 + k) * nu + v] = rhs[k * nu + v];
  }
}

// Value of the predictor polynomial of a cell at reference point (xi, tau).
void eval_qh(const OSolver& S, const std::vector<double>& qhat, const double* xt, double* q) {
  std::vector<double> th(S.Lc);
  st_basis(S, xt, th.data(), nullptr);
  for (int v = 0; v < S.nu; ++v) q[v] = 0.0;
  for (int l = 0; l < S.Lc; ++l)
    for (int v = 0; v < S.nu; ++v) q[v] += th[l] * qhat[l * S.nu + v];
}

// Face quadrature points in physical space for face k of cell i: the face
// vertices are taken in ascending global vertex id; edge: Gauss-Legendre on
// [A,B]; triangle: conical product x = A + s(1-t)(B-A) + t(C-A) with
// Gauss-Legendre in s and Gauss-Jacobi(1,0) in t.  Weights sum to 1.
void face_points(const OSolver& S, long i, int k, std::vector<std::array<double, 3>>& pts, std::vector<double>& wts,
                 double* nrm, double& area) {
  const OMesh& m = *S.mesh;
  int d = m.d, M = S.M;
  std::vector<std::pair<long, int>> fv;
  for (int q = 0; q <= d; ++q)
    if (q != k) fv.push_back({m.cells[i * (d + 1) + q], q});
  std::sort(fv.begin(), fv.end());
  double P[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int r = 0; r < d; ++r)
    for (int a = 0; a < d; ++a) P[r][a] = vx(m, i, fv[r].second, a);
  std::vector<double> xs, ws;
  gauss_legendre01(M + 1, xs, ws);
  pts.clear();
  wts.clear();
  double out[3] = {0, 0, 0};
  if (d == 2) {
    for (int q = 0; q <= M; ++q) {
      pts.push_back({P[0][0] + xs[q] * (P[1][0] - P[0][0]), P[0][1] + xs[q] * (P[1][1] - P[0][1]), 0.0});
      wts.push_back(ws[q]);
    }
    double tx = P[1][0] - P[0][0], ty = P[1][1] - P[0][1];
    area = std::hypot(tx, ty);
    out[0] = ty / area;
    out[1] = -tx / area;
  } else {
    std::vector<double> xt, wt;
    gauss_jacobi10_01(M + 1, xt, wt);
    for (int a = 0; a <= M; ++a)
      for (int b = 0; b <= M; ++b) {
        double s = xs[a], t = xt[b];
        std::array<double, 3> x;
        for (int c = 0; c < 3; ++c) x[c] = P[0][c] + s * (1.0 - t) * (P[1][c] - P[0][c]) + t * (P[2][c] - P[0][c]);
        pts.push_back(x);
        wts.push_back(ws[a] * wt[b]);
      }
    double u[3], w[3];
    for (int c = 0; c < 3; ++c) {
      u[c] = P[1][c] - P[0][c];
      w[c] = P[2][c] - P[0][c];
    }
    double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    double nn = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    area = 0.5 * nn;
    for (int c = 0; c < 3; ++c) out[c] = cr[c] / nn;
  }
  // orient outward from cell i
  double dot = 0.0;
  for (int a = 0; a < d; ++a) dot += out[a] * (P[0][a] - m.bary[i * 3 + a]);
  for (int a = 0; a < 3; ++a) nrm[a] = dot > 0 ? out[a] : -out[a];
}

// ============================================================================
// Moving meshes: the direct ALE step (Secs. 2.2-2.4), two and three space dimensions,
// Euler equations, Rusanov flux with the ALE Jacobian of Eq. (rusanov)
// ============================================================================

// Mesh-velocity choice of Sec. 2.3: ALE_LAGRANGE takes V = v, the local
// fluid velocity (the choice of every moving-mesh test of Sec. 3); ALE_STILL
// takes V = 0, the ALE machinery on a mesh that does not move (it reduces to
// the Eulerian scheme).
enum { ALE_LAGRANGE = 1, ALE_STILL = 2 };

void mesh_velocity(int mode, int d, const double* q, double* V) {
  for (int a = 0; a < d; ++a) V[a] = mode == ALE_LAGRANGE ? q[1 + a] / q[0] : 0.0;
}

double ipow_d(double x, int n) {
  double r = 1.0;
  for (int k = 0; k < n; ++k) r *= x;
  return r;
}

// Space-time predictor on a moving element, Eqs. (PDExi2)-(ODEfinal).  The
// state DOFs q_hat and the geometry DOFs x_hat of the isoparametric map
// (Eq. xh_vh) are iterated together.  Each iteration takes the nodal fluxes
// F_hat and mesh velocities V_hat, the term H of Eq. (Hterm) at every node
// from the xi-derivatives of the nodal interpolants, with d xi / d x the
// inverse of d x_h / d xi at that node and d xi / d t = -(d xi / d x) V, and
// then solves, as written,
//   K_tau^1 q^1 = -dt M H - K_tau^0 q^0        (Eq. CGfinal)
//   K_tau^1 x^1 =  dt M V - K_tau^0 x^0        (Eq. ODEfinal)
// by Gaussian elimination.  Initial guess: w(xi) and the affine map of T_i^n
// at every node; niter (= M+1) iterations.  Vhat: L x d mesh velocities of
// the final nodal states.  With the positivity switch, a cell whose
// predictor leaves the admissible set at a tau > 0 node falls back to its
// cell average at every node (as on fixed meshes).
void ale_predictor_cell(const OSolver& S, long i, const std::vector<Poly>& w, double dt, int mode,
                        std::vector<double>& qhat, std::vector<double>& Vhat, const double* qbar) {
  int d = S.d, nu = S.nu, L = S.Lc, L0 = S.L0, L1 = L - L0;
  const OMesh& m = *S.mesh;
  qhat.assign((size_t)L * nu, 0.0);
  std::vector<double> xh((size_t)L * d);
  for (int l = 0; l < L; ++l) {
    double x[4] = {S.st_nodes[l][0], S.st_nodes[l][1], S.st_nodes[l][2], 0.0};
    for (int v = 0; v < nu; ++v) qhat[l * nu + v] = poly_eval(w[v], x);
    for (int a = 0; a < d; ++a) {
      double xa = vx(m, i, 0, a);
      for (int e = 0; e < d; ++e) xa += (vx(m, i, e + 1, a) - vx(m, i, 0, a)) * S.st_nodes[l][e];
      xh[l * d + a] = xa;
    }
  }
  // dth[e][n][l] = d theta_l / d xi_e at node n
  std::vector<double> dth((size_t)d * L * L);
  for (int e = 0; e < d; ++e)
    for (int l = 0; l < L; ++l) {
      Poly dp = poly_deriv(S.theta[l], e);
      for (int n = 0; n < L; ++n) {
        double x[4] = {S.st_nodes[n][0], S.st_nodes[n][1], S.st_nodes[n][2], S.st_nodes[n][3]};
        dth[((size_t)e * L + n) * L + l] = poly_eval(dp, x);
      }
    }
  std::vector<double> K1((size_t)L1 * L1);
  for (int k = 0; k < L1; ++k)
    for (int l = 0; l < L1; ++l) K1[k * L1 + l] = S.Ktau[k * L + L0 + l];
  std::vector<double> F((size_t)L * d * nu), H((size_t)L * nu), V((size_t)L * d);
  const int nr = nu + d;
  for (int it = 0; it < S.P.niter; ++it) {
    for (int l = 0; l < L; ++l) {
      for (int mm = 0; mm < d; ++mm) flux(S.pde, d, S.P, &qhat[l * nu], mm, &F[((size_t)l * d + mm) * nu]);
      mesh_velocity(mode, d, &qhat[l * nu], &V[l * d]);
    }
    for (int n = 0; n < L; ++n) {
      // Jx[a][e] = d x_a / d xi_e of the isoparametric map at node n
      double Jx[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Ji[3][3];
      for (int a = 0; a < d; ++a)
        for (int e = 0; e < d; ++e) {
          double s = 0.0;
          for (int l = 0; l < L; ++l) s += dth[((size_t)e * L + n) * L + l] * xh[l * d + a];
          Jx[a][e] = s;
        }
      inv3(Jx, d, Ji);  // Ji[e][a] = d xi_e / d x_a
      for (int v = 0; v < nu; ++v) {
        double h = 0.0;
        for (int e = 0; e < d; ++e) {
          double dq = 0.0;
          for (int l = 0; l < L; ++l) dq += dth[((size_t)e * L + n) * L + l] * qhat[l * nu + v];
          double dxidt = 0.0;
          for (int a = 0; a < d; ++a) dxidt -= Ji[e][a] * V[n * d + a];
          h += dq * dxidt;
          for (int mm = 0; mm < d; ++mm) {
            double dF = 0.0;
            for (int l = 0; l < L; ++l) dF += dth[((size_t)e * L + n) * L + l] * F[((size_t)l * d + mm) * nu + v];
            h += Ji[e][mm] * dF;
          }
        }
        H[n * nu + v] = h;
      }
    }
    std::vector<double> rhs((size_t)L1 * nr, 0.0);
    for (int k = 0; k < L1; ++k) {
      for (int v = 0; v < nu; ++v) {
        double s = 0.0;
        for (int l = 0; l < L; ++l) s -= dt * S.Mmat[k * L + l] * H[l * nu + v];
        for (int l = 0; l < L0; ++l) s -= S.Ktau[k * L + l] * qhat[l * nu + v];
        rhs[k * nr + v] = s;
      }
      for (int a = 0; a < d; ++a) {
        double s = 0.0;
        for (int l = 0; l < L; ++l) s += dt * S.Mmat[k * L + l] * V[l * d + a];
        for (int l = 0; l < L0; ++l) s -= S.Ktau[k * L + l] * xh[l * d + a];
        rhs[k * nr + nu + a] = s;
      }
    }
    gauss_solve(L1, K1, rhs, nr);
    for (int k = 0; k < L1; ++k) {
      for (int v = 0; v < nu; ++v) qhat[(L0 + k) * nu + v] = rhs[k * nr + v];
      for (int a = 0; a < d; ++a) xh[(L0 + k) * d + a] = rhs[k * nr + nu + a];
    }
  }
  if (qbar && S.P.positivity) {
    // The fallback takes a tau > 0 node that is inadmissible or whose density
    // or pressure leaves [1/2 min, 2 max] of the tau = 0 nodes' values (a
    // relaxed discrete maximum principle: with V = v the Picard iteration of
    // a cell cut by a strong discontinuity can stop on large, positive
    // oscillations instead of converging).
    double r0 = HUGE_VAL, r1 = -HUGE_VAL, p0 = HUGE_VAL, p1 = -HUGE_VAL;
    for (int l = 0; l < L0; ++l) {
      const double* q = &qhat[(size_t)l * nu];
      const double pl = pressure(S.pde, d, S.P, q);
      r0 = std::min(r0, q[0]);
      r1 = std::max(r1, q[0]);
      p0 = std::min(p0, pl);
      p1 = std::max(p1, pl);
    }
    bool ok = true;
    for (int l = L0; l < L; ++l) {
      const double* q = &qhat[(size_t)l * nu];
      bool fin = true;
      for (int v = 0; v < nu; ++v) fin = fin && std::isfinite(q[v]);
      const double pl = pressure(S.pde, d, S.P, q);
      if (!(fin && q[0] > 0.0 && pl > 0.0)) ok = false;
      if (!(q[0] >= 0.5 * r0 && q[0] <= 2.0 * r1 && pl >= 0.5 * p0 && pl <= 2.0 * p1)) ok = false;
    }
    if (!ok)
      for (int l = 0; l < L; ++l)
        for (int v = 0; v < nu; ++v) qhat[(size_t)l * nu + v] = qbar[v];
  }
  Vhat.assign((size_t)L * d, 0.0);
  for (int l = 0; l < L; ++l) mesh_velocity(mode, d, &qhat[l * nu], &Vhat[l * d]);
}

// Time integrals of the nodal basis at the reference vertices, the weights
// of Eq. (NodesVel): W[v][l] = int_0^1 theta_l(xi_v, tau) dtau with xi_0 = 0
// and xi_v the v-th unit vector, integrated monomial by monomial.
std::vector<double> ale_vertex_weights(const OSolver& S) {
  int d = S.d, L = S.Lc;
  std::vector<double> W((size_t)(d + 1) * L, 0.0);
  for (int v = 0; v <= d; ++v) {
    double xv[3] = {0, 0, 0};
    if (v > 0) xv[v - 1] = 1.0;
    for (int l = 0; l < L; ++l) {
      double s = 0.0;
      for (const Term& t : S.theta[l])
        s += t.c * ipow_d(xv[0], t.e[0]) * ipow_d(xv[1], t.e[1]) * ipow_d(xv[2], t.e[2]) / (t.e[3] + 1);
      W[(size_t)v * L + l] = s;
    }
  }
  return W;
}

// Space-time normal of a lateral face, Eqs. (SurfPar)-(detChi), d = 2.  The
// face is the segment A-B at t^n (XA0, XB0) moving on straight lines to
// (XA1, XB1) at t^{n+1}; x(chi, tau) is the bilinear map of Eq. (SurfPar)
// and t = t^n + tau dt.  The rows of the matrix of Eq. (ChiTransf) below the
// unit vectors are (dx/dchi, dt/dchi = 0) and (dx/dtau, dt/dtau = dt); the
// normal is the cofactor expansion along the first row, (x, y, t) order.
void st_normal(const double* XA0, const double* XB0, const double* XA1, const double* XB1, double chi, double tau,
               double dt, double* n) {
  double r1[3], r2[3];
  for (int a = 0; a < 2; ++a) {
    r1[a] = (1.0 - tau) * (XB0[a] - XA0[a]) + tau * (XB1[a] - XA1[a]);
    r2[a] = (1.0 - chi) * (XA1[a] - XA0[a]) + chi * (XB1[a] - XB0[a]);
  }
  r1[2] = 0.0;
  r2[2] = dt;
  // (-1)^(1+p) times the minor that deletes column p
  n[0] = r1[1] * r2[2] - r1[2] * r2[1];
  n[1] = -(r1[0] * r2[2] - r1[2] * r2[0]);
  n[2] = r1[0] * r2[1] - r1[1] * r2[0];
}

// Space-time normal of a lateral face in three space dimensions, Eqs.
// (BetaBaseFunc)-(detChi): the triangle (A, B, C) at t^n moving on straight
// lines to (A1, B1, C1) at t^{n+1}, x(chi1, chi2, tau) the map of Eq.
// (SurfPar) with the bilinear basis beta_1..beta_6 and t = t^n + tau dt.  The
// rows of the matrix of Eq. (ChiTransf) below the unit vectors are
// (dx/dchi1, 0), (dx/dchi2, 0) and (dx/dtau, dt); component p of the normal is
// (-1)^(1+p) times the 3 x 3 minor that deletes column p, (x, y, z, t) order.
void st_normal3(const double* A0, const double* B0, const double* C0, const double* A1, const double* B1,
                const double* C1, double c1, double c2, double tau, double dt, double* n) {
  double r[3][4];
  for (int a = 0; a < 3; ++a) {
    r[0][a] = (1.0 - tau) * (B0[a] - A0[a]) + tau * (B1[a] - A1[a]);
    r[1][a] = (1.0 - tau) * (C0[a] - A0[a]) + tau * (C1[a] - A1[a]);
    r[2][a] = (1.0 - c1 - c2) * (A1[a] - A0[a]) + c1 * (B1[a] - B0[a]) + c2 * (C1[a] - C0[a]);
  }
  r[0][3] = 0.0;
  r[1][3] = 0.0;
  r[2][3] = dt;
  for (int p = 0; p < 4; ++p) {
    int c[3], k = 0;
    for (int q = 0; q < 4; ++q)
      if (q != p) c[k++] = q;
    const double det = r[0][c[0]] * (r[1][c[1]] * r[2][c[2]] - r[1][c[2]] * r[2][c[1]]) -
                       r[0][c[1]] * (r[1][c[0]] * r[2][c[2]] - r[1][c[2]] * r[2][c[0]]) +
                       r[0][c[2]] * (r[1][c[0]] * r[2][c[1]] - r[1][c[1]] * r[2][c[0]]);
    n[p] = (p % 2 == 0) ? det : -det;
  }
}

// Reference coordinates in cell c of the point at parameter chi on the
// segment from global vertex ga to global vertex gb of that cell: the
// lateral face (chi, tau) sits at the same reference point at every tau.
void ref_on_edge(const OMesh& m, long c, long ga, long gb, double chi, double* xi) {
  int d = m.d;
  double pa[3] = {0, 0, 0}, pb[3] = {0, 0, 0};
  for (int k = 0; k <= d; ++k) {
    long g = m.cells[c * (d + 1) + k];
    if (k > 0 && g == ga) pa[k - 1] = 1.0;
    if (k > 0 && g == gb) pb[k - 1] = 1.0;
  }
  for (int a = 0; a < 3; ++a) xi[a] = pa[a] + chi * (pb[a] - pa[a]);
}

// The same on a triangular face (global vertices ga, gb, gc of cell c) at
// parameters (chi1, chi2): A + chi1 (B - A) + chi2 (C - A) in cell c's frame.
void ref_on_face(const OMesh& m, long c, const long* g, double c1, double c2, double* xi) {
  int d = m.d;
  double p[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int k = 1; k <= d; ++k) {
    long gk = m.cells[c * (d + 1) + k];
    for (int r = 0; r < 3; ++r)
      if (gk == g[r]) p[r][k - 1] = 1.0;
  }
  for (int a = 0; a < 3; ++a) xi[a] = p[0][a] + c1 * (p[1][a] - p[0][a]) + c2 * (p[2][a] - p[0][a]);
}

// One direct ALE ADER-CWENO step on the solver's current mesh:
//   1. reconstruction (fixed stencils, matrices of the current geometry) and
//      the moving-element predictor of every cell;
//   2. nodal solver, Eqs. (NScs), (NScs.weights), (NodesVel): the velocity
//      of vertex k is the mass-weighted mean over its cells j of the time
//      integral of the predictor's mesh velocity at that vertex, with masses
//      rho_j^n |T_j^n| and cells visited in increasing index; new positions
//      by Eq. (newX);
//   3. the space-time control volumes of Eq. (dCi): bottom T_i^n, top
//      T_i^{n+1}, lateral faces (SurfPar) with normals (detChi);
//   4. Eq. (PDEfinal): |T_i^{n+1}| Q_i^{n+1} = |T_i^n| Q_i^n minus the
//      lateral-face integrals of the Rusanov flux of Eq. (rusanov),
//      (F~(q+) + F~(q-)) . n~ / 2 - s_max (q+ - q-) / 2 with
//      F~ = (f, g, Q), s_max = |n~_x| max over both sides of |v.n - V.n| + c
//      (the largest eigenvalue of the ALE Jacobian A_n^V), V.n = -n~_t/|n~_x|
//      the face's own normal velocity; Gauss-Legendre with M+1 points in chi
//      and in tau.  Transmissive boundary: q+ = q-.
// Qnew: nc x nu; xyz_new: nv x d.  The mesh is not moved (ale_move does).
bool ale_step(OSolver& S, const double* Q, double dt, int mode, double* Qnew, double* xyz_new, std::string& err) {
  OMesh& m = *S.mesh;
  int d = m.d, nu = S.nu, L = S.Lc, M = S.M;
  if (S.pde != PDE_EULER || S.P.flux != 0) {
    err = "moving meshes: Euler equations, Rusanov flux";
    return false;
  }
  std::vector<std::vector<double>> pred(m.nc), Vh(m.nc);
  for (long c = 0; c < m.nc; ++c) {
    RecOut R;
    if (!reconstruct_cell(S, Q, c, R, err)) return false;
    ale_predictor_cell(S, c, R.w, dt, mode, pred[c], Vh[c], &Q[c * nu]);
  }
  // nodal solver
  std::vector<double> W = ale_vertex_weights(S);
  std::vector<double> acc((size_t)m.nv * d, 0.0), mu(m.nv, 0.0);
  for (long c = 0; c < m.nc; ++c) {
    double mass = Q[c * nu] * m.vol[c];
    for (int k = 0; k <= d; ++k) {
      long g = m.cells[c * (d + 1) + k];
      for (int a = 0; a < d; ++a) {
        double vkj = 0.0;
        for (int l = 0; l < L; ++l) vkj += W[(size_t)k * L + l] * Vh[c][(size_t)l * d + a];
        acc[g * d + a] += mass * vkj;
      }
      mu[g] += mass;
    }
  }
  for (long g = 0; g < m.nv; ++g)  // a vertex of no cell keeps its position
    for (int a = 0; a < d; ++a)
      xyz_new[g * d + a] = mu[g] > 0.0 ? m.xyz[g * d + a] + dt * (acc[g * d + a] / mu[g]) : m.xyz[g * d + a];
  // geometry at t^{n+1}
  OMesh m1 = m;
  m1.xyz.assign(xyz_new, xyz_new + m.nv * d);
  if (!mesh_geometry(m1, err)) {
    err = "moving mesh: " + err;
    return false;
  }
  // lateral-face rule in (chi) or (chi1, chi2): Gauss-Legendre with M + 1
  // points on the segment; on the triangle the collapsed product chi1 =
  // s (1 - r), chi2 = r of M + 1 Gauss-Legendre points s and M + 1
  // Gauss-Jacobi points r (weight 1 - r), weights times 1/2, the area of the
  // reference triangle (exact to degree 2M + 1); Gauss-Legendre in tau.
  std::vector<double> gx, gw;
  gauss_legendre01(M + 1, gx, gw);
  std::vector<std::array<double, 2>> fchi;
  std::vector<double> fw;
  if (d == 2) {
    for (int q = 0; q <= M; ++q) {
      fchi.push_back({gx[q], 0.0});
      fw.push_back(gw[q]);
    }
  } else {
    std::vector<double> jx, jw;
    gauss_jacobi10_01(M + 1, jx, jw);
    for (int a = 0; a <= M; ++a)
      for (int b = 0; b <= M; ++b) {
        fchi.push_back({gx[a] * (1.0 - jx[b]), jx[b]});
        fw.push_back(0.5 * gw[a] * jw[b]);
      }
  }
  std::vector<double> qm(nu), qp(nu), f(nu), g(nu);
  for (long i = 0; i < m.nc; ++i) {
    std::vector<double> accq(nu, 0.0);
    for (int k = 0; k <= d; ++k) {
      long j = m.nbr[i * (d + 1) + k];
      // face vertices: the cell's local vertices other than k, ordered by
      // global id so that both sides parametrise the face alike
      std::vector<std::pair<long, int>> fv;
      for (int q = 0; q <= d; ++q)
        if (q != k) fv.push_back({m.cells[i * (d + 1) + q], q});
      std::sort(fv.begin(), fv.end());
      long gf[3] = {fv[0].first, fv[1].first, d == 3 ? fv[2].first : -1};
      double P0[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, P1[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int r = 0; r < d; ++r)
        for (int a = 0; a < d; ++a) {
          P0[r][a] = vx(m, i, fv[r].second, a);
          P1[r][a] = vx(m1, i, fv[r].second, a);
        }
      auto normal = [&](double c1, double c2, double tau, double* n) {
        if (d == 2) st_normal(P0[0], P0[1], P1[0], P1[1], c1, tau, dt, n);
        else st_normal3(P0[0], P0[1], P0[2], P1[0], P1[1], P1[2], c1, c2, tau, dt, n);
      };
      // outward orientation from cell i at t^n
      double n0[4];
      normal(0.0, 0.0, 0.0, n0);
      double dot = 0.0;
      for (int a = 0; a < d; ++a) dot += n0[a] * (P0[0][a] - m.bary[i * 3 + a]);
      const double sgn = dot > 0 ? 1.0 : -1.0;
      for (size_t q = 0; q < fchi.size(); ++q) {
        double xi_i[3], xi_j[3];
        if (d == 2) {
          ref_on_edge(m, i, gf[0], gf[1], fchi[q][0], xi_i);
          if (j >= 0) ref_on_edge(m, j, gf[0], gf[1], fchi[q][0], xi_j);
        } else {
          ref_on_face(m, i, gf, fchi[q][0], fchi[q][1], xi_i);
          if (j >= 0) ref_on_face(m, j, gf, fchi[q][0], fchi[q][1], xi_j);
        }
        for (int t = 0; t <= M; ++t) {
          double nt[4];
          normal(fchi[q][0], fchi[q][1], gx[t], nt);
          for (int a = 0; a <= d; ++a) nt[a] *= sgn;
          double xt[4] = {xi_i[0], xi_i[1], xi_i[2], gx[t]};
          eval_qh(S, pred[i], xt, qm.data());
          if (j >= 0) {
            double xtj[4] = {xi_j[0], xi_j[1], xi_j[2], gx[t]};
            eval_qh(S, pred[j], xtj, qp.data());
          } else {
            qp = qm;
          }
          if (S.P.positivity) {
            if (!(qm[0] > 0.0 && pressure(S.pde, d, S.P, qm.data()) > 0.0))
              for (int v = 0; v < nu; ++v) qm[v] = Q[i * nu + v];
            if (!(qp[0] > 0.0 && pressure(S.pde, d, S.P, qp.data()) > 0.0))
              for (int v = 0; v < nu; ++v) qp[v] = j >= 0 ? Q[j * nu + v] : Q[i * nu + v];
          }
          double nx = 0.0;
          for (int a = 0; a < d; ++a) nx += nt[a] * nt[a];
          nx = std::sqrt(nx);
          double un[3] = {0, 0, 0};
          for (int a = 0; a < d; ++a) un[a] = nt[a] / nx;
          double Vn = -nt[d] / nx;
          double sm = 0.0;
          for (const double* qs : {qm.data(), qp.data()}) {
            double vn = 0.0;
            for (int a = 0; a < d; ++a) vn += qs[1 + a] * un[a];
            vn /= qs[0];
            double c = max_speed_normal(S.pde, d, S.P, qs, un) - std::fabs(vn);  // sound speed
            sm = std::max(sm, std::fabs(vn - Vn) + c);
          }
          sm *= nx;
          std::vector<double> G(nu, 0.0);
          for (int mm = 0; mm < d; ++mm) {
            flux(S.pde, d, S.P, qm.data(), mm, f.data());
            flux(S.pde, d, S.P, qp.data(), mm, g.data());
            for (int v = 0; v < nu; ++v) G[v] += 0.5 * (f[v] + g[v]) * nt[mm];
          }
          for (int v = 0; v < nu; ++v) G[v] += 0.5 * (qm[v] + qp[v]) * nt[d] - 0.5 * sm * (qp[v] - qm[v]);
          for (int v = 0; v < nu; ++v) accq[v] += fw[q] * gw[t] * G[v];
        }
      }
    }
    for (int v = 0; v < nu; ++v) Qnew[i * nu + v] = (m.vol[i] * Q[i * nu + v] - accq[v]) / m1.vol[i];
  }
  return true;
}

// Move the mesh to new vertex positions (same topology) and rebuild every
// cell's geometry-dependent matrices for its fixed stencils.
bool ale_move(OSolver& S, const double* xyz, std::string& err) {
  OMesh& m = *S.mesh;
  m.xyz.assign(xyz, xyz + m.nv * m.d);
  if (!mesh_geometry(m, err)) return false;
  for (auto& kv : S.cache) cell_matrices(S, kv.first, kv.second);
  return true;
}

}  // namespace

// ============================================================================
// C API (ctypes)
// ============================================================================
extern "C" {

static void set_err(char* buf, int len, const std::string& s) {
  if (buf && len > 0) {
    std::snprintf(buf, (size_t)len, "%s", s.c_str());
  }
}

void* orc_mesh_new(int d, int64_t nv, const double* xyz, int64_t nc, const int64_t* cells, const double* period,
                   char* err, int errlen) {
  OMesh* m = new OMesh();
  m->d = d;
  m->nv = nv;
  m->nc = nc;
  m->xyz.assign(xyz, xyz + nv * d);
  m->cells.assign(cells, cells + nc * (d + 1));
  for (int a = 0; a < d; ++a)
    if (period && period[a] > 0) {
      m->per[a] = true;
      m->L[a] = period[a];
    }
  std::string e;
  if (!build_mesh(*m, e)) {
    set_err(err, errlen, e);
    delete m;
    return nullptr;
  }
  return m;
}

void orc_mesh_free(void* p) { delete (OMesh*)p; }

// vol[nc], bary[nc*3], h[nc], nbr[nc*(d+1)]
int orc_mesh_geometry(void* p, double* vol, double* bary, double* h, int64_t* nbr) {
  OMesh* m = (OMesh*)p;
  for (long c = 0; c < m->nc; ++c) {
    if (vol) vol[c] = m->vol[c];
    if (bary)
      for (int a = 0; a < 3; ++a) bary[c * 3 + a] = m->bary[c * 3 + a];
    if (h) h[c] = cell_h(*m, c);
    if (nbr)
      for (int k = 0; k <= m->d; ++k) nbr[c * (m->d + 1) + k] = m->nbr[c * (m->d + 1) + k];
  }
  return 0;
}

// params: eps, r, lam0, lams, gamma, ch, cfl, niter, linear_weights, positivity, flux
void* orc_solver_new(void* mesh, int M, int pde, const double* prm, char* err, int errlen) {
  OMesh* m = (OMesh*)mesh;
  if (M < 1 || M > 4 || (pde != PDE_EULER && pde != PDE_MHD)) {
    set_err(err, errlen, "unsupported order or PDE");
    return nullptr;
  }
  OSolver* S = new OSolver();
  S->mesh = m;
  S->M = M;
  S->pde = pde;
  S->d = m->d;
  S->nu = nvars(pde, m->d);
  S->P.eps = prm[0];
  S->P.r = prm[1];
  S->P.lam0 = prm[2];
  S->P.lams = prm[3];
  S->P.gamma = prm[4];
  S->P.ch = prm[5];
  S->P.cfl = prm[6];
  S->P.niter = (int)prm[7];
  S->P.linear_weights = (int)prm[8];
  S->P.positivity = (int)prm[9];
  S->P.flux = (int)prm[10];
  if (S->P.flux < 0 || S->P.flux > 2 || (S->P.flux == 1 && pde != PDE_EULER)) {
    delete S;
    set_err(err, errlen, "unknown flux, or the Osher-type flux outside the Euler equations");
    return nullptr;
  }
  S->Mc = Mcal(M, m->d);
  S->ne = m->d * S->Mc;
  S->mono = monomial_list(m->d, M);
  init_predictor(*S);
  return S;
}

void orc_solver_free(void* p) { delete (OSolver*)p; }

int orc_sizes(void* p, int* out /* Mc, ne, L, L0, nu */) {
  OSolver* S = (OSolver*)p;
  out[0] = S->Mc;
  out[1] = S->ne;
  out[2] = S->Lc;
  out[3] = S->L0;
  out[4] = S->nu;
  return 0;
}

// Central stencil (ne ids, S0[0] = cell) and sectors ((d+1) x d ids, -1 if dropped).
int orc_stencil(void* p, int64_t cell, int64_t* S0, int64_t* sec, char* err, int errlen) {
  OSolver* S = (OSolver*)p;
  std::string e;
  if (!prepare_cell(*S, cell, e)) {
    set_err(err, errlen, e);
    return -1;
  }
  const CellRec& R = S->cache[cell];
  for (int k = 0; k < S->ne; ++k) S0[k] = R.st.S0[k];
  for (int s = 0; s <= S->d; ++s)
    for (int k = 0; k < S->d; ++k) sec[s * S->d + k] = R.st.sector[s].empty() ? -1 : R.st.sector[s][k];
  return 0;
}

// Reconstruction at the lattice nodes for cells ids[0..n) (ids NULL -> all).
// w: n x Mc x nu, popt (nullable): n x Mc x nu, omega/sigma (nullable): n x (d+2) x nu.
int orc_reconstruct(void* p, const double* Q, int64_t n, const int64_t* ids, double* w, double* popt, double* omega,
                    double* sigma, char* err, int errlen) {
  OSolver* S = (OSolver*)p;
  long cnt = ids ? n : S->mesh->nc;
  int nu = S->nu, Mc = S->Mc, d = S->d;
  for (long c = 0; c < cnt; ++c) {
    long i = ids ? ids[c] : c;
    RecOut R;
    std::string e;
    if (!reconstruct_cell(*S, Q, i, R, e)) {
      set_err(err, errlen, e);
      return -1;
    }
    for (int node = 0; node < Mc; ++node) {
      double x[4] = {S->lat[node][0], S->lat[node][1], S->lat[node][2], 0.0};
      for (int v = 0; v < nu; ++v) {
        if (w) w[((size_t)c * Mc + node) * nu + v] = poly_eval(R.w[v], x);
        if (popt) popt[((size_t)c * Mc + node) * nu + v] = poly_eval(R.popt[v], x);
      }
    }
    for (int s = 0; s < d + 2; ++s)
      for (int v = 0; v < nu; ++v) {
        if (omega) omega[((size_t)c * (d + 2) + s) * nu + v] = R.omega[s * nu + v];
        if (sigma) sigma[((size_t)c * (d + 2) + s) * nu + v] = R.sigma[s * nu + v];
      }
  }
  return 0;
}

// Predictor nodal values q_hat (n x L x nu) for cells ids (NULL -> all).
int orc_predictor(void* p, const double* Q, double dt, int64_t n, const int64_t* ids, double* qhat, char* err,
                  int errlen) {
  OSolver* S = (OSolver*)p;
  long cnt = ids ? n : S->mesh->nc;
  int nu = S->nu, L = S->Lc;
  for (long c = 0; c < cnt; ++c) {
    long i = ids ? ids[c] : c;
    RecOut R;
    std::string e;
    if (!reconstruct_cell(*S, Q, i, R, e)) {
      set_err(err, errlen, e);
      return -1;
    }
    std::vector<double> qh;
    predictor_cell(*S, i, R.w, dt, qh, &Q[i * nu]);
    for (int l = 0; l < L; ++l)
      for (int v = 0; v < nu; ++v) qhat[((size_t)c * L + l) * nu + v] = qh[l * nu + v];
  }
  return 0;
}

// Predictor from given reconstruction values at the lattice nodes (Mc x nu);
// galerkin != 0 takes the Galerkin solve of Eq. (CGfinal) instead of the
// closed form.
int orc_predictor_from_w(void* p, int64_t cell, const double* wnodal, double dt, int galerkin, double* qhat) {
  OSolver* S = (OSolver*)p;
  int nu = S->nu, Mc = S->Mc, d = S->d;
  // interpolate: monomial coefficients from lattice values
  std::vector<double> V((size_t)Mc * Mc), C((size_t)Mc * nu);
  for (int n = 0; n < Mc; ++n) {
    for (int k = 0; k < Mc; ++k) {
      double v = 1.0;
      for (int a = 0; a < d; ++a) v *= std::pow(S->lat[n][a], S->mono[k][a]);
      V[n * Mc + k] = v;
    }
    for (int v = 0; v < nu; ++v) C[n * nu + v] = wnodal[n * nu + v];
  }
  gauss_solve(Mc, V, C, nu);
  std::vector<Poly> w(nu);
  for (int v = 0; v < nu; ++v) {
    std::vector<double> c(Mc);
    for (int k = 0; k < Mc; ++k) c[k] = C[k * nu + v];
    w[v] = poly_from_coef(*S, c.data());
  }
  std::vector<double> qh;
  if (galerkin) predictor_cell_galerkin(*S, cell, w, dt, qh);
  else predictor_cell(*S, cell, w, dt, qh, nullptr);
  for (size_t k = 0; k < qh.size(); ++k) qhat[k] = qh[k];
  return 0;
}

// Quadrature-free Rusanov flux of one face (the fixed-mesh formulation the
// paper describes after Eq. osher): with the nodal expansions of the
// predictor and of its flux (Eq. PDEterm), the face and time integrals
// reduce to the integrals I_l of each side's nodal basis over the face and
// [0,1] (normalised by |f|), so the time-averaged normal flux is
//   1/2 sum_l (I-_l F(q-_l) + I+_l F(q+_l)) . n - 1/2 s (qbar+ - qbar-),
// qbar = sum_l I_l q_l the space-time face average of a side's predictor and
// s the larger maximal signal speed along n of the two averages (reading:
// the paper fixes no constant s for this form).  I_l are computed here by
// the face and time Gauss rules (exact: the integrand has degree M).  A
// nodal state that is not admissible contributes its cell average's flux,
// and an inadmissible face average its cell average's speed (positivity
// safeguard, as for the quadrature flux).  G: time-averaged flux per |f|.
void qf_face_flux(const OSolver& S, const double* Q, std::map<long, std::vector<double>>& pred, long i, long j,
                  const std::vector<std::array<double, 3>>& pts, const std::vector<double>& wts, const double* sj,
                  const double* nrm, const std::vector<double>& tx, const std::vector<double>& tw, double* G) {
  const OMesh& m = *S.mesh;
  const int d = S.d, nu = S.nu, L = S.Lc;
  std::vector<double> Ii(L, 0.0), Ij(L, 0.0), th(L);
  for (size_t q = 0; q < pts.size(); ++q) {
    double xi_i[3], xi_j[3];
    to_ref(m, i, pts[q].data(), xi_i);
    if (j >= 0) {
      double xj[3] = {pts[q][0] - sj[0], pts[q][1] - sj[1], pts[q][2] - sj[2]};
      to_ref(m, j, xj, xi_j);
    }
    for (size_t t = 0; t < tx.size(); ++t) {
      double xt[4] = {xi_i[0], xi_i[1], xi_i[2], tx[t]};
      st_basis(S, xt, th.data(), nullptr);
      for (int l = 0; l < L; ++l) Ii[l] += wts[q] * tw[t] * th[l];
      if (j >= 0) {
        double xtj[4] = {xi_j[0], xi_j[1], xi_j[2], tx[t]};
        st_basis(S, xtj, th.data(), nullptr);
        for (int l = 0; l < L; ++l) Ij[l] += wts[q] * tw[t] * th[l];
      }
    }
  }
  // one side: sum_l I_l F_n(q_l) and qbar
  auto side = [&](long c, const std::vector<double>& I, std::vector<double>& Fn, std::vector<double>& qbar) {
    const std::vector<double>& qh = pred[c];
    Fn.assign(nu, 0.0);
    qbar.assign(nu, 0.0);
    std::vector<double> f(nu);
    for (int l = 0; l < L; ++l) {
      const double* ql = &qh[(size_t)l * nu];
      const double* qs = ql;
      if (S.P.positivity && !(ql[0] > 0.0 && pressure(S.pde, d, S.P, ql) > 0.0)) qs = &Q[c * nu];
      for (int mm = 0; mm < d; ++mm) {
        flux(S.pde, d, S.P, qs, mm, f.data());
        for (int v = 0; v < nu; ++v) Fn[v] += I[l] * nrm[mm] * f[v];
      }
      for (int v = 0; v < nu; ++v) qbar[v] += I[l] * ql[v];
    }
  };
  std::vector<double> Fi, qi, Fj, qj;
  side(i, Ii, Fi, qi);
  if (j >= 0) {
    side(j, Ij, Fj, qj);
  } else {  // transmissive boundary: the outer side is the inner one
    Fj = Fi;
    qj = qi;
  }
  const double* si = qi.data();
  const double* sjp = qj.data();
  if (S.P.positivity) {
    if (!(qi[0] > 0.0 && pressure(S.pde, d, S.P, qi.data()) > 0.0)) si = &Q[i * nu];
    if (!(qj[0] > 0.0 && pressure(S.pde, d, S.P, qj.data()) > 0.0)) sjp = j >= 0 ? &Q[j * nu] : &Q[i * nu];
  }
  double smax = std::max(max_speed_normal(S.pde, d, S.P, si, nrm), max_speed_normal(S.pde, d, S.P, sjp, nrm));
  for (int v = 0; v < nu; ++v) G[v] = 0.5 * (Fi[v] + Fj[v]) - 0.5 * smax * (qj[v] - qi[v]);
}

// One ADER-CWENO step, Eq. (PDEfinal) (Eulerian), for cells ids (NULL -> all).
// Qnew: n x nu.
int orc_step(void* p, const double* Q, double dt, int64_t n, const int64_t* ids, double* Qnew, char* err,
             int errlen) {
  OSolver* S = (OSolver*)p;
  const OMesh& m = *S->mesh;
  int d = S->d, nu = S->nu, M = S->M;
  long cnt = ids ? n : m.nc;
  // predictors of every cell involved
  std::map<long, std::vector<double>> pred;
  for (long c = 0; c < cnt; ++c) {
    long i = ids ? ids[c] : c;
    std::vector<long> need(1, i);
    for (int k = 0; k <= d; ++k)
      if (m.nbr[i * (d + 1) + k] >= 0) need.push_back(m.nbr[i * (d + 1) + k]);
    for (long j : need) {
      if (pred.count(j)) continue;
      RecOut R;
      std::string e;
      if (!reconstruct_cell(*S, Q, j, R, e)) {
        set_err(err, errlen, e);
        return -1;
      }
      predictor_cell(*S, j, R.w, dt, pred[j], &Q[j * S->nu]);
    }
  }
  std::vector<double> tx, tw;
  gauss_legendre01(M + 1, tx, tw);
  std::vector<double> qm(nu), qp(nu), fdir(nu);
  for (long c = 0; c < cnt; ++c) {
    long i = ids ? ids[c] : c;
    std::vector<double> acc(nu, 0.0);
    for (int k = 0; k <= d; ++k) {
      long j = m.nbr[i * (d + 1) + k];
      std::vector<std::array<double, 3>> pts;
      std::vector<double> wts;
      double nrm[3], area;
      face_points(*S, i, k, pts, wts, nrm, area);
      double sj[3] = {0, 0, 0};
      if (j >= 0) min_image_shift(m, i, j, sj);
      if (S->P.flux == 2) {
        qf_face_flux(*S, Q, pred, i, j, pts, wts, sj, nrm, tx, tw, fdir.data());
        for (int v = 0; v < nu; ++v) acc[v] += dt * area * fdir[v];
        continue;
      }
      for (size_t q = 0; q < pts.size(); ++q) {
        double xi_i[3], xi_j[3];
        to_ref(m, i, pts[q].data(), xi_i);
        if (j >= 0) {
          double xj[3] = {pts[q][0] - sj[0], pts[q][1] - sj[1], pts[q][2] - sj[2]};
          to_ref(m, j, xj, xi_j);
        }
        for (int t = 0; t <= M; ++t) {
          double xt[4] = {xi_i[0], xi_i[1], xi_i[2], tx[t]};
          eval_qh(*S, pred[i], xt, qm.data());
          if (j >= 0) {
            double xtj[4] = {xi_j[0], xi_j[1], xi_j[2], tx[t]};
            eval_qh(*S, pred[j], xtj, qp.data());
          } else {
            qp = qm;  // transmissive boundary
          }
          if (S->P.positivity) {
            if (!(qm[0] > 0.0 && pressure(S->pde, d, S->P, qm.data()) > 0.0))
              for (int v = 0; v < nu; ++v) qm[v] = Q[i * nu + v];
            if (!(qp[0] > 0.0 && pressure(S->pde, d, S->P, qp.data()) > 0.0))
              for (int v = 0; v < nu; ++v) qp[v] = j >= 0 ? Q[j * nu + v] : Q[i * nu + v];
          }
          // numerical flux, Eq. (rusanov) or (osher), Eulerian normal (n |f| dt, 0)
          numerical_flux(S->pde, d, S->P, qm.data(), qp.data(), nrm, fdir.data());
          for (int v = 0; v < nu; ++v) acc[v] += dt * area * wts[q] * tw[t] * fdir[v];
        }
      }
    }
    for (int v = 0; v < nu; ++v) Qnew[c * nu + v] = Q[i * nu + v] - acc[v] / m.vol[i];
  }
  return 0;
}

// Global time step, Eq. (timestep).
double orc_stable_dt(void* p, const double* Q, double cfl) {
  OSolver* S = (OSolver*)p;
  const OMesh& m = *S->mesh;
  double best = 1e300;
  for (long c = 0; c < m.nc; ++c) {
    double lam = max_speed(S->pde, S->d, S->P, &Q[c * S->nu]);
    best = std::min(best, cell_h(m, c) / lam);
  }
  return cfl * best;
}

// --- building blocks exposed for pins -------------------------------------
int orc_physical_flux(int pde, int d, const double* prm, const double* q, int m, double* f) {
  Params P;
  P.gamma = prm[4];
  P.ch = prm[5];
  flux(pde, d, P, q, m, f);
  return 0;
}

double orc_max_speed_normal(int pde, int d, const double* prm, const double* q, const double* n) {
  Params P;
  P.gamma = prm[4];
  P.ch = prm[5];
  return max_speed_normal(pde, d, P, q, n);
}

// Numerical normal flux (prm[10] selects Rusanov / Osher) and |A_n| (Euler).
int orc_numerical_flux(int pde, int d, const double* prm, const double* qm, const double* qp, const double* n,
                       double* G) {
  Params P;
  P.gamma = prm[4];
  P.ch = prm[5];
  P.flux = (int)prm[10];
  numerical_flux(pde, d, P, qm, qp, n, G);
  return 0;
}

int orc_abs_jacobian(int d, double gamma, const double* q, const double* n, double* out) {
  euler_abs_jacobian(d, gamma, q, n, out);
  return 0;
}

double orc_max_speed(int pde, int d, const double* prm, const double* q) {
  Params P;
  P.gamma = prm[4];
  P.ch = prm[5];
  return max_speed(pde, d, P, q);
}

// kind 0: Gauss-Legendre on [0,1]; kind 1: Gauss-Jacobi weight (1-t) on [0,1]
int orc_gauss_rule(int kind, int n, double* x, double* w) {
  std::vector<double> xs, ws;
  if (kind == 0) gauss_legendre01(n, xs, ws);
  else gauss_jacobi10_01(n, xs, ws);
  for (int i = 0; i < n; ++i) {
    x[i] = xs[i];
    w[i] = ws[i];
  }
  return 0;
}

// Exact integral over T_E of a monomial (nvar spatial dims).
double orc_simplex_integral(int d, const int* e) { return simplex_integral(d, e); }

// Oscillation indicator of the polynomial given by monomial coefficients in
// the solver's monomial order (orc_monomials).
double orc_sigma(void* p, const double* coef) {
  OSolver* S = (OSolver*)p;
  return sigma_of(*S, poly_from_coef(*S, coef));
}

int orc_monomials(void* p, int* exps /* Mc x 3 */) {
  OSolver* S = (OSolver*)p;
  for (int e = 0; e < S->Mc; ++e)
    for (int a = 0; a < 3; ++a) exps[e * 3 + a] = S->mono[e][a];
  return 0;
}

// Space-time nodes (L x 4: xi, eta, zeta, tau).
int orc_st_nodes(void* p, double* out) {
  OSolver* S = (OSolver*)p;
  for (int l = 0; l < S->Lc; ++l)
    for (int a = 0; a < 4; ++a) out[l * 4 + a] = S->st_nodes[l][a];
  return 0;
}

// Face quadrature of face k of a cell (points npts x 3, weights, normal, area).
int orc_face_points(void* p, int64_t cell, int k, double* pts, double* wts, double* nrm, double* area) {
  OSolver* S = (OSolver*)p;
  std::vector<std::array<double, 3>> P;
  std::vector<double> W;
  face_points(*S, cell, k, P, W, nrm, *area);
  for (size_t q = 0; q < P.size(); ++q) {
    for (int a = 0; a < 3; ++a) pts[q * 3 + a] = P[q][a];
    wts[q] = W[q];
  }
  return (int)P.size();
}


// Direct ALE step (Euler, Rusanov): Qnew (nc x nu) and the
// new vertex positions xyz_new (nv x d); the oracle's mesh is then moved to
// them (stencils fixed, matrices rebuilt).  mode: 1 V = v, 2 V = 0.
int orc_ale_step(void* p, const double* Q, double dt, int mode, double* Qnew, double* xyz_new, char* err,
                 int errlen) {
  OSolver* S = (OSolver*)p;
  std::string e;
  if (mode != ALE_LAGRANGE && mode != ALE_STILL) {
    set_err(err, errlen, "unknown mesh-velocity mode");
    return -1;
  }
  if (!ale_step(*S, Q, dt, mode, Qnew, xyz_new, e) || !ale_move(*S, xyz_new, e)) {
    set_err(err, errlen, e);
    return -1;
  }
  return 0;
}

// Moving-element predictor of one cell from its reconstruction: qhat (L x nu)
// and the nodal mesh velocities Vhat (L x d).
int orc_ale_predictor(void* p, const double* Q, double dt, int mode, int64_t cell, double* qhat, double* Vhat,
                      char* err, int errlen) {
  OSolver* S = (OSolver*)p;
  RecOut R;
  std::string e;
  if (!reconstruct_cell(*S, Q, cell, R, e)) {
    set_err(err, errlen, e);
    return -1;
  }
  std::vector<double> qh, vh;
  ale_predictor_cell(*S, cell, R.w, dt, mode, qh, vh, &Q[cell * S->nu]);
  std::memcpy(qhat, qh.data(), sizeof(double) * qh.size());
  std::memcpy(Vhat, vh.data(), sizeof(double) * vh.size());
  return 0;
}

// W[(d+1) x L], Eq. (NodesVel)
int orc_ale_vertex_weights(void* p, double* W) {
  std::vector<double> w = ale_vertex_weights(*(OSolver*)p);
  std::memcpy(W, w.data(), sizeof(double) * w.size());
  return 0;
}

// Space-time normal of a lateral face, Eq. (detChi), d = 2: n[3] = (x, y, t).
int orc_st_normal(const double* XA0, const double* XB0, const double* XA1, const double* XB1, double chi,
                  double tau, double dt, double* n) {
  st_normal(XA0, XB0, XA1, XB1, chi, tau, dt, n);
  return 0;
}

// Space-time normal (x, y, z, t) of a moving triangle, Eq. (detChi), d = 3.
int orc_st_normal3(const double* A0, const double* B0, const double* C0, const double* A1, const double* B1,
                   const double* C1, double c1, double c2, double tau, double dt, double* n) {
  st_normal3(A0, B0, C0, A1, B1, C1, c1, c2, tau, dt, n);
  return 0;
}

// Current vertex positions of the oracle's mesh (nv x d).
int orc_mesh_xyz(void* p, double* xyz) {
  OMesh* m = (OMesh*)p;
  std::memcpy(xyz, m->xyz.data(), sizeof(double) * m->xyz.size());
  return 0;
}

}  // extern "C"
