// Reference-element tables of the ADER-CWENO scheme (host, FP64).
//
// Everything here is universal: it depends on (d, M) only, never on a mesh.
//   * orthonormal Dubiner-type basis psi_l on T_E (Sec. 2.1, Eq. recpolydef),
//     with psi_0 := 1 so that the cell average is the first coefficient;
//   * oscillation-indicator matrix Sigma_lm (Sec. 2.1);
//   * space-time nodal basis theta_l and the predictor matrices of the
//     Picard update of Eq. (CGfinal), in the closed form of its Galerkin
//     solution (exact time integration of the interpolated flux divergence);
//   * space-time Gauss quadrature on faces (Sec. 2.4) as basis tables.
#pragma once
#include <array>
#include <vector>

namespace cw {

int mcal(int M, int d);  // Eq. (cwenoM)

// Gauss-Jacobi rule on [-1,1], weight (1-x)^a (1+x)^b (Golub-Welsch).
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);

// Collapsed (conical product) rule on the unit d-simplex, n points per
// direction, exact to degree 2n-1; weights sum to |T_E| = 1/d!.
struct SimplexQuad {
  int d = 2;
  std::vector<std::array<double, 3>> x;
  std::vector<double> w;
};
SimplexQuad simplex_quad(int d, int n);

// Power-form polynomial in nvar <= 4 variables over an explicit monomial list.
struct PPoly {
  int nvar = 0;
  std::vector<std::array<int, 4>> e;
  std::vector<double> c;
  double eval(const double* x) const;
  PPoly deriv(int var) const;
};
std::vector<std::array<int, 4>> graded_monomials(int nvar, int deg);

// Dubiner-type basis on T_E evaluated pointwise (psi_0 = 1, the others
// orthonormal in L2(T_E)); index order: total degree, then the exponent of
// the last collapsed direction.
struct Dubiner {
  int d = 2, M = 1, n = 0;
  std::vector<double> norm;              // normalisation per function
  std::vector<std::array<int, 3>> pqr;   // Jacobi indices
  std::vector<PPoly> power;              // power-form coefficients (for derivatives)
  // three-term recurrence coefficients of the homogenised Jacobi polynomials
  // P^(alpha,0), per integer alpha and degree k >= 2: p_k = (c2 s + c3 u)
  // p_{k-1} - c4 s^2 p_{k-2}
  std::vector<std::array<double, 3>> rec;  // [(alpha * (M + 1) + k)]
  void init(int d, int M);
  void eval(const double* xi, double* out) const;  // out[n]
 private:
  void jacobi_seq(int alpha, int nmax, double u, double s, double* p) const;
};

// Reference data of one (d, M).
struct RefElem {
  int d = 2, M = 1;
  int Mc = 0, ne = 0, L = 0, L0 = 0, L1 = 0;
  int nqs = 0, nqt = 0, ncode = 0;
  Dubiner psi;
  std::vector<std::array<double, 3>> lattice;  // Mc spatial lattice nodes
  std::vector<std::array<double, 4>> stnode;   // L space-time nodes (xi.., tau in [3])
  // E[n][l-1] = psi_l(lattice n), l = 1..Mc-1
  std::vector<double> E;
  // Sigma restricted to l, m >= 1: (Mc-1) x (Mc-1)
  std::vector<double> Sigma;
  // predictor: q1 = C0 q0 - dt sum_e P_e G_e
  std::vector<double> C0;  // L1 x L0
  std::vector<double> P;   // d x L1 x L
  // face quadrature: code -> table[t][q][l]; weights normalised to 1
  std::vector<double> ftab;  // ncode x nqt x nqs x L
  // integrals of the nodal basis over the face (per |f|) and [0,1]:
  // fint[code][l] = sum_t sum_q wt[t] wq[q] theta_l(point), the tables of
  // the quadrature-free flux
  std::vector<double> fint;  // ncode x L
  std::vector<double> wq, wt;
  std::vector<double> tq;    // time points
  std::vector<double> chi;   // face points (d = 2: parameter along the edge)
  std::vector<double> chi3;  // face points (d = 3: (chi1, chi2) pairs on the triangle)
  // moving-mesh predictor (Secs. 2.2-2.3):
  //   Dxi[(e L + n) L + l] = d theta_l / d xi_e at node n;
  //   Gal = (K_tau^1)^-1 M^1, L1 x L, the Galerkin operator of Eqs. (CGfinal)
  //     and (ODEfinal) (q^1 = C0 q^0 - dt Gal H, x^1 = C0 x^0 + dt Gal V);
  //   Wv[v L + l] = int_0^1 theta_l(reference vertex v, tau) dtau (Eq. NodesVel).
  std::vector<double> Dxi, Gal, Wv;
  void init(int d, int M);
};

// Face code of an ordered tuple of local vertex indices (the face's
// vertices sorted by global vertex id), and its local face index.
int face_code(int d, const int* ordered_local, int* local_face);

// Small dense helpers.
bool lu_solve(int n, std::vector<double> A, std::vector<double>& B, int nrhs);

}  // namespace cw
