// Per-cell reconstruction setup on fixed meshes (Sec. 2.1): the paper
// precomputes and inverts the least-squares matrices once for Eulerian runs;
// this does the same in FP64 on the host with one thread per core.
//
// Stencil rule (the paper fills S_i^0 "recursively with neighbours" without
// fixing the order): breadth-first layers over face neighbours; inside a
// layer candidates are ranked by the squared distance between the
// minimum-image barycentre and b_i, then by that barycentre's coordinates,
// then by the caller's cell index; the first n_e - 1 of the ranked sequence
// join cell i.  The sequence is continued two layers further for the
// sectorial stencils: sector s takes the first d cells whose barycentre
// lies in the open cone at vertex s through the opposite face (strictly
// positive barycentric coordinates for all vertices but s); a sector with
// fewer cells, or with collinear / coplanar barycentres, is dropped.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>

#include "../../include/cweno.h"
#include "host.h"

namespace cw {

namespace {

struct Ctx {
  const MeshHost* m;
  const RefElem* re;
};

inline const double* vtx(const MeshHost& m, int32_t c, int k) { return &m.X[((size_t)c * (m.d + 1) + k) * 3]; }

void jac_inv(const MeshHost& m, int32_t c, double Ji[3][3]) {
  int d = m.d;
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int a = 0; a < d; ++a)
    for (int k = 0; k < d; ++k) J[a][k] = vtx(m, c, k + 1)[a] - vtx(m, c, 0)[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Ji[a][b] = 0.0;
  if (d == 2) {
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det;
    Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det;
    Ji[1][1] = J[0][0] / det;
    return;
  }
  double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
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

// shift that brings cell j next to cell i (minimum image of barycentres)
void shift_of(const MeshHost& m, int32_t i, int32_t j, double* s) {
  for (int a = 0; a < 3; ++a) {
    s[a] = 0.0;
    if (a < m.d && m.per[a]) s[a] = m.Lper[a] * std::nearbyint((m.bary[i * 3 + a] - m.bary[j * 3 + a]) / m.Lper[a]);
  }
}

struct Cand {
  long long k[4];
  int32_t user;
  int32_t cell;
  bool operator<(const Cand& o) const {
    for (int q = 0; q < 4; ++q)
      if (k[q] != o.k[q]) return k[q] < o.k[q];
    return user < o.user;
  }
};

// per-thread scratch of the stencil search: mark[j] == i flags cell j as
// reached from cell i (each cell is searched once, so no reset is needed)
struct Scratch {
  std::vector<int32_t> mark, front, next;
  std::vector<Cand> cand;
};

// ranked BFS sequence (cell i excluded); returns false if the mesh is too small
bool ranked_sequence(const MeshHost& m, int32_t i, int need, std::vector<int32_t>& seq, Scratch& sc) {
  const int nvx = m.d + 1;
  seq.clear();
  if ((int64_t)sc.mark.size() != m.nc) sc.mark.assign(m.nc, -1);
  sc.mark[i] = i;
  std::vector<int32_t>& front = sc.front;
  std::vector<int32_t>& next = sc.next;
  std::vector<Cand>& cand = sc.cand;
  front.assign(1, i);
  const double tol = 1e-9 * m.qscale;
  int done_layer = -1;
  for (int layer = 1;; ++layer) {
    next.clear();
    for (int32_t c : front)
      for (int k = 0; k < nvx; ++k) {
        int32_t j = m.nbr[(size_t)c * nvx + k];
        if (j < 0 || sc.mark[j] == i) continue;
        sc.mark[j] = i;
        next.push_back(j);
      }
    if (next.empty()) break;
    cand.clear();
    for (int32_t j : next) {
      double s[3];
      shift_of(m, i, j, s);
      double b[3] = {0, 0, 0}, d2 = 0.0;
      for (int a = 0; a < m.d; ++a) {
        b[a] = m.bary[j * 3 + a] + s[a];
        double df = b[a] - m.bary[i * 3 + a];
        d2 += df * df;
      }
      Cand cd;
      cd.k[0] = std::llround(d2 / (tol * m.qscale));
      for (int a = 0; a < 3; ++a) cd.k[1 + a] = std::llround(b[a] / tol);
      cd.user = m.perm[j];
      cd.cell = j;
      cand.push_back(cd);
    }
    std::sort(cand.begin(), cand.end());
    for (const Cand& cd : cand) seq.push_back(cd.cell);
    if (done_layer < 0 && (int)seq.size() + 1 >= need) done_layer = layer;
    if (done_layer >= 0 && layer >= done_layer + 2) break;
    front.swap(next);
  }
  return (int)seq.size() + 1 >= need;
}

// reference coordinates (in cell i) of physical point x
void to_ref(const MeshHost& m, int32_t i, const double Ji[3][3], const double* x, double* xi) {
  const double* X0 = vtx(m, i, 0);
  for (int a = 0; a < 3; ++a) xi[a] = 0.0;
  for (int a = 0; a < m.d; ++a)
    for (int b = 0; b < m.d; ++b) xi[a] += Ji[a][b] * (x[b] - X0[b]);
}

// Pseudo-inverse of A (m x n, m >= n, row-major) by modified Gram-Schmidt QR
// with one reorthogonalisation pass: pinv = R^{-1} Q^T (n x m).
bool mgs_pinv(int mrow, int n, const std::vector<double>& A, std::vector<double>& pinv, std::vector<double>& Qm,
              std::vector<double>& Rm) {
  Qm = A;
  Rm.assign((size_t)n * n, 0.0);
  for (int k = 0; k < n; ++k) {
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < k; ++j) {
        double s = 0.0;
        for (int r = 0; r < mrow; ++r) s += Qm[r * n + j] * Qm[r * n + k];
        Rm[j * n + k] += s;
        for (int r = 0; r < mrow; ++r) Qm[r * n + k] -= s * Qm[r * n + j];
      }
    double nn = 0.0;
    for (int r = 0; r < mrow; ++r) nn += Qm[r * n + k] * Qm[r * n + k];
    nn = std::sqrt(nn);
    Rm[k * n + k] = nn;
    if (nn == 0.0) return false;
    for (int r = 0; r < mrow; ++r) Qm[r * n + k] /= nn;
  }
  double dmax = 0.0;
  for (int k = 0; k < n; ++k) dmax = std::max(dmax, std::fabs(Rm[k * n + k]));
  for (int k = 0; k < n; ++k)
    if (std::fabs(Rm[k * n + k]) <= 1e-13 * dmax) return false;
  // pinv = R^{-1} Q^T: back-substitute column by column of Q^T
  pinv.assign((size_t)n * mrow, 0.0);
  for (int r = 0; r < mrow; ++r)
    for (int k = n - 1; k >= 0; --k) {
      double s = Qm[r * n + k];
      for (int j = k + 1; j < n; ++j) s -= Rm[k * n + j] * pinv[j * mrow + r];
      pinv[k * mrow + r] = s / Rm[k * n + k];
    }
  return true;
}

bool inv_small(int d, const double* B, double* Bi) {
  if (d == 2) {
    double det = B[0] * B[3] - B[1] * B[2];
    if (det == 0.0) return false;
    Bi[0] = B[3] / det;
    Bi[1] = -B[1] / det;
    Bi[2] = -B[2] / det;
    Bi[3] = B[0] / det;
    return true;
  }
  double c00 = B[4] * B[8] - B[5] * B[7], c01 = B[5] * B[6] - B[3] * B[8], c02 = B[3] * B[7] - B[4] * B[6];
  double det = B[0] * c00 + B[1] * c01 + B[2] * c02;
  if (det == 0.0) return false;
  Bi[0] = c00 / det;
  Bi[3] = c01 / det;
  Bi[6] = c02 / det;
  Bi[1] = (B[2] * B[7] - B[1] * B[8]) / det;
  Bi[4] = (B[0] * B[8] - B[2] * B[6]) / det;
  Bi[7] = (B[1] * B[6] - B[0] * B[7]) / det;
  Bi[2] = (B[1] * B[5] - B[2] * B[4]) / det;
  Bi[5] = (B[2] * B[3] - B[0] * B[5]) / det;
  Bi[8] = (B[0] * B[4] - B[1] * B[3]) / det;
  return true;
}

double det_small(int d, const double* B) {
  if (d == 2) return B[0] * B[3] - B[1] * B[2];
  return B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) + B[2] * (B[3] * B[7] - B[4] * B[6]);
}

}  // namespace

int build_cell_setup(const MeshHost& m, const RefElem& re, CellSetup& cs, std::string& err, int nthreads,
                     bool with_lsq) {
  const int d = m.d, nvx = d + 1, ne = re.ne, Mc = re.Mc, M = re.M;
  const int64_t nc = m.nc;
  cs = CellSetup();
  cs.ne = ne;
  cs.Mc = Mc;
  cs.d = d;
  cs.sten.assign((size_t)nc * (ne - 1), -1);
  if (with_lsq) cs.R.assign((size_t)nc * (Mc - 1) * (ne - 1), 0.0);
  cs.sec.assign((size_t)nc * nvx * d, -1);
  cs.Binv.assign((size_t)nc * nvx * d * d, 0.0);
  cs.nsec.assign(nc, 0);
  cs.Jinv.assign((size_t)nc * d * d, 0.0);
  // quadrature exact to degree M for the stencil averages
  SimplexQuad Q = simplex_quad(d, (M + 2) / 2);
  double wsum = 0.0;
  for (double w : Q.w) wsum += w;
  std::atomic<int64_t> bad(-1);
  std::atomic<int> badkind(0);
  auto work = [&](int64_t c0, int64_t c1) {
    std::vector<int32_t> seq;
    std::vector<double> A((size_t)(ne - 1) * (Mc - 1)), pinv, Qm, Rm;
    std::vector<std::array<double, 4>> lamseq;  // barycentric coordinates of the sequence's barycentres
    std::vector<std::array<double, 3>> xiseq;   // and their reference coordinates
    Scratch sc;
    double psi[64];
    for (int64_t ii = c0; ii < c1; ++ii) {
      if (bad.load() >= 0) return;
      int32_t i = (int32_t)ii;
      if (!ranked_sequence(m, i, ne, seq, sc)) {
        bad = ii;
        badkind = 1;
        return;
      }
      double Ji[3][3];
      jac_inv(m, i, Ji);
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) cs.Jinv[(size_t)i * d * d + a * d + b] = Ji[a][b];
      for (int k = 0; k < ne - 1; ++k) cs.sten[(size_t)i * (ne - 1) + k] = seq[k];
      // least-squares rows: averages of psi_l (l >= 1) over each stencil cell
      for (int r = 0; r < (with_lsq ? ne - 1 : 0); ++r) {
        int32_t j = seq[r];
        double s[3];
        shift_of(m, i, j, s);
        double acc[64];
        for (int l = 0; l < Mc; ++l) acc[l] = 0.0;
        const double* Xj0 = vtx(m, j, 0);
        for (size_t g = 0; g < Q.w.size(); ++g) {
          double x[3] = {0, 0, 0};
          for (int a = 0; a < d; ++a) {
            x[a] = Xj0[a] + s[a];
            for (int k = 0; k < d; ++k) x[a] += Q.x[g][k] * (vtx(m, j, k + 1)[a] - Xj0[a]);
          }
          double xi[3];
          to_ref(m, i, Ji, x, xi);
          re.psi.eval(xi, psi);
          for (int l = 1; l < Mc; ++l) acc[l] += Q.w[g] * psi[l];
        }
        for (int l = 1; l < Mc; ++l) A[(size_t)r * (Mc - 1) + (l - 1)] = acc[l] / wsum;
      }
      if (with_lsq && !mgs_pinv(ne - 1, Mc - 1, A, pinv, Qm, Rm)) {
        bad = ii;
        badkind = 2;
        return;
      }
      if (with_lsq)
        std::memcpy(&cs.R[(size_t)i * (Mc - 1) * (ne - 1)], pinv.data(), sizeof(double) * (Mc - 1) * (ne - 1));
      // sectors: barycentric coordinates of every sequence cell's
      // (minimum-image) barycentre in cell i, once
      lamseq.resize(seq.size());
      xiseq.resize(seq.size());
      for (size_t q = 0; q < seq.size(); ++q) {
        const int32_t j = seq[q];
        double s[3];
        shift_of(m, i, j, s);
        double b[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) b[a] = m.bary[j * 3 + a] + s[a];
        double xi[3] = {0, 0, 0};
        to_ref(m, i, Ji, b, xi);
        lamseq[q][0] = 1.0;
        for (int a = 0; a < d; ++a) {
          lamseq[q][a + 1] = xi[a];
          lamseq[q][0] -= xi[a];
        }
        for (int a = 0; a < 3; ++a) xiseq[q][a] = xi[a];
      }
      int kept = 0;
      for (int sct = 0; sct < nvx; ++sct) {
        int32_t chosen[3];
        int nch = 0;
        double xib[3][3];
        for (size_t q = 0; q < seq.size(); ++q) {
          bool in = true;
          for (int v = 0; v < nvx; ++v)
            if (v != sct && !(lamseq[q][v] > 1e-9)) in = false;
          if (!in) continue;
          for (int a = 0; a < 3; ++a) xib[nch][a] = xiseq[q][a];
          chosen[nch++] = seq[q];
          if (nch == d) break;
        }
        if (nch < d) continue;
        // degeneracy test on the geometric matrix (xi(b_j) - barycentre of T_E)
        double G[9], B[9], Bi[9];
        for (int k = 0; k < d; ++k)
          for (int a = 0; a < d; ++a) G[k * d + a] = xib[k][a] - 1.0 / nvx;
        if (std::fabs(det_small(d, G)) < 1e-8) continue;
        // B[k][l] = psi_{1+l}(xi(b_jk)) (the degree-1 basis functions)
        for (int k = 0; k < d; ++k) {
          re.psi.eval(xib[k], psi);
          for (int l = 0; l < d; ++l) B[k * d + l] = psi[1 + l];
        }
        if (!inv_small(d, B, Bi)) continue;
        for (int k = 0; k < d; ++k) cs.sec[((size_t)i * nvx + sct) * d + k] = chosen[k];
        for (int q = 0; q < d * d; ++q) cs.Binv[((size_t)i * nvx + sct) * d * d + q] = Bi[q];
        ++kept;
      }
      cs.nsec[i] = (uint8_t)kept;
    }
  };
  int nt = std::max(1, nthreads);
  if (nc < 4096) nt = 1;
  std::vector<std::thread> th;
  int64_t chunk = (nc + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int64_t a = t * chunk, b = std::min<int64_t>(nc, a + chunk);
    if (a >= b) break;
    th.emplace_back(work, a, b);
  }
  for (auto& x : th) x.join();
  if (bad.load() >= 0) {
    int64_t c = m.perm[bad.load()];
    err = (badkind.load() == 1 ? "mesh too small for the central stencil at cell "
                               : "rank-deficient least-squares system at cell ") +
          std::to_string(c);
    return CWENO_EDEGENERATE;
  }
  return CWENO_OK;
}

}  // namespace cw
