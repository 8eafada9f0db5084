// Mesh creation: validation, periodic unwrapping, geometry (Eqs. xietaTransf,
// cellaverage), face matching (Neumann neighbours of Eq. PDEfinal), Morton
// reordering of the cells so that stencil gathers and face sweeps touch
// nearby memory.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/cweno.h"
#include "host.h"

namespace cw {

static double det_dd(int d, const double J[3][3]) {
  if (d == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

static uint64_t spread2(uint64_t x) {  // 31 bits -> every other bit
  x &= 0x7fffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

static uint64_t spread3(uint64_t x) {  // 21 bits -> every third bit
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

int build_mesh(int d, int64_t nv, const double* xyz, int64_t nc, const int32_t* cells, const double* period,
               MeshHost& m, std::string& err) {
  if (d != 2 && d != 3) {
    err = "dim must be 2 or 3";
    return CWENO_EINVAL;
  }
  if (nv <= 0 || nc <= 0 || !xyz || !cells) {
    err = "empty mesh or null pointer";
    return CWENO_EINVAL;
  }
  if (nc > 0x3fffffff) {
    err = "too many cells (limit 2^30)";
    return CWENO_EINVAL;
  }
  const int nvx = d + 1;
  m = MeshHost();
  m.d = d;
  m.nv = nv;
  m.nc = nc;
  m.xyz.assign(xyz, xyz + nv * d);
  for (int a = 0; a < d; ++a)
    if (period && period[a] > 0) {
      m.per[a] = true;
      m.Lper[a] = period[a];
    }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < nv; ++v)
    for (int a = 0; a < d; ++a) {
      double x = xyz[v * d + a];
      if (!std::isfinite(x)) {
        err = "non-finite vertex coordinate";
        return CWENO_EINVAL;
      }
      lo[a] = std::min(lo[a], x);
      hi[a] = std::max(hi[a], x);
    }
  m.qscale = 0.0;
  for (int a = 0; a < d; ++a) m.qscale = std::max(m.qscale, hi[a] - lo[a]);
  // unwrap + geometry in user order
  std::vector<double> Xu((size_t)nc * nvx * 3, 0.0), volu(nc), baryu((size_t)nc * 3, 0.0);
  for (int64_t c = 0; c < nc; ++c) {
    for (int k = 0; k < nvx; ++k) {
      int64_t v = cells[c * nvx + k];
      if (v < 0 || v >= nv) {
        err = "vertex index out of range in cell " + std::to_string(c);
        return CWENO_EINVAL;
      }
      for (int a = 0; a < d; ++a) {
        double x = xyz[v * d + a];
        if (m.per[a] && k > 0) {
          double x0 = xyz[(int64_t)cells[c * nvx] * d + a];
          x += m.Lper[a] * std::nearbyint((x0 - x) / m.Lper[a]);
        }
        Xu[((size_t)c * nvx + k) * 3 + a] = x;
      }
    }
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < d; ++a)
      for (int k = 0; k < d; ++k) J[a][k] = Xu[((size_t)c * nvx + k + 1) * 3 + a] - Xu[((size_t)c * nvx) * 3 + a];
    double det = det_dd(d, J);
    volu[c] = det / (d == 2 ? 2.0 : 6.0);
    if (!(volu[c] > 0.0)) {
      err = "cell " + std::to_string(c) + " has non-positive volume";
      return CWENO_EDEGENERATE;
    }
    for (int a = 0; a < d; ++a) {
      double s = 0.0;
      for (int k = 0; k < nvx; ++k) s += Xu[((size_t)c * nvx + k) * 3 + a];
      baryu[c * 3 + a] = s / nvx;
    }
  }
  // Morton order of barycentres
  double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
  for (int64_t c = 0; c < nc; ++c)
    for (int a = 0; a < d; ++a) {
      blo[a] = std::min(blo[a], baryu[c * 3 + a]);
      bhi[a] = std::max(bhi[a], baryu[c * 3 + a]);
    }
  std::vector<std::pair<uint64_t, int32_t>> key(nc);
  const double qmax = (d == 2) ? 2147483647.0 : 2097151.0;
  for (int64_t c = 0; c < nc; ++c) {
    uint64_t code = 0;
    for (int a = 0; a < d; ++a) {
      double ext = bhi[a] - blo[a];
      double u = ext > 0 ? (baryu[c * 3 + a] - blo[a]) / ext : 0.0;
      uint64_t qv = (uint64_t)std::min(qmax, std::max(0.0, std::floor(u * qmax)));
      code |= (d == 2 ? spread2(qv) : spread3(qv)) << a;
    }
    key[c] = {code, (int32_t)c};
  }
  std::sort(key.begin(), key.end());
  m.perm.resize(nc);
  m.iperm.resize(nc);
  for (int64_t i = 0; i < nc; ++i) {
    m.perm[i] = key[i].second;
    m.iperm[key[i].second] = (int32_t)i;
  }
  m.X.assign((size_t)nc * nvx * 3, 0.0);
  m.vol.resize(nc);
  m.bary.assign((size_t)nc * 3, 0.0);
  m.gv.resize((size_t)nc * nvx);
  for (int64_t i = 0; i < nc; ++i) {
    int64_t c = m.perm[i];
    std::memcpy(&m.X[(size_t)i * nvx * 3], &Xu[(size_t)c * nvx * 3], sizeof(double) * nvx * 3);
    m.vol[i] = volu[c];
    for (int a = 0; a < 3; ++a) m.bary[i * 3 + a] = baryu[c * 3 + a];
    for (int k = 0; k < nvx; ++k) m.gv[i * nvx + k] = cells[c * nvx + k];
  }
  // face matching by sorted global vertex ids
  struct FK {
    int64_t v[3];
    int32_t cell;
    int8_t face;
  };
  std::vector<FK> fk((size_t)nc * nvx);
  for (int64_t i = 0; i < nc; ++i)
    for (int k = 0; k < nvx; ++k) {
      FK& f = fk[i * nvx + k];
      int n = 0;
      for (int q = 0; q < nvx; ++q)
        if (q != k) f.v[n++] = m.gv[i * nvx + q];
      if (d == 2) f.v[2] = -1;
      std::sort(f.v, f.v + d);
      f.cell = (int32_t)i;
      f.face = (int8_t)k;
    }
  std::sort(fk.begin(), fk.end(), [](const FK& a, const FK& b) {
    if (a.v[0] != b.v[0]) return a.v[0] < b.v[0];
    if (a.v[1] != b.v[1]) return a.v[1] < b.v[1];
    if (a.v[2] != b.v[2]) return a.v[2] < b.v[2];
    return a.cell < b.cell;
  });
  m.nbr.assign((size_t)nc * nvx, -1);
  std::vector<int8_t> nbrf((size_t)nc * nvx, -1);
  for (size_t s = 0; s < fk.size();) {
    size_t e = s + 1;
    while (e < fk.size() && fk[e].v[0] == fk[s].v[0] && fk[e].v[1] == fk[s].v[1] && fk[e].v[2] == fk[s].v[2]) ++e;
    if (e - s > 2) {
      err = "a face is shared by more than two cells";
      return CWENO_EINVAL;
    }
    if (e - s == 2) {
      if (fk[s].cell == fk[s + 1].cell) {
        err = "a cell meets itself across a face (mesh too small for its period)";
        return CWENO_EINVAL;
      }
      m.nbr[(size_t)fk[s].cell * nvx + fk[s].face] = fk[s + 1].cell;
      m.nbr[(size_t)fk[s + 1].cell * nvx + fk[s + 1].face] = fk[s].cell;
      nbrf[(size_t)fk[s].cell * nvx + fk[s].face] = fk[s + 1].face;
      nbrf[(size_t)fk[s + 1].cell * nvx + fk[s + 1].face] = fk[s].face;
    }
    s = e;
  }
  // face list ordered by its L cell
  m.cellface.assign((size_t)nc * nvx, -1);
  m.hsize.resize(nc);
  for (int64_t i = 0; i < nc; ++i) {
    double surf = 0.0;
    for (int k = 0; k < nvx; ++k) {
      int32_t j = m.nbr[i * nvx + k];
      // face geometry from cell i
      int lv[3], n = 0;
      for (int q = 0; q < nvx; ++q)
        if (q != k) lv[n++] = q;
      const double* P0 = &m.X[((size_t)i * nvx + lv[0]) * 3];
      const double* P1 = &m.X[((size_t)i * nvx + lv[1]) * 3];
      double nrm[3] = {0, 0, 0}, area;
      if (d == 2) {
        double tx = P1[0] - P0[0], ty = P1[1] - P0[1];
        area = std::sqrt(tx * tx + ty * ty);
        nrm[0] = ty / area;
        nrm[1] = -tx / area;
      } else {
        const double* P2 = &m.X[((size_t)i * nvx + lv[2]) * 3];
        double u[3], w[3];
        for (int a = 0; a < 3; ++a) {
          u[a] = P1[a] - P0[a];
          w[a] = P2[a] - P0[a];
        }
        double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        double nn = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        area = 0.5 * nn;
        for (int a = 0; a < 3; ++a) nrm[a] = cr[a] / nn;
      }
      surf += area;
      double dot = 0.0;
      for (int a = 0; a < d; ++a) dot += nrm[a] * (P0[a] - m.bary[i * 3 + a]);
      if (dot < 0)
        for (int a = 0; a < 3; ++a) nrm[a] = -nrm[a];
      if (j >= 0 && j < i) continue;  // owned by the lower-index neighbour
      if (j == i) continue;
      int32_t f = (int32_t)m.fL.size();
      m.fL.push_back((int32_t)i);
      m.fR.push_back(j);
      for (int a = 0; a < 3; ++a) m.fn.push_back(nrm[a]);
      m.farea.push_back(area);
      // face vertices in ascending global id -> ordered local indices on both sides
      int64_t g[3];
      for (int r = 0; r < d; ++r) g[r] = m.gv[i * nvx + lv[r]];
      std::sort(g, g + d);
      auto codeof = [&](int32_t cell) {
        int ol[3];
        for (int r = 0; r < d; ++r) {
          ol[r] = -1;
          for (int q = 0; q < nvx; ++q)
            if (m.gv[(size_t)cell * nvx + q] == g[r]) ol[r] = q;
        }
        int lf;
        return (uint8_t)face_code(d, ol, &lf);
      };
      m.codeL.push_back(codeof((int32_t)i));
      m.codeR.push_back(j >= 0 ? codeof(j) : 0);
      m.cellface[i * nvx + k] = f * 2;
      if (j >= 0) {
        int kj = nbrf[(size_t)i * nvx + k];
        m.cellface[(size_t)j * nvx + kj] = f * 2 + 1;
      } else {
        m.nbnd++;
      }
    }
    m.hsize[i] = 2.0 * d * m.vol[i] / surf;
  }
  m.nf = (int64_t)m.fL.size();
  return CWENO_OK;
}

}  // namespace cw
