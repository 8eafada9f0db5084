// C ABI: handles, error reporting, device uploads and the step sequence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cweno.h"
#include "ale.h"
#include "api_internal.h"
#include "layout.h"
#include "host.h"
#include "ops.h"
#include "refelem.h"

namespace cw {

static thread_local std::string g_err;
// host threads used by one setup (the serving loop lowers it for its workers)
thread_local int g_setup_threads = 0;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return CWENO_ECUDA;
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Reference tables are universal per (d, M): built once per process.
static std::mutex g_ref_mu;
static std::map<int, std::unique_ptr<RefElem>> g_ref;

const RefElem& ref_elem(int d, int M) {
  std::lock_guard<std::mutex> lk(g_ref_mu);
  int key = d * 16 + M;
  auto it = g_ref.find(key);
  if (it != g_ref.end()) return *it->second;
  std::unique_ptr<RefElem> r(new RefElem());
  r->init(d, M);
  const RefElem& out = *r;
  g_ref[key] = std::move(r);
  return out;
}

// Device bytes cweno_setup allocates for a mesh of nc cells and nf faces.
size_t footprint_estimate(int d, int64_t nc, int64_t nf, int order, int pde, int precision) {
  const int M = order - 1;
  const int Mc = (d == 2) ? (M + 1) * (M + 2) / 2 : (M + 1) * (M + 2) * (M + 3) / 6;
  const int L = (d == 2) ? (M + 1) * (M + 2) * (M + 3) / 6 : (M + 1) * (M + 2) * (M + 3) * (M + 4) / 24;
  const int ne = d * Mc, nvx = d + 1, nv = (pde == CWENO_MHD_GLM) ? 9 : d + 2;
  const size_t es = precision == CWENO_FP32_MIXED ? 4 : 8;
  size_t b = 0;
  b += 8 * nc * nv * 2;                                     // Q, staging
  if (precision == CWENO_FP32_MIXED) b += 8 * nc * ((nv + 1) & ~1);  // hi, lo pairs
  b += 4 * nc + 4 * nc * (ne - 1) + 16 * nc * ((ne + 2) / 4);        // ids, ids in vectors
  b += 16 * nc * (((ne - 1) * (Mc - 1) * es + 15) / 16);             // R_i in vectors
  b += 4 * nc * nvx * d + es * nc * nvx * d * d + nc + es * nc * d * d;
  b += es * nc * nv * L;                                    // q_hat
  b += nf * (8 + 2 + es * d + 8 * d + 8 + 8 * nv);          // faces + G
  b += 4 * nc * nvx + 16 * nc;                              // cell->face, 1/|T|, h
  // reference tables: face basis values per face code, time and space point;
  // per-cell tables (E, Sigma, C0 E, P_e) where they are stored beside them
  const size_t ncode = d == 2 ? 6 : 24, nqs = d == 2 ? M + 1 : (M + 1) * (M + 1);
  b += es * (ncode * (M + 1) * nqs * (L + 3) + ncode * (L + 3) + 256);
  b += es * ((size_t)Mc * (Mc - 1) + (size_t)(Mc - 1) * (Mc - 1) + (size_t)(L - Mc) * (Mc - 1) +
             (size_t)d * (L - Mc) * L) + 4096;
  return b + (size_t)64 * 1024;                             // allocation granularity slack
}

}  // namespace cw

using namespace cw;

struct cweno_mesh {
  MeshHost m;
};

// ---------------------------------------------------------------- helpers
// Stream-ordered allocations on the solver's stream: no device-wide
// synchronisation when solvers come and go while others run (serving).
static int dev_alloc(cweno_solver* s, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CWENO_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  s->allocs.push_back(*p);
  s->bytes += bytes;
  return CWENO_OK;
}

template <typename TV>
static int upload(cweno_solver* s, const std::vector<TV>& h, const void** out) {
  void* p = nullptr;
  int rc = dev_alloc(s, &p, h.size() * sizeof(TV));
  if (rc) return rc;
  if (!h.empty()) {
    // pageable source: staged before the call returns, so h may be released
    cudaError_t e = cudaMemcpyAsync(p, h.data(), h.size() * sizeof(TV), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload");
  }
  *out = p;
  return CWENO_OK;
}

// double matrix in AoS-by-cell (nc x K) -> SoA (K x nc) of type TV
template <typename TV>
static std::vector<TV> soa(const std::vector<double>& a, int64_t nc, int K) {
  std::vector<TV> o((size_t)nc * K);
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < K; ++k) o[(size_t)k * nc + c] = (TV)a[(size_t)c * K + k];
  return o;
}
template <typename TI>
static std::vector<TI> soa_i(const std::vector<TI>& a, int64_t nc, int K) {
  std::vector<TI> o((size_t)nc * K);
  for (int64_t c = 0; c < nc; ++c)
    for (int k = 0; k < K; ++k) o[(size_t)k * nc + c] = a[(size_t)c * K + k];
  return o;
}

static int upload_real(cweno_solver* s, const std::vector<double>& a, int64_t n, int K, const void** out) {
  if (s->prec == CWENO_FP32_MIXED) {
    std::vector<float> v = soa<float>(a, n, K);
    return upload(s, v, out);
  }
  std::vector<double> v = soa<double>(a, n, K);
  return upload(s, v, out);
}

extern "C" {

void cweno_default_params(cweno_params* p, int dim, int pde) {
  if (!p) return;
  p->eps = 1e-14;
  p->r = 4.0;
  p->lambda0 = 1e5;
  p->lambda_s = 1.0;
  p->gamma = pde == CWENO_MHD_GLM ? 5.0 / 3.0 : 1.4;
  p->c_h = 2.0;
  p->cfl = dim == 3 ? 1.0 / 3.0 : 0.5;
  p->picard_iters = 0;
  p->linear_weights = 0;
  p->positivity = 1;
  p->flux = CWENO_FLUX_RUSANOV;
  p->mesh_motion = CWENO_MOTION_FIXED;
}

const char* cweno_last_error(void) { return g_err.c_str(); }

int cweno_nvars(int dim, int pde) { return pde == CWENO_MHD_GLM ? 9 : dim + 2; }

int cweno_mesh_create(int dim, int64_t nv, const double* xyz, int64_t nc, const int32_t* cells, const double* period,
                      cweno_mesh** out) {
  if (!out) return fail(CWENO_EINVAL, "null output handle");
  *out = nullptr;
  std::unique_ptr<cweno_mesh> m(new cweno_mesh());
  std::string err;
  int rc = build_mesh(dim, nv, xyz, nc, cells, period, m->m, err);
  if (rc) return fail(rc, err);
  *out = m.release();
  return CWENO_OK;
}

void cweno_mesh_destroy(cweno_mesh* m) { delete m; }

int cweno_mesh_info(const cweno_mesh* m, int64_t* ncells, int64_t* nfaces, int64_t* nboundary) {
  if (!m) return fail(CWENO_EINVAL, "null mesh");
  if (ncells) *ncells = m->m.nc;
  if (nfaces) *nfaces = m->m.nf;
  if (nboundary) *nboundary = m->m.nbnd;
  return CWENO_OK;
}

int cweno_mesh_stencils(const cweno_mesh* mesh, int order, int32_t* S0, int32_t* sec) {
  if (!mesh || !S0 || !sec) return fail(CWENO_EINVAL, "null argument");
  const MeshHost& m = mesh->m;
  if (order < 2 || order > 5) return fail(CWENO_EINVAL, "order must be 2..5");
  const RefElem& re = ref_elem(m.d, order - 1);
  CellSetup cs;
  std::string err;
  int rc = build_cell_setup(m, re, cs, err, (int)std::max(1u, std::thread::hardware_concurrency()), false);
  if (rc) return fail(rc, err);
  const int ne = re.ne, d = m.d, nvx = d + 1;
  for (int64_t i = 0; i < m.nc; ++i) {
    int64_t u = m.perm[i];
    S0[u * ne] = (int32_t)u;
    for (int k = 0; k < ne - 1; ++k) S0[u * ne + 1 + k] = m.perm[cs.sten[(size_t)i * (ne - 1) + k]];
    for (int q = 0; q < nvx * d; ++q) {
      int32_t c = cs.sec[(size_t)i * nvx * d + q];
      sec[u * nvx * d + q] = c < 0 ? -1 : m.perm[c];
    }
  }
  return CWENO_OK;
}

int cweno_solver_stencils(cweno_solver* s, int32_t* S0, int32_t* sec) {
  if (!s || !S0 || !sec) return fail(CWENO_EINVAL, "null argument");
  CK(cudaSetDevice(s->dev));
  const int64_t N = s->nc;
  const int ne = s->re->ne, d = s->dim, nvx = d + 1;
  std::vector<int32_t> st((size_t)N * (ne - 1)), sc((size_t)N * nvx * d), perm(N);
  CK(cudaMemcpyAsync(st.data(), s->ds.sten, sizeof(int32_t) * st.size(), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(sc.data(), s->ds.sec, sizeof(int32_t) * sc.size(), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(perm.data(), s->ds.perm, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  for (int64_t i = 0; i < N; ++i) {  // SoA, internal order -> caller's cells
    const int64_t u = perm[i];
    S0[u * ne] = (int32_t)u;
    for (int k = 0; k < ne - 1; ++k) S0[u * ne + 1 + k] = perm[st[(size_t)k * N + i]];
    for (int q = 0; q < nvx * d; ++q) {
      const int32_t c = sc[(size_t)q * N + i];
      sec[u * nvx * d + q] = c < 0 ? -1 : perm[c];
    }
  }
  return CWENO_OK;
}

void cweno_solver_destroy(cweno_solver* s) {
  if (!s) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(s->dev);
  cudaStreamSynchronize(s->stream);
  s->ale.reset();
  for (auto& kv : s->graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  for (auto& u : s->ev_used) {
    cudaEventDestroy(u.first.first);
    cudaEventDestroy(u.first.second);
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  for (void* p : s->allocs) cudaFreeAsync(p, s->stream);
  if (s->own_stream) {
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
  }
  if (cur >= 0) cudaSetDevice(cur);
  delete s;
}

int cweno_setup(const cweno_mesh* mesh, int order, int pde, int precision, const cweno_params* params, void* stream,
                cweno_solver** out) {
  if (!out) return fail(CWENO_EINVAL, "null output handle");
  *out = nullptr;
  if (!mesh) return fail(CWENO_EINVAL, "null mesh");
  const MeshHost& m = mesh->m;
  if (order < 2 || order > 5) return fail(CWENO_EINVAL, "order must be 2..5");
  if (pde != CWENO_EULER && pde != CWENO_MHD_GLM) return fail(CWENO_EINVAL, "unknown pde");
  if (order == 5 && pde != CWENO_EULER) return fail(CWENO_EINVAL, "order 5 is built for the Euler equations only");
  if (pde == CWENO_MHD_GLM && m.d != 2) return fail(CWENO_EINVAL, "MHD-GLM is built for 2D meshes only");
  if (precision != CWENO_FP64 && precision != CWENO_FP32_MIXED) return fail(CWENO_EINVAL, "unknown precision");
  cweno_params prm;
  cweno_default_params(&prm, m.d, pde);
  if (params) prm = *params;
  if (prm.r != 4.0) return fail(CWENO_EINVAL, "only r = 4 is built (Eq. weights2)");
  if (!(prm.eps > 0) || !(prm.lambda0 > 0) || !(prm.lambda_s > 0) || !(prm.gamma > 1.0) || !(prm.cfl > 0))
    return fail(CWENO_EINVAL, "bad scheme parameters");
  if (prm.flux != CWENO_FLUX_RUSANOV && prm.flux != CWENO_FLUX_OSHER && prm.flux != CWENO_FLUX_RUSANOV_QF)
    return fail(CWENO_EINVAL, "unknown flux");
  if (prm.flux == CWENO_FLUX_OSHER && pde != CWENO_EULER)
    return fail(CWENO_EINVAL, "the Osher-type flux is built for the Euler equations");
  if (prm.mesh_motion != CWENO_MOTION_FIXED && prm.mesh_motion != CWENO_MOTION_LAGRANGE &&
      prm.mesh_motion != CWENO_MOTION_STILL)
    return fail(CWENO_EINVAL, "unknown mesh motion");
  if (prm.mesh_motion != CWENO_MOTION_FIXED &&
      (pde != CWENO_EULER || order > 4 || prm.flux != CWENO_FLUX_RUSANOV))
    return fail(CWENO_EINVAL, "moving meshes are built for Euler, Rusanov flux, order 2..4");
  const int M = order - 1;
  std::unique_ptr<cweno_solver> s(new cweno_solver());
  s->dim = m.d;
  s->order = order;
  s->M = M;
  s->pde = pde;
  s->prec = precision;
  s->nv = cweno_nvars(m.d, pde);
  s->prm = prm;
  s->ph.gamma = prm.gamma;
  s->ph.ch = prm.c_h;
  s->ph.eps = prm.eps;
  s->ph.lam0 = prm.lambda0;
  s->ph.lams = prm.lambda_s;
  s->ph.niter = prm.picard_iters > 0 ? prm.picard_iters : M + 1;
  s->ph.linear_weights = prm.linear_weights;
  s->ph.positivity = prm.positivity;
  s->ph.flux = prm.flux;
  s->nc = m.nc;
  s->nf = m.nf;
  CK(cudaGetDevice(&s->dev));
  const RefElem& re = ref_elem(m.d, M);
  s->re = &re;
  if (pde == CWENO_EULER && m.d == 2) s->ops = make_ops_euler2(M, precision == CWENO_FP32_MIXED, re);
  else if (pde == CWENO_EULER && m.d == 3) s->ops = make_ops_euler3(M, precision == CWENO_FP32_MIXED, re);
  else s->ops = make_ops_mhd2(M, precision == CWENO_FP32_MIXED, re);
  if (!s->ops) return fail(CWENO_EINVAL, "configuration not built");
  std::string err;
  int rc = CWENO_OK;
  {
    // keep freed blocks in the device's default pool for reuse (serving)
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (s->dev >= 0 && s->dev < 64 && !done[s->dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, s->dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      done[s->dev] = true;
    }
  }
  if (stream) {
    s->stream = (cudaStream_t)stream;
    s->own_stream = false;
  } else {
    CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  const int64_t N = m.nc, F = m.nf;
  const int d = m.d, nvx = d + 1, nv = s->nv;
  DevState& ds = s->ds;
  ds.N = N;
  ds.F = F;
  ds.nv = nv;
  const size_t es = s->ops->elem_size();
  // state
  void* p = nullptr;
  if ((rc = dev_alloc(s.get(), &p, sizeof(double) * N * nv))) return rc;
  ds.Q = (double*)p;
  CK(cudaMemsetAsync(ds.Q, 0, sizeof(double) * N * nv, s->stream));
  if (precision == CWENO_FP32_MIXED) {
    const size_t pb = sizeof(float) * 2 * N * cw::pair_vars(nv);
    if ((rc = dev_alloc(s.get(), &p, pb))) return rc;
    ds.Qp = (float*)p;
    CK(cudaMemsetAsync(ds.Qp, 0, pb, s->stream));
  }
  if ((rc = upload(s.get(), m.perm, (const void**)&ds.perm))) return rc;
  if ((rc = upload(s.get(), m.iperm, (const void**)&ds.iperm))) return rc;
  {
    // Per-cell reconstruction data: stencils, sectors, inverse Jacobians and
    // sector inverses by the device search, then the least-squares inverses
    // R_i; the host search where the device one runs out of its per-thread
    // capacity.  Buffers in the kernels' layouts (layout.h, SoA).
    const int ne1 = re.ne - 1, nsv = cw::sten_vectors(ne1);
    void *bs = nullptr, *bs4 = nullptr, *bsec = nullptr, *bB = nullptr, *bns = nullptr, *bJ = nullptr, *bR = nullptr;
    const int vw = (int)(16 / es);
    const size_t rb = es * (size_t)N * vw * cw::r_vectors(ne1, re.Mc - 1, vw);
    if ((rc = dev_alloc(s.get(), &bs, sizeof(int32_t) * N * ne1))) return rc;
    if ((rc = dev_alloc(s.get(), &bs4, sizeof(int32_t) * N * nsv * 4))) return rc;
    if ((rc = dev_alloc(s.get(), &bsec, sizeof(int32_t) * N * nvx * d))) return rc;
    if ((rc = dev_alloc(s.get(), &bB, es * N * nvx * d * d))) return rc;
    if ((rc = dev_alloc(s.get(), &bns, N))) return rc;
    if ((rc = dev_alloc(s.get(), &bJ, es * N * d * d))) return rc;
    if ((rc = dev_alloc(s.get(), &bR, rb))) return rc;
    CK(cudaMemsetAsync(bsec, 0xff, sizeof(int32_t) * N * nvx * d, s->stream));
    CK(cudaMemsetAsync(bB, 0, es * N * nvx * d * d, s->stream));
    CK(cudaMemsetAsync(bns, 0, N, s->stream));
    CK(cudaMemsetAsync(bR, 0, rb, s->stream));  // the padding of the last R vector is zero
    ds.sten = (const int32_t*)bs;
    ds.sten4 = (const int32_t*)bs4;
    ds.sec = (const int32_t*)bsec;
    ds.Binv = bB;
    ds.nsec = (const uint8_t*)bns;
    ds.Jinv = bJ;
    ds.R = bR;
    rc = cell_setup_device(m, re, precision == CWENO_FP32_MIXED, s->stream, (int32_t*)bs, (int32_t*)bs4,
                           (int32_t*)bsec, bB, (uint8_t*)bns, bJ, bR, err);
    if (rc == kCellSetupOnHost) {
      CellSetup cs;
      const int nth = cw::g_setup_threads > 0 ? cw::g_setup_threads : (int)std::max(1u, std::thread::hardware_concurrency());
      if ((rc = build_cell_setup(m, re, cs, err, nth, false))) return fail(rc, err);
      std::vector<int32_t> s4((size_t)nsv * N * 4);
      for (int64_t i = 0; i < N; ++i)
        for (int r = 0; r < nsv * 4; ++r)
          s4[((size_t)(r / 4) * N + i) * 4 + r % 4] = r < ne1 ? cs.sten[(size_t)i * ne1 + r] : (int32_t)i;
      std::vector<int32_t> st = soa_i(cs.sten, N, ne1), sc = soa_i(cs.sec, N, nvx * d);
      CK(cudaMemcpyAsync(bs, st.data(), sizeof(int32_t) * st.size(), cudaMemcpyHostToDevice, s->stream));
      CK(cudaMemcpyAsync(bs4, s4.data(), sizeof(int32_t) * s4.size(), cudaMemcpyHostToDevice, s->stream));
      CK(cudaMemcpyAsync(bsec, sc.data(), sizeof(int32_t) * sc.size(), cudaMemcpyHostToDevice, s->stream));
      CK(cudaMemcpyAsync(bns, cs.nsec.data(), N, cudaMemcpyHostToDevice, s->stream));
      if (precision == CWENO_FP32_MIXED) {
        std::vector<float> b = soa<float>(cs.Binv, N, nvx * d * d), j = soa<float>(cs.Jinv, N, d * d);
        CK(cudaMemcpyAsync(bB, b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice, s->stream));
        CK(cudaMemcpyAsync(bJ, j.data(), sizeof(float) * j.size(), cudaMemcpyHostToDevice, s->stream));
      } else {
        std::vector<double> b = soa<double>(cs.Binv, N, nvx * d * d), j = soa<double>(cs.Jinv, N, d * d);
        CK(cudaMemcpyAsync(bB, b.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice, s->stream));
        CK(cudaMemcpyAsync(bJ, j.data(), sizeof(double) * j.size(), cudaMemcpyHostToDevice, s->stream));
      }
      rc = lsq_setup_device(m, re, (const int32_t*)bs, bR, precision == CWENO_FP32_MIXED, s->stream, err);
    }
    if (rc) return fail(rc, err);
  }
  if ((rc = dev_alloc(s.get(), &p, es * N * nv * re.L))) return rc;
  ds.qhat = p;
  if ((rc = upload(s.get(), m.fL, (const void**)&ds.fL))) return rc;
  if ((rc = upload(s.get(), m.fR, (const void**)&ds.fR))) return rc;
  if ((rc = upload(s.get(), m.codeL, (const void**)&ds.codeL))) return rc;
  if ((rc = upload(s.get(), m.codeR, (const void**)&ds.codeR))) return rc;
  {
    std::vector<double> fn((size_t)F * d);
    for (int64_t f = 0; f < F; ++f)
      for (int a = 0; a < d; ++a) fn[(size_t)f * d + a] = m.fn[f * 3 + a];
    if ((rc = upload_real(s.get(), fn, F, d, &ds.fn))) return rc;
    std::vector<double> fa((size_t)F * d);
    for (int64_t f = 0; f < F; ++f)
      for (int a = 0; a < d; ++a) fa[(size_t)f * d + a] = m.fn[f * 3 + a] * m.farea[f];
    std::vector<double> fa_soa = soa<double>(fa, F, d);
    if ((rc = upload(s.get(), fa_soa, (const void**)&ds.fa))) return rc;
    if ((rc = upload(s.get(), m.farea, (const void**)&ds.farea))) return rc;
  }
  if ((rc = dev_alloc(s.get(), &p, sizeof(double) * F * nv))) return rc;
  ds.G = (double*)p;
  {
    std::vector<unsigned char> tb(s->ops->table_bytes());
    s->ops->pack_tables(tb.data());
    if ((rc = upload(s.get(), tb, &ds.ftab))) return rc;
  }
  if ((rc = upload(s.get(), soa_i(m.cellface, N, nvx), (const void**)&ds.cellface))) return rc;
  {
    std::vector<double> iv(N);
    for (int64_t i = 0; i < N; ++i) iv[i] = 1.0 / m.vol[i];
    if ((rc = upload(s.get(), iv, (const void**)&ds.invvol))) return rc;
    if ((rc = upload(s.get(), m.hsize, (const void**)&ds.hsize))) return rc;
  }
  if ((rc = dev_alloc(s.get(), &p, sizeof(unsigned long long) * 4 + sizeof(double) + sizeof(int) * 2))) return rc;
  ds.dtmin = (unsigned long long*)p;
  ds.time = (double*)((char*)p + sizeof(unsigned long long) * 4);
  ds.status = (int*)((char*)p + sizeof(unsigned long long) * 4 + sizeof(double));
  {
    unsigned long long init[4] = {0x7ff0000000000000ull, 0x7ff0000000000000ull, 0x7ff0000000000000ull,
                                  0x7ff0000000000000ull};
    CK(cudaMemcpyAsync(ds.dtmin, init, sizeof(init), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemsetAsync(ds.time, 0, sizeof(double) + 2 * sizeof(int), s->stream));
  }
  if ((rc = dev_alloc(s.get(), &p, sizeof(double) * N * nv))) return rc;
  ds.stage = (double*)p;
  CK(s->ops->prepare());
  if (prm.mesh_motion != CWENO_MOTION_FIXED && (rc = ale_create(s.get(), m, err))) return fail(rc, err);
  CK(cudaStreamSynchronize(s->stream));
  *out = s.release();
  return CWENO_OK;
}

int cweno_solver_info(const cweno_solver* s, int* nvars, int* mcal_, int* ne, int* lcal, int64_t* ncells,
                      int64_t* nfaces) {
  if (!s) return fail(CWENO_EINVAL, "null solver");
  if (nvars) *nvars = s->nv;
  if (mcal_) *mcal_ = s->re->Mc;
  if (ne) *ne = s->re->ne;
  if (lcal) *lcal = s->re->L;
  if (ncells) *ncells = s->nc;
  if (nfaces) *nfaces = s->nf;
  return CWENO_OK;
}

int cweno_solver_footprint(const cweno_solver* s, size_t* bytes) {
  if (!s || !bytes) return fail(CWENO_EINVAL, "null argument");
  *bytes = s->bytes;
  return CWENO_OK;
}

// Page-locked host memory that is mapped into the device address space (every
// cudaHostAlloc/cudaHostRegister allocation under unified addressing): the
// state kernels then read or write it in place over the CPU-GPU link instead
// of going through a staging copy. Returns nullptr for pageable memory.
static void* mapped_host(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int cweno_set_state(cweno_solver* s, const double* Q, int on_device) {
  if (!s || !Q) return fail(CWENO_EINVAL, "null argument");
  CK(cudaSetDevice(s->dev));
  const double* src = Q;
  if (!on_device) {
    if (const void* dp = mapped_host(Q)) {
      src = (const double*)dp;
    } else {
      CK(cudaMemcpyAsync(s->ds.stage, Q, sizeof(double) * s->nc * s->nv, cudaMemcpyHostToDevice, s->stream));
      src = s->ds.stage;
    }
  }
  CK(s->ops->set_state(s->ds, src, s->stream));  // also resets dt bound, time, status
  if (s->ale) {
    int rc = ale_refresh(s);  // h of the current mesh for the bound below
    if (rc) return rc;
  }
  CK(s->ops->stable_dt(s->ds, s->ph, 0, s->stream));
  s->cur = 0;
  return CWENO_OK;
}

int cweno_get_state(cweno_solver* s, double* Q, int on_device) {
  if (!s || !Q) return fail(CWENO_EINVAL, "null argument");
  CK(cudaSetDevice(s->dev));
  if (on_device) {
    CK(s->ops->get_state(s->ds, Q, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return CWENO_OK;
  }
  if (void* dp = mapped_host(Q)) {
    CK(s->ops->get_state(s->ds, (double*)dp, s->stream));
  } else {
    CK(s->ops->get_state(s->ds, s->ds.stage, s->stream));
    CK(cudaMemcpyAsync(Q, s->ds.stage, sizeof(double) * s->nc * s->nv, cudaMemcpyDeviceToHost, s->stream));
  }
  CK(cudaStreamSynchronize(s->stream));
  return CWENO_OK;
}

static int ensure_out(cweno_solver* s, size_t bytes) {
  if (s->outbuf_bytes >= bytes) return CWENO_OK;
  void* p = nullptr;
  int rc = dev_alloc(s, &p, bytes);
  if (rc) return rc;
  s->outbuf = (double*)p;
  s->outbuf_bytes = bytes;
  return CWENO_OK;
}

int cweno_reconstruct(cweno_solver* s, double* w, int on_device) {
  if (!s || !w) return fail(CWENO_EINVAL, "null argument");
  CK(cudaSetDevice(s->dev));
  size_t bytes = sizeof(double) * s->nc * s->re->Mc * s->nv;
  double* dst = w;
  if (!on_device) {
    int rc = ensure_out(s, bytes);
    if (rc) return rc;
    dst = s->outbuf;
  }
  if (s->ale) {
    int rc = ale_refresh(s);
    if (rc) return rc;
  }
  CK(s->ops->reconstruct(s->ds, s->ph, dst, s->stream));
  if (!on_device) CK(cudaMemcpyAsync(w, dst, bytes, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return CWENO_OK;
}

int cweno_predictor(cweno_solver* s, double dt, double* qhat, int on_device) {
  if (!s || !qhat || !(dt > 0)) return fail(CWENO_EINVAL, "bad argument");
  if (s->ale) return fail(CWENO_EINVAL, "the predictor of a moving mesh is internal to its step");
  CK(cudaSetDevice(s->dev));
  size_t bytes = sizeof(double) * s->nc * s->re->L * s->nv;
  double* dst = qhat;
  if (!on_device) {
    int rc = ensure_out(s, bytes);
    if (rc) return rc;
    dst = s->outbuf;
  }
  DtArgs a;
  a.fixed = dt;
  a.cur = -1;
  CK(s->ops->rec_pred(s->ds, s->ph, a, s->stream));
  CK(s->ops->qhat_out(s->ds, dst, s->stream));
  if (!on_device) CK(cudaMemcpyAsync(qhat, dst, bytes, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return CWENO_OK;
}

int cweno_stable_dt(cweno_solver* s, double cfl, double* dt) {
  if (!s || !dt || !(cfl > 0)) return fail(CWENO_EINVAL, "bad argument");
  CK(cudaSetDevice(s->dev));
  if (s->ale) {
    int rc = ale_refresh(s);
    if (rc) return rc;
  }
  static const unsigned long long inf = 0x7ff0000000000000ull;
  CK(cudaMemcpyAsync(s->ds.dtmin + 2, &inf, sizeof(inf), cudaMemcpyHostToDevice, s->stream));
  CK(s->ops->stable_dt(s->ds, s->ph, 2, s->stream));
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, s->ds.dtmin + 2, sizeof(bits), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  double h;
  std::memcpy(&h, &bits, sizeof(h));
  *dt = cfl * h;
  return CWENO_OK;
}

}  // extern "C"

namespace cw {
static cudaError_t take_event(cweno_solver* s, cudaEvent_t* e) {
  if (!s->ev_pool.empty()) {
    *e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreate(e);
}

cudaError_t prof_begin(cweno_solver* s, cudaEvent_t* e0) {
  *e0 = nullptr;
  if (!s->profile) return cudaSuccess;
  cudaError_t e = take_event(s, e0);
  return e == cudaSuccess ? cudaEventRecord(*e0, s->stream) : e;
}

cudaError_t prof_end(cweno_solver* s, cudaEvent_t e0, int k) {
  if (!s->profile || !e0) return cudaSuccess;
  cudaEvent_t e1 = nullptr;
  cudaError_t e = take_event(s, &e1);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s->stream);
  if (e == cudaSuccess) s->ev_used.push_back({{e0, e1}, k});
  return e;
}

int enqueue_step(cweno_solver* s, double dt, int cur) {
  DtArgs a;
  a.fixed = dt > 0 ? dt : 0.0;
  a.cfl = s->prm.cfl;
  a.cur = cur;
  for (int k = 0; k < 3; ++k) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (s->profile) {
      CK(take_event(s, &e0));
      CK(take_event(s, &e1));
      CK(cudaEventRecord(e0, s->stream));
    }
    if (k == 0) CK(s->ops->rec_pred(s->ds, s->ph, a, s->stream));
    if (k == 1) CK(s->ops->flux(s->ds, s->ph, a, s->stream));
    if (k == 2) CK(s->ops->update(s->ds, s->ph, a, s->stream));
    if (s->profile) {
      CK(cudaEventRecord(e1, s->stream));
      s->ev_used.push_back({{e0, e1}, k});
    }
  }
  return CWENO_OK;
}
}  // namespace cw

extern "C" {

int ader_cweno_step(cweno_solver* s, double dt) {
  if (!s) return fail(CWENO_EINVAL, "null solver");
  CK(cudaSetDevice(s->dev));
  if (s->ale) return ale_step(s, dt);
  int rc = enqueue_step(s, dt, s->cur);
  if (rc) return rc;
  s->cur ^= 1;
  return CWENO_OK;
}

int ader_cweno_run(cweno_solver* s, int nsteps, double dt) {
  if (!s || nsteps < 0) return fail(CWENO_EINVAL, "bad argument");
  CK(cudaSetDevice(s->dev));
  if (s->ale) {
    for (int k = 0; k < nsteps; ++k) {
      int rc = ale_step(s, dt);
      if (rc) return rc;
    }
    return CWENO_OK;
  }
  for (int k = 0; k < nsteps; ++k) {
    // one graph per (time-step slot, dt): captured on first use, then replayed
    std::pair<int, double> gk(s->cur, dt > 0 ? dt : 0.0);
    cudaGraphExec_t& ex = s->graphs[gk];
    if (!ex) {
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
      bool prof = s->profile;
      s->profile = false;
      int rc = enqueue_step(s, dt, s->cur);
      s->profile = prof;
      cudaError_t e = cudaStreamEndCapture(s->stream, &g);
      if (rc) return rc;
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    }
    CK(cudaGraphLaunch(ex, s->stream));
    s->cur ^= 1;
  }
  return CWENO_OK;
}

int cweno_sync(cweno_solver* s) {
  if (!s) return fail(CWENO_EINVAL, "null solver");
  CK(cudaSetDevice(s->dev));
  int st = 0;
  CK(cudaMemcpyAsync(&st, s->ds.status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (s->ale) {
    int bad = -1;
    int rc = ale_degenerate(s, &bad);
    if (rc) return rc;
    if (bad >= 0)
      return fail(CWENO_EDEGENERATE, "the moving mesh made a least-squares or sector system singular (cell " +
                                         std::to_string(s->ds.N > bad ? bad : -1) + ", internal order)");
  }
  if (st) return fail(CWENO_ENAN, "a step produced NaN or non-positive density / pressure");
  return CWENO_OK;
}

int cweno_get_vertices(cweno_solver* s, double* xyz, int on_device) {
  if (!s || !xyz) return fail(CWENO_EINVAL, "null argument");
  if (!s->ale) return fail(CWENO_EINVAL, "the solver's mesh is fixed");
  CK(cudaSetDevice(s->dev));
  return ale_vertices(s, xyz, on_device);
}

int cweno_get_time(cweno_solver* s, double* t) {
  if (!s || !t) return fail(CWENO_EINVAL, "null argument");
  CK(cudaSetDevice(s->dev));
  CK(cudaMemcpyAsync(t, s->ds.time, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return CWENO_OK;
}

void* cweno_stream(cweno_solver* s) { return s ? (void*)s->stream : nullptr; }

int cweno_profile_enable(cweno_solver* s, int on) {
  if (!s) return fail(CWENO_EINVAL, "null solver");
  s->profile = on != 0;
  return CWENO_OK;
}

int cweno_profile_read(cweno_solver* s, double* ms, int64_t* launches) {
  return cweno_profile_read_stages(s, ms, launches, 3);
}

int cweno_profile_read_stages(cweno_solver* s, double* ms, int64_t* launches, int nstages) {
  if (!s || !ms || !launches) return fail(CWENO_EINVAL, "null argument");
  if (nstages < 1 || nstages > 8) return fail(CWENO_EINVAL, "nstages must be 1..8");
  CK(cudaSetDevice(s->dev));
  CK(cudaStreamSynchronize(s->stream));
  for (int k = 0; k < nstages; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (auto& u : s->ev_used) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, u.first.first, u.first.second));
    if (u.second < nstages) {
      ms[u.second] += t;
      launches[u.second] += 1;
    }
    s->ev_pool.push_back(u.first.first);
    s->ev_pool.push_back(u.first.second);
  }
  s->ev_used.clear();
  return CWENO_OK;
}

}  // extern "C"
