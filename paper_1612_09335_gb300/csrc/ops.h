// Host-side interface to the per-configuration CUDA kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>

#include "refelem.h"

namespace cw {

// Device buffers of one solver (types are erased: T = float or double).
struct DevState {
  int64_t N = 0, F = 0;
  int nv = 0;
  double* Q = nullptr;          // nv x N (FP64 always)
  float* Qp = nullptr;          // N x NVP x 2 FP32 pairs (FP32 mode), layout.h
  const int32_t* perm = nullptr;  // internal -> user
  const int32_t* iperm = nullptr; // user -> internal
  const int32_t* sten = nullptr;  // (ne-1) x N
  const int32_t* sten4 = nullptr; // (ne-1)/4 rounded up x N x 4, layout.h
  const void* R = nullptr;        // vectors of R_i, layout.h
  const int32_t* sec = nullptr;   // (d+1) d x N
  const void* Binv = nullptr;     // (d+1) d d x N
  const uint8_t* nsec = nullptr;  // N
  const void* Jinv = nullptr;     // d d x N
  void* qhat = nullptr;           // L nv x N
  const int32_t* fL = nullptr;
  const int32_t* fR = nullptr;
  const uint8_t* codeL = nullptr;
  const uint8_t* codeR = nullptr;
  const void* fn = nullptr;       // d x F unit normal (arithmetic type)
  const double* fa = nullptr;     // d x F area-weighted normal (FP64)
  const double* farea = nullptr;  // F (FP64)
  double* G = nullptr;            // nv x F face flux integrals (FP64)
  const void* ftab = nullptr;     // face basis table + wq + wt
  const int32_t* cellface = nullptr;  // (d+1) x N
  const double* invvol = nullptr;     // N
  const double* hsize = nullptr;      // N
  unsigned long long* dtmin = nullptr;  // 2 slots (double bits)
  double* time = nullptr;
  int* status = nullptr;
  double* stage = nullptr;        // N x nv (user-order staging)
};

struct PhysParams {
  double gamma = 1.4, ch = 2.0;
  double eps = 1e-14, lam0 = 1e5, lams = 1.0;
  int niter = 2, linear_weights = 0, positivity = 1;
  int flux = 0;  // 0 Rusanov, 1 Osher-type (Euler)
};

// Time step source: fixed > 0, else cfl * (min h/lambda) read from dtmin[cur].
struct DtArgs {
  double fixed = 0.0;
  double cfl = 0.5;
  int cur = 0;  // slot read; the other slot is reset and receives the next bound
};

class Ops {
 public:
  virtual ~Ops() {}
  virtual size_t table_bytes() const = 0;
  virtual void pack_tables(void* host) const = 0;  // face table (device copy made by caller)
  virtual size_t elem_size() const = 0;
  // Kernel attributes and launch shapes for the current device; call before
  // the first launch (and before any stream capture).
  virtual cudaError_t prepare() = 0;
  virtual cudaError_t rec_pred(const DevState& s, const PhysParams& ph, DtArgs dt, cudaStream_t st) = 0;
  virtual cudaError_t reconstruct(const DevState& s, const PhysParams& ph, double* out_user, cudaStream_t st) = 0;
  virtual cudaError_t flux(const DevState& s, const PhysParams& ph, DtArgs dt, cudaStream_t st) = 0;
  virtual cudaError_t update(const DevState& s, const PhysParams& ph, DtArgs dt, cudaStream_t st) = 0;
  virtual cudaError_t stable_dt(const DevState& s, const PhysParams& ph, int slot, cudaStream_t st) = 0;
  virtual cudaError_t set_state(const DevState& s, const double* user_dev, cudaStream_t st) = 0;
  virtual cudaError_t get_state(const DevState& s, double* user_dev, cudaStream_t st) = 0;
  virtual cudaError_t qhat_out(const DevState& s, double* user_dev, cudaStream_t st) = 0;
  // Batched time steps of many solvers of this configuration (serving): the
  // table's size, its host image for nseg solvers (at most batch_max()), and
  // one step of all of them from the device copy of that image.
  virtual size_t batch_bytes() const = 0;
  virtual int batch_max() const = 0;
  virtual void batch_fill(void* host_tab, int nseg, const DevState* const* ds, const PhysParams* const* ph,
                          const DtArgs* dt) const = 0;
  virtual cudaError_t step_batch(const void* dev_tab, int flux, cudaStream_t st) = 0;
};

// Factories (one per translation unit); nullptr if (M, precision) is not built.
std::unique_ptr<Ops> make_ops_euler2(int M, int fp32, const RefElem& re);
std::unique_ptr<Ops> make_ops_euler3(int M, int fp32, const RefElem& re);
// 3D Euler at M = 4, one translation unit per precision (the largest instances)
std::unique_ptr<Ops> make_ops_euler3_p4(int fp32, const RefElem& re);
std::unique_ptr<Ops> make_ops_mhd2(int M, int fp32, const RefElem& re);

}  // namespace cw
