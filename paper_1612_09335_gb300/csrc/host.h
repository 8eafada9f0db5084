// Host-side mesh topology and per-cell reconstruction setup (FP64).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "refelem.h"

namespace cw {

struct MeshHost {
  int d = 2;
  int64_t nv = 0, nc = 0;
  std::vector<double> xyz;       // user vertices nv x d
  bool per[3] = {false, false, false};
  double Lper[3] = {0, 0, 0};
  double qscale = 1.0;           // largest bounding-box extent (ranking tolerances)
  // internal (Morton) order
  std::vector<int32_t> perm;     // internal -> user cell index
  std::vector<int32_t> iperm;    // user -> internal
  std::vector<int64_t> gv;       // nc x (d+1) global vertex ids
  std::vector<double> X;         // nc x (d+1) x 3 unwrapped coordinates
  std::vector<double> vol;       // |T_i|
  std::vector<double> bary;      // nc x 3
  std::vector<double> hsize;     // incircle / insphere diameter
  std::vector<int32_t> nbr;      // nc x (d+1): neighbour across local face k (opposite vertex k), -1 boundary
  // faces (interior first in cell order, boundary faces included)
  int64_t nf = 0, nbnd = 0;
  std::vector<int32_t> fL, fR;   // fR = -1 on the boundary
  std::vector<uint8_t> codeL, codeR;
  std::vector<double> fn;        // nf x 3 unit normal, out of L
  std::vector<double> farea;     // nf
  std::vector<int32_t> cellface; // nc x (d+1): face id * 2 + (cell is R)
};

// Returns 0 or a CWENO_E* code, with a message in err.
int build_mesh(int d, int64_t nv, const double* xyz, int64_t nc, const int32_t* cells, const double* period,
               MeshHost& m, std::string& err);

// Per-cell reconstruction data in internal order (FP64, SoA-ready).
struct CellSetup {
  int ne = 0, Mc = 0, d = 2;
  std::vector<int32_t> sten;    // nc x (ne-1): S_i^0 \ {i}
  std::vector<double> R;        // nc x (Mc-1) x (ne-1): pseudo-inverse rows
  std::vector<int32_t> sec;     // nc x (d+1) x d sector cells, -1 if dropped
  std::vector<double> Binv;     // nc x (d+1) x d x d
  std::vector<uint8_t> nsec;    // kept sectors per cell
  std::vector<double> Jinv;     // nc x d x d, Jinv[e][m] = d xi_e / d x_m
};

// with_lsq = false leaves R empty (the device computes it, lsq_setup_device).
int build_cell_setup(const MeshHost& m, const RefElem& re, CellSetup& cs, std::string& err, int nthreads,
                     bool with_lsq = true);

// Least-squares pseudo-inverses R on the current device (lsq_gpu.cu): d_sten
// the uploaded SoA stencils, d_R the solver's R buffer (FP32 if fp32, else
// FP64), stream a cudaStream_t.  Synchronous on that stream.
int lsq_setup_device(const MeshHost& m, const RefElem& re, const int32_t* d_sten, void* d_R, int fp32,
                     void* stream, std::string& err);
// The same kernel on caller-uploaded vertices d_X (nc x (d+1) x 3) and
// barycentres d_bary (nc x 3); asynchronous on stream, *d_bad receives the
// smallest rank-deficient cell index (atomicMin, caller-initialised).
int lsq_launch_device(const MeshHost& m, const RefElem& re, const double* d_X, const double* d_bary,
                      const int32_t* d_sten, void* d_R, int fp32, int* d_bad, void* stream, std::string& err);
// Stencils, sectors, inverse Jacobians, sector inverses and R_i of every
// cell on the device (setup_gpu.cu), into caller-allocated buffers in the
// kernels' layouts; returns kCellSetupOnHost when a stencil search outgrows
// the device kernel's per-thread capacity (the caller then runs the host
// search), else 0 or a CWENO_E* code with a message in err.
constexpr int kCellSetupOnHost = 1;
int cell_setup_device(const MeshHost& m, const RefElem& re, int fp32, void* stream, int32_t* d_sten, int32_t* d_sten4,
                      int32_t* d_sec, void* d_Binv, uint8_t* d_nsec, void* d_Jinv, void* d_R, std::string& err);

// Moving meshes (ale.cu, two dimensions, FP64): rebuild on the device
// the least-squares pseudo-inverses R and the sector inverses Binv of every
// cell from the unwrapped cell vertices d_X (nc x (d+1) x 3, internal order)
// and barycentres d_bary (nc x 3) of the current mesh, for the fixed
// stencils d_sten and sector cells d_sec (SoA, as uploaded by the setup).
// R and Binv are written as FP32 when fp32 (FP32-mixed solvers), else FP64.
// *d_bad receives the smallest cell index whose system is degenerate.
// Asynchronous on stream (a cudaStream_t).
int ale_matrices_device(const MeshHost& m, const RefElem& re, const double* d_X, const double* d_bary,
                        const int32_t* d_sten, const int32_t* d_sec, void* d_R, void* d_Binv, int fp32, int* d_bad,
                        void* stream);

}  // namespace cw
