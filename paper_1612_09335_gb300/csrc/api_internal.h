// Solver handle layout shared by the C ABI and the serving loop.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/cweno.h"
#include "ops.h"
#include "refelem.h"

namespace cw {
struct Ale;
}

struct cweno_solver {
  int dim = 2, order = 2, M = 1, pde = 0, prec = 0, nv = 4;
  cweno_params prm;
  cw::PhysParams ph;
  const cw::RefElem* re = nullptr;
  std::unique_ptr<cw::Ops> ops;
  cw::DevState ds;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  size_t bytes = 0;
  int cur = 0;
  int64_t nc = 0, nf = 0;
  double* outbuf = nullptr;
  size_t outbuf_bytes = 0;
  std::map<std::pair<int, double>, cudaGraphExec_t> graphs;
  // profiling: (start, stop, kernel) event triples recorded by enqueue_step
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<std::pair<cudaEvent_t, cudaEvent_t>, int>> ev_used;
  // moving mesh (mesh_motion != CWENO_MOTION_FIXED), else empty
  std::shared_ptr<cw::Ale> ale;
};

namespace cw {
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
int enqueue_step(cweno_solver* s, double dt, int cur);
// Profiling of one stage on the solver's stream, a no-op unless profiling is
// on: prof_begin records the start event, prof_end the stop event of stage k.
cudaError_t prof_begin(cweno_solver* s, cudaEvent_t* e0);
cudaError_t prof_end(cweno_solver* s, cudaEvent_t e0, int k);
const RefElem& ref_elem(int d, int M);
size_t footprint_estimate(int d, int64_t nc, int64_t nf, int order, int pde, int precision);
extern thread_local int g_setup_threads;
}  // namespace cw
