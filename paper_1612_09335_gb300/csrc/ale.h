// Moving-mesh (direct ALE) path of a solver: 2D, Euler, FP64 (ale.cu).
#pragma once
#include <string>

#include "api_internal.h"
#include "host.h"

namespace cw {

// Device state of the moving mesh of solver s (vertex positions, incidence
// lists, per-cell periodic shifts, reference tables, scratch).  Returns 0 or
// a CWENO_E* code with a message in err.
int ale_create(cweno_solver* s, const MeshHost& m, std::string& err);
// Geometry, h, 1/|T| and the reconstruction matrices of the current vertices
// (no-op until the mesh moves again).  Asynchronous.
int ale_refresh(cweno_solver* s);
// One direct ALE step (dt <= 0: CFL bound on the current mesh).  Asynchronous.
int ale_step(cweno_solver* s, double dt);
// Current vertices (nv x 2, caller order) into host or device memory; synchronous.
int ale_vertices(cweno_solver* s, double* xyz, int on_device);
// Smallest cell whose least-squares or sector system became singular, or -1.
int ale_degenerate(cweno_solver* s, int* cell);

}  // namespace cw
