/*
 * cweno.h -- C ABI of the GB300 ADER-CWENO library.
 *
 * Fixed-mesh (Eulerian) ADER-CWENO finite-volume method on triangle and
 * tetrahedron meshes, after Dumbser, Boscheri, Semplice & Russo, "Central
 * WENO schemes on unstructured meshes" (arXiv 1612.09335).  One time step
 * is: CWENO reconstruction (Sec. 2.1), local space-time Galerkin predictor
 * (Sec. 2.2), space-time-quadrature Rusanov face fluxes and the conservative
 * one-step update (Sec. 2.4, Eq. PDEfinal with zero mesh velocity).  For
 * the Euler equations the same step also runs on a moving mesh (direct ALE,
 * Secs. 2.2-2.4: cweno_params.mesh_motion, cweno_get_vertices), orders
 * 2..4.
 *
 * Conventions for every call:
 *   - Return value: CWENO_OK (0) or a negative CWENO_E* code.  A message
 *     for the last failure of the calling thread is in cweno_last_error().
 *   - Inputs are copied; the library never keeps a caller pointer.
 *   - Handles are opaque, owned by the library, freed by the matching
 *     *_destroy call (NULL is accepted and ignored).
 *   - Cell arrays are in the caller's cell order (the order of `cells` given
 *     to cweno_mesh_create).  Internally cells are Morton-reordered; the
 *     permutation never shows at this boundary.
 *   - `on_device` != 0 means the pointer is CUDA device memory of the
 *     solver's device, 0 means host memory (pageable or pinned).
 *   - State vectors are AoS by cell: Q[c * nvars + v], FP64, conserved
 *     variables.  Euler (Eqs. eulerTerms, eos): nvars = d + 2,
 *     (rho, rho u, rho v[, rho w], rho E).  Ideal MHD with GLM cleaning
 *     (Eqs. MHDTerms, MHDeos, Gaussian units): nvars = 9,
 *     (rho, rho u, rho v, rho w, rho E, Bx, By, Bz, psi), also in 2D.
 *   - Work is enqueued on the solver's CUDA stream and is asynchronous
 *     unless stated; cweno_sync() waits for it.
 */
#ifndef CWENO_H
#define CWENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CWENO_OK = 0,
  CWENO_EINVAL = -1,      /* bad argument, size or unsupported combination */
  CWENO_EDEGENERATE = -2, /* non-positive cell volume, rank-deficient LSQ, mesh too small */
  CWENO_ENOMEM = -3,      /* device or host allocation failed */
  CWENO_EBUSY = -4,       /* server: request can never be admitted */
  CWENO_ENAN = -5,        /* a step produced NaN / non-positive density or pressure */
  CWENO_ETIMEDOUT = -6,   /* a bounded wait gave up */
  CWENO_ECUDA = -7,       /* CUDA runtime error (message has the CUDA text) */
  CWENO_ENOTFOUND = -8    /* server: unknown request id */
};

enum { CWENO_EULER = 0, CWENO_MHD_GLM = 1 };
enum { CWENO_FP64 = 0, CWENO_FP32_MIXED = 1 };
/* Numerical flux at the space-time face points. */
enum { CWENO_FLUX_RUSANOV = 0, CWENO_FLUX_OSHER = 1, CWENO_FLUX_RUSANOV_QF = 2 };
/* Mesh motion (Secs. 2.3-2.4).  FIXED: the Eulerian scheme on the given
 * mesh.  LAGRANGE: the direct ALE scheme with mesh velocity V = v, the local
 * fluid velocity (the paper's choice for its moving-mesh tests): predictor on
 * the moving element (Eqs. CGfinal, ODEfinal), nodal solver (Eqs. NScs to
 * newX), space-time control volumes (Eqs. dCi to detChi), update of Eq.
 * (PDEfinal).  STILL: the same ALE machinery with V = 0 (it reduces to the
 * Eulerian scheme; a check of the moving-mesh path). */
enum { CWENO_MOTION_FIXED = 0, CWENO_MOTION_LAGRANGE = 1, CWENO_MOTION_STILL = 2 };

typedef struct cweno_mesh cweno_mesh;
typedef struct cweno_solver cweno_solver;
typedef struct cweno_server cweno_server;

/* Scheme parameters.  Defaults (cweno_default_params) are the paper's:
 * eps = 1e-14, r = 4, lambda_0 = 1e5, lambda_s = 1 (Sec. 2.1, after Eq.
 * weights2; the lambdas are normalised to sum 1 over the kept stencils),
 * CFL = 1/d (Eq. timestep), gamma = 1.4 (Euler) or 5/3 (MHD), c_h = 2,
 * Picard iterations of Eq. (CGfinal) = M + 1, positivity scaling on,
 * Rusanov flux. */
typedef struct {
  double eps;          /* epsilon of Eq. (weights2) */
  double r;            /* exponent r of Eq. (weights2); must be 4 */
  double lambda0;      /* raw linear weight of the central stencil */
  double lambda_s;     /* raw linear weight of each sectorial stencil */
  double gamma;        /* ratio of specific heats */
  double c_h;          /* GLM divergence-cleaning speed (MHD) */
  double cfl;          /* CFL number used when ader_cweno_step(dt <= 0) */
  int picard_iters;    /* iterations of Eq. (CGfinal); <= 0 -> M + 1 */
  int linear_weights;  /* test mode: omega := lambda (no indicators) */
  int positivity;      /* 1 (default): scale w toward the cell average where
                          density or pressure would fall below 1e-3 of their
                          cell-average values at a lattice node (Zhang & Shu
                          scaling; not part of the paper, inactive wherever the
                          reconstruction is admissible); 0: the paper's scheme */
  int flux;            /* CWENO_FLUX_RUSANOV (default, Eq. rusanov) or
                          CWENO_FLUX_OSHER: the Osher-type flux of Eq. (osher),
                          |A_n| integrated along the straight path between the
                          two traces by 3-point Gauss-Legendre; Euler only
                          (EINVAL for MHD); or CWENO_FLUX_RUSANOV_QF: the
                          quadrature-free fixed-mesh form described after Eq.
                          (osher): the nodal predictor fluxes contracted with
                          precomputed integrals of the nodal basis over face
                          and time step, Rusanov dissipation with the
                          signal speed of the two sides' space-time face
                          averages */
  int mesh_motion;     /* CWENO_MOTION_FIXED (default), _LAGRANGE or _STILL.
                          Moving meshes: Euler, Rusanov flux, FP64 or
                          FP32-mixed, order 2..4 on triangles and
                          tetrahedra (EINVAL otherwise); the
                          stencils are chosen on the initial mesh and kept
                          (the topology never changes), their least-squares
                          and sector matrices are rebuilt on the device every
                          step in FP64.  FP32-mixed: predictor and face
                          traces in FP32 on deviations from the cell
                          averages, the averages' part of the face
                          integrals, nodal solver and update in FP64 */
} cweno_params;

/* Fill *p with the paper's defaults for dimension `dim` and `pde`. */
void cweno_default_params(cweno_params* p, int dim, int pde);

/* Thread-local text of the last error of this thread ("" if none). */
const char* cweno_last_error(void);

/* Number of conserved variables for (dim, pde): d+2 (Euler) or 9 (MHD). */
int cweno_nvars(int dim, int pde);

/* Mesh from vertices and connectivity (Sec. 2, Eqs. trian, xietaTransf).
 *   dim      2 (triangles) or 3 (tetrahedra)
 *   xyz      nv x dim vertex coordinates (host, row-major)
 *   cells    nc x (dim+1) vertex ids (host); each cell positively oriented:
 *            det[X1-X0, X2-X0(, X3-X0)] > 0 for the affine map of Eq.
 *            (xietaTransf), whose first vertex is X0
 *   period   NULL (bounded domain, transmissive boundary faces) or dim
 *            lengths; entries > 0 make that direction periodic.  Periodic
 *            meshes give each torus vertex once; every cell is unwrapped to
 *            the image nearest its first vertex, which needs cells much
 *            smaller than the period.
 * Errors: EINVAL (bad sizes / ids, a face shared by > 2 cells),
 *         EDEGENERATE (non-positive volume).  Host-only, synchronous. */
int cweno_mesh_create(int dim, int64_t nv, const double* xyz, int64_t nc, const int32_t* cells,
                      const double* period, cweno_mesh** out);
void cweno_mesh_destroy(cweno_mesh* m);
/* Cells, faces (interior + boundary) of a mesh. */
int cweno_mesh_info(const cweno_mesh* m, int64_t* ncells, int64_t* nfaces, int64_t* nboundary);

/* Diagnostic, host only: the stencils cweno_setup would use for `order`,
 * in the caller's cell ids.  S0: nc x n_e (S0[c*n_e] = c, then the ranked
 * breadth-first cells of Eq. stencil); sec: nc x (d+1) x d sector cells
 * (Sec. 2.1 cone rule), -1 where a sector is dropped.  `order` 2..5.
 * Errors as cweno_setup. */
int cweno_mesh_stencils(const cweno_mesh* m, int order, int32_t* S0, int32_t* sec);
/* Diagnostic: the stencils a solver actually uses (found on the device by
 * cweno_setup, or by the host search when a stencil outgrows the device
 * search's capacity), in the layout and caller ids of cweno_mesh_stencils.
 * S0: nc x n_e, sec: nc x (d+1) x d, host.  Synchronous. */
int cweno_solver_stencils(cweno_solver* s, int32_t* S0, int32_t* sec);

/* Current vertex positions, nv x dim FP64 in the caller's vertex order
 * (they move under CWENO_MOTION_LAGRANGE; otherwise the mesh's own).
 * on_device selects a device or host destination.  EINVAL for a solver of
 * a fixed mesh.  Synchronous. */
int cweno_get_vertices(cweno_solver* s, double* xyz, int on_device);

/* Reconstruction setup for `order` = M + 1 in 2..5 (Sec. 2.1): central
 * stencils S_i^0 of n_e = d * M(M,d) cells (Eq. stencil), d+1 sectorial
 * stencils, the FP64 pseudo-inverses of the constrained least-squares
 * problems (Eq. CWENO:Popt, precomputed as the paper prescribes for fixed
 * meshes), the sector inverses (Eq. CWENO:Ps), the universal matrices
 * (Sigma_lm, predictor matrices of Eq. cgPDE) and face quadrature tables;
 * all are uploaded to the current CUDA device.  `precision` selects FP64
 * throughout, or FP32 arithmetic with FP64 setup and FP64 cell-average
 * accumulators.  `stream` is a cudaStream_t (NULL: the library creates a
 * non-blocking stream it owns).  `params` NULL means defaults.
 * Supported: (dim 2 and 3, Euler, order 2..5; order 5 is the paper's
 * fifth-order scheme of Secs. 4.2.1-4.2.2 and the O5 column of its 3D
 * convergence study), (dim 2, MHD, order 2..4).
 * The state is zero until cweno_set_state.
 * Errors: EINVAL, EDEGENERATE (rank-deficient LSQ, mesh too small for the
 * stencil), ENOMEM, ECUDA.  Synchronous. */
int cweno_setup(const cweno_mesh* m, int order, int pde, int precision, const cweno_params* params,
                void* stream, cweno_solver** out);
void cweno_solver_destroy(cweno_solver* s);

/* Sizes: nvars, M(M,d), n_e, L = M(M,d+1) space-time nodes, cells, faces. */
int cweno_solver_info(const cweno_solver* s, int* nvars, int* mcal, int* ne, int* lcal, int64_t* ncells,
                      int64_t* nfaces);
/* Device bytes held by the solver (mesh tables, matrices, state, scratch). */
int cweno_solver_footprint(const cweno_solver* s, size_t* bytes);

/* Cell averages Q (Eq. cellaverage), nc x nvars FP64, copied in / out.
 * set_state also resets the accumulated time and the status word and
 * computes the CFL time-step bound for the next step.
 * on_device = 0: Q is host memory.  Pageable memory goes through a device
 * staging buffer.  Page-locked memory that is mapped into the device address
 * space (cudaHostAlloc, cudaHostRegister, torch pin_memory) is read or
 * written in place by the state kernel over the CPU-GPU link, with no
 * staging copy.  In both cases set_state is asynchronous on the solver's
 * stream for page-locked Q: keep Q unchanged until a later synchronous call
 * (get_state, reconstruct, ...) or a synchronisation of that stream. */
int cweno_set_state(cweno_solver* s, const double* Q, int on_device);
int cweno_get_state(cweno_solver* s, double* Q, int on_device); /* synchronous */

/* CWENO reconstruction of the current state (Eqs. CWENO:Popt .. weights2):
 * w_i evaluated at the M(M,d) equispaced lattice nodes of T_E in the
 * reference frame of each cell (node (i/M, j/M[, k/M]), enumerated with the
 * zeta index outermost, then eta, then xi), written as
 * w_nodal[(c * Mcal + node) * nvars + v].  Synchronous. */
int cweno_reconstruct(cweno_solver* s, double* w_nodal, int on_device);

/* Space-time predictor of the current state for time step dt (Eq. CGfinal),
 * nodal values at the L space-time nodes (principal lattice of the
 * (d+1)-simplex, step 1/M, time level tau = t/M outermost), written as
 * qhat[(c * L + node) * nvars + v].  Diagnostic; synchronous.  EINVAL on
 * a moving mesh (its predictor is internal to the ALE step). */
int cweno_predictor(cweno_solver* s, double dt, double* qhat, int on_device);

/* Global time step of Eq. (timestep) for the current state:
 * cfl * min_i h_i / |lambda_max,i|, h_i the incircle / insphere diameter.
 * Synchronous; returns it in *dt. */
int cweno_stable_dt(cweno_solver* s, double cfl, double* dt);

/* One ADER-CWENO step of length dt (Eq. PDEfinal, Eulerian).  dt <= 0 uses
 * the CFL bound of the current state, computed on the device (no host
 * round trip; the bound for the following step is produced by the update).
 * On a moving mesh (mesh_motion != FIXED) one direct ALE step: geometry and
 * reconstruction matrices of the current mesh, moving-element predictor,
 * nodal solver and new vertices, space-time face fluxes, volume-weighted
 * update; dt <= 0 takes the CFL bound on the current mesh.  Asynchronous. */
int ader_cweno_step(cweno_solver* s, double dt);

/* `nsteps` steps as above; the sequence is captured once into a CUDA graph
 * per solver and replayed (moving meshes: plain launches).  Asynchronous. */
int ader_cweno_run(cweno_solver* s, int nsteps, double dt);

/* Wait for the solver's stream.  Returns ENAN if any step since the last
 * set_state produced NaN or non-positive density / pressure (on a moving
 * mesh also a cell of non-positive area), EDEGENERATE if a moving mesh made
 * a least-squares or sector system singular. */
int cweno_sync(cweno_solver* s);
/* Simulated time accumulated since set_state (synchronous). */
int cweno_get_time(cweno_solver* s, double* t);
/* The solver's CUDA stream (cudaStream_t). */
void* cweno_stream(cweno_solver* s);

/* Measurement: with profiling on, ader_cweno_step brackets each of its three
 * kernels (reconstruction + predictor, face fluxes, update) with CUDA events
 * on the solver's stream (fixed meshes; a moving-mesh step records its
 * stages instead, cweno_profile_read_stages).  cweno_profile_read waits for the stream and
 * returns the summed device milliseconds per kernel (ms[0..2]) and the
 * number of launches per kernel since the last read, then clears them. */
int cweno_profile_enable(cweno_solver* s, int on);
int cweno_profile_read(cweno_solver* s, double* ms, int64_t* launches);
/* The same per stage for moving meshes (the paper has no counterpart: it is
 * instrumentation).  ms[k], launches[k] for k < nstages (1..8): on a moving
 * mesh 0 geometry + least squares + sector inverses, 1 reconstruction, 2
 * predictor, 3 nodal solver, 4 lateral space-time faces, 5 update, 6 CFL
 * bound; on a fixed mesh the three kernels of cweno_profile_read.  Waits for
 * the stream and clears the record, like cweno_profile_read. */
int cweno_profile_read_stages(cweno_solver* s, double* ms, int64_t* launches, int nstages);

/* Measured FMA rate of the current device (the paper has no counterpart: it
 * is the denominator of the FP32 / FP64 pipe fractions a benchmark reports).
 * fp64 = 0 measures FP32 fused multiply-adds, otherwise FP64.  Every thread
 * runs 16 independent FMA chains, in enough blocks to fill every SM; one
 * untimed launch, then one launch timed with CUDA events on a private
 * stream (about 10 ms).  Synchronous.  *tflops receives 2 flops per FMA per
 * second / 1e12, *ms (nullable) the timed launch's milliseconds.  Allocates
 * no device memory. */
int cweno_measure_fma_peak(int fp64, double* tflops, double* ms);

/* CFL time-step bound without any allocation.  The paper has no counterpart:
 * this is for callers that cannot call cudaMalloc (work inside another
 * framework's memory pool, or in a process whose device memory is reserved
 * up front).  It computes
 * cfl * min_i h_i / |lambda_max(Q_i)| like cweno_stable_dt, but for a state in
 * the caller's own buffers:
 *   Q      device, ncells x nvars FP64, AoS by cell (as cweno_set_state)
 *   h      device, ncells FP64, characteristic cell sizes (incircle /
 *          insphere diameters, Eq. timestep)
 *   dt     device, one FP64, receives the bound
 *   stream cudaStream_t (NULL: the legacy default stream); asynchronous.
 * dim 2 or 3 with pde CWENO_EULER, or dim 2 with CWENO_MHD_GLM (EINVAL
 * otherwise, as cweno_setup).
 * Scratch is a file-scope device array of one partial minimum per 256 cells
 * (512 KiB), held by every GPU that loads the library until the process
 * exits, so ncells must not exceed CWENO_NOALLOC_MAX_CELLS (EINVAL
 * otherwise).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current.  The address is
 * kept for the life of the process: after cudaDeviceReset (or any other
 * teardown of the device's primary context) the array lives at a new
 * address, so do not call this entry point again in that process.  Calls
 * that overlap on the GPU share the scratch and race; serialise them (one
 * stream, or events).  Nothing is allocated and nothing is freed. */
#define CWENO_NOALLOC_MAX_CELLS (65536 * 256)
int cweno_stable_dt_noalloc(int dim, int pde, int64_t ncells, const double* Q, const double* h, double gamma,
                            double c_h, double cfl, double* dt, void* stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of independent solves on one GPU.
 * A request owns a mesh (copied), order, initial state, CFL and step count.
 * The server admits requests while their measured device footprint fits the
 * memory budget and a slot is free, sets each one up on a host worker, and
 * groups the admitted requests by configuration (dimension, order, PDE,
 * precision, flux) and size class (cells below 4096, 16384, 65536, above:
 * a tick lasts as long as its members' steps together, so small requests do
 * not wait for large ones).  Each group advances all of its members by one time step
 * per tick: one captured CUDA graph of batched kernels over a table of the
 * members (the reconstruction + predictor, flux and update of every member's
 * cells and faces in the same three launches), replayed every tick with the
 * table rewritten in place as members join and leave.  Groups tick
 * concurrently; finished requests are retired and waiting ones admitted as
 * slots and memory free up.  Results are identical to running the same
 * request alone (same per-cell arithmetic, no cross-request reductions).
 * ------------------------------------------------------------------------- */
typedef struct {
  int dim;
  int64_t nv;
  const double* xyz;     /* nv x dim, host */
  int64_t nc;
  const int32_t* cells;  /* nc x (dim+1), host */
  const double* period;  /* dim or NULL */
  int order;             /* as cweno_setup */
  int pde;               /* CWENO_EULER / CWENO_MHD_GLM */
  int precision;         /* CWENO_FP64 / CWENO_FP32_MIXED */
  const double* Q0;      /* nc x nvars, host */
  double cfl;            /* time step from Eq. (timestep) each step */
  int nsteps;
} cweno_request;

enum { CWENO_REQ_QUEUED = 0, CWENO_REQ_RUNNING = 1, CWENO_REQ_DONE = 2, CWENO_REQ_ERROR = 3 };

/* mem_budget: device bytes the server may hold for admitted requests
 * (0 -> 80% of free memory); max_slots: concurrently admitted requests, each
 * with its own CUDA stream for its setup (<= 0 -> 256, at most 256; a
 * group's batch table holds 64 members, further requests of a configuration
 * wait to join it); nworkers: host threads preparing
 * admitted requests (mesh on the host; stencils, sectors and least-squares
 * inverses on the device; <= 0 -> one per host core).  Admission is first come,
 * first served. */
int serve_create(size_t mem_budget, int max_slots, int nworkers, cweno_server** out);
/* Copies the request; returns its id.  EBUSY if its footprint exceeds the
 * whole budget (it could never be admitted).  Thread-safe. */
int serve_submit(cweno_server* s, const cweno_request* r, uint64_t* id);
/* Status of a request; when DONE and Q_out != NULL copies the final state
 * (nc x nvars, host) and releases the request.  latency_s (nullable) gets
 * submit-to-completion wall time.  Thread-safe, non-blocking. */
int serve_poll(cweno_server* s, uint64_t id, int* status, double* Q_out, double* latency_s);
/* Wait until every submitted request is DONE or ERROR, at most timeout_s
 * seconds (ETIMEDOUT otherwise). */
int serve_drain(cweno_server* s, double timeout_s);
/* Counters: submitted, admitted, completed, peak concurrently admitted,
 * cell-updates completed. */
int serve_stats(cweno_server* s, uint64_t* submitted, uint64_t* admitted, uint64_t* completed,
                uint64_t* peak_running, double* cell_updates);
/* Batching counters: ticks completed (one batched time step of one group)
 * and the member time steps they carried (member_steps / ticks = requests
 * advanced per launch sequence). */
int serve_batch_stats(cweno_server* s, uint64_t* ticks, uint64_t* member_steps);
void serve_destroy(cweno_server* s);

#ifdef __cplusplus
}
#endif
#endif /* CWENO_H */
