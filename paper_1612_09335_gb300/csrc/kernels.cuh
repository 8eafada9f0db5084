// CUDA kernels of the fixed-mesh ADER-CWENO step (sm_103a), templated on
// dimension D, polynomial degree M, PDE and arithmetic type T.
//
//   k_rec_pred  one thread per cell: stencil gather, P_opt = R dQ
//               (Eq. CWENO:Popt), sectorial P_s (Eq. CWENO:Ps), P_0
//               (Eq. CWENO:P0), indicators and nonlinear weights (Eqs.
//               weights, weights2), then the space-time Galerkin predictor
//               (Eq. CGfinal) with the Picard iteration folded into
//               q1 = C0 q0 - dt sum_e P_e G_e,  P_e = (K_tau^1)^-1 K_xi_e;
//               node loops rolled, working set in shared memory; writes
//               the L space-time nodal values.
//   k_flux      one thread per face (persistent grid): the predictor of both
//               sides at the space-time Gauss points of the face, Rusanov
//               flux (Eq. rusanov) with s_max per point, integrated with
//               weights -> G_f = dt |f| sum w G.  Each face once.
//   k_update    one thread per cell, gather by cell (deterministic, no
//               atomics): Q -= (1/|T|) sum_f +-G_f in FP64 (Eq. PDEfinal),
//               admissibility status, and the CFL bound of Eq. (timestep)
//               for the next step (block min + atomicMin on the bits).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <memory>
#include <type_traits>
#include <vector>

#include "layout.h"
#include "ops.h"
#include "pred_pattern.h"

namespace cw {

constexpr int cmcal(int M, int d) {
  return d == 2 ? (M + 1) * (M + 2) / 2
                : d == 3 ? (M + 1) * (M + 2) * (M + 3) / 6 : (M + 1) * (M + 2) * (M + 3) * (M + 4) / 24;
}

// smallest stride >= base, a multiple of vw elements, whose byte size is
// 16 mod 128
constexpr int code_stride(int base, int vw, int esize) {
  int st = (base + vw - 1) / vw * vw;
  while ((st * esize) % 128 != 16) st += vw;
  return st;
}

template <int D_, int M_, int PDE_, typename T_>
struct Cfg {
  static constexpr int D = D_, M = M_, PDE = PDE_;
  using T = T_;
  static constexpr int NV = PDE == 0 ? D + 2 : 9;
  static constexpr int MC = cmcal(M, D);
  static constexpr int MC1 = MC - 1;
  static constexpr int NE = D * MC;
  static constexpr int NS = D + 1;
  static constexpr int L = cmcal(M, D + 1);
  static constexpr int L0 = MC;
  static constexpr int L1 = L - MC;
  static constexpr int NQS = D == 2 ? M + 1 : (M + 1) * (M + 1);
  static constexpr int NQT = M + 1;
  static constexpr int NCODE = D == 2 ? 6 : 24;
  // FP32 pairs per cell (layout.h) and the 16-byte vectors of R_i
  static constexpr int NVP = pair_vars(NV);
  static constexpr int NE1 = NE - 1;
  static constexpr int RV = r_vectors(NE1, MC - 1, 16 / (int)sizeof(T_));
  // face tables: each (code, time point, space point) row of L basis values
  // is padded to a multiple of one 16-byte vector
  static constexpr int VW = 16 / (int)sizeof(T_);
  static constexpr int LP = (L + VW - 1) / VW * VW;
  // per-code stride padded to 16 bytes past a multiple of 128 bytes, so the
  // rows of different face codes read by one warp fall into different
  // shared-memory banks
  static constexpr int CODE_STRIDE = code_stride(NQT * NQS * LP, VW, (int)sizeof(T_));
  static constexpr int TABN = NCODE * CODE_STRIDE;
  // quadrature-free flux: per code, the L integrals of the nodal basis over
  // the face and [0,1] (rows of LP), after the quadrature weights
  static constexpr int QF_OFF = (TABN + NQS + NQT + VW - 1) / VW * VW;
  static constexpr int TAB_TOTAL = QF_OFF + NCODE * LP;
  // face kernel: two threads per face in FP32 (each thread evaluates its
  // own side's traces, the pair swaps them by shuffles and splits the
  // Rusanov points); one thread per face in FP64
#ifdef CW_FLUX_PAIR
  static constexpr int PAIR = CW_FLUX_PAIR;
#else
  static constexpr int PAIR = sizeof(T_) == 4;
#endif
  // passes of the pair kernel over the time points: one pass holds all
  // NQT NQS traces where they fit (2D Euler), otherwise one time point per
  // pass (q_hat re-read per time point, as in the one-thread kernel)
#ifdef CW_PAIR_PASSES
  static constexpr int PAIR_PASSES = CW_PAIR_PASSES;
#else
  static constexpr int PAIR_PASSES = NQT * NQS * NV <= 64 ? 1 : NQT;
#endif
  // groups of space-time points per face side in the pair kernel (threads
  // per face = 2 FLUX_SPLIT)
#ifdef CW_FLUX_SPLIT
  static constexpr int FLUX_SPLIT_REQ = CW_FLUX_SPLIT;
#else
  static constexpr int FLUX_SPLIT_REQ = 1;
#endif
  static constexpr int FLUX_SPLIT = (NQT * NQS) % (FLUX_SPLIT_REQ * PAIR_PASSES) == 0 ? FLUX_SPLIT_REQ : 1;
  // prefetch of the next q_hat chunk in the trace loop where the extra
  // registers are few (measured: faster in 2D Euler, slower for NV >= 5)
  static constexpr bool TR_PREFETCH = VW * NV <= 16;
  // Resident 128-thread blocks per SM requested from the register allocator
  // (measured launch-shape sweeps).  Face kernel (the two-threads-per-face
  // form in FP32): four in FP32 Euler (<= 128 registers) except 3D P3, three
  // in FP32 MHD (<= 168), unconstrained elsewhere.
#ifdef CW_FLUX_MINB
  static constexpr int FLUX_MINB = CW_FLUX_MINB;
#else
  static constexpr int FLUX_MINB = sizeof(T_) != 4 ? 1 : PDE == 1 ? 3 : (D == 3 && M >= 3) ? 1 : 4;
#endif
  // Reconstruction + predictor: four in 2D FP32 Euler up to P3 (<= 128
  // registers), three in 3D FP32 Euler (<= 168; 128 spills); unconstrained
  // where a cap would spill (MHD, FP64, P4).
#ifdef CW_REC_MINB
  static constexpr int REC_MINB = CW_REC_MINB;
#else
  static constexpr int REC_MINB = (sizeof(T_) != 4 || M >= 4) ? 1 : NV == 4 ? 4 : NV == 5 ? 3 : 1;
#endif
  // predictor working set (the fixed part and the current iterate of the L1
  // unknown space-time nodes) kept in shared memory, one column per thread,
  // so that the node loops run rolled: a few kilobytes of code instead of a
  // fully unrolled body that misses the instruction cache
  // Where one block's columns exceed the shared memory of an SM (3D P4 in
  // FP64: 358 KB), each thread keeps its working set in local memory instead.
  static constexpr int PRED_WS_BYTES = 2 * L1 * NV * (int)sizeof(T_) * 128;
  static constexpr bool PRED_WS_LOCAL = PRED_WS_BYTES > 227 * 1024;
  static constexpr int PRED_SMEM_BYTES = PRED_WS_LOCAL ? 0 : PRED_WS_BYTES;
  // reconstruction at the lattice nodes kept in the predictor's working set
  // (where it fits: L0 NV <= 2 L1 NV)
  static constexpr bool STASH = L0 <= 2 * L1;
  // tau = 0 node loop of the predictor unrolled with the zero pattern of P_e
  // (measured: 4 % slower at 2D P3 FP32, the unrolled body costs more in
  // instruction fetch than the skipped FMAs save)
#ifdef CW_TAU0_SPARSE
  static constexpr bool TAU0_SPARSE = CW_TAU0_SPARSE;
#else
  static constexpr bool TAU0_SPARSE = false;
#endif
#ifdef CW_SIDE_AHEAD
  static constexpr bool SIDE_AHEAD = CW_SIDE_AHEAD;
#else
  static constexpr bool SIDE_AHEAD = true;
#endif
#ifdef CW_IDS_AHEAD
  static constexpr bool IDS_AHEAD = CW_IDS_AHEAD;
#else
  static constexpr bool IDS_AHEAD = true;
#endif
  // chunks of four stencil neighbours unrolled together in the gather
#ifdef CW_GATHER_CHUNKS
  static constexpr int GATHER_CHUNKS = CW_GATHER_CHUNKS;
#else
  static constexpr int GATHER_CHUNKS = 1;
#endif
  // Picard node loop unrolled with the compile-time zero pattern of P_e
  // where it has at most ten unknown nodes (measured: P2/P3 3-8 % faster;
  // the 20-node unroll of P4 overflows the instruction cache)
#ifdef CW_PRED_SPARSE
  static constexpr bool PRED_SPARSE = CW_PRED_SPARSE;
#else
  static constexpr bool PRED_SPARSE = L1 <= 10;
#endif
};

template <class C>
struct CellTab {
  using T = typename C::T;
  T E[C::L0][C::MC1];
  T Sig[C::MC1][C::MC1];  // Sigma's diagonal and its upper triangle doubled (symmetric form)
  T CE[C::L1][C::MC1];  // C0 E: known part of the unknown nodes, from w directly
  int sel[C::L1];       // tau = 0 lattice node below each unknown node
  T P[C::D][C::L1][C::L];
};

template <class C>
struct KArgs {
  using T = typename C::T;
  int64_t N, F;
  double* Q;
  float* Qp;  // FP32 pairs (hi, lo) per cell and variable, layout.h
  const int32_t* perm;
  const int32_t* iperm;
  const int32_t* sten4;  // central stencil ids, four per vector, layout.h
  const T* R;
  const int32_t* sec;
  const T* Binv;
  const uint8_t* nsec;
  const T* Jinv;
  T* qhat;
  const int32_t* fL;
  const int32_t* fR;
  const uint8_t* codeL;
  const uint8_t* codeR;
  const T* fn;
  const double* fa;     // area-weighted normal |f| n, FP64, d x F
  const double* farea;  // |f|, FP64
  double* G;            // face flux integrals, FP64
  const T* ftab;
  const int32_t* cellface;
  const double* invvol;
  const double* hsize;
  unsigned long long* dtmin;
  double* time;
  int* status;
  double* out;
  T gamma, ch, eps, lam0, lams;
  int niter, linw, pos, flux;
  double dt_fixed, cfl;
  int cur, reset_next;
};

// The per-cell reference tables (E, Sigma, C0 E, P_e) travel as a kernel
// parameter (constant bank, broadcast reads) where they fit beside KArgs into
// the 32 KB parameter space.  Otherwise (3D P4: 44 KB in FP32, 87 KB in FP64)
// they are stored after the face tables in the same device buffer and read
// from there through the cache.
struct NoCellTab {};
template <class C>
__host__ __device__ constexpr bool cell_tab_in_param() {
  return sizeof(CellTab<C>) + sizeof(KArgs<C>) <= 32000;
}
template <class C>
using CellTabArg = std::conditional_t<cell_tab_in_param<C>(), CellTab<C>, NoCellTab>;
// byte offset of the cell tables in the face-table buffer
template <class C>
__host__ __device__ constexpr size_t cell_tab_offset() {
  return ((size_t)C::TAB_TOTAL * sizeof(typename C::T) + 255) / 256 * 256;
}
template <class C>
__device__ __forceinline__ const CellTab<C>& cell_tab(const KArgs<C>& a, const CellTabArg<C>& tb) {
  if constexpr (cell_tab_in_param<C>())
    return tb;
  else
    return *reinterpret_cast<const CellTab<C>*>(reinterpret_cast<const unsigned char*>(a.ftab) +
                                                 cell_tab_offset<C>());
}

__device__ __forceinline__ double dt_of(double fixed, double cfl, const unsigned long long* dtmin, int cur) {
  return fixed > 0.0 ? fixed : cfl * __longlong_as_double((long long)dtmin[cur]);
}

// ------------------------------------------------------------------ physics
// Normal flux F.n for an arbitrary (not necessarily unit) vector n, which is
// linear in n: used with unit face normals and with rows of d xi / d x.
// Reciprocal and square root in the arithmetic type.  FP32: the PTX
// approximate instructions rcp.approx.ftz.f32 and sqrt.approx.ftz.f32
// (relative error within about 2^-23), which skip the correction sequences
// of IEEE division and square root; the FP32 path is held to tolerances far
// above that.  FP64: correctly rounded.
__device__ __forceinline__ float arcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double arcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float asqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double asqrt(double x) { return sqrt(x); }

template <int D, int PDE, typename T>
struct Phys;

template <int D, typename T>
struct Phys<D, 0, T> {  // Euler, Eqs. (eulerTerms), (eos)
  static constexpr int NV = D + 2;
  struct Prim {
    T rho, ir, v[D], p, E;
  };
  __device__ __forceinline__ static Prim prim(const T* q, T gamma) {
    Prim s;
    s.rho = q[0];
    s.ir = arcp(q[0]);
    T v2 = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      s.v[a] = q[1 + a] * s.ir;
      v2 += s.v[a] * s.v[a];
    }
    s.E = q[D + 1];
    s.p = (gamma - T(1)) * (s.E - T(0.5) * s.rho * v2);
    return s;
  }
  __device__ __forceinline__ static void fluxn(const T* q, const Prim& s, const T* n, T* Fn) {
    T vn = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) vn += s.v[a] * n[a];
    Fn[0] = s.rho * vn;
#pragma unroll
    for (int k = 0; k < D; ++k) Fn[1 + k] = q[1 + k] * vn + s.p * n[k];
    Fn[D + 1] = vn * (s.E + s.p);
  }
  // largest |eigenvalue| in unit direction n
  __device__ __forceinline__ static T smax(const Prim& s, const T* n, T gamma, T /*ch*/) {
    T vn = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) vn += s.v[a] * n[a];
    const T c2 = gamma * s.p * s.ir;
    return fabs(vn) + asqrt(c2 > T(0) ? c2 : T(0));
  }
  // largest |eigenvalue| over all directions
  __device__ __forceinline__ static T speed(const T* q, T gamma, T /*ch*/) {
    Prim s = prim(q, gamma);
    T v2 = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) v2 += s.v[a] * s.v[a];
    const T c2 = gamma * s.p * s.ir;
    return asqrt(v2) + asqrt(c2 > T(0) ? c2 : T(0));
  }
  __device__ __forceinline__ static T pressure(const T* q, T gamma) {
    T m2 = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) m2 += q[1 + a] * q[1 + a];
    return (gamma - T(1)) * (q[D + 1] - T(0.5) * m2 * arcp(q[0]));
  }
  // Dissipation of the Osher-type flux, Eq. (osher): out = sum_j w_j
  // |A_n(psi_j)| (ur - ul) over the 3-point Gauss-Legendre rule on the path
  // psi(s) = ul + s (ur - ul), unit normal n.  |A_n| dq is formed from the
  // characteristic decomposition at psi: linearised primitive variations
  // (drho, du, dp) of dq, wave strengths of the acoustic (vn -+ c), entropy
  // and shear (vn) waves, each scaled by |eigenvalue| times its right
  // eigenvector.
  __device__ __forceinline__ static void osher_dissipation(const T* ul, const T* ur, const T* n, T gamma, T* out) {
    T dq[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      dq[v] = ur[v] - ul[v];
      out[v] = T(0);
    }
    const T sq = T(0.38729833462074168852);  // sqrt(3/5) / 2
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T sj = T(0.5) + (j == 0 ? -sq : j == 1 ? T(0) : sq);
      const T wj = j == 1 ? T(8.0 / 18.0) : T(5.0 / 18.0);
      T q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = ul[v] + sj * dq[v];
      const T rho = q[0], ir = arcp(q[0]);
      T u[D], u2 = T(0), un = T(0), udm = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        u[a] = q[1 + a] * ir;
        u2 += u[a] * u[a];
        un += u[a] * n[a];
        udm += u[a] * dq[1 + a];
      }
      const T p = (gamma - T(1)) * (q[D + 1] - T(0.5) * rho * u2);
      const T c2 = gamma * p * ir;
      const T c = asqrt(c2 > T(0) ? c2 : T(0));
      const T ic2 = arcp(c2);
      const T H = (q[D + 1] + p) * ir;
      // linearised primitive variations at psi
      const T drho = dq[0];
      T du[D], dun = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        du[a] = (dq[1 + a] - u[a] * drho) * ir;
        dun += du[a] * n[a];
      }
      const T dp = (gamma - T(1)) * (dq[D + 1] - udm + T(0.5) * u2 * drho);
      // wave strengths
      const T am = T(0.5) * (dp - rho * c * dun) * ic2;
      const T ap = T(0.5) * (dp + rho * c * dun) * ic2;
      const T a0 = drho - dp * ic2;
      const T lm = fabs(un - c) * wj, lp = fabs(un + c) * wj, l0 = fabs(un) * wj;
      T dut[D], udut = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        dut[a] = du[a] - dun * n[a];
        udut += u[a] * dut[a];
      }
      out[0] += lm * am + lp * ap + l0 * a0;
#pragma unroll
      for (int a = 0; a < D; ++a)
        out[1 + a] += lm * am * (u[a] - c * n[a]) + lp * ap * (u[a] + c * n[a]) + l0 * (a0 * u[a] + rho * dut[a]);
      out[D + 1] += lm * am * (H - c * un) + lp * ap * (H + c * un) + l0 * (a0 * T(0.5) * u2 + rho * udut);
    }
  }
};

template <int D, typename T>
struct Phys<D, 1, T> {  // ideal MHD + GLM, Eqs. (MHDTerms), (MHDeos), Gaussian units
  static constexpr int NV = 9;
  struct Prim {
    T rho, ir, v[3], B[3], p, pt, E, vB, psi;
  };
  __device__ __forceinline__ static Prim prim(const T* q, T gamma) {
    Prim s;
    s.rho = q[0];
    s.ir = arcp(q[0]);
    T v2 = T(0), B2 = T(0), vB = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s.v[a] = q[1 + a] * s.ir;
      s.B[a] = q[5 + a];
      v2 += s.v[a] * s.v[a];
      B2 += s.B[a] * s.B[a];
      vB += s.v[a] * s.B[a];
    }
    s.E = q[4];
    s.psi = q[8];
    const T i8pi = T(0.039788735772973836);  // 1/(8 pi)
    s.p = (gamma - T(1)) * (s.E - T(0.5) * s.rho * v2 - B2 * i8pi);
    s.pt = s.p + B2 * i8pi;
    s.vB = vB;
    return s;
  }
  __device__ __forceinline__ static void fluxn_ch(const T* q, const Prim& s, const T* n, T* Fn, T ch) {
    const T i4pi = T(0.079577471545947673);  // 1/(4 pi)
    T vn = T(0), Bn = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vn += s.v[a] * n[a];
      Bn += s.B[a] * n[a];
    }
    Fn[0] = s.rho * vn;
#pragma unroll
    for (int k = 0; k < 3; ++k) Fn[1 + k] = q[1 + k] * vn - s.B[k] * Bn * i4pi + (k < D ? s.pt * n[k < D ? k : 0] : T(0));
    Fn[4] = vn * (s.E + s.pt) - Bn * s.vB * i4pi;
#pragma unroll
    for (int k = 0; k < 3; ++k) Fn[5 + k] = vn * s.B[k] - Bn * s.v[k] + (k < D ? s.psi * n[k < D ? k : 0] : T(0));
    Fn[8] = ch * ch * Bn;
  }
  __device__ __forceinline__ static T smax(const Prim& s, const T* n, T gamma, T ch) {
    const T i4pi = T(0.079577471545947673);
    T vn = T(0), Bn = T(0), B2 = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      vn += s.v[a] * n[a];
      Bn += s.B[a] * n[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) B2 += s.B[a] * s.B[a];
    T a2 = gamma * s.p * s.ir, b2 = B2 * i4pi * s.ir, bn2 = Bn * Bn * i4pi * s.ir;
    T sum = a2 + b2;
    T disc = sum * sum - T(4) * a2 * bn2;
    disc = disc > T(0) ? disc : T(0);
    T cf2 = T(0.5) * (sum + asqrt(disc));
    T cf = asqrt(cf2 > T(0) ? cf2 : T(0));
    T sp = fabs(vn) + cf;
    return sp > ch ? sp : ch;
  }
  __device__ __forceinline__ static T speed(const T* q, T gamma, T ch) {
    const T i4pi = T(0.079577471545947673);
    Prim s = prim(q, gamma);
    T v2 = T(0), B2 = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      v2 += s.v[a] * s.v[a];
      B2 += s.B[a] * s.B[a];
    }
    T f2 = gamma * s.p * s.ir + B2 * i4pi * s.ir;
    T sp = asqrt(v2) + asqrt(f2 > T(0) ? f2 : T(0));
    return sp > ch ? sp : ch;
  }
  __device__ __forceinline__ static T pressure(const T* q, T gamma) {
    const T i8pi = T(0.039788735772973836);
    T m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    T B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
    return (gamma - T(1)) * (q[4] - T(0.5) * m2 * arcp(q[0]) - B2 * i8pi);
  }
};

template <int D, int PDE, typename T>
__device__ __forceinline__ void flux_normal(const T* q, const typename Phys<D, PDE, T>::Prim& s, const T* n, T* Fn,
                                            T ch) {
  if constexpr (PDE == 0) {
    Phys<D, 0, T>::fluxn(q, s, n, Fn);
  } else {
    Phys<D, 1, T>::fluxn_ch(q, s, n, Fn, ch);
  }
}

// --------------------------------------------------- state access helpers
// The FP32 pairs (hi, lo) of cell j, NVP / 2 16-byte vectors (layout.h)
template <class C>
__device__ __forceinline__ void load_pairs(const float* __restrict__ Qp, int64_t j, float* hi, float* lo) {
  const float4* p = reinterpret_cast<const float4*>(Qp) + j * (C::NVP / 2);
#pragma unroll
  for (int m = 0; m < C::NVP / 2; ++m) {
    const float4 x = __ldg(p + m);
    hi[2 * m] = x.x;
    lo[2 * m] = x.y;
    if (2 * m + 1 < C::NV) {
      hi[2 * m + 1] = x.z;
      lo[2 * m + 1] = x.w;
    }
  }
}

template <class C>
__device__ __forceinline__ void load_state(const KArgs<C>& a, int64_t i, typename C::T* q,
                                           typename C::T* lo) {
  using T = typename C::T;
  if constexpr (std::is_same<T, double>::value) {
#pragma unroll
    for (int v = 0; v < C::NV; ++v) {
      q[v] = a.Q[v * a.N + i];
      lo[v] = 0.0;
    }
  } else {
    load_pairs<C>(a.Qp, i, q, lo);
  }
}

// dq = Q_j - Q_i, formed from the FP32 hi/lo split in mixed mode (the hi
// difference of nearby values is exact, the lo part restores FP64 accuracy)
template <class C>
__device__ __forceinline__ void load_diff(const KArgs<C>& a, int64_t j, const typename C::T* qi,
                                          const typename C::T* qilo, typename C::T* dq) {
  using T = typename C::T;
  if constexpr (std::is_same<T, double>::value) {
#pragma unroll
    for (int v = 0; v < C::NV; ++v) dq[v] = a.Q[v * a.N + j] - qi[v];
  } else {
    float hj[C::NV], lj[C::NV];
    load_pairs<C>(a.Qp, j, hj, lj);
#pragma unroll
    for (int v = 0; v < C::NV; ++v) dq[v] = (hj[v] - qi[v]) + (lj[v] - qilo[v]);
  }
}

template <typename T>
__device__ __forceinline__ T pow4(T x) {
  T y = x * x;
  return y * y;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  __device__ __forceinline__ static float get(const float4& x, int j) {
    return j == 0 ? x.x : j == 1 ? x.y : j == 2 ? x.z : x.w;
  }
  __device__ __forceinline__ static float4 make(const float* a) { return make_float4(a[0], a[1], a[2], a[3]); }
};
template <>
struct Vec16<double> {
  using V = double2;
  __device__ __forceinline__ static double get(const double2& x, int j) { return j == 0 ? x.x : x.y; }
  __device__ __forceinline__ static double2 make(const double* a) { return make_double2(a[0], a[1]); }
};

// The NV values of one space-time node of one cell are contiguous in q_hat
// ([node][cell][var]); with NV * sizeof(T) a multiple of 16 bytes they move
// as 128-bit accesses (coalesced across consecutive cells of a warp).
template <int NV, typename T>
__device__ __forceinline__ void load_node(const T* __restrict__ p, T* out) {
  if constexpr ((NV * sizeof(T)) % 16 == 0) {
    using V = typename Vec16<T>::V;
    constexpr int W = 16 / sizeof(T);
#pragma unroll
    for (int k = 0; k < NV / W; ++k) {
      const V x = __ldg(reinterpret_cast<const V*>(p) + k);
#pragma unroll
      for (int j = 0; j < W; ++j) out[k * W + j] = Vec16<T>::get(x, j);
    }
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = __ldg(p + v);
  }
}

template <int NV, typename T>
__device__ __forceinline__ void store_node(T* __restrict__ p, const T* in) {
  if constexpr ((NV * sizeof(T)) % 16 == 0) {
    using V = typename Vec16<T>::V;
    constexpr int W = 16 / sizeof(T);
#pragma unroll
    for (int k = 0; k < NV / W; ++k) reinterpret_cast<V*>(p)[k] = Vec16<T>::make(in + k * W);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) p[v] = in[v];
  }
}

// ---------------------------------------------------------- rec + predictor
// Positivity scaling toward the cell average (switchable; an addition to the
// paper, the Zhang-Shu scaling limiter): density first, then the pressure,
// both kept above 1e-3 of their cell-average values at every lattice node
// (well above FP32 rounding of Qbar + theta (w - Qbar), and high enough that
// a scaled node cannot reach near-vacuum with a finite momentum, whose
// velocity the cell-average time step would not see); density and pressure
// are concave in the conserved state.  dev(n, v) is the reconstruction's
// deviation from the cell average qb at lattice node n; returns the factor
// theta in (0, 1] that scales it.
template <class C, class Dev>
__device__ __forceinline__ typename C::T positivity_theta(const KArgs<C>& a, const typename C::T* qb, Dev dev) {
  using T = typename C::T;
  constexpr int NV = C::NV;
  using PH = Phys<C::D, C::PDE, T>;
  const T fl = T(1e-3);
  const T rb = qb[0];
  T th = T(1);
#pragma unroll 1
  for (int n = 0; n < C::L0; ++n) {
    const T r = qb[0] + dev(n, 0);
    if (r < fl * rb) {
      const T t = (rb - fl * rb) / (rb - r);
      th = t < th ? t : th;
    }
  }
  const T pb = PH::pressure(qb, a.gamma);
  T thp = T(1);
  if (pb > T(0)) {
#pragma unroll 1
    for (int n = 0; n < C::L0; ++n) {
      T q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = qb[v] + th * dev(n, v);
      if (!(q[0] > T(0))) {
        thp = T(0);
        continue;
      }
      const T pk = PH::pressure(q, a.gamma);
      if (pk < fl * pb) {
        const T t = (pb - fl * pb) / (pb - pk);
        thp = t < thp ? t : thp;
      }
    }
  }
  return th * thp;
}

// One cell: reconstruction, then (unless REC_ONLY) the predictor.
template <class C, bool REC_ONLY>
__device__ __forceinline__ void rec_pred_cell(const KArgs<C>& a, const CellTab<C>& tb, int64_t i) {
  using T = typename C::T;
  constexpr int D = C::D, NV = C::NV, MC1 = C::MC1, NE1 = C::NE - 1, NS = C::NS;
  using PH = Phys<D, C::PDE, T>;
  const int64_t N = a.N;
  if (i >= N) return;

  T qi[NV], qlo[NV];
  load_state<C>(a, i, qi, qlo);

  // ---- P_opt: c = R dQ over the central stencil (constant part is Q_i).
  // Neighbours in chunks of four: one 16-byte vector of ids, whole 16-byte
  // vectors of R (layout.h), four neighbours' differences, then the FMAs.
  T c[MC1][NV];
#pragma unroll
  for (int l = 0; l < MC1; ++l)
#pragma unroll
    for (int v = 0; v < NV; ++v) c[l][v] = T(0);
  {
    using V = typename Vec16<T>::V;
    constexpr int VW = C::VW, NFULL = NE1 / 4, TAIL = NE1 % 4, GPC = 4 * MC1 / VW;
    const V* Rv = reinterpret_cast<const V*>(a.R);
    const int4* S4 = reinterpret_cast<const int4*>(a.sten4);
    // with IDS_AHEAD the id vector of the next chunk is loaded while the
    // current one is in use, so a chunk's gathers wait one round trip, not two
    int4 idn = __ldg(S4 + i);
    auto chunk = [&](int ch, auto nn) {
      constexpr int NN = decltype(nn)::value;
      constexpr int NG = (NN * MC1 + VW - 1) / VW;
      int4 id;
      if constexpr (C::IDS_AHEAD) {
        id = idn;
        if (ch + 1 < sten_vectors(NE1)) idn = __ldg(S4 + (int64_t)(ch + 1) * N + i);
      } else {
        id = __ldg(S4 + (int64_t)ch * N + i);
      }
      const int ids[4] = {id.x, id.y, id.z, id.w};
      T dq[NN][NV];
#pragma unroll
      for (int rr = 0; rr < NN; ++rr) load_diff<C>(a, ids[rr], qi, qlo, dq[rr]);
      T r[NG * VW];
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const V x = __ldg(Rv + (int64_t)(ch * GPC + g) * N + i);
#pragma unroll
        for (int j = 0; j < VW; ++j) r[g * VW + j] = Vec16<T>::get(x, j);
      }
#pragma unroll
      for (int rr = 0; rr < NN; ++rr)
#pragma unroll
        for (int l = 0; l < MC1; ++l)
#pragma unroll
          for (int v = 0; v < NV; ++v) c[l][v] += r[rr * MC1 + l] * dq[rr][v];
    };
#pragma unroll(C::GATHER_CHUNKS)
    for (int ch = 0; ch < NFULL; ++ch) chunk(ch, std::integral_constant<int, 4>());
    if constexpr (TAIL > 0) chunk(NFULL, std::integral_constant<int, TAIL>());
  }

  // ---- sectorial polynomials: g_s = B_s^{-1} dQ_sector
  T g[NS][D][NV];
  bool keep[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int64_t j0 = __ldg(a.sec + (s * D) * N + i);
    keep[s] = j0 >= 0;
#pragma unroll
    for (int e = 0; e < D; ++e)
#pragma unroll
      for (int v = 0; v < NV; ++v) g[s][e][v] = T(0);
    if (keep[s]) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int64_t j = __ldg(a.sec + (s * D + k) * N + i);
        T dq[NV];
        load_diff<C>(a, j, qi, qlo, dq);
#pragma unroll
        for (int e = 0; e < D; ++e) {
          const T b = __ldg(a.Binv + (int64_t)((s * D + e) * D + k) * N + i);
#pragma unroll
          for (int v = 0; v < NV; ++v) g[s][e][v] += b * dq[v];
        }
      }
    }
  }

  // ---- linear weights (normalised over kept stencils), P_0, indicators, weights
  const int ns = a.nsec[i];
  const T lden = arcp(a.lam0 + T(ns) * a.lams);
  const T lam0 = a.lam0 * lden, lams = a.lams * lden;
  const T ilam0 = arcp(lam0);
  T w[MC1][NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    T p0[MC1];
#pragma unroll
    for (int l = 0; l < MC1; ++l) {
      T s = c[l][v];
      if (l < D) {
#pragma unroll
        for (int sc = 0; sc < NS; ++sc) s -= (keep[sc] ? lams : T(0)) * g[sc][l < D ? l : 0][v];
      }
      p0[l] = s * ilam0;
    }
    // sigma = p^T Sigma p in the symmetric form: sum over l of p_l (Sigma_ll
    // p_l + sum over m > l of 2 Sigma_lm p_m)
    T sig0 = T(0);
#pragma unroll
    for (int l = 0; l < MC1; ++l) {
      T t = tb.Sig[l][l] * p0[l];
#pragma unroll
      for (int m = l + 1; m < MC1; ++m) t += tb.Sig[l][m] * p0[m];
      sig0 += p0[l] * t;
    }
    T sig[NS];
    T smin = sig0;
#pragma unroll
    for (int sc = 0; sc < NS; ++sc) {
      T s = T(0);
#pragma unroll
      for (int l = 0; l < D; ++l) {
        T t = tb.Sig[l][l] * g[sc][l][v];
#pragma unroll
        for (int m = l + 1; m < D; ++m) t += tb.Sig[l][m] * g[sc][m][v];
        s += g[sc][l][v] * t;
      }
      sig[sc] = s;
      if (keep[sc] && s < smin) smin = s;
    }
    // omega_s proportional to lambda_s / (sigma_s + eps)^4, scaled by
    // (sigma_min + eps)^4 so that nothing overflows in FP32
    const T num = smin + a.eps;
    T w0 = a.linw ? lam0 : lam0 * pow4(num * arcp(sig0 + a.eps));
    T ws[NS];
    T tot = w0;
#pragma unroll
    for (int sc = 0; sc < NS; ++sc) {
      ws[sc] = keep[sc] ? (a.linw ? lams : lams * pow4(num * arcp(sig[sc] + a.eps))) : T(0);
      tot += ws[sc];
    }
    const T itot = arcp(tot);
    w0 *= itot;
#pragma unroll
    for (int sc = 0; sc < NS; ++sc) ws[sc] *= itot;
#pragma unroll
    for (int l = 0; l < MC1; ++l) {
      T s = w0 * p0[l];
      if (l < D) {
#pragma unroll
        for (int sc = 0; sc < NS; ++sc) s += ws[sc] * g[sc][l < D ? l : 0][v];
      }
      w[l][v] = s;
    }
  }

  T qbar[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) qbar[v] = qi[v] + qlo[v];
  if constexpr (REC_ONLY) {
    if (a.pos) {
      const T theta = positivity_theta<C>(a, qbar, [&](int n, int v) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < MC1; ++l) s += tb.E[n][l] * w[l][v];
        return s;
      });
      if (theta < T(1)) {
#pragma unroll
        for (int l = 0; l < MC1; ++l)
#pragma unroll
          for (int v = 0; v < NV; ++v) w[l][v] *= theta;
      }
    }
    // reconstruction values at the lattice nodes, caller's cell order; in
    // FP32-mixed mode the FP32 deviation is added to the FP64 cell average
    // (hi + lo in FP64), so the deviation stays recoverable to FP32 accuracy
    const int64_t u = a.perm[i];
#pragma unroll
    for (int n = 0; n < C::L0; ++n)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if constexpr (std::is_same<T, float>::value) {
          T s = T(0);
#pragma unroll
          for (int l = 0; l < MC1; ++l) s += tb.E[n][l] * w[l][v];
          a.out[(u * C::MC + n) * NV + v] = ((double)qi[v] + (double)qlo[v]) + (double)s;
        } else {
          T s = qbar[v];
#pragma unroll
          for (int l = 0; l < MC1; ++l) s += tb.E[n][l] * w[l][v];
          a.out[(u * C::MC + n) * NV + v] = (double)s;
        }
      }
    return;
  } else {
    // B: stride between the entries of one thread's working set (128
    // columns in shared memory, or contiguous in local memory)
    constexpr int L0 = C::L0, L1 = C::L1, B = C::PRED_WS_LOCAL ? 1 : 128;
    extern __shared__ __align__(16) unsigned char rp_smem[];
    T ws_local[C::PRED_WS_LOCAL ? 2 * L1 * NV : 1];
    T* sb = C::PRED_WS_LOCAL ? ws_local : reinterpret_cast<T*>(rp_smem) + threadIdx.x;  // fixed part, [(k NV + v) B]
    T* sq = sb + L1 * NV * B;                              // current iterate
    // With STASH, the reconstruction at the L0 lattice nodes (E w, deviation
    // from the cell average) is formed once into the working set: the
    // positivity scaling, the tau = 0 nodes of the predictor and its known
    // part read it.  The known part C0 q0 needs no arithmetic: on the
    // principal lattice every unknown node lies above a tau = 0 node
    // (tb.sel), where C0 = theta_n(xi_k, 0) is 1, and 0 elsewhere.
    constexpr bool STASH = C::STASH;
    T* sw = sb;  // [(n NV + v) B], n < L0
    T theta = T(1);
    if constexpr (STASH) {
#pragma unroll 1
      for (int n = 0; n < L0; ++n)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T s = T(0);
#pragma unroll
          for (int l = 0; l < MC1; ++l) s += tb.E[n][l] * w[l][v];
          sw[(n * NV + v) * B] = s;
        }
      if (a.pos) theta = positivity_theta<C>(a, qbar, [&](int n, int v) { return sw[(n * NV + v) * B]; });
    } else if (a.pos) {
      theta = positivity_theta<C>(a, qbar, [&](int n, int v) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < MC1; ++l) s += tb.E[n][l] * w[l][v];
        return s;
      });
      if (theta < T(1)) {
#pragma unroll
        for (int l = 0; l < MC1; ++l)
#pragma unroll
          for (int v = 0; v < NV; ++v) w[l][v] *= theta;
      }
    }
    // dt is folded into the inverse Jacobian: G_e = F . (dt d xi_e / d x) is
    // linear in the direction, so the scaled directions give dt G_e directly
    const T dt = (T)dt_of(a.dt_fixed, a.cfl, a.dtmin, a.cur);
    T J[D][D];
#pragma unroll
    for (int e = 0; e < D; ++e)
#pragma unroll
      for (int m = 0; m < D; ++m) J[e][m] = dt * __ldg(a.Jinv + (e * D + m) * N + i);
    // Deviations from the cell average: the Picard update subtracts the flux
    // of the cell average, G_e(q) - G_e(Qbar), which P_e annihilates exactly
    // (it differentiates constants to zero); q_hat is stored as q - Qbar.  The
    // arithmetic is identical in exact arithmetic, and constant states stay
    // exactly constant in FP32.
    const T* qb = qbar;
    T Gref[D][NV];
    {
      typename PH::Prim pr = PH::prim(qb, a.gamma);
#pragma unroll
      for (int e = 0; e < D; ++e) flux_normal<D, C::PDE, T>(qb, pr, J[e], Gref[e], a.ch);
    }
    // flux part of the fixed term, -sum_e P_e[:, tau=0 nodes] dt (G_e(q0) - G_e(Qbar));
    // with TAU0_SPARSE the node loop is unrolled and the exact zeros of P_e
    // in the tau = 0 columns are skipped at compile time
    T S[L1][NV];
#pragma unroll
    for (int k = 0; k < L1; ++k)
#pragma unroll
      for (int v = 0; v < NV; ++v) S[k][v] = T(0);
#pragma unroll(C::TAU0_SPARSE ? C::L0 : 1)
    for (int n = 0; n < L0; ++n) {
      T dq0[NV], q0[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T s;
        if constexpr (STASH) {
          s = theta * sw[(n * NV + v) * B];
        } else {
          s = T(0);
#pragma unroll
          for (int l = 0; l < MC1; ++l) s += tb.E[n][l] * w[l][v];
        }
        dq0[v] = s;
        q0[v] = qb[v] + s;
      }
      store_node<NV, T>(a.qhat + ((int64_t)n * N + i) * NV, dq0);
      typename PH::Prim pr = PH::prim(q0, a.gamma);
      T Ge[D][NV];
#pragma unroll
      for (int e = 0; e < D; ++e) {
        flux_normal<D, C::PDE, T>(q0, pr, J[e], Ge[e], a.ch);
#pragma unroll
        for (int v = 0; v < NV; ++v) Ge[e][v] -= Gref[e][v];
      }
#pragma unroll
      for (int k = 0; k < L1; ++k)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T b = S[k][v];
#pragma unroll
          for (int e = 0; e < D; ++e)
            if (!C::TAU0_SPARSE || PredPattern<D, C::M>::nz(e, k, n)) b -= tb.P[e][k][n] * Ge[e][v];
          S[k][v] = b;
        }
    }
    // known part C0 q0, also the initial guess (deviation of the unknown
    // nodes from Qbar); with STASH read from the stash into registers before
    // the working set is overwritten
    if constexpr (STASH) {
      T c0[L1][NV];
#pragma unroll
      for (int k = 0; k < L1; ++k)
#pragma unroll
        for (int v = 0; v < NV; ++v) c0[k][v] = theta * sw[(tb.sel[k] * NV + v) * B];
#pragma unroll
      for (int k = 0; k < L1; ++k)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          sq[(k * NV + v) * B] = c0[k][v];
          sb[(k * NV + v) * B] = c0[k][v] + S[k][v];
        }
    } else {
#pragma unroll
      for (int k = 0; k < L1; ++k)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T c0 = T(0);
#pragma unroll
          for (int l = 0; l < MC1; ++l) c0 += tb.CE[k][l] * w[l][v];
          sq[(k * NV + v) * B] = c0;
          sb[(k * NV + v) * B] = c0 + S[k][v];
        }
    }
    // Picard iterations of Eq. (CGfinal), on deviations
    for (int it = 0; it < a.niter; ++it) {
      T nq[L1][NV];
#pragma unroll
      for (int k = 0; k < L1; ++k)
#pragma unroll
        for (int v = 0; v < NV; ++v) nq[k][v] = sb[(k * NV + v) * B];
      // with PRED_SPARSE the loop is unrolled over the nodes, so the exact
      // zeros of P_e (half to two thirds of the entries, pred_pattern.h) are
      // skipped at compile time and the rest are immediate operands
#pragma unroll(C::PRED_SPARSE ? C::L1 : 1)
      for (int l = 0; l < L1; ++l) {
        T ql[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) ql[v] = qb[v] + sq[(l * NV + v) * B];
        typename PH::Prim pr = PH::prim(ql, a.gamma);
        T Ge[D][NV];
#pragma unroll
        for (int e = 0; e < D; ++e) {
          flux_normal<D, C::PDE, T>(ql, pr, J[e], Ge[e], a.ch);
#pragma unroll
          for (int v = 0; v < NV; ++v) Ge[e][v] -= Gref[e][v];
        }
#pragma unroll
        for (int k = 0; k < L1; ++k)
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            T s = nq[k][v];
#pragma unroll
            for (int e = 0; e < D; ++e)
              if (!C::PRED_SPARSE || PredPattern<D, C::M>::nz(e, k, L0 + l)) s -= tb.P[e][k][L0 + l] * Ge[e][v];
            nq[k][v] = s;
          }
      }
#pragma unroll
      for (int k = 0; k < L1; ++k)
#pragma unroll
        for (int v = 0; v < NV; ++v) sq[(k * NV + v) * B] = nq[k][v];
    }
    // predictor fallback (with the positivity switch; an addition to the
    // paper): a space-time node outside the admissible set (density or
    // pressure <= 0, or not finite) makes the cell's predictor its cell
    // average at every node.  A lattice node scaled close to vacuum can carry
    // a wave speed far above the cell average's, which the time step of Eq.
    // (timestep) does not see.
    bool admissible = true;
    if (a.pos) {
#pragma unroll 1
      for (int k = 0; k < L1; ++k) {
        T q[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) q[v] = qb[v] + sq[(k * NV + v) * B];
        const T pk = PH::pressure(q, a.gamma);
        if (!(q[0] > T(0) && pk > T(0) && isfinite(pk))) admissible = false;
      }
    }
    if (admissible) {
#pragma unroll 1
      for (int k = 0; k < L1; ++k) {
        T q1[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) q1[v] = sq[(k * NV + v) * B];
        store_node<NV, T>(a.qhat + ((int64_t)(L0 + k) * N + i) * NV, q1);
      }
    } else {
      T z[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) z[v] = T(0);
#pragma unroll 1
      for (int l = 0; l < C::L; ++l) store_node<NV, T>(a.qhat + ((int64_t)l * N + i) * NV, z);
    }
  }
}

// One thread per cell, one block per tile of 128 consecutive cells.
template <class C, bool REC_ONLY>
__global__ void __launch_bounds__(128, C::REC_MINB) k_rec_pred(KArgs<C> a, const __grid_constant__ CellTabArg<C> tb) {
  if (!REC_ONLY && a.reset_next && blockIdx.x == 0 && threadIdx.x == 0) a.dtmin[1 - a.cur] = 0x7ff0000000000000ull;
  rec_pred_cell<C, REC_ONLY>(a, cell_tab<C>(a, tb), (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ----------------------------------------------------------------- fluxes
template <class C>
__device__ __forceinline__ void load_chunk(const typename C::T* __restrict__ qhat, int64_t c, int64_t N, int l4,
                                           typename C::T (&ql)[C::VW][C::NV]) {
  using T = typename C::T;
#pragma unroll
  for (int j = 0; j < C::VW; ++j) {
    if (l4 + j < C::L) {
      load_node<C::NV, T>(qhat + ((int64_t)(l4 + j) * N + c) * C::NV, ql[j]);
    } else {
#pragma unroll
      for (int v = 0; v < C::NV; ++v) ql[j][v] = T(0);
    }
  }
}

// Predictor deviations of cell c at NPT consecutive rows (space-time points)
// of its face table, starting at row r0: tr[j][v] += theta_l(point) q_hat_l[v].
// Basis values are read from the padded table as 16-byte vectors, VW nodes
// at a time; with TR_PREFETCH the next chunk of nodes is in flight while the
// current one is used.
template <class C, int NPT>
__device__ __forceinline__ void face_traces(const typename C::T* __restrict__ qhat, int64_t c, int64_t N,
                                            const typename C::T* tcode, int r0, typename C::T (&tr)[NPT][C::NV]) {
  using T = typename C::T;
  using V = typename Vec16<T>::V;
  constexpr int NV = C::NV, L = C::L, LP = C::LP, VW = C::VW;
  T nx[VW][NV];
  if constexpr (C::TR_PREFETCH) load_chunk<C>(qhat, c, N, 0, nx);
#pragma unroll 1
  for (int l4 = 0; l4 < LP; l4 += VW) {
    T ql[VW][NV];
    if constexpr (C::TR_PREFETCH) {
#pragma unroll
      for (int j = 0; j < VW; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) ql[j][v] = nx[j][v];
      if (l4 + VW < LP) load_chunk<C>(qhat, c, N, l4 + VW, nx);
    } else {
      load_chunk<C>(qhat, c, N, l4, ql);
    }
#pragma unroll
    for (int jq = 0; jq < NPT; ++jq) {
      const V th = *reinterpret_cast<const V*>(tcode + (r0 + jq) * LP + l4);
#pragma unroll
      for (int j = 0; j < VW; ++j) {
        if (l4 + j < L) {
          const T tj = Vec16<T>::get(th, j);
#pragma unroll
          for (int v = 0; v < NV; ++v) tr[jq][v] += tj * ql[j][v];
        }
      }
    }
  }
}

// Numerical flux at one space-time point with quadrature weight wgt, from
// the traces ul, ur (cell average + deviation) of both sides:
// facc[m] += wgt (F_m(u-) + F_m(u+)) per direction m, and dacc += wgt s
// (u+ - u-), s the larger of the two sides' maximal signal speeds along n
// (Rusanov, Eq. rusanov), or dacc += wgt int_0^1 |A_n(psi)| ds (u+ - u-)
// (Osher-type, Eq. osher; Euler).  A trace that
// is not an admissible state (density or pressure <= 0) is replaced by its
// cell average at this point (positivity safeguard, with the scaling of the
// reconstruction).
template <class C, bool OSHER>
__device__ __forceinline__ void rusanov_point(const KArgs<C>& a, typename C::T* ul, typename C::T* ur,
                                              const typename C::T* qbL, const typename C::T* qbR,
                                              const typename C::T* n, typename C::T wgt,
                                              typename C::T (&facc)[C::D][C::NV], typename C::T (&dacc)[C::NV]) {
  using T = typename C::T;
  constexpr int D = C::D, NV = C::NV;
  using PH = Phys<D, C::PDE, T>;
  typename PH::Prim pl = PH::prim(ul, a.gamma);
  typename PH::Prim pr = PH::prim(ur, a.gamma);
  if (a.pos) {
    if (!(ul[0] > T(0) && pl.p > T(0))) {
#pragma unroll
      for (int v = 0; v < NV; ++v) ul[v] = qbL[v];
      pl = PH::prim(ul, a.gamma);
    }
    if (!(ur[0] > T(0) && pr.p > T(0))) {
#pragma unroll
      for (int v = 0; v < NV; ++v) ur[v] = qbR[v];
      pr = PH::prim(ur, a.gamma);
    }
  }
#pragma unroll
  for (int m = 0; m < D; ++m) {
    T em[D];
#pragma unroll
    for (int e = 0; e < D; ++e) em[e] = e == m ? T(1) : T(0);
    T fl[NV], fr[NV];
    flux_normal<D, C::PDE, T>(ul, pl, em, fl, a.ch);
    flux_normal<D, C::PDE, T>(ur, pr, em, fr, a.ch);
#pragma unroll
    for (int v = 0; v < NV; ++v) facc[m][v] += wgt * (fl[v] + fr[v]);
  }
  if constexpr (OSHER && C::PDE == 0) {  // Osher-type, Eq. (osher)
    T dis[NV];
    PH::osher_dissipation(ul, ur, n, a.gamma, dis);
#pragma unroll
    for (int v = 0; v < NV; ++v) dacc[v] += wgt * dis[v];
    return;
  }
  const T sl = PH::smax(pl, n, a.gamma, a.ch), sr = PH::smax(pr, n, a.gamma, a.ch);
  const T s = sl > sr ? sl : sr;
  const T ws = wgt * s;
#pragma unroll
  for (int v = 0; v < NV; ++v) dacc[v] += ws * (ur[v] - ul[v]);
}

// G_f = 1/2 dt (sum_m |f| n_m facc[m] - |f| dacc), contracted in FP64 so that
// a constant state gives bit-identical sums on every face and the update
// closes
template <class C>
__device__ __forceinline__ void store_face_integral(const KArgs<C>& a, int64_t f, double dtd,
                                                    const typename C::T (&facc)[C::D][C::NV],
                                                    const typename C::T (&dacc)[C::NV]) {
  double fa[C::D];
#pragma unroll
  for (int m = 0; m < C::D; ++m) fa[m] = a.fa[m * a.F + f];
  const double area = a.farea[f];
#pragma unroll
  for (int v = 0; v < C::NV; ++v) {
    double g = -area * (double)dacc[v];
#pragma unroll
    for (int m = 0; m < C::D; ++m) g += fa[m] * (double)facc[m][v];
    a.G[v * a.F + f] = 0.5 * dtd * g;
  }
}

template <class C>
__device__ __forceinline__ const typename C::T* face_tables(const KArgs<C>& a, int use_smem, unsigned char* smem_raw) {
  using T = typename C::T;
  if (!use_smem) return a.ftab;
  T* st = reinterpret_cast<T*>(smem_raw);
  for (int k = threadIdx.x; k < C::TABN + C::NQS + C::NQT; k += blockDim.x) st[k] = a.ftab[k];
  __syncthreads();
  return st;
}

template <class C>
__device__ __forceinline__ void cell_average(const KArgs<C>& a, int64_t c, typename C::T* qb) {
  if constexpr (std::is_same<typename C::T, double>::value) {
#pragma unroll
    for (int v = 0; v < C::NV; ++v) qb[v] = a.Q[v * a.N + c];
  } else {
    float hi[C::NV], lo[C::NV];
    load_pairs<C>(a.Qp, c, hi, lo);
#pragma unroll
    for (int v = 0; v < C::NV; ++v) qb[v] = hi[v] + lo[v];
  }
}

// One face, one thread: both sides' traces one time point at a time (NQS
// space points), Rusanov flux, space-time quadrature.  `tab` holds the face
// tables, then the space and time quadrature weights.
template <class C, bool OSHER>
__device__ __forceinline__ void flux_one_face(const KArgs<C>& a, const typename C::T* tab, int64_t f, double dtd) {
  using T = typename C::T;
  constexpr int D = C::D, NV = C::NV, NQS = C::NQS, NQT = C::NQT;
  const T* wq = tab + C::TABN;
  const T* wt = wq + NQS;
  const int64_t N = a.N, F = a.F;
  {
    const int64_t Lc = a.fL[f];
    const int64_t Rc = a.fR[f];
    const T* tL = tab + (int)a.codeL[f] * C::CODE_STRIDE;
    const T* tR = tab + (int)a.codeR[f] * C::CODE_STRIDE;
    T n[D];
#pragma unroll
    for (int e = 0; e < D; ++e) n[e] = a.fn[e * F + f];
    // cell averages of both sides: q_hat holds deviations from them
    T qbL[NV], qbR[NV];
    cell_average<C>(a, Lc, qbL);
    if (Rc >= 0) {
      cell_average<C>(a, Rc, qbR);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) qbR[v] = qbL[v];
    }
    T facc[D][NV], dacc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      dacc[v] = T(0);
#pragma unroll
      for (int m = 0; m < D; ++m) facc[m][v] = T(0);
    }
#pragma unroll 1
    for (int t = 0; t < NQT; ++t) {
      T trL[NQS][NV], trR[NQS][NV];
#pragma unroll
      for (int j = 0; j < NQS; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          trL[j][v] = T(0);
          trR[j][v] = T(0);
        }
      face_traces<C, NQS>(a.qhat, Lc, N, tL, t * NQS, trL);
      if (Rc >= 0) {
        face_traces<C, NQS>(a.qhat, Rc, N, tR, t * NQS, trR);
      } else {
#pragma unroll
        for (int j = 0; j < NQS; ++j)
#pragma unroll
          for (int v = 0; v < NV; ++v) trR[j][v] = trL[j][v];  // transmissive
      }
#pragma unroll
      for (int j = 0; j < NQS; ++j) {
        T ul[NV], ur[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          ul[v] = qbL[v] + trL[j][v];
          ur[v] = qbR[v] + trR[j][v];
        }
        rusanov_point<C, OSHER>(a, ul, ur, qbL, qbR, n, wq[j] * wt[t], facc, dacc);
      }
    }
    store_face_integral<C>(a, f, dtd, facc, dacc);
  }
}

// One thread per face, persistent grid.
template <class C, bool OSHER>
__global__ void __launch_bounds__(128, C::FLUX_MINB) k_flux(KArgs<C> a, int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const typename C::T* tab = face_tables<C>(a, use_smem, smem_raw);
  const double dtd = dt_of(a.dt_fixed, a.cfl, a.dtmin, a.cur);
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < a.F; f += (int64_t)gridDim.x * blockDim.x)
    flux_one_face<C, OSHER>(a, tab, f, dtd);
}

// 2 SPLIT threads per face (consecutive lanes), persistent grid.  Lane bit 0
// is the side; the higher bits pick one of SPLIT groups of the NQT x NQS
// space-time points (in time order).  Each thread evaluates its own side's
// traces at its group's points from one pass over that cell's q_hat (or
// PAIR_PASSES passes); the two sides of a group swap traces by warp
// shuffles, each thread takes every other point for the numerical flux, and
// the partial sums of the face's threads are added.  A boundary face
// evaluates its inner cell on both sides (transmissive: the outer trace
// equals the inner one).
// One block iteration of the pair kernel: the 128 threads starting at
// thread index g0 of the face space (TPF threads per face).  `tab` holds the
// face tables, then the space and time quadrature weights.
// The cell and face code a thread of the pair kernel works on at thread base
// g0 (its own side; a boundary face evaluates its inner cell on both sides)
struct PairSide {
  int32_t c, code;
};
template <class C>
__device__ __forceinline__ PairSide pair_side(const KArgs<C>& a, int64_t g0) {
  constexpr int TPF = 2 * C::FLUX_SPLIT;
  const int64_t fg = (g0 + threadIdx.x) / TPF;
  const int64_t f = fg < a.F ? fg : a.F - 1;
  const int32_t Lc = a.fL[f], Rc = a.fR[f];
  const bool own_left = (threadIdx.x & 1) == 0 || Rc < 0;
  return PairSide{own_left ? Lc : Rc, (int32_t)(own_left ? a.codeL[f] : a.codeR[f])};
}

template <class C, bool OSHER>
__device__ __forceinline__ void flux_pair_iter(const KArgs<C>& a, const typename C::T* tab, int64_t g0, double dtd,
                                               PairSide ps) {
  using T = typename C::T;
  constexpr int D = C::D, NV = C::NV, NQS = C::NQS, NP = C::NQT * C::NQS;
  constexpr int SPLIT = C::FLUX_SPLIT, TPF = 2 * SPLIT;
  static_assert(NP % (SPLIT * C::PAIR_PASSES) == 0, "points must divide over the groups and passes");
  const T* wq = tab + C::TABN;
  const T* wt = wq + NQS;
  const int64_t N = a.N, F = a.F;
  const int side = (int)(threadIdx.x & 1);
  const int grp = (int)(threadIdx.x >> 1) & (SPLIT - 1);
  {
    const int64_t fg = (g0 + threadIdx.x) / TPF;
    const bool valid = fg < F;
    const int64_t f = valid ? fg : F - 1;
    const int64_t c = ps.c;
    const T* tc = tab + ps.code * C::CODE_STRIDE;
    T n[D];
#pragma unroll
    for (int e = 0; e < D; ++e) n[e] = a.fn[e * F + f];
    T qb[NV], qo[NV];
    cell_average<C>(a, c, qb);
#pragma unroll
    for (int v = 0; v < NV; ++v) qo[v] = __shfl_xor_sync(0xffffffffu, qb[v], 1);
    const T* qbL = side == 0 ? qb : qo;
    const T* qbR = side == 0 ? qo : qb;
    T facc[D][NV], dacc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      dacc[v] = T(0);
#pragma unroll
      for (int m = 0; m < D; ++m) facc[m][v] = T(0);
    }
    constexpr int NPP = NP / (SPLIT * C::PAIR_PASSES);
#pragma unroll 1
    for (int h = 0; h < C::PAIR_PASSES; ++h) {
      const int p00 = (grp * C::PAIR_PASSES + h) * NPP;  // first point of this pass
      T tr[NPP][NV];
#pragma unroll
      for (int p = 0; p < NPP; ++p)
#pragma unroll
        for (int v = 0; v < NV; ++v) tr[p][v] = T(0);
      face_traces<C, NPP>(a.qhat, c, N, tc, p00, tr);
#pragma unroll
      for (int k = 0; k < (NPP + 1) / 2; ++k) {
        constexpr int LAST = NPP - 1;
        const int p0 = 2 * k, p1 = 2 * k + 1 <= LAST ? 2 * k + 1 : LAST;
        // side 0 takes point p0, side 1 point p1: each sends the partner its
        // own trace at the partner's point
        T mine[NV], other[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T send = side == 0 ? tr[p1][v] : tr[p0][v];
          other[v] = __shfl_xor_sync(0xffffffffu, send, 1);
          mine[v] = side == 0 ? tr[p0][v] : tr[p1][v];
        }
        if (side == 0 || 2 * k + 1 <= LAST) {
          const int p = p00 + (side == 0 ? p0 : p1);
          T ul[NV], ur[NV];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            ul[v] = qbL[v] + (side == 0 ? mine[v] : other[v]);
            ur[v] = qbR[v] + (side == 0 ? other[v] : mine[v]);
          }
          rusanov_point<C, OSHER>(a, ul, ur, qbL, qbR, n, wq[p % NQS] * wt[p / NQS], facc, dacc);
        }
      }
    }
#pragma unroll
    for (int o = 1; o < TPF; o <<= 1)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        dacc[v] += __shfl_xor_sync(0xffffffffu, dacc[v], o);
#pragma unroll
        for (int m = 0; m < D; ++m) facc[m][v] += __shfl_xor_sync(0xffffffffu, facc[m][v], o);
      }
    // FP64 contraction split over the face's threads (thread q takes the
    // variables q, q + TPF, ...), so every FP64 instruction runs on all lanes
    if (valid) {
      const int q = (int)(threadIdx.x % TPF);
      double fa[D];
#pragma unroll
      for (int m = 0; m < D; ++m) fa[m] = a.fa[m * F + f];
      const double area = a.farea[f];
#pragma unroll
      for (int j = 0; j < (NV + TPF - 1) / TPF; ++j) {
        const int v = q + j * TPF;
        if (v >= NV) break;
        T dv = dacc[0];
        T fv[D];
#pragma unroll
        for (int m = 0; m < D; ++m) fv[m] = facc[m][0];
#pragma unroll
        for (int u = 1; u < NV; ++u)
          if (u == v) {
            dv = dacc[u];
#pragma unroll
            for (int m = 0; m < D; ++m) fv[m] = facc[m][u];
          }
        double g = -area * (double)dv;
#pragma unroll
        for (int m = 0; m < D; ++m) g += fa[m] * (double)fv[m];
        a.G[v * F + f] = 0.5 * dtd * g;
      }
    }
  }
}

template <class C, bool OSHER>
__global__ void __launch_bounds__(128, C::FLUX_MINB) k_flux_pair(KArgs<C> a, int use_smem) {
  constexpr int TPF = 2 * C::FLUX_SPLIT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const typename C::T* tab = face_tables<C>(a, use_smem, smem_raw);
  const double dtd = dt_of(a.dt_fixed, a.cfl, a.dtmin, a.cur);
  // block-uniform trip count (the exchanges shuffle over the whole warp); a
  // thread past the last face works on a clamped copy, not written
  // with SIDE_AHEAD the next iteration's cell and code are loaded while the
  // current face is integrated
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t g0 = (int64_t)blockIdx.x * blockDim.x;
  PairSide ps = pair_side<C>(a, g0);
  for (; g0 < TPF * a.F; g0 += stride) {
    PairSide nx = ps;
    if (C::SIDE_AHEAD && g0 + stride < TPF * a.F) nx = pair_side<C>(a, g0 + stride);
    flux_pair_iter<C, OSHER>(a, tab, g0, dtd, ps);
    ps = C::SIDE_AHEAD ? nx : pair_side<C>(a, g0 + stride);
  }
}

// Quadrature-free Rusanov flux (the fixed-mesh form the paper describes
// after Eq. osher), one thread per face, persistent grid.  With the nodal
// expansions of the predictor and its flux (Eq. PDEterm) the face and time
// integrals reduce to the precomputed integrals I_l of each side's nodal
// basis (per code), so the time-averaged normal flux per |f| is
//   1/2 sum_l (I-_l F(q-_l) + I+_l F(q+_l)) . n - 1/2 s (qbar+ - qbar-),
// qbar = Qbar + sum_l I_l q_hat_l the space-time face average of a side's
// predictor, s the larger maximal signal speed along n of the two averages.
// Deviation form: F(Qbar) + sum_l I_l (F(Qbar + q_hat_l) - F(Qbar)) (the I_l
// sum to one), so a constant state gives identical sums on every face.  A
// nodal state that is not admissible contributes F(Qbar); an inadmissible
// face average takes its cell average's speed.
template <class C>
__device__ __forceinline__ void qf_side(const KArgs<C>& a, const typename C::T* __restrict__ qhat, int64_t c,
                                        int64_t N, const typename C::T* Ic, const typename C::T* qb,
                                        typename C::T (&facc)[C::D][C::NV], typename C::T (&dev)[C::NV]) {
  using T = typename C::T;
  using V = typename Vec16<T>::V;
  constexpr int D = C::D, NV = C::NV, L = C::L, LP = C::LP, VW = C::VW;
  using PH = Phys<D, C::PDE, T>;
  T Fb[D][NV];
  {
    typename PH::Prim pb = PH::prim(qb, a.gamma);
#pragma unroll
    for (int m = 0; m < D; ++m) {
      T em[D];
#pragma unroll
      for (int e = 0; e < D; ++e) em[e] = e == m ? T(1) : T(0);
      flux_normal<D, C::PDE, T>(qb, pb, em, Fb[m], a.ch);
#pragma unroll
      for (int v = 0; v < NV; ++v) facc[m][v] += Fb[m][v];
    }
  }
#pragma unroll 1
  for (int l4 = 0; l4 < LP; l4 += VW) {
    T ql[VW][NV];
    load_chunk<C>(qhat, c, N, l4, ql);
    const V iv = *reinterpret_cast<const V*>(Ic + l4);
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      if (l4 + j >= L) continue;
      const T I = Vec16<T>::get(iv, j);
      T q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        q[v] = qb[v] + ql[j][v];
        dev[v] += I * ql[j][v];
      }
      typename PH::Prim pq = PH::prim(q, a.gamma);
      if (a.pos && !(q[0] > T(0) && pq.p > T(0))) continue;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        T em[D];
#pragma unroll
        for (int e = 0; e < D; ++e) em[e] = e == m ? T(1) : T(0);
        T fq[NV];
        flux_normal<D, C::PDE, T>(q, pq, em, fq, a.ch);
#pragma unroll
        for (int v = 0; v < NV; ++v) facc[m][v] += I * (fq[v] - Fb[m][v]);
      }
    }
  }
}

template <class C>
__global__ void __launch_bounds__(128) k_flux_qf(KArgs<C> a) {
  using T = typename C::T;
  constexpr int D = C::D, NV = C::NV, LP = C::LP;
  using PH = Phys<D, C::PDE, T>;
  __shared__ __align__(16) T sI[C::NCODE * LP];
  for (int k = threadIdx.x; k < C::NCODE * LP; k += blockDim.x) sI[k] = a.ftab[C::QF_OFF + k];
  __syncthreads();
  const double dtd = dt_of(a.dt_fixed, a.cfl, a.dtmin, a.cur);
  const int64_t N = a.N, F = a.F;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t Lc = a.fL[f];
    const int64_t Rc = a.fR[f];
    T n[D];
#pragma unroll
    for (int e = 0; e < D; ++e) n[e] = a.fn[e * F + f];
    T qbL[NV], qbR[NV], devL[NV], devR[NV];
    T facc[D][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      devL[v] = T(0);
      devR[v] = T(0);
#pragma unroll
      for (int m = 0; m < D; ++m) facc[m][v] = T(0);
    }
    cell_average<C>(a, Lc, qbL);
    qf_side<C>(a, a.qhat, Lc, N, sI + (int)a.codeL[f] * LP, qbL, facc, devL);
    if (Rc >= 0) {
      cell_average<C>(a, Rc, qbR);
      qf_side<C>(a, a.qhat, Rc, N, sI + (int)a.codeR[f] * LP, qbR, facc, devR);
    } else {  // transmissive: the outer side repeats the inner one
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        qbR[v] = qbL[v];
        devR[v] = devL[v];
#pragma unroll
        for (int m = 0; m < D; ++m) facc[m][v] *= T(2);
      }
    }
    T uL[NV], uR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      uL[v] = qbL[v] + devL[v];
      uR[v] = qbR[v] + devR[v];
    }
    typename PH::Prim pl = PH::prim(uL, a.gamma);
    typename PH::Prim pr = PH::prim(uR, a.gamma);
    if (a.pos) {
      if (!(uL[0] > T(0) && pl.p > T(0))) pl = PH::prim(qbL, a.gamma);
      if (!(uR[0] > T(0) && pr.p > T(0))) pr = PH::prim(qbR, a.gamma);
    }
    const T sl = PH::smax(pl, n, a.gamma, a.ch), sr = PH::smax(pr, n, a.gamma, a.ch);
    const T s = sl > sr ? sl : sr;
    T dacc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) dacc[v] = s * ((qbR[v] - qbL[v]) + (devR[v] - devL[v]));
    store_face_integral<C>(a, f, dtd, facc, dacc);
  }
}

// Block minimum of non-negative ratios folded into *target, which holds the
// bits of a positive double.  Non-negative IEEE values order like their bit
// patterns, so the reduction runs on the integer bits (no FP64 pipe work in
// FP32-mixed mode); a NaN (bits above +inf) never wins.
template <typename T>
__device__ __forceinline__ void block_min_atomic(T val, unsigned long long* target) {
  using U = typename std::conditional<sizeof(T) == 4, unsigned, unsigned long long>::type;
  __shared__ U red[32];
  U b;
  if constexpr (sizeof(T) == 4) {
    b = __reduce_min_sync(0xffffffffu, __float_as_uint(val));
  } else {
    b = (U)__double_as_longlong(val);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const U other = __shfl_xor_sync(0xffffffffu, b, o);
      b = other < b ? other : b;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = b;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    const U inf = sizeof(T) == 4 ? (U)0x7f800000u : (U)0x7ff0000000000000ull;
    b = lane < nw ? red[lane] : inf;
    if constexpr (sizeof(T) == 4) {
      b = __reduce_min_sync(0xffffffffu, b);
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const U other = __shfl_xor_sync(0xffffffffu, b, o);
        b = other < b ? other : b;
      }
    }
    if (lane == 0) {
      double v;
      if constexpr (sizeof(T) == 4) v = (double)__uint_as_float((unsigned)b);
      else v = __longlong_as_double((long long)b);
      if (v > 0.0) atomicMin(target, (unsigned long long)__double_as_longlong(v));
    }
  }
}

// ------------------------------------------------------------------ update
// One cell of the update; returns its ratio h_i / |lambda_max| for the CFL
// bound of the next step (+inf past the last cell).
template <class C>
__device__ __forceinline__ typename C::T update_cell(const KArgs<C>& a, int64_t i) {
  using T = typename C::T;
  constexpr int D = C::D, NV = C::NV;
  using PH = Phys<D, C::PDE, T>;
  const int64_t N = a.N, F = a.F;
  T ratio = T(INFINITY);
  if (i < N) {
    // sum_f +-G_f: the sign of a face's integral is flipped on the bits (no
    // FP64 instruction), the first face starts the sum
    double acc[NV];
#pragma unroll
    for (int k = 0; k <= D; ++k) {
      const int cf = a.cellface[k * N + i];
      const int64_t f = cf >> 1;
      const long long flip = (long long)(cf & 1) << 63;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double g = __longlong_as_double(__double_as_longlong(a.G[v * F + f]) ^ flip);
        acc[v] = k == 0 ? g : acc[v] + g;
      }
    }
    const double iv = a.invvol[i];
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      q[v] = fma(-iv, acc[v], a.Q[v * N + i]);
      a.Q[v * N + i] = q[v];
    }
    T qt[NV];
    if constexpr (std::is_same<T, float>::value) {
      float pr[2 * C::NVP];
#pragma unroll
      for (int v = 0; v < C::NVP; ++v) {
        float hi = 0.f, lo = 0.f;
        if (v < NV) split_hilo(q[v], hi, lo);
        pr[2 * v] = hi;
        pr[2 * v + 1] = lo;
        if (v < NV) qt[v] = hi;
      }
      float4* dst = reinterpret_cast<float4*>(a.Qp) + i * (C::NVP / 2);
#pragma unroll
      for (int m = 0; m < C::NVP / 2; ++m) dst[m] = make_float4(pr[4 * m], pr[4 * m + 1], pr[4 * m + 2], pr[4 * m + 3]);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) qt[v] = q[v];
    }
    // admissibility and the CFL bound in the arithmetic type (FP32 in mixed
    // mode: FP64 divisions and square roots are slow on this part)
    const T pk = PH::pressure(qt, a.gamma);
    if (!(qt[0] > T(0) && pk > T(0) && isfinite(pk))) atomicOr(a.status, 1);
    const T sp = PH::speed(qt, a.gamma, a.ch);
    ratio = (T)a.hsize[i] / sp;
  }
  return ratio;
}

template <class C>
__global__ void __launch_bounds__(256) k_update(KArgs<C> a) {
  const typename C::T ratio = update_cell<C>(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  block_min_atomic(ratio, a.dtmin + (1 - a.cur));
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.time += dt_of(a.dt_fixed, a.cfl, a.dtmin, a.cur);
}

// ------------------------------------------------- batched steps (serving)
// One time step of many solvers of one configuration in each launch.  A
// table in device memory lists the solvers (their kernel arguments) and,
// per kernel, the prefix sums of their work chunks: 128 cells for the
// reconstruction + predictor, 128 threads of the face space for the fluxes,
// 256 cells for the update.  The grids are persistent (sized to the
// resident blocks) and loop over the chunks; a block stages the arguments of
// its chunk's solver in shared memory.  Every cell and face of a solver gets
// the arithmetic of the single-solver kernels (the same device functions),
// and the CFL minimum reduces within a solver's own blocks, so each result
// equals the solver stepped alone.
constexpr int kBatchMaxSeg = 64;
struct BatchHdr {
  int nseg;
  int pad;
  int pref[3][kBatchMaxSeg + 1];
};
template <class C>
struct BatchTab {
  BatchHdr h;
  KArgs<C> a[kBatchMaxSeg];
};

// index of the solver whose chunk range holds chunk c (pref ascending)
__device__ __forceinline__ int batch_seg(const int* pref, int nseg, int c) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// stage the arguments of chunk c's solver into sa; returns the chunk's index
// within that solver
template <class C>
__device__ __forceinline__ int batch_stage(const BatchTab<C>* bt, int kernel, int c, KArgs<C>& sa) {
  const int seg = batch_seg(bt->h.pref[kernel], bt->h.nseg, c);
  __syncthreads();
  const int* src = reinterpret_cast<const int*>(&bt->a[seg]);
  int* dst = reinterpret_cast<int*>(&sa);
  for (int k = threadIdx.x; k < (int)(sizeof(KArgs<C>) / 4); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
  return c - bt->h.pref[kernel][seg];
}

template <class C>
__global__ void __launch_bounds__(128, C::REC_MINB) k_rec_pred_batch(const BatchTab<C>* bt,
                                                                     const __grid_constant__ CellTabArg<C> tb) {
  __shared__ __align__(16) KArgs<C> sa;
  const int total = bt->h.pref[0][bt->h.nseg];
  for (int c = blockIdx.x; c < total; c += gridDim.x) {
    const int lc = batch_stage(bt, 0, c, sa);
    if (lc == 0 && threadIdx.x == 0 && sa.reset_next) sa.dtmin[1 - sa.cur] = 0x7ff0000000000000ull;
    rec_pred_cell<C, false>(sa, cell_tab<C>(sa, tb), (int64_t)lc * 128 + threadIdx.x);
  }
}

template <class C, bool OSHER>
__global__ void __launch_bounds__(128, C::FLUX_MINB) k_flux_batch(const BatchTab<C>* bt, int use_smem) {
  using T = typename C::T;
  __shared__ __align__(16) KArgs<C> sa;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the face tables depend on the configuration only: any solver's copy
  const T* tab = face_tables<C>(bt->a[0], use_smem, smem_raw);
  const int total = bt->h.pref[1][bt->h.nseg];
  for (int c = blockIdx.x; c < total; c += gridDim.x) {
    const int lc = batch_stage(bt, 1, c, sa);
    const double dtd = dt_of(sa.dt_fixed, sa.cfl, sa.dtmin, sa.cur);
    if constexpr (C::PAIR) {
      flux_pair_iter<C, OSHER>(sa, tab, (int64_t)lc * 128, dtd, pair_side<C>(sa, (int64_t)lc * 128));
    } else {
      const int64_t f = (int64_t)lc * 128 + threadIdx.x;
      if (f < sa.F) flux_one_face<C, OSHER>(sa, tab, f, dtd);
    }
  }
}

template <class C>
__global__ void __launch_bounds__(256) k_update_batch(const BatchTab<C>* bt) {
  __shared__ __align__(16) KArgs<C> sa;
  const int total = bt->h.pref[2][bt->h.nseg];
  for (int c = blockIdx.x; c < total; c += gridDim.x) {
    const int lc = batch_stage(bt, 2, c, sa);
    const typename C::T ratio = update_cell<C>(sa, (int64_t)lc * 256 + threadIdx.x);
    block_min_atomic(ratio, sa.dtmin + (1 - sa.cur));
    if (lc == 0 && threadIdx.x == 0) *sa.time += dt_of(sa.dt_fixed, sa.cfl, sa.dtmin, sa.cur);
  }
}

template <class C>
__global__ void __launch_bounds__(256) k_stable_dt(KArgs<C> a, int slot) {
  using T = typename C::T;
  using PH = Phys<C::D, C::PDE, T>;
  const int64_t N = a.N;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  T ratio = T(INFINITY);
  if (i < N) {
    T q[C::NV];
    if constexpr (std::is_same<T, float>::value) {
      float lo[C::NV];
      load_pairs<C>(a.Qp, i, q, lo);
    } else {
#pragma unroll
      for (int v = 0; v < C::NV; ++v) q[v] = a.Q[v * N + i];
    }
    ratio = (T)a.hsize[i] / PH::speed(q, a.gamma, a.ch);
  }
  block_min_atomic(ratio, a.dtmin + slot);
}

// State in the caller's cell order (N x NV, row-major) <-> internal SoA. One
// thread per caller element, so the caller-side accesses (which may be pinned
// host memory read or written directly over the CPU-GPU link) are contiguous
// across a warp; the device side scatters through the user->internal map.
// set_state also restarts the run: the time-step bound of slot 0 (recomputed
// by k_stable_dt next), the accumulated time and the status words.
template <class C>
__global__ void k_set_state(KArgs<C> a, const double* user) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) {
    a.dtmin[0] = 0x7ff0000000000000ull;
    *a.time = 0.0;
    a.status[0] = 0;
    a.status[1] = 0;
  }
  if (e >= a.N * C::NV) return;
  const int64_t u = e / C::NV;
  const int v = (int)(e - u * C::NV);
  const int64_t c = a.iperm[u];
  const double q = user[e];
  a.Q[v * a.N + c] = q;
  if constexpr (std::is_same<typename C::T, float>::value) {
    float hi, lo;
    split_hilo(q, hi, lo);
    reinterpret_cast<float2*>(a.Qp)[c * C::NVP + v] = make_float2(hi, lo);
  }
}

template <class C>
__global__ void k_get_state(KArgs<C> a, double* user) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.N * C::NV) return;
  const int64_t u = e / C::NV;
  const int v = (int)(e - u * C::NV);
  user[e] = a.Q[v * a.N + a.iperm[u]];
}

template <class C>
__global__ void k_qhat_out(KArgs<C> a, double* user) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const int64_t u = a.perm[i];
  for (int l = 0; l < C::L; ++l)
#pragma unroll
    for (int v = 0; v < C::NV; ++v) {
      double qbar;
      if constexpr (std::is_same<typename C::T, float>::value)
        qbar = (double)a.Qp[(i * C::NVP + v) * 2] + (double)a.Qp[(i * C::NVP + v) * 2 + 1];
      else
        qbar = a.Q[v * a.N + i];
      user[(u * C::L + l) * C::NV + v] = qbar + (double)a.qhat[((int64_t)l * a.N + i) * C::NV + v];
    }
}

// ------------------------------------------------------------- host side
template <class C>
class OpsImpl final : public Ops {
 public:
  using T = typename C::T;
  explicit OpsImpl(const RefElem& re) {
    std::memset(&tab_, 0, sizeof(tab_));
    for (int n = 0; n < C::L0; ++n)
      for (int l = 0; l < C::MC1; ++l) tab_.E[n][l] = (T)re.E[n * C::MC1 + l];
    for (int l = 0; l < C::MC1; ++l)
      for (int m = 0; m < C::MC1; ++m)
        tab_.Sig[l][m] = m == l ? (T)re.Sigma[l * C::MC1 + m] : m > l ? (T)(2.0 * re.Sigma[l * C::MC1 + m]) : T(0);
    for (int k = 0; k < C::L1; ++k)
      for (int l = 0; l < C::MC1; ++l) {
        double s = 0.0;
        for (int n = 0; n < C::L0; ++n) s += re.C0[k * C::L0 + n] * re.E[n * C::MC1 + l];
        tab_.CE[k][l] = (T)s;
      }
    for (int e = 0; e < C::D; ++e)
      for (int k = 0; k < C::L1; ++k)
        for (int l = 0; l < C::L; ++l) tab_.P[e][k][l] = (T)re.P[((size_t)e * C::L1 + k) * C::L + l];
    // the tau = 0 node below each unknown node (same spatial coordinates);
    // C0 must be that selection (it is, on the principal lattice: C0[k][n] =
    // theta_n(xi_k, 0) with xi_k a lattice node), else prepare() refuses
    for (int k = 0; k < C::L1; ++k) {
      tab_.sel[k] = -1;
      for (int n = 0; n < C::L0 && tab_.sel[k] < 0; ++n) {
        bool same = true;
        for (int a = 0; a < C::D; ++a) same = same && re.stnode[n][a] == re.stnode[C::L0 + k][a];
        if (same) tab_.sel[k] = n;
      }
      if (tab_.sel[k] < 0) {
        sel_ok_ = false;
        tab_.sel[k] = 0;
      }
      for (int n = 0; n < C::L0; ++n)
        if (std::fabs(re.C0[k * C::L0 + n] - (n == tab_.sel[k] ? 1.0 : 0.0)) > 1e-12) sel_ok_ = false;
    }
    ftab_.assign(C::TAB_TOTAL, T(0));
    for (int code = 0; code < C::NCODE; ++code)
      for (int row = 0; row < C::NQT * C::NQS; ++row)
        for (int l = 0; l < C::L; ++l)
          ftab_[code * C::CODE_STRIDE + row * C::LP + l] =
              (T)re.ftab[((size_t)code * C::NQT * C::NQS + row) * C::L + l];
    for (int q = 0; q < C::NQS; ++q) ftab_[C::TABN + q] = (T)re.wq[q];
    for (int t = 0; t < C::NQT; ++t) ftab_[C::TABN + C::NQS + t] = (T)re.wt[t];
    for (int code = 0; code < C::NCODE; ++code)
      for (int l = 0; l < C::L; ++l) ftab_[C::QF_OFF + code * C::LP + l] = (T)re.fint[(size_t)code * C::L + l];
  }
  // face tables, then (where they are not a kernel parameter) the cell tables
  size_t table_bytes() const override {
    return cell_tab_in_param<C>() ? ftab_.size() * sizeof(T) : cell_tab_offset<C>() + sizeof(CellTab<C>);
  }
  CellTabArg<C> tab_arg() const {
    if constexpr (cell_tab_in_param<C>())
      return tab_;
    else
      return NoCellTab{};
  }
  // shared-memory bytes of the quadrature flux kernels (tables and weights)
  static size_t quad_table_bytes() { return (size_t)(C::TABN + C::NQS + C::NQT) * sizeof(T); }
  void pack_tables(void* host) const override {
    std::memcpy(host, ftab_.data(), ftab_.size() * sizeof(T));
    if constexpr (!cell_tab_in_param<C>()) {
      unsigned char* h = static_cast<unsigned char*>(host);
      std::memset(h + ftab_.size() * sizeof(T), 0, cell_tab_offset<C>() - ftab_.size() * sizeof(T));
      std::memcpy(h + cell_tab_offset<C>(), &tab_, sizeof(tab_));
    }
  }
  size_t elem_size() const override { return sizeof(T); }

  KArgs<C> args(const DevState& s, const PhysParams& ph, DtArgs dt) const {
    KArgs<C> a;
    std::memset(&a, 0, sizeof(a));
    a.N = s.N;
    a.F = s.F;
    a.Q = s.Q;
    a.Qp = s.Qp;
    a.perm = s.perm;
    a.iperm = s.iperm;
    a.sten4 = s.sten4;
    a.R = (const T*)s.R;
    a.sec = s.sec;
    a.Binv = (const T*)s.Binv;
    a.nsec = s.nsec;
    a.Jinv = (const T*)s.Jinv;
    a.qhat = (T*)s.qhat;
    a.fL = s.fL;
    a.fR = s.fR;
    a.codeL = s.codeL;
    a.codeR = s.codeR;
    a.fn = (const T*)s.fn;
    a.fa = s.fa;
    a.farea = s.farea;
    a.G = s.G;
    a.ftab = (const T*)s.ftab;
    a.cellface = s.cellface;
    a.invvol = s.invvol;
    a.hsize = s.hsize;
    a.dtmin = s.dtmin;
    a.time = s.time;
    a.status = s.status;
    a.out = nullptr;
    a.gamma = (T)ph.gamma;
    a.ch = (T)ph.ch;
    a.eps = (T)ph.eps;
    a.lam0 = (T)ph.lam0;
    a.lams = (T)ph.lams;
    a.niter = ph.niter;
    a.linw = ph.linear_weights;
    a.pos = ph.positivity;
    a.flux = ph.flux;
    a.dt_fixed = dt.fixed;
    a.cfl = dt.cfl;
    a.cur = dt.cur;
    a.reset_next = 1;
    return a;
  }

  static unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

  cudaError_t rec_pred(const DevState& s, const PhysParams& ph, DtArgs dt, cudaStream_t st) override {
    KArgs<C> a = args(s, ph, dt);
    if (dt.cur < 0) {  // diagnostic call: keep the next-step bound untouched
      a.cur = 0;
      a.reset_next = 0;
    }
    k_rec_pred<C, false><<<nblk(s.N, 128), 128, C::PRED_SMEM_BYTES, st>>>(a, tab_arg());
    return cudaGetLastError();
  }
  cudaError_t reconstruct(const DevState& s, const PhysParams& ph, double* out, cudaStream_t st) override {
    KArgs<C> a = args(s, ph, DtArgs());
    a.out = out;
    a.reset_next = 0;
    k_rec_pred<C, true><<<nblk(s.N, 128), 128, 0, st>>>(a, tab_arg());
    return cudaGetLastError();
  }
  using FluxKernel = void (*)(KArgs<C>, int);
  // quadrature flux kernel: Rusanov, or Osher-type (Euler only)
  static FluxKernel flux_kernel(bool osher = false) {
    if constexpr (C::PDE == 0) {
      if (osher) {
        if constexpr (C::PAIR) return k_flux_pair<C, true>;
        else return k_flux<C, true>;
      }
    }
    if constexpr (C::PAIR) return k_flux_pair<C, false>;
    else return k_flux<C, false>;
  }
  cudaError_t prepare() override {
    if (C::STASH && !sel_ok_) return cudaErrorInvalidValue;  // C0 is not the lattice selection
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_rec_pred<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             C::PRED_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const size_t smem = quad_table_bytes();
    use_smem_ = smem <= 100 * 1024 ? 1 : 0;
    if (use_smem_) {
      for (int o = 0; o < (C::PDE == 0 ? 2 : 1); ++o) {
        e = cudaFuncSetAttribute(flux_kernel(o == 1), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
    }
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, flux_kernel(), 128, use_smem_ ? smem : 0);
    if (e != cudaSuccess) return e;
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    max_blocks_ = (int64_t)std::max(1, nb) * nsm;
    int nbq = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbq, k_flux_qf<C>, 128, 0);
    if (e != cudaSuccess) return e;
    max_blocks_qf_ = (int64_t)std::max(1, nbq) * nsm;
    // batched kernels (serving): resident grids
    e = cudaFuncSetAttribute(k_rec_pred_batch<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::PRED_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    int nb1 = 0, nb2 = 0, nb3 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb1, k_rec_pred_batch<C>, 128, C::PRED_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (use_smem_) {
      for (int o = 0; o < (C::PDE == 0 ? 2 : 1); ++o) {
        e = cudaFuncSetAttribute(o ? (const void*)k_flux_batch<C, true> : (const void*)k_flux_batch<C, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, k_flux_batch<C, false>, 128, use_smem_ ? smem : 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb3, k_update_batch<C>, 256, 0);
    if (e != cudaSuccess) return e;
    max_blocks_rec_b_ = (int64_t)std::max(1, nb1) * nsm;
    max_blocks_flux_b_ = (int64_t)std::max(1, nb2) * nsm;
    max_blocks_upd_b_ = (int64_t)std::max(1, nb3) * nsm;
    return cudaSuccess;
  }
  cudaError_t flux(const DevState& s, const PhysParams& ph, DtArgs dt, cudaStream_t st) override {
    KArgs<C> a = args(s, ph, dt);
    if (dt.cur < 0) a.cur = 0;
    if (ph.flux == 2) {  // quadrature-free Rusanov
      unsigned nb = (unsigned)std::min<int64_t>(nblk(s.F, 128), max_blocks_qf_);
      k_flux_qf<C><<<nb, 128, 0, st>>>(a);
      return cudaGetLastError();
    }
    const size_t smem = use_smem_ ? quad_table_bytes() : 0;
    unsigned nb = (unsigned)std::min<int64_t>(nblk(s.F * (C::PAIR ? 2 * C::FLUX_SPLIT : 1), 128), max_blocks_);
    flux_kernel(ph.flux == 1)<<<nb, 128, smem, st>>>(a, use_smem_);
    return cudaGetLastError();
  }
  cudaError_t update(const DevState& s, const PhysParams& ph, DtArgs dt, cudaStream_t st) override {
    KArgs<C> a = args(s, ph, dt);
    k_update<C><<<nblk(s.N, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
  }
  cudaError_t stable_dt(const DevState& s, const PhysParams& ph, int slot, cudaStream_t st) override {
    KArgs<C> a = args(s, ph, DtArgs());
    k_stable_dt<C><<<nblk(s.N, 256), 256, 0, st>>>(a, slot);
    return cudaGetLastError();
  }
  cudaError_t set_state(const DevState& s, const double* user, cudaStream_t st) override {
    KArgs<C> a = args(s, PhysParams(), DtArgs());
    k_set_state<C><<<nblk(s.N * C::NV, 256), 256, 0, st>>>(a, user);
    return cudaGetLastError();
  }
  cudaError_t get_state(const DevState& s, double* user, cudaStream_t st) override {
    KArgs<C> a = args(s, PhysParams(), DtArgs());
    k_get_state<C><<<nblk(s.N * C::NV, 256), 256, 0, st>>>(a, user);
    return cudaGetLastError();
  }
  size_t batch_bytes() const override { return sizeof(BatchTab<C>); }
  int batch_max() const override { return kBatchMaxSeg; }
  void batch_fill(void* host_tab, int nseg, const DevState* const* ds, const PhysParams* const* ph,
                  const DtArgs* dt) const override {
    BatchTab<C>* bt = reinterpret_cast<BatchTab<C>*>(host_tab);
    std::memset(&bt->h, 0, sizeof(bt->h));
    bt->h.nseg = nseg;
    const int64_t tpf = C::PAIR ? 2 * C::FLUX_SPLIT : 1;
    for (int k = 0; k < nseg; ++k) {
      bt->a[k] = args(*ds[k], *ph[k], dt[k]);
      bt->h.pref[0][k + 1] = bt->h.pref[0][k] + (int)nblk(ds[k]->N, 128);
      bt->h.pref[1][k + 1] = bt->h.pref[1][k] + (int)nblk(ds[k]->F * tpf, 128);
      bt->h.pref[2][k + 1] = bt->h.pref[2][k] + (int)nblk(ds[k]->N, 256);
    }
  }
  cudaError_t step_batch(const void* dev_tab, int flux, cudaStream_t st) override {
    const BatchTab<C>* bt = reinterpret_cast<const BatchTab<C>*>(dev_tab);
    k_rec_pred_batch<C><<<(unsigned)max_blocks_rec_b_, 128, C::PRED_SMEM_BYTES, st>>>(bt, tab_arg());
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = use_smem_ ? quad_table_bytes() : 0;
    if (flux == 1 && C::PDE == 0) k_flux_batch<C, true><<<(unsigned)max_blocks_flux_b_, 128, smem, st>>>(bt, use_smem_);
    else k_flux_batch<C, false><<<(unsigned)max_blocks_flux_b_, 128, smem, st>>>(bt, use_smem_);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_update_batch<C><<<(unsigned)max_blocks_upd_b_, 256, 0, st>>>(bt);
    return cudaGetLastError();
  }
  cudaError_t qhat_out(const DevState& s, double* user, cudaStream_t st) override {
    KArgs<C> a = args(s, PhysParams(), DtArgs());
    k_qhat_out<C><<<nblk(s.N, 256), 256, 0, st>>>(a, user);
    return cudaGetLastError();
  }

 private:
  CellTab<C> tab_;
  std::vector<T> ftab_;
  int use_smem_ = 0;
  bool sel_ok_ = true;
  int64_t max_blocks_ = 152;
  int64_t max_blocks_qf_ = 152;
  int64_t max_blocks_rec_b_ = 152, max_blocks_flux_b_ = 152, max_blocks_upd_b_ = 152;
};

}  // namespace cw
