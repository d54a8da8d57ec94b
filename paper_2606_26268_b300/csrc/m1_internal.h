// m1_internal.h -- structures shared by the host library and the step
// kernels.  Not part of the public ABI.
#pragma once
#include <cstdint>

#include "m1_math.cuh"

namespace m1 {

enum { kCart = 0, kCyl = 1, kSph = 2 };

// Boundary kinds (the values of the public rad_bc).
enum { BC_OUTFLOW = 0, BC_PERIODIC = 1, BC_REFLECT = 2, BC_FIXED = 3, BC_LTE = 4 };

// Options of the face computation (Sect. 2.5): reconstruction (0 PLM, 1
// LimO3), treatment of |F_f| > E_f (0 f-preserving, 1 flat, 2 clip) and
// Riemann solver (0 HLL, 1 Lax-Friedrichs-Rusanov).  All zero on the
// TMA-staged kernels, which implement only the defaults.
struct Scheme {
  int recon, ffix, riemann;
};

// Per-direction geometry tables, indexed by the padded index ip = i + g
// (g = 2 ghost cells on active directions, 0 on inactive ones); each table
// has len = n + 2 g entries.  Ghost entries describe the cell the ghost
// copies (its width, radius) except TAB_IDXC/TAB_HLO/TAB_HHI, which use the
// extended centre coordinates of the ghost itself.
enum {
  TAB_IDXC = 0,  // 1 / (xc[ip+1] - xc[ip])
  TAB_HLO,       // x_face_lo - xc  (<= 0)
  TAB_HHI,       // x_face_hi - xc  (>= 0)
  TAB_ALO,       // lower-face area / volume factor of this direction
  TAB_AHI,       // upper-face area / volume factor
  TAB_WID,       // coordinate width (dx, dR, dr, dphi, dtheta, dz)
  TAB_MET,       // dir 0: 1/R_c (cyl) or 1/r~ (sph); dir 1 (sph): cot~theta
  TAB_AMLO,      // area/volume factors of the phi component (angular-momentum form)
  TAB_AMHI,
  TAB_RC,        // dir 0: centre radius; dir 1 (sph): sin(theta_c)
  TAB_PHF,       // dir 1 (sph): dtheta / (cos theta_lo - cos theta_hi)
  TAB_N
};

template <class T>
struct GeomDev {
  const T* tab[3];  // tab[d][slot * len[d] + ip]
  int len[3];
};

struct StepDims {
  int ndim;
  int n[3];         // cells per direction
  int g[3];         // ghost depth per direction
  int pn[3];        // padded extents (pn[0] may be rounded up for alignment)
  long long sy, sz; // padded strides of directions 1 and 2
  int bc_lo[3], bc_hi[3];  // BC_* per direction
};

template <class S>
struct Fields {
  S* E;
  S* F[3];
  S* e;
  S* m[3];
};

enum {
  ST_FIX = 0,
  ST_EFLOOR,
  ST_FCLIP,
  ST_ITERS,
  ST_ITMAX,
  ST_FALLBACK,
  ST_NOCONV,
  ST_STEPS,
  ST_N
};

enum { STATUS_NOCONV = 1, STATUS_NONPHYS = 2, STATUS_TIMEOUT = 4, STATUS_BOUNDS = 8 };

// Index check of the debug build (compiled with RAD_DEBUG_CHECKS, the
// library librad_debug.so): an index outside [0, n) sets STATUS_BOUNDS in
// the status word, which the next rad_sync returns as RAD_EBOUNDS, and the
// caller skips the access; there is no trap.  Release builds compile the
// check to `true`.
__device__ __forceinline__ bool index_ok(long long i, long long n, int* status) {
#ifdef RAD_DEBUG_CHECKS
  if (i >= 0 && i < n) return true;
  atomicOr(status, STATUS_BOUNDS);
  return false;
#else
  (void)i;
  (void)n;
  (void)status;
  return true;
#endif
}

// Cells of one padded field array.
__host__ __device__ __forceinline__ long long padded_cells(const StepDims& d) {
  return (long long)d.pn[0] * d.pn[1] * d.pn[2];
}

template <class P>
struct StepArgs {
  using S = typename P::S;
  using T = typename P::T;
  StepDims dim;
  Fields<S> in;   // U^n (read only)
  Fields<S> out;  // U^{n+1}
  // (E*, F*) of the cells queued for the Newton iteration, read back by the
  // queue pass (the output buffer itself, except in the last stage of the
  // two-stage step, where the output buffer still holds U^n)
  Fields<S> stash;
  // irradiation (Sect. 2.9): energy deposited per unit volume and time,
  // -div F_irr, in the padded layout; nullptr: none
  const S* qirr;
  // last stage of the two-stage step: the result written to `out` is the
  // average of the stage result with the U^n that `out` holds at the cell
  // (conserved variables E_r, F_r, m and E_gas = e + |m|^2 / (2 rho))
  int average;
  Scheme scheme;
  // gas evolved by the gas step (general form only): the last stage of the
  // two-stage step reads rho^n of the cell from rho_avg and stores the
  // average of rho there (nullptr otherwise); `hydro` makes the epilogue
  // keep the gas ghosts of the fixed and LTE sides (edge density, e =
  // C_v T_b with the gas temperatures bcT)
  S* rho_avg;
  int hydro;
  double bcT[3][2];
  const S* rho;
  GeomDev<T> geo;
  OpacityDev opac;
  CoupleParams cp;
  T chat, dt, efloor;
  T ratio;        // c / chat
  T inv_chat;
  unsigned long long* stats;
  int* status;
  // first wait on each TMA-staged plane: 0 = the default bounded wait,
  // else that many non-blocking tests; a wait that runs out sets
  // STATUS_TIMEOUT and the CTA stops once its copies in flight have landed
  unsigned int wait_polls;
  int chunk;      // cells along the march axis per CTA
  // uniform Cartesian grids: 1 / width per direction and the largest width
  T uni_inv[3];
  T uni_h;
  // learned guess (Newton mode): cells whose first linearised solve changes T
  // by more than mlp_gate go to a queue solved by the queue pass
  long long* queue;
  unsigned int* queue_count;
  unsigned int queue_cap;  // 0: no learned guess
  float mlp_gate;
  const float* mlp_w;      // parameters of the network (MLP_NPARAM floats)
  // training records of converged solves: float4 (x1, x2, log(T/T^n), gate)
  float* log;
  unsigned int* log_count;
  unsigned int log_cap;    // 0: no logging
  long long log_stride;
};

}  // namespace m1
