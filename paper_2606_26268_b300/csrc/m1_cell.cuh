// m1_cell.cuh -- per-cell end of the step, shared by the fused step kernel
// and the learned-guess queue pass: implicit coupling (Sect. 2.8), E floor,
// scattering update of F (Eq. source_discrete2), |F| <= E, gas bookkeeping
// (Sect. 2.7), stores of the cell and of the ghost copies it feeds, and the
// optional record of the solve for training the learned guess.
#pragma once
#include "m1_internal.h"

namespace m1 {

// Counters of one CTA.  The frequent events (fixed face states, coupling
// iterations) are counted per thread in registers; the rare ones (E floor,
// |F| clip, Newton restart, no convergence, an iteration count above 1) go
// straight to the CTA's shared counters s_rare, so that they hold no
// registers in the step's main loop.  Status bits go to the status word
// directly (rare too).
struct Counters {
  unsigned int fix = 0, iters = 0;
};

enum { RARE_EFLOOR = 0, RARE_FCLIP, RARE_FALLBACK, RARE_NOCONV, RARE_ITMAX, RARE_N };
static __shared__ unsigned int s_rare[RARE_N];

__device__ __forceinline__ void rare_add(int k) { atomicAdd(&s_rare[k], 1u); }

// Zeroes the CTA's shared counters; a barrier must follow before any event.
__device__ __forceinline__ void counters_reset(unsigned long long* s_red, int tid) {
  if (tid < ST_N) s_red[tid] = 0ull;
  if (tid < RARE_N) s_rare[tid] = 0u;
}

// Adds the CTA's counters to stats (one atomic per counter per CTA).  Called
// by every thread of the CTA; s_red holds ST_N shared words zeroed by
// counters_reset.
template <class P>
__device__ __forceinline__ void counters_flush(const StepArgs<P>& a, const Counters& c,
                                               unsigned long long* s_red, int tid) {
  unsigned long long f = c.fix, it = c.iters;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    f += __shfl_down_sync(0xffffffffu, f, off);
    it += __shfl_down_sync(0xffffffffu, it, off);
  }
  __syncthreads();  // every event of the CTA has been counted
  if ((tid & 31) == 0) {
    if (f) atomicAdd(&s_red[ST_FIX], f);
    if (it) atomicAdd(&s_red[ST_ITERS], it);
  }
  __syncthreads();
  if (tid == 0) {
    s_red[ST_EFLOOR] = s_rare[RARE_EFLOOR];
    s_red[ST_FCLIP] = s_rare[RARE_FCLIP];
    s_red[ST_FALLBACK] = s_rare[RARE_FALLBACK];
    s_red[ST_NOCONV] = s_rare[RARE_NOCONV];
    // every finished cell took at least one iteration
    const unsigned int im = s_rare[RARE_ITMAX];
    s_red[ST_ITMAX] = s_red[ST_ITERS] ? (im > 1u ? im : 1u) : 0u;
  }
  __syncthreads();
  if (tid < ST_N && s_red[tid]) {
    if (tid == ST_ITMAX)
      atomicMax(a.stats + tid, s_red[tid]);
    else
      atomicAdd(a.stats + tid, s_red[tid]);
  }
}

// Dimensionless inputs of the converged coupling: the root y = T/T^n of
// (y - 1) + alpha (y^4 - eps) = 0 depends only on
//   alpha = g a T^n^3 / ((1 + g_r) C_v),  eps = E* / (a T^n^4),
// returned as x1 = log10(alpha) / 4 and x2 = log10(eps) / 4, clamped to
// [-2, 2].  lin = alpha |eps - 1| / (1 + 4 alpha) is the relative change of T
// of the first linearised solve (the gate of the learned guess).
__device__ __forceinline__ void coupling_features(const CoupleParams& p, float rho, float e,
                                                  float kp, float Es, float& x1, float& x2,
                                                  float& lin, float& Tn) {
  float Cv = rho * p.f_cvfac;
  Tn = e * rcp_approx(Cv);
  float gr = p.f_dtchat * kp * rho;
  float g = p.f_dtc * kp * rho;
  float aT3 = p.f_a * Tn * Tn * Tn;
  float alpha = g * aT3 * rcp_approx((1.f + gr) * Cv);
  float eps = Es * rcp_approx(aT3 * Tn);
  const float kQ = 0.25f * 0.30102999566398120f;  // log10(x) / 4 = lg2(x) * log10(2) / 4
  x1 = fminf(fmaxf(lg2_approx(fmaxf(alpha, 1e-30f)) * kQ, -2.f), 2.f);
  x2 = fminf(fmaxf(lg2_approx(fmaxf(eps, 1e-30f)) * kQ, -2.f), 2.f);
  lin = alpha * fabsf(eps - 1.f) * rcp_approx(1.f + 4.f * alpha);
}

// The implicit coupling of the cell at padded index ic (Sect. 2.8): the
// single linearised solve when `once`, else the mode of the parameters
// (Newton from T0 > 0 or T^n; with T1 > 0, the single solve's result, Newton
// continues from it or from T0, whichever leaves the smaller residual).
// GEN (the general form) adds the absorption-only mode and the irradiation
// deposit of Sect. 2.9 when the context has them; the default step kernels,
// which such contexts do not use, compile both out.
template <class P, bool GEN = true>
__device__ __forceinline__ CoupleOutT<typename P::T> couple_cell(const StepArgs<P>& a, long long ic,
                                                 typename P::S rho_s, typename P::S e_s,
                                                 typename P::T kp, typename P::T Es, float T0,
                                                 bool once, double T1 = 0.0) {
  using T = typename P::T;
  if constexpr (GEN) {
    const bool ab = a.cp.absorb;
    const T sq = a.qirr ? a.dt * T(__ldg(a.qirr + ic)) : T(0);
    if constexpr (P::kSplit)
      return couple_split(a.cp, float(rho_s), float(e_s), float(kp), float(Es), T0, once,
                          float(sq), ab, float(T1));
    else
      return couple_fp64(a.cp, double(rho_s), double(e_s), double(kp), double(Es), double(T0),
                         once, double(sq), ab, T1);
  } else {
    if constexpr (P::kSplit)
      return couple_split(a.cp, float(rho_s), float(e_s), float(kp), float(Es), T0, once, 0.f,
                          false, float(T1));
    else
      return couple_fp64(a.cp, double(rho_s), double(e_s), double(kp), double(Es), double(T0),
                         once, 0.0, false, T1);
  }
}

// Bookkeeping and stores of the cell at padded index ic with unpadded
// coordinates ci, given its coupling result co.  Us = (E*, F*) after
// transport (E* already floored); I, the type of ic, may be a 32-bit index
// where every padded array has fewer than 2^31 cells.  ghosts = false: the
// caller knows the cell lies at least two cells from every boundary, so it
// feeds no ghost copy.
template <class P, int NDIM, int NC, bool GEN = true, class I = long long>
__device__ __forceinline__ void finish_cell(const StepArgs<P>& a, I ic, const int (&ci)[3],
                                            typename P::T (&Us)[4], typename P::S rho_s,
                                            typename P::S e_s, typename P::T kp,
                                            typename P::T chi, const typename P::T (&mom)[3],
                                            const CoupleOutT<typename P::T>& co, Counters& c,
                                            bool ghosts = true) {
  using S = typename P::S;
  using T = typename P::T;
  const StepDims& Dm = a.dim;
  c.iters += co.iters;
  if (co.iters > 1) atomicMax(&s_rare[RARE_ITMAX], (unsigned int)co.iters);
  if (co.fallback) rare_add(RARE_FALLBACK);
  if (co.noconv) {
    rare_add(RARE_NOCONV);
    atomicOr(a.status, STATUS_NOCONV);
  }
  // record (features, converged log(T/T^n)) for training the learned guess
  if (a.log_cap && a.cp.newton && !co.noconv) {
    long long lin_idx = ci[0] + (long long)Dm.n[0] * (ci[1] + (long long)Dm.n[1] * ci[2]);
    if (lin_idx % a.log_stride == 0) {
      float x1, x2, glin, Tn;
      coupling_features(a.cp, float(rho_s), float(e_s), float(kp), float(Us[0]), x1, x2, glin, Tn);
      unsigned int slot = atomicAdd(a.log_count, 1u);
      if (slot < a.log_cap)
        reinterpret_cast<float4*>(a.log)[slot] =
            make_float4(x1, x2, float(log(double(co.Tnew) / double(Tn))), glin);
    }
  }
  T En = Us[0] + T(co.dE);
  T dE = T(co.dE);
  if (En < a.efloor) {
    En = a.efloor;
    dE = En - Us[0];
    rare_add(RARE_EFLOOR);
  }
  // Eq. (source_discrete2): F^{n+1} (1 + dt chat chi rho) = F*
  T x = a.dt * a.chat * chi * T(rho_s);
  T Fn[3], dF[3];
  T inv = Ops<T>::rcp(T(1) + x);
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    if (v < NC) {
      if constexpr (sizeof(T) == 8) {
        Fn[v] = Us[1 + v] / (T(1) + x);
        dF[v] = Fn[v] - Us[1 + v];
      } else {
        dF[v] = -Us[1 + v] * x * inv;
        Fn[v] = Us[1 + v] + dF[v];
      }
    } else {
      Fn[v] = dF[v] = T(0);
    }
  }
  T nF2 = Fn[0] * Fn[0] + Fn[1] * Fn[1] + Fn[2] * Fn[2];
  if (nF2 > En * En) {
    T r = Ops<T>::div(En, Ops<T>::sqrt_(nF2));
#pragma unroll
    for (int v = 0; v < NC; ++v) {
      Fn[v] *= r;
      dF[v] = Fn[v] - Us[1 + v];
    }
    rare_add(RARE_FCLIP);
  }
  // Sect. 2.7: E_gas + (c/chat) E_r and m + F/chat are conserved; the
  // internal energy takes the kinetic-energy change.
  T mn[3], dke = T(0);
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    T dm = -dF[v] * a.inv_chat;
    mn[v] = mom[v] + dm;
    dke += dm * (T(2) * mom[v] + dm);
  }
  T rr = T(rho_s);
  T en;
  if constexpr (sizeof(T) == 8)
    en = T(e_s) - a.ratio * dE - dke / (T(2) * rr);
  else
    en = T(e_s) - a.ratio * dE - dke * T(0.5) * rcp_approx(rr);
  // Sect. 2.9: E_gas gains dt (-div F_irr) (reloaded here rather than kept
  // live through the coupling)
  if (GEN && a.qirr) en += a.dt * T(__ldg(a.qirr + ic));
  T rfin = T(rho_s);  // the cell's final density
  if (a.average) {
    // last stage of the two-stage step: average with U^n, which the output
    // buffer holds at this cell (only this thread reads or writes it)
    T mo[3] = {0, 0, 0}, ma[3] = {0, 0, 0};
#pragma unroll
    for (int v = 0; v < NC; ++v) {
      mo[v] = T(a.out.m[v][ic]);
      ma[v] = T(0.5) * (mo[v] + mn[v]);
    }
    T h = T(0.5) * Ops<T>::rcp(T(rho_s));
    T ho = h, ha = h;
    if constexpr (GEN) {
      if (a.rho_avg) {  // the gas step moved rho: average it too
        const T rn = T(a.rho_avg[ic]);
        rfin = T(0.5) * (rn + T(rho_s));
        ho = T(0.5) * Ops<T>::rcp(rn);
        ha = T(0.5) * Ops<T>::rcp(rfin);
        a.rho_avg[ic] = S(rfin);
      }
    }
    const T ko = (mo[0] * mo[0] + mo[1] * mo[1] + mo[2] * mo[2]) * ho;
    const T kn = (mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]) * h;
    const T ka = (ma[0] * ma[0] + ma[1] * ma[1] + ma[2] * ma[2]) * ha;
    const T eg = T(0.5) * ((T(a.out.e[ic]) + ko) + (en + kn));
    En = T(0.5) * (T(a.out.E[ic]) + En);
#pragma unroll
    for (int v = 0; v < NC; ++v) {
      Fn[v] = T(0.5) * (T(a.out.F[v][ic]) + Fn[v]);
      mn[v] = ma[v];
    }
    en = eg - ka;
  }
  if (!(En > T(0) && en > T(0))) atomicOr(a.status, STATUS_NONPHYS);  // also NaN
  // stores: own cell and the ghost copies it feeds
  if (!index_ok((long long)ic, padded_cells(Dm), a.status)) return;
  a.out.E[ic] = S(En);
#pragma unroll
  for (int v = 0; v < NC; ++v) {
    a.out.F[v][ic] = S(Fn[v]);
    a.out.m[v][ic] = S(mn[v]);
  }
  a.out.e[ic] = S(en);
  // ghost copies: wrapped (periodic), edge (outflow), mirrored with the
  // normal components negated (reflective), F only (LTE: E, e held); the
  // FIXED sides hold their boundary state
  if (!ghosts) return;
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    const int n = Dm.n[d];
    const int i = ci[d];
    if (i >= 2 && i < n - 2) continue;
    const long long stride = d == 0 ? 1ll : (d == 1 ? Dm.sy : Dm.sz);
#pragma unroll
    for (int gslot = 0; gslot < 4; ++gslot) {
      const bool lo = gslot < 2;
      const int gpos = lo ? gslot - 2 : n + gslot - 2;  // -2, -1, n, n+1
      const int bc = lo ? Dm.bc_lo[d] : Dm.bc_hi[d];
      bool gas_held = false;  // evolved gas: keep the held gas ghosts in step
      if constexpr (GEN) gas_held = a.hydro && (bc == BC_FIXED || bc == BC_LTE);
      if (bc == BC_FIXED && !gas_held) continue;
      int src;
      if (bc == BC_PERIODIC)
        src = lo ? ((gpos % n) + n) % n : gpos % n;
      else if (bc == BC_REFLECT)
        src = min(max(lo ? -1 - gpos : 2 * n - 1 - gpos, 0), n - 1);
      else
        src = lo ? 0 : n - 1;
      if (src != i) continue;
      const long long ig = (long long)ic + (long long)(gpos - i) * stride;
      if (!index_ok(ig, padded_cells(Dm), a.status)) continue;
      if constexpr (GEN) {
        if (a.rho_avg) a.rho_avg[ig] = S(rfin);
        if (gas_held) {
          a.out.e[ig] = S(T(a.cp.cvfac) * rfin * T(a.bcT[d][lo ? 0 : 1]));
#pragma unroll
          for (int v = 0; v < NC; ++v) a.out.m[v][ig] = S(0);
          if (bc == BC_LTE)
#pragma unroll
            for (int v = 0; v < NC; ++v) a.out.F[v][ig] = S(Fn[v]);
          continue;
        }
      }
      const bool refl = bc == BC_REFLECT;
      const bool all = bc != BC_LTE;
      if (all) {
        a.out.E[ig] = S(En);
        a.out.e[ig] = S(en);
      }
#pragma unroll
      for (int v = 0; v < NC; ++v) {
        const bool neg = refl && v == d;
        a.out.F[v][ig] = S(neg ? -Fn[v] : Fn[v]);
        if (all) a.out.m[v][ig] = S(neg ? -mn[v] : mn[v]);
      }
    }
  }
}

}  // namespace m1
