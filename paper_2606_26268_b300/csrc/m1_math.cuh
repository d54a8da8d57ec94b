// m1_math.cuh -- per-state and per-cell arithmetic of the M1 radiation step
// (device code, sm_103a).  Two precision policies:
//   Fp64  : storage, transport and coupling in double, IEEE division/sqrt;
//   Split : float storage and transport (MUFU approximations of rcp, rsqrt,
//           sqrt, ex2, lg2); the coupling's E - a T^4 residual to within one
//           float rounding (compensated float in the single solve, double in
//           the Newton iterations), the remaining well-conditioned coupling
//           products in float.
#pragma once
#include <cstdint>

namespace m1 {

// ---------------------------------------------------------------------------
// scalar helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Packed pairs of FP32 values: the f32x2 arithmetic of sm_100 and later
// does both lanes in one instruction.  A state (E, F0, F1, F2) is two pairs;
// each lane is the IEEE round-to-nearest result of the scalar operation.
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
// a * b + c with one rounding per lane.
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(r)
      : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
  return f2_unpack(r);
}

template <class T> struct Ops;

template <> struct Ops<double> {
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
  static __device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
};

template <> struct Ops<float> {
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp_approx(b); }
  static __device__ __forceinline__ float rcp(float a) { return rcp_approx(a); }
  static __device__ __forceinline__ float sqrt_(float a) { return sqrt_approx(a); }
};

struct Fp64 {
  using S = double;  // storage
  using T = double;  // transport arithmetic
  static constexpr bool kSplit = false;
};
struct Split {
  using S = float;
  using T = float;
  static constexpr bool kSplit = true;
};

// ---------------------------------------------------------------------------
// PLM with the van Leer limiter (Sect. 2.5)
// ---------------------------------------------------------------------------

// Limited slope from the two one-sided slopes: the harmonic mean
// 2 dl dr / (dl + dr) when they have the same sign, else zero.
template <class T>
__device__ __forceinline__ T vanleer(T dl, T dr) {
  T p = dl * dr;
  return p > T(0) ? Ops<T>::div(T(2) * p, dl + dr) : T(0);
}

// ---------------------------------------------------------------------------
// f-preserving face fix, Eq. (f_reconstruct)
// ---------------------------------------------------------------------------

// uf = (Ef, Ff) is the reconstructed face state of the cell uc = (Ec, Fc)
// with nc2 = |Fc|^2.  The reconstructed flux is kept iff f_face <= 1 and
// f_face > f_centre (compared without division: Ef, Ec > 0; in float the
// squared ratios, with f_centre^2 from inv_Ec = 1 / Ec); otherwise
// F_face = F_centre * E_face / E_centre.  Returns true when recomputed.
template <class T, int NC>
__device__ __forceinline__ bool fix_face(T (&uf)[4], const T (&uc)[4], T nc2, T inv_Ec) {
  T nf2 = uf[1] * uf[1];
  if (NC > 1) nf2 += uf[2] * uf[2];
  if (NC > 2) nf2 += uf[3] * uf[3];
  const T Ef = uf[0], Ec = uc[0];
  bool keep;
  if constexpr (sizeof(T) == 8) {
    keep = (nf2 <= Ef * Ef) && (nf2 * (Ec * Ec) > nc2 * (Ef * Ef));
  } else {
    // f_centre^2 = nc2 / Ec^2 is the same for every face state of the cell
    const T Ef2 = Ef * Ef;
    keep = (nf2 <= Ef2) && (nf2 > (nc2 * (inv_Ec * inv_Ec)) * Ef2);
  }
  if constexpr (sizeof(T) == 8) {
    if (!keep) {
      T r = Ef / Ec;
      uf[1] = uc[1] * r;
      if (NC > 1) uf[2] = uc[2] * r;
      if (NC > 2) uf[3] = uc[3] * r;
    }
  } else {
    // selects rather than a branch: lanes of a warp disagree often
    const T r = Ef * inv_Ec;
    uf[1] = keep ? uf[1] : uc[1] * r;
    if (NC > 1) uf[2] = keep ? uf[2] : uc[2] * r;
    if (NC > 2) uf[3] = keep ? uf[3] : uc[3] * r;
  }
  return !keep;
}

// ---------------------------------------------------------------------------
// Closure (Sect. 2.1) and signal speeds (Sect. 2.6) of one state along D
// ---------------------------------------------------------------------------

// Physical flux (chat F_D, chat D_{D j} E) and the eigenvalues lambda_{1,3}
// (units of chat) of the state (E, F) along direction D.
//   f = min(|F|/E, 1), s = sqrt(4 - 3 f^2), xi = (3 + 4 f^2) / (5 + 2 s),
//   D E = a delta + b F F  with a = (1 - xi) E / 2, b = (3 xi - 1) E / (2 |F|^2),
//   lambda = (f cos(theta) +/- zeta) / s.
// zeta^2 of Sect. 2.6 is evaluated in the algebraically identical form
//   zeta^2 = 2 (1 - f^2) (s (1 + c^2) - 2 c^2) / (s + 1),  c = cos(theta),
// which is non-negative term by term and free of the cancellation of
// 4 - 3 f^2 - s as f -> 1.
template <class T, int NC, int D>
__device__ __forceinline__ void state_flux(const T (&u)[4], T chat, T (&flux)[4], T& lm,
                                           T& lp) {
  const T E = u[0];
  const T F[3] = {u[1], u[2], u[3]};
  T nF2 = F[0] * F[0];
  if (NC > 1) nF2 += F[1] * F[1];
  if (NC > 2) nF2 += F[2] * F[2];
  const T Fd = (D < NC) ? F[D] : T(0);
  T f, fc, c2, b;
  T invE = Ops<T>::rcp(E);
  if constexpr (sizeof(T) == 8) {
    T nF = sqrt(nF2);
    f = nF / E;
    if (f > T(1)) f = T(1);
    T cth = (nF > T(0)) ? Fd / nF : T(0);
    fc = f * cth;
    c2 = cth * cth;
    b = T(0);
    T f2 = f * f;
    T s = sqrt(T(4) - T(3) * f2);
    T xi = (T(3) + T(4) * f2) / (T(5) + T(2) * s);
    T a = T(0.5) * (T(1) - xi) * E;
    if (nF > T(0)) b = T(0.5) * (T(3) * xi - T(1)) * E / nF2;
    flux[0] = chat * Fd;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T Fj = (j < NC) ? F[j] : T(0);
      T dj = (j == D ? a : T(0)) + b * Fd * Fj;
      if (j < NC) flux[1 + j] = chat * dj;
    }
    T z2 = T(2) * (T(1) - f2) * (s * (T(1) + c2) - T(2) * c2) / (s + T(1));
    T z = sqrt(z2 > T(0) ? z2 : T(0));
    lp = (fc + z) / s;
    lm = (fc - z) / s;
  } else {
    // |F|^2 is clamped to 1e-37 under the rsqrt: the flush-to-zero rsqrt
    // would turn a denormal or zero |F|^2 into an infinite 1/|F|.  F = 0
    // still gives zero f and zero direction terms, and below the clamp the
    // closure depends on the direction of F only at O(f^2).
    T rn = rsqrt_approx(fmaxf(nF2, T(1e-37)));
    T nF = nF2 * rn;
    f = nF * invE;
    f = f > T(1) ? T(1) : f;
    T cth = Fd * rn;
    fc = f * cth;
    c2 = cth * cth;
    T f2 = f * f;
    T q = T(4) - T(3) * f2;
    T rs = rsqrt_approx(q);
    T s = q * rs;
    // (5 + 2 s)(5 - 2 s) = 25 - 4 s^2 = 3 (3 + 4 f^2), so xi = (5 - 2 s) / 3
    // exactly: (1 - xi) / 2 = (s - 1) / 3 and (3 xi - 1) / 2 = 2 - s, with no
    // division.
    T t = s * T(1.0 / 3.0) - T(1.0 / 3.0);
    T b2 = T(2) - s;
    T Ec = E * chat;
    T ac = t * Ec;
    T bFd = (b2 * Ec) * (cth * rn);
    flux[0] = chat * Fd;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (j < NC) {
        T v = bFd * F[j];
        flux[1 + j] = (j == D) ? v + ac : v;
      }
    }
    // (1 - f^2) / (s + 1) = (s - 1) / 3 since s^2 - 1 = 3 (1 - f^2), and
    // s (1 + c^2) - 2 c^2 = s - c^2 (2 - s)
    T z2 = T(2) * t * (s - c2 * b2);
    T z = sqrt_approx(z2 > T(0) ? z2 : T(0));
    lp = (fc + z) * rs;
    lm = (fc - z) * rs;
  }
}

// Pressure tensor P = D E of a cell-centred state (for the geometric
// sources): P_ij = a delta_ij + b F_i F_j.
template <class T, int NC>
__device__ __forceinline__ void pressure(const T (&u)[4], T& a, T& b) {
  const T E = u[0];
  T nF2 = u[1] * u[1];
  if (NC > 1) nF2 += u[2] * u[2];
  if (NC > 2) nF2 += u[3] * u[3];
  if (sizeof(T) == 4 && !(nF2 > T(1e-37))) nF2 = T(0);
  T nF = Ops<T>::sqrt_(nF2);
  T f = Ops<T>::div(nF, E);
  f = f > T(1) ? T(1) : f;
  T f2 = f * f;
  T s = Ops<T>::sqrt_(T(4) - T(3) * f2);
  T xi = Ops<T>::div(T(3) + T(4) * f2, T(5) + T(2) * s);
  a = T(0.5) * (T(1) - xi) * E;
  b = nF2 > T(0) ? Ops<T>::div(T(0.5) * (T(3) * xi - T(1)) * E, nF2) : T(0);
}

// HLL flux (Sect. 2.5) with the signal speeds of Sect. 2.6:
// S_L = chat min(lm_L, lm_R), S_R = chat max(lp_L, lp_R), limited to
// -/+ 4 chat / (3 tau) when tau > 0.
template <class T, int NV>
__device__ __forceinline__ void hll(const T (&uL)[4], const T (&uR)[4], const T (&fL)[4],
                                    const T (&fR)[4], T lmL, T lpL, T lmR, T lpR, T chat,
                                    T tau, T (&out)[4]) {
  if constexpr (sizeof(T) == 8) {
    T sl = chat * (lmL < lmR ? lmL : lmR);
    T sr = chat * (lpL > lpR ? lpL : lpR);
    if (tau > T(0)) {
      T bound = T(4) * chat / (T(3) * tau);
      if (sl < -bound) sl = -bound;
      if (sr > bound) sr = bound;
    }
    if (sl >= T(0)) {
#pragma unroll
      for (int q = 0; q < NV; ++q) out[q] = fL[q];
    } else if (sr <= T(0)) {
#pragma unroll
      for (int q = 0; q < NV; ++q) out[q] = fR[q];
    } else {
#pragma unroll
      for (int q = 0; q < NV; ++q)
        out[q] = (sr * fL[q] - sl * fR[q] + sl * sr * (uR[q] - uL[q])) / (sr - sl);
    }
  } else {
    // Branch-free form: with S_L <= 0 <= S_R enforced the same expression
    // gives the two upwind cases (S_L = 0 -> F_L, S_R = 0 -> F_R); the
    // thick-limit bound 4 chat / (3 tau) is +inf when tau = 0.
    T bound = (T(4.0 / 3.0) * chat) * rcp_approx(tau);
    T sl = fmaxf(fminf(chat * fminf(lmL, lmR), T(0)), -bound);
    T sr = fminf(fmaxf(chat * fmaxf(lpL, lpR), T(0)), bound);
    T inv = rcp_approx(fmaxf(sr - sl, T(1e-30)));
    T slsr = sl * sr;
    if constexpr (NV == 4) {  // two packed pairs
      const float2 SR = make_float2(sr, sr), MSL = make_float2(-sl, -sl);
      const float2 SLSR = make_float2(slsr, slsr), INV = make_float2(inv, inv);
#pragma unroll
      for (int h = 0; h < 4; h += 2) {
        const float2 du = f2_sub(make_float2(uR[h], uR[h + 1]), make_float2(uL[h], uL[h + 1]));
        float2 acc = f2_mul(MSL, make_float2(fR[h], fR[h + 1]));
        acc = f2_fma(SLSR, du, acc);
        acc = f2_fma(SR, make_float2(fL[h], fL[h + 1]), acc);
        acc = f2_mul(acc, INV);
        out[h] = acc.x;
        out[h + 1] = acc.y;
      }
    } else {
#pragma unroll
      for (int q = 0; q < NV; ++q)
        out[q] = (sr * fL[q] - sl * fR[q] + slsr * (uR[q] - uL[q])) * inv;
    }
  }
}

// Lax-Friedrichs-Rusanov flux (Sect. 2.5) with the local speed
// S = max(|S_L|, |S_R|) of the thick-limited signal speeds of Sect. 2.6:
// (F_L + F_R) / 2 - S (U_R - U_L) / 2.
template <class T, int NV>
__device__ __forceinline__ void lf(const T (&uL)[4], const T (&uR)[4], const T (&fL)[4],
                                   const T (&fR)[4], T lmL, T lpL, T lmR, T lpR, T chat, T tau,
                                   T (&out)[4]) {
  T sl = chat * (lmL < lmR ? lmL : lmR);
  T sr = chat * (lpL > lpR ? lpL : lpR);
  if (tau > T(0)) {
    T bound = Ops<T>::div(T(4) * chat, T(3) * tau);
    if (sl < -bound) sl = -bound;
    if (sr > bound) sr = bound;
  }
  const T S = fabs(sl) > fabs(sr) ? fabs(sl) : fabs(sr);
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = T(0.5) * (fL[q] + fR[q]) - T(0.5) * S * (uR[q] - uL[q]);
}

// LimO3 (Sect. 2.5): the increment phi(theta) dt / 2 from the cell value to
// its face on the side of the one-sided difference dt, theta = dn / dt with
// dn the other one; phi = max(0, min(phi3, max(-theta/2, min(2 theta, phi3,
// 3/2)))), phi3 = (2 + theta) / 3 the unlimited third-order value.  Zero
// when dt = 0.
template <class T>
__device__ __forceinline__ T limo3(T dn, T dt) {
  if (dt == T(0)) return T(0);
  const T th = Ops<T>::div(dn, dt);
  const T p3 = Ops<T>::div(T(2) + th, T(3));
  T a = T(2) * th;
  if (p3 < a) a = p3;
  if (T(1.5) < a) a = T(1.5);
  if (T(-0.5) * th > a) a = T(-0.5) * th;
  if (p3 < a) a = p3;
  if (a < T(0)) a = T(0);
  return T(0.5) * a * dt;
}

// ---------------------------------------------------------------------------
// Opacities
// ---------------------------------------------------------------------------

struct OpacityDev {
  int kind;                    // 0 const, 1 powerlaw, 2 table
  double kappa_p, kappa_r, sigma;
  double k0, a_rho, b_T, kmin, kmax, sigma_ratio;
  int nrho, nT;
  double lrho0, lT0, sr, sT;   // sr = (nrho-1)/(lrho1-lrho0), sT likewise
  const double* tab64;         // log10 kappa, [iT][irho]
  const float* tab32;
  int linear_rho;              // powerlaw with a = 1, b = 0 (kappa = k0 rho)
  // float copies for the split-precision path (no double conversions there)
  float f_kp, f_chi0, f_k0, f_a, f_b, f_kmin, f_kmax, f_s1, f_lrho0, f_lT0, f_sr, f_sT;
  // log2 of C_v / rho = 1 / (mu (Gamma - 1)), and b_T times it and a_rho - b_T, for
  // the opacities from (rho, e) without forming T
  float f_lcv, f_blcv, f_amb;
};

// Opacities per unit mass at (rho, T): kp (Planck), chi = kappa_R + sigma.
__device__ __forceinline__ void opacity(const OpacityDev& o, double rho, double T, double& kp,
                                        double& chi) {
  if (o.kind == 0) {
    kp = o.kappa_p;
    chi = o.kappa_r + o.sigma;
    return;
  }
  double k;
  if (o.kind == 1) {
    k = o.k0 * pow(rho, o.a_rho) * pow(T, o.b_T);
    k = k < o.kmin ? o.kmin : k;
    k = k > o.kmax ? o.kmax : k;
  } else {
    double xr = (log10(rho) - o.lrho0) * o.sr;
    double xt = (log10(T) - o.lT0) * o.sT;
    xr = xr < 0.0 ? 0.0 : (xr > o.nrho - 1 ? double(o.nrho - 1) : xr);
    xt = xt < 0.0 ? 0.0 : (xt > o.nT - 1 ? double(o.nT - 1) : xt);
    int ir = int(floor(xr)), it = int(floor(xt));
    ir = ir > o.nrho - 2 ? o.nrho - 2 : ir;
    it = it > o.nT - 2 ? o.nT - 2 : it;
    double wr = xr - ir, wt = xt - it;
    const double* t = o.tab64 + it * o.nrho + ir;
    double l00 = __ldg(t), l10 = __ldg(t + 1), l01 = __ldg(t + o.nrho), l11 = __ldg(t + o.nrho + 1);
    double lk = (1.0 - wr) * (1.0 - wt) * l00 + wr * (1.0 - wt) * l10 + (1.0 - wr) * wt * l01 +
                wr * wt * l11;
    k = pow(10.0, lk);
  }
  kp = k;
  chi = k * (1.0 + o.sigma_ratio);
}

__device__ __forceinline__ void opacity(const OpacityDev& o, float rho, float T, float& kp,
                                        float& chi) {
  if (o.kind == 0) {
    kp = o.f_kp;
    chi = o.f_chi0;
    return;
  }
  float k;
  if (o.kind == 1) {
    if (o.linear_rho) {
      k = o.f_k0 * rho;
    } else {
      k = o.f_k0 * ex2_approx(o.f_a * lg2_approx(rho) + o.f_b * lg2_approx(T));
    }
    k = k < o.f_kmin ? o.f_kmin : k;
    k = k > o.f_kmax ? o.f_kmax : k;
  } else {
    const float kLog10_2 = 0.30102999566398120f;
    float xr = (lg2_approx(rho) * kLog10_2 - o.f_lrho0) * o.f_sr;
    float xt = (lg2_approx(T) * kLog10_2 - o.f_lT0) * o.f_sT;
    xr = fminf(fmaxf(xr, 0.f), float(o.nrho - 1));
    xt = fminf(fmaxf(xt, 0.f), float(o.nT - 1));
    int ir = min(int(xr), o.nrho - 2), it = min(int(xt), o.nT - 2);
    float wr = xr - ir, wt = xt - it;
    const float* t = o.tab32 + it * o.nrho + ir;
    float l00 = __ldg(t), l10 = __ldg(t + 1), l01 = __ldg(t + o.nrho), l11 = __ldg(t + o.nrho + 1);
    float lk = (1.f - wr) * ((1.f - wt) * l00 + wt * l01) + wr * ((1.f - wt) * l10 + wt * l11);
    k = ex2_approx(lk * 3.32192809488736235f);
  }
  kp = k;
  chi = k * o.f_s1;
}

// The same opacities at (rho, T = e / (rho C_v/rho)) from log2 T = log2 e -
// log2 rho - log2 (C_v/rho), in float: no reciprocal and no T (the power law
// k0 rho^a T^b = k0 2^((a - b) log2 rho + b log2 e - b log2 (C_v/rho))).
__device__ __forceinline__ void opacity_re(const OpacityDev& o, float rho, float e, float& kp,
                                           float& chi) {
  if (o.kind == 0) {
    kp = o.f_kp;
    chi = o.f_chi0;
    return;
  }
  float k;
  if (o.kind == 1) {
    if (o.linear_rho) {
      k = o.f_k0 * rho;
    } else {
      k = o.f_k0 * ex2_approx(fmaf(o.f_amb, lg2_approx(rho), fmaf(o.f_b, lg2_approx(e), -o.f_blcv)));
    }
    k = k < o.f_kmin ? o.f_kmin : k;
    k = k > o.f_kmax ? o.f_kmax : k;
  } else {
    const float kLog10_2 = 0.30102999566398120f;
    const float lr = lg2_approx(rho);
    float xr = (lr * kLog10_2 - o.f_lrho0) * o.f_sr;
    float xt = ((lg2_approx(e) - lr - o.f_lcv) * kLog10_2 - o.f_lT0) * o.f_sT;
    xr = fminf(fmaxf(xr, 0.f), float(o.nrho - 1));
    xt = fminf(fmaxf(xt, 0.f), float(o.nT - 1));
    int ir = min(int(xr), o.nrho - 2), it = min(int(xt), o.nT - 2);
    float wr = xr - ir, wt = xt - it;
    const float* t = o.tab32 + it * o.nrho + ir;
    float l00 = __ldg(t), l10 = __ldg(t + 1), l01 = __ldg(t + o.nrho), l11 = __ldg(t + o.nrho + 1);
    float lk = (1.f - wr) * ((1.f - wt) * l00 + wt * l01) + wr * ((1.f - wt) * l10 + wt * l11);
    k = ex2_approx(lk * 3.32192809488736235f);
  }
  kp = k;
  chi = k * o.f_s1;
}

// ---------------------------------------------------------------------------
// Implicit coupling (Sect. 2.8)
// ---------------------------------------------------------------------------

struct CoupleParams {
  double dt, chat, c, a_rad, cvfac;  // cvfac = 1 / (mu (gamma - 1)): C_v = rho cvfac
  double rtol;
  int maxit, newton;
  int absorb;  // absorption only: E^{n+1} = E* / (1 + g_r), no emission (general form)
  // float copies for the split-precision path
  float f_dtchat, f_dtc, f_cvfac, f_a, f_rtol;
  float f_a_lo;  // a_R - f_a in float: (f_a, f_a_lo) carries a_R to about 48 bits
  int a_is_one;  // a_R == 1 (code units): the emission term needs no scaling
};

// Result of the coupling of one cell, in the precision of the transport
// (double for the FP64 form, float for the split form, whose T^{n+1} and
// E^{n+1} - E* are stored in float).
template <class R>
struct CoupleOutT {
  R dE;          // E^{n+1} - E*
  R Tnew;        // T^{n+1} of the solve
  int iters;
  int fallback;  // restarted from T^n
  int noconv;
  int conv1;     // single solve only: it already passes the Newton convergence test
};
using CoupleOut = CoupleOutT<double>;

// Increments of the 2x2 system of Eq. (implicit_matrix) with T^4 linearised
// about Tk.  With D = E* - a Tk^4, det = (1 + g_r) C_v + 4 g a Tk^3 and
// G = (1 + g_r) (C_v (T^n - Tk) + sq), Cramer's rule gives exactly
//   T^{n+1} - Tk = (G + g D) / det,
//   E^{n+1} - E* = g_r (4 a Tk^3 (C_v (T^n - Tk) + sq) - C_v D) / det,
// which for Tk = T^n is the paper's single solve.  sq = dt (-div F_irr) is
// the irradiation term that Sect. 2.9 adds to the gas row (0 without
// irradiation).  Newton mode repeats the solve with Tk <- T^{n+1} until
// |T^{n+1} - Tk| <= rtol T^{n+1}.
//
// Continuing after the single solve: T1 > 0 is the single solve's T^{n+1},
// which is the first Newton iterate from T^n.  The first attempt then
// starts from T1 (or from the learned guess T0 when T0 is given and leaves
// the smaller residual of the scalar equation
//   r(T) = (1 + g_r) (C_v (T - T^n) - sq) + g (a T^4 - E*)),
// counts the single solve as its first iteration and has maxit - 1 left;
// the restart from T^n after a failure is unchanged.  Without T1 the first
// attempt starts from T0 (or T^n) with maxit iterations.
__device__ __forceinline__ double couple_residual(const CoupleParams& p, double Cv, double g,
                                                  double gr, double Tn, double Es, double sq,
                                                  double T) {
  const double T2 = T * T;
  return (1.0 + gr) * (Cv * (T - Tn) - sq) + g * (p.a_rad * T2 * T2 - Es);
}

__device__ __forceinline__ CoupleOut couple_fp64(const CoupleParams& p, double rho, double e,
                                                 double kp, double Es, double T0,
                                                 bool once = false, double sq = 0.0,
                                                 bool absorb = false, double T1 = 0.0) {
  CoupleOut o{};
  double Cv = rho * p.cvfac;
  double Tn = e / Cv;
  double gr = p.dt * p.chat * kp * rho;
  double g = p.dt * p.c * kp * rho;
  double c1 = (1.0 + gr) * Cv;
  if (T0 <= 0.0) T0 = Tn;
  if (absorb) {  // absorption only: E^{n+1} = E* / (1 + g_r)
    o.dE = Es / (1.0 + gr) - Es;
    o.Tnew = Tn;
    o.iters = 1;
    o.conv1 = 1;
    return o;
  }
  if (!p.newton || once) {
    double aT3 = p.a_rad * Tn * Tn * Tn;
    double D = Es - aT3 * Tn;
    double det = c1 + 4.0 * g * aT3;
    double q = D / det;
    double dT = g * q;
    o.dE = -gr * Cv * q;
    if (sq != 0.0) {
      const double h = sq / det;
      dT += (1.0 + gr) * h;
      o.dE += gr * 4.0 * aT3 * h;
    }
    o.Tnew = Tn + dT;
    o.iters = 1;
    o.conv1 = fabs(dT) <= p.rtol * o.Tnew;
    return o;
  }
  int maxit0 = p.maxit;
  double Tstart = T0;
  if (T1 > 0.0) {
    o.iters = 1;  // the single solve, the first iterate from T^n
    maxit0 = p.maxit - 1;
    Tstart = T1;
    if (T0 > 0.0 && T0 != Tn &&
        fabs(couple_residual(p, Cv, g, gr, Tn, Es, sq, T0)) <
            fabs(couple_residual(p, Cv, g, gr, Tn, Es, sq, T1)))
      Tstart = T0;
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    double Tk = attempt == 0 ? Tstart : Tn;
    const int maxit = attempt == 0 ? maxit0 : p.maxit;
    bool ok = false;
    int it;
    double aT3 = 0.0, D = 0.0, det = 1.0, Tnew = Tk;
    for (it = 1; it <= maxit; ++it) {
      aT3 = p.a_rad * Tk * Tk * Tk;
      D = Es - aT3 * Tk;
      det = c1 + 4.0 * g * aT3;
      double dT = (c1 * (Tn - Tk) + (1.0 + gr) * sq + g * D) / det;
      Tnew = Tk + dT;
      if (!(Tnew > 0.0)) break;
      if (fabs(dT) <= p.rtol * Tnew) {
        ok = true;
        break;
      }
      Tk = Tnew;
    }
    int used = ok ? it : (it > maxit ? maxit : it);
    o.iters += used;
    if (ok || attempt == 1) {
      o.Tnew = Tnew;
      o.dE = gr * (4.0 * aT3 * (Cv * (Tn - Tk) + sq) - Cv * D) / det;
      o.noconv = ok ? 0 : 1;
      return o;
    }
    o.fallback = 1;
  }
  return o;
}

// Split precision: the residual E* - a T^4 of the single solve in
// compensated float (within one float rounding of exact), the T^4 term, the
// residual and the numerator of the Newton iterations in double; det and the
// final products, whose terms are all positive, in float.
__device__ __forceinline__ CoupleOutT<float> couple_split(const CoupleParams& p, float rho, float e,
                                                  float kp, float Es, float T0f,
                                                  bool once = false, float sq = 0.f,
                                                  bool absorb = false, float T1f = 0.f) {
  CoupleOutT<float> o{};
  float Cv = rho * p.f_cvfac;
  float invCv = rcp_approx(Cv);
  float Tf = e * invCv;
  float gr = p.f_dtchat * kp * rho;
  float g = p.f_dtc * kp * rho;
  float c1 = (1.f + gr) * Cv;
  if (absorb) {  // absorption only: E^{n+1} = E* / (1 + g_r)
    o.dE = -Es * gr * rcp_approx(1.f + gr);
    o.Tnew = Tf;
    o.iters = 1;
    o.conv1 = 1;
    return o;
  }
  if (!p.newton || once) {
    // E* - a T^4 without cancellation and without the (slow) FP64 pipe:
    // T^2 = t2 + t2e and t2^2 = t4 + t4e exactly (the FMA remainders), so
    // a T^4 = a (t4 + l4) with l4 = t4e + t2e (2 t2 + t2e) to about 2^-48
    // relative, and with a = f_a + f_a_lo the residual E* - a T^4 comes out
    // within one float rounding of its exact value, as from an FP64
    // evaluation rounded to float
    const float t2 = Tf * Tf;
    const float t2e = fmaf(Tf, Tf, -t2);
    const float t4 = t2 * t2;
    const float l4 = fmaf(t2e, fmaf(2.f, t2, t2e), fmaf(t2, t2, -t4));
    float D;
    if (p.a_is_one) {
      D = (Es - t4) - l4;
    } else {
      const float h = p.f_a * t4;
      const float he = fmaf(p.f_a, t4, -h);
      D = (Es - h) - fmaf(p.f_a, l4, fmaf(p.f_a_lo, t4, he));
    }
    float aT3 = p.f_a * Tf * Tf * Tf;
    float det = c1 + 4.f * g * aT3;
    const float rdet = rcp_approx(det);
    float q = D * rdet;
    float dT = g * q;
    float dE = -gr * Cv * q;
    if (sq != 0.f) {
      const float h = sq * rdet;
      dT += (1.f + gr) * h;
      dE += gr * 4.f * aT3 * h;
    }
    o.Tnew = Tf + dT;
    o.dE = dE;
    o.iters = 1;
    o.conv1 = fabsf(dT) <= p.f_rtol * o.Tnew;
    return o;
  }
  double Tn = double(Tf);
  double c1d = double(c1);
  // continuing after the single solve (see couple_fp64)
  int maxit0 = p.maxit;
  double Tstart = T0f > 0.f ? double(T0f) : Tn;
  if (T1f > 0.f) {
    o.iters = 1;
    maxit0 = p.maxit - 1;
    const double T1 = double(T1f);
    Tstart = T1;
    if (T0f > 0.f && double(T0f) != Tn) {
      const double Cvd = double(Cv), gd = double(g), grd = double(gr);
      if (fabs(couple_residual(p, Cvd, gd, grd, Tn, double(Es), double(sq), double(T0f))) <
          fabs(couple_residual(p, Cvd, gd, grd, Tn, double(Es), double(sq), T1)))
        Tstart = double(T0f);
    }
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    double Tk = attempt == 0 ? Tstart : Tn;
    const int maxit = attempt == 0 ? maxit0 : p.maxit;
    bool ok = false;
    int it;
    double aT3 = 0.0, D = 0.0;
    float det = 1.f;
    double Tnew = Tk;
    for (it = 1; it <= maxit; ++it) {
      aT3 = p.a_rad * Tk * Tk * Tk;
      D = double(Es) - aT3 * Tk;
      det = c1 + 4.f * g * float(aT3);
      double num = c1d * (Tn - Tk) + double(1.f + gr) * double(sq) + double(g) * D;
      double dT = num * double(rcp_approx(det));
      Tnew = Tk + dT;
      if (!(Tnew > 0.0)) break;
      if (fabsf(float(dT)) <= p.f_rtol * float(Tnew)) {
        ok = true;
        break;
      }
      Tk = Tnew;
    }
    int used = ok ? it : (it > maxit ? maxit : it);
    o.iters += used;
    if (ok || attempt == 1) {
      o.Tnew = float(Tnew);
      float inner = float(4.0 * aT3 * (double(Cv) * (Tn - Tk) + double(sq)) - double(Cv) * D);
      o.dE = gr * inner * rcp_approx(det);
      o.noconv = ok ? 0 : 1;
      return o;
    }
    o.fallback = 1;
  }
  return o;
}

}  // namespace m1
