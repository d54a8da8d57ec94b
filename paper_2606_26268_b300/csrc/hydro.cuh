// hydro.cuh -- the gas step that precedes the radiation transport in every
// (sub)step when the gas is evolved (Sect. 2.4 orders a substep as gas step,
// radiation transport, radiation sources).  A Godunov step of the Euler
// equations on Cartesian grids: PLM with the van Leer limiter on the
// primitive variables (rho, v, p), the HLL flux with the Davis signal speeds
// S_L = min(v_L - c_L, v_R - c_R), S_R = max(v_L + c_L, v_R + c_R), and the
// flux divergence of (rho, m, E_gas).
//
// One thread per cell computes the fluxes of its two faces in every active
// direction (each face twice, once by each of its cells) from the padded
// input buffer, whose ghost cells the previous step left up to date.  The
// result (rho*, m*, e*) goes to separate arrays: the radiation kernel that
// follows reads rho* and e* of neighbouring cells for its optical depths
// while it writes the final gas, so it must not read them from the arrays it
// writes.  The thread also writes the ghost copies of rho* and e* that its
// cell feeds.
#pragma once
#include "m1_internal.h"

namespace m1 {

template <class P>
struct HydroArgs {
  using S = typename P::S;
  using T = typename P::T;
  StepDims dim;
  GeomDev<T> geo;
  const S* rho;      // input gas (padded, ghosts valid)
  const S* e;
  const S* m[3];
  S* rho_out;        // gas after the step (padded); ghosts of rho and e written
  S* e_out;
  S* m_out[3];
  T dt, gamma, cvfac;
  T bcT[3][2];       // gas temperature of the fixed and LTE sides
};

// Primitive state (rho, v0, v1, v2, p) of the padded cell ip.
template <class P, int NC>
__device__ __forceinline__ void gas_w(const HydroArgs<P>& h, long long ip,
                                      typename P::T (&w)[5]) {
  using T = typename P::T;
  const T r = T(__ldg(h.rho + ip));
  const T ir = Ops<T>::rcp(r);
  w[0] = r;
#pragma unroll
  for (int v = 0; v < 3; ++v) w[1 + v] = v < NC ? T(__ldg(h.m[v] + ip)) * ir : T(0);
  w[4] = (h.gamma - T(1)) * T(__ldg(h.e + ip));
}

// Conserved state and physical flux along D of a primitive state.
template <class T, int NC, int D>
__device__ __forceinline__ void gas_flux(const T (&w)[5], T gamma, T (&U)[5], T (&f)[5]) {
  const T r = w[0], p = w[4], vd = w[1 + D];
  T v2 = T(0);
#pragma unroll
  for (int v = 0; v < NC; ++v) v2 += w[1 + v] * w[1 + v];
  const T Eg = Ops<T>::div(p, gamma - T(1)) + T(0.5) * r * v2;
  U[0] = r;
  f[0] = r * vd;
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    U[1 + v] = r * w[1 + v];
    f[1 + v] = r * vd * w[1 + v] + (v == D ? p : T(0));
  }
  U[4] = Eg;
  f[4] = (Eg + p) * vd;
}

// HLL flux of the face between the padded cells ip - s and ip along D (s the
// padded stride of D, pi the padded coordinate of ip along D).
template <class P, int NC, int D>
__device__ __forceinline__ void gas_face(const HydroArgs<P>& h, long long ip, long long s, int pi,
                                         typename P::T (&out)[5]) {
  using T = typename P::T;
  T w0[5], w1[5], w2[5], w3[5];
  gas_w<P, NC>(h, ip - 2 * s, w0);
  gas_w<P, NC>(h, ip - s, w1);
  gas_w<P, NC>(h, ip, w2);
  gas_w<P, NC>(h, ip + s, w3);
  const T* tab = h.geo.tab[D];
  const int len = h.geo.len[D];
  const T ix0 = __ldg(tab + TAB_IDXC * len + pi - 2), ix1 = __ldg(tab + TAB_IDXC * len + pi - 1),
          ix2 = __ldg(tab + TAB_IDXC * len + pi);
  const T hh = __ldg(tab + TAB_HHI * len + pi - 1), hl = __ldg(tab + TAB_HLO * len + pi);
  T wl[5], wr[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const T d0 = (w1[q] - w0[q]) * ix0, d1 = (w2[q] - w1[q]) * ix1, d2 = (w3[q] - w2[q]) * ix2;
    wl[q] = w1[q] + vanleer(d0, d1) * hh;
    wr[q] = w2[q] + vanleer(d1, d2) * hl;
  }
  T UL[5], UR[5], fL[5], fR[5];
  gas_flux<T, NC, D>(wl, h.gamma, UL, fL);
  gas_flux<T, NC, D>(wr, h.gamma, UR, fR);
  const T cl = Ops<T>::sqrt_(Ops<T>::div(h.gamma * wl[4], wl[0]));
  const T cr = Ops<T>::sqrt_(Ops<T>::div(h.gamma * wr[4], wr[0]));
  T sl = wl[1 + D] - cl, sr = wr[1 + D] + cr;
  if (wr[1 + D] - cr < sl) sl = wr[1 + D] - cr;
  if (wl[1 + D] + cl > sr) sr = wl[1 + D] + cl;
  if (sl >= T(0)) {
#pragma unroll
    for (int q = 0; q < 5; ++q) out[q] = fL[q];
  } else if (sr <= T(0)) {
#pragma unroll
    for (int q = 0; q < 5; ++q) out[q] = fR[q];
  } else {
    const T inv = Ops<T>::rcp(sr - sl);
#pragma unroll
    for (int q = 0; q < 5; ++q) out[q] = (sr * fL[q] - sl * fR[q] + sl * sr * (UR[q] - UL[q])) * inv;
  }
}

template <class P, int NC, int D>
__device__ __forceinline__ void gas_direction(const HydroArgs<P>& h, long long ic, int pi,
                                              typename P::T (&U)[5]) {
  using T = typename P::T;
  const long long s = D == 0 ? 1ll : (D == 1 ? h.dim.sy : h.dim.sz);
  T flo[5], fhi[5];
  gas_face<P, NC, D>(h, ic, s, pi, flo);
  gas_face<P, NC, D>(h, ic + s, s, pi + 1, fhi);
  const T ih = __ldg(h.geo.tab[D] + TAB_ALO * h.geo.len[D] + pi);  // 1 / width (Cartesian)
#pragma unroll
  for (int q = 0; q < 5; ++q) U[q] -= h.dt * ih * (fhi[q] - flo[q]);
}

template <class P, int NDIM, int NC>
__global__ void __launch_bounds__(128) hydro_kernel(const __grid_constant__ HydroArgs<P> h) {
  using S = typename P::S;
  using T = typename P::T;
  const StepDims& Dm = h.dim;
  const long long N = (long long)Dm.n[0] * Dm.n[1] * Dm.n[2];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
       q += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    long long r = q;
    ci[0] = int(r % Dm.n[0]);
    r /= Dm.n[0];
    ci[1] = int(r % Dm.n[1]);
    ci[2] = int(r / Dm.n[1]);
    const int p0 = ci[0] + Dm.g[0], p1 = ci[1] + Dm.g[1], p2 = ci[2] + Dm.g[2];
    const long long ic = p0 + Dm.sy * p1 + Dm.sz * p2;
    const T rho = T(h.rho[ic]);
    T U[5];
    U[0] = rho;
    T ke = T(0);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      U[1 + v] = v < NC ? T(h.m[v][ic]) : T(0);
      ke += U[1 + v] * U[1 + v];
    }
    U[4] = T(h.e[ic]) + T(0.5) * ke * Ops<T>::rcp(rho);
    gas_direction<P, NC, 0>(h, ic, p0, U);
    if constexpr (NDIM >= 2) gas_direction<P, NC, 1>(h, ic, p1, U);
    if constexpr (NDIM >= 3) gas_direction<P, NC, 2>(h, ic, p2, U);
    T k2 = T(0);
#pragma unroll
    for (int v = 0; v < NC; ++v) k2 += U[1 + v] * U[1 + v];
    const T en = U[4] - T(0.5) * k2 * Ops<T>::rcp(U[0]);
    h.rho_out[ic] = S(U[0]);
    h.e_out[ic] = S(en);
#pragma unroll
    for (int v = 0; v < NC; ++v) h.m_out[v][ic] = S(U[1 + v]);
    // ghost copies of rho* and e* (the optical depths of the radiation step
    // read them): wrapped, edge or mirrored; the fixed and LTE sides take the
    // edge density and e = C_v T_b
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const int n = Dm.n[d];
      const int i = ci[d];
      if (i >= 2 && i < n - 2) continue;
      const long long stride = d == 0 ? 1ll : (d == 1 ? Dm.sy : Dm.sz);
#pragma unroll
      for (int gslot = 0; gslot < 4; ++gslot) {
        const bool lo = gslot < 2;
        const int gpos = lo ? gslot - 2 : n + gslot - 2;
        const int bc = lo ? Dm.bc_lo[d] : Dm.bc_hi[d];
        int src;
        if (bc == BC_PERIODIC)
          src = lo ? ((gpos % n) + n) % n : gpos % n;
        else if (bc == BC_REFLECT)
          src = min(max(lo ? -1 - gpos : 2 * n - 1 - gpos, 0), n - 1);
        else
          src = lo ? 0 : n - 1;
        if (src != i) continue;
        const long long ig = ic + (long long)(gpos - i) * stride;
        h.rho_out[ig] = S(U[0]);
        const bool held = bc == BC_FIXED || bc == BC_LTE;
        h.e_out[ig] = S(held ? h.cvfac * U[0] * h.bcT[d][lo ? 0 : 1] : en);
      }
    }
  }
}

}  // namespace m1
