// m1_step.cuh -- the fused M1 radiation step kernel (sm_103a).
//
// One launch performs, for every cell, the whole Euler step of Sect. 2.4:
// boundary values (ghost layers kept up to date by the previous launch),
// PLM reconstruction, the f-preserving fix of Eq. (f_reconstruct), closure,
// signal speeds with the optically thick limit (Sect. 2.6), HLL fluxes,
// the unsplit flux divergence with the metric terms of the geometry, and
// the implicit coupling of Sect. 2.8 with the gas bookkeeping of Sect. 2.7.
//
// Options of Sect. 2.5 (LimO3, the flat and clipping face treatments, the
// Lax-Friedrichs-Rusanov flux), the absorption-only coupling and the
// irradiation deposit exist in the general instantiation (GEN) only, as
// uniform branches; the default instantiations compile them out.
//
// Work decomposition.  A CTA of TX x TY threads owns an x (and, in 3D, y)
// tile and marches along the slowest active axis (y in 2D, z in 3D).  Thread
// (tx, ty) computes the lower face of its own column in every tile direction;
// tiles overlap by one cell, so each CTA updates (TX-1) x (TY-1) columns.  The
// march direction keeps the column's states, its reconstructed upper face
// state and the lower face flux in registers, so each march face is computed
// once.  The tile directions read a shared-memory plane holding the current
// march plane with a 2-cell halo; the face fluxes are exchanged through
// shared memory.  Optical depths of the halo cells needed by the tile faces
// are computed by the threads that load the halo.
#pragma once
#include "m1_cell.cuh"
#include "m1_internal.h"

namespace m1 {

template <class T>
__device__ __forceinline__ T tabv(const GeomDev<T>& G, int d, int slot, int ip) {
  return __ldg(G.tab[d] + slot * G.len[d] + ip);
}

// Largest physical width of a cell over the active directions (tau and CFL).
template <class T, int NDIM, int GEOM>
__device__ __forceinline__ T cell_hmax(const GeomDev<T>& G, int p0, int p1, int p2) {
  T h = tabv(G, 0, TAB_WID, p0);
  if (NDIM >= 2) {
    T w = tabv(G, 1, TAB_WID, p1);
    if (GEOM != kCart) w *= tabv(G, 0, TAB_RC, p0);
    h = w > h ? w : h;
  }
  if (NDIM >= 3) {
    T w = tabv(G, 2, TAB_WID, p2);
    if (GEOM == kSph) w *= tabv(G, 0, TAB_RC, p0) * tabv(G, 1, TAB_RC, p1);
    h = w > h ? w : h;
  }
  return h;
}

// Opacities and optical depth rho chi h of a cell from its (rho, e).
template <class P, int NDIM, int GEOM, bool UNI = false>
__device__ __forceinline__ typename P::T cell_tau(const StepArgs<P>& a, typename P::S rho,
                                                  typename P::S e, int p0, int p1, int p2,
                                                  typename P::T& kp, typename P::T& chi) {
  using T = typename P::T;
  T r = T(rho);
  if constexpr (sizeof(T) == 8)
    opacity(a.opac, r, T(e) / (r * T(a.cp.cvfac)), kp, chi);
  else
    opacity_re(a.opac, r, T(e), kp, chi);
  if constexpr (UNI) return r * chi * a.uni_h;
  return r * chi * cell_hmax<T, NDIM, GEOM>(a.geo, p0, p1, p2);
}

// Reconstructed state at the face of cell uc at offset h from its centre,
// from the one-sided differences dl = (uc - um) ixl and dr = (up - uc) ixr.
template <class T, int NV>
__device__ __forceinline__ void plm_state(const T (&dl)[4], const T (&dr)[4], const T (&uc)[4],
                                          T h, T (&out)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = (q < NV) ? uc[q] + vanleer(dl[q], dr[q]) * h : T(0);
}

template <class T, int NC>
__device__ __forceinline__ T flux2(const T (&u)[4]) {
  T s = u[1] * u[1];
  if (NC > 1) s += u[2] * u[2];
  if (NC > 2) s += u[3] * u[3];
  return s;
}

// HLL flux from two fixed face states along D.
template <class T, int NC, int D>
__device__ __forceinline__ void riemann(const T (&uL)[4], const T (&uR)[4], T chat, T tau,
                                        T (&out)[4]) {
  T fL[4] = {0, 0, 0, 0}, fR[4] = {0, 0, 0, 0};
  T lmL, lpL, lmR, lpR;
  state_flux<T, NC, D>(uL, chat, fL, lmL, lpL);
  state_flux<T, NC, D>(uR, chat, fR, lmR, lpR);
  hll<T, 1 + NC>(uL, uR, fL, fR, lmL, lpL, lmR, lpR, chat, tau, out);
}

// The Riemann solver the scheme selects (HLL or Lax-Friedrichs-Rusanov).
template <class T, int NC, int D>
__device__ __forceinline__ void riemann_s(const Scheme& sc, const T (&uL)[4], const T (&uR)[4],
                                          T chat, T tau, T (&out)[4]) {
  if (sc.riemann == 0) {
    riemann<T, NC, D>(uL, uR, chat, tau, out);
    return;
  }
  T fL[4] = {0, 0, 0, 0}, fR[4] = {0, 0, 0, 0};
  T lmL, lpL, lmR, lpR;
  state_flux<T, NC, D>(uL, chat, fL, lmL, lpL);
  state_flux<T, NC, D>(uR, chat, fR, lmR, lpR);
  lf<T, 1 + NC>(uL, uR, fL, fR, lmL, lpL, lmR, lpR, chat, tau, out);
}

// The treatment of a face state with |F_f| > E_f that the scheme selects
// (Sect. 2.5): Eq. (f_reconstruct), the cell's flat state, or F_f rescaled
// to |F_f| = E_f.  Returns true when the state was changed.
template <class T, int NC>
__device__ __forceinline__ bool fix_face_s(const Scheme& sc, T (&uf)[4], const T (&uc)[4], T nc2,
                                           T inv_Ec) {
  if (sc.ffix == 0) return fix_face<T, NC>(uf, uc, nc2, inv_Ec);
  const T nf2 = flux2<T, NC>(uf);
  if (nf2 <= uf[0] * uf[0]) return false;
  if (sc.ffix == 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) uf[q] = uc[q];
  } else {
    const T r = Ops<T>::div(uf[0], Ops<T>::sqrt_(nf2));
#pragma unroll
    for (int v = 0; v < NC; ++v) uf[1 + v] *= r;
  }
  return true;
}

// LimO3 lower (lo) and upper (hi) face states of cell u between um and up.
template <class T, int NV>
__device__ __forceinline__ void limo3_states(const T (&um)[4], const T (&u)[4], const T (&up)[4],
                                             T (&lo)[4], T (&hi)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < NV) {
      const T dm = u[q] - um[q], dp = up[q] - u[q];
      lo[q] = u[q] - limo3(dp, dm);
      hi[q] = u[q] + limo3(dm, dp);
    } else {
      lo[q] = hi[q] = T(0);
    }
  }
}

// Face flux from four consecutive cells um2, um1 | u0, up1 along D (the
// face between um1 and u0).  ix_k = 1 / (centre distance) of the pairs
// (um2, um1), (um1, u0), (u0, up1); hh = offset of the upper face of um1,
// hl = offset of the lower face of u0.  Returns which face states the fix
// replaced: bit 0 the upper state of um1, bit 1 the lower state of u0.
// Half of the van Leer limited slope on a uniform grid, in units of the
// cell difference: vl(dl, dr) / 2 = dl dr / (dl + dr) when dl dr > 0.
template <class T>
__device__ __forceinline__ T half_vanleer(T dl, T dr) {
  T p = dl * dr;
  return p > T(0) ? p * rcp_approx(dl + dr) : T(0);
}

// sc: the face options (all zero, the defaults, unless given).
// Lower (lo) and upper (hi) PLM face states of cell uc between um and up on
// a uniform grid, from the van Leer half slope; the float form with four
// components runs on packed pairs.
template <class T, int NV>
__device__ __forceinline__ void uni_states(const T (&um)[4], const T (&uc)[4], const T (&up)[4],
                                           T (&lo)[4], T (&hi)[4]) {
  if constexpr (sizeof(T) == 4 && NV == 4) {
#pragma unroll
    for (int h = 0; h < 4; h += 2) {
      const float2 c = make_float2(uc[h], uc[h + 1]);
      const float2 dl = f2_sub(c, make_float2(um[h], um[h + 1]));
      const float2 dr = f2_sub(make_float2(up[h], up[h + 1]), c);
      const float2 pr = f2_mul(dl, dr), sm = f2_add(dl, dr);
      float2 hs = f2_mul(pr, make_float2(rcp_approx(sm.x), rcp_approx(sm.y)));
      hs.x = pr.x > 0.f ? hs.x : 0.f;
      hs.y = pr.y > 0.f ? hs.y : 0.f;
      const float2 l = f2_sub(c, hs), u = f2_add(c, hs);
      lo[h] = l.x;
      lo[h + 1] = l.y;
      hi[h] = u.x;
      hi[h + 1] = u.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T hs = q < NV ? half_vanleer(uc[q] - um[q], up[q] - uc[q]) : T(0);
      lo[q] = q < NV ? uc[q] - hs : T(0);
      hi[q] = q < NV ? uc[q] + hs : T(0);
    }
  }
}

template <class T, int NC, int D, bool UNI>
__device__ __forceinline__ int face4(const T (&um2)[4], const T (&um1)[4], const T (&u0)[4],
                                     const T (&up1)[4], T ix0, T ix1, T ix2, T hh, T hl, T tau,
                                     T chat, T inv_u0, T n2_u0, T (&out)[4],
                                     Scheme sc = Scheme{0, 0, 0}) {
  constexpr int NV = 1 + NC;
  T uL[4], uR[4];
  if (sc.recon == 1) {
    T lo[4], hi[4];
    limo3_states<T, NV>(um2, um1, u0, lo, uL);
    limo3_states<T, NV>(um1, u0, up1, uR, hi);
  } else if constexpr (UNI && sizeof(T) == 4) {
    T lo[4], hi[4];
    uni_states<T, NV>(um2, um1, u0, lo, uL);
    uni_states<T, NV>(um1, u0, up1, uR, hi);
  } else {
    T d0[4], d1[4], d2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      d0[q] = (um1[q] - um2[q]) * ix0;
      d1[q] = (u0[q] - um1[q]) * ix1;
      d2[q] = (up1[q] - u0[q]) * ix2;
    }
    plm_state<T, NV>(d0, d1, um1, hh, uL);
    plm_state<T, NV>(d1, d2, u0, hl, uR);
  }
  const int fixL = fix_face_s<T, NC>(sc, uL, um1, flux2<T, NC>(um1), Ops<T>::rcp(um1[0]));
  const int fixR = fix_face_s<T, NC>(sc, uR, u0, n2_u0, inv_u0);
  riemann_s<T, NC, D>(sc, uL, uR, chat, tau, out);
  return fixL | (fixR << 1);
}

template <class S, int NC, class T>
__device__ __forceinline__ void load_state(const Fields<S>& f, long long i, T (&u)[4]) {
  u[0] = T(__ldg(f.E + i));
#pragma unroll
  for (int q = 0; q < 3; ++q) u[1 + q] = (q < NC) ? T(__ldg(f.F[q] + i)) : T(0);
}

// MINB: resident CTAs per SM requested from the register allocator.
// One tile of the step: the CTA's (bx, by, bz) block coordinates select the
// x tile, the y tile (3D) and the march chunk.  Called by the single-grid
// kernel below and by the batched kernel of many grids.
// UNI: uniform Cartesian grid (spacing from constants instead of tables; the
// slopes use raw differences, the 1/dx factor cancelling in the van Leer
// mean, and faces sit at -/+ 1/2 in units of the difference).
// GEN: the general form, with the face options of StepArgs::scheme, the
// absorption-only coupling and the irradiation deposit as uniform runtime
// branches; without it those are compiled out (the defaults, no deposit).
template <class P, int NDIM, int GEOM, int NC, bool UNI, int TX, int TY, bool GEN = false>
__device__ __forceinline__ void step_tile(const StepArgs<P>& a, int bx, int by, int bz) {
  using S = typename P::S;
  using T = typename P::T;
  constexpr int NV = 1 + NC;
  constexpr bool TILE_Y = (NDIM == 3);
  constexpr bool MARCH = (NDIM >= 2);
  constexpr int MA = (NDIM == 3) ? 2 : 1;  // march axis
  constexpr int SX = TX + 3;
  constexpr int SY = TILE_Y ? TY + 3 : 1;
  constexpr int OY = TILE_Y ? 2 : 0;
  constexpr int NT = TX * TY;
  constexpr int NHALO = TILE_Y ? 3 * (TX + TY) : 3;

  __shared__ T s_u[NV][SY][SX];
  __shared__ T s_tau[TILE_Y ? TY + 1 : 1][TX + 1];
  __shared__ T s_fx[NV][TY][TX];
  __shared__ T s_fy[TILE_Y ? NV : 1][TILE_Y ? TY : 1][TX];
  __shared__ unsigned long long s_red[ST_N];

  const StepDims& Dm = a.dim;
  const GeomDev<T>& G = a.geo;
  const int tx = threadIdx.x;
  const int ty = TILE_Y ? threadIdx.y : 0;
  const int tid = tx + TX * ty;
  const int x0 = bx * (TX - 1);
  const int y0 = TILE_Y ? by * (TY - 1) : 0;
  const int mblk = MARCH ? (TILE_Y ? bz : by) : 0;
  const int m0 = MARCH ? mblk * a.chunk : 0;
  const int m1 = MARCH ? min(m0 + a.chunk, Dm.n[MA]) : 1;

  counters_reset(s_red, tid);

  const int cx = x0 + tx;
  const int cy = TILE_Y ? y0 + ty : 0;
  const int px = min(cx + Dm.g[0], G.len[0] - 1);                 // table / array x
  const int pxa = min(cx + Dm.g[0], Dm.pn[0] - 1);
  const int py = TILE_Y ? min(cy + Dm.g[1], G.len[1] - 1) : 0;
  const long long base = (long long)pxa + (TILE_Y ? (long long)py * Dm.sy : 0ll);
  const long long ms = MARCH ? (MA == 2 ? Dm.sz : Dm.sy) : 0ll;
  const int gm = MARCH ? Dm.g[MA] : 0;
  const bool in_col = cx < Dm.n[0] && (!TILE_Y || cy < Dm.n[1]);
  const bool upd_col = in_col && tx <= TX - 2 && (!TILE_Y || ty <= TY - 2);
  // a column at least two cells from the boundaries of its tile directions
  // feeds ghost copies only near the ends of the march
  const bool col_inner =
      cx >= 2 && cx < Dm.n[0] - 2 && (!TILE_Y || (cy >= 2 && cy < Dm.n[1] - 2));
  // In the split precision the face fluxes and signal speeds are formed in
  // units of chat (the flux functions take fchat = 1) and the divergence
  // is scaled by dt chat; in FP64 they carry chat as the oracle does.
  const T fchat = P::kSplit ? T(1) : T(a.chat);
  const T dtf = P::kSplit ? T(a.dt) * T(a.chat) : T(a.dt);
  Scheme sc{0, 0, 0};
  if constexpr (GEN) sc = a.scheme;

  // march-plane coordinates for tables: p1 (2D: march; 3D: tile y), p2
  auto p1_of = [&](int m) { return TILE_Y ? py : (MARCH ? m + gm : 0); };
  auto p2_of = [&](int m) { return TILE_Y ? m + gm : 0; };
  // spacing tables, or their constant values on a uniform grid
  auto IXC = [&](int d, int ip) -> T { return UNI ? T(1) : tabv(G, d, TAB_IDXC, ip); };
  auto HHI = [&](int d, int ip) -> T { return UNI ? T(0.5) : tabv(G, d, TAB_HHI, ip); };
  auto HLO = [&](int d, int ip) -> T { return UNI ? T(-0.5) : tabv(G, d, TAB_HLO, ip); };
  auto ALO = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_ALO, ip); };
  auto AHI = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_AHI, ip); };

  Counters cnt;

  // column queue: q[0..2] = states at m, m+1, m+2
  T q[3][4];
  T hiS[4];         // fixed upper face state of cell m along the march axis
  T zlo[4], zhi[4]; // march-face fluxes m-1/2 and m+1/2
  T inv_own = 0, n2_own = 0;  // 1/E and |F|^2 of the own cell (fix of its face states)
  T tau_m = 0, tau_n = 0, kp_m = 0, chi_m = 0, kp_n = 0, chi_n = 0;
  S rho_m = 0, e_m = 0, rho_n = 0, e_n = 0;
#pragma unroll
  for (int v = 0; v < 4; ++v) zlo[v] = zhi[v] = hiS[v] = T(0);

  if constexpr (MARCH) {
    T qm2[4], qm1[4];
    load_state<S, NC>(a.in, base + (long long)(m0 - 2 + gm) * ms, qm2);
    load_state<S, NC>(a.in, base + (long long)(m0 - 1 + gm) * ms, qm1);
    load_state<S, NC>(a.in, base + (long long)(m0 + gm) * ms, q[0]);
    load_state<S, NC>(a.in, base + (long long)(m0 + 1 + gm) * ms, q[1]);
    {
      long long i = base + (long long)(m0 - 1 + gm) * ms;
      S r = __ldg(a.rho + i), e = __ldg(a.in.e + i);
      T kp, chi;
      tau_m = cell_tau<P, NDIM, GEOM, UNI>(a, r, e, px, p1_of(m0 - 1), p2_of(m0 - 1), kp, chi);
    }
    T tau_prev = tau_m;
    {
      long long i = base + (long long)(m0 + gm) * ms;
      rho_m = __ldg(a.rho + i);
      e_m = __ldg(a.in.e + i);
      tau_m = cell_tau<P, NDIM, GEOM, UNI>(a, rho_m, e_m, px, p1_of(m0), p2_of(m0), kp_m, chi_m);
    }
    const int pm = m0 + gm;
    T ix0 = IXC(MA, pm - 2), ix1 = IXC(MA, pm - 1);
    T ix2 = IXC(MA, pm);
    int nf = face4<T, NC, MA, UNI>(qm2, qm1, q[0], q[1], ix0, ix1, ix2, HHI(MA, pm - 1),
                                   HLO(MA, pm), T(0.5) * (tau_prev + tau_m), fchat,
                                   Ops<T>::rcp(q[0][0]), flux2<T, NC>(q[0]), zlo, sc);
    if (upd_col) cnt.fix += nf >> 1;  // the lower march state of cell m0
    // upper face state of cell m0 (fixed), kept for the face m0 + 1/2
    if (sc.recon == 1) {
      T lo[4];
      limo3_states<T, NV>(qm1, q[0], q[1], lo, hiS);
    } else {
      T d1[4], d2[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        d1[v] = (q[0][v] - qm1[v]) * ix1;
        d2[v] = (q[1][v] - q[0][v]) * ix2;
      }
      plm_state<T, NV>(d1, d2, q[0], HHI(MA, pm), hiS);
    }
    inv_own = Ops<T>::rcp(q[0][0]);
    n2_own = flux2<T, NC>(q[0]);
    int nfh = fix_face_s<T, NC>(sc, hiS, q[0], n2_own, inv_own);
    if (upd_col) cnt.fix += nfh;
  } else {
    load_state<S, NC>(a.in, base, q[0]);
    inv_own = Ops<T>::rcp(q[0][0]);
    n2_own = flux2<T, NC>(q[0]);
    rho_m = __ldg(a.rho + base);
    e_m = __ldg(a.in.e + base);
    tau_m = cell_tau<P, NDIM, GEOM, UNI>(a, rho_m, e_m, px, 0, 0, kp_m, chi_m);
  }

  // Halo cell of this thread (each thread owns at most one), decoded once;
  // its values for plane m are loaded one iteration ahead.
  static_assert(NHALO <= NT, "one halo cell per thread");
  const bool has_halo = tid < NHALO;
  int hxs = 0, hys = 0;
  if (has_halo) {
    const int h = tid;
    if (TILE_Y) {
      if (h < 3 * TY) {
        int c = h / TY;
        hxs = c == 0 ? -2 : (c == 1 ? -1 : TX);
        hys = h - c * TY;
      } else {
        int hh = h - 3 * TY;
        int c = hh / TX;
        hys = c == 0 ? -2 : (c == 1 ? -1 : TY);
        hxs = hh - c * TX;
      }
    } else {
      hxs = h == 0 ? -2 : (h == 1 ? -1 : TX);
    }
  }
  const bool halo_tau = has_halo && (TILE_Y ? ((hxs == -1 && hys >= 0 && hys < TY) ||
                                               (hys == -1 && hxs >= 0 && hxs < TX))
                                            : (hxs == -1));
  const int hx = min(max(x0 + hxs + Dm.g[0], 0), Dm.pn[0] - 1);
  const int hy = TILE_Y ? min(max(y0 + hys + Dm.g[1], 0), Dm.pn[1] - 1) : 0;
  const long long hbase = (long long)hx + (TILE_Y ? (long long)hy * Dm.sy : 0ll);
  T hu[4] = {0, 0, 0, 0};
  S hrho = S(1), he = S(1);
  auto load_halo = [&](int m) {
    if (has_halo) {
      long long ih = hbase + (long long)(m + gm) * ms;
      load_state<S, NC>(a.in, ih, hu);
      if (halo_tau) {
        hrho = __ldg(a.rho + ih);
        he = __ldg(a.in.e + ih);
      }
    }
  };
  load_halo(m0);
  // (rho, e) of the cell m + 1 of the own column, loaded one iteration ahead
  S rho_p = S(1), e_p = S(1);
  if constexpr (MARCH) {
    rho_p = __ldg(a.rho + base + (long long)(m0 + 1 + gm) * ms);
    e_p = __ldg(a.in.e + base + (long long)(m0 + 1 + gm) * ms);
  }

  for (int m = m0; m < m1; ++m) {
    const long long ic = base + (long long)(m + gm) * ms;  // own cell
    T mom[3] = {0, 0, 0};
    if constexpr (MARCH) {
      load_state<S, NC>(a.in, ic + 2 * ms, q[2]);
      rho_n = rho_p;
      e_n = e_p;
      rho_p = __ldg(a.rho + ic + 2 * ms);
      e_p = __ldg(a.in.e + ic + 2 * ms);
    }
    if (upd_col) {
#pragma unroll
      for (int v = 0; v < NC; ++v) mom[v] = T(__ldg(a.in.m[v] + ic));
    }
    // own state and tau into the shared plane
#pragma unroll
    for (int v = 0; v < NV; ++v) s_u[v][ty + OY][tx + 2] = q[0][v];
    s_tau[TILE_Y ? ty + 1 : 0][tx + 1] = tau_m;
    // halo of the plane (values loaded in the previous iteration)
    if (has_halo) {
#pragma unroll
      for (int v = 0; v < NV; ++v) s_u[v][hys + OY][hxs + 2] = hu[v];
      if (halo_tau) {
        T kp, chi;
        int tx_ = min(hx, G.len[0] - 1);
        int ty_ = TILE_Y ? min(hy, G.len[1] - 1) : p1_of(m);
        s_tau[TILE_Y ? hys + 1 : 0][hxs + 1] =
            cell_tau<P, NDIM, GEOM, UNI>(a, hrho, he, tx_, ty_, p2_of(m), kp, chi);
      }
    }
    if (MARCH && m + 1 < m1) load_halo(m + 1);
    if constexpr (MARCH)
      tau_n = cell_tau<P, NDIM, GEOM, UNI>(a, rho_n, e_n, px, p1_of(m + 1), p2_of(m + 1), kp_n, chi_n);
    __syncthreads();

    // x face (tx - 1/2)
    {
      T um2[4], um1[4], u0[4], up1[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        um2[v] = v < NV ? s_u[v][ty + OY][tx] : T(0);
        um1[v] = v < NV ? s_u[v][ty + OY][tx + 1] : T(0);
        u0[v] = v < NV ? s_u[v][ty + OY][tx + 2] : T(0);
        up1[v] = v < NV ? s_u[v][ty + OY][tx + 3] : T(0);
      }
      T tau = T(0.5) * (s_tau[TILE_Y ? ty + 1 : 0][tx] + s_tau[TILE_Y ? ty + 1 : 0][tx + 1]);
      T fx[4];
      int nf = face4<T, NC, 0, UNI>(um2, um1, u0, up1, IXC(0, px - 2),
                               IXC(0, px - 1), IXC(0, px),
                               HHI(0, px - 1), HLO(0, px), tau, fchat, inv_own, n2_own, fx,
                               sc);
      // fixed states of updated cells: the lower one of this cell, the upper
      // one of the cell to the left
      const bool row_upd = !TILE_Y || (ty <= TY - 2 && cy < Dm.n[1]);
      if (upd_col) cnt.fix += nf >> 1;
      if (row_upd && tx >= 1 && cx - 1 < Dm.n[0]) cnt.fix += nf & 1;
#pragma unroll
      for (int v = 0; v < NV; ++v) s_fx[v][ty][tx] = fx[v];
    }
    // y face (ty - 1/2), 3D only
    if constexpr (TILE_Y) {
      T um2[4], um1[4], u0[4], up1[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        um2[v] = v < NV ? s_u[v][ty][tx + 2] : T(0);
        um1[v] = v < NV ? s_u[v][ty + 1][tx + 2] : T(0);
        u0[v] = v < NV ? s_u[v][ty + 2][tx + 2] : T(0);
        up1[v] = v < NV ? s_u[v][ty + 3][tx + 2] : T(0);
      }
      T tau = T(0.5) * (s_tau[ty][tx + 1] + s_tau[ty + 1][tx + 1]);
      T fy[4];
      int nf = face4<T, NC, 1, UNI>(um2, um1, u0, up1, IXC(1, py - 2),
                               IXC(1, py - 1), IXC(1, py),
                               HHI(1, py - 1), HLO(1, py), tau, fchat, inv_own, n2_own, fy,
                               sc);
      if (upd_col) cnt.fix += nf >> 1;
      if (ty >= 1 && cy - 1 < Dm.n[1] && tx <= TX - 2 && cx < Dm.n[0]) cnt.fix += nf & 1;
#pragma unroll
      for (int v = 0; v < NV; ++v) s_fy[v][ty][tx] = fy[v];
    }
    // march face m + 1/2 from the column registers
    T hiN[4];
    T inv_n = 0, n2_n = 0;
    if constexpr (MARCH) {
      const int pm = m + 1 + gm;  // padded index of cell m+1
      T loN[4];
      if (sc.recon == 1) {
        limo3_states<T, NV>(q[0], q[1], q[2], loN, hiN);
      } else if constexpr (UNI && sizeof(T) == 4) {
        uni_states<T, NV>(q[0], q[1], q[2], loN, hiN);
      } else {
        T ix1 = IXC(MA, pm - 1), ix2 = IXC(MA, pm);
        T d1[4], d2[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          d1[v] = (q[1][v] - q[0][v]) * ix1;
          d2[v] = (q[2][v] - q[1][v]) * ix2;
        }
        plm_state<T, NV>(d1, d2, q[1], HLO(MA, pm), loN);
        plm_state<T, NV>(d1, d2, q[1], HHI(MA, pm), hiN);
      }
      inv_n = Ops<T>::rcp(q[1][0]);
      n2_n = flux2<T, NC>(q[1]);
      int nf = fix_face_s<T, NC>(sc, loN, q[1], n2_n, inv_n);
      int nf2 = fix_face_s<T, NC>(sc, hiN, q[1], n2_n, inv_n);
      riemann_s<T, NC, MA>(sc, hiS, loN, fchat, T(0.5) * (tau_m + tau_n), zhi);
      // hiN belongs to the face m + 3/2, computed here only if m + 1 < m1
      if (upd_col && m + 1 < m1) cnt.fix += nf + nf2;  // the march states of cell m + 1
    }
    __syncthreads();

    // update of the own cell
    if (upd_col && m < (MARCH ? Dm.n[MA] : 1)) {
      T dU[4] = {0, 0, 0, 0};
      // direction 0
      {
        T flo[4], fhi[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          flo[v] = v < NV ? s_fx[v][ty][tx] : T(0);
          fhi[v] = v < NV ? s_fx[v][ty][tx + 1] : T(0);
        }
        T alo = ALO(0, px), ahi = AHI(0, px);
#pragma unroll
        for (int v = 0; v < NV; ++v) dU[v] -= ahi * fhi[v] - alo * flo[v];
        if (GEOM == kCyl && NC >= 2) {
          dU[2] += ahi * fhi[2] - alo * flo[2];
          dU[2] -= tabv(G, 0, TAB_AMHI, px) * fhi[2] - tabv(G, 0, TAB_AMLO, px) * flo[2];
        }
        if (GEOM == kSph && NC >= 3) {
          dU[3] += ahi * fhi[3] - alo * flo[3];
          dU[3] -= tabv(G, 0, TAB_AMHI, px) * fhi[3] - tabv(G, 0, TAB_AMLO, px) * flo[3];
        }
      }
      const int p1 = p1_of(m), p2 = p2_of(m);
      T met0 = (GEOM != kCart) ? tabv(G, 0, TAB_MET, px) : T(1);
      // direction 1
      if constexpr (NDIM >= 2) {
        T flo[4], fhi[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if constexpr (TILE_Y) {
            flo[v] = v < NV ? s_fy[v][ty][tx] : T(0);
            fhi[v] = v < NV ? s_fy[v][ty + 1][tx] : T(0);
          } else {
            flo[v] = zlo[v];
            fhi[v] = zhi[v];
          }
        }
        T alo = ALO(1, p1), ahi = AHI(1, p1);
        if (GEOM != kCart) {
          alo *= met0;
          ahi *= met0;
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) dU[v] -= ahi * fhi[v] - alo * flo[v];
        if (GEOM == kSph && NC >= 3) {
          dU[3] += ahi * fhi[3] - alo * flo[3];
          dU[3] -= met0 * (tabv(G, 1, TAB_AMHI, p1) * fhi[3] - tabv(G, 1, TAB_AMLO, p1) * flo[3]);
        }
      }
      // direction 2
      if constexpr (NDIM >= 3) {
        T alo = ALO(2, p2), ahi = AHI(2, p2);
        if (GEOM == kSph) {
          T f = met0 * tabv(G, 1, TAB_PHF, p1);
          alo *= f;
          ahi *= f;
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) dU[v] -= ahi * zhi[v] - alo * zlo[v];
      }
      const T (&u)[4] = q[0];
      // inactive theta of a 1D spherical grid: one cell whose faces carry the
      // cell's own physical flux
      if constexpr (GEOM == kSph && NDIM == 1) {
        T fl[4] = {0, 0, 0, 0}, lm, lp;
        state_flux<T, NC, 1>(u, fchat, fl, lm, lp);
        T alo = met0 * ALO(1, 0), ahi = met0 * AHI(1, 0);
#pragma unroll
        for (int v = 0; v < NV; ++v) dU[v] -= (ahi - alo) * fl[v];
        if (NC >= 3) {
          dU[3] += (ahi - alo) * fl[3];
          dU[3] -= met0 * (tabv(G, 1, TAB_AMHI, 0) - tabv(G, 1, TAB_AMLO, 0)) * fl[3];
        }
      }
      // geometric sources of the cell-centred pressure tensor of U^n
      if constexpr (GEOM != kCart) {
        T pa, pb;
        pressure<T, NC>(u, pa, pb);
        if constexpr (GEOM == kCyl) {
          T Fp = NC >= 2 ? u[2] : T(0);
          dU[1] += fchat * met0 * (pa + pb * Fp * Fp);
        } else {
          T Ft = NC >= 2 ? u[2] : T(0), Fp = NC >= 3 ? u[3] : T(0);
          T Ptt = pa + pb * Ft * Ft, Ppp = pa + pb * Fp * Fp, Prt = pb * u[1] * Ft;
          dU[1] += fchat * met0 * (Ptt + Ppp);
          if (NC >= 2) dU[2] += fchat * met0 * (tabv(G, 1, TAB_MET, p1) * Ppp - Prt);
        }
      }
      T Us[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) Us[v] = u[v] + dtf * dU[v];
      if (Us[0] < a.efloor) {
        Us[0] = a.efloor;
        rare_add(RARE_EFLOOR);
      }
      const int ci[3] = {cx, TILE_Y ? cy : (MARCH ? m : 0), TILE_Y ? m : 0};
      // Newton mode with the queue: the single linearised solve here; cells
      // it does not already converge go to the queue pass, which iterates
      // (from T^n or the learned guess) without holding back this warp.
      bool queued = false;
      CoupleOutT<T> co;
      if (a.queue_cap) {
        co = couple_cell<P, GEN>(a, ic, rho_m, e_m, kp_m, Us[0], 0.f, true);
        queued = !co.conv1;
        const unsigned int mask = __activemask();
        const unsigned int want = __ballot_sync(mask, queued);
        unsigned int base_slot = 0;
        const int leader = __ffs(mask) - 1;
        if ((tid & 31) == leader && want) base_slot = atomicAdd(a.queue_count, __popc(want));
        base_slot = __shfl_sync(mask, base_slot, leader);
        if (queued) {
          unsigned int slot = base_slot + __popc(want & ((1u << (tid & 31)) - 1u));
          if (slot < a.queue_cap && index_ok((long long)ic, padded_cells(a.dim), a.status)) {
            a.queue[slot] = ic;
            a.stash.E[ic] = S(Us[0]);
            // the single solve's T^{n+1}: the queue pass continues from it
            a.stash.e[ic] = S(co.Tnew);
#pragma unroll
            for (int v = 0; v < NC; ++v) a.stash.F[v][ic] = S(Us[1 + v]);
          } else {
            queued = false;  // queue full: iterate here
            co = couple_cell<P, GEN>(a, ic, rho_m, e_m, kp_m, Us[0], 0.f, false);
          }
        }
      } else {
        co = couple_cell<P, GEN>(a, ic, rho_m, e_m, kp_m, Us[0], 0.f, false);
      }
      if (!queued)
        finish_cell<P, NDIM, NC, GEN>(a, ic, ci, Us, rho_m, e_m, kp_m, chi_m, mom, co, cnt,
                                      !col_inner || (MARCH && (m < 2 || m >= Dm.n[MA] - 2)));
    }
    if constexpr (MARCH) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        q[0][v] = q[1][v];
        q[1][v] = q[2][v];
        hiS[v] = hiN[v];
        zlo[v] = zhi[v];
      }
      tau_m = tau_n;
      inv_own = inv_n;
      n2_own = n2_n;
      kp_m = kp_n;
      chi_m = chi_n;
      rho_m = rho_n;
      e_m = e_n;
    }
  }

  counters_flush<P>(a, cnt, s_red, tid);
}

template <class P, int NDIM, int GEOM, int NC, bool UNI, int TX, int TY, int MINB, bool GEN>
__global__ void __launch_bounds__(TX * TY, MINB) step_kernel(const __grid_constant__ StepArgs<P> a) {
  step_tile<P, NDIM, GEOM, NC, UNI, TX, TY, GEN>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

}  // namespace m1
