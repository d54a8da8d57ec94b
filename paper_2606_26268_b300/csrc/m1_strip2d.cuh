// m1_strip2d.cuh -- one tile of the fused step on a 2D Cartesian grid as a
// single warp: a strip of 32 columns marching along y, with the row
// exchanged between lanes by warp shuffles instead of shared memory, so
// that a row needs no barrier.
//
// The arithmetic per cell is that of step_tile (m1_step.cuh) for NDIM = 2:
// lane k owns column x0 + k, reconstructs its cell's two x face states once
// (its neighbours' states by shuffles), passes the upper one to lane k + 1
// and computes the x face x0 + k - 1/2 from the upper state of lane k - 1
// and its own lower state; lanes 0..30 update their cell with their own
// face and the face of the lane to their right, so strips overlap by one
// column (31 updated columns per strip).  The cells left of the strip
// (x0 - 2, x0 - 1, whose upper state and optical depth the face x0 - 1/2
// needs) are loaded by lane 0 and the cell right of it (x0 + 32) by lane 31,
// a row ahead.  The march face and the cell update follow step_tile.
// Default form (no face options, absorption-only coupling or irradiation
// deposit).
#pragma once
#include "m1_step.cuh"

namespace m1 {

// Lower (lo) and upper (hi) x face states of cell uc between um and up,
// each fixed with the cell's own centre; returns how many the fix replaced.
template <class T, int NC, bool UNI>
__device__ __forceinline__ int face_states_x(const T (&um)[4], const T (&uc)[4], const T (&up)[4],
                                             T ixl, T ixr, T hl, T hh, T n2c, T invc,
                                             T (&lo)[4], T (&hi)[4]) {
  constexpr int NV = 1 + NC;
  if constexpr (UNI && sizeof(T) == 4) {
    uni_states<T, NV>(um, uc, up, lo, hi);
  } else {
    T dl[4], dr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dl[q] = (uc[q] - um[q]) * ixl;
      dr[q] = (up[q] - uc[q]) * ixr;
    }
    plm_state<T, NV>(dl, dr, uc, hl, lo);
    plm_state<T, NV>(dl, dr, uc, hh, hi);
  }
  return fix_face<T, NC>(lo, uc, n2c, invc) + fix_face<T, NC>(hi, uc, n2c, invc);
}

template <class P, int NC, bool UNI>
__device__ __forceinline__ void step_strip2d(const StepArgs<P>& a, int bx, int by) {
  using S = typename P::S;
  using T = typename P::T;
  constexpr int NDIM = 2, GEOM = kCart, NV = 1 + NC, MA = 1;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ unsigned long long s_red[ST_N];

  const StepDims& Dm = a.dim;
  const GeomDev<T>& G = a.geo;
  const int k = threadIdx.x;  // lane
  const int x0 = bx * 31;
  const int m0 = by * a.chunk;
  const int m1 = min(m0 + a.chunk, Dm.n[1]);
  counters_reset(s_red, k);

  const int cx = x0 + k;
  const int px = min(cx + Dm.g[0], G.len[0] - 1);
  const int pxa = min(cx + Dm.g[0], Dm.pn[0] - 1);
  const long long base = (long long)pxa;
  const long long ms = Dm.sy;
  const int gm = Dm.g[1];
  const bool upd_col = cx < Dm.n[0] && k <= 30;
  // a column at least two cells from the x boundaries feeds ghost copies
  // only near the y boundaries
  const bool x_inner = cx >= 2 && cx < Dm.n[0] - 2;
  // In the split precision the face fluxes and signal speeds are formed in
  // units of chat (the flux functions take fchat = 1) and the divergence
  // is scaled by dt chat; in FP64 they carry chat as the oracle does.
  const T fchat = P::kSplit ? T(1) : T(a.chat);
  const T dtf = P::kSplit ? T(a.dt) * T(a.chat) : T(a.dt);

  auto IXC = [&](int d, int ip) -> T { return UNI ? T(1) : tabv(G, d, TAB_IDXC, ip); };
  auto HHI = [&](int d, int ip) -> T { return UNI ? T(0.5) : tabv(G, d, TAB_HHI, ip); };
  auto HLO = [&](int d, int ip) -> T { return UNI ? T(-0.5) : tabv(G, d, TAB_HLO, ip); };
  auto ALO = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_ALO, ip); };
  auto AHI = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_AHI, ip); };

  __syncthreads();  // counters zeroed
  Counters cnt;
  T q[3][4], hiS[4], zlo[4], zhi[4];
  T inv_own = 0, n2_own = 0;
  T tau_m = 0, tau_n = 0, kp_m = 0, chi_m = 0, kp_n = 0, chi_n = 0;
  S rho_m = 0, e_m = 0, rho_n = 0, e_n = 0;
#pragma unroll
  for (int v = 0; v < 4; ++v) zlo[v] = zhi[v] = hiS[v] = T(0);

  {
    T qm2[4], qm1[4];
    load_state<S, NC>(a.in, base + (long long)(m0 - 2 + gm) * ms, qm2);
    load_state<S, NC>(a.in, base + (long long)(m0 - 1 + gm) * ms, qm1);
    load_state<S, NC>(a.in, base + (long long)(m0 + gm) * ms, q[0]);
    load_state<S, NC>(a.in, base + (long long)(m0 + 1 + gm) * ms, q[1]);
    T tau_prev;
    {
      const long long i = base + (long long)(m0 - 1 + gm) * ms;
      T kp, chi;
      tau_prev = cell_tau<P, NDIM, GEOM, UNI>(a, __ldg(a.rho + i), __ldg(a.in.e + i), px,
                                              m0 - 1 + gm, 0, kp, chi);
    }
    {
      const long long i = base + (long long)(m0 + gm) * ms;
      rho_m = __ldg(a.rho + i);
      e_m = __ldg(a.in.e + i);
      tau_m = cell_tau<P, NDIM, GEOM, UNI>(a, rho_m, e_m, px, m0 + gm, 0, kp_m, chi_m);
    }
    const int pm = m0 + gm;
    const T ix1 = IXC(MA, pm - 1), ix2 = IXC(MA, pm);
    inv_own = Ops<T>::rcp(q[0][0]);
    n2_own = flux2<T, NC>(q[0]);
    const int nf = face4<T, NC, MA, UNI>(qm2, qm1, q[0], q[1], IXC(MA, pm - 2), ix1, ix2,
                                         HHI(MA, pm - 1), HLO(MA, pm),
                                         T(0.5) * (tau_prev + tau_m), fchat, inv_own, n2_own, zlo);
    if (upd_col) cnt.fix += nf >> 1;  // the lower march state of cell m0
    T d1[4], d2[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      d1[v] = (q[0][v] - qm1[v]) * ix1;
      d2[v] = (q[1][v] - q[0][v]) * ix2;
    }
    plm_state<T, NV>(d1, d2, q[0], HHI(MA, pm), hiS);
    const int nfh = fix_face<T, NC>(hiS, q[0], n2_own, inv_own);
    if (upd_col) cnt.fix += nfh;
  }

  // the strip's outside cells: lane 0 columns x0 - 2 (ha) and x0 - 1 (hb,
  // with its rho and e), lane 31 column x0 + 32 (hb)
  const int hxa = min(max(x0 - 2 + Dm.g[0], 0), Dm.pn[0] - 1);
  const int hxb = min(max(x0 + (k == 0 ? -1 : 32) + Dm.g[0], 0), Dm.pn[0] - 1);
  T ha[4] = {0, 0, 0, 0}, hb[4] = {0, 0, 0, 0};
  S hrho = S(1), he = S(1);
  auto load_halo = [&](int m) {
    if (k == 0 || k == 31) {
      const long long ib = hxb + (long long)(m + gm) * ms;
      load_state<S, NC>(a.in, ib, hb);
      if (k == 0) {
        load_state<S, NC>(a.in, hxa + (long long)(m + gm) * ms, ha);
        hrho = __ldg(a.rho + ib);
        he = __ldg(a.in.e + ib);
      }
    }
  };
  load_halo(m0);
  S rho_p = __ldg(a.rho + base + (long long)(m0 + 1 + gm) * ms);
  S e_p = __ldg(a.in.e + base + (long long)(m0 + 1 + gm) * ms);

  for (int m = m0; m < m1; ++m) {
    const long long ic = base + (long long)(m + gm) * ms;  // own cell
    T mom[3] = {0, 0, 0};
    load_state<S, NC>(a.in, ic + 2 * ms, q[2]);
    rho_n = rho_p;
    e_n = e_p;
    rho_p = __ldg(a.rho + ic + 2 * ms);
    e_p = __ldg(a.in.e + ic + 2 * ms);
    if (upd_col) {
#pragma unroll
      for (int v = 0; v < NC; ++v) mom[v] = T(__ldg(a.in.m[v] + ic));
    }
    // the row around this lane's column: its neighbours by shuffles, the
    // outside cells from lanes 0 and 31
    T um1[4], up1[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (v < NV) {
        const T own = q[0][v];
        const T sU1 = __shfl_up_sync(FULL, own, 1);
        const T sD1 = __shfl_down_sync(FULL, own, 1);
        um1[v] = k >= 1 ? sU1 : hb[v];
        up1[v] = k <= 30 ? sD1 : hb[v];
      } else {
        um1[v] = up1[v] = T(0);
      }
    }
    // the two x face states of this lane's cell, fixed with its centre
    T lox[4], hix[4];
    const int nfx = face_states_x<T, NC, UNI>(um1, q[0], up1, IXC(0, px - 1), IXC(0, px),
                                              HLO(0, px), HHI(0, px), n2_own, inv_own, lox, hix);
    if (upd_col) cnt.fix += nfx;
    // the upper state and optical depth of the column left of each lane's
    // face: lane k - 1's, or for lane 0 the outside column x0 - 1
    T uL[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) uL[v] = __shfl_up_sync(FULL, hix[v], 1);
    T tL = __shfl_up_sync(FULL, tau_m, 1);
    if (k == 0) {
      T lo0[4];
      face_states_x<T, NC, UNI>(ha, hb, q[0], IXC(0, px - 2), IXC(0, px - 1), HLO(0, px - 1),
                                HHI(0, px - 1), flux2<T, NC>(hb), Ops<T>::rcp(hb[0]), lo0, uL);
      T kp, chi;
      tL = cell_tau<P, NDIM, GEOM, UNI>(a, hrho, he, min(hxb, G.len[0] - 1), m + gm, 0, kp, chi);
    }
    if (m + 1 < m1) load_halo(m + 1);
    tau_n = cell_tau<P, NDIM, GEOM, UNI>(a, rho_n, e_n, px, m + 1 + gm, 0, kp_n, chi_n);

    // x face (column - 1/2)
    T fx[4];
    riemann<T, NC, 0>(uL, lox, fchat, T(0.5) * (tL + tau_m), fx);
    T fhi[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) fhi[v] = __shfl_down_sync(FULL, fx[v], 1);

    // march face m + 1/2 from the column registers
    T hiN[4];
    const T inv_n = Ops<T>::rcp(q[1][0]);
    const T n2_n = flux2<T, NC>(q[1]);
    {
      const int pm = m + 1 + gm;  // padded index of cell m+1
      T loN[4];
      if constexpr (UNI && sizeof(T) == 4) {
        uni_states<T, NV>(q[0], q[1], q[2], loN, hiN);
      } else {
        const T ix1 = IXC(MA, pm - 1), ix2 = IXC(MA, pm);
        T d1[4], d2[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          d1[v] = (q[1][v] - q[0][v]) * ix1;
          d2[v] = (q[2][v] - q[1][v]) * ix2;
        }
        plm_state<T, NV>(d1, d2, q[1], HLO(MA, pm), loN);
        plm_state<T, NV>(d1, d2, q[1], HHI(MA, pm), hiN);
      }
      const int nf = fix_face<T, NC>(loN, q[1], n2_n, inv_n);
      const int nf2 = fix_face<T, NC>(hiN, q[1], n2_n, inv_n);
      riemann<T, NC, MA>(hiS, loN, fchat, T(0.5) * (tau_m + tau_n), zhi);
      if (upd_col && m + 1 < m1) cnt.fix += nf + nf2;  // the march states of cell m + 1
    }

    // update of the own cell
    if (upd_col) {
      T dU[4] = {0, 0, 0, 0};
      {
        const T alo = ALO(0, px), ahi = AHI(0, px);
#pragma unroll
        for (int v = 0; v < NV; ++v) dU[v] -= ahi * fhi[v] - alo * fx[v];
      }
      {
        const T alo = ALO(1, m + gm), ahi = AHI(1, m + gm);
#pragma unroll
        for (int v = 0; v < NV; ++v) dU[v] -= ahi * zhi[v] - alo * zlo[v];
      }
      const T (&u)[4] = q[0];
      T Us[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) Us[v] = u[v] + dtf * dU[v];
      if (Us[0] < a.efloor) {
        Us[0] = a.efloor;
        rare_add(RARE_EFLOOR);
      }
      const int ci[3] = {cx, m, 0};
      bool queued = false;
      CoupleOutT<T> co;
      if (a.queue_cap) {
        co = couple_cell<P, false>(a, ic, rho_m, e_m, kp_m, Us[0], 0.f, true);
        queued = !co.conv1;
        const unsigned int mask = __activemask();
        const unsigned int want = __ballot_sync(mask, queued);
        unsigned int base_slot = 0;
        const int leader = __ffs(mask) - 1;
        if (k == leader && want) base_slot = atomicAdd(a.queue_count, __popc(want));
        base_slot = __shfl_sync(mask, base_slot, leader);
        if (queued) {
          const unsigned int slot = base_slot + __popc(want & ((1u << k) - 1u));
          if (slot < a.queue_cap && index_ok((long long)ic, padded_cells(a.dim), a.status)) {
            a.queue[slot] = ic;
            a.stash.E[ic] = S(Us[0]);
            // the single solve's T^{n+1}: the queue pass continues from it
            a.stash.e[ic] = S(co.Tnew);
#pragma unroll
            for (int v = 0; v < NC; ++v) a.stash.F[v][ic] = S(Us[1 + v]);
          } else {
            queued = false;  // queue full: iterate here
            co = couple_cell<P, false>(a, ic, rho_m, e_m, kp_m, Us[0], 0.f, false);
          }
        }
      } else {
        co = couple_cell<P, false>(a, ic, rho_m, e_m, kp_m, Us[0], 0.f, false);
      }
      if (!queued)
        finish_cell<P, NDIM, NC, false>(a, ic, ci, Us, rho_m, e_m, kp_m, chi_m, mom, co, cnt,
                                        !x_inner || m < 2 || m >= Dm.n[1] - 2);
    }
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
  counters_flush<P>(a, cnt, s_red, k);
}

template <class P, int NC, bool UNI, int MINB>
__global__ void __launch_bounds__(32, MINB) step_strip2d_kernel(const __grid_constant__ StepArgs<P> a) {
  step_strip2d<P, NC, UNI>(a, blockIdx.x, blockIdx.y);
}

}  // namespace m1
