// m1_step_tma2.cuh -- the fused step kernel for 3D Cartesian grids in the
// split precision, with TMA-staged planes and non-overlapping tiles.
//
// A CTA of TX x TY threads updates exactly its TX x TY columns and marches
// along z (same per-cell arithmetic as step_tile).  The planes of E, F, rho
// and e, with a 2-cell halo on every side, arrive by TMA in a ring of plane
// slots (as in m1_step_tma.cuh).  Tile origins are multiples of TX, so the
// boxes need no alignment shift.
//
// Each z plane is done in two phases separated by a barrier.
//   Phase 1.  Every thread reconstructs the x and y face states of its own
//   cell (one limited slope per direction, both face states, both fixed with
//   the cell's own centre).  It keeps the lower states in registers and
//   publishes the upper ones in shared memory.  The threads of the last
//   three warps also produce the states of the halo ring the tile faces
//   need: the upper state of column -1 and row -1, the lower state of
//   column TX and row TY, with those cells' optical depths.
//   Phase 2.  Every thread computes the HLL flux of its lower x and y faces
//   from its neighbour's published upper state and its own lower state.  The
//   threads of the first two warps also compute the tile's upper faces (x
//   face TX - 1/2 per row, y face TY - 1/2 per column).
// The march face and the cell update follow as in the other kernels.
// Compared with overlapping tiles, no thread computes faces for a cell it
// does not update, and each cell's slope is computed once per direction.
#pragma once
#include "m1_step.cuh"
#include "m1_step_tma.cuh"
#include "tma.cuh"

namespace m1 {

template <int TX, int TY>
struct Tma2Tile {
  static constexpr int BX = TX + 4;                  // box columns (-2 .. TX+1)
  static constexpr int BY = TY + 4;                  // box rows (-2 .. TY+1)
  static constexpr int BOX = BX * BY;
  static constexpr int BOXP = (BOX + 31) / 32 * 32;  // 128-byte aligned stride
  static constexpr int NHALO = 2 * (TX + TY);        // halo face states per plane
  static constexpr int NEXTRA = TX + TY;             // upper tile faces per plane
};

// Plane rings: E and F of a plane in one of kTma2RingEF slots, rho and e in
// one of kTma2RingRE slots (rho and e of a plane are needed one plane later
// than its E and F, and are released one plane earlier).  One mbarrier per
// E/F slot tracks the E/F of plane k together with the rho/e of plane k - 1,
// which the same iteration needs first.
constexpr int kTma2RingEF = 4;
constexpr int kTma2RingRE = 4;

template <int NC, int TX, int TY>
constexpr size_t tma2_smem_bytes() {
  return size_t(kTma2RingEF * (NC + 1) + kTma2RingRE * 2) * Tma2Tile<TX, TY>::BOXP *
             sizeof(float) +
         128;
}

// Lower and upper reconstructed states of cell uc along one direction from
// its neighbours um (below) and up (above), each fixed with the cell's own
// centre; returns how many the fix replaced.  ixl, ixr: inverse centre
// distances of (um, uc) and (uc, up); hl, hh: offsets of the two faces.
template <class T, int NC, bool UNI>
__device__ __forceinline__ int face_states(const T (&um)[4], const T (&uc)[4], const T (&up)[4],
                                           T ixl, T ixr, T hl, T hh, T n2c, T invc, T (&lo)[4],
                                           T (&hi)[4]) {
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

__device__ __forceinline__ float4 f4_of(const float (&u)[4]) {
  return make_float4(u[0], u[1], u[2], u[3]);
}
__device__ __forceinline__ void f4_to(float4 v, float (&u)[4]) {
  u[0] = v.x;
  u[1] = v.y;
  u[2] = v.z;
  u[3] = v.w;
}

// One of the two states (the upper if `upper`), for the halo ring.
template <class T, int NC, bool UNI>
__device__ __forceinline__ void face_state1(const T (&um)[4], const T (&uc)[4], const T (&up)[4],
                                            T ixl, T ixr, T h, bool upper, T (&out)[4]) {
  constexpr int NV = 1 + NC;
  if constexpr (UNI && sizeof(T) == 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T hs = q < NV ? half_vanleer(uc[q] - um[q], up[q] - uc[q]) : T(0);
      out[q] = q < NV ? (upper ? uc[q] + hs : uc[q] - hs) : T(0);
    }
  } else {
    T dl[4], dr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dl[q] = (uc[q] - um[q]) * ixl;
      dr[q] = (up[q] - uc[q]) * ixr;
    }
    plm_state<T, NV>(dl, dr, uc, h, out);
  }
  fix_face<T, NC>(out, uc, flux2<T, NC>(uc), Ops<T>::rcp(uc[0]));
}

// GEN: the general coupling and epilogue (absorption only, irradiation,
// evolved gas); the face computation is always the default scheme.
// UYZ: directions 1 and 2 evenly spaced (a curvilinear grid stretched in
// its first direction only): their reconstruction takes the uniform form,
// while the area/volume ratios stay tabulated.
template <class P, int NC, bool UNI, int TX, int TY, int MINB, bool GEN = false, int GEOM = kCart,
          bool UYZ = false>
__global__ void __launch_bounds__(TX * TY, MINB)
    step_tma2_kernel(const __grid_constant__ StepArgs<P> a, const __grid_constant__ TmaMaps tm) {
  static_assert(P::kSplit, "TMA staging is built for the split precision");
  using S = typename P::S;
  using T = typename P::T;
  using TL = Tma2Tile<TX, TY>;
  constexpr int NDIM = 3;
  constexpr int NV = 1 + NC, RF = kTma2RingEF, RR = kTma2RingRE;
  constexpr int BX = TL::BX, BY = TL::BY, BOXP = TL::BOXP;
  constexpr int SLOT_EF = NV * BOXP, SLOT_RE = 2 * BOXP;
  constexpr int FR = NC + 1, FE = NC + 2;  // tensor maps of rho and e
  constexpr int NT = TX * TY;
  constexpr uint32_t TX_EF = uint32_t(NV) * BX * BY * sizeof(float);
  constexpr uint32_t TX_RE = 2u * BX * BY * sizeof(float);
  static_assert(TL::NHALO <= 96 && NT >= 160, "halo states on the last three warps");
  static_assert(TL::NEXTRA <= 64, "upper tile faces on the first two warps");
  static_assert(NC == 3, "float4 states; the upper y faces take the x solver with F_x, F_y exchanged");

  extern __shared__ unsigned char s_dyn[];
  float* const s_ef =
      reinterpret_cast<float*>(s_dyn + ((128u - (smem_addr(s_dyn) & 127u)) & 127u));
  float* const s_re = s_ef + RF * SLOT_EF;
  __shared__ __align__(8) unsigned long long s_bar[RF];  // E/F of plane k and rho/e of k - 1
  __shared__ T s_tau[TY + 2][TX + 2];   // [row + 1][col + 1], rows/cols -1 .. TY/TX
  // states and fluxes as float4 (E, F0, F1, F2): one shared-memory access each
  __shared__ float4 s_hx[TY][TX + 1];  // upper x state of column c at [c + 1], c = -1 .. TX-1
  __shared__ float4 s_hy[TY + 1][TX];  // upper y state of row k at [k + 1], k = -1 .. TY-1
  __shared__ float4 s_lx[TY];          // lower x state of column TX
  __shared__ float4 s_ly[TX];          // lower y state of row TY
  __shared__ float4 s_fx[TY][TX + 1];  // x face c - 1/2 at [c], c = 0 .. TX
  __shared__ float4 s_fy[TY + 1][TX];  // y face k - 1/2 at [k], k = 0 .. TY
  __shared__ unsigned long long s_red[ST_N];
  __shared__ int s_abort;

  const StepDims& Dm = a.dim;
  const GeomDev<T>& G = a.geo;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TX * ty;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int m0 = blockIdx.z * a.chunk;
  const int m1 = min(m0 + a.chunk, Dm.n[2]);
  const int jlast = m1 - m0 + 3;  // plane j <-> z = m0 - 2 + j

  const int cx = x0 + tx, cy = y0 + ty;
  const int px = min(cx + 2, G.len[0] - 1);
  const int py = min(cy + 2, G.len[1] - 1);
  const long long base = (long long)min(cx + 2, Dm.pn[0] - 1) + (long long)py * Dm.sy;
  const long long ms = Dm.sz;
  const bool in_col = cx < Dm.n[0] && cy < Dm.n[1];
  // a column at least two cells from the x and y boundaries feeds ghost
  // copies only near the z boundaries
  const bool xy_inner = cx >= 2 && cx < Dm.n[0] - 2 && cy >= 2 && cy < Dm.n[1] - 2;
  const T chat = a.chat;
  // The face fluxes and signal speeds are formed in units of chat (the
  // solver called with chat = 1) and the divergence takes dt chat.
  const T dtc = T(a.dt) * chat;
  const int own = (ty + 2) * BX + tx + 2;

  constexpr bool U1 = UNI || UYZ;  // directions 1 and 2 evenly spaced
  auto even = [](int d) { return d == 0 ? UNI : U1; };
  auto IXC = [&](int d, int ip) -> T { return even(d) ? T(1) : tabv(G, d, TAB_IDXC, ip); };
  auto HHI = [&](int d, int ip) -> T { return even(d) ? T(0.5) : tabv(G, d, TAB_HHI, ip); };
  auto HLO = [&](int d, int ip) -> T { return even(d) ? T(-0.5) : tabv(G, d, TAB_HLO, ip); };
  auto ALO = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_ALO, ip); };
  auto AHI = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_AHI, ip); };
  static_assert((RF & (RF - 1)) == 0 && (RR & (RR - 1)) == 0, "power-of-two rings");
  // E/F of plane j in slot j % RF; rho/e of plane j >= 1 in slot (j - 1) % RR
  // (plane 0 is read for its E and F only).
  auto slot = [&](int j) -> const float* { return s_ef + (j & (RF - 1)) * SLOT_EF; };
  auto rslot = [&](int j) -> const float* { return s_re + ((j - 1) & (RR - 1)) * SLOT_RE; };
  int issued = -1;
  auto issue = [&](int k) {  // thread 0: E/F of plane k and rho/e of plane k - 1 (k >= 2)
    issued = k;
    unsigned long long* bar = &s_bar[k & (RF - 1)];
    float* dst = s_ef + (k & (RF - 1)) * SLOT_EF;
    mbar_arrive_expect_tx(bar, k >= 2 ? TX_EF + TX_RE : TX_EF);
    const int z = m0 + k;  // padded z of plane m0 - 2 + k
#pragma unroll
    for (int f = 0; f < NV; ++f) tma_load_3d(dst + f * BOXP, &tm.m[f], x0, y0, z, bar);
    if (k >= 2) {
      float* rdst = s_re + ((k - 2) & (RR - 1)) * SLOT_RE;
      tma_load_3d(rdst, &tm.m[FR], x0, y0, z - 1, bar);
      tma_load_3d(rdst + BOXP, &tm.m[FE], x0, y0, z - 1, bar);
    }
  };
  bool ok = true;
  // plane k's E/F and plane k - 1's rho/e
  auto wait = [&](int k) {
    unsigned long long* bar = &s_bar[k & (RF - 1)];
    const uint32_t par = uint32_t((k / RF) & 1);
    if (!(a.wait_polls ? mbar_test(bar, par, a.wait_polls) : mbar_wait(bar, par, kWaitLimit))) {
      ok = false;
      s_abort = 1;
    }
  };
  auto state_at = [&](const float* sl, int idx, T (&u)[4]) {
    u[0] = sl[idx];
#pragma unroll
    for (int v = 0; v < 3; ++v) u[1 + v] = v < NC ? sl[(1 + v) * BOXP + idx] : T(0);
  };

  if (tid == 0) {
    for (int s = 0; s < RF; ++s) mbar_init(&s_bar[s], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  counters_reset(s_red, tid);
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < RF && k <= jlast; ++k) issue(k);

  Counters cnt;
  T q[3][4], hiS[4], zlo[4], zhi[4];
  T inv_own, n2_own, tau_m, tau_n = 0, kp_m, chi_m, kp_n = 0, chi_n = 0;
#pragma unroll
  for (int v = 0; v < 4; ++v) zlo[v] = zhi[v] = hiS[v] = T(0);

  // prologue: planes m0-2 .. m0+1 (j = 0..3) for the face m0 - 1/2
  for (int j = 0; j < 4; ++j) wait(j);  // E/F of planes 0 .. 3, rho/e of 1 and 2
  {
    T qm2[4], qm1[4];
    state_at(slot(0), own, qm2);
    state_at(slot(1), own, qm1);
    state_at(slot(2), own, q[0]);
    state_at(slot(3), own, q[1]);
    T kp, chi;
    const T tau_prev = cell_tau<P, NDIM, GEOM, UNI>(a, rslot(1)[own], rslot(1)[BOXP + own], px,
                                                    py, m0 + 1, kp, chi);
    tau_m = cell_tau<P, NDIM, GEOM, UNI>(a, rslot(2)[own], rslot(2)[BOXP + own], px, py, m0 + 2,
                                         kp_m, chi_m);
    const int pm = m0 + 2;
    inv_own = Ops<T>::rcp(q[0][0]);
    n2_own = flux2<T, NC>(q[0]);
    int nf = face4<T, NC, 2, U1>(qm2, qm1, q[0], q[1], IXC(2, pm - 2), IXC(2, pm - 1),
                                  IXC(2, pm), HHI(2, pm - 1), HLO(2, pm),
                                  T(0.5) * (tau_prev + tau_m), T(1), inv_own, n2_own, zlo);
    if (in_col) cnt.fix += nf >> 1;  // the lower z state of cell m0
    T d1[4], d2[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      d1[v] = (q[0][v] - qm1[v]) * IXC(2, pm - 1);
      d2[v] = (q[1][v] - q[0][v]) * IXC(2, pm);
    }
    plm_state<T, NV>(d1, d2, q[0], HHI(2, pm), hiS);
    int nfh = fix_face<T, NC>(hiS, q[0], n2_own, inv_own);
    if (in_col) cnt.fix += nfh;
  }
  // every thread has read plane 0: its slot takes plane RF
  __syncthreads();
  if (tid == 0 && RF <= jlast) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(RF);
  }

  // The halo item and the upper tile face of a thread are recomputed from
  // its index where they are used, not kept in registers across the march:
  // the index is read by an asm statement that is not hoisted out of the loop.
  auto fresh_tid = [&]() -> int {
    unsigned int x, y;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(x));
    asm volatile("mov.u32 %0, %%tid.y;" : "=r"(y));
    return int(x + TX * y);
  };

  for (int m = m0; m < m1; ++m) {
    const int j = m - m0 + 2;  // plane m
    // 32-bit cell index: the TMA-staged shapes run only where a padded array
    // has fewer than 2^31 cells
    const unsigned int ic = unsigned(base) + unsigned(m + 2) * unsigned(ms);
    wait(j + 2);  // E/F of plane j + 2, rho/e of plane j + 1
    const float* sl0 = slot(j);
    const float* rl0 = rslot(j);
    const float* rl1 = rslot(j + 1);
    state_at(slot(j + 2), own, q[2]);
    // --- phase 1: face states of the own cell (x and y) and of the halo
    T lox[4], loy[4];
    {
      T um[4], up[4], hx[4], hy[4];
      state_at(sl0, own - 1, um);
      state_at(sl0, own + 1, up);
      int nf = face_states<T, NC, UNI>(um, q[0], up, IXC(0, px - 1), IXC(0, px), HLO(0, px),
                                       HHI(0, px), n2_own, inv_own, lox, hx);
      state_at(sl0, own - BX, um);
      state_at(sl0, own + BX, up);
      nf += face_states<T, NC, U1>(um, q[0], up, IXC(1, py - 1), IXC(1, py), HLO(1, py),
                                    HHI(1, py), n2_own, inv_own, loy, hy);
      if (in_col) cnt.fix += nf;
      s_hx[ty][tx + 1] = f4_of(hx);
      s_hy[ty + 1][tx] = f4_of(hy);
    }
    s_tau[ty + 1][tx + 1] = tau_m;
    // halo face state of this thread (the last three warps): item h of
    //   [0, TY): upper x of column -1, row h       [TY, 2TY): lower x of column TX
    //   [2TY, 2TY+TX): upper y of row -1, col c    [2TY+TX, 2TY+2TX): lower y of row TY
    const int h = fresh_tid() - (NT - 96);
    if (h >= 0 && h < TL::NHALO) {
      const bool h_x = h < 2 * TY;                       // x-direction item
      const bool h_hi = h_x ? h < TY : h < 2 * TY + TX;  // upper state wanted
      const int h_rc =
          h_x ? (h < TY ? h : h - TY) : (h < 2 * TY + TX ? h - 2 * TY : h - 2 * TY - TX);
      // smem position of the item's cell, its neighbours' stride, table indices
      const int h_row = h_x ? h_rc + 2 : (h_hi ? 1 : TY + 2);
      const int h_col = h_x ? (h_hi ? 1 : TX + 2) : h_rc + 2;
      const int h_idx = h_row * BX + h_col;
      const int h_step = h_x ? 1 : BX;
      const int h_px = min(x0 + h_col, G.len[0] - 1);
      const int h_py = min(y0 + h_row, G.len[1] - 1);
      const int h_p = h_x ? h_px : h_py;  // padded index along the item's direction
      T uc[4], um[4], up[4], st[4];
      state_at(sl0, h_idx, uc);
      state_at(sl0, h_idx - h_step, um);
      state_at(sl0, h_idx + h_step, up);
      const int d = h_x ? 0 : 1;
      face_state1<T, NC, UNI>(um, uc, up, IXC(d, h_p - 1), IXC(d, h_p),
                              h_hi ? HHI(d, h_p) : HLO(d, h_p), h_hi, st);
      const float4 s4 = f4_of(st);
      if (h_x) {
        if (h_hi)
          s_hx[h_rc][0] = s4;
        else
          s_lx[h_rc] = s4;
      } else {
        if (h_hi)
          s_hy[0][h_rc] = s4;
        else
          s_ly[h_rc] = s4;
      }
      T kp, chi;
      s_tau[h_row - 1][h_col - 1] = cell_tau<P, NDIM, GEOM, UNI>(
          a, rl0[h_idx], rl0[BOXP + h_idx], h_px, h_py, m + 2, kp, chi);
    }
    tau_n = cell_tau<P, NDIM, GEOM, UNI>(a, rl1[own], rl1[BOXP + own], px, py, m + 3, kp_n,
                                         chi_n);
    __syncthreads();
    if (s_abort) break;
    // the E/F of plane j - 1 (last read in iteration m - 1 or the prologue)
    // and the rho/e of plane j - 2 are no longer read: their slots take the
    // E/F of plane j + 3 and the rho/e of plane j + 2
    if (tid == 0 && j + 3 <= jlast) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(j + 3);
    }

    // --- phase 2: HLL fluxes of the lower x and y faces (and upper tile faces)
    {
      T uL[4], f[4];
      f4_to(s_hx[ty][tx], uL);
      riemann<T, NC, 0>(uL, lox, T(1), T(0.5) * (s_tau[ty + 1][tx] + s_tau[ty + 1][tx + 1]), f);
      s_fx[ty][tx] = f4_of(f);
      f4_to(s_hy[ty][tx], uL);
      riemann<T, NC, 1>(uL, loy, T(1), T(0.5) * (s_tau[ty][tx + 1] + s_tau[ty + 1][tx + 1]), f);
      s_fy[ty][tx] = f4_of(f);
    }
    // upper tile face of this thread (the first two warps): x face TX - 1/2
    // of row e (e < TY) or y face TY - 1/2 of column e - TY
    const int e = fresh_tid();
    if (e < TL::NEXTRA) {
      const bool e_x = e < TY;
      // x faces (rows e < TY) and y faces (columns e - TY) share one call of
      // the x solver: a y face enters with F_x and F_y exchanged, and its
      // flux leaves with them exchanged back, so a warp holding both kinds
      // does not run the solver twice
      const int c = e - TY;
      float4 l4, r4;
      T tau_e;
      if (e_x) {
        l4 = s_hx[e][TX];
        r4 = s_lx[e];
        tau_e = T(0.5) * (s_tau[e + 1][TX] + s_tau[e + 1][TX + 1]);
      } else {
        l4 = s_hy[TY][c];
        r4 = s_ly[c];
        l4 = make_float4(l4.x, l4.z, l4.y, l4.w);
        r4 = make_float4(r4.x, r4.z, r4.y, r4.w);
        tau_e = T(0.5) * (s_tau[TY][c + 1] + s_tau[TY + 1][c + 1]);
      }
      T uL[4], uR[4], f[4];
      f4_to(l4, uL);
      f4_to(r4, uR);
      riemann<T, NC, 0>(uL, uR, T(1), tau_e, f);
      if (e_x)
        s_fx[e][TX] = f4_of(f);
      else
        s_fy[TY][c] = make_float4(f[0], f[2], f[1], f[3]);
    }
    // march face m + 1/2 from the column registers
    T hiN[4];
    T inv_n = Ops<T>::rcp(q[1][0]);
    T n2_n = flux2<T, NC>(q[1]);
    {
      const int pm = m + 3;  // padded z of cell m + 1
      T loN[4];
      if constexpr (U1) {
        uni_states<T, NV>(q[0], q[1], q[2], loN, hiN);
      } else {
        T ix1 = IXC(2, pm - 1), ix2 = IXC(2, pm);
        T d1[4], d2[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          d1[v] = (q[1][v] - q[0][v]) * ix1;
          d2[v] = (q[2][v] - q[1][v]) * ix2;
        }
        plm_state<T, NV>(d1, d2, q[1], HLO(2, pm), loN);
        plm_state<T, NV>(d1, d2, q[1], HHI(2, pm), hiN);
      }
      int nf = fix_face<T, NC>(loN, q[1], n2_n, inv_n);
      int nf2 = fix_face<T, NC>(hiN, q[1], n2_n, inv_n);
      riemann<T, NC, 2>(hiS, loN, T(1), T(0.5) * (tau_m + tau_n), zhi);
      if (in_col && m + 1 < m1) cnt.fix += nf + nf2;  // the z states of cell m + 1
    }
    __syncthreads();

    // update of the own cell
    if (in_col) {
      // the gas momentum is loaded here rather than with the plane: three
      // registers fewer across both phases
      T mom[3] = {0, 0, 0};
#pragma unroll
      for (int v = 0; v < NC; ++v) mom[v] = T(__ldg(a.in.m[v] + ic));
      const T (&u)[4] = q[0];
      T Us[4];
      T fxl[4], fxh[4], fyl[4], fyh[4];
      f4_to(s_fx[ty][tx], fxl);
      f4_to(s_fx[ty][tx + 1], fxh);
      f4_to(s_fy[ty][tx], fyl);
      f4_to(s_fy[ty + 1][tx], fyh);
      if constexpr (GEOM == kCart && NV == 4) {  // flux divergence on packed pairs
        const float2 mx = make_float2(-AHI(0, px), -AHI(0, px)), px_ = make_float2(ALO(0, px), ALO(0, px));
        const float2 my = make_float2(-AHI(1, py), -AHI(1, py)), py_ = make_float2(ALO(1, py), ALO(1, py));
        const float2 mz = make_float2(-AHI(2, m + 2), -AHI(2, m + 2));
        const float2 pz = make_float2(ALO(2, m + 2), ALO(2, m + 2));
        const float2 dt2 = make_float2(dtc, dtc);
#pragma unroll
        for (int h = 0; h < 4; h += 2) {
          float2 d = f2_mul(mx, make_float2(fxh[h], fxh[h + 1]));
          d = f2_fma(px_, make_float2(fxl[h], fxl[h + 1]), d);
          d = f2_fma(my, make_float2(fyh[h], fyh[h + 1]), d);
          d = f2_fma(py_, make_float2(fyl[h], fyl[h + 1]), d);
          d = f2_fma(mz, make_float2(zhi[h], zhi[h + 1]), d);
          d = f2_fma(pz, make_float2(zlo[h], zlo[h + 1]), d);
          const float2 us = f2_fma(dt2, d, make_float2(u[h], u[h + 1]));
          Us[h] = us.x;
          Us[h + 1] = us.y;
        }
      } else {
        // unsplit divergence with the factorised area/volume ratios; on
        // curvilinear grids the angular-momentum form of the phi component
        // and the geometric sources of the centred pressure tensor
        T dU[4] = {0, 0, 0, 0};
        {
          const T alo = ALO(0, px), ahi = AHI(0, px);
#pragma unroll
          for (int v = 0; v < NV; ++v) dU[v] -= ahi * fxh[v] - alo * fxl[v];
          if constexpr (GEOM != kCart) {
            constexpr int PH = GEOM == kCyl ? 2 : 3;  // the phi component
            const T fhi = fxh[PH], flo = fxl[PH];
            dU[PH] += ahi * fhi - alo * flo;
            dU[PH] -= tabv(G, 0, TAB_AMHI, px) * fhi - tabv(G, 0, TAB_AMLO, px) * flo;
          }
        }
        const T met0 = GEOM != kCart ? tabv(G, 0, TAB_MET, px) : T(1);
        {
          T alo = ALO(1, py), ahi = AHI(1, py);
          if constexpr (GEOM != kCart) {
            alo *= met0;
            ahi *= met0;
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) dU[v] -= ahi * fyh[v] - alo * fyl[v];
          if constexpr (GEOM == kSph) {
            const T fhi = fyh[3], flo = fyl[3];
            dU[3] += ahi * fhi - alo * flo;
            dU[3] -= met0 * (tabv(G, 1, TAB_AMHI, py) * fhi - tabv(G, 1, TAB_AMLO, py) * flo);
          }
        }
        {
          T alo = ALO(2, m + 2), ahi = AHI(2, m + 2);
          if constexpr (GEOM == kSph) {
            const T f = met0 * tabv(G, 1, TAB_PHF, py);
            alo *= f;
            ahi *= f;
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) dU[v] -= ahi * zhi[v] - alo * zlo[v];
        }
        if constexpr (GEOM != kCart) {
          T pa, pb;
          pressure<T, NC>(u, pa, pb);
          if constexpr (GEOM == kCyl) {
            dU[1] += met0 * (pa + pb * u[2] * u[2]);
          } else {
            const T Ft = u[2], Fp = u[3];
            const T Ptt = pa + pb * Ft * Ft, Ppp = pa + pb * Fp * Fp, Prt = pb * u[1] * Ft;
            dU[1] += met0 * (Ptt + Ppp);
            dU[2] += met0 * (tabv(G, 1, TAB_MET, py) * Ppp - Prt);
          }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) Us[v] = u[v] + dtc * dU[v];
      }
      if (Us[0] < a.efloor) {
        Us[0] = a.efloor;
        rare_add(RARE_EFLOOR);
      }
      const S rho_m = rl0[own], e_m = rl0[BOXP + own];
      const int ci[3] = {cx, cy, m};
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
          unsigned int qs = base_slot + __popc(want & ((1u << (tid & 31)) - 1u));
          if (qs < a.queue_cap && index_ok((long long)ic, padded_cells(a.dim), a.status)) {
            a.queue[qs] = ic;
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
                                      !xy_inner || m < 2 || m >= Dm.n[2] - 2);
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
  }

  if (!ok) atomicOr(a.status, STATUS_TIMEOUT);
  __syncthreads();
  if (s_abort && tid == 0) {
    // let the copies still in flight land (bounded) before the CTA exits
    // (the last phase issued on each slot: the earlier ones completed first)
    for (int k = issued - RF + 1 > 0 ? issued - RF + 1 : 0; k <= issued; ++k)
      mbar_wait(&s_bar[k & (RF - 1)], uint32_t((k / RF) & 1), kWaitLimit);
  }
  counters_flush<P>(a, cnt, s_red, tid);
}

}  // namespace m1
