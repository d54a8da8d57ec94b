// m1_step_tma3.cuh -- the fused step kernel for 3D split grids with
// TMA-staged planes, non-overlapping tiles and one barrier per plane.
//
// The per-cell arithmetic is that of step_tma2_kernel; the work of a plane is
// arranged so that one CTA barrier separates the two kinds of exchange.  In
// the iteration of plane j (z = m0 - 2 + j):
//   Phase 1.  Every thread reconstructs the x and y face states of its own
//   cell of plane j and publishes the upper ones; the last two or three warps
//   add the states of the halo ring with their optical depths; the first one
//   or two warps compute the tile's upper x and y faces of plane j - 1,
//   whose states plane j - 1 published.
//   Barrier.
//   Phase 2.  Every thread computes the HLL fluxes of its lower x and y faces
//   of plane j, the march face j - 1/2 from its column registers, and updates
//   its cell of plane j - 1 from the fluxes plane j - 1 left in shared memory.
// A plane's face states and fluxes share one shared-memory buffer (a face's
// flux overwrites the state the same thread read for it), and three such
// buffers rotate over the planes, so that no phase writes a buffer that the
// other phase of a neighbouring plane, which may run at the same time in a
// slower warp, still reads.  States and fluxes are float4 (E, F0, F1, F2).
// Compared with two barriers per plane, the halo states and the upper tile
// faces, which fall on a few warps, now run side by side in one phase.
#pragma once
#include "m1_step_tma2.cuh"

namespace m1 {

constexpr int kTma3RingEF = 4;  // E/F plane slots
constexpr int kTma3RingRE = 4;  // rho/e plane slots (plane j - 1 is read in phase 2 of plane j)

template <int NC, int TX, int TY>
constexpr size_t tma3_smem_bytes() {
  return size_t(kTma3RingEF * (NC + 1) + kTma3RingRE * 2) * Tma2Tile<TX, TY>::BOXP *
             sizeof(float) +
         128;
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

template <class P, int NC, bool UNI, int TX, int TY, int MINB, bool GEN = false, int GEOM = kCart,
          bool UYZ = false>
__global__ void __launch_bounds__(TX * TY, MINB)
    step_tma3_kernel(const __grid_constant__ StepArgs<P> a, const __grid_constant__ TmaMaps tm) {
  static_assert(P::kSplit, "TMA staging is built for the split precision");
  using S = typename P::S;
  using T = typename P::T;
  static_assert(sizeof(T) == 4, "float4 exchange");
  using TL = Tma2Tile<TX, TY>;
  constexpr int NDIM = 3;
  constexpr int NV = 1 + NC, RF = kTma3RingEF, RR = kTma3RingRE;
  constexpr int BX = TL::BX, BY = TL::BY, BOXP = TL::BOXP;
  constexpr int SLOT_EF = NV * BOXP, SLOT_RE = 2 * BOXP;
  constexpr int FR = NC + 1, FE = NC + 2;  // tensor maps of rho and e
  constexpr int NT = TX * TY;
  constexpr uint32_t TX_EF = uint32_t(NV) * BX * BY * sizeof(float);
  constexpr uint32_t TX_RE = 2u * BX * BY * sizeof(float);
  constexpr int HALO_WARPS = (TL::NHALO + 31) / 32;
  constexpr int UPPER_WARPS = (TL::NEXTRA + 31) / 32;
  static_assert(HALO_WARPS + UPPER_WARPS <= NT / 32, "halo and upper faces on distinct warps");
  static_assert(NC == 3, "float4 states; the upper y faces take the x solver with F_x, F_y exchanged");

  extern __shared__ unsigned char s_dyn[];
  float* const s_ef =
      reinterpret_cast<float*>(s_dyn + ((128u - (smem_addr(s_dyn) & 127u)) & 127u));
  float* const s_re = s_ef + RF * SLOT_EF;
  __shared__ __align__(8) unsigned long long s_bar[RF + RR];  // E/F slots, then rho/e slots
  // buffer j % 3: the upper x state of column c - 1 at [c] (c = 0 .. TX), then
  // the flux of x face c - 1/2; likewise y with rows
  __shared__ float4 s_hx[3][TY][TX + 1];
  __shared__ float4 s_hy[3][TY + 1][TX];
  __shared__ float4 s_lx[2][TY];           // lower x state of column TX (buffer j % 2)
  __shared__ float4 s_ly[2][TX];           // lower y state of row TY
  __shared__ T s_tau[2][TY + 2][TX + 2];  // [row + 1][col + 1], rows/cols -1 .. TY/TX
  __shared__ unsigned long long s_red[ST_N];
  // a wait that ran out in the iteration of plane j sets s_abort[j & 1]; with
  // one barrier per plane a faster thread may already wait for the next plane
  // while a slower one reads the flag of this one
  __shared__ int s_abort[2];

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
  // The face fluxes and signal speeds are formed in units of chat (the
  // solver called with chat = 1) and the divergence takes dt chat.
  const T dtc = T(a.dt) * T(a.chat);
  const int own = (ty + 2) * BX + tx + 2;

  constexpr bool U1 = UNI || UYZ;  // directions 1 and 2 evenly spaced
  auto even = [](int d) { return d == 0 ? UNI : U1; };
  auto IXC = [&](int d, int ip) -> T { return even(d) ? T(1) : tabv(G, d, TAB_IDXC, ip); };
  auto HHI = [&](int d, int ip) -> T { return even(d) ? T(0.5) : tabv(G, d, TAB_HHI, ip); };
  auto HLO = [&](int d, int ip) -> T { return even(d) ? T(-0.5) : tabv(G, d, TAB_HLO, ip); };
  auto ALO = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_ALO, ip); };
  auto AHI = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_AHI, ip); };
  // E/F of plane j in slot j % RF; rho/e of plane j >= 1 in slot (j - 1) % RR
  // (plane 0 is read for its E and F only).
  auto slot = [&](int j) -> const float* { return s_ef + (j % RF) * SLOT_EF; };
  auto rslot = [&](int j) -> const float* { return s_re + ((j - 1) % RR) * SLOT_RE; };
  int ef_issued = -1, re_issued = 0;
  auto issue_ef = [&](int j) {  // thread 0: E and F of plane j
    ef_issued = j;
    unsigned long long* bar = &s_bar[j % RF];
    float* dst = s_ef + (j % RF) * SLOT_EF;
    mbar_arrive_expect_tx(bar, TX_EF);
    const int z = m0 + j;  // padded z of plane m0 - 2 + j
#pragma unroll
    for (int f = 0; f < NV; ++f) tma_load_3d(dst + f * BOXP, &tm.m[f], x0, y0, z, bar);
  };
  auto issue_re = [&](int j) {  // thread 0: rho and e of plane j >= 1
    re_issued = j;
    unsigned long long* bar = &s_bar[RF + (j - 1) % RR];
    float* dst = s_re + ((j - 1) % RR) * SLOT_RE;
    mbar_arrive_expect_tx(bar, TX_RE);
    const int z = m0 + j;
    tma_load_3d(dst, &tm.m[FR], x0, y0, z, bar);
    tma_load_3d(dst + BOXP, &tm.m[FE], x0, y0, z, bar);
  };
  bool ok = true;
  int cur = 0;  // abort flag of the current iteration
  auto wait_bar = [&](unsigned long long* bar, uint32_t par) {
    if (!(a.wait_polls ? mbar_test(bar, par, a.wait_polls) : mbar_wait(bar, par, kWaitLimit))) {
      ok = false;
      s_abort[cur] = 1;
    }
  };
  auto wait = [&](int j) { wait_bar(&s_bar[j % RF], uint32_t((j / RF) & 1)); };
  auto wait_re = [&](int j) {
    wait_bar(&s_bar[RF + (j - 1) % RR], uint32_t(((j - 1) / RR) & 1));
  };
  auto state_at = [&](const float* sl, int idx, T (&u)[4]) {
    u[0] = sl[idx];
#pragma unroll
    for (int v = 0; v < 3; ++v) u[1 + v] = v < NC ? sl[(1 + v) * BOXP + idx] : T(0);
  };

  if (tid == 0) {
    for (int s = 0; s < RF + RR; ++s) mbar_init(&s_bar[s], 1);
    mbar_fence_init();
    s_abort[0] = s_abort[1] = 0;
  }
  counters_reset(s_red, tid);
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < RF && j <= jlast; ++j) issue_ef(j);
    for (int j = 1; j <= RR && j <= jlast - 1; ++j) issue_re(j);
  }

  Counters cnt;
  // column registers: qm = plane j - 1, q0 = plane j, qp = plane j + 1
  T qm[4], q0[4], qp[4], hiS[4], zlo[4];
  T inv0, n20;              // 1 / E and |F|^2 of plane j
  T tau_m, kp_m, chi_m;     // optical depth and opacities of plane j - 1
#pragma unroll
  for (int v = 0; v < 4; ++v) zlo[v] = hiS[v] = T(0);

  // prologue: planes 0 .. 2 for the upper z state of plane 1 (z = m0 - 1)
  wait(0);
  wait(1);
  wait(2);
  wait_re(1);
  {
    T qa[4];
    state_at(slot(0), own, qa);
    state_at(slot(1), own, qm);
    state_at(slot(2), own, q0);
    tau_m = cell_tau<P, NDIM, GEOM, UNI>(a, rslot(1)[own], rslot(1)[BOXP + own], px, py, m0 + 1,
                                         kp_m, chi_m);
    const int pm = m0 + 1;  // padded z of plane 1
    if constexpr (U1) {
      T lo[4];
      uni_states<T, NV>(qa, qm, q0, lo, hiS);
    } else {
      T d1[4], d2[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        d1[v] = (qm[v] - qa[v]) * IXC(2, pm - 1);
        d2[v] = (q0[v] - qm[v]) * IXC(2, pm);
      }
      plm_state<T, NV>(d1, d2, qm, HHI(2, pm), hiS);
    }
    fix_face<T, NC>(hiS, qm, flux2<T, NC>(qm), Ops<T>::rcp(qm[0]));
  }
  inv0 = Ops<T>::rcp(q0[0]);
  n20 = flux2<T, NC>(q0);

  // halo face state of this thread (the last HALO_WARPS warps): item h of
  //   [0, TY): upper x of column -1, row h       [TY, 2TY): lower x of column TX
  //   [2TY, 2TY+TX): upper y of row -1, col c    [2TY+TX, 2TY+2TX): lower y of row TY
  const int h = tid - (NT - 32 * HALO_WARPS);
  const bool has_h = h >= 0 && h < TL::NHALO;
  const bool h_x = h < 2 * TY;                       // x-direction item
  const bool h_hi = h_x ? h < TY : h < 2 * TY + TX;  // upper state wanted
  const int h_rc = h_x ? (h < TY ? h : h - TY) : (h < 2 * TY + TX ? h - 2 * TY : h - 2 * TY - TX);
  // smem position of the item's cell, its neighbours' stride, table indices
  const int h_row = h_x ? h_rc + 2 : (h_hi ? 1 : TY + 2);
  const int h_col = h_x ? (h_hi ? 1 : TX + 2) : h_rc + 2;
  const int h_idx = h_row * BX + h_col;
  const int h_step = h_x ? 1 : BX;
  const int h_px = min(x0 + h_col, G.len[0] - 1);
  const int h_py = min(y0 + h_row, G.len[1] - 1);
  const int h_p = h_x ? h_px : h_py;  // padded index along the item's direction
  // upper tile face of this thread (the first UPPER_WARPS warps): x face
  // TX - 1/2 of row e (e < TY) or y face TY - 1/2 of column e - TY
  const int e = tid;
  const bool has_e = e < TL::NEXTRA;
  const bool e_x = e < TY;

  for (int j = 2; j <= jlast - 1; ++j) {
    const bool own_j = j <= jlast - 2;  // plane j holds cells of this chunk
    const bool upd = j >= 3;            // so does plane j - 1
    const int m = m0 + j - 2;           // z of plane j
    const int b3 = j % 3, bp3 = (j + 2) % 3;  // state/flux buffers of planes j, j - 1
    const int b2 = j & 1, bp2 = b2 ^ 1;       // halo and optical-depth buffers
    cur = b2;  // the prologue's waits report with plane 2's
    wait(j + 1);
    wait_re(j);
    const float* sl0 = slot(j);
    const float* rl0 = rslot(j);
    state_at(slot(j + 1), own, qp);
    // --- phase 1: optical depth and face states of plane j; the tile's upper
    // faces of plane j - 1
    // the upper faces first: the own face states then live only in registers
    if (upd && has_e) {
      // x faces (rows e < TY) and y faces (columns e - TY) share one call of
      // the x solver: a y face enters with F_x and F_y exchanged, and its
      // flux leaves with them exchanged back, so a warp holding both kinds
      // does not run the solver twice
      const int c = e - TY;
      float4 l4, r4;
      T tau_e;
      if (e_x) {
        l4 = s_hx[bp3][e][TX];
        r4 = s_lx[bp2][e];
        tau_e = T(0.5) * (s_tau[bp2][e + 1][TX] + s_tau[bp2][e + 1][TX + 1]);
      } else {
        l4 = s_hy[bp3][TY][c];
        r4 = s_ly[bp2][c];
        l4 = make_float4(l4.x, l4.z, l4.y, l4.w);
        r4 = make_float4(r4.x, r4.z, r4.y, r4.w);
        tau_e = T(0.5) * (s_tau[bp2][TY][c + 1] + s_tau[bp2][TY + 1][c + 1]);
      }
      T uL[4], uR[4], f[4];
      f4_to(l4, uL);
      f4_to(r4, uR);
      riemann<T, NC, 0>(uL, uR, T(1), tau_e, f);
      if (e_x)
        s_hx[bp3][e][TX] = f4_of(f);
      else
        s_hy[bp3][TY][c] = make_float4(f[0], f[2], f[1], f[3]);
    }
    T lox[4], loy[4];
    if (own_j) {
      T um[4], up[4], hx[4], hy[4];
      state_at(sl0, own - 1, um);
      state_at(sl0, own + 1, up);
      int nf = face_states<T, NC, UNI>(um, q0, up, IXC(0, px - 1), IXC(0, px), HLO(0, px),
                                       HHI(0, px), n20, inv0, lox, hx);
      state_at(sl0, own - BX, um);
      state_at(sl0, own + BX, up);
      nf += face_states<T, NC, U1>(um, q0, up, IXC(1, py - 1), IXC(1, py), HLO(1, py),
                                    HHI(1, py), n20, inv0, loy, hy);
      if (in_col) cnt.fix += nf;
      s_hx[b3][ty][tx + 1] = f4_of(hx);
      s_hy[b3][ty + 1][tx] = f4_of(hy);
      if (has_h) {
        T uc[4], st[4];
        state_at(sl0, h_idx, uc);
        state_at(sl0, h_idx - h_step, um);
        state_at(sl0, h_idx + h_step, up);
        const int d = h_x ? 0 : 1;
        face_state1<T, NC, UNI>(um, uc, up, IXC(d, h_p - 1), IXC(d, h_p),
                                h_hi ? HHI(d, h_p) : HLO(d, h_p), h_hi, st);
        const float4 s4 = f4_of(st);
        if (h_x) {
          if (h_hi)
            s_hx[b3][h_rc][0] = s4;
          else
            s_lx[b2][h_rc] = s4;
        } else {
          if (h_hi)
            s_hy[b3][0][h_rc] = s4;
          else
            s_ly[b2][h_rc] = s4;
        }
        T kp, chi;
        s_tau[b2][h_row - 1][h_col - 1] = cell_tau<P, NDIM, GEOM, UNI>(
            a, rl0[h_idx], rl0[BOXP + h_idx], h_px, h_py, m + 2, kp, chi);
      }
    }
    T kp0, chi0;
    const T tau0 =
        cell_tau<P, NDIM, GEOM, UNI>(a, rl0[own], rl0[BOXP + own], px, py, m + 2, kp0, chi0);
    s_tau[b2][ty + 1][tx + 1] = tau0;
    __syncthreads();
    if (s_abort[b2]) break;
    if (tid == 0) {
      // E/F of plane j - 1 and rho/e of plane j - 2 are no longer read
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (j == 2 && RF <= jlast) issue_ef(RF);
      if (j + RF - 1 <= jlast && j + RF - 1 > RF) issue_ef(j + RF - 1);
      if (j + 2 <= jlast - 1 && j + 2 > RR) issue_re(j + 2);
    }

    // --- phase 2: HLL fluxes of the lower x and y faces of plane j, the march
    // face j - 1/2 and the update of plane j - 1
    if (own_j) {
      T uL[4], f[4];
      f4_to(s_hx[b3][ty][tx], uL);
      riemann<T, NC, 0>(uL, lox, T(1), T(0.5) * (s_tau[b2][ty + 1][tx] + s_tau[b2][ty + 1][tx + 1]),
                        f);
      s_hx[b3][ty][tx] = f4_of(f);
      f4_to(s_hy[b3][ty][tx], uL);
      riemann<T, NC, 1>(uL, loy, T(1), T(0.5) * (s_tau[b2][ty][tx + 1] + s_tau[b2][ty + 1][tx + 1]),
                        f);
      s_hy[b3][ty][tx] = f4_of(f);
    }
    T zhi[4], hiN[4];
    {
      const int pz = m + 2;  // padded z of plane j
      T loN[4];
      if constexpr (U1) {
        uni_states<T, NV>(qm, q0, qp, loN, hiN);
      } else {
        const T ix1 = IXC(2, pz - 1), ix2 = IXC(2, pz);
        T d1[4], d2[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          d1[v] = (q0[v] - qm[v]) * ix1;
          d2[v] = (qp[v] - q0[v]) * ix2;
        }
        plm_state<T, NV>(d1, d2, q0, HLO(2, pz), loN);
        plm_state<T, NV>(d1, d2, q0, HHI(2, pz), hiN);
      }
      const int nf = fix_face<T, NC>(loN, q0, n20, inv0);
      const int nf2 = fix_face<T, NC>(hiN, q0, n20, inv0);
      riemann<T, NC, 2>(hiS, loN, T(1), T(0.5) * (tau_m + tau0), zhi);
      if (in_col && own_j) cnt.fix += nf + nf2;  // the z states of plane j
    }
    if (upd && in_col) {
      const long long icm = base + (long long)(m + 1) * ms;  // cell of plane j - 1
      T mom[3] = {0, 0, 0};
#pragma unroll
      for (int v = 0; v < NC; ++v) mom[v] = T(__ldg(a.in.m[v] + icm));
      const T (&u)[4] = qm;
      const int pu = m + 1;  // padded z of plane j - 1
      T Us[4];
      if constexpr (GEOM == kCart && NV == 4) {  // flux divergence on packed pairs
        // one face's float4 at a time: d += w * (F_lo, F_hi pairs)
        float2 d0 = make_float2(0.f, 0.f), d1 = d0;
        auto acc = [&](float4 f, float w) {
          const float2 w2 = make_float2(w, w);
          d0 = f2_fma(w2, make_float2(f.x, f.y), d0);
          d1 = f2_fma(w2, make_float2(f.z, f.w), d1);
        };
        acc(s_hx[bp3][ty][tx + 1], -AHI(0, px));
        acc(s_hx[bp3][ty][tx], ALO(0, px));
        acc(s_hy[bp3][ty + 1][tx], -AHI(1, py));
        acc(s_hy[bp3][ty][tx], ALO(1, py));
        acc(make_float4(zhi[0], zhi[1], zhi[2], zhi[3]), -AHI(2, pu));
        acc(make_float4(zlo[0], zlo[1], zlo[2], zlo[3]), ALO(2, pu));
        const float2 dt2 = make_float2(dtc, dtc);
        const float2 u0 = f2_fma(dt2, d0, make_float2(u[0], u[1]));
        const float2 u1 = f2_fma(dt2, d1, make_float2(u[2], u[3]));
        Us[0] = u0.x;
        Us[1] = u0.y;
        Us[2] = u1.x;
        Us[3] = u1.y;
      } else {
        T fxl[4], fxh[4], fyl[4], fyh[4];
        f4_to(s_hx[bp3][ty][tx], fxl);
        f4_to(s_hx[bp3][ty][tx + 1], fxh);
        f4_to(s_hy[bp3][ty][tx], fyl);
        f4_to(s_hy[bp3][ty + 1][tx], fyh);
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
            dU[PH] += ahi * fxh[PH] - alo * fxl[PH];
            dU[PH] -= tabv(G, 0, TAB_AMHI, px) * fxh[PH] - tabv(G, 0, TAB_AMLO, px) * fxl[PH];
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
            dU[3] += ahi * fyh[3] - alo * fyl[3];
            dU[3] -= met0 * (tabv(G, 1, TAB_AMHI, py) * fyh[3] - tabv(G, 1, TAB_AMLO, py) * fyl[3]);
          }
        }
        {
          T alo = ALO(2, pu), ahi = AHI(2, pu);
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
      const float* rlm = rslot(j - 1);
      const S rho_m = rlm[own], e_m = rlm[BOXP + own];
      const int ci[3] = {cx, cy, m - 1};
      bool queued = false;
      CoupleOut co;
      if (a.queue_cap) {
        co = couple_cell<P, GEN>(a, icm, rho_m, e_m, kp_m, Us[0], 0.f, true);
        queued = !co.conv1;
        const unsigned int mask = __activemask();
        const unsigned int want = __ballot_sync(mask, queued);
        unsigned int base_slot = 0;
        const int leader = __ffs(mask) - 1;
        if ((tid & 31) == leader && want) base_slot = atomicAdd(a.queue_count, __popc(want));
        base_slot = __shfl_sync(mask, base_slot, leader);
        if (queued) {
          unsigned int qs = base_slot + __popc(want & ((1u << (tid & 31)) - 1u));
          if (qs < a.queue_cap) {
            a.queue[qs] = icm;
            a.stash.E[icm] = S(Us[0]);
            // the single solve's T^{n+1}: the queue pass continues from it
            a.stash.e[icm] = S(co.Tnew);
#pragma unroll
            for (int v = 0; v < NC; ++v) a.stash.F[v][icm] = S(Us[1 + v]);
          } else {
            queued = false;  // queue full: iterate here
            co = couple_cell<P, GEN>(a, icm, rho_m, e_m, kp_m, Us[0], 0.f, false);
          }
        }
      } else {
        co = couple_cell<P, GEN>(a, icm, rho_m, e_m, kp_m, Us[0], 0.f, false);
      }
      if (!queued)
        finish_cell<P, NDIM, NC, GEN>(a, icm, ci, Us, rho_m, e_m, kp_m, chi_m, mom, co, cnt);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qm[v] = q0[v];
      q0[v] = qp[v];
      hiS[v] = hiN[v];
      zlo[v] = zhi[v];
    }
    tau_m = tau0;
    kp_m = kp0;
    chi_m = chi0;
    inv0 = Ops<T>::rcp(q0[0]);
    n20 = flux2<T, NC>(q0);
  }

  if (!ok) atomicOr(a.status, STATUS_TIMEOUT);
  __syncthreads();
  if ((s_abort[0] | s_abort[1]) && tid == 0) {
    // let the copies still in flight land (bounded) before the CTA exits
    // (the last phase issued on each slot: the earlier ones completed first)
    for (int j = ef_issued - RF + 1 > 0 ? ef_issued - RF + 1 : 0; j <= ef_issued; ++j)
      mbar_wait(&s_bar[j % RF], uint32_t((j / RF) & 1), kWaitLimit);
    for (int j = re_issued - RR + 1 > 1 ? re_issued - RR + 1 : 1; j <= re_issued; ++j)
      mbar_wait(&s_bar[RF + (j - 1) % RR], uint32_t(((j - 1) / RR) & 1), kWaitLimit);
  }
  counters_flush<P>(a, cnt, s_red, tid);
}

}  // namespace m1
