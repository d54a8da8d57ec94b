// m1_step_tma.cuh -- the fused step kernel for 3D Cartesian grids in the
// split precision, with the march planes staged by TMA.
//
// Same method, tile decomposition and per-cell arithmetic as step_tile
// (m1_step.cuh): a CTA of TX x TY threads owns an overlapped x-y tile and
// marches along z.  The difference is how the planes reach the CTA.  One
// thread loads each z plane of the tile, with its halo (columns -2..TX, rows
// -2..TY) and for all the fields the step reads (E, F, rho, e), as TMA boxes
// into a ring of R plane slots, each slot tracked by an mbarrier.  A plane
// is issued one iteration before it is first needed; every thread then reads
// its own column, its neighbours and the halo from shared memory.  This removes the
// per-thread halo loads, the register copies that prefetched them and the
// shared-memory stores of the state.
//
// Box geometry.  A TMA box must start at an x coordinate that is a multiple
// of 16 bytes, but tile origins are multiples of TX - 1 cells.  The box
// therefore starts at the origin rounded down to 4 elements and is BX >= TX
// + 6 columns wide; xo = origin - start selects the tile inside it.  Boxes
// that reach past the array are zero-filled by TMA; those cells are outside
// the domain and none of their results is stored.
#pragma once
#include "m1_step.cuh"
#include "tma.cuh"

namespace m1 {

struct TmaMaps {
  CUtensorMap m[6];  // E, F[0..NC-1], rho, e of the input buffer
};

template <int TX, int TY>
struct TmaTile {
  static constexpr int BX = (TX + 6 + 3) / 4 * 4;    // box columns
  static constexpr int BY = TY + 3;                  // box rows
  static constexpr int BOX = BX * BY;                // floats per box
  static constexpr int BOXP = (BOX + 31) / 32 * 32;  // 128-byte aligned stride
};

constexpr int kTmaRing = 5;  // plane slots

// dynamic shared memory of the ring, with the alignment slack
template <int NC, int TX, int TY>
constexpr size_t tma_smem_bytes() {
  return size_t(kTmaRing) * (NC + 3) * TmaTile<TX, TY>::BOXP * sizeof(float) + 128;
}

// GEN: the general coupling and epilogue (absorption only, irradiation,
// evolved gas); the face computation is always the default scheme.
template <class P, int NC, bool UNI, int TX, int TY, int MINB, bool GEN = false>
__global__ void __launch_bounds__(TX * TY, MINB)
    step_tma_kernel(const __grid_constant__ StepArgs<P> a, const __grid_constant__ TmaMaps tm) {
  static_assert(P::kSplit, "TMA staging is built for the split precision");
  using S = typename P::S;
  using T = typename P::T;
  constexpr int NDIM = 3, GEOM = kCart;
  constexpr int NV = 1 + NC, NF = NC + 3, R = kTmaRing;
  constexpr int BX = TmaTile<TX, TY>::BX, BY = TmaTile<TX, TY>::BY;
  constexpr int BOXP = TmaTile<TX, TY>::BOXP;
  constexpr int SLOT = NF * BOXP;
  constexpr int FR = NC + 1, FE = NC + 2;  // field index of rho and e in a slot
  constexpr uint32_t TX_BYTES = uint32_t(NF) * BX * BY * sizeof(float);

  // ring of R plane slots in dynamic shared memory, aligned here to the
  // 128 bytes a TMA destination needs (128 bytes of slack are allocated)
  // (the pointer is formed from s_dyn by an offset, so that the compiler
  // keeps the shared state space and addresses the slots directly)
  extern __shared__ unsigned char s_dyn[];
  float* const s_ring =
      reinterpret_cast<float*>(s_dyn + ((128u - (smem_addr(s_dyn) & 127u)) & 127u));
  __shared__ __align__(8) unsigned long long s_bar[R];
  __shared__ T s_tau[TY + 1][TX + 1];
  __shared__ T s_fx[NV][TY][TX];
  __shared__ T s_fy[NV][TY][TX];
  __shared__ unsigned long long s_red[ST_N];
  __shared__ int s_abort;

  const StepDims& Dm = a.dim;
  const GeomDev<T>& G = a.geo;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TX * ty;
  const int x0 = blockIdx.x * (TX - 1), y0 = blockIdx.y * (TY - 1);
  const int m0 = blockIdx.z * a.chunk;
  const int m1 = min(m0 + a.chunk, Dm.n[2]);
  const int xs = x0 & ~3, xo = x0 - xs;  // box start (padded x) and tile offset in the box
  const int jlast = m1 - m0 + 3;         // plane j <-> z = m0 - 2 + j, j = 0..jlast

  const int cx = x0 + tx, cy = y0 + ty;
  const int px = min(cx + 2, G.len[0] - 1);
  const int py = min(cy + 2, G.len[1] - 1);
  const long long base = (long long)min(cx + 2, Dm.pn[0] - 1) + (long long)py * Dm.sy;
  const long long ms = Dm.sz;
  const bool in_col = cx < Dm.n[0] && cy < Dm.n[1];
  const bool upd_col = in_col && tx <= TX - 2 && ty <= TY - 2;
  // The face fluxes and signal speeds are formed in units of chat (the
  // flux functions take chat = 1) and the divergence is scaled by dt chat.
  const T dtc = T(a.dt) * T(a.chat);
  const int own = (ty + 2) * BX + tx + 2 + xo;  // own cell inside a box

  auto IXC = [&](int d, int ip) -> T { return UNI ? T(1) : tabv(G, d, TAB_IDXC, ip); };
  auto HHI = [&](int d, int ip) -> T { return UNI ? T(0.5) : tabv(G, d, TAB_HHI, ip); };
  auto HLO = [&](int d, int ip) -> T { return UNI ? T(-0.5) : tabv(G, d, TAB_HLO, ip); };
  auto ALO = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_ALO, ip); };
  auto AHI = [&](int d, int ip) -> T { return UNI ? a.uni_inv[d] : tabv(G, d, TAB_AHI, ip); };
  auto slot = [&](int j) -> const float* { return s_ring + (j % R) * SLOT; };
  int jissued = -1;  // thread 0: last plane issued
  auto issue = [&](int j) {  // thread 0: plane j into its slot
    jissued = j;
    unsigned long long* bar = &s_bar[j % R];
    float* dst = s_ring + (j % R) * SLOT;
    mbar_arrive_expect_tx(bar, TX_BYTES);
    const int z = m0 + j;  // padded z of plane m0 - 2 + j
#pragma unroll
    for (int f = 0; f < NF; ++f) tma_load_3d(dst + f * BOXP, &tm.m[f], xs, y0, z, bar);
  };
  bool ok = true;
  auto wait = [&](int j) {
    const uint32_t par = uint32_t((j / R) & 1);
    if (!(a.wait_polls ? mbar_test(&s_bar[j % R], par, a.wait_polls)
                       : mbar_wait(&s_bar[j % R], par, kWaitLimit))) {
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
    for (int s = 0; s < R; ++s) mbar_init(&s_bar[s], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  counters_reset(s_red, tid);
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < R && j <= jlast; ++j) issue(j);

  Counters cnt;
  T q[3][4], hiS[4], zlo[4], zhi[4];
  T inv_own, n2_own, tau_m, tau_n = 0, kp_m, chi_m, kp_n = 0, chi_n = 0;
#pragma unroll
  for (int v = 0; v < 4; ++v) zlo[v] = zhi[v] = hiS[v] = T(0);

  // prologue: planes m0-2 .. m0+1 (j = 0..3) for the face m0 - 1/2
  for (int j = 0; j < 4; ++j) wait(j);
  {
    T qm2[4], qm1[4];
    state_at(slot(0), own, qm2);
    state_at(slot(1), own, qm1);
    state_at(slot(2), own, q[0]);
    state_at(slot(3), own, q[1]);
    T kp, chi;
    const T tau_prev = cell_tau<P, NDIM, GEOM, UNI>(a, slot(1)[FR * BOXP + own],
                                                    slot(1)[FE * BOXP + own], px, py, m0 + 1,
                                                    kp, chi);
    tau_m = cell_tau<P, NDIM, GEOM, UNI>(a, slot(2)[FR * BOXP + own], slot(2)[FE * BOXP + own],
                                         px, py, m0 + 2, kp_m, chi_m);
    const int pm = m0 + 2;
    inv_own = Ops<T>::rcp(q[0][0]);
    n2_own = flux2<T, NC>(q[0]);
    int nf = face4<T, NC, 2, UNI>(qm2, qm1, q[0], q[1], IXC(2, pm - 2), IXC(2, pm - 1),
                                  IXC(2, pm), HHI(2, pm - 1), HLO(2, pm),
                                  T(0.5) * (tau_prev + tau_m), T(1), inv_own, n2_own, zlo);
    if (upd_col) cnt.fix += nf >> 1;  // the lower march state of cell m0
    T d1[4], d2[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      d1[v] = (q[0][v] - qm1[v]) * IXC(2, pm - 1);
      d2[v] = (q[1][v] - q[0][v]) * IXC(2, pm);
    }
    plm_state<T, NV>(d1, d2, q[0], HHI(2, pm), hiS);
    int nfh = fix_face<T, NC>(hiS, q[0], n2_own, inv_own);
    if (upd_col) cnt.fix += nfh;
  }

  // halo cells whose optical depth this thread supplies: column -1 of row
  // tid (tid < TY) or row -1 of column tid - TY (TY <= tid < TY + TX)
  const bool htau_col = tid < TY, htau_row = tid >= TY && tid < TY + TX;
  const int hidx = htau_col ? (tid + 2) * BX + 1 + xo : BX + (tid - TY) + 2 + xo;
  const int hpx = htau_col ? min(x0 + 1, G.len[0] - 1) : min(x0 + (tid - TY) + 2, G.len[0] - 1);
  const int hpy = htau_col ? min(y0 + tid + 2, G.len[1] - 1) : min(y0 + 1, G.len[1] - 1);

  for (int m = m0; m < m1; ++m) {
    const int j = m - m0 + 2;  // plane m
    const long long ic = base + (long long)(m + 2) * ms;
    wait(j + 2);
    const float* sl0 = slot(j);
    const float* sl1 = slot(j + 1);
    state_at(slot(j + 2), own, q[2]);
    T mom[3] = {0, 0, 0};
    if (upd_col) {
#pragma unroll
      for (int v = 0; v < NC; ++v) mom[v] = T(__ldg(a.in.m[v] + ic));
    }
    s_tau[ty + 1][tx + 1] = tau_m;
    if (htau_col || htau_row) {
      T kp, chi;
      s_tau[htau_col ? tid + 1 : 0][htau_col ? 0 : tid - TY + 1] = cell_tau<P, NDIM, GEOM, UNI>(
          a, sl0[FR * BOXP + hidx], sl0[FE * BOXP + hidx], hpx, hpy, m + 2, kp, chi);
    }
    tau_n = cell_tau<P, NDIM, GEOM, UNI>(a, sl1[FR * BOXP + own], sl1[FE * BOXP + own], px, py,
                                         m + 3, kp_n, chi_n);
    __syncthreads();
    if (s_abort) break;
    // plane j - 2 (= m - 2) was last read in iteration m - 2: its slot is free
    // (the proxy fence orders those reads before the TMA writes into it)
    if (tid == 0 && j + 3 <= jlast) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(j + 3);
    }

    // x face (tx - 1/2)
    {
      T um2[4], um1[4], u0[4], up1[4];
      const int r0 = (ty + 2) * BX + tx + xo;
      state_at(sl0, r0, um2);
      state_at(sl0, r0 + 1, um1);
      state_at(sl0, r0 + 2, u0);
      state_at(sl0, r0 + 3, up1);
      T tau = T(0.5) * (s_tau[ty + 1][tx] + s_tau[ty + 1][tx + 1]);
      T fx[4];
      int nf = face4<T, NC, 0, UNI>(um2, um1, u0, up1, IXC(0, px - 2), IXC(0, px - 1), IXC(0, px),
                                    HHI(0, px - 1), HLO(0, px), tau, T(1), inv_own, n2_own, fx);
      if (upd_col) cnt.fix += nf >> 1;
      if (ty <= TY - 2 && cy < Dm.n[1] && tx >= 1 && cx - 1 < Dm.n[0]) cnt.fix += nf & 1;
#pragma unroll
      for (int v = 0; v < NV; ++v) s_fx[v][ty][tx] = fx[v];
    }
    // y face (ty - 1/2)
    {
      T um2[4], um1[4], u0[4], up1[4];
      const int c0 = ty * BX + tx + 2 + xo;
      state_at(sl0, c0, um2);
      state_at(sl0, c0 + BX, um1);
      state_at(sl0, c0 + 2 * BX, u0);
      state_at(sl0, c0 + 3 * BX, up1);
      T tau = T(0.5) * (s_tau[ty][tx + 1] + s_tau[ty + 1][tx + 1]);
      T fy[4];
      int nf = face4<T, NC, 1, UNI>(um2, um1, u0, up1, IXC(1, py - 2), IXC(1, py - 1), IXC(1, py),
                                    HHI(1, py - 1), HLO(1, py), tau, T(1), inv_own, n2_own, fy);
      if (upd_col) cnt.fix += nf >> 1;
      if (ty >= 1 && cy - 1 < Dm.n[1] && tx <= TX - 2 && cx < Dm.n[0]) cnt.fix += nf & 1;
#pragma unroll
      for (int v = 0; v < NV; ++v) s_fy[v][ty][tx] = fy[v];
    }
    // march face m + 1/2 from the column registers
    T hiN[4];
    T inv_n = Ops<T>::rcp(q[1][0]);
    T n2_n = flux2<T, NC>(q[1]);
    {
      const int pm = m + 3;  // padded z of cell m + 1
      T loN[4];
      if constexpr (UNI) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          T hs = v < NV ? half_vanleer(q[1][v] - q[0][v], q[2][v] - q[1][v]) : T(0);
          loN[v] = q[1][v] - hs;
          hiN[v] = q[1][v] + hs;
        }
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
      if (upd_col && m + 1 < m1) cnt.fix += nf + nf2;  // the march states of cell m + 1
    }
    __syncthreads();

    // update of the own cell
    if (upd_col) {
      T dU[4] = {0, 0, 0, 0};
      {
        T alo = ALO(0, px), ahi = AHI(0, px);
#pragma unroll
        for (int v = 0; v < NV; ++v) dU[v] -= ahi * s_fx[v][ty][tx + 1] - alo * s_fx[v][ty][tx];
      }
      {
        T alo = ALO(1, py), ahi = AHI(1, py);
#pragma unroll
        for (int v = 0; v < NV; ++v) dU[v] -= ahi * s_fy[v][ty + 1][tx] - alo * s_fy[v][ty][tx];
      }
      {
        T alo = ALO(2, m + 2), ahi = AHI(2, m + 2);
#pragma unroll
        for (int v = 0; v < NV; ++v) dU[v] -= ahi * zhi[v] - alo * zlo[v];
      }
      const T (&u)[4] = q[0];
      T Us[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) Us[v] = u[v] + dtc * dU[v];
      if (Us[0] < a.efloor) {
        Us[0] = a.efloor;
        rare_add(RARE_EFLOOR);
      }
      const S rho_m = sl0[FR * BOXP + own], e_m = sl0[FE * BOXP + own];
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
      if (!queued) finish_cell<P, NDIM, NC, GEN>(a, ic, ci, Us, rho_m, e_m, kp_m, chi_m, mom, co, cnt);
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
    for (int j = jissued - R + 1 > 0 ? jissued - R + 1 : 0; j <= jissued; ++j)
      mbar_wait(&s_bar[j % R], uint32_t((j / R) & 1), kWaitLimit);
  }

  counters_flush<P>(a, cnt, s_red, tid);
}

}  // namespace m1
