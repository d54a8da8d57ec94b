// hydro.cuh -- the gas step that precedes the radiation transport in every
// (sub)step when the gas is evolved (Sect. 2.4 orders a substep as gas step,
// radiation transport, radiation sources).  A Godunov step of the Euler
// equations on Cartesian grids: PLM with the van Leer limiter on the
// primitive variables (rho, v, p), the HLL flux with the Davis signal speeds
// S_L = min(v_L - c_L, v_R - c_R), S_R = max(v_L + c_L, v_R + c_R), and the
// flux divergence of (rho, m, E_gas).
//
// The kernel reads the padded input buffer, whose ghost cells the previous
// step left up to date, and computes every face flux once.  The result
// (rho*, m*, e*) goes to separate arrays: the radiation kernel that
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
  T inv_gm1;         // 1 / (Gamma - 1)
  T uni_inv[3];      // 1 / h per direction (uniform grids)
  T bcT[3][2];       // gas temperature of the fixed and LTE sides
  int* status;       // status word (the debug build's index checks)
};

// Conserved state and physical flux along D of a primitive state.
template <class T, int NC, int D>
__device__ __forceinline__ void gas_flux(const T (&w)[5], T inv_gm1, T (&U)[5], T (&f)[5]) {
  const T r = w[0], p = w[4], vd = w[1 + D];
  T v2 = T(0);
#pragma unroll
  for (int v = 0; v < NC; ++v) v2 += w[1 + v] * w[1 + v];
  const T Eg = p * inv_gm1 + T(0.5) * r * v2;
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

// HLL flux of the face between the cells of primitive states w1 and w2 along
// D, with their outer neighbours w0 and w3: ix0..ix2 the inverse centre
// distances of (w0, w1), (w1, w2), (w2, w3), hh and hl the offsets of the face
// from the centres of w1 and w2.
// UNI: uniform spacing; the faces sit half a cell from the centres and the
// limited half slope is d0 d1 / (d0 + d1) of the raw differences (the tables
// are not read).
template <class T, int NC, int D, bool UNI = false>
__device__ __forceinline__ void gas_riemann(const T (&w0)[5], const T (&w1)[5], const T (&w2)[5],
                                            const T (&w3)[5], T ix0, T ix1, T ix2, T hh, T hl,
                                            T gamma, T inv_gm1, T (&out)[5]) {
  T wl[5], wr[5];
  auto half = [](T a, T b) {
    const T p = a * b;
    return p > T(0) ? Ops<T>::div(p, a + b) : T(0);
  };
  if constexpr (UNI && sizeof(T) == 4) {
    // components (0, 1) and (2, 3) on packed FP32 pairs, 4 alone
#pragma unroll
    for (int h = 0; h < 4; h += 2) {
      const float2 c0 = make_float2(w0[h], w0[h + 1]), c1 = make_float2(w1[h], w1[h + 1]);
      const float2 c2 = make_float2(w2[h], w2[h + 1]), c3 = make_float2(w3[h], w3[h + 1]);
      const float2 d0 = f2_sub(c1, c0), d1 = f2_sub(c2, c1), d2 = f2_sub(c3, c2);
      const float2 pa = f2_mul(d0, d1), sa = f2_add(d0, d1);
      const float2 pb = f2_mul(d1, d2), sb = f2_add(d1, d2);
      float2 ha = f2_mul(pa, make_float2(rcp_approx(sa.x), rcp_approx(sa.y)));
      float2 hb = f2_mul(pb, make_float2(rcp_approx(sb.x), rcp_approx(sb.y)));
      ha.x = pa.x > 0.f ? ha.x : 0.f;
      ha.y = pa.y > 0.f ? ha.y : 0.f;
      hb.x = pb.x > 0.f ? hb.x : 0.f;
      hb.y = pb.y > 0.f ? hb.y : 0.f;
      const float2 l = f2_add(c1, ha), r = f2_sub(c2, hb);
      wl[h] = l.x;
      wl[h + 1] = l.y;
      wr[h] = r.x;
      wr[h + 1] = r.y;
    }
    wl[4] = w1[4] + half(w1[4] - w0[4], w2[4] - w1[4]);
    wr[4] = w2[4] - half(w2[4] - w1[4], w3[4] - w2[4]);
  } else if constexpr (UNI) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const T d0 = w1[q] - w0[q], d1 = w2[q] - w1[q], d2 = w3[q] - w2[q];
      wl[q] = w1[q] + half(d0, d1);
      wr[q] = w2[q] - half(d1, d2);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const T d0 = (w1[q] - w0[q]) * ix0, d1 = (w2[q] - w1[q]) * ix1, d2 = (w3[q] - w2[q]) * ix2;
      wl[q] = w1[q] + vanleer(d0, d1) * hh;
      wr[q] = w2[q] + vanleer(d1, d2) * hl;
    }
  }
  T UL[5], UR[5], fL[5], fR[5];
  gas_flux<T, NC, D>(wl, inv_gm1, UL, fL);
  gas_flux<T, NC, D>(wr, inv_gm1, UR, fR);
  const T cl = Ops<T>::sqrt_(Ops<T>::div(gamma * wl[4], wl[0]));
  const T cr = Ops<T>::sqrt_(Ops<T>::div(gamma * wr[4], wr[0]));
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
    if constexpr (sizeof(T) == 4) {  // components (0, 1), (2, 3) packed, 4 alone
      const float2 SR = make_float2(sr, sr), MSL = make_float2(-sl, -sl);
      const float2 SLSR = make_float2(sl * sr, sl * sr), INV = make_float2(inv, inv);
#pragma unroll
      for (int h = 0; h < 4; h += 2) {
        const float2 du = f2_sub(make_float2(UR[h], UR[h + 1]), make_float2(UL[h], UL[h + 1]));
        float2 acc = f2_mul(MSL, make_float2(fR[h], fR[h + 1]));
        acc = f2_fma(SLSR, du, acc);
        acc = f2_fma(SR, make_float2(fL[h], fL[h + 1]), acc);
        acc = f2_mul(acc, INV);
        out[h] = acc.x;
        out[h + 1] = acc.y;
      }
      out[4] = (sr * fL[4] - sl * fR[4] + sl * sr * (UR[4] - UL[4])) * inv;
    } else {
#pragma unroll
      for (int q = 0; q < 5; ++q) out[q] = (sr * fL[q] - sl * fR[q] + sl * sr * (UR[q] - UL[q])) * inv;
    }
  }
}

template <class T>
__device__ __forceinline__ T gtab(const GeomDev<T>& G, int d, int slot, int ip) {
  return __ldg(G.tab[d] + slot * G.len[d] + ip);
}

// The gas step.  A CTA of TX x TY threads owns a TX x TY tile of cells in x
// (and y) and marches along z (3D).  Per z plane the CTA stages the
// primitive states of the tile and a 2-cell halo in shared memory; each
// thread computes the flux of its cell's lower x (and y) face, the threads of
// the last column (row) also the upper tile face, and every face is computed
// once.  The z faces come from the column's states held in registers, the
// upper face of one plane being the lower face of the next.
template <class P, int NDIM, int NC, int TX, int TY, bool UNI>
__global__ void __launch_bounds__(TX * TY, (TX * TY >= 256 && P::kSplit) ? 3 : 1) hydro_kernel(const __grid_constant__ HydroArgs<P> h) {
  using S = typename P::S;
  using T = typename P::T;
  constexpr bool HY = NDIM >= 2, HZ = NDIM >= 3;
  constexpr int SX = TX + 4, SY = HY ? TY + 4 : 1, OY = HY ? 2 : 0;
  constexpr int NT = TX * TY;
  __shared__ T s_w[5][SY][SX];
  __shared__ T s_fx[5][TY][TX + 1];
  __shared__ T s_fy[5][HY ? TY + 1 : 1][TX];
  // split precision: the tile's own input (rho, m, e) staged with the plane,
  // so that the update reads it from shared memory (FP64 reads it again)
  constexpr bool SU = P::kSplit;
  // (two copies: the update of plane z reads one while the next plane is
  // staged into the other)
  __shared__ T s_u[SU ? 2 : 1][SU ? 5 : 1][SU ? TY : 1][SU ? TX : 1];
  int ub = 0;

  const StepDims& Dm = h.dim;
  const GeomDev<T>& G = h.geo;
  const int tx = threadIdx.x, ty = HY ? threadIdx.y : 0;
  const int tid = tx + TX * ty;
  const int x0 = blockIdx.x * TX, y0 = HY ? blockIdx.y * TY : 0;
  const int cx = x0 + tx, cy = y0 + ty;
  const bool upd = cx < Dm.n[0] && (!HY || cy < Dm.n[1]);
  const int chunk = HZ ? (Dm.n[2] + gridDim.z - 1) / gridDim.z : 1;
  const int z0 = HZ ? blockIdx.z * chunk : 0;
  const int z1 = HZ ? min(z0 + chunk, Dm.n[2]) : 1;
  // padded coordinates of the own cell (clamped inside the array for the
  // threads past the grid's edge, which update nothing)
  const int px = min(cx, Dm.n[0] - 1) + Dm.g[0];
  const int py = HY ? min(cy, Dm.n[1] - 1) + Dm.g[1] : 0;
  const long long col = px + Dm.sy * (long long)py;
  const long long sz = Dm.sz;
  const int gz = Dm.g[2];

  auto prim = [&](long long ip, T (&w)[5]) {
    const T r = T(__ldg(h.rho + ip));
    const T ir = Ops<T>::rcp(r);
    w[0] = r;
#pragma unroll
    for (int v = 0; v < 3; ++v) w[1 + v] = v < NC ? T(__ldg(h.m[v] + ip)) * ir : T(0);
    w[4] = (h.gamma - T(1)) * T(__ldg(h.e + ip));
  };

  // the own column's states at z - 2 .. z + 2, and the flux of the face below
  T wz[5][5];
  T fzlo[5] = {0, 0, 0, 0, 0};
  if constexpr (HZ) {
#pragma unroll
    for (int k = 0; k < 4; ++k) prim(col + (long long)(z0 - 2 + k + gz) * sz, wz[k]);
    const int pz = z0 + gz;
    gas_riemann<T, NC, 2, UNI>(wz[0], wz[1], wz[2], wz[3], gtab(G, 2, TAB_IDXC, pz - 2),
                          gtab(G, 2, TAB_IDXC, pz - 1), gtab(G, 2, TAB_IDXC, pz),
                          gtab(G, 2, TAB_HHI, pz - 1), gtab(G, 2, TAB_HLO, pz), h.gamma, h.inv_gm1, fzlo);
  }

  // The plane (tile plus a 2-cell halo, coordinates clamped to the padded
  // array) is loaded into registers one plane ahead, so that its loads are in
  // flight while the previous plane's faces are computed, and staged in
  // shared memory as primitive states.
  constexpr int KS = (SX * SY + NT - 1) / NT;  // staged cells per thread
  S pre[KS][5];
  auto load_plane = [&](int z) {
    const long long zoff = (long long)(z + gz) * sz;
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      const int k = tid + kk * NT;
      if (k < SX * SY) {
        const int iy = k / SX, ix = k - iy * SX;
        const int gx = min(max(x0 - 2 + ix + Dm.g[0], 0), Dm.n[0] + 2 * Dm.g[0] - 1);
        const int gy = HY ? min(max(y0 - OY + iy + Dm.g[1], 0), Dm.n[1] + 2 * Dm.g[1] - 1) : 0;
        const long long ip = gx + Dm.sy * (long long)gy + zoff;
        pre[kk][0] = __ldg(h.rho + ip);
#pragma unroll
        for (int v = 0; v < 3; ++v) pre[kk][1 + v] = v < NC ? __ldg(h.m[v] + ip) : S(0);
        pre[kk][4] = __ldg(h.e + ip);
      }
    }
  };
  auto store_plane = [&]() {
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
      const int k = tid + kk * NT;
      if (k < SX * SY) {
        const int iy = k / SX, ix = k - iy * SX;
        const T r = T(pre[kk][0]);
        const T ir = Ops<T>::rcp(r);
        s_w[0][iy][ix] = r;
#pragma unroll
        for (int v = 0; v < 3; ++v) s_w[1 + v][iy][ix] = T(pre[kk][1 + v]) * ir;
        s_w[4][iy][ix] = (h.gamma - T(1)) * T(pre[kk][4]);
        if constexpr (SU) {
          const int ux = ix - 2, uy = iy - OY;
          if (ux >= 0 && ux < TX && uy >= 0 && uy < TY) {
#pragma unroll
            for (int q = 0; q < 5; ++q) s_u[ub][q][uy][ux] = T(pre[kk][q]);
          }
        }
      }
    }
  };
  // the own column two planes above the current one, loaded an iteration
  // ahead
  S zpre[5];
  auto load_col = [&](int zz) {
    const long long ip = col + (long long)(zz + gz) * sz;
    zpre[0] = __ldg(h.rho + ip);
#pragma unroll
    for (int v = 0; v < 3; ++v) zpre[1 + v] = v < NC ? __ldg(h.m[v] + ip) : S(0);
    zpre[4] = __ldg(h.e + ip);
  };
  if constexpr (HZ) load_col(z0 + 2);
  load_plane(z0);

  for (int z = z0; z < z1; ++z) {
    const long long zoff = (long long)(z + gz) * sz;
    store_plane();
    if constexpr (HZ) {
      const T r = T(zpre[0]);
      const T ir = Ops<T>::rcp(r);
      wz[4][0] = r;
#pragma unroll
      for (int v = 0; v < 3; ++v) wz[4][1 + v] = v < NC ? T(zpre[1 + v]) * ir : T(0);
      wz[4][4] = (h.gamma - T(1)) * T(zpre[4]);
      if (z + 1 < z1) load_col(z + 3);
    }
    __syncthreads();
    if (z + 1 < z1) load_plane(z + 1);
    // faces of the tile directions: the lower x (and y) face of the own cell;
    // the tile's upper faces (one per row and per column) go to the first
    // threads of the CTA, so that they occupy as few warps as possible
    auto xface = [&](int row, int c, T (&f)[5]) {  // face between tile columns c - 1 and c
      T a0[5], a1[5], a2[5], a3[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        a0[q] = s_w[q][row + OY][c];
        a1[q] = s_w[q][row + OY][c + 1];
        a2[q] = s_w[q][row + OY][c + 2];
        a3[q] = s_w[q][row + OY][c + 3];
      }
      const int pc = min(x0 + c, Dm.n[0]) + Dm.g[0];
      gas_riemann<T, NC, 0, UNI>(a0, a1, a2, a3, gtab(G, 0, TAB_IDXC, pc - 2),
                            gtab(G, 0, TAB_IDXC, pc - 1), gtab(G, 0, TAB_IDXC, pc),
                            gtab(G, 0, TAB_HHI, pc - 1), gtab(G, 0, TAB_HLO, pc), h.gamma,
                            h.inv_gm1, f);
    };
    auto yface = [&](int r, int cl, T (&f)[5]) {  // face between tile rows r - 1 and r
      T a0[5], a1[5], a2[5], a3[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        a0[q] = s_w[q][r][cl + 2];
        a1[q] = s_w[q][r + 1][cl + 2];
        a2[q] = s_w[q][r + 2][cl + 2];
        a3[q] = s_w[q][r + 3][cl + 2];
      }
      const int pr = min(y0 + r, Dm.n[1]) + Dm.g[1];
      gas_riemann<T, NC, 1, UNI>(a0, a1, a2, a3, gtab(G, 1, TAB_IDXC, pr - 2),
                            gtab(G, 1, TAB_IDXC, pr - 1), gtab(G, 1, TAB_IDXC, pr),
                            gtab(G, 1, TAB_HHI, pr - 1), gtab(G, 1, TAB_HLO, pr), h.gamma,
                            h.inv_gm1, f);
    };
    {
      T f[5];
      xface(ty, tx, f);
#pragma unroll
      for (int q = 0; q < 5; ++q) s_fx[q][ty][tx] = f[q];
      if constexpr (HY) {
        yface(ty, tx, f);
#pragma unroll
        for (int q = 0; q < 5; ++q) s_fy[q][ty][tx] = f[q];
      }
      if (tid < TY) {
        xface(tid, TX, f);
#pragma unroll
        for (int q = 0; q < 5; ++q) s_fx[q][tid][TX] = f[q];
      }
      if constexpr (HY) {
        if (tid >= TY && tid < TY + TX) {
          yface(TY, tid - TY, f);
#pragma unroll
          for (int q = 0; q < 5; ++q) s_fy[q][TY][tid - TY] = f[q];
        }
      }
    }
    // z face above the own cell
    T fzhi[5] = {0, 0, 0, 0, 0};
    if constexpr (HZ) {
      const int pz = z + 1 + gz;
      gas_riemann<T, NC, 2, UNI>(wz[1], wz[2], wz[3], wz[4], gtab(G, 2, TAB_IDXC, pz - 2),
                            gtab(G, 2, TAB_IDXC, pz - 1), gtab(G, 2, TAB_IDXC, pz),
                            gtab(G, 2, TAB_HHI, pz - 1), gtab(G, 2, TAB_HLO, pz), h.gamma, h.inv_gm1, fzhi);
    }
    __syncthreads();
    if (upd) {
      const long long ic = col + zoff;
      T U[5];
      {
        const T r = SU ? s_u[ub][0][ty][tx] : T(__ldg(h.rho + ic));
        U[0] = r;
        T ke = T(0);
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          U[1 + v] = v < NC ? (SU ? s_u[ub][1 + v][ty][tx] : T(__ldg(h.m[v] + ic))) : T(0);
          ke += U[1 + v] * U[1 + v];
        }
        U[4] = (SU ? s_u[ub][4][ty][tx] : T(__ldg(h.e + ic))) + T(0.5) * ke * Ops<T>::rcp(r);
      }
      {
        const T ih = UNI ? h.uni_inv[0] : gtab(G, 0, TAB_ALO, px);
#pragma unroll
        for (int q = 0; q < 5; ++q) U[q] -= h.dt * ih * (s_fx[q][ty][tx + 1] - s_fx[q][ty][tx]);
      }
      if constexpr (HY) {
        const T ih = UNI ? h.uni_inv[1] : gtab(G, 1, TAB_ALO, py);
#pragma unroll
        for (int q = 0; q < 5; ++q) U[q] -= h.dt * ih * (s_fy[q][ty + 1][tx] - s_fy[q][ty][tx]);
      }
      if constexpr (HZ) {
        const T ih = UNI ? h.uni_inv[2] : gtab(G, 2, TAB_ALO, z + gz);
#pragma unroll
        for (int q = 0; q < 5; ++q) U[q] -= h.dt * ih * (fzhi[q] - fzlo[q]);
      }
      T k2 = T(0);
#pragma unroll
      for (int v = 0; v < NC; ++v) k2 += U[1 + v] * U[1 + v];
      const T en = U[4] - T(0.5) * k2 * Ops<T>::rcp(U[0]);
      // (the debug build skips the stores of a cell whose index fails its check)
      const bool store_ok = index_ok((long long)ic, padded_cells(Dm), h.status);
      if (store_ok) {
        h.rho_out[ic] = S(U[0]);
        h.e_out[ic] = S(en);
#pragma unroll
        for (int v = 0; v < NC; ++v) h.m_out[v][ic] = S(U[1 + v]);
      }
      // ghost copies of rho* and e* (the optical depths of the radiation
      // step read them): wrapped, edge or mirrored; the fixed and LTE sides
      // take the edge density and e = C_v T_b
      const int ci[3] = {cx, cy, z};
#pragma unroll
      for (int d = 0; d < NDIM; ++d) {
        const int n = Dm.n[d];
        const int i = ci[d];
        if (!store_ok || (i >= 2 && i < n - 2)) continue;
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
          if (!index_ok(ig, padded_cells(Dm), h.status)) continue;
          h.rho_out[ig] = S(U[0]);
          const bool held = bc == BC_FIXED || bc == BC_LTE;
          h.e_out[ig] = S(held ? h.cvfac * U[0] * h.bcT[d][lo ? 0 : 1] : en);
        }
      }
    }
    if constexpr (HZ) {
#pragma unroll
      for (int q = 0; q < 5; ++q) fzlo[q] = fzhi[q];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int q = 0; q < 5; ++q) wz[k][q] = wz[k + 1][q];
    }
    // No barrier here: the next plane's staging writes s_w, which the faces
    // of this plane read before the second barrier, and the other copy of
    // s_u; its faces write s_fx, s_fy only after its first barrier, which
    // every thread reaches after this update.
    if constexpr (SU) ub ^= 1;
  }
}

// The CFL step with the gas: the largest over cells of
// sum_d max(chat, |v_d| + c_s) / h_d (c_s = sqrt(Gamma (Gamma - 1) e / rho)),
// reduced into *out as the bits of a non-negative double (whose order is
// the order of the bit patterns).  Computed in the precision of the
// transport (FP32 for the split form, whose step only needs the CFL bound
// to rounding; FP64 for the FP64 form), with one reciprocal of rho per cell.
template <class P>
struct GasCflArgs {
  using S = typename P::S;
  using T = typename P::T;
  StepDims dim;
  GeomDev<T> geo;
  const S* rho;
  const S* e;
  const S* m[3];
  double chat, gamma;
  unsigned long long* out;
};

template <class P, int NDIM, int NC>
__global__ void __launch_bounds__(256) gas_cfl_kernel(const __grid_constant__ GasCflArgs<P> g) {
  using T = typename P::T;
  const StepDims& Dm = g.dim;
  const long long N = (long long)Dm.n[0] * Dm.n[1] * Dm.n[2];
  const T chat = T(g.chat), gg1 = T(g.gamma * (g.gamma - 1.0));
  T worst = T(0);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N;
       q += (long long)gridDim.x * blockDim.x) {
    long long r = q;
    const int i = int(r % Dm.n[0]);
    r /= Dm.n[0];
    const int j = int(r % Dm.n[1]);
    const int k = int(r / Dm.n[1]);
    const int pc[3] = {i + Dm.g[0], j + Dm.g[1], k + Dm.g[2]};
    const long long ic = pc[0] + Dm.sy * pc[1] + Dm.sz * pc[2];
    const T ir = T(1) / T(g.rho[ic]);
    const T cs = Ops<T>::sqrt_(gg1 * T(g.e[ic]) * ir);
    T sum = T(0);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const T vd = T(g.m[d][ic]) * ir;
      const T v = (vd < T(0) ? -vd : vd) + cs;
      const T w = g.geo.tab[d][TAB_WID * g.geo.len[d] + pc[d]];
      sum += (v > chat ? v : chat) / w;
    }
    worst = sum > worst ? sum : worst;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const T o = __shfl_down_sync(0xffffffffu, worst, off);
    worst = o > worst ? o : worst;
  }
  if ((threadIdx.x & 31) == 0)
    atomicMax(g.out, static_cast<unsigned long long>(__double_as_longlong(double(worst))));
}

}  // namespace m1
