// queue_cell.cuh -- per-cell work of the queue pass (cells the step kernel
// left for the Newton iteration, optionally started from the learned guess)
// and the block reduction of the step counters.
#pragma once
#include "m1_cell.cuh"
#include "mlp.cuh"

namespace m1 {

// One queued cell: (E*, F*) left in the output buffer by the step kernel,
// gas state from the input buffer, opacities at (rho, T^n), the learned guess
// T0 = T^n exp(net(x1, x2)) when the network is set and the first linearised
// change exceeds the gate (else T^n), then the common end of the step.
template <class P, int NDIM, int NC>
__device__ __forceinline__ void queue_cell(const StepArgs<P>& a, long long ic,
                                           const float* s_w, Counters& cnt) {
  using S = typename P::S;
  using T = typename P::T;
  const StepDims& Dm = a.dim;
  long long r = ic;
  int ci[3];
  ci[0] = int(r % Dm.pn[0]) - Dm.g[0];
  r /= Dm.pn[0];
  ci[1] = int(r % Dm.pn[1]) - Dm.g[1];
  ci[2] = int(r / Dm.pn[1]) - Dm.g[2];
  T Us[4] = {T(a.out.E[ic]), 0, 0, 0};
#pragma unroll
  for (int v = 0; v < NC; ++v) Us[1 + v] = T(a.out.F[v][ic]);
  T mom[3] = {0, 0, 0};
#pragma unroll
  for (int v = 0; v < NC; ++v) mom[v] = T(a.in.m[v][ic]);
  const S rho = a.rho[ic], e = a.in.e[ic];
  T kp, chi;
  {
    T rr = T(rho);
    T Temp;
    if constexpr (sizeof(T) == 8)
      Temp = T(e) / (rr * T(a.cp.cvfac));
    else
      Temp = T(e) * rcp_approx(rr * a.cp.f_cvfac);
    opacity(a.opac, rr, Temp, kp, chi);
  }
  float T0 = 0.f;  // T^n
  if (a.mlp_w) {
    float x1, x2, lin, Tn;
    coupling_features(a.cp, float(rho), float(e), float(kp), float(Us[0]), x1, x2, lin, Tn);
    if (lin > a.mlp_gate) {
      const float guess = mlp_forward(s_w, x1, x2);
      T0 = Tn * ex2_approx(fminf(fmaxf(guess, -20.f), 20.f) * 1.44269504088896341f);
    }
  }
  const CoupleOut co = couple_cell<P>(a, rho, e, kp, Us[0], T0, false);
  finish_cell<P, NDIM, NC>(a, ic, ci, Us, rho, e, kp, chi, mom, co, cnt);
}

}  // namespace m1
