// queue_cell.cuh -- per-cell work of the queue pass: the cells the step
// kernel left for the Newton iteration, optionally started from the learned
// guess.
#pragma once
#include "m1_cell.cuh"
#include "mlp.cuh"

namespace m1 {

// A cell the step kernel queued: (E*, F*) and the single solve's T^{n+1}
// (T1, in the stash's e) left in the stash buffer, gas state from the input
// buffer, opacities at (rho, T^n).
template <class P>
struct QueuedCell {
  using S = typename P::S;
  using T = typename P::T;
  long long ic;
  int ci[3];
  T Us[4], mom[3], kp, chi;
  S rho, e, T1;
};

template <class P, int NC>
__device__ __forceinline__ void queue_load(const StepArgs<P>& a, long long ic, QueuedCell<P>& c) {
  using T = typename P::T;
  const StepDims& Dm = a.dim;
  c.ic = ic;
  long long r = ic;
  c.ci[0] = int(r % Dm.pn[0]) - Dm.g[0];
  r /= Dm.pn[0];
  c.ci[1] = int(r % Dm.pn[1]) - Dm.g[1];
  c.ci[2] = int(r / Dm.pn[1]) - Dm.g[2];
  c.Us[0] = T(a.stash.E[ic]);
  c.T1 = a.stash.e[ic];
  c.Us[1] = c.Us[2] = c.Us[3] = T(0);
  c.mom[0] = c.mom[1] = c.mom[2] = T(0);
#pragma unroll
  for (int v = 0; v < NC; ++v) {
    c.Us[1 + v] = T(a.stash.F[v][ic]);
    c.mom[v] = T(a.in.m[v][ic]);
  }
  c.rho = a.rho[ic];
  c.e = a.in.e[ic];
  T rr = T(c.rho);
  if constexpr (sizeof(T) == 8)
    opacity(a.opac, rr, T(c.e) / (rr * T(a.cp.cvfac)), c.kp, c.chi);
  else
    opacity_re(a.opac, rr, T(c.e), c.kp, c.chi);
}

// The Newton iteration continued from the single solve's T1, or from the
// learned guess T0 when that leaves the smaller residual, then the common
// end of the step.
template <class P, int NDIM, int NC>
__device__ __forceinline__ void queue_solve(const StepArgs<P>& a, QueuedCell<P>& c, float T0,
                                            Counters& cnt) {
  const auto co =
      couple_cell<P>(a, c.ic, c.rho, c.e, c.kp, c.Us[0], T0, false, double(c.T1));
  finish_cell<P, NDIM, NC>(a, c.ic, c.ci, c.Us, c.rho, c.e, c.kp, c.chi, c.mom, co, cnt);
}

// Starting temperature from the network output g = log(T/T^n).
__device__ __forceinline__ float guess_temperature(float Tn, float g) {
  return Tn * ex2_approx(fminf(fmaxf(g, -20.f), 20.f) * 1.44269504088896341f);
}

}  // namespace m1
