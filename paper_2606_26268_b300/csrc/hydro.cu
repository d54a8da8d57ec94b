// hydro.cu -- instantiations and launcher of the gas step (hydro.cuh).
#include "hydro.cuh"
#include "hydro_launch.h"

namespace m1 {

template <class P, int NDIM, int NC>
cudaError_t hydro_launch(const void* args, cudaStream_t s) {
  const HydroArgs<P>& h = *static_cast<const HydroArgs<P>*>(args);
  const long long N = (long long)h.dim.n[0] * h.dim.n[1] * h.dim.n[2];
  const long long blocks = (N + 127) / 128;
  const int grid = int(blocks < 148 * 64 ? blocks : 148 * 64);
  hydro_kernel<P, NDIM, NC><<<grid, 128, 0, s>>>(h);
  return cudaGetLastError();
}

template <class P>
static HydroFn pick(int ndim, int nc) {
  if (ndim == 1 && nc == 1) return &hydro_launch<P, 1, 1>;
  if (ndim == 1 && nc == 2) return &hydro_launch<P, 1, 2>;
  if (ndim == 1 && nc == 3) return &hydro_launch<P, 1, 3>;
  if (ndim == 2 && nc == 2) return &hydro_launch<P, 2, 2>;
  if (ndim == 2 && nc == 3) return &hydro_launch<P, 2, 3>;
  if (ndim == 3 && nc == 3) return &hydro_launch<P, 3, 3>;
  return nullptr;
}

HydroFn select_hydro(bool split, int ndim, int nc) {
  return split ? pick<Split>(ndim, nc) : pick<Fp64>(ndim, nc);
}

}  // namespace m1
