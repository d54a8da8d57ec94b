// hydro.cu -- instantiations and launcher of the gas step (hydro.cuh).
#include "hydro.cuh"
#include "hydro_launch.h"

namespace m1 {

// CTA tiles: 32 x 8 cells marching 16 planes along z (3D), 32 x 8 (2D), 128
// cells (1D).
template <class P, int NDIM, int NC, bool UNI>
cudaError_t hydro_launch(const void* args, cudaStream_t s) {
  const HydroArgs<P>& h = *static_cast<const HydroArgs<P>*>(args);
  const int* n = h.dim.n;
  if constexpr (NDIM == 3) {
    dim3 grid((n[0] + 31) / 32, (n[1] + 7) / 8, (n[2] + 15) / 16);
    hydro_kernel<P, 3, NC, 32, 8, UNI><<<grid, dim3(32, 8), 0, s>>>(h);
  } else if constexpr (NDIM == 2) {
    dim3 grid((n[0] + 31) / 32, (n[1] + 7) / 8, 1);
    hydro_kernel<P, 2, NC, 32, 8, UNI><<<grid, dim3(32, 8), 0, s>>>(h);
  } else {
    hydro_kernel<P, 1, NC, 128, 1, UNI><<<(n[0] + 127) / 128, dim3(128, 1), 0, s>>>(h);
  }
  return cudaGetLastError();
}

template <class P, bool UNI>
static HydroFn pick(int ndim, int nc) {
  if (ndim == 1 && nc == 1) return &hydro_launch<P, 1, 1, UNI>;
  if (ndim == 1 && nc == 2) return &hydro_launch<P, 1, 2, UNI>;
  if (ndim == 1 && nc == 3) return &hydro_launch<P, 1, 3, UNI>;
  if (ndim == 2 && nc == 2) return &hydro_launch<P, 2, 2, UNI>;
  if (ndim == 2 && nc == 3) return &hydro_launch<P, 2, 3, UNI>;
  if (ndim == 3 && nc == 3) return &hydro_launch<P, 3, 3, UNI>;
  return nullptr;
}

HydroFn select_hydro(bool split, int ndim, int nc, bool uniform) {
  if (uniform) return split ? pick<Split, true>(ndim, nc) : pick<Fp64, true>(ndim, nc);
  return split ? pick<Split, false>(ndim, nc) : pick<Fp64, false>(ndim, nc);
}

template <class P, int NDIM, int NC>
cudaError_t gas_cfl_launch(const void* args, cudaStream_t s) {
  const GasCflArgs<P>& g = *static_cast<const GasCflArgs<P>*>(args);
  const long long N = (long long)g.dim.n[0] * g.dim.n[1] * g.dim.n[2];
  const long long blocks = (N + 255) / 256;
  const int grid = int(blocks < 148 * 8 ? blocks : 148 * 8);
  gas_cfl_kernel<P, NDIM, NC><<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

template <class P>
static HydroFn pick_cfl(int ndim, int nc) {
  if (ndim == 1 && nc == 1) return &gas_cfl_launch<P, 1, 1>;
  if (ndim == 1 && nc == 2) return &gas_cfl_launch<P, 1, 2>;
  if (ndim == 1 && nc == 3) return &gas_cfl_launch<P, 1, 3>;
  if (ndim == 2 && nc == 2) return &gas_cfl_launch<P, 2, 2>;
  if (ndim == 2 && nc == 3) return &gas_cfl_launch<P, 2, 3>;
  if (ndim == 3 && nc == 3) return &gas_cfl_launch<P, 3, 3>;
  return nullptr;
}

HydroFn select_gas_cfl(bool split, int ndim, int nc) {
  return split ? pick_cfl<Split>(ndim, nc) : pick_cfl<Fp64>(ndim, nc);
}

}  // namespace m1
