// step_launch.cuh -- launch configuration of the step kernel.
#pragma once
#include "m1_step.cuh"
#include "step_launch.h"

namespace m1 {

// 3D: 32 x 8 thread tiles (31 x 7 updated columns) marching 32 planes;
// 2D: 128-thread rows (127 updated columns) marching 64 rows; 1D: 128 cells.
template <class P, int NDIM, int GEOM, int NC>
cudaError_t launch_step(const void* vargs, cudaStream_t s) {
  StepArgs<P> a = *static_cast<const StepArgs<P>*>(vargs);
  const int* n = a.dim.n;
  if constexpr (NDIM == 3) {
    constexpr int TX = 32, TY = 8;
    a.chunk = n[2] < 32 ? n[2] : 32;
    dim3 grid((n[0] + TX - 2) / (TX - 1), (n[1] + TY - 2) / (TY - 1), (n[2] + a.chunk - 1) / a.chunk);
    step_kernel<P, 3, GEOM, NC, TX, TY><<<grid, dim3(TX, TY), 0, s>>>(a);
  } else if constexpr (NDIM == 2) {
    constexpr int TX = 128;
    a.chunk = n[1] < 64 ? n[1] : 64;
    dim3 grid((n[0] + TX - 2) / (TX - 1), (n[1] + a.chunk - 1) / a.chunk);
    step_kernel<P, 2, GEOM, NC, TX, 1><<<grid, dim3(TX, 1), 0, s>>>(a);
  } else {
    constexpr int TX = 128;
    a.chunk = 1;
    dim3 grid((n[0] + TX - 2) / (TX - 1));
    step_kernel<P, 1, GEOM, NC, TX, 1><<<grid, dim3(TX, 1), 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace m1
