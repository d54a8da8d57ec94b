// step_launch.cuh -- launch configurations of the step kernel.
#pragma once
#include <cstring>

#include "m1_step.cuh"
#include "m1_step_tma.cuh"
#include "m1_step_tma2.cuh"
#include "m1_strip2d.cuh"
#include "step_launch.h"

namespace m1 {

template <class P, int NDIM, int GEOM, int NC, bool UNI, int TX, int TY, int MINB, bool GEN>
cudaError_t launch_shape(StepArgs<P> a, cudaStream_t s, int chunk) {
  const int* n = a.dim.n;
  if constexpr (NDIM == 3) {
    a.chunk = chunk > 0 ? chunk : 32;
    if (a.chunk > n[2]) a.chunk = n[2];
    dim3 grid((n[0] + TX - 2) / (TX - 1), (n[1] + TY - 2) / (TY - 1), (n[2] + a.chunk - 1) / a.chunk);
    step_kernel<P, 3, GEOM, NC, UNI, TX, TY, MINB, GEN><<<grid, dim3(TX, TY), 0, s>>>(a);
  } else if constexpr (NDIM == 2) {
    a.chunk = chunk > 0 ? chunk : 64;
    if (a.chunk > n[1]) a.chunk = n[1];
    dim3 grid((n[0] + TX - 2) / (TX - 1), (n[1] + a.chunk - 1) / a.chunk);
    step_kernel<P, 2, GEOM, NC, UNI, TX, 1, MINB, GEN><<<grid, dim3(TX, 1), 0, s>>>(a);
  } else {
    a.chunk = 1;
    dim3 grid((n[0] + TX - 2) / (TX - 1));
    step_kernel<P, 1, GEOM, NC, UNI, TX, 1, MINB, GEN><<<grid, dim3(TX, 1), 0, s>>>(a);
  }
  return cudaGetLastError();
}

// One warp per strip of 31 updated columns of a 2D Cartesian grid.
template <class P, int NC, bool UNI, int MINB>
cudaError_t launch_strip2d(StepArgs<P> a, cudaStream_t s, int chunk) {
  const int* n = a.dim.n;
  a.chunk = chunk > 0 ? chunk : 64;
  if (a.chunk > n[1]) a.chunk = n[1];
  dim3 grid((n[0] + 30) / 31, (n[1] + a.chunk - 1) / a.chunk);
  step_strip2d_kernel<P, NC, UNI, MINB><<<grid, 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <class P, int NC, bool UNI, int TX, int TY, int MINB, bool GEN>
cudaError_t launch_tma(StepArgs<P> a, const void* tma, cudaStream_t s, int chunk) {
  if (!tma) return cudaErrorInvalidValue;
  const int* n = a.dim.n;
  a.chunk = chunk > 0 ? chunk : 32;
  if (a.chunk > n[2]) a.chunk = n[2];
  constexpr size_t smem = tma_smem_bytes<NC, TX, TY>();
  auto kern = step_tma_kernel<P, NC, UNI, TX, TY, MINB, GEN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  TmaMaps maps;
  std::memcpy(&maps, tma, sizeof(maps));
  dim3 grid((n[0] + TX - 2) / (TX - 1), (n[1] + TY - 2) / (TY - 1), (n[2] + a.chunk - 1) / a.chunk);
  kern<<<grid, dim3(TX, TY), smem, s>>>(a, maps);
  return cudaGetLastError();
}

template <class P, int NC, bool UNI, int TX, int TY, int MINB, bool GEN, int GEOM = kCart,
          bool UYZ = false>
cudaError_t launch_tma2(StepArgs<P> a, const void* tma, cudaStream_t s, int chunk) {
  if (!tma) return cudaErrorInvalidValue;
  const int* n = a.dim.n;
  a.chunk = chunk > 0 ? chunk : 32;
  if (a.chunk > n[2]) a.chunk = n[2];
  constexpr size_t smem = tma2_smem_bytes<NC, TX, TY>();
  auto kern = step_tma2_kernel<P, NC, UNI, TX, TY, MINB, GEN, GEOM, UYZ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  TmaMaps maps;
  std::memcpy(&maps, tma, sizeof(maps));
  dim3 grid((n[0] + TX - 1) / TX, (n[1] + TY - 1) / TY, (n[2] + a.chunk - 1) / a.chunk);
  kern<<<grid, dim3(TX, TY), smem, s>>>(a, maps);
  return cudaGetLastError();
}

// CTA shapes.  3D: 32x8 (2 or 3 CTAs/SM), 32x16, 64x8, and for the split
// precision on Cartesian grids the TMA-staged 32x8 with overlapping tiles
// (variants 4, 5) and with non-overlapping tiles (6, 7), and the TMA-staged
// non-overlapping 16x16 (8, 9), each at 2 or 3 CTAs/SM; 2D rows of 128, 256
// or 64 threads, rows of 64 and 128 threads held to 80 registers (24 warps
// per SM; variants 3, 4), and in the default form one warp per strip of 31
// columns with the row exchanged by shuffles (variants 5, 6: 24 or 16
// strips per SM); 1D: 128.  Curvilinear 3D
// grids in the split precision: the default shape, the TMA-staged
// non-overlapping 32x8 at 2 or 3 CTAs/SM (variants 1, 2) and 16x16 at 3
// (variant 3); other curvilinear
// grids the default shape only.  The general form (GEN: face options,
// absorption only, irradiation, evolved gas) has the TMA-staged shapes only
// when it keeps the default face scheme (TMA_OK).  UYZ: directions 1 and 2
// evenly spaced (for the TMA-staged curvilinear shapes).
template <class P, int NDIM, int GEOM, int NC, bool UNI, bool GEN = false, bool TMA_OK = true,
          bool UYZ = false>
struct Shapes {
  static constexpr bool tma = TMA_OK && P::kSplit && GEOM == kCart && NDIM == 3;
  static constexpr bool tma_curv = TMA_OK && P::kSplit && GEOM != kCart && NDIM == 3;
  static constexpr int count =
      tma_curv ? 4
               : ((GEOM != kCart || NDIM == 1) ? 1 : (NDIM == 3 ? (tma ? 10 : 4) : (GEN ? 5 : 7)));
  static cudaError_t launch(const void* vargs, const void* maps, cudaStream_t s, int variant,
                            int chunk) {
    const StepArgs<P>& a = *static_cast<const StepArgs<P>*>(vargs);
    if (variant < 0 || variant >= count) variant = 0;
    if constexpr (NDIM == 3) {
      if constexpr (tma_curv) {
        if (variant == 1) return launch_tma2<P, NC, UNI, 32, 8, 2, GEN, GEOM, UYZ>(a, maps, s, chunk);
        if (variant == 2) return launch_tma2<P, NC, UNI, 32, 8, 3, GEN, GEOM, UYZ>(a, maps, s, chunk);
        if (variant == 3) return launch_tma2<P, NC, UNI, 16, 16, 3, GEN, GEOM, UYZ>(a, maps, s, chunk);
        return launch_shape<P, 3, GEOM, NC, UNI, 32, 8, 2, GEN>(a, s, chunk);
      }
      if constexpr (tma) {
        if (variant == 4) return launch_tma<P, NC, UNI, 32, 8, 2, GEN>(a, maps, s, chunk);
        if (variant == 5) return launch_tma<P, NC, UNI, 32, 8, 3, GEN>(a, maps, s, chunk);
        if (variant == 6) return launch_tma2<P, NC, UNI, 32, 8, 2, GEN>(a, maps, s, chunk);
        if (variant == 7) return launch_tma2<P, NC, UNI, 32, 8, 3, GEN>(a, maps, s, chunk);
        if (variant == 8) return launch_tma2<P, NC, UNI, 16, 16, 2, GEN>(a, maps, s, chunk);
        if (variant == 9) return launch_tma2<P, NC, UNI, 16, 16, 3, GEN>(a, maps, s, chunk);
      }
      if constexpr (count > 1) {
        if (variant == 1) return launch_shape<P, 3, GEOM, NC, UNI, 32, 8, 3, GEN>(a, s, chunk);
        if (variant == 2) return launch_shape<P, 3, GEOM, NC, UNI, 32, 16, 1, GEN>(a, s, chunk);
        if (variant == 3) return launch_shape<P, 3, GEOM, NC, UNI, 64, 8, 1, GEN>(a, s, chunk);
      }
      return launch_shape<P, 3, GEOM, NC, UNI, 32, 8, 2, GEN>(a, s, chunk);
    } else if constexpr (NDIM == 2) {
      if constexpr (count > 1) {
        if (variant == 1) return launch_shape<P, 2, GEOM, NC, UNI, 256, 1, 1, GEN>(a, s, chunk);
        if (variant == 2) return launch_shape<P, 2, GEOM, NC, UNI, 64, 1, 1, GEN>(a, s, chunk);
        if (variant == 3) return launch_shape<P, 2, GEOM, NC, UNI, 64, 1, 12, GEN>(a, s, chunk);
        if (variant == 4) return launch_shape<P, 2, GEOM, NC, UNI, 128, 1, 6, GEN>(a, s, chunk);
        if constexpr (!GEN && GEOM == kCart) {
          if (variant == 5) return launch_strip2d<P, NC, UNI, 24>(a, s, chunk);
          if (variant == 6) return launch_strip2d<P, NC, UNI, 16>(a, s, chunk);
        }
      }
      return launch_shape<P, 2, GEOM, NC, UNI, 128, 1, 1, GEN>(a, s, chunk);
    } else {
      return launch_shape<P, 1, GEOM, NC, UNI, 128, 1, 1, GEN>(a, s, chunk);
    }
  }
};

template <class P, int NDIM, int GEOM, int NC, bool UNI = false, bool GEN = false,
          bool TMA_OK = true, bool UYZ = false>
LaunchEntry entry() {
  using Sh = Shapes<P, NDIM, GEOM, NC, UNI, GEN, TMA_OK, UYZ>;
  LaunchEntry e{&Sh::launch, Sh::count, {}};
  if constexpr (Sh::tma) {
    for (int v = 4; v < 6; ++v) {
      e.tma_box[v][0] = TmaTile<32, 8>::BX;
      e.tma_box[v][1] = TmaTile<32, 8>::BY;
    }
    for (int v = 6; v < 8; ++v) {
      e.tma_box[v][0] = Tma2Tile<32, 8>::BX;
      e.tma_box[v][1] = Tma2Tile<32, 8>::BY;
    }
    for (int v = 8; v < 10; ++v) {
      e.tma_box[v][0] = Tma2Tile<16, 16>::BX;
      e.tma_box[v][1] = Tma2Tile<16, 16>::BY;
    }
  }
  if constexpr (Sh::tma_curv) {
    for (int v = 1; v < 3; ++v) {
      e.tma_box[v][0] = Tma2Tile<32, 8>::BX;
      e.tma_box[v][1] = Tma2Tile<32, 8>::BY;
    }
    e.tma_box[3][0] = Tma2Tile<16, 16>::BX;
    e.tma_box[3][1] = Tma2Tile<16, 16>::BY;
  }
  return e;
}

}  // namespace m1
