// step_launch.h -- launchers of the step kernel instantiations.
#pragma once
#include <cuda_runtime.h>

// Launches one step; `args` points to the StepArgs of the policy and `tma`
// to the six tensor maps (CUtensorMap: E, F0..F2, rho, e of the input
// buffer) of the TMA-staged variants (ignored by the others).  `variant`
// selects the CTA shape (0 = default; see step_launch.cuh) and `chunk` the
// number of cells each CTA marches (0 = default).
typedef cudaError_t (*LaunchFn)(const void* args, const void* tma, cudaStream_t stream,
                                int variant, int chunk);

constexpr int kMaxVariants = 10;

struct LaunchEntry {
  LaunchFn fn;
  int variants;                    // number of CTA shapes instantiated
  int tma_box[kMaxVariants][2];    // TMA box (columns, rows) of a TMA-staged variant, else 0
};

// The launcher for (precision, active directions, geometry, carried flux
// components, spacing, general form, face options); uniform: bit 0 every
// direction of a Cartesian grid evenly spaced, bit 1 directions 1 and 2
// evenly spaced;
// fn == nullptr when that combination is not instantiated.  The general form
// carries the absorption-only coupling, the irradiation deposit and the
// evolved gas, and with `options` the face options of Sect. 2.5, which the
// TMA-staged shapes do not implement.
LaunchEntry select_launch(bool split, int ndim, int geom, int nc, int uniform, bool general,
                          bool options);
