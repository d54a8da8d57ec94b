// step_launch.h -- launchers of the step kernel instantiations.
#pragma once
#include <cuda_runtime.h>

// Launches one step; `args` points to the StepArgs of the policy.  `variant`
// selects the CTA shape (0 = default; see step_launch.cuh) and `chunk` the
// number of cells each CTA marches (0 = default).
typedef cudaError_t (*LaunchFn)(const void* args, cudaStream_t stream, int variant, int chunk);

struct LaunchEntry {
  LaunchFn fn;
  int variants;  // number of CTA shapes instantiated
};

// The launcher for (precision, active directions, geometry, carried flux
// components, uniform Cartesian spacing); fn == nullptr when that
// combination is not instantiated.
LaunchEntry select_launch(bool split, int ndim, int geom, int nc, bool uniform);
