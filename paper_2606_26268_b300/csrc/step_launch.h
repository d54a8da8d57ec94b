// step_launch.h -- launchers of the step kernel instantiations.
#pragma once
#include <cuda_runtime.h>

// Launches one step; `args` points to the StepArgs of the policy.
typedef cudaError_t (*LaunchFn)(const void* args, cudaStream_t stream);

// The launcher for (precision, active directions, geometry, carried flux
// components), or nullptr when that combination is not instantiated.
LaunchFn select_launch(bool split, int ndim, int geom, int nc);
