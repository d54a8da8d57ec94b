// hydro_launch.h -- host launcher of the gas step.
#pragma once
#include <cuda_runtime.h>

namespace m1 {

// Launches the gas step; `args` points to the HydroArgs of the precision
// policy.  nullptr for combinations not instantiated.
typedef cudaError_t (*HydroFn)(const void* args, cudaStream_t stream);
HydroFn select_hydro(bool split, int ndim, int nc, bool uniform);

// Launches the reduction of the gas CFL rate; `args` points to the
// GasCflArgs of the precision policy.
HydroFn select_gas_cfl(bool split, int ndim, int nc);

}  // namespace m1
