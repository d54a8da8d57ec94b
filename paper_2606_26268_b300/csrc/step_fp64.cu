// step_fp64.cu -- step kernel instantiations for the Fp64 precision policy
// (default form).
#include "step_tables.cuh"

namespace m1 {
LaunchEntry select_fp64(int ndim, int geom, int nc, int uni) {
  return select_table<Fp64, false>(ndim, geom, nc, uni, true);
}
}  // namespace m1
