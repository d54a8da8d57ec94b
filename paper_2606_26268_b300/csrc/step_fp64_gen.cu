// step_fp64_gen.cu -- step kernel instantiations for the Fp64 precision policy
// in the general form (face options, absorption only, irradiation).
#include "step_tables.cuh"

namespace m1 {
LaunchEntry select_fp64_gen(int ndim, int geom, int nc, int uni, bool tma) {
  return select_table<Fp64, true>(ndim, geom, nc, uni, tma);
}
}  // namespace m1
