// step_split_gen.cu -- step kernel instantiations for the Split precision policy
// in the general form (face options, absorption only, irradiation).
#include "step_tables.cuh"

namespace m1 {
LaunchEntry select_split_gen(int ndim, int geom, int nc, int uni, bool tma) {
  return select_table<Split, true>(ndim, geom, nc, uni, tma);
}
}  // namespace m1
