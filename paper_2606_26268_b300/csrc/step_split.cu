// step_split.cu -- step kernel instantiations for the Split precision policy
// (default form).
#include "step_tables.cuh"

namespace m1 {
LaunchEntry select_split(int ndim, int geom, int nc, int uni) {
  return select_table<Split, false>(ndim, geom, nc, uni, true);
}
}  // namespace m1
