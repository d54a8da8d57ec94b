// step_select.cu -- maps (precision, ndim, geometry, components) to a launcher.
#include "step_launch.h"

namespace m1 {
LaunchEntry select_fp64(int ndim, int geom, int nc, bool uni);
LaunchEntry select_split(int ndim, int geom, int nc, bool uni);
}  // namespace m1

LaunchEntry select_launch(bool split, int ndim, int geom, int nc, bool uniform) {
  return split ? m1::select_split(ndim, geom, nc, uniform) : m1::select_fp64(ndim, geom, nc, uniform);
}
