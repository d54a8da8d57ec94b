// step_select.cu -- maps (precision, ndim, geometry, components) to the
// single-grid and batched launchers.
#include "step_launch.h"

namespace m1 {
LaunchEntry select_fp64(int ndim, int geom, int nc, int uni);
LaunchEntry select_split(int ndim, int geom, int nc, int uni);
LaunchEntry select_fp64_gen(int ndim, int geom, int nc, int uni, bool tma);
LaunchEntry select_split_gen(int ndim, int geom, int nc, int uni, bool tma);
}  // namespace m1

LaunchEntry select_launch(bool split, int ndim, int geom, int nc, int uniform, bool general,
                          bool options) {
  if (general)
    return split ? m1::select_split_gen(ndim, geom, nc, uniform, !options)
                 : m1::select_fp64_gen(ndim, geom, nc, uniform, !options);
  return split ? m1::select_split(ndim, geom, nc, uniform) : m1::select_fp64(ndim, geom, nc, uniform);
}

#include "batch_launch.h"

namespace m1 {
BatchEntry select_batch_fp64(int ndim, int nc, bool uni);
BatchEntry select_batch_split(int ndim, int nc, bool uni);
}  // namespace m1

BatchEntry select_batch(bool split, int ndim, int nc, bool uniform) {
  return split ? m1::select_batch_split(ndim, nc, uniform) : m1::select_batch_fp64(ndim, nc, uniform);
}
