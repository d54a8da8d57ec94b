// step_split.cu -- step kernel instantiations for the Split precision policy.
#include "step_launch.cuh"

namespace m1 {
LaunchEntry select_split(int ndim, int geom, int nc, bool uni) {
  if (geom == kCart && uni) {
    if (ndim == 1 && nc == 1) return entry<Split, 1, kCart, 1, true>();
    if (ndim == 1 && nc == 2) return entry<Split, 1, kCart, 2, true>();
    if (ndim == 1 && nc == 3) return entry<Split, 1, kCart, 3, true>();
    if (ndim == 2 && nc == 2) return entry<Split, 2, kCart, 2, true>();
    if (ndim == 2 && nc == 3) return entry<Split, 2, kCart, 3, true>();
    if (ndim == 3 && nc == 3) return entry<Split, 3, kCart, 3, true>();
    return LaunchEntry{nullptr, 0};
  }
  if (geom == kCart) {
    if (ndim == 1 && nc == 1) return entry<Split, 1, kCart, 1>();
    if (ndim == 1 && nc == 2) return entry<Split, 1, kCart, 2>();
    if (ndim == 1 && nc == 3) return entry<Split, 1, kCart, 3>();
    if (ndim == 2 && nc == 2) return entry<Split, 2, kCart, 2>();
    if (ndim == 2 && nc == 3) return entry<Split, 2, kCart, 3>();
    if (ndim == 3 && nc == 3) return entry<Split, 3, kCart, 3>();
    return LaunchEntry{nullptr, 0};
  }
  if (nc != 3) return LaunchEntry{nullptr, 0};
  if (geom == kCyl) {
    if (ndim == 1) return entry<Split, 1, kCyl, 3>();
    if (ndim == 2) return entry<Split, 2, kCyl, 3>();
    if (ndim == 3) return entry<Split, 3, kCyl, 3>();
  }
  if (geom == kSph) {
    if (ndim == 1) return entry<Split, 1, kSph, 3>();
    if (ndim == 2) return entry<Split, 2, kSph, 3>();
    if (ndim == 3) return entry<Split, 3, kSph, 3>();
  }
  return LaunchEntry{nullptr, 0};
}
}  // namespace m1
