// step_tables.cuh -- the instantiated (precision, active directions,
// geometry, carried components, uniform spacing) combinations of the step
// kernel, as one table for the default form and the general form (GEN).
#pragma once
#include "step_launch.cuh"

namespace m1 {

// tma: offer the TMA-staged shapes (split 3D; the general form only when it
// keeps the default face scheme).  uni: bit 0 every direction evenly spaced,
// bit 1 directions 1 and 2 evenly spaced.
template <class P, bool GEN>
LaunchEntry select_table(int ndim, int geom, int nc, int uni_mask, bool tma) {
  const bool uni = uni_mask & 1, uyz = uni_mask & 2;
  if (geom == kCart && uni) {
    if (ndim == 1 && nc == 1) return entry<P, 1, kCart, 1, true, GEN>();
    if (ndim == 1 && nc == 2) return entry<P, 1, kCart, 2, true, GEN>();
    if (ndim == 1 && nc == 3) return entry<P, 1, kCart, 3, true, GEN>();
    if (ndim == 2 && nc == 2) return entry<P, 2, kCart, 2, true, GEN>();
    if (ndim == 2 && nc == 3) return entry<P, 2, kCart, 3, true, GEN>();
    if (ndim == 3 && nc == 3)
      return tma ? entry<P, 3, kCart, 3, true, GEN, true>() : entry<P, 3, kCart, 3, true, GEN, false>();
    return LaunchEntry{nullptr, 0};
  }
  if (geom == kCart) {
    if (ndim == 1 && nc == 1) return entry<P, 1, kCart, 1, false, GEN>();
    if (ndim == 1 && nc == 2) return entry<P, 1, kCart, 2, false, GEN>();
    if (ndim == 1 && nc == 3) return entry<P, 1, kCart, 3, false, GEN>();
    if (ndim == 2 && nc == 2) return entry<P, 2, kCart, 2, false, GEN>();
    if (ndim == 2 && nc == 3) return entry<P, 2, kCart, 3, false, GEN>();
    if (ndim == 3 && nc == 3)
      return tma ? entry<P, 3, kCart, 3, false, GEN, true>() : entry<P, 3, kCart, 3, false, GEN, false>();
    return LaunchEntry{nullptr, 0};
  }
  if (nc != 3) return LaunchEntry{nullptr, 0};
  if (geom == kCyl) {
    if (ndim == 1) return entry<P, 1, kCyl, 3, false, GEN>();
    if (ndim == 2) return entry<P, 2, kCyl, 3, false, GEN>();
    if (ndim == 3) {
      if (!tma) return entry<P, 3, kCyl, 3, false, GEN, false>();
      return uyz ? entry<P, 3, kCyl, 3, false, GEN, true, true>() : entry<P, 3, kCyl, 3, false, GEN, true>();
    }
  }
  if (geom == kSph) {
    if (ndim == 1) return entry<P, 1, kSph, 3, false, GEN>();
    if (ndim == 2) return entry<P, 2, kSph, 3, false, GEN>();
    if (ndim == 3) {
      if (!tma) return entry<P, 3, kSph, 3, false, GEN, false>();
      return uyz ? entry<P, 3, kSph, 3, false, GEN, true, true>() : entry<P, 3, kSph, 3, false, GEN, true>();
    }
  }
  return LaunchEntry{nullptr, 0};
}

}  // namespace m1
