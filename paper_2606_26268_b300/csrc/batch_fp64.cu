// batch_fp64.cu -- batched kernel instantiations, FP64 precision policy.
#include "batch.cuh"

namespace m1 {
BatchEntry select_batch_fp64(int ndim, int nc, bool uni) {
  if (uni) {
    if (ndim == 2 && nc == 2) return batch_entry<Fp64, 2, 2, true>();
    if (ndim == 2 && nc == 3) return batch_entry<Fp64, 2, 3, true>();
    if (ndim == 3 && nc == 3) return batch_entry<Fp64, 3, 3, true>();
  } else {
    if (ndim == 2 && nc == 2) return batch_entry<Fp64, 2, 2, false>();
    if (ndim == 2 && nc == 3) return batch_entry<Fp64, 2, 3, false>();
    if (ndim == 3 && nc == 3) return batch_entry<Fp64, 3, 3, false>();
  }
  return BatchEntry{nullptr, nullptr, nullptr, 0, {0, 0, 0, 0}, {0, 0, 0, 0}};
}
}  // namespace m1
