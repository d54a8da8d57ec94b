// batch.cuh -- kernels that advance many independent Cartesian grids with
// one launch per step: a persistent step kernel that takes tiles of any grid
// from a shared work list, and a queue pass over the queues of all grids.
// Each tile runs exactly the single-grid tile code (step_tile), so a grid
// advanced in a batch gets the same values as when it is stepped alone.
#pragma once
#include "batch_launch.h"
#include "m1_step.cuh"
#include "queue_cell.cuh"

namespace m1 {

// Copies one grid's step arguments into shared memory (8-byte words).
template <class P>
__device__ __forceinline__ void copy_args(StepArgs<P>* dst, const StepArgs<P>* src, int tid,
                                          int nt) {
  static_assert(sizeof(StepArgs<P>) % 8 == 0, "argument block of whole words");
  constexpr int W = int(sizeof(StepArgs<P>) / 8);
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (int i = tid; i < W; i += nt) d[i] = __ldg(s + i);
}

// Persistent step: every CTA repeatedly takes the next tile of the work list
// (one atomic per tile), loads that grid's arguments into shared memory and
// runs the tile.  No CTA waits on another: the last CTA to retire resets the
// counters for the next launch, which the stream orders after this one.
template <class P, int NDIM, int NC, bool UNI, int TX, int TY, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB)
    batch_step_kernel(const StepArgs<P>* __restrict__ args, const int4* __restrict__ items,
                      int nitems, unsigned int* ctl) {
  __shared__ StepArgs<P> s_args;
  __shared__ int s_item;
  constexpr int NT = TX * TY;
  const int tid = threadIdx.x + TX * (NDIM == 3 ? threadIdx.y : 0);
  for (;;) {
    if (tid == 0) s_item = int(atomicAdd(ctl, 1u));
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int4 w = __ldg(items + it);
    copy_args<P>(&s_args, args + w.x, tid, NT);
    __syncthreads();
    step_tile<P, NDIM, kCart, NC, UNI, TX, TY>(s_args, w.y, w.z, w.w);
    __syncthreads();  // s_args and s_item are rewritten by the next tile
  }
  if (tid == 0) {
    __threadfence();
    const unsigned int done = atomicAdd(ctl + 1, 1u);
    if (done == gridDim.x - 1) {  // every CTA has taken its last item
      ctl[0] = 0u;
      ctl[1] = 0u;
    }
  }
}

// Queue pass over all grids: the queues are concatenated in grid order
// (prefix sums of their lengths in shared memory) and walked grid-stride;
// each cell is finished by the same code as in the single-grid queue pass.
template <class P, int NDIM, int NC>
__global__ void __launch_bounds__(128)
    batch_queue_kernel(const StepArgs<P>* __restrict__ args, int count,
                       const unsigned int* __restrict__ counts) {
  extern __shared__ __align__(16) float s_w[];
  __shared__ unsigned int s_off[kBatchMaxGrids + 1];
  __shared__ unsigned long long s_red[ST_N];
  if (threadIdx.x == 0) {
    unsigned int acc = 0;
    s_off[0] = 0;
    for (int g = 0; g < count; ++g) {
      acc += min(counts[g], args[g].queue_cap);
      s_off[g + 1] = acc;
    }
  }
  __syncthreads();
  const unsigned int total = s_off[count];
  if (blockIdx.x * blockDim.x >= total) return;  // no queued cell for this block
  const float* w = args[0].mlp_w;
  if (w) load_mlp_weights(s_w, w);
  counters_reset(s_red, threadIdx.x);
  __syncthreads();
  Counters cnt;
  for (unsigned int q = blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += gridDim.x * blockDim.x) {
    // grid g with s_off[g] <= q < s_off[g + 1]
    int lo = 0, hi = count;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_off[mid] <= q)
        lo = mid;
      else
        hi = mid;
    }
    const StepArgs<P>& a = args[lo];
    queue_cell<P, NDIM, NC>(a, a.queue[q - s_off[lo]], s_w, cnt);
  }
  counters_flush<P>(args[0], cnt, s_red, threadIdx.x);
}

template <class P, int NDIM, int NC, bool UNI, int TX, int TY, int MINB>
struct BatchShape {
  static cudaError_t launch(const void* args, const int4* items, int nitems, unsigned int* ctl,
                            int blocks, cudaStream_t s) {
    batch_step_kernel<P, NDIM, NC, UNI, TX, TY, MINB>
        <<<blocks, dim3(TX, NDIM == 3 ? TY : 1), 0, s>>>(
            static_cast<const StepArgs<P>*>(args), items, nitems, ctl);
    return cudaGetLastError();
  }
  static cudaError_t occupancy(int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        per_sm, batch_step_kernel<P, NDIM, NC, UNI, TX, TY, MINB>, TX * TY, 0);
  }
};

// CTA shapes: 2D rows of 128, 256 or 64 threads marching along y; 3D 32x8
// (2 or 3 CTAs/SM) marching along z.
template <class P, int NDIM, int NC, bool UNI>
struct BatchShapes {
  static constexpr int count = NDIM == 3 ? 2 : 3;
  static cudaError_t step(const void* args, const int4* items, int nitems, unsigned int* ctl,
                          int variant, int blocks, cudaStream_t s) {
    if constexpr (NDIM == 3) {
      if (variant == 1)
        return BatchShape<P, 3, NC, UNI, 32, 8, 3>::launch(args, items, nitems, ctl, blocks, s);
      return BatchShape<P, 3, NC, UNI, 32, 8, 2>::launch(args, items, nitems, ctl, blocks, s);
    } else {
      if (variant == 1)
        return BatchShape<P, 2, NC, UNI, 256, 1, 1>::launch(args, items, nitems, ctl, blocks, s);
      if (variant == 2)
        return BatchShape<P, 2, NC, UNI, 64, 1, 1>::launch(args, items, nitems, ctl, blocks, s);
      return BatchShape<P, 2, NC, UNI, 128, 1, 1>::launch(args, items, nitems, ctl, blocks, s);
    }
  }
  static cudaError_t occupancy(int variant, int* per_sm) {
    if constexpr (NDIM == 3) {
      if (variant == 1) return BatchShape<P, 3, NC, UNI, 32, 8, 3>::occupancy(per_sm);
      return BatchShape<P, 3, NC, UNI, 32, 8, 2>::occupancy(per_sm);
    } else {
      if (variant == 1) return BatchShape<P, 2, NC, UNI, 256, 1, 1>::occupancy(per_sm);
      if (variant == 2) return BatchShape<P, 2, NC, UNI, 64, 1, 1>::occupancy(per_sm);
      return BatchShape<P, 2, NC, UNI, 128, 1, 1>::occupancy(per_sm);
    }
  }
  static cudaError_t qpass(const void* args, int count, const unsigned int* counts, bool mlp,
                           cudaStream_t s) {
    const size_t smem = mlp ? MLP_NPARAM_PAD * sizeof(float) : 0;
    batch_queue_kernel<P, NDIM, NC><<<148 * 4, 128, smem, s>>>(
        static_cast<const StepArgs<P>*>(args), count, counts);
    return cudaGetLastError();
  }
};

template <class P, int NDIM, int NC, bool UNI>
BatchEntry batch_entry() {
  using B = BatchShapes<P, NDIM, NC, UNI>;
  BatchEntry e{&B::step, &B::qpass, &B::occupancy, B::count, {0, 0, 0, 0}, {1, 1, 1, 1}};
  if (NDIM == 3) {
    e.tx[0] = e.tx[1] = 32;
    e.ty[0] = e.ty[1] = 8;
  } else {
    e.tx[0] = 128;
    e.tx[1] = 256;
    e.tx[2] = 64;
  }
  return e;
}

}  // namespace m1
