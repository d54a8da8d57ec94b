// batch.cuh -- kernels that advance many independent Cartesian grids with
// one launch per step: a persistent step kernel that takes tiles of any grid
// from a shared work list, and a queue pass over the queues of all grids.
// Each tile runs exactly the single-grid tile code (step_tile), so a grid
// advanced in a batch gets the same values as when it is stepped alone.
#pragma once
#include <type_traits>

#include "batch_launch.h"
#include "m1_step.cuh"
#include "m1_strip2d.cuh"
#include "mlp_tc.cuh"
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
// STRIP: 2D tiles as one warp per strip (step_strip2d, TX = 32).
template <class P, int NDIM, int NC, bool UNI, int TX, int TY, int MINB, bool STRIP = false>
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
    if constexpr (STRIP)
      step_strip2d<P, NC, UNI>(s_args, w.y, w.z);
    else
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
// (prefix sums of their lengths in shared memory) and walked 128 cells per
// CTA at a time; each cell is finished by the same code as in the
// single-grid queue pass, with the learned guess on the tensor cores when the
// network is set.
template <class P, int NDIM, int NC>
__device__ __forceinline__ const StepArgs<P>& grid_of(const StepArgs<P>* args,
                                                     const unsigned int* s_off, int count,
                                                     unsigned int q, unsigned int& local) {
  int lo = 0, hi = count;  // grid g with s_off[g] <= q < s_off[g + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (s_off[mid] <= q)
      lo = mid;
    else
      hi = mid;
  }
  local = q - s_off[lo];
  return args[lo];
}

template <class P, int NDIM, int NC, bool MLP>
__global__ void __launch_bounds__(TC_ROWS)
    batch_queue_kernel(const StepArgs<P>* __restrict__ args, int count,
                       const unsigned int* __restrict__ counts) {
  __shared__ unsigned int s_off[kBatchMaxGrids + 1];
  __shared__ unsigned long long s_red[ST_N];
  // the network's shared state only when it is used
  __shared__ typename std::conditional<MLP, TcMlpSmem, int>::type s_tc;
  __shared__ unsigned int s_wsum[TC_ROWS / 32];
  const int tid = threadIdx.x;
  // prefix sums of the queue lengths, TC_ROWS grids at a time: each thread
  // loads one grid's length and the block scans them (warp shuffles, then
  // the warp totals), so the loads are not one thread's chain over all grids
  {
    const int lane = tid & 31, w = tid >> 5;
    unsigned int carry = 0;
    if (tid == 0) s_off[0] = 0;
    for (int g0 = 0; g0 < count; g0 += TC_ROWS) {
      const int g = g0 + tid;
      unsigned int v = g < count ? min(counts[g], args[g].queue_cap) : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (lane == 31) s_wsum[w] = v;
      __syncthreads();
      unsigned int before = 0, all = 0;
#pragma unroll
      for (int k = 0; k < TC_ROWS / 32; ++k) {
        before += k < w ? s_wsum[k] : 0u;
        all += s_wsum[k];
      }
      if (g < count) s_off[g + 1] = carry + before + v;
      carry += all;
      __syncthreads();  // s_wsum is rewritten by the next group
    }
  }
  const unsigned int total = s_off[count];
  const unsigned int first = blockIdx.x * TC_ROWS;
  if (first >= total) return;  // no queued cell for this block
  counters_reset(s_red, tid);
  if constexpr (MLP)
    tc_mlp_setup(s_tc, args[0].mlp_w, tid);  // ends with a barrier
  else
    __syncthreads();
  Counters cnt;
  for (unsigned int base = first; base < total; base += gridDim.x * TC_ROWS) {
    const unsigned int q = base + tid;
    const bool valid = q < total;
    unsigned int local = 0;
    const StepArgs<P>& a = grid_of<P, NDIM, NC>(args, s_off, count, valid ? q : 0u, local);
    QueuedCell<P> c;
    float T0 = 0.f;
    if (valid) queue_load<P, NC>(a, a.queue[local], c);
    if constexpr (MLP) {
      float x1 = 0.f, x2 = 0.f, lin = 0.f, Tn = 0.f;
      if (valid)
        coupling_features(a.cp, float(c.rho), float(c.e), float(c.kp), float(c.Us[0]), x1, x2,
                          lin, Tn);
      const bool gated = valid && lin > a.mlp_gate;
      if (__syncthreads_or(gated)) {
        const float g = tc_mlp_forward(s_tc, gated ? x1 : 0.f, gated ? x2 : 0.f, tid);
        if (gated) T0 = guess_temperature(Tn, g);
      }
    }
    if (valid) queue_solve<P, NDIM, NC>(a, c, T0, cnt);
  }
  if constexpr (MLP) {
    tc_mlp_teardown(s_tc, tid);
    if (tid == 0 && s_tc.err) atomicOr(args[0].status, STATUS_TIMEOUT);
  }
  counters_flush<P>(args[0], cnt, s_red, tid);
}

template <class P, int NDIM, int NC, bool UNI, int TX, int TY, int MINB, bool STRIP = false>
struct BatchShape {
  static cudaError_t launch(const void* args, const int4* items, int nitems, unsigned int* ctl,
                            int blocks, cudaStream_t s) {
    batch_step_kernel<P, NDIM, NC, UNI, TX, TY, MINB, STRIP>
        <<<blocks, dim3(TX, NDIM == 3 ? TY : 1), 0, s>>>(
            static_cast<const StepArgs<P>*>(args), items, nitems, ctl);
    return cudaGetLastError();
  }
  static cudaError_t occupancy(int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        per_sm, batch_step_kernel<P, NDIM, NC, UNI, TX, TY, MINB, STRIP>, TX * TY, 0);
  }
};

// CTA shapes: 2D rows of 128, 256 or 64 threads marching along y, rows of
// 64 and 128 threads held to 80 or 64 registers so that 24 or 32 warps fit
// on an SM, and one warp per strip of 31 columns (24 or 16 strips per SM);
// 3D 32x8 (2 or 3 CTAs/SM) marching along z.
template <class P, int NDIM, int NC, bool UNI>
struct BatchShapes {
  static constexpr int count = NDIM == 3 ? 2 : 8;
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
      if (variant == 3)
        return BatchShape<P, 2, NC, UNI, 64, 1, 12>::launch(args, items, nitems, ctl, blocks, s);
      if (variant == 4)
        return BatchShape<P, 2, NC, UNI, 128, 1, 6>::launch(args, items, nitems, ctl, blocks, s);
      if (variant == 5)
        return BatchShape<P, 2, NC, UNI, 64, 1, 16>::launch(args, items, nitems, ctl, blocks, s);
      if (variant == 6)
        return BatchShape<P, 2, NC, UNI, 32, 1, 24, true>::launch(args, items, nitems, ctl, blocks, s);
      if (variant == 7)
        return BatchShape<P, 2, NC, UNI, 32, 1, 16, true>::launch(args, items, nitems, ctl, blocks, s);
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
      if (variant == 3) return BatchShape<P, 2, NC, UNI, 64, 1, 12>::occupancy(per_sm);
      if (variant == 4) return BatchShape<P, 2, NC, UNI, 128, 1, 6>::occupancy(per_sm);
      if (variant == 5) return BatchShape<P, 2, NC, UNI, 64, 1, 16>::occupancy(per_sm);
      if (variant == 6) return BatchShape<P, 2, NC, UNI, 32, 1, 24, true>::occupancy(per_sm);
      if (variant == 7) return BatchShape<P, 2, NC, UNI, 32, 1, 16, true>::occupancy(per_sm);
      return BatchShape<P, 2, NC, UNI, 128, 1, 1>::occupancy(per_sm);
    }
  }
  static cudaError_t qpass(const void* args, int count, const unsigned int* counts, bool mlp,
                           cudaStream_t s) {
    if (mlp)
      batch_queue_kernel<P, NDIM, NC, true><<<148 * 4, TC_ROWS, 0, s>>>(
          static_cast<const StepArgs<P>*>(args), count, counts);
    else
      batch_queue_kernel<P, NDIM, NC, false><<<148 * 4, TC_ROWS, 0, s>>>(
          static_cast<const StepArgs<P>*>(args), count, counts);
    return cudaGetLastError();
  }
};

template <class P, int NDIM, int NC, bool UNI>
BatchEntry batch_entry() {
  using B = BatchShapes<P, NDIM, NC, UNI>;
  BatchEntry e{&B::step, &B::qpass, &B::occupancy, B::count, {}, {1, 1, 1, 1, 1, 1, 1, 1}};
  if (NDIM == 3) {
    e.tx[0] = e.tx[1] = 32;
    e.ty[0] = e.ty[1] = 8;
  } else {
    e.tx[0] = 128;
    e.tx[1] = 256;
    e.tx[2] = 64;
    e.tx[3] = 64;
    e.tx[4] = 128;
    e.tx[5] = 64;
    e.tx[6] = e.tx[7] = 32;
  }
  return e;
}

}  // namespace m1
