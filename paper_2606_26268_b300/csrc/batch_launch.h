// batch_launch.h -- launchers of the batched kernels (many independent grids
// advanced by one persistent launch per step).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

// Largest number of grids in one batch (the queue pass keeps the prefix sum
// of the per-grid queue lengths in shared memory).
constexpr int kBatchMaxGrids = 1024;

// Persistent step over the tile work list `items` (int4: grid, bx, by, bz,
// as the single-grid kernel numbers its CTAs): `blocks` CTAs of shape
// `variant` take items through the counter ctl[0]; the last CTA to finish
// resets ctl[0] and ctl[1].  `args` is the device array of the grids' step
// arguments.
typedef cudaError_t (*BatchStepFn)(const void* args, const int4* items, int nitems,
                                   unsigned int* ctl, int variant, int blocks, cudaStream_t s);
// Queue pass over every grid's queue of cells left for the Newton iteration;
// counts[i] is the length of grid i's queue.  mlp: the parameters of the
// learned guess are set in the arguments.
typedef cudaError_t (*BatchQueueFn)(const void* args, int count, const unsigned int* counts,
                                    bool mlp, cudaStream_t s);
// Resident CTAs per SM of the persistent step kernel of shape `variant`.
typedef cudaError_t (*BatchOccFn)(int variant, int* per_sm);

struct BatchEntry {
  BatchStepFn step;
  BatchQueueFn qpass;
  BatchOccFn occupancy;
  int variants;
  int tx[8], ty[8];  // CTA shape of each variant
};

// The batched launchers for (precision, active directions, carried flux
// components, uniform spacing); step == nullptr when not instantiated
// (Cartesian 2D and 3D only).
BatchEntry select_batch(bool split, int ndim, int nc, bool uniform);
