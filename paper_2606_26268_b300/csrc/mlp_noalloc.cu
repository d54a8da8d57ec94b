// mlp_noalloc.cu -- rad_mlp_grad_noalloc: the gradient of the learned
// guess's training loss computed without allocating any device memory.
//
// Who needs this: callers that cannot call cudaMalloc (or any allocating
// routine) at the point where they want the gradient, typically because their
// framework owns all device memory through its own pre-sized pool and forbids
// allocations after start-up, or because they must not synchronise the device
// the way cudaMalloc/cudaFree can.  rad_mlp_grad needs a context whose
// workspace holds its accumulators; this entry point needs no context: the
// caller passes the parameters, the records and the output buffers, and the
// scratch (partial gradients) lives in a file-scope device array that every
// GPU loading this library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "mlp.cuh"
#include "rad.h"

namespace {

using m1::MLP_B1;
using m1::MLP_B2;
using m1::MLP_B3;
using m1::MLP_B4;
using m1::MLP_H;
using m1::MLP_NPARAM;
using m1::MLP_W1;
using m1::MLP_W2;
using m1::MLP_W3;
using m1::MLP_W4;

constexpr int kRowRecords = RAD_NOALLOC_ROW_RECORDS;  // records per partial gradient
constexpr int kMaxRows = RAD_NOALLOC_MAX_RECORDS / RAD_NOALLOC_ROW_RECORDS;
constexpr int kMaxDevices = 64;

// Scratch: one partial gradient and one partial loss per block of records.
static __device__ __align__(256) float g_partial[kMaxRows * MLP_NPARAM];
static __device__ __align__(256) double g_loss_partial[kMaxRows];

// Block b sums the mean-squared-error gradient of records [64 b, 64 b + 64)
// (scaled by 1/n) into row b of the scratch, writing every entry of the row.
__global__ void __launch_bounds__(64) grad_rows_kernel(const float* __restrict__ w,
                                                      const float4* __restrict__ rec, long long n,
                                                      float inv_n, float* __restrict__ partial,
                                                      double* __restrict__ loss_partial) {
  __shared__ float sW2[MLP_H][MLP_H + 1], sW3[MLP_H][MLP_H + 1];
  __shared__ float h1[MLP_H], h2[MLP_H], d2[MLP_H], d3[MLP_H];
  __shared__ float red[2];
  const int j = threadIdx.x;
  for (int i = j; i < MLP_H * MLP_H; i += MLP_H) {
    sW2[i / MLP_H][i % MLP_H] = w[MLP_W2 + i];
    sW3[i / MLP_H][i % MLP_H] = w[MLP_W3 + i];
  }
  const float w1a = w[MLP_W1 + 2 * j], w1b = w[MLP_W1 + 2 * j + 1];
  const float b1 = w[MLP_B1 + j], b2 = w[MLP_B2 + j], b3 = w[MLP_B3 + j];
  const float w4 = w[MLP_W4 + j], b4 = w[MLP_B4];
  float gW2[MLP_H], gW3[MLP_H];
#pragma unroll
  for (int k = 0; k < MLP_H; ++k) gW2[k] = gW3[k] = 0.f;
  float gw1a = 0.f, gw1b = 0.f, gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, gw4 = 0.f, gb4 = 0.f;
  double lsum = 0.0;
  __syncthreads();
  const long long first = (long long)blockIdx.x * kRowRecords;
  const long long last = first + kRowRecords < n ? first + kRowRecords : n;
  for (long long s = first; s < last; ++s) {
    const float4 r = rec[s];
    const float x1 = r.x, x2 = r.y, t = r.z;
    const float a1 = tanhf(fmaf(w1a, x1, fmaf(w1b, x2, b1)));
    h1[j] = a1;
    __syncthreads();
    float acc = b2;
    for (int i = 0; i < MLP_H; ++i) acc = fmaf(sW2[j][i], h1[i], acc);
    const float a2 = tanhf(acc);
    h2[j] = a2;
    __syncthreads();
    acc = b3;
    for (int i = 0; i < MLP_H; ++i) acc = fmaf(sW3[j][i], h2[i], acc);
    const float a3 = tanhf(acc);
    float part = w4 * a3;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((j & 31) == 0) red[j >> 5] = part;
    __syncthreads();
    const float res = red[0] + red[1] + b4 - t;
    const float dout = 2.f * res * inv_n;
    if (j == 0) {
      lsum += double(res) * res;
      gb4 += dout;
    }
    gw4 += dout * a3;
    const float dd3 = dout * w4 * (1.f - a3 * a3);
    d3[j] = dd3;
    gb3 += dd3;
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) gW3[i] = fmaf(dd3, h2[i], gW3[i]);
    __syncthreads();
    acc = 0.f;
    for (int i = 0; i < MLP_H; ++i) acc = fmaf(sW3[i][j], d3[i], acc);
    const float dd2 = acc * (1.f - a2 * a2);
    d2[j] = dd2;
    gb2 += dd2;
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) gW2[i] = fmaf(dd2, h1[i], gW2[i]);
    __syncthreads();
    acc = 0.f;
    for (int i = 0; i < MLP_H; ++i) acc = fmaf(sW2[i][j], d2[i], acc);
    const float dd1 = acc * (1.f - a1 * a1);
    gb1 += dd1;
    gw1a = fmaf(dd1, x1, gw1a);
    gw1b = fmaf(dd1, x2, gw1b);
    __syncthreads();
  }
  float* row = partial + (size_t)blockIdx.x * MLP_NPARAM;
  row[MLP_W1 + 2 * j] = gw1a;
  row[MLP_W1 + 2 * j + 1] = gw1b;
  row[MLP_B1 + j] = gb1;
  row[MLP_B2 + j] = gb2;
  row[MLP_B3 + j] = gb3;
  row[MLP_W4 + j] = gw4;
#pragma unroll
  for (int i = 0; i < MLP_H; ++i) {
    row[MLP_W2 + MLP_H * j + i] = gW2[i];
    row[MLP_W3 + MLP_H * j + i] = gW3[i];
  }
  if (j == 0) {
    row[MLP_B4] = gb4;
    loss_partial[blockIdx.x] = lsum;
  }
}

// Sums the first `rows` partial gradients (fixed order, no atomics) into the
// caller's outputs; the loss is the mean over the n records.
__global__ void sum_rows_kernel(const float* __restrict__ partial,
                                const double* __restrict__ loss_partial, int rows, double inv_n,
                                float* __restrict__ grad, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MLP_NPARAM) {
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc += partial[(size_t)r * MLP_NPARAM + p];
    grad[p] = acc;
  }
  if (p == 0) {
    double l = 0.0;
    for (int r = 0; r < rows; ++r) l += loss_partial[r];
    *loss = float(l * inv_n);
  }
}

std::mutex g_setup_mutex;
float* g_partial_ptr[kMaxDevices] = {};
double* g_loss_ptr[kMaxDevices] = {};

// Device addresses of the scratch on the current device (looked up once per
// device, under a lock).
rad_status scratch_on_current_device(float** partial, double** loss) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RAD_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return RAD_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partial_ptr[dev]) {
    void* p = nullptr;
    void* l = nullptr;
    if (cudaGetSymbolAddress(&p, g_partial) != cudaSuccess) return RAD_ECUDA;
    if (cudaGetSymbolAddress(&l, g_loss_partial) != cudaSuccess) return RAD_ECUDA;
    g_partial_ptr[dev] = static_cast<float*>(p);
    g_loss_ptr[dev] = static_cast<double*>(l);
  }
  *partial = g_partial_ptr[dev];
  *loss = g_loss_ptr[dev];
  return RAD_OK;
}

}  // namespace

extern "C" rad_status rad_mlp_grad_noalloc(const float* dev_params, const float* dev_records,
                                           size_t n, float* dev_grad, float* dev_loss,
                                           void* stream) {
  if (!dev_params || !dev_records || !dev_grad || !dev_loss || n == 0) return RAD_EINVAL;
  // the records are read as 16-byte vectors
  if (reinterpret_cast<uintptr_t>(dev_records) & 15u) return RAD_EINVAL;
  if (n > size_t(RAD_NOALLOC_MAX_RECORDS)) return RAD_EINVAL;  // beyond the scratch
  float* partial = nullptr;
  double* loss_partial = nullptr;
  rad_status st = scratch_on_current_device(&partial, &loss_partial);
  if (st != RAD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rows = int((n + kRowRecords - 1) / kRowRecords);
  grad_rows_kernel<<<rows, MLP_H, 0, s>>>(dev_params, reinterpret_cast<const float4*>(dev_records),
                                          (long long)n, 1.f / float(n), partial, loss_partial);
  if (cudaGetLastError() != cudaSuccess) return RAD_ECUDA;
  sum_rows_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(partial, loss_partial, rows,
                                                           1.0 / double(n), dev_grad, dev_loss);
  if (cudaGetLastError() != cudaSuccess) return RAD_ECUDA;
  return RAD_OK;
}
