// mlp.cu -- kernels of the learned starting guess: the queue pass of the
// step (network guess on the tensor cores, then the unchanged Newton
// iteration, for the cells the step kernel queued), and the training kernels
// (forward + backward over a mini-batch with block-level gradient
// accumulation, Adam update), the gradient of a given batch and plain FP32
// prediction.
#include <cuda_runtime.h>

#include <cmath>

#include "m1_cell.cuh"
#include "mlp.cuh"
#include "mlp_launch.h"
#include "mlp_tc.cuh"
#include "queue_cell.cuh"

namespace m1 {

// ---------------------------------------------------------------------------
// queue pass
// ---------------------------------------------------------------------------

// Queue pass without the learned guess: Newton from T^n.
template <class P, int NDIM, int NC>
__global__ void __launch_bounds__(128) queue_pass_kernel(const __grid_constant__ StepArgs<P> a) {
  __shared__ unsigned long long s_red[ST_N];
  const unsigned int count = min(*a.queue_count, a.queue_cap);
  if (blockIdx.x * blockDim.x >= count) return;  // no queued cell for this block
  counters_reset(s_red, threadIdx.x);
  __syncthreads();
  Counters cnt;
  for (unsigned int q = blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += gridDim.x * blockDim.x) {
    QueuedCell<P> c;
    queue_load<P, NC>(a, a.queue[q], c);
    queue_solve<P, NDIM, NC>(a, c, 0.f, cnt);
  }
  counters_flush<P>(a, cnt, s_red, threadIdx.x);
}

// Queue pass with the learned guess: the CTA takes 128 queued cells at a
// time; if any of them passes the gate, the network runs for all 128 on the
// tensor cores (rows of cells below the gate are ignored), and each gated
// cell starts its Newton iteration from T^n exp(output).
template <class P, int NDIM, int NC>
__global__ void __launch_bounds__(TC_ROWS, 5) queue_pass_tc_kernel(const __grid_constant__ StepArgs<P> a) {
  __shared__ TcMlpSmem s;
  __shared__ unsigned long long s_red[ST_N];
  const unsigned int count = min(*a.queue_count, a.queue_cap);
  const unsigned int first = blockIdx.x * TC_ROWS;
  if (first >= count) return;  // no queued cell for this block
  const int tid = threadIdx.x;
  counters_reset(s_red, tid);
  tc_mlp_setup(s, a.mlp_w, tid);  // ends with a barrier
  Counters cnt;
  for (unsigned int base = first; base < count; base += gridDim.x * TC_ROWS) {
    const unsigned int q = base + tid;
    const bool valid = q < count;
    QueuedCell<P> c;
    float x1 = 0.f, x2 = 0.f, lin = 0.f, Tn = 0.f;
    if (valid) {
      queue_load<P, NC>(a, a.queue[q], c);
      coupling_features(a.cp, float(c.rho), float(c.e), float(c.kp), float(c.Us[0]), x1, x2, lin,
                        Tn);
    }
    const bool gated = valid && lin > a.mlp_gate;
    float T0 = 0.f;
    if (__syncthreads_or(gated)) {
      const float g = tc_mlp_forward(s, gated ? x1 : 0.f, gated ? x2 : 0.f, tid);
      if (gated) T0 = guess_temperature(Tn, g);
    }
    if (valid) queue_solve<P, NDIM, NC>(a, c, T0, cnt);
  }
  tc_mlp_teardown(s, tid);
  if (tid == 0 && s.err) atomicOr(a.status, STATUS_TIMEOUT);
  counters_flush<P>(a, cnt, s_red, tid);
}

template <class P, int NDIM, int NC>
cudaError_t launch_queue_pass(const void* vargs, cudaStream_t s) {
  const StepArgs<P>& a = *static_cast<const StepArgs<P>*>(vargs);
  if (a.mlp_w)
    queue_pass_tc_kernel<P, NDIM, NC><<<148 * 5, TC_ROWS, 0, s>>>(a);
  else
    queue_pass_kernel<P, NDIM, NC><<<148 * 4, 128, 0, s>>>(a);
  return cudaGetLastError();
}

QueueFn select_queue_pass(bool split, int ndim, int nc) {
#define M1_Q(PP, D, C) \
  if (ndim == D && nc == C) return launch_queue_pass<PP, D, C>;
  if (split) {
    M1_Q(Split, 1, 1) M1_Q(Split, 1, 2) M1_Q(Split, 1, 3) M1_Q(Split, 2, 2) M1_Q(Split, 2, 3)
    M1_Q(Split, 3, 3)
  } else {
    M1_Q(Fp64, 1, 1) M1_Q(Fp64, 1, 2) M1_Q(Fp64, 1, 3) M1_Q(Fp64, 2, 2) M1_Q(Fp64, 2, 3)
    M1_Q(Fp64, 3, 3)
  }
#undef M1_Q
  return nullptr;
}

// ---------------------------------------------------------------------------
// training
// ---------------------------------------------------------------------------

// Mean-squared-error gradient over samples (a_perm k + c_perm) mod n,
// k in [b0, b0 + bsize): one block of 64 threads per sample at a time,
// thread j owning unit j of every layer; the block accumulates its share of
// the gradient in registers and adds it to `grad` at the end.
__global__ void __launch_bounds__(64) mlp_grad_kernel(const float* __restrict__ w,
                                                     const float4* __restrict__ rec, long long n,
                                                     unsigned long long a_perm,
                                                     unsigned long long c_perm, long long b0,
                                                     int bsize, float inv_b, float* grad,
                                                     double* loss) {
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
  for (int k = blockIdx.x; k < bsize; k += gridDim.x) {
    unsigned long long idx = (a_perm * (unsigned long long)(b0 + k) + c_perm) % (unsigned long long)n;
    float4 r = rec[idx];
    const float x1 = r.x, x2 = r.y, t = r.z;
    float a1 = tanhf(fmaf(w1a, x1, fmaf(w1b, x2, b1)));
    h1[j] = a1;
    __syncthreads();
    float acc = b2;
#pragma unroll 16
    for (int i = 0; i < MLP_H; ++i) acc = fmaf(sW2[j][i], h1[i], acc);
    const float a2 = tanhf(acc);
    h2[j] = a2;
    __syncthreads();
    acc = b3;
#pragma unroll 16
    for (int i = 0; i < MLP_H; ++i) acc = fmaf(sW3[j][i], h2[i], acc);
    const float a3 = tanhf(acc);
    float part = w4 * a3;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((j & 31) == 0) red[j >> 5] = part;
    __syncthreads();
    const float out = red[0] + red[1] + b4;
    const float res = out - t;
    const float dout = 2.f * res * inv_b;
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
#pragma unroll 16
    for (int i = 0; i < MLP_H; ++i) acc = fmaf(sW3[i][j], d3[i], acc);
    const float dd2 = acc * (1.f - a2 * a2);
    d2[j] = dd2;
    gb2 += dd2;
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) gW2[i] = fmaf(dd2, h1[i], gW2[i]);
    __syncthreads();
    acc = 0.f;
#pragma unroll 16
    for (int i = 0; i < MLP_H; ++i) acc = fmaf(sW2[i][j], d2[i], acc);
    const float dd1 = acc * (1.f - a1 * a1);
    gb1 += dd1;
    gw1a = fmaf(dd1, x1, gw1a);
    gw1b = fmaf(dd1, x2, gw1b);
    __syncthreads();
  }
  atomicAdd(grad + MLP_W1 + 2 * j, gw1a);
  atomicAdd(grad + MLP_W1 + 2 * j + 1, gw1b);
  atomicAdd(grad + MLP_B1 + j, gb1);
  atomicAdd(grad + MLP_B2 + j, gb2);
  atomicAdd(grad + MLP_B3 + j, gb3);
  atomicAdd(grad + MLP_W4 + j, gw4);
#pragma unroll
  for (int i = 0; i < MLP_H; ++i) {
    atomicAdd(grad + MLP_W2 + MLP_H * j + i, gW2[i]);
    atomicAdd(grad + MLP_W3 + MLP_H * j + i, gW3[i]);
  }
  if (j == 0) {
    atomicAdd(grad + MLP_B4, gb4);
    atomicAdd(loss, lsum);
  }
}

// Adam (Kingma & Ba 2015): m, v moments, bias-corrected step; clears grad.
__global__ void mlp_adam_kernel(float* w, float* grad, float* m, float* v, float lr, float beta1,
                                float beta2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MLP_NPARAM) return;
  float g = grad[i];
  float mi = beta1 * m[i] + (1.f - beta1) * g;
  float vi = beta2 * v[i] + (1.f - beta2) * g * g;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  grad[i] = 0.f;
}

__global__ void mlp_predict_kernel(const float* __restrict__ w, const float4* __restrict__ rec,
                                   long long n, float* out) {
  extern __shared__ __align__(16) float s_w[];
  load_mlp_weights(s_w, w);
  __syncthreads();
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    float4 r = rec[q];
    out[q] = mlp_forward(s_w, r.x, r.y);
  }
}

// Prediction on the tensor cores (the path of the queue pass), 128 records per
// CTA at a time; a bounded wait that ran out sets STATUS_TIMEOUT in *status.
__global__ void __launch_bounds__(TC_ROWS) mlp_predict_tc_kernel(const float* __restrict__ w,
                                                                 const float4* __restrict__ rec,
                                                                 long long n, float* out,
                                                                 int* status) {
  __shared__ TcMlpSmem s;
  const int tid = threadIdx.x;
  tc_mlp_setup(s, w, tid);
  for (long long base = (long long)blockIdx.x * TC_ROWS; base < n;
       base += (long long)gridDim.x * TC_ROWS) {
    const long long q = base + tid;
    const float4 r = q < n ? rec[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float g = tc_mlp_forward(s, r.x, r.y, tid);
    if (q < n) out[q] = g;
  }
  tc_mlp_teardown(s, tid);
  if (tid == 0 && s.err) atomicOr(status, STATUS_TIMEOUT);
}

cudaError_t mlp_predict_tc_launch(const float* w, const float4* rec, long long n, float* out,
                                  int* status, cudaStream_t s) {
  long long blocks = (n + TC_ROWS - 1) / TC_ROWS;
  if (blocks > 148 * 4) blocks = 148 * 4;
  if (blocks < 1) blocks = 1;
  mlp_predict_tc_kernel<<<int(blocks), TC_ROWS, 0, s>>>(w, rec, n, out, status);
  return cudaGetLastError();
}

cudaError_t mlp_grad_launch(const float* w, const float4* rec, long long n,
                            unsigned long long a_perm, unsigned long long c_perm, long long b0,
                            int bsize, float* grad, double* loss, cudaStream_t s) {
  int blocks = (bsize + 7) / 8;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  mlp_grad_kernel<<<blocks, MLP_H, 0, s>>>(w, rec, n, a_perm, c_perm, b0, bsize, 1.f / bsize,
                                           grad, loss);
  return cudaGetLastError();
}

cudaError_t mlp_adam_launch(float* w, float* grad, float* m, float* v, float lr, int step,
                            cudaStream_t s) {
  const float beta1 = 0.9f, beta2 = 0.999f;
  float c1 = float(1.0 / (1.0 - std::pow(double(beta1), step)));
  float c2 = float(1.0 / (1.0 - std::pow(double(beta2), step)));
  mlp_adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(w, grad, m, v, lr, beta1, beta2, 1e-8f,
                                                           c1, c2);
  return cudaGetLastError();
}

cudaError_t mlp_predict_launch(const float* w, const float4* rec, long long n, float* out,
                               cudaStream_t s) {
  const size_t smem = MLP_NPARAM_PAD * sizeof(float);
  long long blocks = (n + 127) / 128;
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (blocks < 1) blocks = 1;
  mlp_predict_kernel<<<int(blocks), 128, smem, s>>>(w, rec, n, out);
  return cudaGetLastError();
}

int mlp_nparam() { return MLP_NPARAM; }

}  // namespace m1
