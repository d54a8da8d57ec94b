// mlp.cuh -- the small network that supplies the starting temperature of
// the coupling iteration in Newton mode (an extension of the method, not in
// the paper).  Input: the two dimensionless numbers of the converged coupling
// (see coupling_features); output: log(T^{n+1} / T^n).  Three tanh hidden
// layers of 64 units.  Parameters are one float vector:
//   W1 (64 x 2, row-major), b1 (64), W2 (64 x 64), b2, W3 (64 x 64), b3,
//   w4 (64), b4 (1).
#pragma once

namespace m1 {

constexpr int MLP_H = 64;
constexpr int MLP_W1 = 0;
constexpr int MLP_B1 = MLP_W1 + MLP_H * 2;
constexpr int MLP_W2 = MLP_B1 + MLP_H;
constexpr int MLP_B2 = MLP_W2 + MLP_H * MLP_H;
constexpr int MLP_W3 = MLP_B2 + MLP_H;
constexpr int MLP_B3 = MLP_W3 + MLP_H * MLP_H;
constexpr int MLP_W4 = MLP_B3 + MLP_H;
constexpr int MLP_B4 = MLP_W4 + MLP_H;
constexpr int MLP_NPARAM = MLP_B4 + 1;  // 8577
// parameters as whole float4 words (the buffers holding them are allocated in
// 256-byte pieces, so the padded tail is readable)
constexpr int MLP_NPARAM_PAD = (MLP_NPARAM + 3) / 4 * 4;

// Copies the parameters into shared memory (s_w: MLP_NPARAM_PAD floats,
// 16-byte aligned) with 16-byte loads, several in flight per thread.
__device__ __forceinline__ void load_mlp_weights(float* s_w, const float* w) {
  const float4* src = reinterpret_cast<const float4*>(w);
  float4* dst = reinterpret_cast<float4*>(s_w);
#pragma unroll 4
  for (int i = threadIdx.x; i < MLP_NPARAM_PAD / 4; i += blockDim.x) dst[i] = __ldg(src + i);
}

__device__ __forceinline__ float tanh_approx(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Forward pass of one sample with the parameters in shared memory.
__device__ __forceinline__ float mlp_forward(const float* __restrict__ w, float x1, float x2) {
  float h1[MLP_H], h2[MLP_H];
#pragma unroll
  for (int j = 0; j < MLP_H; ++j)
    h1[j] = tanh_approx(fmaf(w[MLP_W1 + 2 * j], x1, fmaf(w[MLP_W1 + 2 * j + 1], x2, w[MLP_B1 + j])));
#pragma unroll
  for (int j = 0; j < MLP_H; ++j) {
    float acc = w[MLP_B2 + j];
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) acc = fmaf(w[MLP_W2 + MLP_H * j + k], h1[k], acc);
    h2[j] = tanh_approx(acc);
  }
  float out = w[MLP_B4];
#pragma unroll 1
  for (int j = 0; j < MLP_H; ++j) {
    float acc = w[MLP_B3 + j];
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) acc = fmaf(w[MLP_W3 + MLP_H * j + k], h2[k], acc);
    out = fmaf(w[MLP_W4 + j], tanh_approx(acc), out);
  }
  return out;
}

}  // namespace m1
