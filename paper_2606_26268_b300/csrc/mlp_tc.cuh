// mlp_tc.cuh -- the learned starting guess evaluated for 128 samples at a
// time on the 5th-generation tensor cores (tcgen05).
//
// The two 64 x 64 hidden layers are products [128 x 64] x [64 x 64] with
// bf16 operands in shared memory and FP32 accumulators in tensor memory
// (64 TMEM columns, one lane per sample).  One elected thread issues the
// four K = 16 steps of each product and commits them to an mbarrier; every
// warp then reads its 32 lanes back with tcgen05.ld.  The input layer (2
// inputs), biases, tanh and the output layer (64 -> 1) stay in FP32 on the
// CUDA cores.  bf16 operands cost about three significant digits, which is
// far below the accuracy the starting guess needs (the iteration converges
// to its own tolerance from any positive start).
//
// Operand layout in shared memory (K-major, no swizzle): 8 x 8 core
// matrices of 8 rows x 16 bytes, stored row-group-major, so that element
// (r, k) of a [rows x 64] bf16 matrix sits at byte
//   ((r / 8) * 8 + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
// Core matrices adjacent along K are 128 bytes apart (the descriptor's
// leading byte offset) and adjacent along rows 1024 bytes apart (its stride
// byte offset); a K = 16 step advances the start address by 256 bytes.
#pragma once
#include <cuda_bf16.h>

#include "mlp.cuh"
#include "tma.cuh"

namespace m1 {

constexpr int TC_ROWS = 128;                       // samples per product
constexpr uint32_t TC_LBO = 128, TC_SBO = 1024;    // bytes, see above
constexpr uint32_t TC_A_BYTES = TC_ROWS * MLP_H * 2;  // 16 KB
constexpr uint32_t TC_W_BYTES = MLP_H * MLP_H * 2;    // 8 KB
constexpr uint32_t TC_TMEM_COLS = 64;  // allocation (power of 2 >= 32): the N = 64 accumulators

// Instruction descriptor of tcgen05.mma kind::f16: D in F32 (bits 4-5 = 1),
// A and B in BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N = 64 (bits 17-22 = N / 8), M = 128 (bits 24-28 = M / 16).
constexpr uint32_t TC_IDESC =
    (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t tc_offset(int r, int k) {
  return uint32_t(((r >> 3) * 8 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (each >> 4), descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((TC_LBO >> 4) & 0x3FFFu) << 16) |
         (uint64_t((TC_SBO >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %4, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(uint32_t(accumulate)), "r"(TC_IDESC)
      : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared state of a CTA that evaluates the network on tensor cores.
struct TcMlpSmem {
  alignas(1024) unsigned char a[TC_A_BYTES];   // activations of the 128 samples
  alignas(1024) unsigned char w2[TC_W_BYTES];  // W2 (out x in) as bf16
  alignas(1024) unsigned char w3[TC_W_BYTES];  // W3
  float w1[2 * MLP_H], b1[MLP_H], b2[MLP_H], b3[MLP_H], w4[MLP_H], b4;
  alignas(8) unsigned long long bar;            // MMA completion
  uint32_t tmem;                                // TMEM base address
  int err;                                      // a bounded wait ran out
  int issued;                                   // thread 0 committed a product
  uint32_t last_parity;                         // phase of its last commit
};

// Writes 64 activations of row r (this thread) into the operand tile as bf16.
__device__ __forceinline__ void tc_store_row(unsigned char* tile, int r, const float (&h)[MLP_H]) {
#pragma unroll
  for (int kk = 0; kk < MLP_H / 8; ++kk) {
    uint4 u;
    __nv_bfloat162 p0 = __floats2bfloat162_rn(h[8 * kk + 0], h[8 * kk + 1]);
    __nv_bfloat162 p1 = __floats2bfloat162_rn(h[8 * kk + 2], h[8 * kk + 3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(h[8 * kk + 4], h[8 * kk + 5]);
    __nv_bfloat162 p3 = __floats2bfloat162_rn(h[8 * kk + 6], h[8 * kk + 7]);
    u.x = *reinterpret_cast<uint32_t*>(&p0);
    u.y = *reinterpret_cast<uint32_t*>(&p1);
    u.z = *reinterpret_cast<uint32_t*>(&p2);
    u.w = *reinterpret_cast<uint32_t*>(&p3);
    *reinterpret_cast<uint4*>(tile + tc_offset(r, 8 * kk)) = u;
  }
}

// Setup by all TC_ROWS threads of the CTA: parameters into shared memory
// (hidden weights as bf16 operand tiles), the completion barrier and the
// TMEM columns (allocated by warp 0).  Ends with a barrier.
__device__ __forceinline__ void tc_mlp_setup(TcMlpSmem& s, const float* __restrict__ w, int tid) {
  // element i = tid + TC_ROWS j of each hidden matrix, 2 U loads in flight
  // per round: a load, convert and store per element in turn would wait for
  // every load in sequence
  constexpr int PER = MLP_H * MLP_H / TC_ROWS, U = 8;
  static_assert(PER % U == 0, "whole rounds");
#pragma unroll 1
  for (int j0 = 0; j0 < PER; j0 += U) {
    float v2[U], v3[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      v2[u] = __ldg(w + MLP_W2 + tid + TC_ROWS * (j0 + u));
      v3[u] = __ldg(w + MLP_W3 + tid + TC_ROWS * (j0 + u));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = tid + TC_ROWS * (j0 + u);
      const int n = i / MLP_H, k = i % MLP_H;
      *reinterpret_cast<__nv_bfloat16*>(s.w2 + tc_offset(n, k)) = __float2bfloat16_rn(v2[u]);
      *reinterpret_cast<__nv_bfloat16*>(s.w3 + tc_offset(n, k)) = __float2bfloat16_rn(v3[u]);
    }
  }
  for (int i = tid; i < 2 * MLP_H; i += TC_ROWS) s.w1[i] = w[MLP_W1 + i];
  if (tid < MLP_H) {
    s.b1[tid] = w[MLP_B1 + tid];
    s.b2[tid] = w[MLP_B2 + tid];
    s.b3[tid] = w[MLP_B3 + tid];
    s.w4[tid] = w[MLP_W4 + tid];
  }
  if (tid == 0) {
    s.b4 = w[MLP_B4];
    s.err = 0;
    s.issued = 0;
    s.last_parity = 0;
    mbar_init(&s.bar, 1);
    mbar_fence_init();
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&s.tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // operand tiles written by the generic proxy, read by the tensor cores
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Releases the TMEM columns (all TC_ROWS threads; after the last forward).
// After a wait that ran out, the product last committed may still be
// writing the columns: thread 0 waits for it (bounded) before warp 0 frees
// them.
__device__ __forceinline__ void tc_mlp_teardown(TcMlpSmem& s, int tid) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && s.err && s.issued) mbar_wait(&s.bar, s.last_parity, kWaitLimit);
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem),
                 "r"(TC_TMEM_COLS)
                 : "memory");
}

// One hidden layer on the tensor cores: TMEM <- A (activations) x W^T, then
// this thread's 64 accumulators + bias through tanh into h.  `parity`: phase
// of the completion barrier this product completes.  Once a wait of the CTA
// has run out (s.err, read after the barrier that precedes the layer), no
// further product is issued and the accumulators are not read: the outputs
// are then meaningless and the launch reports STATUS_TIMEOUT.  A thread
// whose own wait runs out does not read the columns either, since the
// product may still be writing them.
__device__ __forceinline__ void tc_layer(TcMlpSmem& s, const unsigned char* wtile,
                                         const float* __restrict__ bias, uint32_t parity, int tid,
                                         float (&h)[MLP_H]) {
  const bool skip = *static_cast<volatile int*>(&s.err) != 0;
  if (tid == 0 && !skip) {
    const uint32_t a0 = smem_addr(s.a), b0 = smem_addr(wtile);
#pragma unroll
    for (int ks = 0; ks < MLP_H / 16; ++ks)
      tc_mma(s.tmem, tc_desc(a0 + ks * 256), tc_desc(b0 + ks * 256), ks > 0);
    tc_commit(&s.bar);
    s.issued = 1;
    s.last_parity = parity;
  }
  const bool done = !skip && mbar_wait(&s.bar, parity, kWaitLimit);
  if (!skip && !done) s.err = 1;
  tc_fence_after();
  const uint32_t lane = uint32_t(tid & ~31) << 16;  // this warp's 32 TMEM lanes
#pragma unroll
  for (int c = 0; c < MLP_H / 16; ++c) {
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = 0.f;
    // tcgen05.ld is warp-collective: the warp reads only if all its lanes
    // saw the product complete
    if (__all_sync(0xffffffffu, done)) {
      tc_ld16(s.tmem + lane + uint32_t(16 * c), v);
      tc_wait_ld();
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) h[16 * c + i] = tanh_approx(v[i] + bias[16 * c + i]);
  }
}

// Forward pass of the sample of this thread (x1, x2) for all TC_ROWS
// threads of the CTA together; returns the network output.
__device__ __forceinline__ float tc_mlp_forward(TcMlpSmem& s, float x1, float x2, int tid) {
  float h[MLP_H];
#pragma unroll
  for (int j = 0; j < MLP_H; ++j)
    h[j] = tanh_approx(fmaf(s.w1[2 * j], x1, fmaf(s.w1[2 * j + 1], x2, s.b1[j])));
  tc_store_row(s.a, tid, h);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tc_layer(s, s.w2, s.b2, 0u, tid, h);
  // every warp has read its accumulators and the product has read A
  tc_store_row(s.a, tid, h);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tc_layer(s, s.w3, s.b3, 1u, tid, h);
  float out = s.b4;
#pragma unroll
  for (int j = 0; j < MLP_H; ++j) out = fmaf(s.w4[j], h[j], out);
  tc_fence_before();
  __syncthreads();  // the next forward overwrites A and the accumulators
  tc_fence_after();
  return out;
}

}  // namespace m1
