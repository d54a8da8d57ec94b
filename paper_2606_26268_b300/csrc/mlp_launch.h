// mlp_launch.h -- host launchers of the learned-guess kernels.
#pragma once
#include <cuda_runtime.h>

namespace m1 {

// Queue pass of one step (`args` points to the StepArgs of the policy).
typedef cudaError_t (*QueueFn)(const void* args, cudaStream_t stream);
QueueFn select_queue_pass(bool split, int ndim, int nc);

int mlp_nparam();
cudaError_t mlp_grad_launch(const float* w, const float4* rec, long long n,
                            unsigned long long a_perm, unsigned long long c_perm, long long b0,
                            int bsize, float* grad, double* loss, cudaStream_t s);
cudaError_t mlp_adam_launch(float* w, float* grad, float* m, float* v, float lr, int step,
                            cudaStream_t s);
cudaError_t mlp_predict_launch(const float* w, const float4* rec, long long n, float* out,
                               cudaStream_t s);
cudaError_t mlp_predict_tc_launch(const float* w, const float4* rec, long long n, float* out,
                                  int* status, cudaStream_t s);

}  // namespace m1
