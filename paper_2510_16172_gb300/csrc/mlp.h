// mlp.h -- host/device interface of the tensor-core kernels of the learned warm start.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace fpt {

enum EpilogueOp { EPI_STORE = 0, EPI_ATOMIC = 1, EPI_BIAS_GELU = 2, EPI_GELU_GRAD = 3 };

// D[M x N] = sum_k A(m, k) B(n, k); A(m, k) = A[m * sam + k * sak], B(n, k) = B[n * sbn + k * sbk].
struct GemmArgs {
  int M, N, K;
  const __nv_bfloat16* A;
  long long sam, sak;
  const __nv_bfloat16* B;
  long long sbn, sbk;
  int op;                 // EpilogueOp
  const float* bias;      // [N] (EPI_STORE, EPI_BIAS_GELU) or null
  float* C;               // FP32 output D (+bias) / pre-activation / dZ, or null where optional
  long long scm, scn;
  __nv_bfloat16* H;       // BF16 output: activation (EPI_BIAS_GELU) or dZ (EPI_GELU_GRAD)
  long long shm, shn;
  const float* Zin;       // pre-activation for EPI_GELU_GRAD
  long long szm, szn;
  int* err;               // device error word (MMA completion timeout)
};

cudaError_t launch_gemm(const GemmArgs& g, int k_split, cudaStream_t stream);

}  // namespace fpt
