// mlp.h -- host/device interface of the tensor-core kernels of the learned warm start.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fpt_device.cuh"

namespace fpt {

constexpr int kMlpIn = 64, kMlpHidden = 256, kMlpOut = 16;
// offsets of the parameter blocks in the flat FP32 vector
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + 256 * 64, kOffW2 = kOffB1 + 256, kOffB2 = kOffW2 + 256 * 256,
              kOffW3 = kOffB2 + 256, kOffB3 = kOffW3 + 256 * 256, kOffW4 = kOffB3 + 256, kOffB4 = kOffW4 + 16 * 256,
              kMlpParams = kOffB4 + 16;

// EPI_ATOMIC adds the product into C: the split-K partial products of the weight gradients, one per
// CTA, go in by TMA tensor reduce-adds (row- or column-major C), else by atomics.
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
  float* C;               // FP32 output: D (+bias) / gelu'(pre-activation) (EPI_BIAS_GELU) / dZ, or null where optional
  long long scm, scn;
  __nv_bfloat16* H;       // BF16 output: activation (EPI_BIAS_GELU) or dZ (EPI_GELU_GRAD)
  long long shm, shn;
  __nv_bfloat16* Ht;      // optional second copy of H with its own strides (the transpose, for the backward)
  long long shtm, shtn;
  const float* Zin;       // EPI_GELU_GRAD: gelu' at the pre-activation, as the forward's EPI_BIAS_GELU wrote it
  long long szm, szn;
  float* colsum;          // EPI_GELU_GRAD: the column sums of the FP32 result are added here ([N]), or null
  int* err;               // device error word (MMA completion timeout)
};

cudaError_t launch_gemm(const GemmArgs& g, int k_split, cudaStream_t stream);
// dst [C][R] = src [R][C]^T (bf16)
cudaError_t launch_bf16_transpose(const __nv_bfloat16* src, int R, int C, __nv_bfloat16* dst, cudaStream_t stream);
// The transposed BF16 weights of layers 2-4 (W^T [in][out]) from the BF16 parameter copy.
constexpr int kMlpWtElems = 256 * 256 + 256 * 256 + 256 * 16;
cudaError_t launch_mlp_transpose_weights(const __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t stream);
cudaError_t launch_mlp_features(const SceneDev& S, const BatchDev& B, int n, const PathRec* list, uint64_t first,
                                uint64_t count, float inv_scale, __nv_bfloat16* X, float* G, cudaStream_t stream);
cudaError_t launch_mlp_loss(const float* G, const float* Y, const float* T, uint64_t B, float* dY,
                            __nv_bfloat16* dYb, __nv_bfloat16* dYt, float* loss, cudaStream_t stream);
cudaError_t launch_colsum(const float* A, uint64_t B, int N, float* out, cudaStream_t stream);
cudaError_t launch_adam(float* w, float* m, float* v, const float* g, int n, float lr, float c1, float c2,
                        __nv_bfloat16* wb, cudaStream_t stream);
cudaError_t launch_to_bf16(const float* src, __nv_bfloat16* dst, int n, cudaStream_t stream);
constexpr size_t kMlpTiledBytes = 9 * 32768 + 4 * 2048;  // weights pre-tiled for the fused inference
cudaError_t launch_mlp_tile_weights(const __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t stream);
cudaError_t launch_mlp_infer(const SceneDev& S, const BatchDev& B, int n, const PathRec* list, uint64_t count,
                             float inv_scale, const __nv_bfloat16* wt, const float* params, float* T, int* err,
                             cudaStream_t stream, int n_sm);
// Rows perm(first .. first + B - 1) of (X [n][64], T [n][8], G [n][12]) into (Xb, Tb, Gb), perm = the
// seeded permutation of [0, n) drawn by key.
cudaError_t launch_mlp_gather(const __nv_bfloat16* X, const float* T, const float* G, uint64_t n, uint64_t first,
                              uint64_t B, uint64_t key, __nv_bfloat16* Xb, float* Tb, float* Gb, __nv_bfloat16* Xt,
                              cudaStream_t stream);
cudaError_t launch_mlp_accumulate(float* dst, const float* src, float w, cudaStream_t stream);
// One CTA waits, for at most `limit_ns` (1 ns .. 1 s), on an mbarrier that receives an arrival only
// when `arrive` != 0; a wait that runs out sets *err (if 0) to the MMA-timeout code.  `elapsed`
// (device, optional) receives the wait's duration in nanoseconds of the global timer.
cudaError_t launch_bounded_wait_check(uint32_t limit_ns, int arrive, int* err, unsigned long long* elapsed,
                                      cudaStream_t stream);
cudaError_t launch_mlp_start(const SceneDev& S, const BatchDev& B, int n, const PathRec* list, uint64_t first,
                             uint64_t count, const float* Y, float* T, cudaStream_t stream);

}  // namespace fpt
