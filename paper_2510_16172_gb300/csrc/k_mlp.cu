// k_mlp.cu -- tensor-core (tcgen05) kernels of the learned warm start.
//
// A small MLP (3 hidden layers of 256, GELU) maps the geometry of a candidate
// sequence (TX, RX and the first four objects) to starting parameters t for
// the solver.  Weights are BF16, accumulation FP32 in tensor memory,
// activations are rounded to BF16 between layers.
//
// gemm_kernel: D[M x N] = sum_k A(m, k) B(n, k) for one 128-row tile per CTA,
// N <= 256, K in chunks of 64.  Operands are gathered from global memory with
// arbitrary element strides into the canonical K-major shared-memory layout
// (tc.cuh), so transposed operands of the backward pass need no copies.  One
// thread issues four 128 x N x 16 MMAs per chunk and commits them to an
// mbarrier; the epilogue reads the accumulator from TMEM (one warp per 32 rows)
// and applies: plain store, atomic add (split-K over the batch), bias + GELU
// with a BF16 activation, or the GELU derivative for the backward pass.
#include <cuda_bf16.h>

#include "fpt_kernels.h"
#include "mlp.h"
#include "tc.cuh"

namespace fpt {

constexpr int kGemmKC = 64;                  // K per chunk
constexpr uint32_t kWaitTries = 1u << 24;    // bounded mbarrier polls
constexpr int ERR_MMA_TIMEOUT = 3;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Gather rows [r0, r0 + 128) x k [k0, k0 + 64) of a strided bf16 matrix into a
// 128 x 64 K-major tile (zero outside rows < R, k < K).
__device__ __forceinline__ void load_tile(unsigned char* tile, const __nv_bfloat16* src, long long s_r, long long s_k,
                                          int R, int K, int r0, int k0, int rows) {
  const bool vec = (s_k == 1) && ((s_r & 7) == 0) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
  if (vec) {
    // 16-byte chunks: (row, group of 8 along k)
    for (int idx = threadIdx.x; idx < rows * (kGemmKC / 8); idx += blockDim.x) {
      const int r = idx / (kGemmKC / 8), kg = idx % (kGemmKC / 8);
      const int gr = r0 + r, gk = k0 + kg * 8;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (gr < R && gk + 8 <= K) {
        v = *reinterpret_cast<const uint4*>(src + (long long)gr * s_r + gk);
      } else if (gr < R && gk < K) {
        __nv_bfloat16 e[8];
        for (int q = 0; q < 8; ++q) e[q] = gk + q < K ? src[(long long)gr * s_r + gk + q] : __float2bfloat16(0.f);
        v = *reinterpret_cast<uint4*>(e);
      }
      *reinterpret_cast<uint4*>(tile + tc::kmajor_offset(r, kg * 8, kGemmKC)) = v;
    }
  } else {
    // element gather, consecutive threads along rows (coalesced when rows are contiguous)
    for (int idx = threadIdx.x; idx < rows * kGemmKC; idx += blockDim.x) {
      const int r = idx % rows, k = idx / rows;
      const int gr = r0 + r, gk = k0 + k;
      __nv_bfloat16 v = __float2bfloat16(0.f);
      if (gr < R && gk < K) v = src[(long long)gr * s_r + (long long)gk * s_k];
      *reinterpret_cast<__nv_bfloat16*>(tile + tc::kmajor_offset(r, k, kGemmKC)) = v;
    }
  }
}

constexpr int kGemmSmem = 128 * kGemmKC * 2 + 256 * kGemmKC * 2;  // A and B tiles (48 KB)

__global__ void __launch_bounds__(128) gemm_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char gemm_smem[];
  unsigned char* sA = gemm_smem;
  unsigned char* sB = gemm_smem + 128 * kGemmKC * 2;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128;
  const int n_pad = (g.N + 15) & ~15;
  const uint32_t ncols = n_pad <= 32 ? 32 : (n_pad <= 64 ? 64 : (n_pad <= 128 ? 128 : 256));
  // K range of this split
  const int k_per = ((g.K + gridDim.y * kGemmKC - 1) / (gridDim.y * kGemmKC)) * kGemmKC;
  const int kb = blockIdx.y * k_per, ke = min(g.K, kb + k_per);
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, ncols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc::idesc_bf16(128, n_pad);
  uint32_t phase = 0;
  int issued = 0;
  for (int k0 = kb; k0 < ke; k0 += kGemmKC) {
    load_tile(sA, g.A, g.sam, g.sak, g.M, g.K, m0, k0, 128);
    load_tile(sB, g.B, g.sbn, g.sbk, g.N, g.K, 0, k0, n_pad);
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < kGemmKC / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, (kGemmKC / 8) * 128);
        const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, (kGemmKC / 8) * 128);
        tc::mma_bf16(tmem, ad, bd, idesc, (issued | kk) ? 1u : 0u);
      }
      tc::mma_commit(&bar);
    }
    issued = 1;
    // the tiles are reused by the next chunk: wait until the MMAs have read them
    if (!tc::mbar_wait(&bar, phase, kWaitTries)) atomicExch(&s_fail, 1);
    phase ^= 1u;
    tc::fence_after_sync();
    __syncthreads();
    if (s_fail) break;
  }
  if (s_fail) {
    if (threadIdx.x == 0 && g.err) atomicCAS(g.err, 0, ERR_MMA_TIMEOUT);
    // give MMAs still in flight a (bounded) chance to finish before TMEM is freed
    tc::mbar_wait(&bar, phase, kWaitTries);
  } else if (issued) {
    // epilogue: warp w owns TMEM lanes (rows) 32 w .. 32 w + 31
    const int m = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < n_pad; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (m < g.M) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int n = c0 + q;
          if (n >= g.N) continue;
          float x = v[q];
          switch (g.op) {
            case EPI_STORE:
              if (g.bias) x += g.bias[n];
              g.C[(long long)m * g.scm + (long long)n * g.scn] = x;
              break;
            case EPI_ATOMIC:
              atomicAdd(g.C + (long long)m * g.scm + (long long)n * g.scn, x);
              break;
            case EPI_BIAS_GELU: {
              if (g.bias) x += g.bias[n];
              if (g.C) g.C[(long long)m * g.scm + (long long)n * g.scn] = x;
              g.H[(long long)m * g.shm + (long long)n * g.shn] = __float2bfloat16(gelu(x));
            } break;
            case EPI_GELU_GRAD: {
              const float dz = x * gelu_grad(g.Zin[(long long)m * g.szm + (long long)n * g.szn]);
              if (g.C) g.C[(long long)m * g.scm + (long long)n * g.scn] = dz;
              g.H[(long long)m * g.shm + (long long)n * g.shn] = __float2bfloat16(dz);
            } break;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

cudaError_t launch_gemm(const GemmArgs& g, int k_split, cudaStream_t stream) {
  if (g.N < 1 || g.N > 256 || g.M < 1 || g.K < 1 || k_split < 1) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((g.M + 127) / 128, k_split);
  gemm_kernel<<<grid, 128, kGemmSmem, stream>>>(g);
  return cudaGetLastError();
}

}  // namespace fpt
