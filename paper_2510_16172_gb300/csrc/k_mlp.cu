// k_mlp.cu -- tensor-core (tcgen05) kernels of the learned warm start.
//
// A small MLP (3 hidden layers of 256, GELU) maps the geometry of a candidate
// sequence (TX, RX and the first four objects) to starting parameters t for
// the solver.  Weights are BF16, accumulation FP32 in tensor memory,
// activations are rounded to BF16 between layers.
//
// GEMMs D[M x N] = sum_k A(m, k) B(n, k), N <= 256, K in chunks of 64.  Operands whose rows are
// contiguous and 16-byte aligned go to gemm_ws_kernel: persistent, one CTA per SM over (128-row tile,
// K split) items, the chunks loaded by TMA into a two-stage ring (128-byte swizzled K-major tiles), one
// thread issuing the MMAs into two TMEM accumulators, twelve epilogue warps staging the outputs in shared
// memory for TMA tensor stores.
// Other strides take gemm_kernel, one tile per CTA with the operands gathered element by element.  The
// training pass keeps every operand K-major: its epilogues also write the transposes that the weight
// gradients read.  Epilogues: plain store; addition into the output (the weight gradients' split-K
// partial products, by TMA reduce-adds); bias + GELU with a BF16 activation (and its transpose) and, for
// training, the GELU derivative at the pre-activation; or the backward's product with that derivative
// (and its transpose).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "fpt_kernels.h"
#include "mlp.h"
#include "tc.cuh"

namespace fpt {

constexpr int kGemmKC = 64;                  // K per chunk
constexpr uint32_t kWaitNs = 1000000000u;   // mbarrier waits give up after 1 s
constexpr int ERR_MMA_TIMEOUT = 3;

// GELU in its tanh form (Hendrycks and Gimpel, arXiv:1606.08415):
//   gelu(z) = z/2 (1 + tanh(u)),  u = sqrt(2/pi) (z + 0.044715 z^3),
// with the hardware tanh approximation (PTX tanh.approx.f32, relative error
// about 2^-11, below the BF16 rounding that follows every activation).  One
// MUFU operation per activation: the epilogues of the inference kernel
// evaluate 768 of them per path.
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// u = z (K0 + K0 K1 z^2) and gelu = h + h tanh(u) with h = z/2: six operations.
constexpr float kGeluK0 = 0.79788456080286536f;  // sqrt(2 / pi)
constexpr float kGeluK1 = 0.044715f;
constexpr float kGeluK01 = 0.0356774081363001f;  // K0 K1
__device__ __forceinline__ float gelu(float z) {
  const float h = 0.5f * z;
  return fmaf(h, tanh_approx(z * fmaf(kGeluK01, z * z, kGeluK0)), h);
}
// gelu(z) and, in d, its derivative gelu'(z) = (1 + th) / 2 + (z / 2) (1 - th^2) K0 (1 + 3 K1 z^2), from one
// tanh.  The training forward keeps gelu'(Z) for the backward (dZ = dH gelu'(Z)), so the backward's
// epilogue multiplies instead of evaluating the derivative again.
__device__ __forceinline__ float gelu_with_grad(float z, float& d) {
  const float z2 = z * z;
  const float th = tanh_approx(z * fmaf(kGeluK01, z2, kGeluK0));
  const float h = 0.5f * z;
  d = 0.5f * (1.f + th) + 0.5f * z * (1.f - th * th) * kGeluK0 * fmaf(3.f * kGeluK1, z2, 1.f);
  return fmaf(h, th, h);
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

// 16 bytes global -> shared, asynchronous (cp.async), the bytes past src_bytes (0..16) zero-filled.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kPending>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(kPending) : "memory");
}

// Rows [r0, r0 + rows) x k [k0, k0 + 64) of a row-major bf16 matrix whose rows start on 16-byte
// boundaries into the K-major tile layout, with asynchronous 16-byte copies (zero outside rows < R,
// k < K).  Consecutive threads take consecutive 16-byte pieces of a row: a warp reads four whole rows.
__device__ __forceinline__ void load_tile_async(unsigned char* tile, const __nv_bfloat16* src, long long s_r, int R,
                                                int K, int r0, int k0, int rows) {
  for (int idx = threadIdx.x; idx < rows * (kGemmKC / 8); idx += blockDim.x) {
    const int r = idx / (kGemmKC / 8), kg = idx % (kGemmKC / 8);
    const int gr = r0 + r, gk = k0 + kg * 8;
    const int valid = gr < R ? min(max(K - gk, 0), 8) : 0;
    const __nv_bfloat16* p = valid ? src + (long long)gr * s_r + gk : src;
    cp_async16(tile + tc::kmajor_offset(r, kg * 8, kGemmKC), p, (uint32_t)valid * 2u);
  }
}

// Operands that the pipelined path takes: unit stride along k, rows 16-byte aligned.
__host__ __device__ inline bool gemm_vectorised(const GemmArgs& g) {
  const bool a = g.sak == 1 && (g.sam % 8) == 0 && (reinterpret_cast<uintptr_t>(g.A) & 15) == 0;
  const bool b = g.sbk == 1 && (g.sbn % 8) == 0 && (reinterpret_cast<uintptr_t>(g.B) & 15) == 0;
  return a && b;
}

constexpr int kGemmStages = 2;                                      // K chunks in flight
constexpr int kGemmTileA = 128 * kGemmKC * 2;                       // 16 KB
constexpr int kGemmStageBytes = kGemmTileA + 256 * kGemmKC * 2;     // A + B (N <= 256): 48 KB
constexpr int kGemmSmem = kGemmStages * kGemmStageBytes;            // 96 KB: two CTAs per SM
// Epilogue staging: each warp's 32 accumulator rows, 64 columns at a time, in a private slab of the
// (by then idle) pipeline buffers; rows padded to 65 floats so that both the row-wise and the
// column-wise passes hit 32 different banks.
constexpr int kEpiCols = 64, kEpiStride = kEpiCols + 1;
static_assert(4 * 32 * kEpiStride * 4 <= kGemmSmem, "epilogue slabs");

// Epilogue of one warp's 32 accumulator rows (TMEM lanes 32 w .. 32 w + 31, matrix rows mrow0 ..).  Per
// 64-column slab: (a) the accumulator (+ bias) goes from TMEM to the warp's staging slab, lane = row;
// (b) row by row, consecutive lanes on consecutive columns, the row-major outputs are formed and stored
// (coalesced; Zin read the same way), and the final value is kept in the slab; (c) column by column,
// consecutive lanes on consecutive rows, the transposed copy Ht is stored (coalesced too).
__device__ __forceinline__ void gemm_epilogue_staged(const GemmArgs& g, uint32_t tmem_warp, int mrow0, int lane,
                                                     int n_pad, float* slab) {
  for (int c0 = 0; c0 < n_pad; c0 += kEpiCols) {
    const int cols = min(kEpiCols, n_pad - c0);
    for (int cc = 0; cc < cols; cc += 16) {
      float v[16];
      tc::tmem_ld16(tmem_warp + (uint32_t)(c0 + cc), v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int n = c0 + cc + q;
        float x = v[q];
        if ((g.op == EPI_STORE || g.op == EPI_BIAS_GELU) && g.bias && n < g.N) x += g.bias[n];
        slab[lane * kEpiStride + cc + q] = x;
      }
    }
    __syncwarp();
    for (int r = 0; r < 32; ++r) {
      const int m = mrow0 + r;
      if (m >= g.M) break;  // r is the same for the whole warp
      for (int cc = lane; cc < cols; cc += 32) {
        const int n = c0 + cc;
        if (n >= g.N) continue;
        const float x = slab[r * kEpiStride + cc];
        float y = x;
        switch (g.op) {
          case EPI_STORE:
            g.C[(long long)m * g.scm + (long long)n * g.scn] = x;
            break;
          case EPI_ATOMIC:
            atomicAdd(g.C + (long long)m * g.scm + (long long)n * g.scn, x);
            break;
          case EPI_BIAS_GELU: {
            float d;
            y = __bfloat162float(__float2bfloat16(gelu_with_grad(x, d)));
            if (g.C) g.C[(long long)m * g.scm + (long long)n * g.scn] = d;
            g.H[(long long)m * g.shm + (long long)n * g.shn] = __float2bfloat16(y);
            break;
          }
          case EPI_GELU_GRAD:
            y = x * g.Zin[(long long)m * g.szm + (long long)n * g.szn];
            if (g.C) g.C[(long long)m * g.scm + (long long)n * g.scn] = y;
            g.H[(long long)m * g.shm + (long long)n * g.shn] = __float2bfloat16(y);
            break;
        }
        slab[r * kEpiStride + cc] = y;
      }
    }
    __syncwarp();
    if (g.op == EPI_GELU_GRAD && g.colsum) {  // this warp's rows of each column (rows past M hold no value)
      const int rows = min(32, g.M - mrow0);
      for (int cc = lane; cc < cols; cc += 32) {
        if (c0 + cc >= g.N) continue;
        float acc = 0.f;
        for (int r = 0; r < rows; ++r) acc += slab[r * kEpiStride + cc];
        atomicAdd(g.colsum + c0 + cc, acc);
      }
    }
    if (g.Ht) {
      const int m = mrow0 + lane;
      for (int cc = 0; cc < cols; ++cc) {
        const int n = c0 + cc;
        if (n < g.N && m < g.M)
          g.Ht[(long long)m * g.shtm + (long long)n * g.shtn] = __float2bfloat16(slab[lane * kEpiStride + cc]);
      }
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(128) gemm_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char gemm_smem[];
  __shared__ __align__(8) uint64_t bar[kGemmStages];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128;
  const int n_pad = (g.N + 15) & ~15;
  const uint32_t ncols = n_pad <= 32 ? 32 : (n_pad <= 64 ? 64 : (n_pad <= 128 ? 128 : 256));
  // K range of this split
  const int k_per = ((g.K + gridDim.y * kGemmKC - 1) / (gridDim.y * kGemmKC)) * kGemmKC;
  const int kb = blockIdx.y * k_per, ke = min(g.K, kb + k_per);
  const int n_chunks = ke > kb ? (ke - kb + kGemmKC - 1) / kGemmKC : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGemmStages; ++s) tc::mbar_init(&bar[s], 1);
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
  auto stage_a = [&](int s) { return gemm_smem + s * kGemmStageBytes; };
  auto stage_b = [&](int s) { return gemm_smem + s * kGemmStageBytes + kGemmTileA; };
  auto issue = [&](int c) {  // one thread: the four MMAs of chunk c, then its commit
    const int s = c % kGemmStages;
    tc::fence_after_sync();
    const uint32_t a0 = tc::smem_u32(stage_a(s)), b0 = tc::smem_u32(stage_b(s));
#pragma unroll
    for (int kk = 0; kk < kGemmKC / 16; ++kk) {
      const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, (kGemmKC / 8) * 128);
      const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, (kGemmKC / 8) * 128);
      tc::mma_bf16(tmem, ad, bd, idesc, (c | kk) ? 1u : 0u);
    }
    tc::mma_commit(&bar[s]);
  };
  // chunk c's MMAs have completed: its stage barrier's phase number c / kGemmStages.  A thread whose
  // bounded wait runs out sets s_fail, which every thread reads only after the next barrier.
  auto wait_chunk = [&](int c) {
    if (tc::mbar_wait(&bar[c % kGemmStages], (uint32_t)((c / kGemmStages) & 1), kWaitNs)) return true;
    atomicExch(&s_fail, 1);
    return false;
  };
  if (gemm_vectorised(g)) {
    // pipelined: chunks load (cp.async, one commit group per chunk) kGemmStages - 1 ahead of the MMAs
    for (int c = 0; c < kGemmStages - 1; ++c) {
      if (c < n_chunks) {
        load_tile_async(stage_a(c), g.A, g.sam, g.M, g.K, m0, kb + c * kGemmKC, 128);
        load_tile_async(stage_b(c), g.B, g.sbn, g.N, g.K, 0, kb + c * kGemmKC, n_pad);
      }
      cp_async_commit();
    }
    for (int c = 0; c < n_chunks; ++c) {
      cp_async_wait<kGemmStages - 2>();  // this thread's copies of chunk c (group c) have landed
      tc::fence_async_smem();
      __syncthreads();
      if (s_fail) break;  // the same value for every thread after the barrier
      if (threadIdx.x == 0) issue(c);
      // refill the stage of chunk c - 1 with chunk c + kGemmStages - 1 once chunk c - 1's MMAs, queued ahead
      // of chunk c's, have read it
      const int cn = c + kGemmStages - 1;
      if (cn < n_chunks && (c == 0 || wait_chunk(c - 1))) {
        const int sn = cn % kGemmStages;
        load_tile_async(stage_a(sn), g.A, g.sam, g.M, g.K, m0, kb + cn * kGemmKC, 128);
        load_tile_async(stage_b(sn), g.B, g.sbn, g.N, g.K, 0, kb + cn * kGemmKC, n_pad);
      }
      cp_async_commit();
    }
    cp_async_wait<0>();
  } else {
    // element gathers from arbitrary strides: one stage, each chunk waited for before the next
    for (int c = 0; c < n_chunks; ++c) {
      load_tile(stage_a(0), g.A, g.sam, g.sak, g.M, g.K, m0, kb + c * kGemmKC, 128);
      load_tile(stage_b(0), g.B, g.sbn, g.sbk, g.N, g.K, 0, kb + c * kGemmKC, n_pad);
      tc::fence_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) {
        const int s = c % kGemmStages;
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(stage_a(0)), b0 = tc::smem_u32(stage_b(0));
#pragma unroll
        for (int kk = 0; kk < kGemmKC / 16; ++kk) {
          const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, (kGemmKC / 8) * 128);
          const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, (kGemmKC / 8) * 128);
          tc::mma_bf16(tmem, ad, bd, idesc, (c | kk) ? 1u : 0u);
        }
        tc::mma_commit(&bar[s]);
      }
      wait_chunk(c);  // the tile is reused by the next chunk
      tc::fence_after_sync();
      __syncthreads();
      if (s_fail) break;
    }
  }
  __syncthreads();
  if (n_chunks > 0 && !s_fail) wait_chunk(n_chunks - 1);  // the last commit: every MMA has completed
  tc::fence_after_sync();
  __syncthreads();
  if (s_fail) {
    if (threadIdx.x == 0 && g.err) atomicCAS(g.err, 0, ERR_MMA_TIMEOUT);
    // give MMAs still in flight a (bounded) chance to finish before TMEM is freed
    if (n_chunks > 0) tc::mbar_wait(&bar[(n_chunks - 1) % kGemmStages], (uint32_t)(((n_chunks - 1) / kGemmStages) & 1),
                                    kWaitNs);
  } else if (n_chunks > 0) {
    // epilogue: warp w owns TMEM lanes (rows) 32 w .. 32 w + 31; the pipeline buffers are idle now
    float* slab = reinterpret_cast<float*>(gemm_smem) + warp * 32 * kEpiStride;
    gemm_epilogue_staged(g, tmem + ((uint32_t)(warp * 32) << 16), m0 + warp * 32, lane, n_pad, slab);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---- persistent warp-specialised GEMM (TMA operands) -------------------------------------------------
// One CTA per SM walks the (128-row tile, K split) items.  Warp 0 (one thread) loads each 64-wide K chunk
// of A (128 rows) and B (n_pad rows) with one TMA tile load per operand into a ring of kWsStages stages,
// in the 128-byte swizzled K-major layout; rows past M or N and k past K arrive as zeros.  Warp 1 (one
// thread) issues four 128 x n_pad x 16 MMAs per chunk into one of two TMEM accumulators (columns 0-255,
// 256-511), releases the chunk's stage by a commit to `empty` and announces a finished tile by a commit
// to `acc_full`.  Warps 2-13 are the epilogue: three warps per 32-lane quarter of TMEM (a warp may read the
// quarter given by its index mod 4), each on every third group of 16 columns, one output row per lane.
// Each 32 x 16 group is staged in shared memory and written by TMA tensor stores (full lines, no
// per-lane store traffic); outputs whose strides a tensor map cannot describe are stored by the lanes.
// The warps hand the accumulator back through `acc_empty`, so the MMAs of the tile after next may start
// while this tile's epilogue runs.  Every wait is bounded; a timeout sets the CTA's fail flag, which every
// role polls and leaves on.
constexpr int kWsStages = 2;     // operand ring stages when the epilogue stages BF16 outputs
constexpr int kWsStagesMax = 3;  // ... and when it stages only the FP32 box (plain stores, reduce-adds)
constexpr int kWsEpiWarps = 12;
constexpr int kWsGroupStride = kWsEpiWarps / 4;  // epilogue warps per 32-lane quarter of TMEM
constexpr int kWsThreads = 32 * (2 + kWsEpiWarps);
constexpr int kWsTileA = 128 * 128;                       // 128 rows x 128 bytes
constexpr int kWsStageBytes = kWsTileA + 256 * 128;       // + B, up to 256 rows: 48 KB
// the ring, two 4 KB output staging buffers per epilogue warp, slack to align the ring to 1024 bytes
constexpr int kWsSmem = kWsStages * kWsStageBytes + kWsEpiWarps * 2 * 4096 + 1024;
static_assert(kWsStagesMax * kWsStageBytes + kWsEpiWarps * 2 * 2048 + 1024 <= kWsSmem, "ring and staging");

struct WsItem {
  int m0, kb, ke, split;
};
__device__ __forceinline__ WsItem ws_item(const GemmArgs& g, int item, int m_tiles, int k_per) {
  WsItem w;
  w.m0 = (item % m_tiles) * 128;
  w.split = item / m_tiles;
  w.kb = w.split * k_per;
  w.ke = min(g.K, w.kb + k_per);
  return w;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Which outputs may use 16-byte vector accesses (unit stride along n, row strides and bases aligned).
struct EpiVec {
  bool c, h, z, bias;
};
__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
__device__ __forceinline__ EpiVec epi_vec(const GemmArgs& g) {
  EpiVec v;
  v.c = g.scn == 1 && g.scm % 4 == 0 && aligned16(g.C);
  v.h = g.shn == 1 && g.shm % 8 == 0 && aligned16(g.H);
  v.z = g.szn == 1 && g.szm % 4 == 0 && aligned16(g.Zin);
  v.bias = aligned16(g.bias);
  return v;
}

__device__ __forceinline__ void store16_f32(float* p, const float (&x)[16], bool vec, int nv, long long sn) {
  if (vec) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (i < nv) p[i * sn] = x[i];
  }
}
__device__ __forceinline__ void store16_bf16(__nv_bfloat16* p, const float (&x)[16], bool vec, int nv, long long sn) {
  if (vec) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&b2);
    }
    uint4* q = reinterpret_cast<uint4*>(p);
    q[0] = make_uint4(w[0], w[1], w[2], w[3]);
    q[1] = make_uint4(w[4], w[5], w[6], w[7]);
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (i < nv) p[i * sn] = __float2bfloat16(x[i]);
  }
}

// Sum of x[i] over the warp's 32 lanes for each of the 16 columns i: a transposing butterfly (16 shuffles).
// Returns the sum of column ((lane >> 1) & 8) | ((lane >> 1) & 4) | ((lane >> 1) & 2) | ((lane >> 1) & 1),
// i.e. column lane / 2 in bit-reversed halves: lane bits 4, 3, 2, 1 select column bits 3, 2, 1, 0.
__device__ __forceinline__ float warp_colsum16(const float (&x)[16], int lane) {
  float a[8], b[4], c[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float send = h16 ? x[i] : x[i + 8];
    const float keep = h16 ? x[i + 8] : x[i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = h8 ? a[i] : a[i + 4];
    const float keep = h8 ? a[i + 4] : a[i];
    b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h4 ? b[i] : b[i + 2];
    const float keep = h4 ? b[i + 2] : b[i];
    c[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const float d = (h2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h2 ? c[0] : c[1], 2);
  return d + __shfl_xor_sync(0xffffffffu, d, 1);
}
__device__ __forceinline__ int warp_colsum16_column(int lane) {
  return ((lane >> 1) & 8) | ((lane >> 1) & 4) | ((lane >> 1) & 2) | ((lane >> 1) & 1);
}

// Z[m][n0 .. n0 + 15] (zero past N or M) into registers; 16-byte loads when aligned and whole.
__device__ __forceinline__ void load_z16(const GemmArgs& g, const EpiVec& ev, int m, bool row, int n0, float (&z)[16]) {
  const float* zp = g.Zin + (long long)m * g.szm + (long long)n0 * g.szn;
  const int nv = min(16, g.N - n0);
  if (row && nv == 16 && ev.z) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(zp) + i);
      z[4 * i] = t.x;
      z[4 * i + 1] = t.y;
      z[4 * i + 2] = t.z;
      z[4 * i + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = row && i < nv ? zp[i * g.szn] : 0.f;
  }
}

// Staging of one warp's 32 x 16 output group for the TMA tensor stores (two buffers per warp, used in
// turn): the FP32 box in the 64-byte swizzled layout (row r, 16-byte chunk c at r 64 + 16 (c ^ (r / 2 mod 4))),
// the BF16 box in the 32-byte swizzled layout (r 32 + 16 (c ^ (r / 4 mod 2))), the transposed BF16 box
// plainly (column n of the group at n 64, row r at 2 r).  Consecutive lanes (rows) hit different banks
// in all three.
constexpr int kStgC = 0, kStgH = 2048, kStgHt = 3072, kStgBytes = 4096;
constexpr int kOutC = 1, kOutH = 2, kOutHt = 4;  // outputs that go through TMA stores
constexpr int kOutCt = 8;  // EPI_ATOMIC into a column-major destination: the FP32 box staged transposed

struct OutMaps {
  const CUtensorMap* c;
  const CUtensorMap* h;
  const CUtensorMap* ht;
  int flags;
};

// One warp's share of a finished 128 x n_pad accumulator: its lane quarter, column groups j0, j0 + kWsGroupStride, ...
// m = this lane's output row, mrow0 = the warp's first row.  Each output goes out through a TMA store of the
// staged group when its tensor map exists (flags), else with this lane's own stores.  gi counts the warp's
// groups (it picks the staging buffer).  For EPI_GELU_GRAD the pre-activations of the next group are
// loaded while the current one is worked on, and the column sums of dZ are added to s_col.
template <int OP>
__device__ __forceinline__ void ws_epilogue(const GemmArgs& g, const EpiVec& ev, uint32_t tacc, int m, int mrow0,
                                            int j0, int n_groups, float* s_col, const OutMaps& om,
                                            unsigned char* stg, int stg_bytes, int& gi) {
  const int lane = lane_id();
  const bool row = m < g.M;
  const bool has_c = OP == EPI_STORE || OP == EPI_ATOMIC || g.C != nullptr;
  const bool has_h = OP == EPI_BIAS_GELU || OP == EPI_GELU_GRAD;
  const bool has_ht = has_h && g.Ht != nullptr;
  const bool tma_c = has_c && (om.flags & (kOutC | kOutCt)), tma_h = has_h && (om.flags & kOutH),
             tma_ht = has_ht && (om.flags & kOutHt);
  const bool any_tma = tma_c || tma_h || tma_ht;
  float zq[16];  // the pre-activations of the next column group (EPI_GELU_GRAD)
  if (OP == EPI_GELU_GRAD && j0 < n_groups) load_z16(g, ev, m, row, 16 * j0, zq);
  for (int j = j0; j < n_groups; j += kWsGroupStride) {
    const int n0 = 16 * j;
    const int nv = min(16, g.N - n0);
    const bool full = nv == 16;
    float x[16];
    __syncwarp();
    tc::tmem_ld16(tacc + (uint32_t)n0, x);
    if ((OP == EPI_STORE || OP == EPI_BIAS_GELU) && g.bias) {
      if (full && ev.bias) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 b = __ldg(reinterpret_cast<const float4*>(g.bias + n0) + i);
          x[4 * i] += b.x;
          x[4 * i + 1] += b.y;
          x[4 * i + 2] += b.z;
          x[4 * i + 3] += b.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (i < nv) x[i] += g.bias[n0 + i];
      }
    }
    float h[16];  // the BF16 output (rounded when stored): the activation, or dZ
    if (OP == EPI_GELU_GRAD) {
      float z[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) z[i] = zq[i];
      if (j + kWsGroupStride < n_groups) load_z16(g, ev, m, row, 16 * (j + kWsGroupStride), zq);
#pragma unroll
      for (int i = 0; i < 16; ++i) x[i] = row ? x[i] * z[i] : 0.f;
      if (s_col) {
        const float cs = warp_colsum16(x, lane);
        if ((lane & 1) == 0) {
          const int c = warp_colsum16_column(lane);
          if (c < nv) atomicAdd(s_col + n0 + c, cs);
        }
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) h[i] = x[i];
    } else if (OP == EPI_BIAS_GELU) {
      if (has_c) {  // training: the FP32 output is gelu'(Z) for the backward
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float d;
          h[i] = gelu_with_grad(x[i], d);
          x[i] = d;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) h[i] = gelu(x[i]);
      }
    }
    // this lane's own stores for the outputs without a tensor map
    if (row) {
      if (has_c && !tma_c) {
        if (OP == EPI_ATOMIC) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (i < nv) atomicAdd(g.C + (long long)m * g.scm + (long long)(n0 + i) * g.scn, x[i]);
        } else {
          store16_f32(g.C + (long long)m * g.scm + (long long)n0 * g.scn, x, full && ev.c, nv, g.scn);
        }
      }
      if (has_h && !tma_h) store16_bf16(g.H + (long long)m * g.shm + (long long)n0 * g.shn, h, full && ev.h, nv, g.shn);
      if (has_ht && !tma_ht) {
        __nv_bfloat16* tp = g.Ht + (long long)m * g.shtm + (long long)n0 * g.shtn;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (i < nv) tp[i * g.shtn] = __float2bfloat16(h[i]);
      }
    }
    if (!any_tma) continue;
    // the staged group: wait until the engine has read this buffer's previous group, fill it, store it
    unsigned char* buf = stg + (gi & 1) * stg_bytes;
    ++gi;
    if (lane == 0) tc::bulk_wait_read<1>();
    __syncwarp();
    if (tma_c && (om.flags & kOutCt)) {  // column n of the group at n 128 bytes, row r at 4 r
      float* tb = reinterpret_cast<float*>(buf + kStgC) + lane;
#pragma unroll
      for (int i = 0; i < 16; ++i) tb[32 * i] = x[i];
    } else if (tma_c) {
      unsigned char* cb = buf + kStgC + lane * 64;
      const int sw = (lane >> 1) & 3;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        *reinterpret_cast<float4*>(cb + 16 * (c ^ sw)) = make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
    }
    if (tma_h) {
      unsigned char* hb = buf + kStgH + lane * 32;
      const int sw = (lane >> 2) & 1;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const __nv_bfloat162 b2 = __floats2bfloat162_rn(h[8 * c + 2 * i], h[8 * c + 2 * i + 1]);
          w[i] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        *reinterpret_cast<uint4*>(hb + 16 * (c ^ sw)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    if (tma_ht) {
      __nv_bfloat16* tb = reinterpret_cast<__nv_bfloat16*>(buf + kStgHt) + lane;
#pragma unroll
      for (int i = 0; i < 16; ++i) tb[32 * i] = __float2bfloat16(h[i]);
    }
    tc::fence_async_smem();
    __syncwarp();
    if (lane == 0 && mrow0 < g.M) {
      if (tma_c) {
        if (OP == EPI_ATOMIC) {
          if (om.flags & kOutCt)
            tc::tma_reduce_add_2d(om.c, buf + kStgC, mrow0, n0);
          else
            tc::tma_reduce_add_2d(om.c, buf + kStgC, n0, mrow0);
        } else {
          tc::tma_store_2d(om.c, buf + kStgC, n0, mrow0);
        }
      }
      if (tma_h) tc::tma_store_2d(om.h, buf + kStgH, n0, mrow0);
      if (tma_ht) tc::tma_store_2d(om.ht, buf + kStgHt, mrow0, n0);
      tc::bulk_commit();
    }
  }
}

__global__ void __launch_bounds__(kWsThreads, 1)
    gemm_ws_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmH,
                   const __grid_constant__ CUtensorMap tmHt, int out_flags, GemmArgs g, int m_tiles, int n_items,
                   int k_per) {
  extern __shared__ unsigned char ws_raw[];
  __shared__ __align__(8) uint64_t full[kWsStagesMax], empty[kWsStagesMax], acc_full[2], acc_empty[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  __shared__ int s_last_q;             // the MMA thread's last committed chunk (-1: none)
  __shared__ int s_armed[kWsStagesMax];  // each stage's last phase handed to the TMA engine (-1: none)
  __shared__ float s_col[256];         // this CTA's column sums (EPI_GELU_GRAD with colsum)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned all = 0xffffffffu;
  const int n_pad = (g.N + 15) & ~15;
  // outputs staged only in the FP32 slot leave room for a deeper operand ring (long K of the weight
  // gradients); the BF16 outputs need the whole 4 KB staging buffers
  const bool fp32_only = g.op == EPI_STORE || g.op == EPI_ATOMIC;
  const int stages = fp32_only ? kWsStagesMax : kWsStages;
  const int stg_bytes = fp32_only ? 2048 : kStgBytes;
  unsigned char* ring = ws_raw + ((1024u - (tc::smem_u32(ws_raw) & 1023u)) & 1023u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kWsStagesMax; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
      s_armed[s] = -1;
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kWsEpiWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    s_last_q = -1;
  }
  const bool want_col = g.op == EPI_GELU_GRAD && g.colsum != nullptr;
  if (want_col)
    for (int k = threadIdx.x; k < 256; k += blockDim.x) s_col[k] = 0.f;
  if (warp == 0) {
    tc::tmem_alloc(&s_tmem, 512);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  auto stage_a = [&](int s) { return ring + s * kWsStageBytes; };
  auto stage_b = [&](int s) { return ring + s * kWsStageBytes + kWsTileA; };
  auto failed = [&]() { return *reinterpret_cast<volatile int*>(&s_fail) != 0; };

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      const uint32_t tx_bytes = (uint32_t)(128 + n_pad) * 128u;
      int q = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
        const WsItem w = ws_item(g, item, m_tiles, k_per);
        for (int k0 = w.kb; k0 < w.ke; k0 += kGemmKC, ++q) {
          const int s = q % stages, u = q / stages;
          if (u > 0) {  // the stage's previous chunk has been read by its MMAs
            ok = !failed() && tc::mbar_wait(&empty[s], (uint32_t)((u - 1) & 1), kWaitNs);
            if (!ok) break;
          }
          tc::mbar_expect_tx(&full[s], tx_bytes);
          s_armed[s] = u;
          tc::tma_load_2d(stage_a(s), &tmA, k0, w.m0, &full[s]);
          tc::tma_load_2d(stage_b(s), &tmB, k0, 0, &full[s]);
        }
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int q = 0, i = 0;
      bool ok = true;
      const uint32_t idesc = tc::idesc_bf16(128, (uint32_t)n_pad);
      for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x, ++i) {
        const WsItem w = ws_item(g, item, m_tiles, k_per);
        const int b = i & 1, v = i >> 1;
        if (v > 0) ok = !failed() && tc::mbar_wait(&acc_empty[b], (uint32_t)((v - 1) & 1), kWaitNs);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(b * 256);
        for (int k0 = w.kb, c = 0; k0 < w.ke; k0 += kGemmKC, ++q, ++c) {
          const int s = q % stages, u = q / stages;
          ok = !failed() && tc::mbar_wait(&full[s], (uint32_t)(u & 1), kWaitNs);
          if (!ok) break;
          tc::fence_after_sync();
          const uint64_t ad = tc::smem_desc_sw128(tc::smem_u32(stage_a(s)));
          const uint64_t bd = tc::smem_desc_sw128(tc::smem_u32(stage_b(s)));
#pragma unroll
          for (int kk = 0; kk < kGemmKC / 16; ++kk)
            tc::mma_bf16(d, ad + 2u * kk, bd + 2u * kk, idesc, (c | kk) ? 1u : 0u);
          tc::mma_commit(&empty[s]);
          s_last_q = q;
        }
        if (!ok) break;
        tc::mma_commit(&acc_full[b]);
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
    __syncwarp();
  } else {
    // ---- epilogue ----
    const int quarter = warp & 3;            // the TMEM lanes this warp may read
    const int j0 = (warp - 2) >> 2;          // its column groups: j0, j0 + kWsGroupStride, ...
    const int n_groups = n_pad / 16;
    const EpiVec ev = epi_vec(g);
    const OutMaps om{&tmC, &tmH, &tmHt, out_flags};
    unsigned char* stg = ring + stages * kWsStageBytes + (warp - 2) * 2 * stg_bytes;
    int gi = 0;
    int i = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++i) {
      const WsItem w = ws_item(g, item, m_tiles, k_per);
      const int b = i & 1, v = i >> 1;
      const bool ok = __all_sync(all, !failed() && tc::mbar_wait(&acc_full[b], (uint32_t)(v & 1), kWaitNs));
      if (!ok) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      tc::fence_after_sync();
      const uint32_t tacc = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
      const int mrow0 = w.m0 + quarter * 32;
      const int m = mrow0 + lane;
      switch (g.op) {
        case EPI_STORE:
          ws_epilogue<EPI_STORE>(g, ev, tacc, m, mrow0, j0, n_groups, nullptr, om, stg, stg_bytes, gi);
          break;
        case EPI_ATOMIC:
          ws_epilogue<EPI_ATOMIC>(g, ev, tacc, m, mrow0, j0, n_groups, nullptr, om, stg, stg_bytes, gi);
          break;
        case EPI_BIAS_GELU:
          ws_epilogue<EPI_BIAS_GELU>(g, ev, tacc, m, mrow0, j0, n_groups, nullptr, om, stg, stg_bytes, gi);
          break;
        default:
          ws_epilogue<EPI_GELU_GRAD>(g, ev, tacc, m, mrow0, j0, n_groups, want_col ? s_col : nullptr, om,
                                     stg, stg_bytes, gi);
          break;
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
    // every TMA store of this warp has completed before its staging buffers go away
    if (lane == 0) tc::bulk_wait_all();
    __syncwarp();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (s_fail && threadIdx.x == 0) {
    if (g.err) atomicCAS(g.err, 0, ERR_MMA_TIMEOUT);
    // let the copies and MMAs already issued finish (bounded) before shared and tensor memory go away
    for (int s = 0; s < stages; ++s)
      if (s_armed[s] >= 0) tc::mbar_wait(&full[s], (uint32_t)(s_armed[s] & 1), kWaitNs);
    const int q = s_last_q;
    if (q >= 0) tc::mbar_wait(&empty[q % stages], (uint32_t)((q / stages) & 1), kWaitNs);
  }
  __syncthreads();
  if (want_col && !s_fail)
    for (int k = threadIdx.x; k < g.N; k += blockDim.x) atomicAdd(g.colsum + k, s_col[k]);
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// A tiled tensor map of `rank` dimensions (dims innermost first, strides in bytes for dimensions 1..),
// elements outside the tensor read as zero and are not written.
static bool encode_map(CUtensorMap* map, CUtensorMapDataType type, int rank, const void* base, const cuuint64_t* dims,
                       const cuuint64_t* strides, const cuuint32_t* box, CUtensorMapSwizzle swizzle) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  for (int d = 0; d + 1 < rank; ++d)
    if (strides[d] % 16 != 0) return false;
  const cuuint32_t elem[3] = {1, 1, 1};
  return enc(map, type, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, elem,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The {k, row} view of a row-major BF16 matrix (rows x K, row stride ld elements) in 64 x box_rows boxes
// with 128-byte swizzling.
static bool encode_operand(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, long long ld, int box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2u};
  const cuuint32_t box[2] = {(cuuint32_t)kGemmKC, (cuuint32_t)box_rows};
  return encode_map(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

// Tensor maps of the epilogue's outputs (32-row x 16-column boxes, laid out as the staging buffers are);
// returns the kOut* flags of the outputs that have one.
static int encode_outputs(const GemmArgs& g, CUtensorMap* tmC, CUtensorMap* tmH, CUtensorMap* tmHt) {
  int flags = 0;
  if (g.op == EPI_ATOMIC) {
    if (g.scn == 1) {  // row-major destination: boxes as the FP32 stores
      const cuuint64_t dims[2] = {(cuuint64_t)g.N, (cuuint64_t)g.M};
      const cuuint64_t strides[1] = {(cuuint64_t)g.scm * 4u};
      const cuuint32_t box[2] = {16, 32};
      if (encode_map(tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, g.C, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B))
        flags |= kOutC;
    } else if (g.scm == 1) {  // column-major destination: the transposed box
      const cuuint64_t dims[2] = {(cuuint64_t)g.M, (cuuint64_t)g.N};
      const cuuint64_t strides[1] = {(cuuint64_t)g.scn * 4u};
      const cuuint32_t box[2] = {32, 16};
      if (encode_map(tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, g.C, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE))
        flags |= kOutCt;
    }
  } else if (g.C && g.scn == 1) {
    const cuuint64_t dims[2] = {(cuuint64_t)g.N, (cuuint64_t)g.M};
    const cuuint64_t strides[1] = {(cuuint64_t)g.scm * 4u};
    const cuuint32_t box[2] = {16, 32};
    if (encode_map(tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, g.C, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B))
      flags |= kOutC;
  }
  if ((g.op == EPI_BIAS_GELU || g.op == EPI_GELU_GRAD) && g.H && g.shn == 1) {
    const cuuint64_t dims[2] = {(cuuint64_t)g.N, (cuuint64_t)g.M};
    const cuuint64_t strides[1] = {(cuuint64_t)g.shm * 2u};
    const cuuint32_t box[2] = {16, 32};
    if (encode_map(tmH, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.H, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_32B))
      flags |= kOutH;
  }
  if ((g.op == EPI_BIAS_GELU || g.op == EPI_GELU_GRAD) && g.Ht && g.shtm == 1) {
    const cuuint64_t dims[2] = {(cuuint64_t)g.M, (cuuint64_t)g.N};
    const cuuint64_t strides[1] = {(cuuint64_t)g.shtn * 2u};
    const cuuint32_t box[2] = {32, 16};
    if (encode_map(tmHt, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.Ht, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_NONE))
      flags |= kOutHt;
  }
  return flags;
}

cudaError_t launch_gemm(const GemmArgs& g, int k_split, cudaStream_t stream) {
  if (g.N < 1 || g.N > 256 || g.M < 1 || g.K < 1 || k_split < 1) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(gemm_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (gemm_vectorised(g)) {
    const int n_pad = (g.N + 15) & ~15;
    CUtensorMap tmA, tmB;
    if (encode_operand(&tmA, g.A, g.M, g.K, g.sam, 128) && encode_operand(&tmB, g.B, g.N, g.K, g.sbn, n_pad)) {
      // persistent: one CTA per SM over the (tile, split) items
      const int m_tiles = (g.M + 127) / 128;
      const int k_per = ((g.K + k_split * kGemmKC - 1) / (k_split * kGemmKC)) * kGemmKC;
      const int splits = (g.K + k_per - 1) / k_per;
      const int n_items = m_tiles * splits;
      int dev = 0, n_sm = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      const int grid = n_items < n_sm ? n_items : n_sm;
      CUtensorMap tmC{}, tmH{}, tmHt{};
      const int out_flags = encode_outputs(g, &tmC, &tmH, &tmHt);
      gemm_ws_kernel<<<grid, kWsThreads, kWsSmem, stream>>>(tmA, tmB, tmC, tmH, tmHt, out_flags, g, m_tiles, n_items,
                                                            k_per);
      count_launch();
      return cudaGetLastError();
    }
  }
  dim3 grid((g.M + 127) / 128, k_split);
  gemm_kernel<<<grid, 128, kGemmSmem, stream>>>(g);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// features, loss, bias gradients, Adam, learned start
// ---------------------------------------------------------------------------

// 64 features of one path (see include/fpt.h): origin o = (TX + RX)/2, scale S;
// per interaction the orthogonal projections of TX and RX onto the object's
// affine hull in its own parameters, their distances to it, the first basis
// length, and the distance-weighted combination of the two projections.  Also
// the per-slot Gram matrix A^T A / S^2 (g11, g12, g22) of the loss.
__device__ __forceinline__ void path_features(const SceneDev& S, const PathDesc& d, float inv_scale,
                                              __nv_bfloat16* f, float* G) {
  float tx[3], rx[3], o[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    tx[c] = S.tx32[kEnd32 * d.tx + c] + S.tx32[kEnd32 * d.tx + 3 + c];
    rx[c] = S.rx32[kEnd32 * d.rx + c] + S.rx32[kEnd32 * d.rx + 3 + c];
    o[c] = 0.5f * (tx[c] + rx[c]);
  }
  float v[kMlpIn], gram[12];
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) v[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 12; ++k) gram[k] = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[c] = (tx[c] - o[c]) * inv_scale;
    v[3 + c] = (rx[c] - o[c]) * inv_scale;
  }
  const bool valid = !(d.flags & ST_INVALID);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s < d.n && valid) {
      const float* r = S.rec32 + kRec32 * d.ids[s];
      const bool edge = S.aux[kAux * d.ids[s] + 2] != 0.f;
      float b[3], a1[3], a2[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        b[c] = r[c] + r[3 + c];
        a1[c] = r[6 + c];
        a2[c] = r[9 + c];
      }
      const float g11 = a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2];
      const float g12 = a1[0] * a2[0] + a1[1] * a2[1] + a1[2] * a2[2];
      const float g22 = a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2];
      const float det = g11 * g22 - g12 * g12;
      float tau[2][2], dist[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float* pt = q == 0 ? tx : rx;
        float rr[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) rr[c] = pt[c] - b[c];
        const float c1 = a1[0] * rr[0] + a1[1] * rr[1] + a1[2] * rr[2];
        const float c2 = a2[0] * rr[0] + a2[1] * rr[1] + a2[2] * rr[2];
        if (edge) {
          tau[q][0] = c1 / g11;
          tau[q][1] = 0.f;
        } else {
          tau[q][0] = (g22 * c1 - g12 * c2) / det;
          tau[q][1] = (g11 * c2 - g12 * c1) / det;
        }
        float e2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float e = rr[c] - tau[q][0] * a1[c] - tau[q][1] * a2[c];
          e2 += e * e;
        }
        dist[q] = sqrtf(e2) * inv_scale;
      }
      const int base = 6 + 11 * s;
      v[base] = 1.f;
      v[base + 1] = edge ? 1.f : 0.f;
      v[base + 2] = tau[0][0];
      v[base + 3] = tau[0][1];
      v[base + 4] = tau[1][0];
      v[base + 5] = tau[1][1];
      v[base + 6] = dist[0];
      v[base + 7] = dist[1];
      v[base + 8] = sqrtf(g11) * inv_scale;
      const float dsum = dist[0] + dist[1];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        v[base + 9 + k] = dsum > 0.f ? (dist[1] * tau[0][k] + dist[0] * tau[1][k]) / dsum
                                     : 0.5f * (tau[0][k] + tau[1][k]);
      const float is2 = inv_scale * inv_scale;
      gram[3 * s] = g11 * is2;
      gram[3 * s + 1] = g12 * is2;
      gram[3 * s + 2] = g22 * is2;
    }
  }
#pragma unroll
  for (int k = 0; k < kMlpIn; k += 8) {
    __nv_bfloat16 e[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) e[q] = __float2bfloat16(v[k + q]);
    *reinterpret_cast<uint4*>(f + k) = *reinterpret_cast<uint4*>(e);
  }
  if (G)
#pragma unroll
    for (int k = 0; k < 12; ++k) G[k] = gram[k];
}

// all paths of a batch (global index order) or one order slice (local index order)
__global__ void mlp_features_kernel(SceneDev S, BatchDev B, int n, const PathRec* list, uint64_t first,
                                    uint64_t count, float inv_scale, __nv_bfloat16* X, float* G) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (uint64_t)gridDim.x * blockDim.x) {
    PathDesc d;
    if (n > 0)
      fetch_path(B, n, list, first + k, d);
    else
      decode_global(B, first + k, d);
    path_features(S, d, inv_scale, X + k * kMlpIn, G ? G + k * 12 : nullptr);
  }
}

// loss (1/B) sum_b sum_s dy_s^T G_s dy_s (G_s = A_s^T A_s / S^2 per slot, zero for unused slots) and dY
// Per sample: d = Y[:8] - T, the Gram-weighted loss sum_s d_s^T G_s d_s and its gradient dY = (2 / B) G d
// (the padded outputs 8..15 get zero), in FP32, BF16 and transposed BF16.  vec: the rows of G, Y, T and the
// outputs start on 16-byte boundaries (16-byte loads and stores).
__global__ void mlp_loss_kernel(const float* __restrict__ G, const float* __restrict__ Y,
                                const float* __restrict__ T, uint64_t B, float* __restrict__ dY,
                                __nv_bfloat16* __restrict__ dYb, __nv_bfloat16* __restrict__ dYt, float* loss,
                                int vec) {
  float acc = 0.f;
  const float w = 2.f / (float)B;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (uint64_t)gridDim.x * blockDim.x) {
    float gm[12], y[8], t[8];
    if (vec) {
      const float4* gp = reinterpret_cast<const float4*>(G + b * 12);
      const float4* yp = reinterpret_cast<const float4*>(Y + b * kMlpOut);
      const float4* tp = reinterpret_cast<const float4*>(T + b * 8);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float4 v = __ldg(gp + q);
        gm[4 * q] = v.x;
        gm[4 * q + 1] = v.y;
        gm[4 * q + 2] = v.z;
        gm[4 * q + 3] = v.w;
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float4 v = yp[q], u = __ldg(tp + q);
        y[4 * q] = v.x;
        y[4 * q + 1] = v.y;
        y[4 * q + 2] = v.z;
        y[4 * q + 3] = v.w;
        t[4 * q] = u.x;
        t[4 * q + 1] = u.y;
        t[4 * q + 2] = u.z;
        t[4 * q + 3] = u.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 12; ++q) gm[q] = G[b * 12 + q];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        y[q] = Y[b * kMlpOut + q];
        t[q] = T[b * 8 + q];
      }
    }
    float g[kMlpOut];
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) g[k] = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float g11 = gm[3 * s], g12 = gm[3 * s + 1], g22 = gm[3 * s + 2];
      const float d0 = y[2 * s] - t[2 * s];
      const float d1 = y[2 * s + 1] - t[2 * s + 1];
      const float m0 = g11 * d0 + g12 * d1, m1 = g12 * d0 + g22 * d1;
      acc += d0 * m0 + d1 * m1;
      g[2 * s] = w * m0;
      g[2 * s + 1] = w * m1;
    }
    if (vec) {
      float4* dp = reinterpret_cast<float4*>(dY + b * kMlpOut);
#pragma unroll
      for (int q = 0; q < 4; ++q) dp[q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
      uint32_t wv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(g[2 * q], g[2 * q + 1]);
        wv[q] = *reinterpret_cast<const uint32_t*>(&b2);
      }
      uint4* bp = reinterpret_cast<uint4*>(dYb + b * kMlpOut);
      bp[0] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      bp[1] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
    } else {
#pragma unroll
      for (int k = 0; k < kMlpOut; ++k) {
        dY[b * kMlpOut + k] = g[k];
        dYb[b * kMlpOut + k] = __float2bfloat16(g[k]);
      }
    }
    if (dYt) {
#pragma unroll
      for (int k = 0; k < kMlpOut; ++k) dYt[(uint64_t)k * B + b] = __float2bfloat16(g[k]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / (float)B);
}

// out[n] += sum_b A[b][n]  (bias gradients), A: [B][N] row-major
// out[n] += sum_b A[b][n]: each thread one column and a strided set of rows (four sums in flight), then
// the block's row lanes combined in shared memory and one atomic per column and block.
__global__ void colsum_kernel(const float* __restrict__ A, uint64_t B, int N, float* out) {
  __shared__ float part[256];
  const int n = threadIdx.x % N;
  const int lanes = blockDim.x / N;
  const int rl = threadIdx.x / N;
  const uint64_t step = (uint64_t)gridDim.x * lanes;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  uint64_t b = (uint64_t)blockIdx.x * lanes + rl;
  if (rl < lanes) {
    for (; b + 3 * step < B; b += 4 * step) {
      a0 += A[b * N + n];
      a1 += A[(b + step) * N + n];
      a2 += A[(b + 2 * step) * N + n];
      a3 += A[(b + 3 * step) * N + n];
    }
    for (; b < B; b += step) a0 += A[b * N + n];
  }
  part[threadIdx.x] = rl < lanes ? (a0 + a1) + (a2 + a3) : 0.f;
  __syncthreads();
  if (threadIdx.x < N) {
    float acc = 0.f;
    for (int r = 0; r < lanes; ++r) acc += part[r * N + threadIdx.x];
    atomicAdd(out + threadIdx.x, acc);
  }
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr, float c1, float c2,
                            __nv_bfloat16* __restrict__ wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
  }
}

// dst [C][R] = src [R][C]^T through a 32 x 32 shared-memory tile (both sides coalesced)
__global__ void bf16_transpose_kernel(const __nv_bfloat16* __restrict__ src, int R, int C,
                                      __nv_bfloat16* __restrict__ dst) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < R && c < C) tile[i][threadIdx.x] = src[(long long)r * C + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < R && c < C) dst[(long long)c * R + r] = tile[threadIdx.x][i];
  }
}

// W^T of layers 2, 3 (256 x 256) and 4 (16 x 256 -> 256 x 16), back to back in wt
__global__ void mlp_transpose_weights_kernel(const __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt) {
  const int n2 = 256 * 256, n4 = 16 * 256;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * n2 + n4; idx += gridDim.x * blockDim.x) {
    if (idx < 2 * n2) {
      const int l = idx / n2, e = idx % n2;  // wt element (in = e / 256, out = e % 256)
      const int in = e / 256, out = e % 256;
      wt[idx] = wb[(l == 0 ? kOffW2 : kOffW3) + out * 256 + in];
    } else {
      const int e = idx - 2 * n2;  // (in = e / 16, out = e % 16)
      const int in = e / 16, out = e % 16;
      wt[idx] = wb[kOffW4 + out * 256 + in];
    }
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16(src[i]);
}

// Starting parameters of a path of order n from the network's outputs y (slots 1-4; an edge's
// second parameter -- bit s of `edges` -- and the later slots start at 1/2, and so does an output
// that is not finite or beyond 1e3, and every slot of an invalid sequence).  The slot loop runs over
// compile-time indices so that y stays in registers.
__device__ __forceinline__ void write_start(int n, bool use, unsigned edges, const float (&y)[8], float2* To) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s < n) {
      float t0 = 0.5f, t1 = 0.5f;
      if (use) {
        if (isfinite(y[2 * s]) && fabsf(y[2 * s]) < 1e3f) t0 = y[2 * s];
        if (!((edges >> s) & 1u) && isfinite(y[2 * s + 1]) && fabsf(y[2 * s + 1]) < 1e3f) t1 = y[2 * s + 1];
      }
      To[s] = make_float2(t0, t1);
    }
  }
  for (int s = 4; s < n; ++s) To[s] = make_float2(0.5f, 0.5f);
}

// bit s: slot s (s < 4) of the path is an edge
__device__ __forceinline__ unsigned edge_mask(const SceneDev& S, const PathDesc& d) {
  unsigned m = 0;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (s < d.n && S.aux[kAux * d.ids[s] + 2] != 0.f) m |= 1u << s;
  return m;
}

// learned start from unfused network outputs Y [count][16] (local indices first .. first + count)
__global__ void mlp_start_kernel(SceneDev S, BatchDev B, int n, const PathRec* list, uint64_t first, uint64_t count,
                                 const float* __restrict__ Y, float* __restrict__ T) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (uint64_t)gridDim.x * blockDim.x) {
    PathDesc d;
    fetch_path(B, n, list, first + k, d);
    float y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) y[i] = Y[k * kMlpOut + i];
    write_start(d.n, !(d.flags & ST_INVALID), edge_mask(S, d), y,
                reinterpret_cast<float2*>(T) + d.g * (uint64_t)B.n_max);
  }
}

// ---------------------------------------------------------------------------
// Fused, persistent inference for the learned start (two CTAs per SM).
//
// Per tile of 128 paths: features are computed straight into the shared
// activation tile (K-major, K = 64), then four layers run on the tensor cores
// with the accumulator in TMEM; each epilogue adds the bias, applies GELU and
// writes the BF16 activations back into the same tile (K = 256) for the next
// layer; the last one writes the starting parameters into T.  The weights are
// pre-tiled in global memory as 19 units, each K-major in core matrices: for
// layers 1-3 all 256 outputs x 32 input columns (16 KB, two MMAs with N = 256
// into the whole TMEM accumulator; an MMA costs about the same time whatever
// its N, so the widest one wastes least), for the output layer all of it, 16
// outputs x 256 columns as four 64-column chunks (8 KB, sixteen MMAs with
// N = 16: one unit instead of four, each unit paying a copy's latency).  They
// stream through two 16 KB shared buffers,
// prefetched one unit ahead: lane 0 of warp 0 waits for the MMAs that last read
// a buffer before refilling it.  A CTA's steps are serial -- features,
// MMAs, CUDA-core epilogue -- so the kernel is sized (103 KB of shared memory,
// 256 TMEM columns, at most 117 registers) for two CTAs per SM, whose phases
// interleave.  All waits are bounded.
// ---------------------------------------------------------------------------
constexpr int kInferThreads = 256;
constexpr int kInferCtasPerSm = 2;
constexpr int kUnitsPerTile = 19;  // streamed units: W1 2 K-halves, W2 and W3 8 each, W4 whole

// One K = 16 MMA (M = 128) occupies an SM's tensor pipe for about the same time whatever N is (measured on
// the GB300: ~131 cycles for N = 64, 128 and 256), so the hidden layers run with N = 256: a unit of W1-W3
// is all 256 outputs x 32 input columns (16 KB, two MMAs); the output layer (16 outputs) is one unit of
// four 64-column chunks (2 KB each, four MMAs each).
__host__ __device__ constexpr int unit_layer(int u) { return u < 2 ? 0 : (u < 10 ? 1 : (u < 18 ? 2 : 3)); }
// first input column of unit u within its layer
__host__ __device__ constexpr int unit_k0(int u) {
  return u < 2 ? 32 * u : (u < 10 ? 32 * (u - 2) : (u < 18 ? 32 * (u - 10) : 0));
}
__host__ __device__ constexpr bool unit_ends_layer(int u) { return u == 1 || u == 9 || u == 17 || u == 18; }
__host__ __device__ constexpr uint32_t unit_bytes(int u) { return u < 18 ? 256u * 32u * 2u : 4u * 16u * 64u * 2u; }
__host__ __device__ constexpr uint32_t unit_offset(int u) { return (uint32_t)(u < 18 ? u : 18) * 16384u; }
// the output layer's 64-column chunk c (16 x 64, 2 KB) within the tiled weights
__host__ __device__ constexpr uint32_t w4_chunk_offset(int c) { return unit_offset(18) + (uint32_t)c * 2048u; }
// the units of a tile cover the tiled weights once, back to back
__host__ __device__ constexpr bool units_tile_weights() {
  for (int u = 0; u + 1 < kUnitsPerTile; ++u)
    if (unit_offset(u) + unit_bytes(u) != unit_offset(u + 1)) return false;
  return unit_offset(kUnitsPerTile - 1) + unit_bytes(kUnitsPerTile - 1) == kMlpTiledBytes &&
         kMlpTiledBytes == 2u * (kMlpHidden * kMlpIn + 2 * kMlpHidden * kMlpHidden + kMlpOut * kMlpHidden);
}
static_assert(units_tile_weights(), "weight units");

// bf16 parameter copy ([out][in] per layer) -> the streamed units, each K-major in core matrices of 8 rows
// x 8 columns: a W1-W3 unit (256 rows x 32 columns) has core matrix (row group, column group) at
// (group * 4 + column group) * 128 bytes; a W4 chunk (16 x 64) at (group * 8 + column group) * 128.
__global__ void mlp_tile_weights_kernel(const __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt) {
  const int n1 = 256 * 64, n2 = 256 * 256, n4 = 16 * 256;
  const int total = n1 + 2 * n2 + n4;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int layer, r, k, K, off;
    if (idx < n1) {
      layer = 0; K = 64; off = kOffW1; r = idx / K; k = idx % K;
    } else if (idx < n1 + n2) {
      layer = 1; K = 256; off = kOffW2; r = (idx - n1) / K; k = (idx - n1) % K;
    } else if (idx < n1 + 2 * n2) {
      layer = 2; K = 256; off = kOffW3; r = (idx - n1 - n2) / K; k = (idx - n1 - n2) % K;
    } else {
      layer = 3; K = 256; off = kOffW4; r = (idx - n1 - 2 * n2) / K; k = (idx - n1 - 2 * n2) % K;
    }
    uint32_t byte;
    if (layer < 3) {
      const int u = (layer == 0 ? 0 : (layer == 1 ? 2 : 10)) + k / 32;
      byte = unit_offset(u) + tc::kmajor_offset(r, k % 32, 32);
    } else {
      byte = w4_chunk_offset(k / 64) + tc::kmajor_offset(r, k % 64, 64);
    }
    wt[byte / 2] = wb[off + r * K + k];
  }
}

struct InferSmem {
  unsigned char act[128 * 256 * 2];
  unsigned char wbuf[2][128 * 64 * 2];
  float bias[3 * 256 + 16];
  uint64_t row_g[128];     // the tile's paths: global index,
  uint32_t row_info[128];  // order | (sequence usable) << 8 | edge mask << 16 (order 0: no path)
  uint64_t full[2], done[2], layer;
  uint32_t tmem;
  int fail;
};

// Path source, fixed per launch: kSrcEnum, an exhaustive batch's enumeration of order n; kSrcRec, a
// bucket of records of order n <= kMaxBfgsOrder (the ids in the record); kSrcRecDecode, a bucket of
// longer sequences (ids decoded from the global index).
enum { kSrcEnum = 0, kSrcRec = 1, kSrcRecDecode = 2 };

template <int kSrc>
__device__ __forceinline__ void infer_fetch(const BatchDev& B, int n, const PathRec* list, uint64_t j, PathDesc& d) {
  if constexpr (kSrc == kSrcEnum) {
    decode_exhaustive_order(B, n, j, d);
  } else {
    load_rec(list, j, d);
    if constexpr (kSrc == kSrcRecDecode) decode_global(B, d.g, d);
  }
}

template <int kSrc>
__global__ void __launch_bounds__(kInferThreads, kInferCtasPerSm) mlp_infer_kernel(SceneDev S, BatchDev B, int n,
                                                                     const PathRec* __restrict__ list, uint64_t count,
                                                                     float inv_scale,
                                                                     const __nv_bfloat16* __restrict__ wt,
                                                                     const float* __restrict__ params, float* T,
                                                                     int* err) {
  extern __shared__ __align__(1024) unsigned char infer_smem[];
  InferSmem& sm = *reinterpret_cast<InferSmem*>(infer_smem);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t n_tiles = (count + 127) / 128;
  const uint64_t my_tiles = blockIdx.x < n_tiles ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const uint64_t total_q = my_tiles * kUnitsPerTile;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&sm.full[b], 1);
      tc::mbar_init(&sm.done[b], 1);
    }
    tc::mbar_init(&sm.layer, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sm.fail = 0;
  }
  for (int i = tid; i < 256; i += blockDim.x) {
    sm.bias[i] = params[kOffB1 + i];
    sm.bias[256 + i] = params[kOffB2 + i];
    sm.bias[512 + i] = params[kOffB3 + i];
  }
  if (tid < 16) sm.bias[768 + tid] = params[kOffB4 + tid];
  if (warp == 0) {
    tc::tmem_alloc(&sm.tmem, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sm.tmem;
  const char* wsrc = reinterpret_cast<const char*>(wt);
  uint32_t full_ph = 0u, done_ph = 0u, layer_ph = 0u;  // mbarrier phases, one bit per buffer
  if (tid == 0 && total_q > 0) {
    tc::mbar_expect_tx(&sm.full[0], unit_bytes(0));
    tc::bulk_g2s(sm.wbuf[0], wsrc + unit_offset(0), unit_bytes(0), &sm.full[0]);
  }
  uint64_t q = 0;
  for (uint64_t ti = 0; ti < my_tiles; ++ti) {
    const uint64_t first = (blockIdx.x + ti * gridDim.x) * 128;
    // features of the tile's 128 paths (K = 64 layout)
    if (tid < 128) {
      __nv_bfloat16 f[kMlpIn];
      if (first + tid < count) {
        PathDesc d;
        infer_fetch<kSrc>(B, n, list, first + tid, d);
        path_features(S, d, inv_scale, f, nullptr);
        sm.row_g[tid] = d.g;
        sm.row_info[tid] = (uint32_t)d.n | (d.flags & ST_INVALID ? 0u : 1u << 8) | (edge_mask(S, d) << 16);
      } else {
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) f[k] = __float2bfloat16(0.f);
        sm.row_info[tid] = 0u;
      }
#pragma unroll
      for (int g8 = 0; g8 < kMlpIn / 8; ++g8)
        *reinterpret_cast<uint4*>(sm.act + tc::kmajor_offset(tid, g8 * 8, 64)) = reinterpret_cast<uint4*>(f)[g8];
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    for (int lq = 0; lq < kUnitsPerTile; ++lq, ++q) {
      const int b = (int)(q & 1);
      const int layer = unit_layer(lq), k0 = unit_k0(lq);
      // warp 0 issues the copies and MMAs: lane 0 works while its warp-mates wait at the warp
      // barrier, so that their mbarrier polls below never hold up the issuing lane
      if (warp == 0) {
        if (lane == 0) {
          // refill the other buffer with the next chunk once the MMAs that read it (chunk q - 1) are done
          if (q + 1 < total_q) {
            const int nb = b ^ 1;
            if (q >= 1) {
              if (!tc::mbar_wait(&sm.done[nb], (done_ph >> nb) & 1u, kWaitNs)) sm.fail = 1;
              done_ph ^= 1u << nb;
            }
            const int nq = (lq + 1) % kUnitsPerTile;
            tc::mbar_expect_tx(&sm.full[nb], unit_bytes(nq));
            tc::bulk_g2s(sm.wbuf[nb], wsrc + unit_offset(nq), unit_bytes(nq), &sm.full[nb]);
          }
          if (!tc::mbar_wait(&sm.full[b], (full_ph >> b) & 1u, kWaitNs)) sm.fail = 1;
          full_ph ^= 1u << b;
          tc::fence_after_sync();
          const uint32_t K_act = layer == 0 ? 64u : 256u;
          const uint32_t a0 = tc::smem_u32(sm.act), w0 = tc::smem_u32(sm.wbuf[b]);
          if (!sm.fail) {
            // the unit's first descriptors; each next K = 16 step starts 256 bytes further, i.e. 16 more
            // in the 14-bit start-address field (shared addresses stay below 2^18: the field never carries)
            const uint64_t ad = tc::smem_desc(a0 + (uint32_t)(k0 / 8) * 128u, 128u, (K_act / 8u) * 128u);
            if (layer < 3) {  // 256 outputs x 32 columns: two MMAs with N = 256
              const uint64_t bd = tc::smem_desc(w0, 128u, 4u * 128u);
              const uint32_t idesc = tc::idesc_bf16(128, 256);
              tc::mma_bf16(tmem, ad, bd, idesc, k0 > 0 ? 1u : 0u);
              tc::mma_bf16(tmem, ad + 16u, bd + 16u, idesc, 1u);
            } else {  // 16 outputs x 256 columns: four 64-column chunks of four MMAs with N = 16
              const uint32_t idesc = tc::idesc_bf16(128, 16);
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                // chunk c: activation columns 64 c .. 64 c + 63 (eight 8-column groups of 128 bytes on), and its
                // 2 KB of weights
                const uint64_t bd = tc::smem_desc(w0 + (uint32_t)c * 2048u, 128u, 8u * 128u);
                const uint64_t adc = ad + 64u * (uint64_t)c;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  tc::mma_bf16(tmem, adc + 16u * kk, bd + 16u * kk, idesc, (c > 0 || kk > 0) ? 1u : 0u);
              }
            }
          }
          tc::mma_commit(&sm.done[b]);
          if (unit_ends_layer(lq)) tc::mma_commit(&sm.layer);
        }
        __syncwarp();
      }
      if (!unit_ends_layer(lq)) continue;
      // end of a layer: wait for its MMAs, then the epilogue
      if (!tc::mbar_wait(&sm.layer, layer_ph, kWaitNs)) sm.fail = 1;
      layer_ph ^= 1u;
      tc::fence_after_sync();
      const int rg = warp & 3;  // TMEM lane group of this warp
      const int row = rg * 32 + lane;
      if (layer < 3) {
        const int c0 = (warp >> 2) * 128;
        const float* bias = sm.bias + layer * 256;
        for (int cc = c0; cc < c0 + 128; cc += 32) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(rg * 32) << 16) + (uint32_t)cc, v);
#pragma unroll
          for (int g8 = 0; g8 < 4; ++g8) {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int c = g8 * 8 + 2 * k;
              const __nv_bfloat162 p = __floats2bfloat162_rn(gelu(v[c] + bias[cc + c]), gelu(v[c + 1] + bias[cc + c + 1]));
              w[k] = *reinterpret_cast<const uint32_t*>(&p);
            }
            *reinterpret_cast<uint4*>(sm.act + tc::kmajor_offset(row, cc + g8 * 8, 256)) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      } else if (warp < 4) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(rg * 32) << 16), v);
        const uint32_t info = sm.row_info[row];
        if (info & 0xFFu) {
          float y[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) y[i] = v[i] + sm.bias[768 + i];
          write_start((int)(info & 0xFFu), (info >> 8) & 1u, info >> 16, y,
                      reinterpret_cast<float2*>(T) + sm.row_g[row] * (uint64_t)B.n_max);
        }
      }
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      if (sm.fail) break;
    }
    if (sm.fail) break;
  }
  if (sm.fail && tid == 0) {
    if (err) atomicCAS(err, 0, ERR_MMA_TIMEOUT);
    tc::mbar_wait(&sm.layer, layer_ph, kWaitNs);  // let MMAs in flight finish before TMEM is freed
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// Training data order: a seeded pseudo-random permutation of [0, n) per epoch, evaluated index by index
// (a four-round Feistel network on 2h-bit words, 2^(2h) >= n, with cycle walking back into [0, n)), and
// the gather of one mini-batch's rows into contiguous buffers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t feistel(uint64_t x, int h, uint64_t key) {
  const uint64_t mask = (1ULL << h) - 1ULL;
  uint64_t l = x >> h, r = x & mask;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint64_t f = mix64(r ^ (key + 0x9E3779B97F4A7C15ULL * (uint64_t)(k + 1))) & mask;
    const uint64_t nl = r;
    r = l ^ f;
    l = nl;
  }
  return (l << h) | r;
}

// Position k of the permutation of [0, n) drawn by `key` (n >= 1).  The walk stays on k's cycle of the
// Feistel permutation, which holds k itself, so it returns a value below n; the bound only guards the loop.
__device__ __forceinline__ uint64_t perm_index(uint64_t k, uint64_t n, int h, uint64_t key) {
  uint64_t x = k;
  for (int i = 0; i < (1 << 20); ++i) {
    x = feistel(x, h, key);
    if (x < n) return x;
  }
  return k;
}

// Row i of the batch = sample perm(first + i): X (128 bytes), T (32) and G (48) copied with 16-byte loads
// and stores; with Xt, also the transposed features Xt[k][i] (consecutive threads, consecutive i).
__global__ void mlp_gather_kernel(const __nv_bfloat16* __restrict__ X, const float* __restrict__ T,
                                  const float* __restrict__ G, uint64_t n, uint64_t first, uint64_t B, int h,
                                  uint64_t key, __nv_bfloat16* __restrict__ Xb, float* __restrict__ Tb,
                                  float* __restrict__ Gb, __nv_bfloat16* __restrict__ Xt, int vec_tg) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t src = perm_index(first + i, n, h, key);
    const uint4* xs = reinterpret_cast<const uint4*>(X + src * kMlpIn);
    uint4* xd = reinterpret_cast<uint4*>(Xb + i * kMlpIn);
    uint4 xv[kMlpIn / 8];
#pragma unroll
    for (int q = 0; q < kMlpIn / 8; ++q) xv[q] = __ldg(xs + q);
    if (vec_tg) {
      const float4* ts = reinterpret_cast<const float4*>(T + src * 8);
      const float4* gs = reinterpret_cast<const float4*>(G + src * 12);
      float4* td = reinterpret_cast<float4*>(Tb + i * 8);
      float4* gd = reinterpret_cast<float4*>(Gb + i * 12);
      const float4 t0 = __ldg(ts), t1 = __ldg(ts + 1);
      const float4 g0 = __ldg(gs), g1 = __ldg(gs + 1), g2 = __ldg(gs + 2);
      td[0] = t0;
      td[1] = t1;
      gd[0] = g0;
      gd[1] = g1;
      gd[2] = g2;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) Tb[i * 8 + q] = T[src * 8 + q];
#pragma unroll
      for (int q = 0; q < 12; ++q) Gb[i * 12 + q] = G[src * 12 + q];
    }
#pragma unroll
    for (int q = 0; q < kMlpIn / 8; ++q) xd[q] = xv[q];
    if (Xt) {
      const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(xv);
#pragma unroll
      for (int k = 0; k < kMlpIn; ++k) Xt[(uint64_t)k * B + i] = e[k];
    }
  }
}

// dst += w * src (one value: a batch's loss into its epoch's mean)
__global__ void mlp_accumulate_kernel(float* dst, const float* src, float w) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst += w * *src;
}

cudaError_t launch_mlp_gather(const __nv_bfloat16* X, const float* T, const float* G, uint64_t n, uint64_t first,
                              uint64_t B, uint64_t key, __nv_bfloat16* Xb, float* Tb, float* Gb, __nv_bfloat16* Xt,
                              cudaStream_t stream) {
  int h = 1;
  while ((1ULL << (2 * h)) < n) ++h;
  const uint64_t want = (B + 255) / 256;
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const int vec_tg = a16(T) && a16(G) && a16(Tb) && a16(Gb);
  mlp_gather_kernel<<<(unsigned)(want < 4096 ? (want ? want : 1) : 4096), 256, 0, stream>>>(X, T, G, n, first, B, h,
                                                                                           key, Xb, Tb, Gb, Xt, vec_tg);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_accumulate(float* dst, const float* src, float w, cudaStream_t stream) {
  mlp_accumulate_kernel<<<1, 32, 0, stream>>>(dst, src, w);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_tile_weights(const __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t stream) {
  mlp_tile_weights_kernel<<<128, 256, 0, stream>>>(wb, wt);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const SceneDev& S, const BatchDev& B, int n, const PathRec* list, uint64_t count,
                             float inv_scale, const __nv_bfloat16* wt, const float* params, float* T, int* err,
                             cudaStream_t stream, int n_sm) {
  if (!count) return cudaSuccess;
  static bool attr = false;
  const int smem = (int)sizeof(InferSmem);
  if (!attr) {
    for (auto k : {mlp_infer_kernel<kSrcEnum>, mlp_infer_kernel<kSrcRec>, mlp_infer_kernel<kSrcRecDecode>}) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
    }
    attr = true;
  }
  const uint64_t tiles = (count + 127) / 128;
  const uint64_t cap = (uint64_t)n_sm * kInferCtasPerSm;
  const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
  auto kern = list == nullptr ? mlp_infer_kernel<kSrcEnum>
                              : (n > kMaxBfgsOrder ? mlp_infer_kernel<kSrcRecDecode> : mlp_infer_kernel<kSrcRec>);
  kern<<<grid, kInferThreads, smem, stream>>>(S, B, n, list, count, inv_scale, wt, params, T, err);
  count_launch();
  return cudaGetLastError();
}

static unsigned grid_1d(uint64_t n, int threads, int cap) {
  uint64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < (uint64_t)cap ? (g ? g : 1) : (uint64_t)cap);
}

cudaError_t launch_mlp_features(const SceneDev& S, const BatchDev& B, int n, const PathRec* list, uint64_t first,
                                uint64_t count, float inv_scale, __nv_bfloat16* X, float* G, cudaStream_t stream) {
  if (!count) return cudaSuccess;
  mlp_features_kernel<<<grid_1d(count, 128, 4096), 128, 0, stream>>>(S, B, n, list, first, count, inv_scale, X, G);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_loss(const float* G, const float* Y, const float* T, uint64_t B, float* dY,
                            __nv_bfloat16* dYb, __nv_bfloat16* dYt, float* loss, cudaStream_t stream) {
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const int vec = a16(G) && a16(Y) && a16(T) && a16(dY) && a16(dYb);
  mlp_loss_kernel<<<grid_1d(B, 256, 1024), 256, 0, stream>>>(G, Y, T, B, dY, dYb, dYt, loss, vec);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_colsum(const float* A, uint64_t B, int N, float* out, cudaStream_t stream) {
  if (N < 1 || N > 256) return cudaErrorInvalidValue;
  const int threads = (256 / N) * N;
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint64_t rows_per_block = (uint64_t)(threads / N) * 16;  // at least 16 rows per thread
  uint64_t blocks = (B + rows_per_block - 1) / rows_per_block;
  if (blocks > (uint64_t)(4 * n_sm)) blocks = 4 * n_sm;
  if (blocks < 1) blocks = 1;
  colsum_kernel<<<(unsigned)blocks, 256, 0, stream>>>(A, B, N, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_adam(float* w, float* m, float* v, const float* g, int n, float lr, float c1, float c2,
                        __nv_bfloat16* wb, cudaStream_t stream) {
  adam_kernel<<<grid_1d(n, 256, 1024), 256, 0, stream>>>(w, m, v, g, n, lr, c1, c2, wb);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bf16_transpose(const __nv_bfloat16* src, int R, int C, __nv_bfloat16* dst, cudaStream_t stream) {
  if (R < 1 || C < 1) return cudaSuccess;
  dim3 grid((C + 31) / 32, (R + 31) / 32);
  bf16_transpose_kernel<<<grid, dim3(32, 8), 0, stream>>>(src, R, C, dst);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_transpose_weights(const __nv_bfloat16* wb, __nv_bfloat16* wt, cudaStream_t stream) {
  mlp_transpose_weights_kernel<<<264, 512, 0, stream>>>(wb, wt);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* src, __nv_bfloat16* dst, int n, cudaStream_t stream) {
  to_bf16_kernel<<<grid_1d(n, 256, 1024), 256, 0, stream>>>(src, dst, n);
  count_launch();
  return cudaGetLastError();
}

// Check of the bounded waits that every tensor-core kernel here relies on.  Thread 0 initialises an
// mbarrier that expects one arrival; unless `arrive` is set, nothing ever arrives on it, so its phase
// never completes.  The wait gives up after `limit_ns` and records ERR_MMA_TIMEOUT in the error word,
// the same path a GEMM or inference CTA takes when an MMA or a TMA copy does not complete.
// `elapsed` (optional) receives the nanoseconds the wait took.
__global__ void bounded_wait_check_kernel(uint32_t limit_ns, int arrive, int* err, unsigned long long* elapsed) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (arrive) tc::mbar_arrive(&bar);
  const uint64_t t0 = tc::global_ns();
  const bool ok = tc::mbar_wait(&bar, 0u, limit_ns);
  const uint64_t t1 = tc::global_ns();
  if (!ok && err) atomicCAS(err, 0, ERR_MMA_TIMEOUT);
  if (elapsed) *elapsed = (unsigned long long)(t1 - t0);
}

cudaError_t launch_bounded_wait_check(uint32_t limit_ns, int arrive, int* err, unsigned long long* elapsed,
                                      cudaStream_t stream) {
  if (limit_ns < 1 || limit_ns > kWaitNs) return cudaErrorInvalidValue;
  bounded_wait_check_kernel<<<1, 32, 0, stream>>>(limit_ns, arrive, err, elapsed);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_start(const SceneDev& S, const BatchDev& B, int n, const PathRec* list, uint64_t first,
                             uint64_t count, const float* Y, float* T, cudaStream_t stream) {
  if (!count) return cudaSuccess;
  mlp_start_kernel<<<grid_1d(count, 128, 4096), 128, 0, stream>>>(S, B, n, list, first, count, Y, T);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fpt
