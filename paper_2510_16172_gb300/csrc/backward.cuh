// backward.cuh -- implicit-differentiation backward, one thread per path.
//
// Sec. III-D: at a solution grad_T L = 0 (Eq. 8), so for a loss
// l = sum_i dX_i . x_i + dL L the vector-Jacobian product through T*(theta)
// is u^T d(grad_T L)/dtheta with H u = -v, v = dl/dT = A^T dX + dL grad_T L
// (Eq. 11-13; H symmetric).  With w_i = A_i u_i, Dw_j = w_j - w_{j-1} (zero
// beyond the ends) and q_j = M_j Dw_j (M_j = (I - u_j u_j^T)/|z_j|), the
// per-path gradient, including the explicit dependence of l on theta, is
//   e_i        = dX_i + dL (u_i - u_{i+1}) + (q_i - q_{i+1})
//   dl/db_i    = e_i
//   dl/da_ik   = e_i t_ik + (u_i - u_{i+1}) u_ik       (k = 1, 2)
//   dl/dTX     = -dL u_0 - q_0,     dl/dRX = dL u_N + q_N
// The per-path terms are summed over paths (per CTA in shared memory, then in
// FP64 in global memory) and mapped to vertices by the chain rule of the
// object records (plane: b = v0, a1 = v1 - v0, a2 = v3 - v0; edge: b = e0,
// a1 = e1 - e0).
#pragma once

#include "fpt_kernels.h"
#include "vjp.cuh"

namespace fpt {

template <int N>
__global__ void __launch_bounds__(kThreads) backward_kernel(SceneDev S, BatchDev B, BackwardCfg cfg,
                                                            uint64_t n_local, const PathRec* __restrict__ list,
                                                            const float* __restrict__ T,
                                                            const uint8_t* __restrict__ status,
                                                            const float* __restrict__ dX,
                                                            const float* __restrict__ dLv, double* gacc,
                                                            uint32_t* __restrict__ rescue_list,
                                                            unsigned* __restrict__ rescue_count) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* s_rec = reinterpret_cast<float*>(smem_raw);
  float* s_aux = s_rec + S.n_obj * kRec32;
  float* s_acc = s_aux + S.n_obj * kAux;
  const int n_acc = S.n_obj * 9 + 3 * (S.n_tx + S.n_rx);
  const int acc_tx = S.n_obj * 9, acc_rx = acc_tx + 3 * S.n_tx;
  stage(s_rec, S.rec32, S.n_obj * kRec32);
  stage(s_aux, S.aux, S.n_obj * kAux);
  if (cfg.acc_in_smem)
    for (int k = threadIdx.x; k < n_acc; k += blockDim.x) s_acc[k] = 0.f;
  __syncthreads();
  const int n_max = B.n_max;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // listed launch: only the paths the select pass found with a cotangent
  const uint64_t n_iter = cfg.sel ? (uint64_t)*cfg.sel_count : n_local;
  int tiles = 0;
  for (uint64_t j0 = (uint64_t)blockIdx.x * blockDim.x; j0 < n_iter; j0 += stride) {
    const bool have = j0 + threadIdx.x < n_iter;
    const uint64_t j = have && cfg.sel ? (uint64_t)cfg.sel[j0 + threadIdx.x] : j0 + threadIdx.x;
    PathDesc d;
    float gb[N][9];  // per slot: d/db (3), d/da1 (3), d/da2 (3)
    float gtx[3] = {0.f, 0.f, 0.f}, grx[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int k = 0; k < 9; ++k) gb[i][k] = 0.f;
    bool use = false;
    uint8_t st = 0;
    float dl = 0.f;
    if (have) {
      fetch_path_n<N>(B, list, j, d);
      st = d.flags;
      if (status) st |= status[d.g];
      use = !(st & (ST_REPEAT | ST_INVALID | ST_DEGENERATE | ST_NONFINITE));
      // a path with no cotangent contributes exactly zero: skip it
      if (use) {
        dl = dLv ? dLv[d.g] : ((cfg.dl_mask && (st & cfg.dl_mask) == cfg.dl_mask) ? 1.f : 0.f);
        use = dl != 0.f || has_point_cotangent<N>(dX, d.g, n_max);
      }
    } else {
      d.tx = d.rx = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) d.ids[i] = -1;
    }
    if (use) {
      const uint64_t g = d.g;
      // geometry (FP32, hi/lo differences of b) and parameters
      float bh[N + 2][3], bl[N + 2][3], a[N][2][3];
      bool edge[N];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        bh[0][c] = __ldg(S.tx32 + kEnd32 * d.tx + c);
        bl[0][c] = __ldg(S.tx32 + kEnd32 * d.tx + 3 + c);
        bh[N + 1][c] = __ldg(S.rx32 + kEnd32 * d.rx + c);
        bl[N + 1][c] = __ldg(S.rx32 + kEnd32 * d.rx + 3 + c);
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float* r = s_rec + kRec32 * d.ids[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          bh[i + 1][c] = r[c];
          bl[i + 1][c] = r[3 + c];
          a[i][0][c] = r[6 + c];
          a[i][1][c] = r[9 + c];
        }
        edge[i] = s_aux[kAux * d.ids[i] + 2] != 0.f;
      }
      const float2* Ti = reinterpret_cast<const float2*>(T) + g * (uint64_t)n_max;
      float t[N][2];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float2 v = Ti[i];
        t[i][0] = v.x;
        t[i][1] = v.y;
      }
      float z[N + 1][3];
#pragma unroll
      for (int jj = 0; jj <= N; ++jj)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float x = (bh[jj + 1][c] - bh[jj][c]) + (bl[jj + 1][c] - bl[jj][c]);
          if (jj < N) x += fmaf(a[jj][1][c], t[jj][1], a[jj][0][c] * t[jj][0]);
          if (jj > 0) x -= fmaf(a[jj - 1][1][c], t[jj - 1][1], a[jj - 1][0][c] * t[jj - 1][0]);
          z[jj][c] = x;
        }
      float dx[N][3];
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) dx[i][c] = dX ? dX[(g * (uint64_t)n_max + i) * 3 + c] : 0.f;
      if (!path_vjp<float, N>(z, a, t, edge, dx, dl, cfg.cond_fp64, gb, gtx, grx)) {
        // FP32 pivots failed: the FP64 pass over the rescue list adds this path
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int k = 0; k < 9; ++k) gb[i][k] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) gtx[c] = grx[c] = 0.f;
        rescue_list[atomicAdd(rescue_count, 1u)] = (uint32_t)j;
      }
    }
    // sums over paths
    const bool sm = cfg.acc_in_smem != 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int id = d.ids[i];
      warp_accumulate<9>(s_acc, id >= 0 ? 9 * id : -1, gb[i], sm, gacc, 9 * id);
    }
    warp_accumulate<3>(s_acc, have ? acc_tx + 3 * d.tx : -1, gtx, sm, gacc, acc_tx + 3 * d.tx);
    warp_accumulate<3>(s_acc, have ? acc_rx + 3 * d.rx : -1, grx, sm, gacc, acc_rx + 3 * d.rx);
    if (sm && ++tiles >= cfg.flush_tiles) {
      tiles = 0;
      __syncthreads();
      for (int k = threadIdx.x; k < n_acc; k += blockDim.x) {
        float x = s_acc[k];
        if (x != 0.f) {
          atomicAdd(gacc + k, (double)x);
          s_acc[k] = 0.f;
        }
      }
      __syncthreads();
    }
  }
  if (cfg.acc_in_smem) {
    __syncthreads();
    for (int k = threadIdx.x; k < n_acc; k += blockDim.x) {
      float x = s_acc[k];
      if (x != 0.f) atomicAdd(gacc + k, (double)x);
    }
  }
}

// List the paths of a slice that carry a cotangent (no dX: those with a non-zero length cotangent
// and a status that the backward does not skip), by local index.  A CTA takes kSelChunk consecutive
// local indices at a time (kSelPer per thread), lists its chunk's paths in index order and claims
// their place in the list with one atomic.  Consecutive list entries are then neighbouring
// sequences, which mostly share their endpoints and leading objects, so the adjoint's warps find
// uniform accumulator targets and sum them by shuffles.
constexpr int kSelThreads = 256, kSelPer = 16, kSelChunk = kSelThreads * kSelPer;
template <int N>
__global__ void __launch_bounds__(kSelThreads) backward_select_kernel(BatchDev B, BackwardCfg cfg, uint64_t n_local,
                                                                      const PathRec* list,
                                                                      const uint8_t* __restrict__ status,
                                                                      const float* __restrict__ dLv) {
  for (uint64_t c0 = (uint64_t)blockIdx.x * kSelChunk; c0 < n_local; c0 += (uint64_t)gridDim.x * kSelChunk) {
    const uint64_t j0 = c0 + (uint64_t)threadIdx.x * kSelPer;
    unsigned bits = 0;
    SliceWalk walk;
    bool whole = false;  // the thread's 16 statuses read with one 16-byte load
    if (status != nullptr && list == nullptr && dLv == nullptr && j0 + kSelPer <= n_local) {
      // exhaustive batch, mask cotangent: 16 consecutive paths of one TX/RX pair whose statuses start on
      // a 16-byte boundary
      SliceWalk w0;
      const uint64_t g0 = w0.next(B, N, j0);
      if (w0.left + 1 >= (uint64_t)kSelPer && (reinterpret_cast<uintptr_t>(status + g0) & 15u) == 0) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(status + g0));
        const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < kSelPer; ++k) {
          const uint8_t st = (uint8_t)(wd[k >> 2] >> (8 * (k & 3)));
          const bool take = !(st & (ST_REPEAT | ST_INVALID | ST_DEGENERATE | ST_NONFINITE)) && cfg.dl_mask &&
                            (st & cfg.dl_mask) == cfg.dl_mask;
          bits |= (take ? 1u : 0u) << k;
        }
        whole = true;
      }
    }
#pragma unroll 4
    for (int k = 0; k < kSelPer && !whole; ++k) {
      const uint64_t j = j0 + k;
      if (j >= n_local) break;
      uint64_t g;
      uint8_t st;
      if (status) {  // the solver wrote the sequence's REPEAT / INVALID_INPUT bits into its status
        g = list != nullptr ? slice_global(B, N, list, j) : walk.next(B, N, j);
        st = status[g];
      } else {
        PathDesc d;
        fetch_path_n<N>(B, list, j, d);
        g = d.g;
        st = d.flags;
      }
      bool take = false;
      if (!(st & (ST_REPEAT | ST_INVALID | ST_DEGENERATE | ST_NONFINITE)))
        take = dLv ? dLv[g] != 0.f : (cfg.dl_mask && (st & cfg.dl_mask) == cfg.dl_mask);
      bits |= (take ? 1u : 0u) << k;
    }
    cta_append_ordered<kSelThreads>(bits, j0, cfg.sel, cfg.sel_count);
  }
}

// FP64 pass over the paths whose FP32 pivots failed: FP64 records, segment
// vectors, Hessian and VJP, summed straight into the FP64 accumulators.
template <int N>
__global__ void __launch_bounds__(kThreads, kLongOrderMinBlocks<N>)
    backward_rescue_kernel(SceneDev S, BatchDev B, BackwardCfg cfg, const PathRec* __restrict__ list,
        const float* __restrict__ T, const uint8_t* __restrict__ status, const float* __restrict__ dX,
        const float* __restrict__ dLv, double* gacc, const uint32_t* __restrict__ rescue_list,
        const unsigned* __restrict__ rescue_count) {
  const uint64_t n = *rescue_count;
  const int n_max = B.n_max;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    PathDesc d;
    fetch_path_n<N>(B, list, rescue_list[k], d);
    const uint64_t g = d.g;
    uint8_t st = d.flags;
    if (status) st |= status[g];
    // the fused polish also lists paths whose polish went to the FP64 pass: their final status decides
    if (st & (ST_REPEAT | ST_INVALID | ST_DEGENERATE | ST_NONFINITE)) continue;
    double a[N][2][3], t[N][2], z[N + 1][3], dx[N][3];
    bool edge[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) a[i][q][c] = S.rec64[kRec64 * d.ids[i] + 3 + 3 * q + c];
      const float2 v = reinterpret_cast<const float2*>(T)[g * (uint64_t)n_max + i];
      t[i][0] = v.x;
      t[i][1] = v.y;
      edge[i] = S.aux[kAux * d.ids[i] + 2] != 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) dx[i][c] = dX ? (double)dX[(g * (uint64_t)n_max + i) * 3 + c] : 0.0;
    }
#pragma unroll
    for (int jj = 0; jj <= N; ++jj)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double b1 = jj < N ? S.rec64[kRec64 * d.ids[jj] + c] : S.rx64[3 * d.rx + c];
        const double b0 = jj > 0 ? S.rec64[kRec64 * d.ids[jj - 1] + c] : S.tx64[3 * d.tx + c];
        double x = b1 - b0;
        if (jj < N) x += a[jj][0][c] * t[jj][0] + a[jj][1][c] * t[jj][1];
        if (jj > 0) x -= a[jj - 1][0][c] * t[jj - 1][0] + a[jj - 1][1][c] * t[jj - 1][1];
        z[jj][c] = x;
      }
    const double dl = dLv ? (double)dLv[g] : ((cfg.dl_mask && (st & cfg.dl_mask) == cfg.dl_mask) ? 1.0 : 0.0);
    bool any = dl != 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < 3; ++c) any = any || dx[i][c] != 0.0;
    if (!any) continue;  // no cotangent: the path contributes exactly zero
    double gb[N][9], gtx[3], grx[3];
    if (!path_vjp<double, N>(z, a, t, edge, dx, dl, 1e-10, gb, gtx, grx)) {
      // singular even in FP64: the path is left out of the sums and counted
      if (cfg.dropped) atomicAdd(cfg.dropped, 1u);
      continue;
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int q = 0; q < 9; ++q) atomicAdd(gacc + 9 * d.ids[i] + q, gb[i][q]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicAdd(gacc + 9 * S.n_obj + 3 * d.tx + c, gtx[c]);
      atomicAdd(gacc + 9 * S.n_obj + 3 * S.n_tx + 3 * d.rx + c, grx[c]);
    }
  }
}
// FP64 adjoint over the listed paths (a few percent of a slice of n_local paths).
template <int N>
cudaError_t launch_backward_rescue_n(const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg,
                                            uint64_t n_local, const PathRec* list, const float* T,
                                            const uint8_t* status, const float* dX, const float* dL, double* gacc,
                                            cudaStream_t stream, int n_sm, const uint32_t* rescue_list,
                                            const unsigned* rescue_count) {
  const uint64_t rwant = (n_local / 16 + kThreads - 1) / kThreads;
  const unsigned rgrid = (unsigned)(rwant < (uint64_t)n_sm * 4 ? (rwant ? rwant : 1) : (uint64_t)n_sm * 4);
  backward_rescue_kernel<N><<<rgrid, kThreads, 0, stream>>>(S, B, cfg, list, T, status, dX, dL, gacc, rescue_list,
                                                             rescue_count);
  count_launch();
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_backward_n(const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg_in,
                                     uint64_t n_local, const PathRec* list, const float* T, const uint8_t* status,
                                     const float* dX, const float* dL, double* gacc, cudaStream_t stream, int n_sm,
                                     uint32_t* rescue_list, unsigned* rescue_count) {
  BackwardCfg cfg = cfg_in;
  if (dX != nullptr || cfg.sel == nullptr || cfg.sel_count == nullptr) {
    cfg.sel = nullptr;  // point cotangents: every path takes part
    cfg.sel_count = nullptr;
  } else {
    cudaError_t e = cudaMemsetAsync(cfg.sel_count, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    const uint64_t want = (n_local + kSelChunk - 1) / kSelChunk;
    const unsigned g = (unsigned)(want < (uint64_t)n_sm * 8 ? want : (uint64_t)n_sm * 8);
    if (g == 0) return cudaSuccess;
    backward_select_kernel<N><<<g, kSelThreads, 0, stream>>>(B, cfg, n_local, list, status, dL);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t base = (size_t)S.n_obj * (kRec32 + kAux) * sizeof(float);
  const size_t accb = (size_t)(S.n_obj * 9 + 3 * (S.n_tx + S.n_rx)) * sizeof(float);
  size_t smem = base + accb;
  if (smem > 160 * 1024) {
    cfg.acc_in_smem = 0;
    smem = base;
  }
  if (smem > 160 * 1024) return cudaErrorInvalidValue;  // scene too large for this kernel
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(backward_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backward_kernel<N>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t want = (n_local + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)n_sm * (uint64_t)per_sm;
  unsigned grid = (unsigned)(want < cap ? want : cap);
  if (grid == 0) return cudaSuccess;
  e = cudaMemsetAsync(rescue_count, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  backward_kernel<N><<<grid, kThreads, smem, stream>>>(S, B, cfg, n_local, list, T, status, dX, dL, gacc, rescue_list,
                                                        rescue_count);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_backward_rescue_n<N>(S, B, cfg, n_local, list, T, status, dX, dL, gacc, stream, n_sm, rescue_list,
                                     rescue_count);
}

// The launchers of one order as an explicitly instantiable unit (see PolishOrder).
template <int N>
struct BackwardOrder {
  static cudaError_t launch(const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg, uint64_t n_local,
                            const PathRec* list, const float* T, const uint8_t* status, const float* dX,
                            const float* dL, double* gacc, cudaStream_t stream, int n_sm, uint32_t* rescue_list,
                            unsigned* rescue_count);
  static cudaError_t rescue(const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg, uint64_t n_local,
                            const PathRec* list, const float* T, const uint8_t* status, const float* dX,
                            const float* dL, double* gacc, cudaStream_t stream, int n_sm,
                            const uint32_t* rescue_list, const unsigned* rescue_count);
};

template <int N>
cudaError_t BackwardOrder<N>::launch(const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg, uint64_t n_local,
                                     const PathRec* list, const float* T, const uint8_t* status, const float* dX,
                                     const float* dL, double* gacc, cudaStream_t stream, int n_sm,
                                     uint32_t* rescue_list, unsigned* rescue_count) {
  return launch_backward_n<N>(S, B, cfg, n_local, list, T, status, dX, dL, gacc, stream, n_sm, rescue_list,
                              rescue_count);
}

template <int N>
cudaError_t BackwardOrder<N>::rescue(const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg, uint64_t n_local,
                                     const PathRec* list, const float* T, const uint8_t* status, const float* dX,
                                     const float* dL, double* gacc, cudaStream_t stream, int n_sm,
                                     const uint32_t* rescue_list, const unsigned* rescue_count) {
  return launch_backward_rescue_n<N>(S, B, cfg, n_local, list, T, status, dX, dL, gacc, stream, n_sm, rescue_list,
                                     rescue_count);
}

}  // namespace fpt
