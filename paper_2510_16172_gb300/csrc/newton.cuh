// newton.cuh -- FP32 Newton + fixed-point line search for the longer sequences.
//
// The BFGS kernels hold the packed inverse-Hessian estimate of a path in
// registers: M(M+1)/2 floats for M = 2n unknowns, 55 at n = 5 but 210 at
// n = 10.  For orders above the BFGS orders the direction comes from the
// exact Hessian of Eq. 5 instead, which is block tridiagonal with 2 x 2 blocks
// (blocktri.cuh: 3 + 4 + 4 floats per slot, factorised by block LDL^T in
// O(n)).  The step size along p = -H^{-1} g is given by rounds of the Eq. 6
// fixed point exactly as in the BFGS kernels (alpha from 1, redone from 0 when
// it gives alpha <= 0), and the stop rules are theirs (world-space step
// tolerance, iteration cap, kink ahead, non-finite).  L is convex in T, so its
// Hessian is positive semidefinite and the Newton direction descends; where
// the factorisation meets a pivot at the rounding level (segments in line:
// a straight-through minimiser) the step falls back to p = -g.
#pragma once

#include "bfgs.cuh"
#include "blocktri.cuh"

namespace fpt {

// Pivot test of the solver's factorisation (smallest eigenvalue of a pivot
// block against its own largest diagonal entry).
constexpr float kNewtonCond = 1e-6f;

template <int N>
struct NewtonState {
  Geo<N> G;
  bool edge[N];
  float t[N][2], g[2 * N], z[N + 1][3], e[N + 1];
  uint64_t gidx;
  int it;
  uint8_t st;
  bool conv;
};

template <int N>
__device__ __forceinline__ bool newton_start(NewtonState<N>& P, const BatchDev& B, const Tables& tb,
                                             const PathRec* list, uint64_t j, int max_iters, const float* T_start) {
  PathDesc d;
  fetch_path_n<N>(B, list, j, d);
  P.gidx = d.g;
  P.st = d.flags;
  P.it = 0;
  P.conv = false;
  load_geo<N, kAllQuads<N>>(d, tb, P.G);
#pragma unroll
  for (int i = 0; i < N; ++i)  // an edge's record carries a zero second basis vector
    P.edge[i] = P.G.a[i][1][0] == 0.f && P.G.a[i][1][1] == 0.f && P.G.a[i][1][2] == 0.f;
  if (T_start) {
    const float2* Ts = reinterpret_cast<const float2*>(T_start) + d.g * (uint64_t)B.n_max;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float2 v = Ts[i];
      P.t[i][0] = v.x;
      P.t[i][1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) P.t[i][0] = P.t[i][1] = 0.5f;
  }
  if (P.st & ST_SKIP) return false;
  grad_eval<N, kAllQuads<N>>(P.G, P.t, P.z, P.e, P.g);
  return max_iters > 0;
}

// One Newton step with the Eq. 6 step size.  Returns true when the path is done.
template <int N>
__device__ __forceinline__ bool newton_step(NewtonState<N>& P, const SolveCfg& cfg) {
  constexpr int M = 2 * N;
  float p[M];
  {
    float u[N + 1][3], il[N + 1];
#pragma unroll
    for (int j = 0; j <= N; ++j) {
      il[j] = rsqrtf(fmaxf(P.e[j], 1e-30f));
#pragma unroll
      for (int c = 0; c < 3; ++c) u[j][c] = P.z[j][c] * il[j];
    }
    BlockTri<float, N> F;
    const bool ok = factor_hessian<float, N>(u, il, P.G.a, P.edge, kNewtonCond, F);
    float r[M];
#pragma unroll
    for (int k = 0; k < M; ++k) r[k] = -P.g[k];
    float gp = 0.f;
    if (ok) {
      solve_hessian<float, N>(F, r, p);
#pragma unroll
      for (int k = 0; k < M; ++k) gp = fmaf(P.g[k], p[k], gp);
    }
    if (!ok || !(gp < 0.f) || !isfinite(gp))
#pragma unroll
      for (int k = 0; k < M; ++k) p[k] = r[k];
  }
  float v[N][3], vmax2 = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int c = 0; c < 3; ++c) v[i][c] = fmaf(P.G.a[i][1][c], p[2 * i + 1], P.G.a[i][0][c] * p[2 * i]);
    vmax2 = fmaxf(vmax2, fmaf(v[i][2], v[i][2], fmaf(v[i][1], v[i][1], v[i][0] * v[i][0])));
  }
  float qa[N + 1], qc[N + 1];
#pragma unroll
  for (int jj = 0; jj <= N; ++jj) {
    float q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float x = 0.f;
      if (jj < N) x += v[jj][c];
      if (jj > 0) x -= v[jj - 1][c];
      q[c] = x;
    }
    qa[jj] = fmaf(q[2], P.z[jj][2], fmaf(q[1], P.z[jj][1], q[0] * P.z[jj][0]));
    qc[jj] = fmaf(q[2], q[2], fmaf(q[1], q[1], q[0] * q[0]));
  }
  float alpha = fixed_point<N>(P.e, qa, qc, 1.f, cfg.fp_iters);
  if (!(alpha > 0.f)) alpha = fixed_point<N>(P.e, qa, qc, 0.f, cfg.fp_iters);
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < 2; ++c) P.t[i][c] = fmaf(alpha, p[2 * i + c], P.t[i][c]);
  grad_eval<N, kAllQuads<N>>(P.G, P.t, P.z, P.e, P.g);
  ++P.it;
  P.conv = alpha * alpha * vmax2 <= cfg.tol2;
  float emin = P.e[0];
#pragma unroll
  for (int jj = 1; jj <= N; ++jj) emin = fminf(emin, P.e[jj]);
  bool bad = !isfinite(alpha);
#pragma unroll
  for (int k = 0; k < M; ++k) bad = bad || !isfinite(P.g[k]);
  if (bad) P.st |= ST_NONFINITE;
  const bool kink = emin < cfg.stop2 && !P.conv && P.it >= kKinkMinIters;
  if (kink) P.st |= ST_DEGENERATE;
  return P.it >= cfg.max_iters || bad || kink || (P.conv && !cfg.fixed_iters);
}

template <int N>
__device__ __forceinline__ void newton_finish(const NewtonState<N>& P, int n_max, float* __restrict__ T_out,
                                              uint8_t* __restrict__ status_out, uint8_t* __restrict__ iters_out) {
  float2* To = reinterpret_cast<float2*>(T_out) + P.gidx * (uint64_t)n_max;
#pragma unroll
  for (int i = 0; i < N; ++i) To[i] = make_float2(P.t[i][0], P.t[i][1]);
#pragma unroll 1
  for (int i = N; i < n_max; ++i) To[i] = make_float2(0.f, 0.f);  // unused slots of shorter sequences
  status_out[P.gidx] = P.st | (P.conv ? ST_CONVERGED : 0);
  if (iters_out) iters_out[P.gidx] = (uint8_t)(P.it > 255 ? 255 : P.it);
}

// One path per thread per tile; a warp leaves its loop when all 32 lanes are done.
template <int N>
__global__ void __launch_bounds__(kThreads) newton_kernel(SceneDev S, BatchDev B, SolveCfg cfg, uint64_t n_local,
                                                          const PathRec* __restrict__ list,
                                                          float* __restrict__ T_out, uint8_t* __restrict__ status_out,
                                                          uint8_t* __restrict__ iters_out, int use_smem) {
  extern __shared__ __align__(16) float s_tab[];
  const Tables tb = stage_tables(S, B, use_smem, s_tab);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j0 = (uint64_t)blockIdx.x * blockDim.x; j0 < n_local; j0 += stride) {
    const uint64_t j = j0 + threadIdx.x;
    const bool have = j < n_local;
    NewtonState<N> P;
    bool active = false;
    if (have) active = newton_start<N>(P, B, tb, list, j, cfg.max_iters, cfg.init_from_T ? T_out : nullptr);
    while (__any_sync(0xffffffffu, active))
      if (active && newton_step<N>(P, cfg)) active = false;
    if (have) newton_finish<N>(P, B.n_max, T_out, status_out, iters_out);
  }
}

// The launcher of one order as an explicitly instantiable unit (k_high.cu).
template <int N>
struct NewtonOrder {
  static cudaError_t launch(const BfgsLaunch& a);
};

template <int N>
cudaError_t NewtonOrder<N>::launch(const BfgsLaunch& a) {
  int use_smem = 0;
  const size_t smem = smem_tables_bytes(a.S, a.B, &use_smem);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(newton_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_kernel<N>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint64_t want = (a.n_local + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)a.n_sm * (uint64_t)per_sm;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  if (grid == 0) return cudaSuccess;
  newton_kernel<N><<<grid, kThreads, smem, a.stream>>>(a.S, a.B, a.cfg, a.n_local, a.list, a.T, a.status, a.iters,
                                                        use_smem);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fpt
