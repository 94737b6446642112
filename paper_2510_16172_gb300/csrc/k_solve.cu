// k_solve.cu -- FP32 BFGS + fixed-point line search, one thread per path.
//
// Sec. III-C: BFGS on the inverse Hessian of L(T; A, B) (Eq. 5) with the step
// size along p = -H g given by rounds of the fixed point of Eq. 6 instead of
// an inexact line search.  Unified d = 2 parameters (edges carry a zero
// second basis vector, Sec. III-B), so every path of order N has M = 2N
// unknowns and the same instruction stream.  The iterate t, the gradient and
// the packed inverse-Hessian estimate (M(M+1)/2 floats) stay in registers; the
// scene's FP32 object records are staged in shared memory.  A warp leaves its
// BFGS loop when every lane has met its stop rule (__any_sync).
//
// Readings of points the paper leaves open: H_0 = I; every step starts the
// fixed point at alpha = 1 and, if that yields alpha <= 0, restarts it at
// alpha = 0 (one round from 0 is a majorise-minimise step, positive along a
// descent direction); the update is skipped unless s^T y > 1e-6 |s| |y|
// (tested as (s^T y)^2 > 1e-12 |s|^2 |y|^2 with s^T y > 0).
#include "fpt_kernels.h"

namespace fpt {

template <int N>
struct Geo {
  float db[N + 1][3];  // Delta b_j: b of the segment's end minus b of its start
  float a[N][2][3];    // basis vectors of each object
};

// Packed upper-triangular index of a symmetric M x M matrix.
template <int M>
__host__ __device__ constexpr int hidx(int r, int c) {
  return r <= c ? r * M - r * (r - 1) / 2 + (c - r) : c * M - c * (c - 1) / 2 + (r - c);
}

template <int N>
__device__ __forceinline__ void load_geo(const PathDesc& d, const float* rec, const SceneDev& S, Geo<N>& G) {
  float bh[N + 2][3], bl[N + 2][3];
  const float* tx = S.tx32 + kEnd32 * d.tx;
  const float* rx = S.rx32 + kEnd32 * d.rx;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bh[0][c] = __ldg(tx + c);
    bl[0][c] = __ldg(tx + 3 + c);
    bh[N + 1][c] = __ldg(rx + c);
    bl[N + 1][c] = __ldg(rx + 3 + c);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float* r = rec + kRec32 * d.ids[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      bh[i + 1][c] = r[c];
      bl[i + 1][c] = r[3 + c];
      G.a[i][0][c] = r[6 + c];
      G.a[i][1][c] = r[9 + c];
    }
  }
#pragma unroll
  for (int j = 0; j <= N; ++j)
#pragma unroll
    for (int c = 0; c < 3; ++c) G.db[j][c] = (bh[j + 1][c] - bh[j][c]) + (bl[j + 1][c] - bl[j][c]);
}

// z_j = x_{j+1} - x_j for j = 0..N, e_j = |z_j|^2, and g = grad_T L (Eq. 5):
// g_i = A_i^T (u_i - u_{i+1}) with u_j = z_j / |z_j|.
template <int N>
__device__ __forceinline__ void grad_eval(const Geo<N>& G, const float (&t)[N][2], float (&z)[N + 1][3],
                                          float (&e)[N + 1], float (&g)[2 * N]) {
  float w[N][3];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) w[i][c] = fmaf(G.a[i][1][c], t[i][1], G.a[i][0][c] * t[i][0]);
  float u[N + 1][3];
#pragma unroll
  for (int j = 0; j <= N; ++j) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float v = G.db[j][c];
      if (j < N) v += w[j][c];
      if (j > 0) v -= w[j - 1][c];
      z[j][c] = v;
    }
    e[j] = fmaf(z[j][2], z[j][2], fmaf(z[j][1], z[j][1], z[j][0] * z[j][0]));
    float r = rsqrtf(fmaxf(e[j], 1e-30f));
#pragma unroll
    for (int c = 0; c < 3; ++c) u[j][c] = z[j][c] * r;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float d0 = u[i][0] - u[i + 1][0], d1 = u[i][1] - u[i + 1][1], d2 = u[i][2] - u[i + 1][2];
    g[2 * i] = fmaf(G.a[i][0][2], d2, fmaf(G.a[i][0][1], d1, G.a[i][0][0] * d0));
    g[2 * i + 1] = fmaf(G.a[i][1][2], d2, fmaf(G.a[i][1][1], d1, G.a[i][1][0] * d0));
  }
}

// Eq. 6: alpha <- -sum_j (q_j.z_j)/|z_j + alpha q_j| / sum_j (q_j.q_j)/|z_j + alpha q_j|,
// with |z_j + alpha q_j|^2 = e_j + alpha (2 qa_j + alpha qc_j).
template <int N>
__device__ __forceinline__ float fixed_point(const float (&e)[N + 1], const float (&qa)[N + 1],
                                             const float (&qc)[N + 1], float alpha, int rounds) {
  for (int k = 0; k < rounds; ++k) {
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int j = 0; j <= N; ++j) {
      float r2 = fmaf(alpha, fmaf(alpha, qc[j], 2.f * qa[j]), e[j]);
      float r = rsqrtf(fmaxf(r2, 1e-30f));
      num = fmaf(qa[j], r, num);
      den = fmaf(qc[j], r, den);
    }
    alpha = den > 1e-30f ? -__fdividef(num, den) : 0.f;
  }
  return alpha;
}

// Per-path solver state, all in registers.
template <int N>
struct PathState {
  static constexpr int M = 2 * N;
  static constexpr int HP = M * (M + 1) / 2;
  Geo<N> G;
  float t[N][2], g[M], H[HP], z[N + 1][3], e[N + 1];
  uint64_t gidx;
  int it;
  uint8_t st;
  bool conv;
};

// Decode a path, load its geometry, start at the object centroids (t = 1/2)
// with H = I and evaluate the first gradient.  Returns false for paths that
// are never solved (repeats, invalid input).
template <int N>
__device__ __forceinline__ bool path_start(PathState<N>& P, const BatchDev& B, const SceneDev& S, const float* rec,
                                           int n, const uint64_t* list, uint64_t j, int max_iters,
                                           const float* T_start) {
  constexpr int M = PathState<N>::M;
  PathDesc d;
  fetch_path(B, n, list, j, d);
  P.gidx = d.g;
  P.st = d.flags;
  P.it = 0;
  P.conv = false;
  load_geo<N>(d, rec, S, P.G);
  if (T_start) {  // learned start written by the network pass
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
#pragma unroll
  for (int r = 0; r < M; ++r)
#pragma unroll
    for (int c = r; c < M; ++c) P.H[hidx<M>(r, c)] = (r == c) ? 1.f : 0.f;
  if (P.st & ST_SKIP) return false;
  grad_eval<N>(P.G, P.t, P.z, P.e, P.g);
  return max_iters > 0;
}

// One BFGS step (Sec. III-C) with the Eq. 6 step size.  Returns true when the
// path is done (tolerance met, cap reached, kink ahead or non-finite).
template <int N>
__device__ __forceinline__ bool bfgs_step(PathState<N>& P, const SolveCfg& cfg) {
  constexpr int M = PathState<N>::M;
  // direction p = -H g
  float p[M];
#pragma unroll
  for (int r = 0; r < M; ++r) {
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < M; ++c) acc = fmaf(P.H[hidx<M>(r, c)], P.g[c], acc);
    p[r] = -acc;
  }
  // world-space direction per object and per segment: q_j = Delta A_j p_j
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
  // step and new gradient
  float s[M];
#pragma unroll
  for (int r = 0; r < M; ++r) {
    s[r] = alpha * p[r];
    P.t[r / 2][r % 2] += s[r];
  }
  float gn[M];
  grad_eval<N>(P.G, P.t, P.z, P.e, gn);
  float y[M], sy = 0.f, ss = 0.f, yy = 0.f;
#pragma unroll
  for (int r = 0; r < M; ++r) {
    y[r] = gn[r] - P.g[r];
    sy = fmaf(s[r], y[r], sy);
    ss = fmaf(s[r], s[r], ss);
    yy = fmaf(y[r], y[r], yy);
    P.g[r] = gn[r];
  }
  // BFGS inverse update: H += -rho (Hy s^T + s (Hy)^T) + (rho^2 y^T H y + rho) s s^T
  if (sy > 0.f && sy * sy > 1e-12f * (ss * yy)) {
    const float rho = __fdividef(1.f, sy);
    float Hy[M], yHy = 0.f;
#pragma unroll
    for (int r = 0; r < M; ++r) {
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < M; ++c) acc = fmaf(P.H[hidx<M>(r, c)], y[c], acc);
      Hy[r] = acc;
      yHy = fmaf(y[r], acc, yHy);
    }
    const float beta = fmaf(rho * rho, yHy, rho);
    float wv[M], mv[M];
#pragma unroll
    for (int r = 0; r < M; ++r) {
      wv[r] = fmaf(beta, s[r], -rho * Hy[r]);
      mv[r] = -rho * Hy[r];
    }
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
      for (int c = r; c < M; ++c) {
        float h = P.H[hidx<M>(r, c)];
        h = fmaf(s[r], wv[c], h);
        P.H[hidx<M>(r, c)] = fmaf(mv[r], s[c], h);
      }
  }
  ++P.it;
  const float ws2 = alpha * alpha * vmax2;
  P.conv = ws2 <= cfg.tol2;
  float emin = P.e[0];
#pragma unroll
  for (int jj = 1; jj <= N; ++jj) emin = fminf(emin, P.e[jj]);
  const bool bad = !isfinite(sy) || !isfinite(alpha);
  if (bad) P.st |= ST_NONFINITE;
  return P.it >= cfg.max_iters || bad || emin < cfg.stop2 || (P.conv && !cfg.fixed_iters);
}

template <int N>
__device__ __forceinline__ void path_finish(const PathState<N>& P, int n_max, float* __restrict__ T_out,
                                            uint8_t* __restrict__ status_out, uint8_t* __restrict__ iters_out) {
  float2* To = reinterpret_cast<float2*>(T_out) + P.gidx * (uint64_t)n_max;
#pragma unroll
  for (int i = 0; i < kMaxOrder; ++i)
    if (i < n_max) To[i] = i < N ? make_float2(P.t[i][0], P.t[i][1]) : make_float2(0.f, 0.f);
  status_out[P.gidx] = P.st | (P.conv ? ST_CONVERGED : 0);
  if (iters_out) iters_out[P.gidx] = (uint8_t)(P.it > 255 ? 255 : P.it);
}

// One path per thread per tile; a warp leaves its BFGS loop when all 32 lanes are done.
template <int N>
__global__ void __launch_bounds__(kThreads) bfgs_kernel(SceneDev S, BatchDev B, SolveCfg cfg, uint64_t n_local,
                                                        const uint64_t* __restrict__ list, float* __restrict__ T_out,
                                                        uint8_t* __restrict__ status_out,
                                                        uint8_t* __restrict__ iters_out, int use_smem) {
  extern __shared__ float s_rec[];
  const float* rec = S.rec32;
  if (use_smem) {
    stage(s_rec, S.rec32, S.n_obj * kRec32);
    __syncthreads();
    rec = s_rec;
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j0 = (uint64_t)blockIdx.x * blockDim.x; j0 < n_local; j0 += stride) {
    const uint64_t j = j0 + threadIdx.x;
    const bool have = j < n_local;
    PathState<N> P;
    bool active = false;
    if (have) active = path_start<N>(P, B, S, rec, N, list, j, cfg.max_iters, cfg.init_from_T ? T_out : nullptr);
    while (__any_sync(0xffffffffu, active))
      if (active && bfgs_step<N>(P, cfg)) active = false;
    if (have) path_finish<N>(P, B.n_max, T_out, status_out, iters_out);
  }
}

// Lane refill: a lane whose path is done writes it out and takes the next path
// of its warp's chunk (chunks of kChunk paths are claimed from a global
// counter), so lanes do not idle behind the warp's slowest path.  To amortise
// the divergent start-up code, lanes refill only when at least cfg.refill of
// them are free, or when none is busy.
constexpr int kChunk = 256;

template <int N>
__global__ void __launch_bounds__(kThreads) bfgs_refill_kernel(SceneDev S, BatchDev B, SolveCfg cfg, uint64_t n_local,
                                                               const uint64_t* __restrict__ list,
                                                               float* __restrict__ T_out,
                                                               uint8_t* __restrict__ status_out,
                                                               uint8_t* __restrict__ iters_out, int use_smem,
                                                               unsigned long long* __restrict__ work) {
  extern __shared__ float s_rec[];
  const float* rec = S.rec32;
  if (use_smem) {
    stage(s_rec, S.rec32, S.n_obj * kRec32);
    __syncthreads();
    rec = s_rec;
  }
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  uint64_t next = 0, end = 0;  // warp-uniform: unclaimed part of the warp's chunk
  bool more = true;            // warp-uniform: the global counter may still have work
  PathState<N> P;
  bool active = false;
  for (;;) {
    unsigned free_mask = __ballot_sync(full, !active);
    const int n_free = __popc(free_mask);
    if (more && (n_free >= cfg.refill || n_free == 32)) {
      // hand out paths to free lanes, claiming new chunks as needed
      while (more && free_mask) {
        if (next >= end) {
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(work, (unsigned long long)kChunk);
          base = __shfl_sync(full, base, 0);
          if (base >= n_local) {
            more = false;
            break;
          }
          next = base;
          end = base + kChunk < n_local ? base + kChunk : n_local;
        }
        const uint64_t avail = end - next;
        const int take = (int)(avail < (uint64_t)__popc(free_mask) ? avail : (uint64_t)__popc(free_mask));
        const bool mine = (free_mask >> lane) & 1u;
        const int rank = __popc(free_mask & lt_mask);
        bool got = mine && rank < take;
        const unsigned got_mask = __ballot_sync(full, got);
        if (got) {
          const uint64_t j = next + (uint64_t)rank;
          if (path_start<N>(P, B, S, rec, N, list, j, cfg.max_iters, cfg.init_from_T ? T_out : nullptr)) {
            active = true;
          } else {
            path_finish<N>(P, B.n_max, T_out, status_out, iters_out);
          }
        }
        next += (uint64_t)take;
        free_mask &= ~got_mask;
        // lanes whose new path needs no solving are free again
        free_mask |= __ballot_sync(full, got && !active);
      }
    }
    if (!__any_sync(full, active)) {
      if (!more) break;
      continue;
    }
    if (active && bfgs_step<N>(P, cfg)) {
      path_finish<N>(P, B.n_max, T_out, status_out, iters_out);
      active = false;
    }
  }
}

template <int N>
static cudaError_t launch_bfgs_n(const SceneDev& S, const BatchDev& B, const SolveCfg& cfg, uint64_t n_local,
                                 const uint64_t* list, float* T, uint8_t* status, uint8_t* iters, cudaStream_t stream,
                                 int n_sm, unsigned long long* work) {
  size_t smem = (size_t)S.n_obj * kRec32 * sizeof(float);
  int use_smem = smem <= 96 * 1024;
  if (!use_smem) smem = 0;
  const bool refill = cfg.refill > 0 && work != nullptr;
  const void* fn = refill ? (const void*)bfgs_refill_kernel<N> : (const void*)bfgs_kernel<N>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t want = (n_local + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)n_sm * (uint64_t)per_sm;
  unsigned grid = (unsigned)(want < cap ? want : cap);
  if (grid == 0) return cudaSuccess;
  if (refill) {
    e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    bfgs_refill_kernel<N><<<grid, kThreads, smem, stream>>>(S, B, cfg, n_local, list, T, status, iters, use_smem,
                                                             work);
  } else {
    bfgs_kernel<N><<<grid, kThreads, smem, stream>>>(S, B, cfg, n_local, list, T, status, iters, use_smem);
  }
  return cudaGetLastError();
}

cudaError_t launch_bfgs(int n, const SceneDev& S, const BatchDev& B, const SolveCfg& cfg, uint64_t n_local,
                        const uint64_t* list, float* T, uint8_t* status, uint8_t* iters, cudaStream_t stream,
                        int n_sm, unsigned long long* work) {
  switch (n) {
    case 1: return launch_bfgs_n<1>(S, B, cfg, n_local, list, T, status, iters, stream, n_sm, work);
    case 2: return launch_bfgs_n<2>(S, B, cfg, n_local, list, T, status, iters, stream, n_sm, work);
    case 3: return launch_bfgs_n<3>(S, B, cfg, n_local, list, T, status, iters, stream, n_sm, work);
    case 4: return launch_bfgs_n<4>(S, B, cfg, n_local, list, T, status, iters, stream, n_sm, work);
    case 5: return launch_bfgs_n<5>(S, B, cfg, n_local, list, T, status, iters, stream, n_sm, work);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpt
