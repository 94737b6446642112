// k_polish.cu -- stationarity polish, residual and validity, one thread per path.
//
// After BFGS (Sec. III-C) each path takes `steps` Newton steps on Eq. 5 whose
// gradient is formed in FP64 (z_j from FP64 geometry, FP64 norms) and whose
// Hessian system (block tridiagonal, blocktri.cuh) is solved in FP32, or in
// FP64 when a pivot is ill-conditioned.  The first-order condition of Eq. 8
// measures the result: rho = max_i |A_i delta_i| (metres), where delta solves
// H delta = -grad_T L at the returned FP32 parameters (the factorisation from
// the last step is reused).  The validity test (Sec. I, Sec. III: points
// inside their objects) uses closed intervals on t.
//
// The same kernel evaluates rho, validity and the boundary distance at
// caller-given parameters (POLISH_VALIDITY) without changing them.
#include "blocktri.cuh"
#include "fpt_kernels.h"

namespace fpt {

template <int N>
struct Geo64 {
  double p0[3], pe[3];  // TX, RX (recentred)
  double b[N][3], a[N][2][3];
};

// FP64 segment data and gradient at t.
template <int N>
__device__ __forceinline__ void grad64(const Geo64<N>& G, const double (&t)[N][2], double (&len)[N + 1],
                                       double (&u)[N + 1][3], double (&g)[2 * N]) {
  double x[N + 2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x[0][c] = G.p0[c];
    x[N + 1][c] = G.pe[c];
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) x[i + 1][c] = fma(G.a[i][1][c], t[i][1], fma(G.a[i][0][c], t[i][0], G.b[i][c]));
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    double z0 = x[j + 1][0] - x[j][0], z1 = x[j + 1][1] - x[j][1], z2 = x[j + 1][2] - x[j][2];
    double e = fma(z2, z2, fma(z1, z1, z0 * z0));
    double r = e > 0.0 ? rsqrt(e) : 0.0;
    len[j] = e * r;
    u[j][0] = z0 * r;
    u[j][1] = z1 * r;
    u[j][2] = z2 * r;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double d0 = u[i][0] - u[i + 1][0], d1 = u[i][1] - u[i + 1][1], d2 = u[i][2] - u[i + 1][2];
    g[2 * i] = fma(G.a[i][0][2], d2, fma(G.a[i][0][1], d1, G.a[i][0][0] * d0));
    g[2 * i + 1] = fma(G.a[i][1][2], d2, fma(G.a[i][1][1], d1, G.a[i][1][0] * d0));
  }
}

template <int N>
__device__ __forceinline__ bool factor_any(const double (&u)[N + 1][3], const double (&len)[N + 1],
                                           const float (&a32)[N][2][3], const Geo64<N>& G, const bool (&edge)[N],
                                           float cond, BlockTri<float, N>& F32, BlockTri<double, N>& F64,
                                           bool& use64) {
  float uf[N + 1][3], ilf[N + 1];
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    ilf[j] = (float)(1.0 / len[j]);
#pragma unroll
    for (int c = 0; c < 3; ++c) uf[j][c] = (float)u[j][c];
  }
  use64 = false;
  if (factor_hessian<float, N>(uf, ilf, a32, edge, cond, F32)) return true;
  use64 = true;
  double il[N + 1];
#pragma unroll
  for (int j = 0; j <= N; ++j) il[j] = 1.0 / len[j];
  return factor_hessian<double, N>(u, il, G.a, edge, (double)cond * 1e-6, F64);
}

template <int N>
__device__ __forceinline__ void newton_step(const BlockTri<float, N>& F32, const BlockTri<double, N>& F64, bool use64,
                                            const double (&g)[2 * N], double (&delta)[2 * N]) {
  if (use64) {
    double r[2 * N];
#pragma unroll
    for (int k = 0; k < 2 * N; ++k) r[k] = -g[k];
    solve_hessian<double, N>(F64, r, delta);
  } else {
    float r[2 * N], x[2 * N];
#pragma unroll
    for (int k = 0; k < 2 * N; ++k) r[k] = (float)(-g[k]);
    solve_hessian<float, N>(F32, r, x);
#pragma unroll
    for (int k = 0; k < 2 * N; ++k) delta[k] = (double)x[k];
  }
}

template <int N>
__global__ void __launch_bounds__(kThreads) polish_kernel(SceneDev S, BatchDev B, PolishCfg cfg, uint64_t n_local,
                                                          const uint64_t* __restrict__ list, float* __restrict__ T,
                                                          float* __restrict__ X, float* __restrict__ Lout,
                                                          uint8_t* __restrict__ status, float* __restrict__ rho_out,
                                                          uint8_t* __restrict__ mask_out,
                                                          float* __restrict__ bdist_out, int use_smem) {
  constexpr int M = 2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const double* rec64 = S.rec64;
  const float* rec32 = S.rec32;
  const float* aux = S.aux;
  if (use_smem) {
    double* s64 = reinterpret_cast<double*>(smem_raw);
    float* s32 = reinterpret_cast<float*>(s64 + S.n_obj * kRec64);
    float* sax = s32 + S.n_obj * kRec32;
    stage(s64, S.rec64, S.n_obj * kRec64);
    stage(s32, S.rec32, S.n_obj * kRec32);
    stage(sax, S.aux, S.n_obj * kAux);
    __syncthreads();
    rec64 = s64;
    rec32 = s32;
    aux = sax;
  }
  const int n_max = B.n_max;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_local; j += stride) {
    PathDesc d;
    fetch_path(B, N, list, j, d);
    const uint64_t g = d.g;
    uint8_t st = d.flags;
    if (cfg.mode == POLISH_SOLVE) st |= status[g] & (ST_CONVERGED | ST_NONFINITE);
    // geometry
    Geo64<N> G;
    float a32[N][2][3];
    bool edge[N];
    float h1[N], h2[N];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      G.p0[c] = __ldg(S.tx64 + 3 * d.tx + c);
      G.pe[c] = __ldg(S.rx64 + 3 * d.rx + c);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const double* r = rec64 + kRec64 * d.ids[i];
      const float* r32 = rec32 + kRec32 * d.ids[i];
      const float* ax = aux + kAux * d.ids[i];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        G.b[i][c] = r[c];
        G.a[i][0][c] = r[3 + c];
        G.a[i][1][c] = r[6 + c];
        a32[i][0][c] = r32[6 + c];
        a32[i][1][c] = r32[9 + c];
      }
      h1[i] = ax[0];
      h2[i] = ax[1];
      edge[i] = ax[2] != 0.f;
    }
    // parameters
    const float2* Ti = reinterpret_cast<const float2*>(T) + g * (uint64_t)n_max;
    float tf[N][2];
    double t[N][2];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float2 v = Ti[i];
      tf[i][0] = v.x;
      tf[i][1] = v.y;
      t[i][0] = v.x;
      t[i][1] = v.y;
    }
    double len[N + 1], u[N + 1][3], gr[M];
    float rho = INFINITY;
    bool finite = true;
#pragma unroll
    for (int i = 0; i < N; ++i) finite = finite && isfinite(tf[i][0]) && isfinite(tf[i][1]);
    if (!finite) st |= ST_NONFINITE;
    if (!(st & ST_INVALID) && finite) {
      grad64<N>(G, t, len, u, gr);
      double lmin = len[0];
#pragma unroll
      for (int k = 1; k <= N; ++k) lmin = fmin(lmin, len[k]);
      if (!(st & ST_REPEAT) && lmin >= (double)cfg.deg_tol) {
        BlockTri<float, N> F32;
        BlockTri<double, N> F64;
        bool use64;
        bool ok = factor_any<N>(u, len, a32, G, edge, cfg.cond_fp64, F32, F64, use64);
        if (use64) st |= ST_FP64;
        if (ok) {
          double delta[M];
          const int steps = cfg.mode == POLISH_SOLVE ? cfg.steps : 0;
          for (int s = 0; s < steps; ++s) {
            newton_step<N>(F32, F64, use64, gr, delta);
#pragma unroll
            for (int i = 0; i < N; ++i) {
              tf[i][0] = (float)(t[i][0] + delta[2 * i]);
              tf[i][1] = edge[i] ? tf[i][1] : (float)(t[i][1] + delta[2 * i + 1]);
              t[i][0] = tf[i][0];
              t[i][1] = tf[i][1];
            }
            grad64<N>(G, t, len, u, gr);
          }
          // residual at the returned parameters
          newton_step<N>(F32, F64, use64, gr, delta);
          float worst = 0.f;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            float w2 = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              float w = a32[i][0][c] * (float)delta[2 * i] + a32[i][1][c] * (float)delta[2 * i + 1];
              w2 = fmaf(w, w, w2);
            }
            worst = fmaxf(worst, w2);
          }
          rho = sqrtf(worst);
          if (!isfinite(rho)) rho = INFINITY;
        }
        lmin = len[0];
#pragma unroll
        for (int k = 1; k <= N; ++k) lmin = fmin(lmin, len[k]);
      }
      if (!(st & ST_REPEAT) && !(lmin >= (double)cfg.deg_tol)) st |= ST_DEGENERATE;
    }
    // validity (closed intervals) and boundary distance
    bool inside = true;
    float bd = INFINITY;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float t0 = tf[i][0], t1 = tf[i][1];
      inside = inside && t0 >= 0.f && t0 <= 1.f && (edge[i] || (t1 >= 0.f && t1 <= 1.f));
      float di = fminf(t0, 1.f - t0) * h1[i];
      if (!edge[i]) di = fminf(di, fminf(t1, 1.f - t1) * h2[i]);
      bd = fminf(bd, di);
    }
    if (st & ST_INVALID) inside = false;
    if (inside) st |= ST_VALID;
    const bool solved = rho <= cfg.solved_tol && !(st & (ST_DEGENERATE | ST_REPEAT | ST_NONFINITE | ST_INVALID));
    if (solved) st |= ST_SOLVED;
    if (cfg.mode == POLISH_SOLVE) {
      float2* To = reinterpret_cast<float2*>(T) + g * (uint64_t)n_max;
#pragma unroll
      for (int i = 0; i < N; ++i) To[i] = make_float2(tf[i][0], tf[i][1]);
      status[g] = st;
      if (X) {
        float* Xo = X + g * (uint64_t)n_max * 3;
#pragma unroll
        for (int i = 0; i < kMaxOrder; ++i)
          if (i < n_max)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              double x = i < N ? fma(G.a[i][1][c], t[i][1], fma(G.a[i][0][c], t[i][0], G.b[i][c])) + S.centre[c] : 0.0;
              Xo[3 * i + c] = (float)x;
            }
      }
      if (Lout) {
        double Ls = 0.0;
        if (!(st & ST_INVALID) && finite) {
          if (st & ST_REPEAT) grad64<N>(G, t, len, u, gr);
#pragma unroll
          for (int k = 0; k <= N; ++k) Ls += len[k];
        } else {
          Ls = NAN;
        }
        Lout[g] = (float)Ls;
      }
    }
    if (rho_out) rho_out[g] = rho;
    if (mask_out) mask_out[g] = inside ? 1 : 0;
    if (bdist_out) bdist_out[g] = bd;
  }
}

template <int N>
static cudaError_t launch_polish_n(const SceneDev& S, const BatchDev& B, const PolishCfg& cfg, uint64_t n_local,
                                   const uint64_t* list, float* T, float* X, float* L, uint8_t* status, float* rho,
                                   uint8_t* mask, float* bdist, cudaStream_t stream, int n_sm) {
  size_t smem = (size_t)S.n_obj * (kRec64 * sizeof(double) + (kRec32 + kAux) * sizeof(float));
  int use_smem = smem <= 160 * 1024;
  if (!use_smem) smem = 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(polish_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, polish_kernel<N>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t want = (n_local + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)n_sm * (uint64_t)per_sm;
  unsigned grid = (unsigned)(want < cap ? want : cap);
  if (grid == 0) return cudaSuccess;
  polish_kernel<N><<<grid, kThreads, smem, stream>>>(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist,
                                                      use_smem);
  return cudaGetLastError();
}

cudaError_t launch_polish(int n, const SceneDev& S, const BatchDev& B, const PolishCfg& cfg, uint64_t n_local,
                          const uint64_t* list, float* T, float* X, float* L, uint8_t* status, float* rho,
                          uint8_t* mask, float* bdist, cudaStream_t stream, int n_sm, int* err) {
  (void)err;
  switch (n) {
    case 1: return launch_polish_n<1>(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist, stream, n_sm);
    case 2: return launch_polish_n<2>(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist, stream, n_sm);
    case 3: return launch_polish_n<3>(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist, stream, n_sm);
    case 4: return launch_polish_n<4>(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist, stream, n_sm);
    case 5: return launch_polish_n<5>(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist, stream, n_sm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpt
