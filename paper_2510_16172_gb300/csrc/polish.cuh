// polish.cuh -- stationarity polish, residual and validity, one thread per path.
//
// After BFGS (Sec. III-C) each path takes `steps` Newton steps on Eq. 5 whose
// gradient is formed in extended precision and whose Hessian system (block
// tridiagonal, blocktri.cuh) is solved in FP32, or in FP64 when a pivot is
// ill-conditioned.  The extended precision is double-float arithmetic (ff.cuh,
// about 2^-46 relative; the default, since GB300's FP64 rate is a small
// fraction of its FP32 rate) or FP64 (validation mode).  The parameters are
// carried in that precision through the steps.  The first-order condition of
// Eq. 8 measures the result: rho = max_i |A_i delta_i| (metres), where delta
// solves H delta = -grad_T L at the final parameters (H factorised there);
// T, X and L are then rounded to FP32 for output.
// The validity test (Sec. I, Sec. III: points inside their objects) uses
// closed intervals on the output t.
//
// The same kernel evaluates rho, validity and the boundary distance at
// caller-given parameters (POLISH_VALIDITY) without changing them.
#pragma once

#include "ff.cuh"
#include "fpt_kernels.h"
#include "vjp.cuh"

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

// Double-float geometry of one path: Delta b_j as pairs, basis vectors as
// (hi, lo) floats.
template <int N>
struct GeoFF {
  ff db[N + 1][3];
  float ah[N][2][3], al[N][2][3];
};

// Double-float segment data and gradient at t (pairs).  Outputs the unit
// directions and inverse lengths rounded to float (for the Hessian), the
// lengths, and the gradient g_i = A_i^T (u_i - u_{i+1}) in float (the
// difference u_i - u_{i+1} is formed in double-float before rounding).
template <int N>
__device__ __forceinline__ void gradff(const GeoFF<N>& G, const ff (&t)[N][2], float (&uf)[N + 1][3],
                                       float (&ilf)[N + 1], ff (&len)[N + 1], float (&g)[2 * N],
                                       float (&dd)[N][3]) {
  ff uo[N + 1][3];
  ff w[N][3];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ff p1 = two_prod(G.ah[i][0][c], t[i][0].hi);
      ff p2 = two_prod(G.ah[i][1][c], t[i][1].hi);
      ff sm = two_sum(p1.hi, p2.hi);
      float lo = __fadd_rn(sm.lo, __fadd_rn(p1.lo, p2.lo));
      lo = __fmaf_rn(G.ah[i][0][c], t[i][0].lo, lo);
      lo = __fmaf_rn(G.al[i][0][c], t[i][0].hi, lo);
      lo = __fmaf_rn(G.ah[i][1][c], t[i][1].lo, lo);
      lo = __fmaf_rn(G.al[i][1][c], t[i][1].hi, lo);
      w[i][c] = two_sum(sm.hi, lo);
    }
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    ff z[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ff v = G.db[j][c];
      if (j < N) v = ff_add(v, w[j][c]);
      if (j > 0) v = ff_sub(v, w[j - 1][c]);
      z[c] = v;
    }
    // |z|^2 in double-float
    ff p0 = two_prod(z[0].hi, z[0].hi), p1 = two_prod(z[1].hi, z[1].hi), p2 = two_prod(z[2].hi, z[2].hi);
    ff s1 = two_sum(p0.hi, p1.hi);
    ff s2 = two_sum(s1.hi, p2.hi);
    float lo = __fadd_rn(__fadd_rn(s1.lo, s2.lo), __fadd_rn(__fadd_rn(p0.lo, p1.lo), p2.lo));
    float cross = __fmaf_rn(z[0].hi, z[0].lo, __fmaf_rn(z[1].hi, z[1].lo, __fmul_rn(z[2].hi, z[2].lo)));
    lo = __fmaf_rn(2.f, cross, lo);
    ff e = fast_two_sum(s2.hi, lo);
    ff r = e.hi > 0.f ? ff_rsqrt(e) : ff{0.f, 0.f};
    len[j] = ff_mul(e, r);
    ilf[j] = r.hi;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uo[j][c] = ff_mul(z[c], r);
      uf[j][c] = uo[j][c].hi;
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float (&d)[3] = dd[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ff dc = ff_sub(uo[i][c], uo[i + 1][c]);
      d[c] = __fadd_rn(dc.hi, dc.lo);
    }
    g[2 * i] = fmaf(G.ah[i][0][2], d[2], fmaf(G.ah[i][0][1], d[1], G.ah[i][0][0] * d[0]));
    g[2 * i + 1] = fmaf(G.ah[i][1][2], d[2], fmaf(G.ah[i][1][1], d[1], G.ah[i][1][0] * d[0]));
  }
}

// Validity (closed intervals on the output t) and signed boundary distance.
template <int N>
__device__ __forceinline__ bool validity(const float (&tf)[N][2], const bool (&edge)[N], const float (&h1)[N],
                                         const float (&h2)[N], float& bd) {
  bool inside = true;
  bd = INFINITY;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float t0 = tf[i][0], t1 = tf[i][1];
    inside = inside && t0 >= 0.f && t0 <= 1.f && (edge[i] || (t1 >= 0.f && t1 <= 1.f));
    float di = fminf(t0, 1.f - t0) * h1[i];
    if (!edge[i]) di = fminf(di, fminf(t1, 1.f - t1) * h2[i]);
    bd = fminf(bd, di);
  }
  return inside;
}

__device__ __forceinline__ uint8_t final_status(uint8_t st, bool inside, float rho, float solved_tol) {
  if (st & ST_INVALID) inside = false;
  if (inside) st |= ST_VALID;
  if (rho <= solved_tol && !(st & (ST_DEGENERATE | ST_REPEAT | ST_NONFINITE | ST_INVALID))) st |= ST_SOLVED;
  return st;
}

template <int N>
__device__ __forceinline__ float world_max(const float (&a)[N][2][3], const float (&delta)[2 * N]) {
  float worst = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float w2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float w = fmaf(a[i][1][c], delta[2 * i + 1], a[i][0][c] * delta[2 * i]);
      w2 = fmaf(w, w, w2);
    }
    worst = fmaxf(worst, w2);
  }
  float r = sqrtf(worst);
  return isfinite(r) ? r : INFINITY;
}

// H^{-1}(-g) with the FP32 factorisation, or the FP64 one when the FP32 pivots failed.
template <int N>
__device__ __forceinline__ void newton_dir(const BlockTri<float, N>& F32, const BlockTri<double, N>& F64, bool use64,
                                           const float (&g)[2 * N], float (&delta)[2 * N]) {
  if (use64) {
    double r[2 * N], x[2 * N];
#pragma unroll
    for (int k = 0; k < 2 * N; ++k) r[k] = -(double)g[k];
    solve_hessian<double, N>(F64, r, x);
#pragma unroll
    for (int k = 0; k < 2 * N; ++k) delta[k] = (float)x[k];
  } else {
    float r[2 * N];
#pragma unroll
    for (int k = 0; k < 2 * N; ++k) r[k] = -g[k];
    solve_hessian<float, N>(F32, r, delta);
  }
}

// ---------------------------------------------------------------------------
// double-float polish (default)
// ---------------------------------------------------------------------------
// Register budget of the double-float polish: up to order 3 the kernel fits in
// 168 registers without spilling, which allows 3 CTAs per SM instead of 2; at
// order 4 the same bound spills 48 bytes (left alone ptxas takes 231 registers,
// two CTAs per SM).
template <int N>
constexpr int kPolishMinBlocks = N <= 4 ? 3 : 1;

// Output slots a kernel of order N writes in its unrolled loop (slots past N
// get zeros); in batches with longer sequences the host clears the later slots
// before the solve.
template <int N>
constexpr int kSlots = N > kMaxBfgsOrder ? N : kMaxBfgsOrder;

// use_smem bits of the polish kernels: records staged, gradient sums in shared memory.
constexpr int kSmemRecords = 1;
constexpr int kSmemAcc = 2;

// kGrad: the implicit backward fused in (fpt_solve_grad).  The polished path's
// geometry, unit directions, inverse lengths, u_i - u_{i+1} and the Hessian
// factorisation at the returned point are still in registers, so the VJP
// costs one block-tridiagonal solve and the sums.  The adjoint's stricter
// pivot test is taken on the same factorisation; paths that fail it -- or
// whose polish went to the FP64 pass -- are listed for the FP64 adjoint pass.
template <int N, bool kGrad>
__global__ void __launch_bounds__(kThreads, kPolishMinBlocks<N>) polish_ff_kernel(
    SceneDev S, BatchDev B, PolishCfg cfg, uint64_t n_local, const PathRec* __restrict__ list,
    float* __restrict__ T, float* __restrict__ X, float* __restrict__ Lout, uint8_t* __restrict__ status,
    float* __restrict__ rho_out, uint8_t* __restrict__ mask_out, float* __restrict__ bdist_out, int use_smem,
    uint32_t* __restrict__ rescue_list, unsigned* __restrict__ rescue_count, GradCfg gc,
    const uint32_t* __restrict__ in_list, const unsigned* __restrict__ in_count, uint32_t* __restrict__ step_list,
    unsigned* __restrict__ step_count, float* __restrict__ step_delta) {
  constexpr int M = 2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const float* rec32 = S.rec32;
  const float* reclo = S.reclo;
  const float* aux = S.aux;
  float* s_acc = nullptr;
  if (use_smem & kSmemRecords) {
    float* s32 = reinterpret_cast<float*>(smem_raw);
    float* slo = s32 + S.n_obj * kRec32;
    float* sax = slo + S.n_obj * kRecLo;
    stage(s32, S.rec32, S.n_obj * kRec32);
    stage(slo, S.reclo, S.n_obj * kRecLo);
    stage(sax, S.aux, S.n_obj * kAux);
    rec32 = s32;
    reclo = slo;
    aux = sax;
    s_acc = sax + S.n_obj * kAux;
  }
  const int n_acc = S.n_obj * 9 + 3 * (S.n_tx + S.n_rx);
  const int acc_tx = S.n_obj * 9, acc_rx = acc_tx + 3 * S.n_tx;
  const bool sm_acc = kGrad && (use_smem & kSmemAcc);
  if (sm_acc)
    for (int k = threadIdx.x; k < n_acc; k += blockDim.x) s_acc[k] = 0.f;
  __syncthreads();
  const int n_max = B.n_max;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // second pass: only the paths the first pass listed for a Newton step
  const uint64_t n_iter = in_list ? (uint64_t)*in_count : n_local;
  int tiles = 0;
  for (uint64_t k0 = (uint64_t)blockIdx.x * blockDim.x; k0 < n_iter; k0 += stride) {
    const uint64_t k = k0 + threadIdx.x;
    const bool have = k < n_iter;
    const uint64_t j = have ? (in_list ? (uint64_t)in_list[k] : k) : 0;
    // per-path gradient terms (kGrad), summed over the warp below
    float gb[N][9], gtx[3], grx[3];
    int acc_id[N], acc_t = -1, acc_r = -1;
    if constexpr (kGrad) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        acc_id[i] = -1;
#pragma unroll
        for (int k = 0; k < 9; ++k) gb[i][k] = 0.f;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) gtx[c] = grx[c] = 0.f;
    }
    if (have) {
      PathDesc d;
      fetch_path_n<N>(B, list, j, d);
      const uint64_t g = d.g;
      uint8_t st = d.flags;
      if (cfg.mode == POLISH_SOLVE) st |= status[g] & (ST_CONVERGED | ST_NONFINITE | ST_DEGENERATE);
      // geometry: b as hi + lo, A as hi + lo
      GeoFF<N> G;
      bool edge[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float* r = rec32 + kRec32 * d.ids[i];
        const float* rl = reclo + kRecLo * d.ids[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          G.ah[i][0][c] = r[6 + c];
          G.ah[i][1][c] = r[9 + c];
          G.al[i][0][c] = rl[c];
          G.al[i][1][c] = rl[3 + c];
        }
        edge[i] = aux[kAux * d.ids[i] + 2] != 0.f;
      }
      {
        float bh[N + 2][3], bl[N + 2][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          bh[0][c] = __ldg(S.tx32 + kEnd32 * d.tx + c);
          bl[0][c] = __ldg(S.tx32 + kEnd32 * d.tx + 3 + c);
          bh[N + 1][c] = __ldg(S.rx32 + kEnd32 * d.rx + c);
          bl[N + 1][c] = __ldg(S.rx32 + kEnd32 * d.rx + 3 + c);
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const float* r = rec32 + kRec32 * d.ids[i];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            bh[i + 1][c] = r[c];
            bl[i + 1][c] = r[3 + c];
          }
        }
#pragma unroll
        for (int jj = 0; jj <= N; ++jj)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            ff sd = two_sum(bh[jj + 1][c], -bh[jj][c]);
            G.db[jj][c] = fast_two_sum(sd.hi, __fadd_rn(sd.lo, __fsub_rn(bl[jj + 1][c], bl[jj][c])));
          }
      }
      // parameters
      const float2* Ti = reinterpret_cast<const float2*>(T) + g * (uint64_t)n_max;
      ff t[N][2];
      bool finite = true;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float2 v = Ti[i];
        t[i][0] = ff{v.x, 0.f};
        t[i][1] = ff{v.y, 0.f};
        finite = finite && isfinite(v.x) && isfinite(v.y);
      }
      if (!finite) st |= ST_NONFINITE;
      float rho = INFINITY;
      ff len[N + 1];
#pragma unroll
      for (int k = 0; k <= N; ++k) len[k] = ff{0.f, 0.f};
      // state the fused backward reuses
      float uf[N + 1][3], ilf[N + 1], dd[N][3];
      BlockTri<float, N> F32;
      bool fact_ok = false, adj_ok = false, listed64 = false, pending = false;
      if (!(st & ST_INVALID) && finite) {
        // Newton steps, then the residual: one gradient, factorisation and solve per pass (one code copy each)
        const int steps = cfg.mode == POLISH_SOLVE ? cfg.steps : 0;
        // the second pass starts with the Newton step the first pass computed (same arithmetic as one pass)
        float delta[M];
        bool stepped = in_list != nullptr;
        if (stepped) {
#pragma unroll
          for (int q = 0; q < M; ++q) delta[q] = step_delta[k * M + q];
        }
        for (int s = stepped ? 1 : 0;; ++s) {
          if (stepped) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
              ff a0 = two_sum(t[i][0].hi, delta[2 * i]);
              t[i][0] = fast_two_sum(a0.hi, __fadd_rn(a0.lo, t[i][0].lo));
              if (!edge[i]) {
                ff a1 = two_sum(t[i][1].hi, delta[2 * i + 1]);
                t[i][1] = fast_two_sum(a1.hi, __fadd_rn(a1.lo, t[i][1].lo));
              }
            }
          }
          float gr[M];
          gradff<N>(G, t, uf, ilf, len, gr, dd);
          float lmin = len[0].hi;
#pragma unroll
          for (int k = 1; k <= N; ++k) lmin = fminf(lmin, len[k].hi);
          if ((st & (ST_REPEAT | ST_DEGENERATE)) || !(lmin >= cfg.deg_tol)) {
            if (!(st & ST_REPEAT)) st |= ST_DEGENERATE;  // a kink: no Newton system
            break;
          }
          bool strict = true;
          fact_ok = factor_hessian<float, N>(uf, ilf, G.ah, edge, cfg.cond_fp64, F32, kGrad ? gc.cond_adj : 0.f,
                                             &strict);
          if (!fact_ok) {
            // FP32 pivots failed: the FP64 pass over the rescue list redoes this path
            st |= ST_FP64;
            rescue_list[atomicAdd(rescue_count, 1u)] = (uint32_t)j;
            listed64 = true;
            break;
          }
          float r[M];
#pragma unroll
          for (int q = 0; q < M; ++q) r[q] = -gr[q];
          solve_hessian<float, N>(F32, r, delta);
          if (s >= steps || (step_list && s == 0)) {
            // at the returned point: the residual, and for the adjoint its own pivot test.  The first
            // pass returns the solver's point when it already meets the bound; otherwise it lists the
            // path with its Newton step, and the second pass continues from there.
            const float r0 = world_max<N>(G.ah, delta);
            if (s >= steps || r0 <= cfg.solved_tol || (cfg.radius > 0.f && r0 > cfg.radius)) {
              rho = r0;
              adj_ok = strict;
            } else {
              // one atomic per group of lanes that list a path here together
              const unsigned grp = __activemask();
              const int lane = (int)(threadIdx.x & 31), first = __ffs(grp) - 1;
              unsigned slot = 0;
              if (lane == first) slot = atomicAdd(step_count, (unsigned)__popc(grp));
              slot = __shfl_sync(grp, slot, first) + (unsigned)__popc(grp & ((1u << lane) - 1u));
              step_list[slot] = (uint32_t)j;
#pragma unroll
              for (int q = 0; q < M; ++q) step_delta[(uint64_t)slot * M + q] = delta[q];
              pending = true;
            }
            break;
          }
          stepped = true;
        }
      }
      float tf[N][2], h1[N], h2[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        tf[i][0] = t[i][0].hi;
        tf[i][1] = t[i][1].hi;
        h1[i] = aux[kAux * d.ids[i]];
        h2[i] = aux[kAux * d.ids[i] + 1];
      }
      float bd;
      const bool inside = validity<N>(tf, edge, h1, h2, bd);
      st = final_status(st, inside, rho, cfg.solved_tol);
      if constexpr (kGrad) {
        if (pending) {
          // the second pass forms this path's adjoint
        } else if (listed64) {
          // the FP64 polish decides this path's status; the FP64 adjoint pass reads it
          gc.rescue_list[atomicAdd(gc.rescue_count, 1u)] = (uint32_t)j;
        } else if (!(st & (ST_REPEAT | ST_INVALID | ST_DEGENERATE | ST_NONFINITE)) &&
                   (has_point_cotangent<N>(gc.dX, g, n_max) ||
                    (gc.dL ? gc.dL[g] != 0.f : (gc.dl_mask && (st & gc.dl_mask) == gc.dl_mask)))) {
          // (a path with no cotangent contributes exactly zero and is skipped)
          if (fact_ok && adj_ok) {
            const float dl = gc.dL ? gc.dL[g] : ((gc.dl_mask && (st & gc.dl_mask) == gc.dl_mask) ? 1.f : 0.f);
            float dx[N][3];
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
              for (int c = 0; c < 3; ++c) dx[i][c] = gc.dX ? gc.dX[(g * (uint64_t)n_max + i) * 3 + c] : 0.f;
            vjp_solved<float, N>(uf, ilf, dd, G.ah, tf, F32, dx, dl, gb, gtx, grx);
#pragma unroll
            for (int i = 0; i < N; ++i) acc_id[i] = d.ids[i];
            acc_t = d.tx;
            acc_r = d.rx;
          } else {
            gc.rescue_list[atomicAdd(gc.rescue_count, 1u)] = (uint32_t)j;
          }
        }
      }
      if (cfg.mode == POLISH_SOLVE && !pending) {
        float2* To = reinterpret_cast<float2*>(T) + g * (uint64_t)n_max;
#pragma unroll
        for (int i = 0; i < N; ++i) To[i] = make_float2(tf[i][0], tf[i][1]);
        status[g] = st;
        if (X) {
          float* Xo = X + g * (uint64_t)n_max * 3;
#pragma unroll
          for (int i = 0; i < kSlots<N>; ++i)
            if (i < n_max)
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                float x = 0.f;
                if (i < N) {
                  ff p1 = two_prod(G.ah[i][0][c], t[i][0].hi);
                  ff p2 = two_prod(G.ah[i][1][c], t[i][1].hi);
                  float lo = __fadd_rn(p1.lo, p2.lo);
                  lo = __fmaf_rn(G.ah[i][0][c], t[i][0].lo, lo);
                  lo = __fmaf_rn(G.al[i][0][c], t[i][0].hi, lo);
                  lo = __fmaf_rn(G.ah[i][1][c], t[i][1].lo, lo);
                  lo = __fmaf_rn(G.al[i][1][c], t[i][1].hi, lo);
                  ff w = ff_add(p1, ff{p2.hi, lo});
                  const float* rb = rec32 + kRec32 * d.ids[i];
                  ff xr = ff_add(ff{rb[c], rb[3 + c]}, w);
                  ff xw = ff_add(xr, ff{S.centre_hi[c], S.centre_lo[c]});
                  x = __fadd_rn(xw.hi, xw.lo);
                }
                Xo[3 * i + c] = x;
              }
        }
        if (Lout) {
          ff Ls{0.f, 0.f};
#pragma unroll
          for (int k = 0; k <= N; ++k) Ls = ff_add(Ls, len[k]);
          Lout[g] = (!(st & ST_INVALID) && finite) ? __fadd_rn(Ls.hi, Ls.lo) : NAN;
        }
      }
      if (!pending) {
        if (rho_out) rho_out[g] = rho;
        if (mask_out) mask_out[g] = (st & ST_VALID) ? 1 : 0;
        if (bdist_out) bdist_out[g] = bd;
      }
    }
    if constexpr (kGrad) {
      // sums over paths (all lanes of the warp take part)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int id = acc_id[i];
        warp_accumulate<9>(s_acc, id >= 0 ? 9 * id : -1, gb[i], sm_acc, gc.gacc, 9 * id);
      }
      warp_accumulate<3>(s_acc, acc_t >= 0 ? acc_tx + 3 * acc_t : -1, gtx, sm_acc, gc.gacc, acc_tx + 3 * acc_t);
      warp_accumulate<3>(s_acc, acc_r >= 0 ? acc_rx + 3 * acc_r : -1, grx, sm_acc, gc.gacc, acc_rx + 3 * acc_r);
      if (sm_acc && ++tiles >= gc.flush_tiles) {
        tiles = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < n_acc; k += blockDim.x) {
          const float x = s_acc[k];
          if (x != 0.f) {
            atomicAdd(gc.gacc + k, (double)x);
            s_acc[k] = 0.f;
          }
        }
        __syncthreads();
      }
    }
  }
  if (sm_acc) {
    __syncthreads();
    for (int k = threadIdx.x; k < n_acc; k += blockDim.x) {
      const float x = s_acc[k];
      if (x != 0.f) atomicAdd(gc.gacc + k, (double)x);
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 polish (validation mode: polish_fp64 = 1)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kThreads, kLongOrderMinBlocks<N>)
    polish64_kernel(SceneDev S, BatchDev B, PolishCfg cfg, uint64_t n_local, const PathRec* __restrict__ list,
        float* __restrict__ T, float* __restrict__ X, float* __restrict__ Lout, uint8_t* __restrict__ status,
        float* __restrict__ rho_out, uint8_t* __restrict__ mask_out, float* __restrict__ bdist_out, int use_smem,
        const uint32_t* __restrict__ rescue_list, const unsigned* __restrict__ rescue_count) {
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
  // rescue mode: only the paths the double-float pass listed
  const uint64_t n_iter = rescue_list ? (uint64_t)*rescue_count : n_local;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_iter; k += stride) {
    const uint64_t j = rescue_list ? (uint64_t)rescue_list[k] : k;
    PathDesc d;
    fetch_path_n<N>(B, list, j, d);
    const uint64_t g = d.g;
    uint8_t st = d.flags;
    if (cfg.mode == POLISH_SOLVE) st |= status[g] & (ST_CONVERGED | ST_NONFINITE | ST_DEGENERATE);
    if (rescue_list) st |= ST_FP64;
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
    const float2* Ti = reinterpret_cast<const float2*>(T) + g * (uint64_t)n_max;
    double t[N][2];
    bool finite = true;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float2 v = Ti[i];
      t[i][0] = v.x;
      t[i][1] = v.y;
      finite = finite && isfinite(v.x) && isfinite(v.y);
    }
    if (!finite) st |= ST_NONFINITE;
    double len[N + 1], u[N + 1][3], gr[M];
#pragma unroll
    for (int k = 0; k <= N; ++k) len[k] = 0.0;
    float rho = INFINITY;
    if (!(st & ST_INVALID) && finite) {
      // Newton steps, then the residual, each with the Hessian factorised at the current point
      const int steps = cfg.mode == POLISH_SOLVE ? cfg.steps : 0;
      for (int s = 0;; ++s) {
        grad64<N>(G, t, len, u, gr);
        double lmin = len[0];
#pragma unroll
        for (int k = 1; k <= N; ++k) lmin = fmin(lmin, len[k]);
        if ((st & (ST_REPEAT | ST_DEGENERATE)) || !(lmin >= (double)cfg.deg_tol)) {
          if (!(st & ST_REPEAT)) st |= ST_DEGENERATE;  // a kink: no Newton system
          break;
        }
        BlockTri<float, N> F32;
        BlockTri<double, N> F64;
        float uf[N + 1][3], ilf[N + 1];
#pragma unroll
        for (int jj = 0; jj <= N; ++jj) {
          ilf[jj] = (float)(1.0 / len[jj]);
#pragma unroll
          for (int c = 0; c < 3; ++c) uf[jj][c] = (float)u[jj][c];
        }
        bool use64 = false;
        bool ok = factor_hessian<float, N>(uf, ilf, a32, edge, cfg.cond_fp64, F32);
        if (!ok) {
          use64 = true;
          double il[N + 1];
#pragma unroll
          for (int jj = 0; jj <= N; ++jj) il[jj] = 1.0 / len[jj];
          ok = factor_hessian<double, N>(u, il, G.a, edge, (double)cfg.cond_fp64 * 1e-6, F64);
          st |= ST_FP64;
        }
        if (!ok) break;
        float gf[M], delta[M];
#pragma unroll
        for (int k = 0; k < M; ++k) gf[k] = (float)gr[k];
        newton_dir<N>(F32, F64, use64, gf, delta);
        if (s >= steps) {
          rho = world_max<N>(a32, delta);
          break;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
          t[i][0] += (double)delta[2 * i];
          if (!edge[i]) t[i][1] += (double)delta[2 * i + 1];
        }
      }
    }
    float tf[N][2];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      tf[i][0] = (float)t[i][0];
      tf[i][1] = (float)t[i][1];
    }
    float bd;
    const bool inside = validity<N>(tf, edge, h1, h2, bd);
    st = final_status(st, inside, rho, cfg.solved_tol);
    if (cfg.mode == POLISH_SOLVE) {
      float2* To = reinterpret_cast<float2*>(T) + g * (uint64_t)n_max;
#pragma unroll
      for (int i = 0; i < N; ++i) To[i] = make_float2(tf[i][0], tf[i][1]);
      status[g] = st;
      if (X) {
        float* Xo = X + g * (uint64_t)n_max * 3;
#pragma unroll
        for (int i = 0; i < kSlots<N>; ++i)
          if (i < n_max)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              double x = i < N ? fma(G.a[i][1][c], t[i][1], fma(G.a[i][0][c], t[i][0], G.b[i][c])) + S.centre[c] : 0.0;
              Xo[3 * i + c] = (float)x;
            }
      }
      if (Lout) {
        double Ls = 0.0;
#pragma unroll
        for (int k = 0; k <= N; ++k) Ls += len[k];
        Lout[g] = (!(st & ST_INVALID) && finite) ? (float)Ls : NAN;
      }
    }
    if (rho_out) rho_out[g] = rho;
    if (mask_out) mask_out[g] = (st & ST_VALID) ? 1 : 0;
    if (bdist_out) bdist_out[g] = bd;
  }
}

template <int N>
cudaError_t launch_polish_n(const SceneDev& S, const BatchDev& B, const PolishCfg& cfg, uint64_t n_local,
                                   const PathRec* list, float* T, float* X, float* L, uint8_t* status, float* rho,
                                   uint8_t* mask, float* bdist, cudaStream_t stream, int n_sm, uint32_t* rescue_list,
                                   unsigned* rescue_count, const GradCfg* grad, uint32_t* step_list,
                                   unsigned* step_count, float* step_delta) {
  const bool f64 = cfg.fp64 != 0;
  const size_t smem64 = (size_t)S.n_obj * (kRec64 * sizeof(double) + (kRec32 + kAux) * sizeof(float));
  const size_t smemff = (size_t)S.n_obj * (kRec32 + kRecLo + kAux) * sizeof(float);
  auto grid_of = [&](const void* fn, size_t smem, uint64_t n, unsigned& grid) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    uint64_t want = (n + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)n_sm * (uint64_t)per_sm;
    grid = (unsigned)(want < cap ? want : cap);
    return cudaSuccess;
  };
  const size_t s64 = smem64 <= 160 * 1024 ? smem64 : 0;
  unsigned grid = 0;
  cudaError_t e;
  if (f64 && !grad) {
    e = grid_of((const void*)polish64_kernel<N>, s64, n_local, grid);
    if (e != cudaSuccess || grid == 0) return e;
    polish64_kernel<N><<<grid, kThreads, s64, stream>>>(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist,
                                                         s64 != 0, nullptr, nullptr);
    count_launch();
    return cudaGetLastError();
  }
  if (f64) return cudaErrorInvalidValue;  // the fused backward runs with the double-float polish only
  // shared memory: records, and with the fused backward its per-CTA sums
  int use_smem = 0;
  size_t sff = 0;
  if (smemff <= 160 * 1024) {
    use_smem = kSmemRecords;
    sff = smemff;
    if (grad && grad->acc_in_smem) {
      const size_t acc = (size_t)(9 * S.n_obj + 3 * (S.n_tx + S.n_rx)) * sizeof(float);
      if (sff + acc <= 160 * 1024) {
        use_smem |= kSmemAcc;
        sff += acc;
      }
    }
  }
  e = cudaMemsetAsync(rescue_count, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  GradCfg gc{};
  if (grad) {
    gc = *grad;
    e = cudaMemsetAsync(gc.rescue_count, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
  }
  // adaptive polish: the first pass lists the paths that still need their Newton steps, the second
  // pass (a grid for a quarter of the slice; it strides over the list) takes them
  const bool two_pass = step_list != nullptr && step_delta != nullptr && cfg.mode == POLISH_SOLVE && cfg.steps > 0;
  if (two_pass) {
    e = cudaMemsetAsync(step_count, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
  }
  for (int pass = 0; pass < (two_pass ? 2 : 1); ++pass) {
    const uint32_t* in_l = pass == 1 ? step_list : nullptr;
    const unsigned* in_c = pass == 1 ? step_count : nullptr;
    uint32_t* out_l = two_pass && pass == 0 ? step_list : nullptr;
    unsigned* out_c = two_pass && pass == 0 ? step_count : nullptr;
    const uint64_t n_grid = pass == 1 ? (n_local + 3) / 4 : n_local;
    if (grad) {
      e = grid_of((const void*)polish_ff_kernel<N, true>, sff, n_grid, grid);
      if (e != cudaSuccess || grid == 0) return e;
      polish_ff_kernel<N, true><<<grid, kThreads, sff, stream>>>(S, B, cfg, n_local, list, T, X, L, status, rho,
                                                                 mask, bdist, use_smem, rescue_list, rescue_count, gc,
                                                                 in_l, in_c, out_l, out_c, step_delta);
    } else {
      e = grid_of((const void*)polish_ff_kernel<N, false>, sff, n_grid, grid);
      if (e != cudaSuccess || grid == 0) return e;
      polish_ff_kernel<N, false><<<grid, kThreads, sff, stream>>>(S, B, cfg, n_local, list, T, X, L, status, rho,
                                                                  mask, bdist, use_smem, rescue_list, rescue_count,
                                                                  gc, in_l, in_c, out_l, out_c, step_delta);
    }
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // FP64 pass over the listed paths (its grid covers a few percent of the paths)
  e = grid_of((const void*)polish64_kernel<N>, s64, (n_local + 15) / 16, grid);
  if (e != cudaSuccess || grid == 0) return e;
  polish64_kernel<N><<<grid, kThreads, s64, stream>>>(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist,
                                                       s64 != 0, rescue_list, rescue_count);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess || !grad) return e;
  // FP64 adjoint for the paths the fused kernel listed (final T and status are in place)
  BackwardCfg bc{gc.cond_adj, gc.deg_tol, 0, 0, gc.dL ? (uint8_t)0 : gc.dl_mask};
  bc.dropped = gc.dropped;
  return launch_backward_rescue(N, S, B, bc, n_local, list, T, status, gc.dX, gc.dL, gc.gacc, stream, n_sm,
                                gc.rescue_list, gc.rescue_count);
}

// The launcher of one order as an explicitly instantiable unit: orders up to
// the BFGS orders are instantiated with the dispatcher (k_polish.cu), the
// longer ones each in their own object (k_high.cu).
template <int N>
struct PolishOrder {
  static cudaError_t launch(const SceneDev& S, const BatchDev& B, const PolishCfg& cfg, uint64_t n_local,
                            const PathRec* list, float* T, float* X, float* L, uint8_t* status, float* rho,
                            uint8_t* mask, float* bdist, cudaStream_t stream, int n_sm, uint32_t* rescue_list,
                            unsigned* rescue_count, const GradCfg* grad, uint32_t* step_list, unsigned* step_count,
                            float* step_delta);
};

template <int N>
cudaError_t PolishOrder<N>::launch(const SceneDev& S, const BatchDev& B, const PolishCfg& cfg, uint64_t n_local,
                                   const PathRec* list, float* T, float* X, float* L, uint8_t* status, float* rho,
                                   uint8_t* mask, float* bdist, cudaStream_t stream, int n_sm,
                                   uint32_t* rescue_list, unsigned* rescue_count, const GradCfg* grad,
                                   uint32_t* step_list, unsigned* step_count, float* step_delta) {
  return launch_polish_n<N>(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist, stream, n_sm, rescue_list,
                            rescue_count, grad, step_list, step_count, step_delta);
}

}  // namespace fpt
