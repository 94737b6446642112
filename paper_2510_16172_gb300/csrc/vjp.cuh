// vjp.cuh -- per-path vector-Jacobian product of the solution (Sec. III-D)
// and the warp-aggregated sums over paths, shared by the backward kernels and
// the fused polish + backward.
//
// At a solution grad_T L = 0 (Eq. 8), so for a loss l = sum_i dX_i . x_i + dL L
// the product through T*(theta) is u^T d(grad_T L)/dtheta with H u = -v,
// v = dl/dT = A^T dX + dL grad_T L (Eq. 11-13; H symmetric).
#pragma once

#include "blocktri.cuh"

namespace fpt {

// A path carries a point cotangent when one of its dX entries is non-zero.  A path whose
// cotangents are all zero contributes exactly zero to the sums, so the adjoint skips it.
template <int N>
__device__ __forceinline__ bool has_point_cotangent(const float* __restrict__ dX, uint64_t g, int n_max) {
  if (!dX) return false;
  const float* p = dX + g * (uint64_t)n_max * 3;
  bool any = false;
#pragma unroll
  for (int k = 0; k < 3 * N; ++k) any = any || p[k] != 0.f;
  return any;
}

// Warp-aggregated accumulate of `cnt` values into acc[base + k] (or, without
// shared accumulators, into gacc[gbase + k]).  Lanes with base < 0 add
// nothing.  If every adding lane has the same base the warp sums its values
// and one lane adds them (the common case: neighbouring paths share objects).
// Otherwise the lanes that share a target are grouped and each group's values
// are summed onto one lane first, so that no two lanes of the warp add to the
// same address: a float atomic on shared memory is a compare-and-swap loop,
// which every colliding lane would repeat.  Groups that are contiguous runs of
// lanes (neighbouring entries of an index-ordered path list) are summed by a
// segmented scan, other groups by pulling one member per round.  CNT <= 32.
template <int CNT>
__device__ __forceinline__ void warp_accumulate(float* acc, int base, const float (&v)[CNT], bool shared_acc,
                                                double* gacc, int gbase) {
  const unsigned full = 0xffffffffu;
  const unsigned adding = __ballot_sync(full, base >= 0);
  if (!adding) return;
  const int lane = (int)(threadIdx.x & 31);
  const int leader = __ffs(adding) - 1;
  const int b0 = __shfl_sync(full, base, leader);
  const bool uniform = __all_sync(full, base < 0 || base == b0);
  if (uniform) {
    // butterfly sums leave every lane with all CNT totals; lane k adds total k, so the CNT
    // additions are one warp instruction instead of CNT single-lane ones
    const int g0 = __shfl_sync(full, gbase, leader);
    float mine = 0.f;
#pragma unroll
    for (int k = 0; k < CNT; ++k) {
      float x = base >= 0 ? v[k] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(full, x, o);
      if (lane == k) mine = x;
    }
    if (lane < CNT) {
      if (shared_acc)
        atomicAdd(acc + b0 + lane, mine);
      else
        atomicAdd(gacc + g0 + lane, (double)mine);
    }
    return;
  }
  const unsigned peers = __match_any_sync(full, base);  // the lanes with this lane's target
  const int first = __ffs(peers) - 1;
  const unsigned gsize = (unsigned)__popc(peers);
  const unsigned maxg = __reduce_max_sync(full, base >= 0 ? gsize : 1u);
  float s[CNT];
#pragma unroll
  for (int k = 0; k < CNT; ++k) s[k] = v[k];
  bool owner = base >= 0;  // the lane that adds its group's sum (every adding lane when all targets differ)
  if (maxg > 1) {
    const bool run = base < 0 || (peers >> first) == (gsize == 32u ? full : (1u << gsize) - 1u);
    if (maxg > 4 && __all_sync(full, run)) {
      // segmented inclusive scan: the last lane of each run ends with the run's sum
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const bool in = lane - o >= first;
#pragma unroll
        for (int k = 0; k < CNT; ++k) {
          const float y = __shfl_up_sync(full, s[k], o);
          if (in) s[k] += y;
        }
      }
      owner = base >= 0 && lane == 31 - __clz(peers);
    } else {
      // the first lane of each group pulls its other members' values, one member per round
      unsigned rest = peers & (peers - 1u);
      for (unsigned r = 1; r < maxg; ++r) {
        const bool pull = lane == first && rest != 0u;
        const int src = pull ? __ffs(rest) - 1 : lane;
#pragma unroll
        for (int k = 0; k < CNT; ++k) {
          const float y = __shfl_sync(full, v[k], src);
          if (pull) s[k] += y;
        }
        if (pull) rest &= rest - 1u;
      }
      owner = base >= 0 && lane == first;
    }
  }
  if (owner) {
#pragma unroll
    for (int k = 0; k < CNT; ++k) {
      if (shared_acc)
        atomicAdd(acc + base + k, s[k]);
      else
        atomicAdd(gacc + gbase + k, (double)s[k]);
    }
  }
}

// Per-path VJP (Sec. III-D) from the unit segment directions u_j, inverse
// lengths il_j, dd_i = u_i - u_{i+1}, the basis vectors a, the parameters t and
// a factorisation F of the Hessian: solve H lam = -v with v = A^T dX + dL g,
// g_i = A_i^T dd_i, and form the per-slot gradients (d/db, d/da1, d/da2) and
// the TX / RX gradients.
template <typename R, int N>
__device__ __forceinline__ void vjp_solved(const R (&u)[N + 1][3], const R (&il)[N + 1], const R (&dd)[N][3],
                                           const R (&a)[N][2][3], const R (&t)[N][2], const BlockTri<R, N>& F,
                                           const R (&dx)[N][3], R dl, R (&gb)[N][9], R (&gtx)[3], R (&grx)[3]) {
  constexpr int M = 2 * N;
  R r[M], lam[M];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const R gk = a[i][k][0] * dd[i][0] + a[i][k][1] * dd[i][1] + a[i][k][2] * dd[i][2];
      const R ak = a[i][k][0] * dx[i][0] + a[i][k][1] * dx[i][1] + a[i][k][2] * dx[i][2];
      r[2 * i + k] = -(ak + dl * gk);
    }
  solve_hessian<R, N>(F, r, lam);
  // q_j = M_j Dw_j with w_i = A_i lam_i
  R q[N + 1][3];
#pragma unroll
  for (int jj = 0; jj <= N; ++jj) {
    R dw[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      R x = R(0);
      if (jj < N) x += a[jj][0][c] * lam[2 * jj] + a[jj][1][c] * lam[2 * jj + 1];
      if (jj > 0) x -= a[jj - 1][0][c] * lam[2 * jj - 2] + a[jj - 1][1][c] * lam[2 * jj - 1];
      dw[c] = x;
    }
    const R ud = u[jj][0] * dw[0] + u[jj][1] * dw[1] + u[jj][2] * dw[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) q[jj][c] = (dw[c] - u[jj][c] * ud) * il[jj];
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R e = dx[i][c] + dl * dd[i][c] + (q[i][c] - q[i + 1][c]);
      gb[i][c] = e;
      gb[i][3 + c] = e * t[i][0] + dd[i][c] * lam[2 * i];
      gb[i][6 + c] = e * t[i][1] + dd[i][c] * lam[2 * i + 1];
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gtx[c] = -dl * u[0][c] - q[0][c];
    grx[c] = dl * u[N][c] + q[N][c];
  }
}

// Per-path VJP from the segment vectors z_j in precision R: factorise the
// Hessian at z and call vjp_solved.  Returns false (and no gradient) if the
// pivot test fails.
template <typename R, int N>
__device__ __forceinline__ bool path_vjp(const R (&z)[N + 1][3], const R (&a)[N][2][3], const R (&t)[N][2],
                                         const bool (&edge)[N], const R (&dx)[N][3], R dl, R cond,
                                         R (&gb)[N][9], R (&gtx)[3], R (&grx)[3]) {
  R u[N + 1][3], il[N + 1];
#pragma unroll
  for (int jj = 0; jj <= N; ++jj) {
    const R e = z[jj][0] * z[jj][0] + z[jj][1] * z[jj][1] + z[jj][2] * z[jj][2];
    const R r = e > R(0) ? rsqrt_r<R>(e) : R(0);
    il[jj] = r;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[jj][c] = z[jj][c] * r;
  }
  R dd[N][3];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) dd[i][c] = u[i][c] - u[i + 1][c];
  BlockTri<R, N> F;
  if (!factor_hessian<R, N>(u, il, a, edge, cond, F)) return false;
  vjp_solved<R, N>(u, il, dd, a, t, F, dx, dl, gb, gtx, grx);
  return true;
}

}  // namespace fpt
