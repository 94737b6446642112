// blocktri.cuh -- exact Hessian of Eq. 5 and its block-tridiagonal solve.
//
// With u_j = z_j / |z_j| and M_j = (I - u_j u_j^T) / |z_j| (the derivative of
// u_j with respect to z_j), the Hessian of L(T; A, B) in the unified d = 2
// parameters is block tridiagonal with 2 x 2 blocks:
//   H_ii     = A_i^T (M_i + M_{i+1}) A_i      (slot i touches segments i, i+1)
//   H_i,i+1  = -A_i^T M_{i+1} A_{i+1}
// It is the matrix of the optimality condition used by implicit
// differentiation (Sec. III-D, Eq. 9-12).  An edge's zero second basis vector
// gives a zero row and column; its diagonal entry is set to the edge's first
// diagonal entry so that the coordinate stays decoupled (its right-hand side
// is always zero) and the pivot test sees the path's own scale.
//
// The solve is block LDL^T (block Thomas): D_0 = H_00,
// C_i = H_{i-1,i}^T D_{i-1}^{-1}, D_i = H_ii - C_i H_{i-1,i}; a pivot block
// that is not positive definite, or whose smallest eigenvalue is below
// cond * (largest diagonal entry of its own H_ii), marks the factorisation as
// failed: the elimination cancelled that block down to noise.  The test is
// per block, so objects of very different sizes or distances (a scaling, not
// an ill-conditioning) do not trigger it.
#pragma once

namespace fpt {

template <typename R, int N>
struct BlockTri {
  R Dinv[N][3];     // inverse pivot blocks, symmetric (a, b, c) = [[a b][b c]]
  R C[N][2][2];     // C_i for i >= 1
  R Up[N][2][2];    // H_{i,i+1} for i < N-1
};

template <typename R>
__device__ __forceinline__ R rsqrt_r(R x);
template <>
__device__ __forceinline__ float rsqrt_r<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_r<double>(double x) { return rsqrt(x); }

template <typename R>
__device__ __forceinline__ R sqrt_r(R x);
template <>
__device__ __forceinline__ float sqrt_r<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double sqrt_r<double>(double x) { return sqrt(x); }

// u [N+1][3] unit segment directions, il [N+1] inverse lengths, a [N][2][3],
// edge[N] flags.  Returns false if a pivot fails the test with `cond`; if
// strict_ok is given, it also receives the outcome of the test with
// cond_strict (one factorisation serving two accuracy needs).
template <typename R, int N>
__device__ __forceinline__ bool factor_hessian(const R (&u)[N + 1][3], const R (&il)[N + 1], const R (&a)[N][2][3],
                                               const bool (&edge)[N], R cond, BlockTri<R, N>& F,
                                               R cond_strict = R(0), bool* strict_ok = nullptr) {
  // M_j packed (xx, xy, xz, yy, yz, zz)
  R Mj[N + 1][6];
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    Mj[j][0] = (R(1) - u[j][0] * u[j][0]) * il[j];
    Mj[j][1] = -u[j][0] * u[j][1] * il[j];
    Mj[j][2] = -u[j][0] * u[j][2] * il[j];
    Mj[j][3] = (R(1) - u[j][1] * u[j][1]) * il[j];
    Mj[j][4] = -u[j][1] * u[j][2] * il[j];
    Mj[j][5] = (R(1) - u[j][2] * u[j][2]) * il[j];
  }
  auto mul = [](const R* m, const R* v, R* o) {
    o[0] = m[0] * v[0] + m[1] * v[1] + m[2] * v[2];
    o[1] = m[1] * v[0] + m[3] * v[1] + m[4] * v[2];
    o[2] = m[2] * v[0] + m[4] * v[1] + m[5] * v[2];
  };
  auto dot = [](const R* x, const R* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
  R Hd[N][3];
  R maxdiag = R(0);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    R Ms[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Ms[k] = Mj[i][k] + Mj[i + 1][k];
    R m0[3], m1[3];
    mul(Ms, a[i][0], m0);
    mul(Ms, a[i][1], m1);
    Hd[i][0] = dot(a[i][0], m0);
    Hd[i][1] = dot(a[i][0], m1);
    Hd[i][2] = dot(a[i][1], m1);
    if (edge[i]) {
      Hd[i][1] = R(0);
      Hd[i][2] = Hd[i][0];
    }
    maxdiag = Hd[i][0] > maxdiag ? Hd[i][0] : maxdiag;
    maxdiag = Hd[i][2] > maxdiag ? Hd[i][2] : maxdiag;
    if (i + 1 < N) {
      R n0[3], n1[3];
      mul(Mj[i + 1], a[i + 1][0], n0);
      mul(Mj[i + 1], a[i + 1][1], n1);
      F.Up[i][0][0] = -dot(a[i][0], n0);
      F.Up[i][0][1] = -dot(a[i][0], n1);
      F.Up[i][1][0] = -dot(a[i][1], n0);
      F.Up[i][1][1] = -dot(a[i][1], n1);
      if (edge[i]) F.Up[i][1][0] = F.Up[i][1][1] = R(0);
      if (edge[i + 1]) F.Up[i][0][1] = F.Up[i][1][1] = R(0);
    }
  }
  bool ok = maxdiag > R(0);
  R D[3] = {Hd[0][0], Hd[0][1], Hd[0][2]};
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (i > 0) {
      // C_i = Up_{i-1}^T Dinv_{i-1};  D_i = Hd_i - C_i Up_{i-1}
      const R(&U)[2][2] = F.Up[i - 1];
      const R* Di = F.Dinv[i - 1];
      R c00 = U[0][0] * Di[0] + U[1][0] * Di[1];
      R c01 = U[0][0] * Di[1] + U[1][0] * Di[2];
      R c10 = U[0][1] * Di[0] + U[1][1] * Di[1];
      R c11 = U[0][1] * Di[1] + U[1][1] * Di[2];
      F.C[i][0][0] = c00;
      F.C[i][0][1] = c01;
      F.C[i][1][0] = c10;
      F.C[i][1][1] = c11;
      D[0] = Hd[i][0] - (c00 * U[0][0] + c01 * U[1][0]);
      D[1] = Hd[i][1] - (c00 * U[0][1] + c01 * U[1][1]);
      D[2] = Hd[i][2] - (c10 * U[0][1] + c11 * U[1][1]);
    }
    R det = D[0] * D[2] - D[1] * D[1];
    R half_tr = R(0.5) * (D[0] + D[2]);
    R half_df = R(0.5) * (D[0] - D[2]);
    R lam_min = half_tr - sqrt_r<R>(half_df * half_df + D[1] * D[1]);
    const R own = Hd[i][0] > Hd[i][2] ? Hd[i][0] : Hd[i][2];
    ok = ok && D[0] > R(0) && det > R(0) && lam_min > cond * own;
    if (strict_ok) *strict_ok = *strict_ok && lam_min > cond_strict * own;
    R idet = R(1) / det;
    F.Dinv[i][0] = D[2] * idet;
    F.Dinv[i][1] = -D[1] * idet;
    F.Dinv[i][2] = D[0] * idet;
  }
  return ok;
}

// x = H^{-1} r
template <typename R, int N>
__device__ __forceinline__ void solve_hessian(const BlockTri<R, N>& F, const R (&r)[2 * N], R (&x)[2 * N]) {
  R y[N][2];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    y[i][0] = r[2 * i];
    y[i][1] = r[2 * i + 1];
    if (i > 0) {
      y[i][0] -= F.C[i][0][0] * y[i - 1][0] + F.C[i][0][1] * y[i - 1][1];
      y[i][1] -= F.C[i][1][0] * y[i - 1][0] + F.C[i][1][1] * y[i - 1][1];
    }
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    R b0 = y[i][0], b1 = y[i][1];
    if (i + 1 < N) {
      b0 -= F.Up[i][0][0] * x[2 * i + 2] + F.Up[i][0][1] * x[2 * i + 3];
      b1 -= F.Up[i][1][0] * x[2 * i + 2] + F.Up[i][1][1] * x[2 * i + 3];
    }
    x[2 * i] = F.Dinv[i][0] * b0 + F.Dinv[i][1] * b1;
    x[2 * i + 1] = F.Dinv[i][1] * b0 + F.Dinv[i][2] * b1;
  }
}

}  // namespace fpt
