// unrolled.cuh -- automatic differentiation through the solver's iterations (reverse mode).
//
// Sec. IV-B compares the implicit backward with differentiating through the
// solver steps.  This kernel is that comparison done natively: for one path
// per thread it runs exactly K steps of the unified d = 2 solver from t = 1/2
// (H_0 = I, Eq. 6 rounds from alpha = 1 redone from 0 when they give alpha <= 0,
// alpha capped, BFGS inverse update under the curvature guard), writing the
// iterate, gradient and inverse-Hessian estimate of every step to a tape in
// global memory, then sweeps the steps backwards, forming the adjoints of every
// operation by hand, and sums the parameter adjoints of the loss
// sum dX . X_K + dL L_K like the implicit backward.  The intermediate values of
// a step are recomputed from its tape entry during the sweep.  Above order 5
// the inverse Hessian (forward) and its adjoint (reverse sweep) share one
// column of shared memory per thread, and the sweep reads each step's H from
// the tape where it stands.
#pragma once

#include "bfgs.cuh"
#include <type_traits>

#include "vjp.cuh"

namespace fpt {

// H_k of a step read where it stands on the tape (entry q of thread `me` at
// p[q * stride]), for the orders whose H does not fit in registers.
struct TapeH {
  const float* p;
  uint64_t stride;
  __device__ __forceinline__ float operator[](int q) const { return p[q * stride]; }
};

// Floats of dynamic shared memory for the H columns of a CTA (they precede the sums).
template <int N>
constexpr int kUnrolledSmemH = N > kMaxBfgsOrder ? (2 * N) * (2 * N + 1) / 2 * kThreads : 0;

template <int N>
struct Adj {
  float db[N + 1][3];  // adjoint of Delta b_j
  float a[N][2][3];    // adjoint of the basis vectors
  float bx[N][3];      // adjoint of b_i through the points X_i = A_i t_i + b_i of the loss
};

// Forward of one Eq. 6 attempt from alpha0; records alpha before each round.
template <int N>
__device__ __forceinline__ float fp_forward(const float (&e)[N + 1], const float (&qa)[N + 1], const float (&qc)[N + 1],
                                            float alpha, int rounds, float* hist) {
  for (int k = 0; k < rounds; ++k) {
    hist[k] = alpha;
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int j = 0; j <= N; ++j) {
      const float w = fmaf(alpha, fmaf(alpha, qc[j], 2.f * qa[j]), e[j]);
      const float r = rsqrtf(fmaxf(w, 1e-30f));
      num = fmaf(qa[j], r, num);
      den = fmaf(qc[j], r, den);
    }
    alpha = den > 1e-30f ? fminf(-__fdividef(num, den), kAlphaMax) : 0.f;
  }
  return alpha;
}

// Reverse of the rounds: abar is d(loss)/d(final alpha); adds to eb, qab, qcb.
template <int N>
__device__ __forceinline__ void fp_reverse(const float (&e)[N + 1], const float (&qa)[N + 1], const float (&qc)[N + 1],
                                           int rounds, const float* hist, float abar, float (&eb)[N + 1],
                                           float (&qab)[N + 1], float (&qcb)[N + 1]) {
  for (int k = rounds - 1; k >= 0; --k) {
    const float al = hist[k];
    float w[N + 1], r[N + 1], num = 0.f, den = 0.f;
#pragma unroll
    for (int j = 0; j <= N; ++j) {
      w[j] = fmaf(al, fmaf(al, qc[j], 2.f * qa[j]), e[j]);
      r[j] = rsqrtf(fmaxf(w[j], 1e-30f));
      num = fmaf(qa[j], r[j], num);
      den = fmaf(qc[j], r[j], den);
    }
    // a constant result (no denominator, or the cap): nothing flows further back
    if (!(den > 1e-30f) || -__fdividef(num, den) >= kAlphaMax) return;
    const float numb = -abar / den;
    const float denb = abar * num / (den * den);
    float alb = 0.f;
#pragma unroll
    for (int j = 0; j <= N; ++j) {
      qab[j] += numb * r[j];
      qcb[j] += denb * r[j];
      const float rb = numb * qa[j] + denb * qc[j];
      const float wb = w[j] > 1e-30f ? -0.5f * rb * r[j] * r[j] * r[j] : 0.f;
      eb[j] += wb;
      qab[j] += 2.f * al * wb;
      qcb[j] += al * al * wb;
      alb += wb * (2.f * qa[j] + 2.f * al * qc[j]);
    }
    abar = alb;
  }
}

// Reverse of grad_eval at t: adjoints gb (of g), zb (of z), eb (of e = |z|^2) -> tb, adj.
template <int N>
__device__ __forceinline__ void grad_reverse(const Geo<N>& G, const float (&t)[N][2], const float (&z)[N + 1][3],
                                             const float (&gb)[2 * N], const float (&zb)[N + 1][3],
                                             const float (&eb)[N + 1], float (&tb)[N][2], Adj<N>& adj) {
  float u[N + 1][3], r[N + 1];
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const float e = fmaf(z[j][2], z[j][2], fmaf(z[j][1], z[j][1], z[j][0] * z[j][0]));
    r[j] = rsqrtf(fmaxf(e, 1e-30f));
#pragma unroll
    for (int c = 0; c < 3; ++c) u[j][c] = z[j][c] * r[j];
  }
  float ub[N + 1][3];
#pragma unroll
  for (int j = 0; j <= N; ++j)
#pragma unroll
    for (int c = 0; c < 3; ++c) ub[j][c] = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float db[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float d = u[i][c] - u[i + 1][c];
      db[c] = G.a[i][0][c] * gb[2 * i] + G.a[i][1][c] * gb[2 * i + 1];
      adj.a[i][0][c] += gb[2 * i] * d;
      adj.a[i][1][c] += gb[2 * i + 1] * d;
      ub[i][c] += db[c];
      ub[i + 1][c] -= db[c];
    }
  }
  float wb[N][3];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) wb[i][c] = 0.f;
#pragma unroll
  for (int j = 0; j <= N; ++j) {
    const float uu = u[j][0] * ub[j][0] + u[j][1] * ub[j][1] + u[j][2] * ub[j][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float zbar = zb[j][c] + (ub[j][c] - u[j][c] * uu) * r[j] + 2.f * eb[j] * z[j][c];
      adj.db[j][c] += zbar;
      if (j < N) wb[j][c] += zbar;
      if (j > 0) wb[j - 1][c] -= zbar;
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s = fmaf(G.a[i][k][c], wb[i][c], s);
        adj.a[i][k][c] += wb[i][c] * t[i][k];
      }
      tb[i][k] += s;
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads, kLongOrderMinBlocks<N>)
    unrolled_grad_kernel(SceneDev S, BatchDev B, int K, int R, uint64_t n_local, const PathRec* __restrict__ list,
        const float* __restrict__ dX, const float* __restrict__ dLv, float dl_all, double* gacc,
        float* __restrict__ tape, float* __restrict__ T_out, uint8_t* __restrict__ status_out, bool sm) {
  constexpr unsigned Q = kAllQuads<N>;
  constexpr int M = 2 * N;
  constexpr int HP = M * (M + 1) / 2;
  constexpr int STRIDE = M + HP;  // tape entry: t, H (g is recomputed from t)
  constexpr bool kRegH = N <= kMaxBfgsOrder;
  extern __shared__ __align__(16) float s_dyn[];
  float* s_acc = s_dyn + kUnrolledSmemH<N>;
  const int n_acc = S.n_obj * 9 + 3 * (S.n_tx + S.n_rx);
  const int acc_tx = S.n_obj * 9, acc_rx = acc_tx + 3 * S.n_tx;
  if (sm)
    for (int k = threadIdx.x; k < n_acc; k += blockDim.x) s_acc[k] = 0.f;
  __syncthreads();
  const Tables tb_g{S.rec32, S.tx32, S.rx32, B.alphabet, B.type_pos};
  const uint64_t n_thr = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t me = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  auto tp = [&](int step, int f) -> float& { return tape[((uint64_t)step * STRIDE + f) * n_thr + me]; };
  float hist[kUnrolledMaxRounds];
  int tiles = 0;
  for (uint64_t j0 = (uint64_t)blockIdx.x * blockDim.x; j0 < n_local; j0 += n_thr) {
    const uint64_t j = j0 + threadIdx.x;
    const bool have = j < n_local;
    float gbv[N][9], gtx[3] = {0.f, 0.f, 0.f}, grx[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int k = 0; k < 9; ++k) gbv[i][k] = 0.f;
    int acc_id[N], acc_t = -1, acc_r = -1;
#pragma unroll
    for (int i = 0; i < N; ++i) acc_id[i] = -1;
    if (have) {
      PathDesc d;
      fetch_path_n<N>(B, list, j, d);
      Geo<N> G;
      load_geo<N, Q>(d, tb_g, G);
      uint8_t st = d.flags;
      const int Kp = (st & ST_SKIP) ? 0 : K;  // sequences that are never solved take no steps and add nothing
      // ---- forward: K steps, taped ----
      float t[N][2], g[M], z[N + 1][3], e[N + 1];
      std::conditional_t<kRegH, float[HP], SmemH> H;
      if constexpr (!kRegH) H.p = s_dyn + threadIdx.x;
#pragma unroll
      for (int i = 0; i < N; ++i) t[i][0] = t[i][1] = 0.5f;
#pragma unroll
      for (int r = 0; r < M; ++r)
#pragma unroll
        for (int c = r; c < M; ++c) H[hidx<M>(r, c)] = r == c ? 1.f : 0.f;
      grad_eval<N, Q>(G, t, z, e, g);
      for (int k = 0; k < Kp; ++k) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          tp(k, 2 * i) = t[i][0];
          tp(k, 2 * i + 1) = t[i][1];
        }
#pragma unroll
        for (int q = 0; q < HP; ++q) tp(k, M + q) = H[q];
        float p[M];
#pragma unroll
        for (int r = 0; r < M; ++r) {
          float acc = 0.f;
#pragma unroll
          for (int c = 0; c < M; ++c) acc = fmaf(H[hidx<M>(r, c)], g[c], acc);
          p[r] = -acc;
        }
        float v[N][3], qa[N + 1], qc[N + 1];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int c = 0; c < 3; ++c) v[i][c] = fmaf(G.a[i][1][c], p[2 * i + 1], G.a[i][0][c] * p[2 * i]);
#pragma unroll
        for (int jj = 0; jj <= N; ++jj) {
          float q[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) q[c] = (jj < N ? v[jj][c] : 0.f) - (jj > 0 ? v[jj - 1][c] : 0.f);
          qa[jj] = fmaf(q[2], z[jj][2], fmaf(q[1], z[jj][1], q[0] * z[jj][0]));
          qc[jj] = fmaf(q[2], q[2], fmaf(q[1], q[1], q[0] * q[0]));
        }
        float alpha = fp_forward<N>(e, qa, qc, 1.f, R, hist);
        if (!(alpha > 0.f)) alpha = fp_forward<N>(e, qa, qc, 0.f, R, hist);
        float s[M];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            s[2 * i + c] = __fmul_rn(alpha, p[2 * i + c]);
            t[i][c] = __fadd_rn(t[i][c], s[2 * i + c]);
          }
        float gn[M];
        grad_eval<N, Q>(G, t, z, e, gn);
        float y[M], sy = 0.f, ss = 0.f, yy = 0.f;
#pragma unroll
        for (int r = 0; r < M; ++r) {
          y[r] = gn[r] - g[r];
          sy = fmaf(s[r], y[r], sy);
          ss = fmaf(s[r], s[r], ss);
          yy = fmaf(y[r], y[r], yy);
          g[r] = gn[r];
        }
        if (sy > 0.f && sy * sy > 1e-12f * (ss * yy)) {
          const float rho = __fdividef(1.f, sy);
          float Hy[M], yHy = 0.f;
#pragma unroll
          for (int r = 0; r < M; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < M; ++c) acc = fmaf(H[hidx<M>(r, c)], y[c], acc);
            Hy[r] = acc;
            yHy = fmaf(y[r], acc, yHy);
          }
          const float beta = fmaf(rho * rho, yHy, rho);
#pragma unroll
          for (int r = 0; r < M; ++r)
#pragma unroll
            for (int c = r; c < M; ++c) {
              float h = H[hidx<M>(r, c)];
              h = fmaf(s[r], fmaf(beta, s[c], -rho * Hy[c]), h);
              H[hidx<M>(r, c)] = fmaf(-rho * Hy[r], s[c], h);
            }
        }
      }
      // ---- loss seeds at the final iterate ----
      const float dl = dLv ? dLv[d.g] : dl_all;
      Adj<N> adj;
#pragma unroll
      for (int jj = 0; jj <= N; ++jj)
#pragma unroll
        for (int c = 0; c < 3; ++c) adj.db[jj][c] = 0.f;
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int c = 0; c < 3; ++c) adj.a[i][0][c] = adj.a[i][1][c] = adj.bx[i][c] = 0.f;
      float tb[N][2], gb[M], zb[N + 1][3], eb[N + 1];
      std::conditional_t<kRegH, float[HP], SmemH> Hb;  // the forward's H is no longer needed
      if constexpr (!kRegH) Hb.p = s_dyn + threadIdx.x;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float dx[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) dx[c] = dX ? dX[(d.g * (uint64_t)B.n_max + i) * 3 + c] : 0.f;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          tb[i][k] = G.a[i][k][0] * dx[0] + G.a[i][k][1] * dx[1] + G.a[i][k][2] * dx[2];
#pragma unroll
          for (int c = 0; c < 3; ++c) adj.a[i][k][c] += dx[c] * t[i][k];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) adj.bx[i][c] = dx[c];
      }
#pragma unroll
      for (int jj = 0; jj <= N; ++jj) {
        const float rr = rsqrtf(fmaxf(e[jj], 1e-30f));
#pragma unroll
        for (int c = 0; c < 3; ++c) zb[jj][c] = dl * z[jj][c] * rr;
        eb[jj] = 0.f;
      }
#pragma unroll
      for (int r = 0; r < M; ++r) gb[r] = 0.f;
#pragma unroll
      for (int q = 0; q < HP; ++q) Hb[q] = 0.f;
      // ---- reverse sweep ----
      for (int k = Kp - 1; k >= 0; --k) {
        // recompute step k from its tape entry
        float tk[N][2], gk[M], zk[N + 1][3], ek[N + 1];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          tk[i][0] = tp(k, 2 * i);
          tk[i][1] = tp(k, 2 * i + 1);
        }
        std::conditional_t<kRegH, float[HP], TapeH> Hk;
        if constexpr (kRegH) {
#pragma unroll
          for (int q = 0; q < HP; ++q) Hk[q] = tp(k, M + q);
        } else {
          Hk = TapeH{&tp(k, M), n_thr};
        }
        grad_eval<N, Q>(G, tk, zk, ek, gk);  // the same arithmetic as the forward: the same bits
        float p[M];
#pragma unroll
        for (int r = 0; r < M; ++r) {
          float acc = 0.f;
#pragma unroll
          for (int c = 0; c < M; ++c) acc = fmaf(Hk[hidx<M>(r, c)], gk[c], acc);
          p[r] = -acc;
        }
        float v[N][3], q[N + 1][3], qa[N + 1], qc[N + 1];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int c = 0; c < 3; ++c) v[i][c] = fmaf(G.a[i][1][c], p[2 * i + 1], G.a[i][0][c] * p[2 * i]);
#pragma unroll
        for (int jj = 0; jj <= N; ++jj) {
#pragma unroll
          for (int c = 0; c < 3; ++c) q[jj][c] = (jj < N ? v[jj][c] : 0.f) - (jj > 0 ? v[jj - 1][c] : 0.f);
          qa[jj] = fmaf(q[jj][2], zk[jj][2], fmaf(q[jj][1], zk[jj][1], q[jj][0] * zk[jj][0]));
          qc[jj] = fmaf(q[jj][2], q[jj][2], fmaf(q[jj][1], q[jj][1], q[jj][0] * q[jj][0]));
        }
        float alpha = fp_forward<N>(ek, qa, qc, 1.f, R, hist);
        if (!(alpha > 0.f)) alpha = fp_forward<N>(ek, qa, qc, 0.f, R, hist);
        float s[M], t1[N][2];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            s[2 * i + c] = __fmul_rn(alpha, p[2 * i + c]);
            t1[i][c] = __fadd_rn(tk[i][c], s[2 * i + c]);
          }
        float z1[N + 1][3], e1[N + 1], g1[M];
        grad_eval<N, Q>(G, t1, z1, e1, g1);
        float y[M], sy = 0.f, ss = 0.f, yy = 0.f;
#pragma unroll
        for (int r = 0; r < M; ++r) {
          y[r] = g1[r] - gk[r];
          sy = fmaf(s[r], y[r], sy);
          ss = fmaf(s[r], s[r], ss);
          yy = fmaf(y[r], y[r], yy);
        }
        // Hb turns from the adjoint of H_{k+1} into that of H_k in place: the update's
        // reverse reads the former only before it adds the first term of the latter
        float sb[M], yb[M];
#pragma unroll
        for (int r = 0; r < M; ++r) sb[r] = yb[r] = 0.f;
        if (sy > 0.f && sy * sy > 1e-12f * (ss * yy)) {
          // H' = H + s wv^T + mv s^T (packed r <= c), wv = beta s - rho Hy, mv = -rho Hy
          const float rho = __fdividef(1.f, sy);
          float Hy[M], yHy = 0.f;
#pragma unroll
          for (int r = 0; r < M; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < M; ++c) acc = fmaf(Hk[hidx<M>(r, c)], y[c], acc);
            Hy[r] = acc;
            yHy = fmaf(y[r], acc, yHy);
          }
          const float beta = fmaf(rho * rho, yHy, rho);
          float wvb[M], mvb[M];
#pragma unroll
          for (int r = 0; r < M; ++r) wvb[r] = mvb[r] = 0.f;
#pragma unroll
          for (int r = 0; r < M; ++r)
#pragma unroll
            for (int c = r; c < M; ++c) {
              const float hb = Hb[hidx<M>(r, c)];
              const float wv_c = fmaf(beta, s[c], -rho * Hy[c]);
              const float mv_r = -rho * Hy[r];
              sb[r] += hb * wv_c;
              wvb[c] += hb * s[r];
              mvb[r] += hb * s[c];
              sb[c] += hb * mv_r;
            }
          float betab = 0.f, rhob = 0.f, Hyb[M];
#pragma unroll
          for (int c = 0; c < M; ++c) {
            betab += wvb[c] * s[c];
            sb[c] += wvb[c] * beta;
            rhob -= wvb[c] * Hy[c] + mvb[c] * Hy[c];
            Hyb[c] = -rho * (wvb[c] + mvb[c]);
          }
          rhob += betab * (2.f * rho * yHy + 1.f);
          const float yHyb = betab * rho * rho;
#pragma unroll
          for (int r = 0; r < M; ++r) {
            yb[r] += yHyb * Hy[r];
            Hyb[r] += yHyb * y[r];
          }
#pragma unroll
          for (int r = 0; r < M; ++r)
#pragma unroll
            for (int c = 0; c < M; ++c) {
              Hb[hidx<M>(r, c)] += Hyb[r] * y[c];
              yb[c] += Hyb[r] * Hk[hidx<M>(r, c)];
            }
          const float syb = -rho * rho * rhob;
#pragma unroll
          for (int r = 0; r < M; ++r) {
            sb[r] += syb * y[r];
            yb[r] += syb * s[r];
          }
        }
        // y = g_{k+1} - g_k
        float gbk[M];
#pragma unroll
        for (int r = 0; r < M; ++r) {
          gb[r] += yb[r];
          gbk[r] = -yb[r];
        }
        // (z, e, g) at t_{k+1}
        float tb1[N][2];
#pragma unroll
        for (int i = 0; i < N; ++i) tb1[i][0] = tb1[i][1] = 0.f;
        grad_reverse<N>(G, t1, z1, gb, zb, eb, tb1, adj);
        // t_{k+1} = t_k + alpha p
        float alphab = 0.f, pb[M];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float tot = tb[i][c] + tb1[i][c];
            tb[i][c] = tot;
            sb[2 * i + c] += tot;
          }
#pragma unroll
        for (int r = 0; r < M; ++r) {
          alphab = fmaf(sb[r], p[r], alphab);
          pb[r] = alpha * sb[r];
        }
        // Eq. 6 rounds of the attempt that gave alpha
        float ebk[N + 1], qab[N + 1], qcb[N + 1];
#pragma unroll
        for (int jj = 0; jj <= N; ++jj) ebk[jj] = qab[jj] = qcb[jj] = 0.f;
        fp_reverse<N>(ek, qa, qc, R, hist, alphab, ebk, qab, qcb);
        // qa = q.z, qc = q.q; q_j = v_j - v_{j-1}; v_i = A_i p_i
        float zbk[N + 1][3], vb[N][3];
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int c = 0; c < 3; ++c) vb[i][c] = 0.f;
#pragma unroll
        for (int jj = 0; jj <= N; ++jj)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float qb = qab[jj] * zk[jj][c] + 2.f * qcb[jj] * q[jj][c];
            zbk[jj][c] = qab[jj] * q[jj][c];
            if (jj < N) vb[jj][c] += qb;
            if (jj > 0) vb[jj - 1][c] -= qb;
          }
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int k2 = 0; k2 < 2; ++k2) {
            float sacc = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              sacc = fmaf(G.a[i][k2][c], vb[i][c], sacc);
              adj.a[i][k2][c] += vb[i][c] * p[2 * i + k2];
            }
            pb[2 * i + k2] += sacc;
          }
        // p = -H g
#pragma unroll
        for (int r = 0; r < M; ++r)
#pragma unroll
          for (int c = 0; c < M; ++c) {
            Hb[hidx<M>(r, c)] -= pb[r] * gk[c];
            gbk[c] -= pb[r] * Hk[hidx<M>(r, c)];
          }
        // adjoint state of step k
#pragma unroll
        for (int r = 0; r < M; ++r) gb[r] = gbk[r];
#pragma unroll
        for (int jj = 0; jj <= N; ++jj) {
          eb[jj] = ebk[jj];
#pragma unroll
          for (int c = 0; c < 3; ++c) zb[jj][c] = zbk[jj][c];
        }
      }
      // the start t_0 = 1/2 is a constant: only the geometry of (z_0, e_0, g_0) receives adjoints
      {
        float t0[N][2], z0[N + 1][3], e0[N + 1], g0[M], tdump[N][2];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          t0[i][0] = t0[i][1] = 0.5f;
          tdump[i][0] = tdump[i][1] = 0.f;
        }
        grad_eval<N, Q>(G, t0, z0, e0, g0);
        grad_reverse<N>(G, t0, z0, gb, zb, eb, tdump, adj);
      }
      // per-slot sums: d/db (objects, from Delta b and the points), d/da1, d/da2; TX and RX
      bool finite = !(st & ST_SKIP);
#pragma unroll
      for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          gbv[i][c] = adj.bx[i][c] + adj.db[i][c] - adj.db[i + 1][c];
          gbv[i][3 + c] = adj.a[i][0][c];
          gbv[i][6 + c] = adj.a[i][1][c];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) finite = finite && isfinite(gbv[i][k]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gtx[c] = -adj.db[0][c];
        grx[c] = adj.db[N][c];
        finite = finite && isfinite(gtx[c]) && isfinite(grx[c]);
      }
      if (finite) {
#pragma unroll
        for (int i = 0; i < N; ++i) acc_id[i] = d.ids[i];
        acc_t = d.tx;
        acc_r = d.rx;
      } else if (!(st & ST_SKIP)) {
        st |= ST_NONFINITE;
      }
      if (T_out) {
        float2* To = reinterpret_cast<float2*>(T_out) + d.g * (uint64_t)B.n_max;
#pragma unroll
        for (int i = 0; i < N; ++i) To[i] = make_float2(t[i][0], t[i][1]);
      }
      if (status_out) status_out[d.g] = st;
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
      warp_accumulate<9>(s_acc, acc_id[i] >= 0 ? 9 * acc_id[i] : -1, gbv[i], sm, gacc, 9 * acc_id[i]);
    warp_accumulate<3>(s_acc, acc_t >= 0 ? acc_tx + 3 * acc_t : -1, gtx, sm, gacc, acc_tx + 3 * acc_t);
    warp_accumulate<3>(s_acc, acc_r >= 0 ? acc_rx + 3 * acc_r : -1, grx, sm, gacc, acc_rx + 3 * acc_r);
    if (sm && ++tiles >= 64) {
      tiles = 0;
      __syncthreads();
      for (int k = threadIdx.x; k < n_acc; k += blockDim.x) {
        const float x = s_acc[k];
        if (x != 0.f) {
          atomicAdd(gacc + k, (double)x);
          s_acc[k] = 0.f;
        }
      }
      __syncthreads();
    }
  }
  if (sm) {
    __syncthreads();
    for (int k = threadIdx.x; k < n_acc; k += blockDim.x) {
      const float x = s_acc[k];
      if (x != 0.f) atomicAdd(gacc + k, (double)x);
    }
  }
}

// The launcher of one order as an explicitly instantiable unit (orders 6-10 in k_high.cu).
template <int N>
struct UnrolledOrder {
  static cudaError_t launch(const SceneDev& S, const BatchDev& B, int steps, int rounds, uint64_t n_local,
                            const PathRec* list, const float* dX, const float* dL, float dl_all, double* gacc,
                            float* tape, size_t tape_floats, float* T_out, uint8_t* status, cudaStream_t stream,
                            int n_sm);
};

template <int N>
cudaError_t UnrolledOrder<N>::launch(const SceneDev& S, const BatchDev& B, int steps, int rounds, uint64_t n_local,
                                     const PathRec* list, const float* dX, const float* dL, float dl_all,
                                     double* gacc, float* tape, size_t tape_floats, float* T_out, uint8_t* status,
                                     cudaStream_t stream, int n_sm) {
  constexpr int M = 2 * N;
  constexpr int STRIDE = M + M * (M + 1) / 2;
  size_t smem = (size_t)(9 * S.n_obj + 3 * (S.n_tx + S.n_rx)) * sizeof(float);
  const bool sm = smem <= 64 * 1024;  // else the sums go straight to the FP64 accumulators
  if (!sm) smem = 0;
  smem += (size_t)kUnrolledSmemH<N> * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(unrolled_grad_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, unrolled_grad_kernel<N>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint64_t want = (n_local + kThreads - 1) / kThreads;
  uint64_t grid = want < (uint64_t)n_sm * per_sm ? want : (uint64_t)n_sm * per_sm;
  // the tape bounds the number of resident paths
  const uint64_t per_thread = (uint64_t)steps * STRIDE;
  const uint64_t max_threads = per_thread ? tape_floats / per_thread : grid * kThreads;
  if (grid * kThreads > max_threads) grid = max_threads / kThreads;
  if (grid == 0) return n_local ? cudaErrorMemoryAllocation : cudaSuccess;
  unrolled_grad_kernel<N><<<(unsigned)grid, kThreads, smem, stream>>>(S, B, steps, rounds, n_local, list, dX, dL,
                                                                       dl_all, gacc, tape, T_out, status, sm);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fpt
