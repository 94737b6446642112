// bfgs.cuh -- FP32 BFGS + fixed-point line search, one thread per path.
//
// Sec. III-C: BFGS on the inverse Hessian of L(T; A, B) (Eq. 5) with the step
// size along p = -H g given by rounds of the fixed point of Eq. 6 instead of
// an inexact line search.  The iterate t, the gradient and the packed
// inverse-Hessian estimate (M(M+1)/2 floats) stay in registers; the scene's
// FP32 object records are staged in shared memory.  A warp leaves its BFGS
// loop when every lane has met its stop rule.
//
// Interaction-type patterns.  In the unified parameterisation (Sec. III-B)
// every object has two parameters; an edge carries a zero second basis
// vector.  That parameter then has a zero gradient in every iteration, so
// with H_0 = I its step is zero, its row and column of H stay those of the
// identity, and it never changes the other entries: the quantities it
// touches are exact zeros in FP32 too.  The kernels are therefore templated
// on the pattern Q of a sequence (bit i set: slot i is a planar reflector
// with two parameters; clear: an edge with one) and leave the edge's dead
// parameter out of g, p, s, y and H.  The remaining arithmetic is the
// unified kernel's, term for term and in the same order, so the iterates are
// the same; Q = all ones over all sequences of an order is the unified
// kernel itself, kept for solves with the specialisation off and as the
// reference the pattern kernels are tested against.
//
// Readings of points the paper leaves open: H_0 = I; every step starts the
// fixed point at alpha = 1 and, if that yields alpha <= 0, restarts it at
// alpha = 0 (one round from 0 is a majorise-minimise step, positive along a
// descent direction); the update is skipped unless s^T y > 1e-6 |s| |y|
// (tested as (s^T y)^2 > 1e-12 |s|^2 |y|^2 with s^T y > 0).
#pragma once

#include <type_traits>
#include <utility>

#include "fpt_kernels.h"

namespace fpt {

// Unknowns of a pattern: slot i has dim(i) parameters starting at off(i).
// Where the unified kernel forms fmaf(a2, t2, a1 * t1) with a2 = 0, the
// pattern kernel forms the rounded product a1 * t1 with __fmul_rn.  That and
// the other products that feed an addition (u_j, the step s) use the _rn
// intrinsics, which the compiler never fuses, so every instantiation rounds
// the same way whatever its code layout.
template <int N, unsigned Q>
struct Pat {
  static constexpr __host__ __device__ bool quad(int i) { return ((Q >> i) & 1u) != 0u; }
  static constexpr __host__ __device__ int dim(int i) { return quad(i) ? 2 : 1; }
  static constexpr __host__ __device__ int off(int i) {
    return N <= kMaxBfgsOrder ? i + (i > 0 && quad(0)) + (i > 1 && quad(1)) + (i > 2 && quad(2)) +
                                    (i > 3 && quad(3)) + (i > 4 && quad(4))
                              : 2 * i;  // above the pattern orders only the unified kernel (Q all ones)
  }
  static constexpr int M = off(N);
  static constexpr int HP = M * (M + 1) / 2;
};

template <int N>
constexpr unsigned kAllQuads = (1u << N) - 1u;

template <int N>
struct Geo {
  float db[N + 1][3];  // Delta b_j: b of the segment's end minus b of its start
  float a[N][2][3];    // basis vectors of each object (a[i][1] unused for edge slots)
};

// Packed upper-triangular index of a symmetric M x M matrix.
template <int M>
__host__ __device__ constexpr int hidx(int r, int c) {
  return r <= c ? r * M - r * (r - 1) / 2 + (c - r) : c * M - c * (c - 1) / 2 + (r - c);
}

// Lookup tables of a launch, in shared memory where they fit.
struct Tables {
  const float* rec;         // FP32 object records [n_obj][kRec32]
  const float* tx;          // endpoints [n][kEnd32]
  const float* rx;
  const int32_t* alphabet;  // [n_alpha] (nullptr for explicit batches)
  const int32_t* type_pos;  // [n_alpha] (exhaustive batches)
};

// Exhaustive batch, sequences of order N and pattern Q only: local index j
// over n_pairs * prod_i |alphabet part of slot i| paths.  The alphabet's
// reflectors and edges are listed (ascending positions) in type_pos.  The
// decoded sequence and its global index g are those of the full enumeration.
// One order of a batch holds at most 2^32 paths (checked by the host), so the
// local index arithmetic is 32-bit.
template <int N, unsigned Q>
__device__ __forceinline__ void decode_exhaustive_pattern(const BatchDev& B, const Tables& tb, uint64_t j,
                                                          PathDesc& d) {
  const uint32_t nq = (uint32_t)B.n_alpha_quad, ne = (uint32_t)(B.n_alpha - B.n_alpha_quad);
  const uint32_t cnt = B.fd_pat.d;
  const uint32_t j32 = (uint32_t)j;
  const uint32_t pair = fdiv(j32, B.fd_pat);
  uint32_t r = j32 - pair * cnt;
  d.n = N;
  d.tx = (int)fdiv(pair, B.fd_rx);
  d.rx = (int)(pair - (uint32_t)d.tx * (uint32_t)B.n_rx);
  int pos[N];
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    const uint32_t base = Pat<N, Q>::quad(i) ? nq : ne;
    const uint32_t q = fdiv(r, Pat<N, Q>::quad(i) ? B.fd_quad : B.fd_edge);
    pos[i] = tb.type_pos[(Pat<N, Q>::quad(i) ? 0u : nq) + (r - q * base)];
    r = q;
  }
  uint64_t rg = 0;
  d.flags = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    rg = rg * (uint64_t)B.n_alpha + (uint64_t)pos[i];
    const int o = tb.alphabet[pos[i]];
    d.ids[i] = o;
    if (i > 0 && d.ids[i - 1] == o) d.flags |= ST_REPEAT;
  }
  d.g = (uint64_t)pair * B.per_pair + B.offset[N] + rg;
}

// Where a kernel's paths come from; each source is its own instantiation so
// that a kernel carries only the decoding it needs.
enum BfgsSource {
  SRC_ORDER = 0,    // exhaustive batch: every sequence of order N, decoded from the local index
  SRC_PATTERN = 1,  // exhaustive batch: the sequences of pattern Q only
  SRC_LIST = 2,     // seeded / explicit batch: a bucket of decoded path records
};

template <int N, unsigned Q, int kSrc>
__device__ __forceinline__ void fetch_path_q(const BatchDev& B, const Tables& tb, const PathRec* list, uint64_t j,
                                             PathDesc& d) {
  if constexpr (kSrc == SRC_LIST) {
    load_rec(list, j, d);
    if constexpr (N > kMaxBfgsOrder) decode_global<N>(B, d.g, d);  // longer records keep g, not the ids
  } else if constexpr (kSrc == SRC_PATTERN) {
    decode_exhaustive_pattern<N, Q>(B, tb, j, d);
  } else {
    decode_exhaustive_order<N>(B, N, j, d);
  }
}

template <int N, unsigned Q>
__device__ __forceinline__ void load_geo(const PathDesc& d, const Tables& tb, Geo<N>& G) {
  float bh[N + 2][3], bl[N + 2][3];
  const float* tx = tb.tx + kEnd32 * d.tx;
  const float* rx = tb.rx + kEnd32 * d.rx;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bh[0][c] = tx[c];
    bl[0][c] = tx[3 + c];
    bh[N + 1][c] = rx[c];
    bl[N + 1][c] = rx[3 + c];
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float* r = tb.rec + kRec32 * d.ids[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      bh[i + 1][c] = r[c];
      bl[i + 1][c] = r[3 + c];
      G.a[i][0][c] = r[6 + c];
      G.a[i][1][c] = Pat<N, Q>::quad(i) ? r[9 + c] : 0.f;
    }
  }
#pragma unroll
  for (int j = 0; j <= N; ++j)
#pragma unroll
    for (int c = 0; c < 3; ++c) G.db[j][c] = (bh[j + 1][c] - bh[j][c]) + (bl[j + 1][c] - bl[j][c]);
}

// z_j = x_{j+1} - x_j for j = 0..N, e_j = |z_j|^2, and g = grad_T L (Eq. 5):
// g_i = A_i^T (u_i - u_{i+1}) with u_j = z_j / |z_j|.
template <int N, unsigned Q>
__device__ __forceinline__ void grad_eval(const Geo<N>& G, const float (&t)[N][2], float (&z)[N + 1][3],
                                          float (&e)[N + 1], float (&g)[Pat<N, Q>::M], float (&rz)[N + 1]) {
  using P = Pat<N, Q>;
  float w[N][3];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      w[i][c] = P::quad(i) ? fmaf(G.a[i][1][c], t[i][1], G.a[i][0][c] * t[i][0]) : __fmul_rn(G.a[i][0][c], t[i][0]);
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
    rz[j] = r;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[j][c] = __fmul_rn(z[j][c], r);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float d0 = u[i][0] - u[i + 1][0], d1 = u[i][1] - u[i + 1][1], d2 = u[i][2] - u[i + 1][2];
    g[P::off(i)] = fmaf(G.a[i][0][2], d2, fmaf(G.a[i][0][1], d1, G.a[i][0][0] * d0));
    if (P::quad(i)) g[P::off(i) + 1] = fmaf(G.a[i][1][2], d2, fmaf(G.a[i][1][1], d1, G.a[i][1][0] * d0));
  }
}

template <int N, unsigned Q>
__device__ __forceinline__ void grad_eval(const Geo<N>& G, const float (&t)[N][2], float (&z)[N + 1][3],
                                          float (&e)[N + 1], float (&g)[Pat<N, Q>::M]) {
  float rz[N + 1];
  grad_eval<N, Q>(G, t, z, e, g, rz);
}

// Eq. 6: alpha <- -sum_j (q_j.z_j)/|z_j + alpha q_j| / sum_j (q_j.q_j)/|z_j + alpha q_j|,
// with |z_j + alpha q_j|^2 = e_j + alpha (2 qa_j + alpha qc_j).  Steps are capped at
// kAlphaMax times the quasi-Newton step, which keeps many rounds at a vanishing
// direction (a converged path run for a fixed step count) finite.
constexpr float kAlphaMax = 1e3f;
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
    alpha = den > 1e-30f ? fminf(-__fdividef(num, den), kAlphaMax) : 0.f;
  }
  return alpha;
}

// The inverse-Hessian estimate of a path of order above kMaxBfgsOrder: 2n(2n+1)/2
// floats (210 at n = 10) do not fit a thread's registers next to its iterate,
// so entry k of thread x lives at s_H[k * kThreads + x] (consecutive threads,
// consecutive banks).
struct SmemH {
  float* p;
  __device__ __forceinline__ float& operator[](int k) const { return p[k * kThreads]; }
};

// Per-path solver state, in registers (H in shared memory above kMaxBfgsOrder).
template <int N, unsigned Q>
struct PathState {
  static constexpr int M = Pat<N, Q>::M;
  static constexpr int HP = Pat<N, Q>::HP;
  Geo<N> G;
  // the packed inverse-Hessian estimate: registers up to the BFGS register orders, a column of
  // shared memory (one float per thread and entry) for the longer sequences
  std::conditional_t<(N <= kMaxBfgsOrder), float[HP], SmemH> H;
  float t[N][2], g[M], z[N + 1][3], e[N + 1];
  float rz[N + 1];  // 1 / |z_j| at t, as the gradient evaluated it (the next step's alpha = 0 round reuses it)
  uint64_t gidx;
  int it;
  uint8_t st;
  bool conv;
};

// Decode a path, load its geometry, start at the object centroids (t = 1/2)
// or at the given start, with H = I, and evaluate the first gradient.
// Returns false for paths that are never solved (repeats, invalid input).
template <int N, unsigned Q, int kSrc>
__device__ __forceinline__ bool path_start(PathState<N, Q>& P, const BatchDev& B, const Tables& tb,
                                           const PathRec* list, uint64_t j, int max_iters, const float* T_start) {
  constexpr int M = PathState<N, Q>::M;
  PathDesc d;
  fetch_path_q<N, Q, kSrc>(B, tb, list, j, d);
  P.gidx = d.g;
  P.st = d.flags;
  P.it = 0;
  P.conv = false;
  load_geo<N, Q>(d, tb, P.G);
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
  grad_eval<N, Q>(P.G, P.t, P.z, P.e, P.g, P.rz);
  return max_iters > 0;
}

// One BFGS step (Sec. III-C) with the Eq. 6 step size.  Returns true when the
// path is done (tolerance met, cap reached, kink ahead or non-finite).
template <int N, unsigned Q>
__device__ __forceinline__ bool bfgs_step(PathState<N, Q>& P, const SolveCfg& cfg) {
  using Pt = Pat<N, Q>;
  constexpr int M = Pt::M;
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
    for (int c = 0; c < 3; ++c)
      v[i][c] = Pt::quad(i) ? fmaf(P.G.a[i][1][c], p[Pt::off(i) + 1], P.G.a[i][0][c] * p[Pt::off(i)])
                            : __fmul_rn(P.G.a[i][0][c], p[Pt::off(i)]);
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
  float alpha;
  if (cfg.fp_iters == 1) {
    // one round: the rounds from alpha = 1 and from alpha = 0 side by side, so that the lanes that need
    // the second (about a third of the steps) do not run it alone; the same values as fixed_point()
    float n1 = 0.f, d1 = 0.f, n0 = 0.f, d0 = 0.f;
#pragma unroll
    for (int jj = 0; jj <= N; ++jj) {
      const float r1 = rsqrtf(fmaxf(fmaf(1.f, fmaf(1.f, qc[jj], 2.f * qa[jj]), P.e[jj]), 1e-30f));
      // 1 / |z_j| at t: kept from the gradient evaluation up to order 4 (the same value), evaluated again
      // for the longer sequences, where four or more reflectors would spill the extra registers
      float r0;
      if constexpr (N <= 4)
        r0 = P.rz[jj];
      else
        r0 = rsqrtf(fmaxf(P.e[jj], 1e-30f));
      n1 = fmaf(qa[jj], r1, n1);
      d1 = fmaf(qc[jj], r1, d1);
      n0 = fmaf(qa[jj], r0, n0);
      d0 = fmaf(qc[jj], r0, d0);
    }
    const float a1 = d1 > 1e-30f ? fminf(-__fdividef(n1, d1), kAlphaMax) : 0.f;
    const float a0 = d0 > 1e-30f ? fminf(-__fdividef(n0, d0), kAlphaMax) : 0.f;
    alpha = a1 > 0.f ? a1 : a0;
  } else {
    alpha = fixed_point<N>(P.e, qa, qc, 1.f, cfg.fp_iters);
    if (!(alpha > 0.f)) alpha = fixed_point<N>(P.e, qa, qc, 0.f, cfg.fp_iters);
  }
  // step and new gradient
  float s[M];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (c < Pt::dim(i)) {
        const int r = Pt::off(i) + c;
        s[r] = __fmul_rn(alpha, p[r]);
        P.t[i][c] = __fadd_rn(P.t[i][c], s[r]);
      }
  float gn[M];
  grad_eval<N, Q>(P.G, P.t, P.z, P.e, gn, P.rz);
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
  // a segment collapsing before convergence, past the first steps (a start may put two points close
  // together): the path runs into a kink of L, not a smooth minimiser
  const bool kink = emin < cfg.stop2 && !P.conv && P.it >= kKinkMinIters;
  if (kink) P.st |= ST_DEGENERATE;
  return P.it >= cfg.max_iters || bad || kink || (P.conv && !cfg.fixed_iters);
}

template <int N, unsigned Q>
__device__ __forceinline__ void path_finish(const PathState<N, Q>& P, int n_max, float* __restrict__ T_out,
                                            uint8_t* __restrict__ status_out, uint8_t* __restrict__ iters_out) {
  float2* To = reinterpret_cast<float2*>(T_out) + P.gidx * (uint64_t)n_max;
  // slots from N to n_max - 1 are zero; those past kMaxBfgsOrder were cleared before the solve
  constexpr int kSlots = N > kMaxBfgsOrder ? N : kMaxBfgsOrder;
#pragma unroll
  for (int i = 0; i < kSlots; ++i)
    if (i < n_max) To[i] = i < N ? make_float2(P.t[i][0], P.t[i][1]) : make_float2(0.f, 0.f);
  status_out[P.gidx] = P.st | (P.conv ? ST_CONVERGED : 0);
  if (iters_out) iters_out[P.gidx] = (uint8_t)(P.it > 255 ? 255 : P.it);
}

// Shared-memory staging of a launch's tables: bit 0 of `use_smem` stages the
// object records, bit 1 also the endpoints and the alphabet tables (the host
// sizes the dynamic shared memory to match, smem_tables_bytes).
__device__ __forceinline__ Tables stage_tables(const SceneDev& S, const BatchDev& B, int use_smem, float* smem) {
  Tables tb{S.rec32, S.tx32, S.rx32, B.alphabet, B.type_pos};
  if (use_smem & 1) {
    stage(smem, S.rec32, S.n_obj * kRec32);
    tb.rec = smem;
    smem += S.n_obj * kRec32;
  }
  if (use_smem & 2) {
    stage(smem, S.tx32, S.n_tx * kEnd32);
    tb.tx = smem;
    smem += S.n_tx * kEnd32;
    stage(smem, S.rx32, S.n_rx * kEnd32);
    tb.rx = smem;
    smem += S.n_rx * kEnd32;
    int32_t* si = reinterpret_cast<int32_t*>(smem);
    if (B.alphabet) {
      stage(si, B.alphabet, B.n_alpha);
      tb.alphabet = si;
      si += B.n_alpha;
    }
    if (B.type_pos) {
      stage(si, B.type_pos, B.n_alpha);
      tb.type_pos = si;
    }
  }
  __syncthreads();
  return tb;
}

// Bytes of shared memory for stage_tables and the matching use_smem flags
// (records up to 96 KB; endpoints and alphabet tables too if the total stays
// within 64 KB, so that several CTAs still fit on an SM).
inline size_t smem_tables_bytes(const SceneDev& S, const BatchDev& B, int* use_smem) {
  const size_t rec = (size_t)S.n_obj * kRec32 * sizeof(float);
  const size_t ends = (size_t)(S.n_tx + S.n_rx) * kEnd32 * sizeof(float) +
                      (size_t)((B.alphabet ? 1 : 0) + (B.type_pos ? 1 : 0)) * B.n_alpha * sizeof(int32_t);
  *use_smem = 0;
  if (rec > 96 * 1024) return 0;
  *use_smem = 1;
  if (rec + ends > 64 * 1024) return rec;
  *use_smem = 3;
  return rec + ends;
}

// Floats of dynamic shared memory that hold the CTA's inverse-Hessian columns
// (sequences above kMaxBfgsOrder; they precede the staged tables).
template <int N, unsigned Q>
constexpr int kSmemHFloats = N > kMaxBfgsOrder ? Pat<N, Q>::HP * kThreads : 0;

// One path per thread per tile; a warp leaves its BFGS loop when all 32 lanes are done.
template <int N>
__global__ void __launch_bounds__(kThreads) bfgs_kernel(SceneDev S, BatchDev B, SolveCfg cfg, uint64_t n_local,
                                                        const PathRec* __restrict__ list, float* __restrict__ T_out,
                                                        uint8_t* __restrict__ status_out,
                                                        uint8_t* __restrict__ iters_out, int use_smem) {
  constexpr unsigned Q = kAllQuads<N>;
  extern __shared__ __align__(16) float s_tab[];
  const Tables tb = stage_tables(S, B, use_smem, s_tab + kSmemHFloats<N, Q>);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j0 = (uint64_t)blockIdx.x * blockDim.x; j0 < n_local; j0 += stride) {
    const uint64_t j = j0 + threadIdx.x;
    const bool have = j < n_local;
    PathState<N, Q> P;
    if constexpr (kSmemHFloats<N, Q> > 0) P.H.p = s_tab + threadIdx.x;
    bool active = false;
    if (have)
      active = list ? path_start<N, Q, SRC_LIST>(P, B, tb, list, j, cfg.max_iters, cfg.init_from_T ? T_out : nullptr)
                    : path_start<N, Q, SRC_ORDER>(P, B, tb, list, j, cfg.max_iters, cfg.init_from_T ? T_out : nullptr);
    while (__any_sync(0xffffffffu, active))
      if (active && bfgs_step<N, Q>(P, cfg)) active = false;
    if (have) path_finish<N, Q>(P, B.n_max, T_out, status_out, iters_out);
  }
}

// Lane refill: a lane whose path is done writes it out and takes the next path
// of its warp's chunk (chunks of cfg.chunk paths are claimed from a global
// counter), so lanes do not idle behind the warp's slowest path.  To amortise
// the divergent start-up code, lanes refill only when at least cfg.refill of
// them are free, or when none is busy; a finished path stays in its lane's
// registers until then, so that writing it out shares that divergent pass.  The chunk is sized per launch so that
// every warp claims several chunks (a short tail) but few atomics are needed.

// CTAs per SM that the register allocation of the refill kernels targets: four up to
// order 3, whose kernels all fit 128 registers without spilling (left to itself, ptxas
// gives some order-3 pattern kernels 137 and so only three CTAs per SM); three for the
// order-5 patterns with three or four reflectors (185-206 registers left alone, 165-168
// and at most 8 bytes of spills bounded; the other order-5 patterns fit three CTAs or,
// with five reflectors at 231 registers, would spill far more); no other constraint.
template <int N, unsigned Q>
constexpr int kBfgsMinCtas = N <= 3 ? 4 : (N == 5 && __builtin_popcount(Q) >= 3 && __builtin_popcount(Q) <= 4 ? 3 : 1);

template <int N, unsigned Q, int kSrc>
__global__ void __launch_bounds__(kThreads, kBfgsMinCtas<N, Q>) bfgs_refill_kernel(SceneDev S, BatchDev B, SolveCfg cfg, uint64_t n_local,
                                                               const PathRec* __restrict__ list,
                                                               float* __restrict__ T_out,
                                                               uint8_t* __restrict__ status_out,
                                                               uint8_t* __restrict__ iters_out, int use_smem,
                                                               unsigned long long* __restrict__ work) {
  extern __shared__ __align__(16) float s_tab[];
  const Tables tb = stage_tables(S, B, use_smem, s_tab + kSmemHFloats<N, Q>);
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  uint64_t next = 0, end = 0;  // warp-uniform: unclaimed part of the warp's chunk
  bool more = true;            // warp-uniform: the global counter may still have work
  PathState<N, Q> P;
  if constexpr (kSmemHFloats<N, Q> > 0) P.H.p = s_tab + threadIdx.x;
  bool active = false;
  bool owed = false;  // the lane's finished path is written out at the next refill (one divergent pass for both)
  for (;;) {
    unsigned free_mask = __ballot_sync(full, !active);
    const int n_free = __popc(free_mask);
    if (more && (n_free >= cfg.refill || n_free == 32)) {
      if (owed) {
        path_finish<N, Q>(P, B.n_max, T_out, status_out, iters_out);
        owed = false;
      }
      // hand out paths to the free lanes in one pass: the rest of the warp's chunk, then (claimed first)
      // the next chunk.  A lane whose new path needs no solving (a repeat) writes it out and stays free
      // until the next refill rather than costing the warp another pass.
      const uint64_t want = (uint64_t)n_free;
      const uint64_t avail = end - next;
      uint64_t nb = 0, ne = 0;  // the newly claimed chunk, if any
      if (avail < want) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(work, (unsigned long long)cfg.chunk);
        base = __shfl_sync(full, base, 0);
        if (base >= n_local) {
          more = false;
        } else {
          nb = base;
          ne = base + cfg.chunk < n_local ? base + cfg.chunk : n_local;
        }
      }
      const uint64_t have = avail + (ne - nb);
      const uint64_t take = have < want ? have : want;
      const bool mine = (free_mask >> lane) & 1u;
      const uint64_t rank = (uint64_t)__popc(free_mask & lt_mask);
      if (mine && rank < take) {
        const uint64_t j = rank < avail ? next + rank : nb + (rank - avail);
        if (path_start<N, Q, kSrc>(P, B, tb, list, j, cfg.max_iters, cfg.init_from_T ? T_out : nullptr)) {
          active = true;
        } else {
          path_finish<N, Q>(P, B.n_max, T_out, status_out, iters_out);
        }
      }
      if (take <= avail) {
        next += take;
      } else {
        next = nb + (take - avail);
        end = ne;
      }
    }
    if (!__any_sync(full, active)) {
      if (!more) break;
      continue;
    }
    if (active && bfgs_step<N, Q>(P, cfg)) {
      active = false;
      owed = true;
    }
  }
  if (owed) path_finish<N, Q>(P, B.n_max, T_out, status_out, iters_out);
}

// Arguments of one BFGS launch over a slice of paths.
struct BfgsLaunch {
  SceneDev S;
  BatchDev B;
  SolveCfg cfg;
  uint64_t n_local;
  const PathRec* list;  // nullptr: exhaustive batch, decoded from the local index
  float* T;
  uint8_t* status;
  uint8_t* iters;
  cudaStream_t stream;
  int n_sm;
  unsigned long long* work;  // chunk counter of the refill kernel
};

template <int N, unsigned Q, int kSrc>
cudaError_t launch_bfgs_nq(const BfgsLaunch& a) {
  int use_smem = 0;
  size_t smem = smem_tables_bytes(a.S, a.B, &use_smem);
  if constexpr (kSmemHFloats<N, Q> > 0) {
    // the inverse-Hessian columns first; the tables stay in global memory when both do not fit
    const size_t hb = (size_t)kSmemHFloats<N, Q> * sizeof(float);
    if (hb + smem > kMaxSmemBytes) {
      use_smem = 0;
      smem = 0;
    }
    smem += hb;
  }
  constexpr bool kPat = kSrc == SRC_PATTERN || Q != kAllQuads<N>;
  const bool refill = kPat || (a.cfg.refill > 0 && a.work != nullptr);
  const void* fn;
  if constexpr (kPat)
    fn = (const void*)bfgs_refill_kernel<N, Q, kSrc>;
  else
    fn = refill ? (const void*)bfgs_refill_kernel<N, Q, kSrc> : (const void*)bfgs_kernel<N>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint64_t want = (a.n_local + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)a.n_sm * (uint64_t)per_sm;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  if (grid == 0) return cudaSuccess;
  if (refill) {
    if (a.work == nullptr) return cudaErrorInvalidValue;
    e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), a.stream);
    if (e != cudaSuccess) return e;
    // at least ~8 chunks per warp, in whole warps of paths
    SolveCfg cfg = a.cfg;
    BatchDev B = a.B;
    if constexpr (kSrc == SRC_PATTERN) {
      uint64_t cnt = 1;
      for (int i = 0; i < N; ++i)
        cnt *= Pat<N, Q>::quad(i) ? (uint64_t)a.B.n_alpha_quad : (uint64_t)(a.B.n_alpha - a.B.n_alpha_quad);
      B.fd_pat = make_fastdiv(cnt);
    }
    const uint64_t per = a.n_local / ((uint64_t)grid * (kThreads / 32) * 8);
    cfg.chunk = (int)(per >= (uint64_t)kMaxChunk ? kMaxChunk : (per < 32 ? 32 : per / 32 * 32));
    bfgs_refill_kernel<N, Q, kSrc><<<grid, kThreads, smem, a.stream>>>(a.S, B, cfg, a.n_local, a.list, a.T,
                                                                       a.status, a.iters, use_smem, a.work);
    count_launch();
  } else {
    if constexpr (!kPat) {
      bfgs_kernel<N><<<grid, kThreads, smem, a.stream>>>(a.S, a.B, a.cfg, a.n_local, a.list, a.T, a.status, a.iters,
                                                          use_smem);
      count_launch();
    }
  }
  return cudaGetLastError();
}

// The unified kernel of order N (every slot with two parameters) as an
// explicitly instantiable unit: the BFGS register orders are instantiated with
// the dispatcher (k_bfgs.cu), the longer sequences each in their own object
// (k_high.cu).
template <int N>
struct BfgsOrder {
  static cudaError_t launch(const BfgsLaunch& a);
};

template <int N>
cudaError_t BfgsOrder<N>::launch(const BfgsLaunch& a) {
  if (a.list != nullptr) return launch_bfgs_nq<N, kAllQuads<N>, SRC_LIST>(a);
  return launch_bfgs_nq<N, kAllQuads<N>, SRC_ORDER>(a);
}

// Pattern kernels Q0 .. Q0 + sizeof...(I) - 1 of order N and one path source behind one switch.
template <int N, unsigned Q0, int kSrc, unsigned... I>
cudaError_t dispatch_patterns(unsigned q, const BfgsLaunch& a, std::integer_sequence<unsigned, I...>) {
  using Fn = cudaError_t (*)(const BfgsLaunch&);
  static constexpr Fn tab[] = {&launch_bfgs_nq<N, Q0 + I, kSrc>...};
  if (q < Q0 || q >= Q0 + sizeof...(I)) return cudaErrorInvalidValue;
  return tab[q - Q0](a);
}

// Pattern kernels Q0 .. Q0 + QN - 1 of order N for both path sources.  Each
// range is instantiated in its own object (k_bfgs_pat.cu compiled once per
// entry of FPT_BFGS_RANGES) so that the ~120 kernels compile in parallel.
template <int N, unsigned Q0, unsigned QN>
cudaError_t launch_bfgs_range(unsigned q, const BfgsLaunch& a) {
  if (a.list != nullptr) return dispatch_patterns<N, Q0, SRC_LIST>(q, a, std::make_integer_sequence<unsigned, QN>{});
  return dispatch_patterns<N, Q0, SRC_PATTERN>(q, a, std::make_integer_sequence<unsigned, QN>{});
}

// (order, first pattern, pattern count) of every pattern object.
#define FPT_BFGS_RANGES(X)                                                                                        \
  X(1, 0, 2) X(2, 0, 4) X(3, 0, 8) X(4, 0, 8) X(4, 8, 8) X(5, 0, 4) X(5, 4, 4) X(5, 8, 4) X(5, 12, 4) X(5, 16, 4) \
  X(5, 20, 4) X(5, 24, 4) X(5, 28, 4)

}  // namespace fpt
