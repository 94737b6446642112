/*
 * Fermat path oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU reference for the batched Fermat
 * path solve of "Fast, Differentiable, GPU-Accelerated Ray Tracing for
 * Multiple Diffraction and Reflection Paths" (arXiv 2510.16172).  Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg load this
 * library.  It shares no code, header or constant table with the CUDA path.
 *
 * What it computes (each function cites its passage):
 *   - object records x = A t + b                      (Sec. III-B, Eq. 3)
 *   - candidate-sequence enumeration                   (Sec. III, first paragraph)
 *   - total length, gradient and Hessian of Eq. 5      (Sec. III-B, Eq. 4-5)
 *   - ground truth X* = argmin of Eq. 1-2 over the affine hulls of the
 *     objects: damped Newton on the reduced parameterisation (d = 1 for
 *     edges, d = 2 for planes) -- the "high-precision solver on a CPU" of
 *     Sec. IV-A.  Textbook Newton with backtracking, not the Carluccio-Albani
 *     variant.
 *   - the paper's own solver in FP64: BFGS on the inverse Hessian (Sec. III-C)
 *     with the fixed-point step-size update of Eq. 6, on the unified d = 2
 *     parameterisation (edges carry a zero second basis vector, Sec. III-B).
 *   - the validity test: every point inside its object (Sec. I, Sec. III)
 *   - the stationarity residual: world-space length of the Newton step
 *   - the implicit-differentiation VJP of Sec. III-D, Eq. 8-13, with the
 *     Jacobian of the optimality condition formed densely.
 *
 * Precision: FP64 throughout.  Parallelism: independent paths split across
 * POSIX threads; nothing inside a path is reordered.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NMAX 10 /* longest sequence handled (Fig. 3 goes to n = 10) */
#define ORC_MMAX (2 * ORC_NMAX)

enum { ORC_QUAD = 0, ORC_EDGE = 1 };

/* per-path status bits (same meaning as the library's, defined independently) */
enum {
  ORC_VALID = 1,
  ORC_CONVERGED = 2,
  ORC_SOLVED = 4,
  ORC_DEGENERATE = 16,
  ORC_REPEAT = 32,
  ORC_NONFINITE = 64,
  ORC_INVALID_INPUT = 128
};

/* ------------------------------------------------------------------------ */
/* Objects (Sec. III-B, Eq. 3): x = A t + b.                                  */
/* A plane is given by corners v0, v1, v3 of a parallelogram: b = v0,         */
/* A = [v1 - v0, v3 - v0], inside <=> t in [0,1]^2.  An edge e0 -> e1:        */
/* b = e0, A = [e1 - e0, 0] (zero second basis vector), inside <=> t1 in [0,1] */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n;                    /* number of interactions */
  double x0[3], xe[3];      /* start (TX) and end (RX) points */
  int type[ORC_NMAX];
  double b[ORC_NMAX][3];
  double col[ORC_NMAX][2][3]; /* columns of A_i; col[i][1] = 0 for edges */
} orc_path;

static void vsub(const double* a, const double* b, double* r) {
  r[0] = a[0] - b[0];
  r[1] = a[1] - b[1];
  r[2] = a[2] - b[2];
}
static double vdot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double vnorm(const double* a) { return sqrt(vdot(a, a)); }

/* object record from its vertex description; returns 0 on success */
int orc_object_record(int type, const double* v /*[3][3]*/, double* b, double* a1, double* a2) {
  for (int k = 0; k < 9; ++k)
    if (!isfinite(v[k])) return -1;
  for (int k = 0; k < 3; ++k) {
    b[k] = v[k];
    a1[k] = v[3 + k] - v[k];
    a2[k] = (type == ORC_QUAD) ? v[6 + k] - v[k] : 0.0;
  }
  if (type == ORC_QUAD) {
    double c[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
    if (vnorm(c) < 1e-9) return -2; /* zero area */
  } else if (type == ORC_EDGE) {
    if (vnorm(a1) < 1e-9) return -2; /* zero length */
  } else {
    return -3;
  }
  return 0;
}

/* dimension of object i in the reduced parameterisation */
static int dim_of(const orc_path* P, int i) { return P->type[i] == ORC_EDGE ? 1 : 2; }

/* interaction points x_0..x_{n+1} for unified parameters t[i][2] (Eq. 3) */
static void points_of(const orc_path* P, const double (*t)[2], double (*x)[3]) {
  memcpy(x[0], P->x0, sizeof(double) * 3);
  for (int i = 0; i < P->n; ++i)
    for (int k = 0; k < 3; ++k)
      x[i + 1][k] = P->b[i][k] + P->col[i][0][k] * t[i][0] + P->col[i][1][k] * t[i][1];
  memcpy(x[P->n + 1], P->xe, sizeof(double) * 3);
}

/* total length L(T; A, B) of Eq. 5 */
double orc_length_t(const orc_path* P, const double (*t)[2]) {
  double x[ORC_NMAX + 2][3], z[3], L = 0.0;
  points_of(P, t, x);
  for (int j = 0; j <= P->n; ++j) {
    vsub(x[j + 1], x[j], z);
    L += vnorm(z);
  }
  return L;
}

/* Segment vectors z_j = x_{j+1} - x_j, lengths and unit vectors. */
typedef struct {
  double z[ORC_NMAX + 1][3], len[ORC_NMAX + 1], u[ORC_NMAX + 1][3];
} orc_segments;

/* With eps > 0 the segment length |z| is replaced by the smooth
 * r = sqrt(|z|^2 + eps^2) (len = r, u = z / r); eps = 0 is Eq. 5 itself. */
static void segments_eps(const orc_path* P, const double (*t)[2], double eps, orc_segments* S) {
  double x[ORC_NMAX + 2][3];
  points_of(P, t, x);
  for (int j = 0; j <= P->n; ++j) {
    vsub(x[j + 1], x[j], S->z[j]);
    S->len[j] = sqrt(vdot(S->z[j], S->z[j]) + eps * eps);
    for (int k = 0; k < 3; ++k) S->u[j][k] = S->len[j] > 0 ? S->z[j][k] / S->len[j] : 0.0;
  }
}

static void segments_of(const orc_path* P, const double (*t)[2], orc_segments* S) { segments_eps(P, t, 0.0, S); }

static double smoothed_length(const orc_path* P, const double (*t)[2], double eps) {
  orc_segments S;
  segments_eps(P, t, eps, &S);
  double L = 0.0;
  for (int j = 0; j <= P->n; ++j) L += S.len[j];
  return L;
}

/* Gradient of Eq. 5 w.r.t. t_i (unified d = 2): dL/dt_ik = col_ik . (u_{i-1} - u_i),
 * since x_i enters z_{i-1} with + and z_i with -. */
static void gradient_unified(const orc_path* P, const orc_segments* S, double (*g)[2]) {
  for (int i = 0; i < P->n; ++i) {
    double d[3];
    vsub(S->u[i], S->u[i + 1], d);
    g[i][0] = vdot(P->col[i][0], d);
    g[i][1] = vdot(P->col[i][1], d);
  }
}

/* M_j = d u_j / d z_j = (I - u_j u_j^T) / |z_j| */
static void proj_over_len(const orc_segments* S, int j, double M[3][3]) {
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) M[a][c] = ((a == c ? 1.0 : 0.0) - S->u[j][a] * S->u[j][c]) / S->len[j];
}

static double quad_form(const double* p, double M[3][3], const double* q) {
  double r = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) r += p[a] * M[a][c] * q[c];
  return r;
}

/* ------------------------------------------------------------------------ */
/* Reduced parameterisation: unknown vector w of size m = sum_i d_i.          */
/* ------------------------------------------------------------------------ */

static int reduced_size(const orc_path* P, int* off) {
  int m = 0;
  for (int i = 0; i < P->n; ++i) {
    off[i] = m;
    m += dim_of(P, i);
  }
  return m;
}

static void reduced_to_unified(const orc_path* P, const int* off, const double* w, double (*t)[2]) {
  for (int i = 0; i < P->n; ++i) {
    t[i][0] = w[off[i]];
    t[i][1] = dim_of(P, i) == 2 ? w[off[i] + 1] : 0.5;
  }
}

/* gradient (m) and exact Hessian (m x m) of Eq. 5 in the reduced coordinates.
 * d2L/dt_ik dt_il   = col_ik^T (M_{i-1} + M_i) col_il
 * d2L/dt_ik dt_i+1l = -col_ik^T M_i col_{i+1,l}                              */
static void grad_hess_reduced(const orc_path* P, const int* off, const orc_segments* S, double* g, double* H, int m) {
  double gu[ORC_NMAX][2];
  gradient_unified(P, S, gu);
  for (int i = 0; i < P->n; ++i)
    for (int k = 0; k < dim_of(P, i); ++k) g[off[i] + k] = gu[i][k];
  if (!H) return;
  memset(H, 0, sizeof(double) * m * m);
  double Mj[ORC_NMAX + 1][3][3];
  for (int j = 0; j <= P->n; ++j) proj_over_len(S, j, Mj[j]);
  for (int i = 0; i < P->n; ++i) {
    double Ms[3][3];
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) Ms[a][c] = Mj[i][a][c] + Mj[i + 1][a][c];
    for (int k = 0; k < dim_of(P, i); ++k) {
      for (int l = 0; l < dim_of(P, i); ++l) H[(off[i] + k) * m + off[i] + l] = quad_form(P->col[i][k], Ms, P->col[i][l]);
      if (i + 1 < P->n)
        for (int l = 0; l < dim_of(P, i + 1); ++l) {
          double h = -quad_form(P->col[i][k], Mj[i + 1], P->col[i + 1][l]);
          H[(off[i] + k) * m + off[i + 1] + l] = h;
          H[(off[i + 1] + l) * m + off[i] + k] = h;
        }
    }
  }
}

/* Solve H x = r by Gaussian elimination with partial pivoting (H copied).
 * Returns 0 on success, -1 if a pivot is (numerically) zero. */
static int dense_solve(const double* H, const double* r, double* x, int m) {
  double a[ORC_MMAX][ORC_MMAX + 1];
  double scale = 0.0;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) {
      a[i][j] = H[i * m + j];
      if (fabs(a[i][j]) > scale) scale = fabs(a[i][j]);
    }
    a[i][m] = r[i];
  }
  if (scale == 0.0) return -1;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int i = c + 1; i < m; ++i)
      if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
    if (fabs(a[piv][c]) <= 1e-300 || fabs(a[piv][c]) < 1e-15 * scale) return -1;
    if (piv != c)
      for (int j = 0; j <= m; ++j) {
        double tmp = a[c][j];
        a[c][j] = a[piv][j];
        a[piv][j] = tmp;
      }
    for (int i = c + 1; i < m; ++i) {
      double f = a[i][c] / a[c][c];
      for (int j = c; j <= m; ++j) a[i][j] -= f * a[c][j];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = a[i][m];
    for (int j = i + 1; j < m; ++j) s -= a[i][j] * x[j];
    x[i] = s / a[i][i];
  }
  return 0;
}

/* largest world-space displacement max_i |A_i dt_i| of a reduced step */
static double world_step(const orc_path* P, const int* off, const double* dw) {
  double worst = 0.0;
  for (int i = 0; i < P->n; ++i) {
    double d[3] = {0, 0, 0};
    for (int k = 0; k < dim_of(P, i); ++k)
      for (int c = 0; c < 3; ++c) d[c] += P->col[i][k][c] * dw[off[i] + k];
    double s = vnorm(d);
    if (s > worst) worst = s;
  }
  return worst;
}

static double path_scale(const orc_path* P) {
  double s = 1.0;
  for (int k = 0; k < 3; ++k) {
    if (fabs(P->x0[k]) > s) s = fabs(P->x0[k]);
    if (fabs(P->xe[k]) > s) s = fabs(P->xe[k]);
  }
  for (int i = 0; i < P->n; ++i)
    for (int k = 0; k < 3; ++k)
      if (fabs(P->b[i][k]) > s) s = fabs(P->b[i][k]);
  return s;
}

static double min_len(const orc_path* P, const orc_segments* S) {
  double m = INFINITY;
  for (int j = 0; j <= P->n; ++j)
    if (S->len[j] < m) m = S->len[j];
  return m;
}

/* ------------------------------------------------------------------------ */
/* Stationarity residual: rho = max_i |A_i delta_i| (metres), where          */
/* delta = -H^{-1} grad L is the exact Newton step at the given T (Eq. 8:   */
/* a solution makes grad_T L vanish, and rho measures how far it is).       */
/* ------------------------------------------------------------------------ */
double orc_residual(const orc_path* P, const double (*t)[2]) {
  int off[ORC_NMAX];
  int m = reduced_size(P, off);
  orc_segments S;
  segments_of(P, t, &S);
  if (!(min_len(P, &S) > 0)) return INFINITY;
  double g[ORC_MMAX], H[ORC_MMAX * ORC_MMAX], d[ORC_MMAX], r[ORC_MMAX];
  grad_hess_reduced(P, off, &S, g, H, m);
  for (int i = 0; i < m; ++i) r[i] = -g[i];
  if (dense_solve(H, r, d, m) != 0) return INFINITY;
  return world_step(P, off, d);
}

/* ------------------------------------------------------------------------ */
/* Ground-truth minimiser of Eq. 4 (reduced parameters d = 1 / 2).           */
/* L is convex but not smooth where a segment has zero length, and Newton or */
/* gradient iterations can stall at such a kink although it is not the      */
/* minimum.  So the minimiser is reached by smoothing and continuation:     */
/* every |z_j| becomes sqrt(|z_j|^2 + eps^2) (smooth, strictly convex), and  */
/* damped Newton (Newton direction, steepest descent if that is not a       */
/* descent direction, Armijo backtracking) minimises it for                 */
/* eps = 1e-2, 1e-4, ..., 1e-12 times the scene scale in turn, each stage   */
/* starting from the previous minimiser.  A last stage with eps = 0 is the  */
/* exact problem.  Start: object centroids (t = 1/2).  Stage stop: world-   */
/* space Newton step <= 1e-12 x scene scale (or 1e-6 eps).  If the smoothed */
/* minimiser keeps a segment shorter than deg_tol the exact minimiser is a  */
/* kink: DEGENERATE, the last smoothed point is returned.                   */
/* ------------------------------------------------------------------------ */
static int newton_stage(const orc_path* P, const int* off, int m, double eps, double tol, double scale,
                        int max_iters, double* w, int* iters) {
  double g[ORC_MMAX], H[ORC_MMAX * ORC_MMAX], d[ORC_MMAX], r[ORC_MMAX], wt[ORC_MMAX];
  double t[ORC_NMAX][2], tt[ORC_NMAX][2];
  orc_segments S;
  for (int it = 0; it < max_iters; ++it, ++*iters) {
    reduced_to_unified(P, off, w, t);
    segments_eps(P, (const double (*)[2])t, eps, &S);
    if (!(min_len(P, &S) > 0)) return 0;
    grad_hess_reduced(P, off, &S, g, H, m);
    for (int i = 0; i < m; ++i) r[i] = -g[i];
    int ok = dense_solve(H, r, d, m) == 0;
    double slope = 0.0;
    for (int i = 0; i < m; ++i) slope += g[i] * d[i];
    double ws = ok ? world_step(P, off, d) : INFINITY;
    if (ws <= tol) { /* converged: take the last (tiny) Newton step */
      for (int i = 0; i < m; ++i) w[i] += d[i];
      return 1;
    }
    double L0 = smoothed_length(P, (const double (*)[2])t, eps);
    if (!ok || !(slope < 0)) {
      for (int i = 0; i < m; ++i) d[i] = -g[i];
      slope = 0.0;
      for (int i = 0; i < m; ++i) slope -= g[i] * g[i];
    } else if (ws <= 1e-6 * scale) {
      /* local quadratic region: the decrease is below FP64 resolution of L,
       * so take the full Newton step unless L visibly grows */
      for (int i = 0; i < m; ++i) wt[i] = w[i] + d[i];
      reduced_to_unified(P, off, wt, tt);
      if (smoothed_length(P, (const double (*)[2])tt, eps) <= L0 * (1.0 + 1e-13)) {
        memcpy(w, wt, sizeof(double) * m);
        continue;
      }
    }
    double alpha = 1.0;
    for (;;) {
      for (int i = 0; i < m; ++i) wt[i] = w[i] + alpha * d[i];
      reduced_to_unified(P, off, wt, tt);
      if (smoothed_length(P, (const double (*)[2])tt, eps) <= L0 + 1e-4 * alpha * slope) break;
      alpha *= 0.5;
      if (alpha < 1e-30) return 0; /* no decrease possible at this precision */
    }
    memcpy(w, wt, sizeof(double) * m);
  }
  return 0;
}

int orc_newton_solve(const orc_path* P, int max_iters, double deg_tol, double (*t)[2], int* iters_out) {
  int off[ORC_NMAX];
  int m = reduced_size(P, off);
  double scale = path_scale(P);
  double w[ORC_MMAX];
  for (int i = 0; i < m; ++i) w[i] = 0.5;
  int iters = 0, status = 0;
  orc_segments S;
  for (double f = 1e-2; f >= 1e-12; f *= 1e-2) {
    double eps = f * scale;
    newton_stage(P, off, m, eps, fmax(1e-12 * scale, 1e-6 * eps), scale, max_iters, w, &iters);
  }
  reduced_to_unified(P, off, w, t);
  segments_of(P, (const double (*)[2])t, &S);
  if (min_len(P, &S) < deg_tol) {
    status |= ORC_DEGENERATE;
  } else {
    double w_exact[ORC_MMAX];
    memcpy(w_exact, w, sizeof(double) * m);
    if (newton_stage(P, off, m, 0.0, 1e-12 * scale, scale, max_iters, w_exact, &iters)) {
      status |= ORC_CONVERGED;
      memcpy(w, w_exact, sizeof(double) * m);
    }
    reduced_to_unified(P, off, w, t);
    segments_of(P, (const double (*)[2])t, &S);
    if (min_len(P, &S) < deg_tol) status |= ORC_DEGENERATE;
  }
  if (iters_out) *iters_out = iters;
  for (int i = 0; i < P->n; ++i)
    if (!isfinite(t[i][0]) || !isfinite(t[i][1])) status |= ORC_NONFINITE;
  return status;
}

/* ------------------------------------------------------------------------ */
/* The paper's solver (Sec. III-C) in FP64 on the unified d = 2 unknowns.    */
/*   H_0 = I (inverse-Hessian estimate); p = -H g;                          */
/*   step size: fp_iters rounds of Eq. 6 starting from alpha0;              */
/*   T += alpha p; BFGS inverse update (skipped when s^T y is not positive);*/
/*   stop when the world-space step max_i |A_i s_i| <= tol_step, or after   */
/*   max_iters steps (Sec. III-C runs a fixed count; tol_step = 0 does so). */
/* Options: alpha0 for the first step and for later steps, and whether H is */
/* rescaled by s^T y / y^T y before the first update.                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  int max_iters, fp_iters, scale_h0, safeguard;
  double alpha0_first, alpha0, tol_step;
  double stop_len; /* stop when a segment gets shorter than this (heading into a kink); 0 = never */
} orc_bfgs_params;

static void grad_flat(const orc_path* P, const orc_segments* S, double* g) {
  double gu[ORC_NMAX][2];
  gradient_unified(P, S, gu);
  for (int i = 0; i < P->n; ++i) {
    g[2 * i] = gu[i][0];
    g[2 * i + 1] = gu[i][1];
  }
}

/* A_i p_i in world space for a flat unified vector p */
static void apply_cols(const orc_path* P, const double* p, int i, double* out) {
  for (int c = 0; c < 3; ++c) out[c] = P->col[i][0][c] * p[2 * i] + P->col[i][1][c] * p[2 * i + 1];
}

/* Eq. 6: fixed-point update of the step size along direction p.             */
/* Steps are capped at this many quasi-Newton steps (keeps rounds at a vanishing direction finite). */
#define ORC_ALPHA_MAX 1e3

double orc_fixed_point_alpha(const orc_path* P, const orc_segments* S, const double* p, double alpha, int fp_iters) {
  int n = P->n;
  double q[ORC_NMAX + 1][3], Ap[ORC_NMAX + 2][3];
  memset(Ap, 0, sizeof(Ap));
  for (int i = 0; i < n; ++i) apply_cols(P, p, i, Ap[i + 1]); /* Ap[0] = Ap[n+1] = 0 */
  for (int j = 0; j <= n; ++j) vsub(Ap[j + 1], Ap[j], q[j]); /* Delta A_j p_j */
  for (int k = 0; k < fp_iters; ++k) {
    double num = 0.0, den = 0.0;
    for (int j = 0; j <= n; ++j) {
      double v[3];
      for (int c = 0; c < 3; ++c) v[c] = S->z[j][c] + alpha * q[j][c];
      double r = vnorm(v);
      if (!(r > 0)) continue;
      num += vdot(q[j], S->z[j]) / r;
      den += vdot(q[j], q[j]) / r;
    }
    if (!(den > 1e-300)) return 0.0;
    alpha = -num / den;
    if (alpha > ORC_ALPHA_MAX) alpha = ORC_ALPHA_MAX; /* step cap (same reading as the GPU solver) */
  }
  return alpha;
}

/* t holds the start on entry when start_given is set (a learned start), else t = 1/2 */
int orc_bfgs_solve(const orc_path* P, const orc_bfgs_params* prm, double (*t)[2], int* iters_out, int start_given) {
  int n = P->n, m = 2 * n;
  double H[ORC_MMAX][ORC_MMAX], g[ORC_MMAX], gn[ORC_MMAX], p[ORC_MMAX], s[ORC_MMAX], y[ORC_MMAX];
  if (!start_given)
    for (int i = 0; i < n; ++i) t[i][0] = t[i][1] = 0.5;
  for (int a = 0; a < m; ++a)
    for (int c = 0; c < m; ++c) H[a][c] = (a == c) ? 1.0 : 0.0;
  orc_segments S;
  segments_of(P, t, &S);
  int status = 0, it = 0;
  if (!(min_len(P, &S) > 0)) {
    if (iters_out) *iters_out = 0;
    return ORC_DEGENERATE;
  }
  grad_flat(P, &S, g);
  for (it = 0; it < prm->max_iters; ++it) {
    for (int a = 0; a < m; ++a) {
      p[a] = 0.0;
      for (int c = 0; c < m; ++c) p[a] -= H[a][c] * g[c];
    }
    double alpha = orc_fixed_point_alpha(P, &S, p, it == 0 ? prm->alpha0_first : prm->alpha0, prm->fp_iters);
    /* safeguard: a non-positive step means the iteration started beyond the
     * line minimum; restart it at alpha = 0, where one round of Eq. 6 is a
     * majorise-minimise step and so positive along a descent direction */
    if (!(alpha > 0.0) && prm->safeguard) alpha = orc_fixed_point_alpha(P, &S, p, 0.0, prm->fp_iters);
    for (int a = 0; a < m; ++a) s[a] = alpha * p[a];
    for (int i = 0; i < n; ++i) {
      t[i][0] += s[2 * i];
      t[i][1] += s[2 * i + 1];
    }
    segments_of(P, t, &S);
    if (!(min_len(P, &S) > 0)) {
      status |= ORC_DEGENERATE;
      ++it;
      break;
    }
    grad_flat(P, &S, gn);
    double sy = 0.0, ss = 0.0, yy = 0.0;
    for (int a = 0; a < m; ++a) {
      y[a] = gn[a] - g[a];
      sy += s[a] * y[a];
      ss += s[a] * s[a];
      yy += y[a] * y[a];
    }
    if (sy > 1e-12 * sqrt(ss * yy) && sy > 0) {
      if (it == 0 && prm->scale_h0) {
        double gam = sy / yy;
        for (int a = 0; a < m; ++a)
          for (int c = 0; c < m; ++c) H[a][c] *= gam;
      }
      /* H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T  (Nocedal-Wright 6.17) */
      double rho = 1.0 / sy, Hy[ORC_MMAX], yHy = 0.0;
      for (int a = 0; a < m; ++a) {
        Hy[a] = 0.0;
        for (int c = 0; c < m; ++c) Hy[a] += H[a][c] * y[c];
        yHy += y[a] * Hy[a];
      }
      for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c)
          H[a][c] += -rho * (Hy[a] * s[c] + s[a] * Hy[c]) + (rho * rho * yHy + rho) * s[a] * s[c];
    }
    memcpy(g, gn, sizeof(double) * m);
    double ws = 0.0;
    for (int i = 0; i < n; ++i) {
      double d[3];
      apply_cols(P, s, i, d);
      if (vnorm(d) > ws) ws = vnorm(d);
    }
    if (ws <= prm->tol_step) {
      status |= ORC_CONVERGED;
      ++it;
      break;
    }
    if (min_len(P, &S) < prm->stop_len) {
      ++it;
      break;
    }
  }
  if (iters_out) *iters_out = it;
  for (int i = 0; i < n; ++i)
    if (!isfinite(t[i][0]) || !isfinite(t[i][1])) status |= ORC_NONFINITE;
  return status;
}

/* ------------------------------------------------------------------------ */
/* Validity (Sec. I / Sec. III: points must lie inside their object).        */
/* Closed intervals.  Boundary distance: signed in-plane distance (metres)   */
/* to the nearest side line, minimised over the path's objects; positive     */
/* inside.                                                                   */
/* ------------------------------------------------------------------------ */
static double side_distance(const orc_path* P, int i, const double* ti) {
  if (P->type[i] == ORC_EDGE) {
    double l = vnorm(P->col[i][0]);
    return fmin(ti[0], 1.0 - ti[0]) * l;
  }
  const double *a1 = P->col[i][0], *a2 = P->col[i][1];
  double c[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
  double area = vnorm(c);
  double h1 = area / vnorm(a2), h2 = area / vnorm(a1);
  return fmin(fmin(ti[0], 1.0 - ti[0]) * h1, fmin(ti[1], 1.0 - ti[1]) * h2);
}

int orc_validity(const orc_path* P, const double (*t)[2], double* boundary_dist) {
  int inside = 1;
  double dmin = INFINITY;
  for (int i = 0; i < P->n; ++i) {
    int ok = t[i][0] >= 0.0 && t[i][0] <= 1.0;
    if (P->type[i] == ORC_QUAD) ok = ok && t[i][1] >= 0.0 && t[i][1] <= 1.0;
    inside = inside && ok;
    double d = side_distance(P, i, t[i]);
    if (d < dmin) dmin = d;
  }
  if (boundary_dist) *boundary_dist = dmin;
  return inside;
}

/* ------------------------------------------------------------------------ */
/* Implicit differentiation (Sec. III-D).                                    */
/* Loss l = sum_i dX_i . x_i* + dL * L*.  With v = dl/dT at T* (reduced):    */
/*   solve H^T u = -v                              (Eq. 12, H symmetric)     */
/*   dl/dtheta = u^T d(grad_T L)/dtheta + dl/dtheta|_T      (Eq. 13 + direct) */
/* theta per path = (x0[3], xe[3], then per slot b_i[3], col_i1[3], col_i2[3]).*/
/* d(grad_T L)/dtheta is formed column by column: perturb one scalar of      */
/* theta symbolically, propagate dx -> dz -> du -> d(grad).                  */
/* ------------------------------------------------------------------------ */
#define ORC_NTHETA (6 + 9 * ORC_NMAX)

int orc_vjp(const orc_path* P, const double (*t)[2], const double* dX /*[n][3]*/, double dL, double* dtheta /*[6+9n]*/) {
  int n = P->n, off[ORC_NMAX];
  int m = reduced_size(P, off);
  orc_segments S;
  segments_of(P, t, &S);
  if (!(min_len(P, &S) > 0)) return -1;
  double g[ORC_MMAX], H[ORC_MMAX * ORC_MMAX], v[ORC_MMAX], u[ORC_MMAX], r[ORC_MMAX];
  grad_hess_reduced(P, off, &S, g, H, m);
  /* v = dl/dT = A_i^T dX_i + dL * grad_T L */
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < dim_of(P, i); ++k) v[off[i] + k] = vdot(P->col[i][k], dX + 3 * i) + dL * g[off[i] + k];
  for (int a = 0; a < m; ++a) r[a] = -v[a];
  if (dense_solve(H, r, u, m) != 0) return -2;
  double M[ORC_NMAX + 1][3][3];
  for (int j = 0; j <= n; ++j) proj_over_len(&S, j, M[j]);
  int np = 6 + 9 * n;
  for (int pidx = 0; pidx < np; ++pidx) {
    /* which scalar of theta: endpoint or slot parameter */
    double dx[ORC_NMAX + 2][3];
    double dcol[ORC_NMAX][2][3];
    memset(dx, 0, sizeof(dx));
    memset(dcol, 0, sizeof(dcol));
    if (pidx < 3) {
      dx[0][pidx] = 1.0;
    } else if (pidx < 6) {
      dx[n + 1][pidx - 3] = 1.0;
    } else {
      int q = pidx - 6, i = q / 9, w = q % 9, c = w % 3;
      if (w < 3) {
        dx[i + 1][c] = 1.0; /* d b_i */
      } else {
        int k = (w < 6) ? 0 : 1; /* d col_ik */
        if (k == 1 && P->type[i] == ORC_EDGE) {
          dtheta[pidx] = 0.0; /* structurally zero column */
          continue;
        }
        dcol[i][k][c] = 1.0;
        dx[i + 1][c] = t[i][k];
      }
    }
    /* d(grad)_ik = dcol_ik . (u_{i-1} - u_i) + col_ik . (M_{i-1} dz_{i-1} - M_i dz_i) */
    double dz[ORC_NMAX + 1][3], du[ORC_NMAX + 1][3];
    for (int j = 0; j <= n; ++j) {
      vsub(dx[j + 1], dx[j], dz[j]);
      for (int a = 0; a < 3; ++a) du[j][a] = M[j][a][0] * dz[j][0] + M[j][a][1] * dz[j][1] + M[j][a][2] * dz[j][2];
    }
    double acc = 0.0;
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < dim_of(P, i); ++k) {
        double dd[3], d0[3];
        vsub(S.u[i], S.u[i + 1], d0);
        vsub(du[i], du[i + 1], dd);
        double dg = vdot(dcol[i][k], d0) + vdot(P->col[i][k], dd);
        acc += u[off[i] + k] * dg;
      }
    /* explicit dependence of the loss on theta at fixed T */
    double direct = 0.0;
    for (int i = 0; i < n; ++i) direct += vdot(dX + 3 * i, dx[i + 1]);
    for (int j = 0; j <= n; ++j) direct += dL * vdot(S.u[j], dz[j]);
    dtheta[pidx] = acc + direct;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Candidate sequences (Sec. III: all ordered sequences of n objects, for   */
/* n = lo..hi).  Exhaustive order: within one TX/RX pair, orders ascending, */
/* then lexicographic in the alphabet index with the first interaction the  */
/* most significant digit (the order of itertools.product).                 */
/* ------------------------------------------------------------------------ */
uint64_t orc_exhaustive_per_pair(int K, int lo, int hi) {
  uint64_t tot = 0, p = 1;
  for (int n = 1; n <= hi; ++n) {
    p *= (uint64_t)K;
    if (n >= lo) tot += p;
  }
  return tot;
}

int orc_exhaustive_decode(int K, int lo, int hi, uint64_t r, int32_t* digits) {
  uint64_t p = 1;
  for (int n = 1; n < lo; ++n) p *= (uint64_t)K;
  for (int n = lo; n <= hi; ++n) {
    p *= (uint64_t)K;
    if (r < p) {
      for (int j = n - 1; j >= 0; --j) {
        digits[j] = (int32_t)(r % (uint64_t)K);
        r /= (uint64_t)K;
      }
      return n;
    }
    r -= p;
  }
  return -1;
}

/* splitmix64 finaliser (Steele, Lea & Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014): the output function of the generator. */
static uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* counter-based draw: the (8 g + slot + 1)-th state of a splitmix64 stream seeded with seed */
uint64_t orc_draw(uint64_t seed, uint64_t g, int slot) {
  return sm64_mix(seed + 0x9E3779B97F4A7C15ULL * (8ULL * g + (uint64_t)slot + 1ULL));
}

/* seeded sequence: order uniform in [lo, hi]; first object uniform; each next
 * object uniform among the K-1 objects different from its predecessor. */
int orc_seeded_decode(uint64_t seed, int K, int lo, int hi, uint64_t g, int32_t* digits) {
  int n = lo + (int)(orc_draw(seed, g, 0) % (uint64_t)(hi - lo + 1));
  digits[0] = (int32_t)(orc_draw(seed, g, 1) % (uint64_t)K);
  for (int j = 1; j < n; ++j)
    digits[j] = (int32_t)((digits[j - 1] + 1 + (int32_t)(orc_draw(seed, g, j + 1) % (uint64_t)(K - 1))) % K);
  return n;
}

/* decode many global indices at once (ids [M][n_max], -1 in unused slots) */
void orc_decode_batch(int mode, uint64_t seed, int K, int lo, int hi, uint64_t per_pair, int n_rx, const int32_t* alphabet,
                      int64_t M, const uint64_t* g, int n_max, int32_t* ids, int32_t* order, int32_t* tx_idx,
                      int32_t* rx_idx) {
  for (int64_t k = 0; k < M; ++k) {
    int32_t digits[ORC_NMAX];
    int n = mode == 0 ? orc_exhaustive_decode(K, lo, hi, g[k] % per_pair, digits)
                      : orc_seeded_decode(seed, K, lo, hi, g[k], digits);
    order[k] = n;
    for (int j = 0; j < n_max; ++j) ids[k * n_max + j] = j < n ? alphabet[digits[j]] : -1;
    uint64_t pair = g[k] / per_pair;
    tx_idx[k] = (int32_t)(pair / (uint64_t)n_rx);
    rx_idx[k] = (int32_t)(pair % (uint64_t)n_rx);
  }
}

/* ------------------------------------------------------------------------ */
/* Batch drivers (independent paths across threads).                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  /* scene */
  int K;
  const uint8_t* types;
  const double* verts; /* [K][3][3] */
  int n_tx, n_rx;
  const double *tx, *rx; /* [n][3] */
  /* paths */
  int64_t M;
  int n_max;
  const int32_t* ids;   /* [M][n_max] object ids */
  const int32_t* order; /* [M] */
  const int32_t* tx_idx; /* [M] */
  const int32_t* rx_idx; /* [M] */
  /* solver */
  int solver; /* 0 = Newton (ground truth), 1 = paper BFGS + Eq. 6 */
  int max_iters;
  orc_bfgs_params bfgs;
  double solved_tol; /* stationarity tolerance in metres */
  double deg_tol;    /* shortest segment of a non-degenerate solution (metres) */
  /* outputs (any may be NULL) */
  const double* T_start; /* [M][n_max][2] BFGS start, or NULL for t = 1/2 */
  double* T;   /* [M][n_max][2] */
  double* X;   /* [M][n_max][3] */
  double* L;   /* [M] */
  double* rho; /* [M] */
  double* bdist; /* [M] */
  int32_t* status;
  int32_t* iters;
  /* backward (optional) */
  const double* dX; /* [M][n_max][3] */
  const double* dL; /* [M] */
  double* dtheta;   /* [M][6 + 9 n_max] per-path parameter gradients */
  int n_threads;
} orc_batch;

static int build_path(const orc_batch* B, int64_t p, orc_path* P) {
  int n = B->order[p];
  if (n < 1 || n > ORC_NMAX || n > B->n_max) return ORC_INVALID_INPUT;
  int ti = B->tx_idx[p], ri = B->rx_idx[p];
  if (ti < 0 || ti >= B->n_tx || ri < 0 || ri >= B->n_rx) return ORC_INVALID_INPUT;
  P->n = n;
  memcpy(P->x0, B->tx + 3 * ti, sizeof(double) * 3);
  memcpy(P->xe, B->rx + 3 * ri, sizeof(double) * 3);
  int st = 0;
  for (int i = 0; i < n; ++i) {
    int o = B->ids[p * B->n_max + i];
    if (o < 0 || o >= B->K) return ORC_INVALID_INPUT;
    P->type[i] = B->types[o];
    if (orc_object_record(B->types[o], B->verts + 9 * o, P->b[i], P->col[i][0], P->col[i][1]) != 0)
      return ORC_INVALID_INPUT;
    if (i > 0 && B->ids[p * B->n_max + i - 1] == o) st |= ORC_REPEAT;
  }
  return st;
}

static void run_one(const orc_batch* B, int64_t p) {
  orc_path P;
  double t[ORC_NMAX][2];
  int st = build_path(B, p, &P), it = 0;
  for (int i = 0; i < ORC_NMAX; ++i) t[i][0] = t[i][1] = 0.5;
  if (B->T_start)
    for (int i = 0; i < P.n && i < B->n_max; ++i) {
      t[i][0] = B->T_start[(p * B->n_max + i) * 2];
      t[i][1] = P.type[i] == ORC_EDGE ? 0.5 : B->T_start[(p * B->n_max + i) * 2 + 1];
    }
  if (!(st & ORC_INVALID_INPUT) && !(st & ORC_REPEAT)) {
    if (B->solver == 0)
      st |= orc_newton_solve(&P, B->max_iters, B->deg_tol, t, &it);
    else
      st |= orc_bfgs_solve(&P, &B->bfgs, t, &it, B->T_start != NULL);
    orc_segments S;
    segments_of(&P, (const double (*)[2])t, &S);
    if (min_len(&P, &S) < B->deg_tol) st |= ORC_DEGENERATE;
  }
  double rho = INFINITY, bd = -INFINITY;
  if (!(st & ORC_INVALID_INPUT)) {
    if (orc_validity(&P, (const double (*)[2])t, &bd)) st |= ORC_VALID;
    if (!(st & (ORC_REPEAT | ORC_DEGENERATE | ORC_NONFINITE))) {
      rho = orc_residual(&P, (const double (*)[2])t);
      if (rho <= B->solved_tol) st |= ORC_SOLVED;
    }
  }
  int nm = B->n_max;
  if (B->T)
    for (int i = 0; i < nm; ++i) {
      B->T[(p * nm + i) * 2 + 0] = i < P.n ? t[i][0] : 0.0;
      B->T[(p * nm + i) * 2 + 1] = i < P.n ? t[i][1] : 0.0;
    }
  if (B->X && !(st & ORC_INVALID_INPUT)) {
    double x[ORC_NMAX + 2][3];
    points_of(&P, (const double (*)[2])t, x);
    for (int i = 0; i < nm; ++i)
      for (int c = 0; c < 3; ++c) B->X[(p * nm + i) * 3 + c] = i < P.n ? x[i + 1][c] : 0.0;
  }
  if (B->L) B->L[p] = (st & ORC_INVALID_INPUT) ? NAN : orc_length_t(&P, (const double (*)[2])t);
  if (B->rho) B->rho[p] = rho;
  if (B->bdist) B->bdist[p] = bd;
  if (B->status) B->status[p] = st;
  if (B->iters) B->iters[p] = it;
  if (B->dtheta) {
    int np = 6 + 9 * nm;
    double* out = B->dtheta + p * np;
    for (int k = 0; k < np; ++k) out[k] = 0.0;
    int usable = !(st & (ORC_INVALID_INPUT | ORC_REPEAT | ORC_DEGENERATE | ORC_NONFINITE));
    if (usable) {
      double dx[ORC_NMAX][3];
      for (int i = 0; i < P.n; ++i)
        for (int c = 0; c < 3; ++c) dx[i][c] = B->dX ? B->dX[(p * nm + i) * 3 + c] : 0.0;
      double dth[ORC_NTHETA];
      if (orc_vjp(&P, (const double (*)[2])t, &dx[0][0], B->dL ? B->dL[p] : 0.0, dth) == 0)
        for (int k = 0; k < 6 + 9 * P.n; ++k) out[k] = dth[k];
    }
  }
}

typedef struct {
  const orc_batch* B;
  int64_t lo, hi;
} orc_chunk;

static void* run_chunk(void* arg) {
  orc_chunk* c = (orc_chunk*)arg;
  for (int64_t p = c->lo; p < c->hi; ++p) run_one(c->B, p);
  return NULL;
}

int orc_solve_batch(const orc_batch* B) {
  int nt = B->n_threads > 0 ? B->n_threads : 1;
  if (nt > 256) nt = 256;
  if (nt == 1 || B->M < 64) {
    for (int64_t p = 0; p < B->M; ++p) run_one(B, p);
    return 0;
  }
  pthread_t th[256];
  orc_chunk ch[256];
  for (int k = 0; k < nt; ++k) {
    ch[k].B = B;
    ch[k].lo = B->M * k / nt;
    ch[k].hi = B->M * (k + 1) / nt;
    if (pthread_create(&th[k], NULL, run_chunk, &ch[k]) != 0) {
      run_chunk(&ch[k]);
      th[k] = 0;
    }
  }
  for (int k = 0; k < nt; ++k)
    if (th[k]) pthread_join(th[k], NULL);
  return 0;
}

/* single-path entry points for the tests: the path is given by arrays */
static void path_from_arrays(int n, const int32_t* types, const double* b, const double* cols, const double* x0,
                             const double* xe, orc_path* P) {
  P->n = n;
  memcpy(P->x0, x0, sizeof(double) * 3);
  memcpy(P->xe, xe, sizeof(double) * 3);
  for (int i = 0; i < n; ++i) {
    P->type[i] = types[i];
    memcpy(P->b[i], b + 3 * i, sizeof(double) * 3);
    memcpy(P->col[i][0], cols + 6 * i, sizeof(double) * 3);
    memcpy(P->col[i][1], cols + 6 * i + 3, sizeof(double) * 3);
  }
}

double orc_path_length(int n, const int32_t* types, const double* b, const double* cols, const double* x0,
                       const double* xe, const double* t) {
  orc_path P;
  path_from_arrays(n, types, b, cols, x0, xe, &P);
  return orc_length_t(&P, (const double (*)[2])t);
}

/* gradient (unified, 2n) and exact Hessian (unified 2n x 2n; rows/columns of
 * an edge's second coordinate are zero) of Eq. 5 */
int orc_path_grad_hess(int n, const int32_t* types, const double* b, const double* cols, const double* x0,
                       const double* xe, const double* t, double* g, double* H) {
  orc_path P;
  path_from_arrays(n, types, b, cols, x0, xe, &P);
  /* treat every object as a plane here: the unified parameterisation */
  orc_path Q = P;
  for (int i = 0; i < n; ++i) Q.type[i] = ORC_QUAD;
  orc_segments S;
  segments_of(&Q, (const double (*)[2])t, &S);
  if (!(min_len(&Q, &S) > 0)) return -1;
  int off[ORC_NMAX];
  int m = reduced_size(&Q, off);
  grad_hess_reduced(&Q, off, &S, g, H, m);
  return 0;
}

int orc_path_solve(int n, const int32_t* types, const double* b, const double* cols, const double* x0,
                   const double* xe, int solver, int max_iters, int fp_iters, double alpha0_first, double alpha0,
                   int scale_h0, int safeguard, double tol_step, double deg_tol, double* t, double* rho,
                   int* iters) {
  orc_path P;
  path_from_arrays(n, types, b, cols, x0, xe, &P);
  int st;
  if (solver == 0) {
    st = orc_newton_solve(&P, max_iters, deg_tol, (double (*)[2])t, iters);
  } else {
    orc_bfgs_params prm = {max_iters, fp_iters, scale_h0, safeguard, alpha0_first, alpha0, tol_step, 0.0};
    st = orc_bfgs_solve(&P, &prm, (double (*)[2])t, iters, 0);
  }
  if (rho) *rho = orc_residual(&P, (const double (*)[2])t);
  return st;
}

double orc_path_residual(int n, const int32_t* types, const double* b, const double* cols, const double* x0,
                         const double* xe, const double* t) {
  orc_path P;
  path_from_arrays(n, types, b, cols, x0, xe, &P);
  return orc_residual(&P, (const double (*)[2])t);
}

double orc_path_fixed_point(int n, const int32_t* types, const double* b, const double* cols, const double* x0,
                            const double* xe, const double* t, const double* p, double alpha0, int fp_iters) {
  orc_path P;
  path_from_arrays(n, types, b, cols, x0, xe, &P);
  orc_segments S;
  segments_of(&P, (const double (*)[2])t, &S);
  return orc_fixed_point_alpha(&P, &S, p, alpha0, fp_iters);
}

int orc_path_vjp(int n, const int32_t* types, const double* b, const double* cols, const double* x0,
                 const double* xe, const double* t, const double* dX, double dL, double* dtheta) {
  orc_path P;
  path_from_arrays(n, types, b, cols, x0, xe, &P);
  return orc_vjp(&P, (const double (*)[2])t, dX, dL, dtheta);
}
