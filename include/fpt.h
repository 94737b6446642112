/*
 * fpt.h -- C ABI of the batched Fermat path library (CUDA, sm_103a).
 *
 * The library finds ray paths between transmitters (TX) and receivers (RX)
 * that interact, in a given order, with planar reflectors and straight
 * diffraction edges.  For every candidate interaction sequence it minimises
 * the total path length (Fermat's principle) over one point per object,
 * following "Fast, Differentiable, GPU-Accelerated Ray Tracing for Multiple
 * Diffraction and Reflection Paths" (arXiv 2510.16172):
 *
 *   - candidate sequences: all ordered sequences of n objects, n = lo..hi
 *     (Sec. III, first paragraph);
 *   - unified parameterisation x_i = A_i t_i + b_i with t_i in R^2; an edge
 *     uses a zero second basis vector (Sec. III-B, Eq. 3);
 *   - objective: L(T; A, B) = sum_i |x_{i+1} - x_i|, x_0 = TX, x_{n+1} = RX
 *     (Sec. III-B, Eq. 4-5);
 *   - solver: BFGS on the inverse Hessian with the fixed-point step-size
 *     update of Eq. 6 (Sec. III-C), in FP32;
 *   - validity: each point inside its object (Sec. I, Sec. III);
 *   - gradients: implicit differentiation at grad_T L = 0 (Sec. III-D,
 *     Eq. 8-13).
 *
 * Conventions.
 *   - All calls are asynchronous on the context's CUDA stream unless stated.
 *     Device pointers are caller-owned and must stay valid until the stream
 *     reaches the call.  Host pointers are read before the call returns.
 *   - Objects: type FPT_QUAD (planar reflector) is the parallelogram with
 *     corners v0, v1, v1 + v3 - v0, v3, given as verts = (v0, v1, v3); its
 *     record is b = v0, A = [v1 - v0, v3 - v0] and t in [0,1]^2 is inside.
 *     Type FPT_EDGE (straight edge e0 -> e1) is given as verts = (e0, e1, *);
 *     b = e0, A = [e1 - e0, 0] and t_1 in [0,1] is inside.
 *   - Path index g (uint64) enumerates a batch; per-path arrays are indexed
 *     by g.  n_max is the batch's largest order; per-path slot arrays have
 *     n_max slots and unused slots are written as zero.
 *   - No call traps or faults on bad data: invalid per-path input gets the
 *     FPT_ST_INVALID_INPUT status bit.  Launch or argument errors are
 *     returned as fpt_status; fpt_last_error() gives a message.
 */
#ifndef FPT_H
#define FPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#pragma GCC visibility push(default) /* the library is built with -fvisibility=hidden */
#endif

typedef enum {
  FPT_OK = 0,
  FPT_EINVAL = 1,       /* bad argument (null pointer, size, degenerate object, ...) */
  FPT_ENOMEM = 2,       /* device or host allocation failed */
  FPT_ECUDA = 3,        /* a CUDA runtime call failed */
  FPT_EDEVICE = 4,      /* a kernel reported an error through the device error word */
  FPT_EUNSUPPORTED = 5  /* valid request outside what the library supports */
} fpt_status;

enum { FPT_QUAD = 0, FPT_EDGE = 1 };

/* per-path status bits (uint8) */
enum {
  FPT_ST_VALID = 1,         /* every point lies inside its object (closed test) */
  FPT_ST_CONVERGED = 2,     /* BFGS stopped on its world-space step tolerance */
  FPT_ST_SOLVED = 4,        /* stationarity residual <= solved_tol and not DEGENERATE/REPEAT/NONFINITE */
  FPT_ST_FP64 = 8,          /* the Hessian solve was redone in FP64 (ill-conditioned) */
  FPT_ST_DEGENERATE = 16,   /* a kink of L: a segment shorter than deg_tol at the solution, or BFGS ran a
                               segment below kink_stop before converging */
  FPT_ST_REPEAT = 32,       /* the same object twice in a row: not solved */
  FPT_ST_NONFINITE = 64,    /* NaN/Inf met */
  FPT_ST_INVALID_INPUT = 128 /* object id, order or TX/RX index out of range */
};

/* Solver parameters.  fpt_default_params() fills the defaults shown. */
typedef struct {
  int32_t max_iters;   /* BFGS step cap (64).  Sec. III-C runs a fixed count; see fixed_iters. */
  int32_t fp_iters;    /* rounds of the Eq. 6 fixed point per BFGS step (1; the paper also uses 64) */
  int32_t polish;      /* Newton steps with an FP64 gradient after BFGS (1; 0..2) */
  int32_t fixed_iters; /* 1: every path runs exactly max_iters steps (Sec. III-C); 0: stop on tol_step (0) */
  float tol_step;      /* BFGS stops when max_i |A_i s_i| <= tol_step metres (1e-4) */
  float solved_tol;    /* stationarity residual bound for FPT_ST_SOLVED, metres (1e-5) */
  float deg_tol;       /* a solution segment shorter than this (metres) is DEGENERATE (1e-3) */
  float cond_fp64;     /* Hessian pivot ratio below which the adjoint solve is redone in FP64 (1e-4); the
                          polish, which needs less accuracy, uses 1e-2 x this value */
  int32_t init_mode;   /* 0: plain init, t = 1/2 (object centroid).  1: learned (fpt_set_init_mlp) */
  int32_t polish_fp64; /* 0: polish gradient in double-float FP32 arithmetic (~2^-46, default); 1: in FP64 */
  int32_t refill;      /* lanes of a warp that must be free before it takes new paths (8); 0: one path per
                          lane until the whole warp is done */
  int32_t specialize;  /* 1: BFGS runs one kernel per interaction-type pattern (reflector/edge per slot), which
                          drops the edge's always-zero second parameter from the iteration and yields the same
                          iterates as the unified kernel, for every order whose non-empty pattern buckets all
                          hold at least 2048 paths per SM; 2: for every order; 0: the unified kernel of
                          Sec. III-B only (1; refill = 0 implies 0) */
  int32_t fuse_adjoint; /* fpt_solve_grad only.  1: each path's adjoint is formed inside the polish kernel;
                           0: the adjoint kernels of fpt_backward run after the solve (0; measured faster on
                           GB300 at order 3, where the fused kernel's larger code and register footprint lower
                           its issue rate more than the shared decoding saves) */
  float kink_stop;      /* BFGS stops a path, and flags it DEGENERATE, when one of its segments is shorter than
                           this (metres) after 4 or more steps without convergence: it is running into a kink,
                           where L is not smooth (0 = 0.1 deg_tol).  Larger values save BFGS steps on
                           kinked paths but also stop some regular paths whose iterates pass close to a kink */
  int32_t polish_all;   /* 0: a path whose residual at the BFGS point already meets solved_tol is returned as is,
                           the others take the `polish` Newton steps (0); 1: every path takes them */
  float polish_radius;  /* adaptive polish: Newton steps are taken only from a point whose residual is at most
                           this (metres; farther points are not near a stationary path and stay unsolved;
                           0.1; 0 = no limit) */
  int32_t reserved[4]; /* must be zero */
} fpt_solve_params;

typedef struct fpt_ctx fpt_ctx;
typedef struct fpt_scene fpt_scene;
typedef struct fpt_batch fpt_batch;

/* Defaults listed in fpt_solve_params. */
void fpt_default_params(fpt_solve_params* p);

/* Create a context on CUDA device `device`, launching on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  The context owns its
 * device workspace.  Returns FPT_ECUDA if the device cannot be used. */
fpt_status fpt_create(fpt_ctx** out, int device, void* cuda_stream);
void fpt_destroy(fpt_ctx* ctx);
/* Switch the context's stream.  No synchronisation (legal inside a stream
 * capture): work issued on the old stream, uploads included, must be complete
 * (fpt_sync) or otherwise ordered before the new stream's next use. */
fpt_status fpt_set_stream(fpt_ctx* ctx, void* cuda_stream);
/* Message for the last error on this context (static storage, never NULL). */
const char* fpt_last_error(const fpt_ctx* ctx);
/* How the backward calls (fpt_backward, fpt_solve_grad, fpt_backward_noalloc)
 * sum the per-path gradient terms of Sec. III-D over paths.  smem = 1 (the
 * default): each CTA adds its paths' terms into FP32 partial sums in shared
 * memory and adds those into the FP64 totals every flush_tiles of its tiles
 * of 128 paths (64 by default) and when it ends; a smaller flush_tiles puts
 * fewer terms into each FP32 partial sum (more accurate, more global
 * atomics).  smem = 0: every term is added straight into the FP64 totals.
 * Scenes whose partial sums do not fit shared memory always use smem = 0.
 * FPT_EINVAL unless flush_tiles >= 1 and smem is 0 or 1. */
fpt_status fpt_set_accumulation(fpt_ctx* ctx, int32_t flush_tiles, int32_t smem);
/* Wait for the stream, then check the device error word: FPT_EDEVICE if a
 * kernel flagged an error since the last check (the word is then cleared). */
fpt_status fpt_sync(fpt_ctx* ctx);

/* Scene upload (Sec. III-B, Eq. 3).  types: host uint8 [n_obj] (FPT_QUAD /
 * FPT_EDGE); verts: host double [n_obj][3][3].  The library builds object
 * records in FP32 (hi + lo parts) and FP64 on the device, relative to the
 * scene centre.  FPT_EINVAL on non-finite vertices, a zero-area plane or a
 * zero-length edge (< 1e-9 m), or n_obj outside [1, 65535].  The records
 * are built on the host and copied asynchronously on the context's stream
 * (ordered before every later call on it; the host inputs may be reused on
 * return, the scene keeps its own copies until fpt_scene_free). */
fpt_status fpt_scene_upload(fpt_ctx* ctx, const uint8_t* types, const double* verts, int32_t n_obj,
                            fpt_scene** out);
void fpt_scene_free(fpt_scene* scene);
/* Scene from a caller-owned DEVICE array verts [n_obj][3][3] FP32 (layout of
 * fpt_scene_upload) and host types [n_obj].  The records are built by a kernel
 * on the context's stream (as fpt_scene_update_vertices), relative to `centre`
 * (host double[3]; NULL = the origin), which the library cannot take from
 * device data without waiting for it; nothing waits for the device.
 * FPT_EINVAL on bad types, a non-finite centre or n_obj outside [1, 65535];
 * non-finite or degenerate objects set the device error word (FPT_EDEVICE at
 * fpt_sync).  The scene has no endpoints until fpt_set_endpoints[_device]. */
fpt_status fpt_scene_upload_device(fpt_ctx* ctx, const uint8_t* types, const float* verts, int32_t n_obj,
                                   const double* centre, fpt_scene** out);
/* TX and RX positions (x_0 and x_{n+1} of Eq. 2): host double [n][3].
 * Copied to the device asynchronously on the context's stream, as the scene.
 * Replacing the endpoints of a scene frees its old device copies first (which
 * waits for the device).  FPT_EINVAL on non-finite input or n < 1. */
fpt_status fpt_set_endpoints(fpt_scene* scene, const double* tx, int32_t n_tx, const double* rx, int32_t n_rx);

/* TX and RX positions from caller-owned DEVICE arrays: tx [n_tx][3], rx
 * [n_rx][3] FP32 (for example torch tensors that an optimisation loop updates
 * from the gradients of Sec. III-D).  A kernel on the context's stream builds
 * the endpoint records from them (each FP32 value taken exactly, relative to
 * the scene centre); nothing passes through host memory and the call does not
 * wait for the device, except when a count exceeds what the scene's endpoint
 * buffers already hold (the first call, or more endpoints than before: the
 * buffers are then reallocated).  The arrays are read when the stream reaches
 * the call and may change afterwards.  FPT_EINVAL on null pointers or n < 1;
 * non-finite coordinates set the device error word (FPT_EDEVICE at fpt_sync).
 * Batches are tied to the counts n_tx, n_rx as with fpt_set_endpoints. */
fpt_status fpt_set_endpoints_device(fpt_scene* scene, const float* tx, int32_t n_tx, const float* rx, int32_t n_rx);
/* Replace the geometry of every object from a caller-owned DEVICE array verts
 * [n_obj][3][3] FP32 (plane: v0, v1, v3; edge: e0, e1, unused), in the layout
 * of fpt_scene_upload.  Object types and the scene centre stay those of the
 * upload.  The records (Sec. III-B, Eq. 3), side heights and occluder records
 * are rebuilt in place by a kernel on the context's stream: no allocation, no
 * wait for the device; calls already issued on the stream use the old
 * geometry, later calls the new.  Non-finite vertices, zero-area planes and
 * zero-length edges (< 1e-9 m) set the device error word (FPT_EDEVICE at
 * fpt_sync) instead of being refused. */
fpt_status fpt_scene_update_vertices(fpt_scene* scene, const float* verts);

/* Candidate sequences (Sec. III).
 * Exhaustive: for every (tx, rx) pair, every ordered sequence over the
 *   alphabet (host int32 object ids; NULL = all objects) of order lo..hi.
 *   g = (tx * n_rx + rx) * per_pair + r; r runs over order lo first, each
 *   order in lexicographic order with the first interaction most significant.
 * Seeded: per_pair sequences for each pair; sequence g has order
 *   lo + h(g,0) mod (hi-lo+1), first object h(g,1) mod K and each next object
 *   (prev + 1 + h(g,j+1) mod (K-1)) mod K (no immediate repeats), where
 *   h(g,s) is splitmix64's output function applied to
 *   seed + 0x9E3779B97F4A7C15 * (8 g + s + 1).
 * Explicit: caller-owned device arrays ids [n][n_max] (object ids),
 *   order [n], tx_idx [n], rx_idx [n]; n = 0 is an empty batch (the arrays
 *   may then be NULL): every call on it succeeds, writes no per-path output
 *   (those pointers may be NULL too) and returns zero gradients.
 * FPT_EINVAL on lo < 1, hi > 10, lo > hi, empty alphabet or ids out of range
 * (host-checked arrays only).  A batch records the object types of the
 * scene it was built for; calls that pass a scene with other types return
 * FPT_EINVAL.  The alphabet tables are copied asynchronously on the
 * context's stream.  Seeded and explicit batches are bucketed on the device
 * by (order, interaction-type pattern) on their first use (synchronous). */
fpt_status fpt_batch_exhaustive(fpt_ctx* ctx, const fpt_scene* scene, const int32_t* alphabet, int32_t n_alpha,
                                int32_t order_lo, int32_t order_hi, fpt_batch** out);
fpt_status fpt_batch_seeded(fpt_ctx* ctx, const fpt_scene* scene, const int32_t* alphabet, int32_t n_alpha,
                            uint64_t seed, uint64_t per_pair, int32_t order_lo, int32_t order_hi, fpt_batch** out);
fpt_status fpt_batch_explicit(fpt_ctx* ctx, const fpt_scene* scene, const int32_t* ids_dev, const uint8_t* order_dev,
                              const int32_t* tx_idx_dev, const int32_t* rx_idx_dev, uint64_t n, int32_t n_max,
                              fpt_batch** out);
/* Number of paths and slots per path of a batch. */
fpt_status fpt_batch_size(const fpt_batch* batch, uint64_t* n_paths, int32_t* n_max);
void fpt_batch_free(fpt_batch* batch);
/* Write the batch's sequences (device outputs: ids [N][n_max] int32, order
 * [N] uint8, tx_idx [N], rx_idx [N] int32; any may be NULL). */
fpt_status fpt_enumerate(fpt_ctx* ctx, const fpt_batch* batch, int32_t* ids_out, uint8_t* order_out,
                         int32_t* tx_idx_out, int32_t* rx_idx_out);

/* Solve every path of the batch (Sec. III-C): plain init t = 1/2, BFGS with
 * Eq. 6 step sizes in FP32 (for orders 6-10 the inverse-Hessian estimate is
 * kept in shared memory; `specialize` applies to orders 1-5), then up to
 * `polish` Newton steps whose gradient
 * is formed in extended precision and whose block-tridiagonal Hessian system
 * is solved in FP32 (FP64 when ill-conditioned), then the validity test and
 * the stationarity residual rho = max_i |A_i delta_i| of the Newton step at
 * the returned T (paths already within solved_tol at the BFGS point skip the
 * steps unless polish_all = 1).  Device outputs (caller-owned; any but status_out may be NULL):
 *   T_out [N][n_max][2] float   parameters t_i (edges: t_i2 stays 1/2)
 *   X_out [N][n_max][3] float   world points x_i
 *   L_out [N] float             path length
 *   status_out [N] uint8        FPT_ST_* bits (required)
 *   iters_out [N] uint8         BFGS steps taken (saturates at 255)
 *   rho_out [N] float           stationarity residual, metres (inf if undefined) */
fpt_status fpt_solve(fpt_ctx* ctx, const fpt_scene* scene, const fpt_batch* batch, const fpt_solve_params* params,
                     float* T_out, float* X_out, float* L_out, uint8_t* status_out, uint8_t* iters_out,
                     float* rho_out);

/* Validity and stationarity at caller-given parameters T [N][n_max][2]
 * (device).  Outputs (device, any may be NULL): mask [N] uint8 (1 = inside),
 * bdist [N] float (signed in-plane distance to the nearest side line,
 * metres, minimised over the path; positive inside), rho [N] float. */
fpt_status fpt_validity(fpt_ctx* ctx, const fpt_scene* scene, const fpt_batch* batch, const float* T,
                        uint8_t* mask_out, float* bdist_out, float* rho_out);

/* Implicit-differentiation backward (Sec. III-D, Eq. 8-13) at solutions T
 * [N][n_max][2] (device).  Cotangents (device, may be NULL = zero):
 * dX [N][n_max][3] for the points, dL [N] for the lengths.  When dL is NULL
 * and dL_status_mask is non-zero, the length cotangent of a path is 1 if its
 * status holds every bit of the mask and 0 otherwise (e.g. FPT_ST_VALID |
 * FPT_ST_SOLVED differentiates the sum of the valid paths' lengths).  Per
 * path: v = A^T dX + dL grad_T L, solve H u = -v with the block-tridiagonal
 * Hessian H (FP32; FP64 if ill-conditioned), then u^T d(grad_T L)/dtheta plus
 * the explicit terms.  Paths with status REPEAT/DEGENERATE/NONFINITE/
 * INVALID_INPUT in `status` (device [N], may be NULL) contribute nothing,
 * and so do paths whose cotangents are all zero (skipped) and paths whose
 * Hessian is singular in FP64 too (counted by fpt_backward_dropped).
 * Gradients are summed over paths into device outputs that the call
 * overwrites (any may be NULL): g_tx [n_tx][3], g_rx [n_rx][3],
 * g_vertices [n_obj][3][3] (plane: v0, v1, v3; edge: e0, e1, zeros).
 * Uses a context-owned FP64 accumulator of 9 n_obj + 3 (n_tx + n_rx) values. */
fpt_status fpt_backward(fpt_ctx* ctx, const fpt_scene* scene, const fpt_batch* batch, const float* T,
                        const uint8_t* status, const float* dX, const float* dL, uint8_t dL_status_mask,
                        float* g_tx, float* g_rx, float* g_vertices);

/* Solve and backward in one call, for cotangents known when the solve starts
 * (Sec. III-C then Sec. III-D): the outputs of fpt_solve and the gradients of
 * fpt_backward(T_out, status_out, dX, dL, dL_status_mask).  The adjoint of
 * each path is formed either by the adjoint kernels of fpt_backward after
 * the solve (params->fuse_adjoint = 0, the default) or inside the polish
 * kernel from the state it already holds (fuse_adjoint = 1: geometry,
 * segment directions, lengths and Hessian factorisation at the returned
 * point); paths whose FP32 pivots fail the adjoint's test (or whose polish
 * ran in FP64) get an FP64 adjoint pass.  Gradients agree with fpt_backward
 * to FP32 rounding.  Requires polish >= 1 and polish_fp64 = 0 (FPT_EINVAL /
 * FPT_EUNSUPPORTED otherwise); status_out is required.  dX [N][n_max][3], dL [N] device or NULL; the
 * gradient outputs are overwritten as in fpt_backward. */
fpt_status fpt_solve_grad(fpt_ctx* ctx, const fpt_scene* scene, const fpt_batch* batch, const fpt_solve_params* params,
                          const float* dX, const float* dL, uint8_t dL_status_mask, float* T_out, float* X_out,
                          float* L_out, uint8_t* status_out, uint8_t* iters_out, float* rho_out, float* g_tx,
                          float* g_rx, float* g_vertices);

/* Obstruction of paths by the scene's planar objects (Sec. I: a candidate ray
 * is discarded when it is obstructed, as well as when an interaction point
 * falls outside its object).  For every path whose status holds all bits of
 * status_mask (status device [N], may be NULL when the mask is 0), with points
 * x_1..x_n from the parameters T [N][n_max][2] (device) and x_0 = TX,
 * x_{n+1} = RX: segment j (from x_j to x_{j+1}) is blocked when a planar
 * object other than the two objects at its ends has the segment's ends on
 * opposite sides of its plane, each more than tol metres from it (tol <= 0:
 * 1e-4), and the crossing point inside its closed parallelogram.  Edges block
 * nothing.  blocked_out [N] uint16 (device): bit j set = segment j blocked
 * (0 for paths not tested and for REPEAT / INVALID_INPUT sequences).  FPT_EINVAL
 * on missing arguments; FPT_EUNSUPPORTED above 3938 planar objects (their
 * 52-byte records are staged in shared memory). */
fpt_status fpt_occlusion(fpt_ctx* ctx, const fpt_scene* scene, const fpt_batch* batch, const float* T,
                         const uint8_t* status, uint8_t status_mask, float tol, uint16_t* blocked_out);

/* Gradient by automatic differentiation through the solver's iterations, the
 * alternative the implicit backward is compared with (Sec. IV-B, Fig. 3).
 * Every path of the batch runs exactly `steps` steps of the unified solver of
 * Sec. III-C (d = 2 unknowns per interaction, an edge's second basis vector
 * zero) from t = 1/2: H_0 = I, p = -H g, `fp_iters` rounds of the Eq. 6 fixed
 * point from alpha = 1 (redone from alpha = 0 when they give alpha <= 0; alpha
 * at most 1e3 times the quasi-Newton step), t += alpha p, and the BFGS inverse
 * update unless s.y <= 0 or (s.y)^2 <= 1e-12 |s|^2 |y|^2.  No convergence test,
 * polish or validity test runs.  The gradient of
 *   sum over paths of dX . X + dL L   (X, L at the last iterate)
 * with respect to TX, RX and the object vertices is then formed in reverse
 * mode through all steps (the line-search rounds and the inverse-Hessian
 * updates included), one path per GPU thread, with each step's iterate and
 * inverse Hessian kept on a context-owned device tape of steps (2n + 2n(2n+1)/2)
 * floats per resident thread (at most 16 GiB; fewer resident threads when it is
 * short).  steps in [0, 4096], fp_iters in [1, 64] (FPT_EINVAL otherwise).
 * dX [N][n_max][3], dL [N] device or NULL (zero).  T_out [N][n_max][2] (the last
 * iterate) and status_out [N] (REPEAT / INVALID as in fpt_solve, NONFINITE when
 * the path's gradient is not finite: it is then left out of the sums) are
 * optional.  Gradient outputs as in fpt_backward. */
fpt_status fpt_backward_unrolled(fpt_ctx* ctx, const fpt_scene* scene, const fpt_batch* batch, int32_t steps,
                                 int32_t fp_iters, const float* dX, const float* dL, float* T_out, uint8_t* status_out,
                                 float* g_tx, float* g_rx, float* g_vertices);

/* fpt_backward without any device allocation, for callers that cannot
 * allocate: for example a host application whose GPU memory is entirely
 * reserved by another allocator (a framework's caching pool), or a latency-
 * critical loop that forbids cudaMalloc / cudaFree because they can
 * synchronise the device.  The paper has no counterpart; arguments, outputs
 * and results are those of fpt_backward.
 * Its scratch (FP64 gradient sums, the list and counter of the FP64 pass) is
 * one fixed array inside the library, about 4.5 MB on every GPU that loads
 * the library, held until the process exits.  Limits: 9 n_obj + 3 (n_tx +
 * n_rx) <= 65536 and at most 2^20 paths of any one order in the batch;
 * larger inputs return FPT_EINVAL with a message.  Seeded and explicit
 * batches must already be bucketed (any earlier fpt_solve or fpt_backward
 * on the batch does that).
 * The array's device address is looked up, with the device current, when a
 * context is created on that device (fpt_create) and cached; a device reset
 * (cudaDeviceReset) can move the array, so create a new context after one
 * before calling this again.  Every call reuses the same array and clears the
 * sums it needs; calls that overlap on the GPU (different streams or
 * contexts, same device) race on it and must be serialised by the caller. */
fpt_status fpt_backward_noalloc(fpt_ctx* ctx, const fpt_scene* scene, const fpt_batch* batch, const float* T,
                                const uint8_t* status, const float* dX, const float* dL, uint8_t dL_status_mask,
                                float* g_tx, float* g_rx, float* g_vertices);

/* Paths left out of the sums of the most recent fpt_backward, fpt_solve_grad
 * or fpt_backward_noalloc call on this context because their Hessian failed
 * the pivot test in FP32 and again in FP64 (singular: such a path has no
 * well-defined implicit gradient and contributes nothing).  Synchronises the
 * context's stream. */
fpt_status fpt_backward_dropped(fpt_ctx* ctx, uint64_t* count);

/* Number of paths whose status has all bits of `mask` set (device status
 * [n]; result written to *count on the host after a stream sync). */
fpt_status fpt_count_status(fpt_ctx* ctx, const uint8_t* status, uint64_t n, uint8_t mask, uint64_t* count);

/* ---------------------------------------------------------------------------
 * Learned warm start (the paper names better initial candidates as future work,
 * Sec. V).  A network maps the geometry of a sequence to starting parameters:
 * features (64, BF16) -> 256 -> 256 -> 256 (GELU, tanh form) -> 8 outputs (t of the first
 * four interactions), BF16 weights, FP32 accumulation on the tensor cores,
 * activations rounded to BF16 between layers.  Features of a path of order n,
 * with o = (TX + RX) / 2 and S the model's length scale (metres):
 *   f[0..2] = (TX - o)/S, f[3..5] = (RX - o)/S, and for slot s < min(n, 4) at
 *   6 + 11 s: [1, is_edge, tau_TX (2), tau_RX (2), d_TX, d_RX, |a1|/S, w (2)]
 *   where tau_P are the parameters of the orthogonal projection of P onto the
 *   object's affine hull (edge: tau_2 = 0), d_P its distance to the hull / S,
 *   and w = (d_RX tau_TX + d_TX tau_RX) / (d_TX + d_RX); all else 0.  These are
 *   TX, RX and the object's origin and basis, expressed in the object's frame.
 * Parameters (FP32, FPT_MLP_NPARAMS floats, in this order): W1 [256][64], b1
 * [256], W2 [256][256], b2 [256], W3 [256][256], b3 [256], W4 [16][256], b4
 * [16] (rows / entries 8..15 of the last layer are zero).
 * Training loss of a batch of B samples with targets t* [B][8] and per-slot
 * Gram matrices G [B][4][3] = (a1.a1, a1.a2, a2.a2) / S^2 (zero for unused
 * slots):  (1/B) sum_b sum_s (y_s - t*_s)^T G_s (y_s - t*_s), the squared
 * world-space error of the predicted points in units of S.
 * ------------------------------------------------------------------------- */
#define FPT_MLP_FEATURES 64
#define FPT_MLP_OUT 16
#define FPT_MLP_NPARAMS 152336
typedef struct fpt_mlp fpt_mlp;

/* New network with seeded uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights
 * and zero biases (splitmix64 stream of `seed`), length scale S > 0 metres. */
fpt_status fpt_mlp_create(fpt_ctx* ctx, uint64_t seed, float length_scale, fpt_mlp** out);
void fpt_mlp_free(fpt_mlp* mlp);
/* Copy the FP32 parameters to / from host memory [FPT_MLP_NPARAMS]; set also
 * resets the Adam state.  Synchronous. */
fpt_status fpt_mlp_get_params(const fpt_mlp* mlp, float* host_params);
fpt_status fpt_mlp_set_params(fpt_mlp* mlp, const float* host_params);
/* Save / load parameters, Adam moments, step count and length scale to a
 * versioned binary file (host path).  FPT_EINVAL on a bad file. */
fpt_status fpt_mlp_save(const fpt_mlp* mlp, const char* path);
fpt_status fpt_mlp_load(fpt_ctx* ctx, const char* path, fpt_mlp** out);
/* Features of every path of a batch: device bf16 output [N][64]; G_out
 * (device float [N][4][3], may be NULL) receives the loss's Gram matrices. */
fpt_status fpt_mlp_features(fpt_ctx* ctx, const fpt_mlp* mlp, const fpt_scene* scene, const fpt_batch* batch,
                            void* X_out, float* G_out);
/* Forward pass: X device bf16 [B][64] -> Y device float [B][16]. */
fpt_status fpt_mlp_forward(fpt_ctx* ctx, fpt_mlp* mlp, const void* X, uint64_t B, float* Y);
/* Loss and its gradient with respect to the parameters (device float
 * [FPT_MLP_NPARAMS], overwritten) for X [B][64], targets T [B][8] and Gram
 * matrices G [B][4][3] (device); *loss receives the loss on the host
 * (synchronises). */
fpt_status fpt_mlp_loss_grad(fpt_ctx* ctx, fpt_mlp* mlp, const void* X, const float* T, const float* G, uint64_t B,
                             float* loss, float* grad_out);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * loss of this batch; *loss (host, may be NULL) receives the batch loss. */
fpt_status fpt_mlp_train_step(fpt_ctx* ctx, fpt_mlp* mlp, const void* X, const float* T, const float* G, uint64_t B,
                              float lr, float* loss);
/* Training schedule of fpt_mlp_train. */
typedef struct {
  int32_t epochs;     /* passes over the samples (>= 1) */
  int32_t batch;      /* samples per Adam step (>= 128); the last partial batch of an epoch is left out */
  float lr;           /* learning rate of the first epoch (> 0) */
  float lr_decay;     /* factor applied to the learning rate after every epoch (> 0; 0.5 halves it) */
  uint64_t seed;      /* seed of the sample order: every epoch visits the samples in a new pseudo-random order */
  int32_t reserved[4]; /* must be zero */
} fpt_train_params;
/* Train the network on n samples (device arrays as for fpt_mlp_loss_grad: X
 * bf16 [n][64], targets T [n][8], Gram matrices G [n][4][3]): for every epoch
 * a seeded permutation of the samples (a Feistel-network permutation drawn
 * from seed and epoch, evaluated on the device), then floor(n / batch) Adam
 * steps on consecutive slices of it; everything runs on the context's stream
 * without waiting for the device.  loss_per_epoch (host [epochs], may be
 * NULL) receives each epoch's mean batch loss (the call then synchronises
 * once at its end).  FPT_EINVAL on bad parameters or n < batch. */
fpt_status fpt_mlp_train(fpt_ctx* ctx, fpt_mlp* mlp, const void* X, const float* T, const float* G, uint64_t n,
                         const fpt_train_params* params, float* loss_per_epoch);
/* The learned start of every path of a batch: T_out [N][n_max][2] (device)
 * receives the starting parameters fpt_solve uses with init_mode = 1 and this
 * network (the first min(n, 4) interactions from the network, an edge's
 * second parameter, later interactions and non-finite outputs at 1/2, unused
 * slots 0), computed by the fused tensor-core inference kernel. */
fpt_status fpt_mlp_infer(fpt_ctx* ctx, fpt_mlp* mlp, const fpt_scene* scene, const fpt_batch* batch, float* T_out);
/* Network used by fpt_solve when init_mode = 1 (NULL detaches).  The network's
 * prediction seeds the first min(n, 4) interactions of each path; further
 * interactions, edges' second coordinate and non-finite predictions use the
 * plain start t = 1/2. */
fpt_status fpt_set_init_mlp(fpt_ctx* ctx, fpt_mlp* mlp);

/* Tensor-core GEMM used by the warm-start network's layers (tcgen05, BF16 in,
 * FP32 accumulation in tensor memory): C[M][N] = A[M][K] W[N][K]^T (+ bias[N]).
 * A, W: device bf16, row-major; bias: device float [N] or NULL; C: device
 * float [M][N].  1 <= N <= 256, M, K >= 1.  FPT_EDEVICE (via fpt_sync) if the
 * tensor core does not complete within its bounded wait. */
fpt_status fpt_tc_gemm_bf16(fpt_ctx* ctx, int32_t M, int32_t N, int32_t K, const void* A, const void* W,
                            const float* bias, float* C);

/* Check of the bounded waits.  Every tensor-core kernel (the GEMMs and the
 * fused inference) gives up an mbarrier wait after 1 s of the GPU's global
 * timer, sets the context's device error word and returns, so that a TMA copy
 * or an MMA that never completes shows up as FPT_EDEVICE from the next
 * fpt_sync (which clears the word) instead of a hung stream.  This call
 * launches one CTA that waits, with the same helper and a limit of limit_us
 * microseconds (1 <= limit_us <= 10^6, else FPT_EINVAL), on an mbarrier that
 * receives its one expected arrival only when arrive != 0.  With arrive == 0
 * the wait runs out and the following fpt_sync returns FPT_EDEVICE; with
 * arrive != 0 it completes at once and the error word is left alone.
 * elapsed_ns (host, optional) receives the wait's duration in nanoseconds;
 * passing it makes the call synchronise the stream. */
fpt_status fpt_check_bounded_wait(fpt_ctx* ctx, uint32_t limit_us, int arrive, uint64_t* elapsed_ns);

/* Kernel timing.  While enabled, the kernels of each class that one call
 * launches are bracketed by CUDA events on the context's stream, and
 * fpt_profile_read() returns, per kernel class, the summed device time in
 * milliseconds and the number of kernels launched (it synchronises the
 * stream; reset != 0 clears the sums). */
enum { FPT_K_BFGS = 0, FPT_K_POLISH = 1, FPT_K_BACKWARD = 2, FPT_K_OTHER = 3, FPT_K_MLP = 4, FPT_K_COUNT = 5 };
fpt_status fpt_profile_enable(fpt_ctx* ctx, int on);
fpt_status fpt_profile_read(fpt_ctx* ctx, double* ms, uint64_t* launches, int reset);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif
#endif /* FPT_H */
