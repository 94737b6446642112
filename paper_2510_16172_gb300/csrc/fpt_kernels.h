// fpt_kernels.h -- launch wrappers of the CUDA kernels (host side).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fpt_device.cuh"

namespace fpt {

constexpr int kThreads = 128;  // threads per CTA for all path kernels
// Minimum CTAs per SM for the launch bounds of the per-order kernels that spill at orders above
// kMaxBfgsOrder (unrolled AD, FP64 polish, FP64 adjoint): 1 there, so that ptxas gives them the
// full 255 registers instead of settling on a smaller budget and spilling more; unspecified (0)
// at the register-resident orders.
template <int N>
constexpr int kLongOrderMinBlocks = N > kMaxBfgsOrder ? 1 : 0;
constexpr size_t kMaxSmemBytes = 200 * 1024;  // dynamic shared memory a path kernel may request

// Kernels launched by the calling thread; the API's profiler reads the
// difference around each call.
extern thread_local uint64_t tl_kernel_launches;
inline void count_launch() { ++tl_kernel_launches; }

constexpr int kMaxChunk = 256;  // most paths a warp of the refill kernel claims at a time
constexpr int kKinkMinIters = 4;  // BFGS steps before the kink stop applies

struct SolveCfg {
  int max_iters;    // BFGS step cap
  int fp_iters;     // Eq. 6 rounds per step
  int fixed_iters;  // 1: run every path for max_iters steps
  float tol2;       // (world-space step tolerance)^2
  float stop2;      // a segment shorter than sqrt(stop2) before convergence stops BFGS: DEGENERATE (a kink)
  int refill;       // lane refill threshold (free lanes before a warp takes new paths); 0 = one path per lane per tile
  int init_from_T;  // 1: start from the parameters already in T (learned start); 0: t = 1/2
  int chunk;        // paths a warp claims at a time (refill kernel; set per launch)
};

enum PolishMode { POLISH_SOLVE = 0, POLISH_VALIDITY = 1 };

struct PolishCfg {
  int mode;          // PolishMode
  int steps;         // Newton steps applied (solve mode)
  float solved_tol;  // residual bound for ST_SOLVED
  float deg_tol;     // shortest segment of a regular solution
  float cond_fp64;   // pivot ratio that triggers the FP64 Hessian solve
  int fp64;          // 1: FP64 gradients in the polish (validation); 0: double-float
  float radius;      // adaptive polish: largest first residual from which the Newton steps are taken (0 = any)
};

struct BackwardCfg {
  float cond_fp64;
  float deg_tol;
  int acc_in_smem;   // accumulate per CTA in shared memory before the FP64 global sum
  int flush_tiles;   // flush the shared accumulators every this many CTA tiles
  uint8_t dl_mask;   // with no dL array: dL = 1 where (status & dl_mask) == dl_mask (0 = no length term)
  // scratch for a list of the paths with a cotangent (room for the slice, and its counter): without dX,
  // a select pass lists them first so the adjoint's warps run full (nullptr: every path is visited)
  uint32_t* sel = nullptr;
  unsigned* sel_count = nullptr;
  // counter of the paths whose Hessian also fails the FP64 pivot test (left out of the sums; nullptr: not counted)
  unsigned* dropped = nullptr;
};

// Per-order launches (n = 1..kMaxOrder).  `list` = nullptr for exhaustive batches.
// BFGS: pattern < 0 runs the unified kernel over every sequence of order n;
// pattern = Q in [0, 2^n) runs the kernel of that interaction-type pattern
// over a slice holding only sequences of pattern Q.
cudaError_t launch_bfgs(int n, int pattern, const SceneDev& S, const BatchDev& B, const SolveCfg& cfg, uint64_t n_local,
                        const PathRec* list, float* T, uint8_t* status, uint8_t* iters, cudaStream_t stream,
                        int n_sm, unsigned long long* work);
// The implicit backward fused into the polish (fpt_solve_grad): cotangents
// known at solve time, sums into FP64 accumulators.
struct GradCfg {
  const float* dX;          // [N][n_max][3] or nullptr
  const float* dL;          // [N] or nullptr
  uint8_t dl_mask;          // with no dL array: dL = 1 where (status & dl_mask) == dl_mask (0 = no length term)
  float cond_adj;           // pivot test of the adjoint solve
  float deg_tol;
  double* gacc;             // 9 n_obj + 3 (n_tx + n_rx) FP64 accumulators
  uint32_t* rescue_list;    // paths whose adjoint runs in the FP64 pass (n_local entries)
  unsigned* rescue_count;
  int flush_tiles;          // flush the shared accumulators every this many CTA tiles
  int acc_in_smem = 1;      // 0: every path's terms go straight into the FP64 accumulators
  unsigned* dropped = nullptr;  // as BackwardCfg::dropped
};

// Double-float polish, then an FP64 pass over the paths whose FP32 pivots failed
// (rescue_list: scratch of n_local entries; rescue_count: one device counter).
// With grad != nullptr the same kernel also forms each path's VJP from its
// polished state and sums it, and an FP64 adjoint pass follows.  With a
// step_list (n_local entries) and step_delta (n_local x 2n floats) the
// polish is adaptive: paths whose residual already meets solved_tol at the
// solver's point keep it, the others are listed with their first Newton step
// and finish in a second pass.
cudaError_t launch_polish(int n, const SceneDev& S, const BatchDev& B, const PolishCfg& cfg, uint64_t n_local,
                          const PathRec* list, float* T, float* X, float* L, uint8_t* status, float* rho,
                          uint8_t* mask, float* bdist, cudaStream_t stream, int n_sm, uint32_t* rescue_list,
                          unsigned* rescue_count, const GradCfg* grad = nullptr, uint32_t* step_list = nullptr,
                          unsigned* step_count = nullptr, float* step_delta = nullptr);
// Adjoint + sums, then an FP64 pass over the paths whose FP32 pivots failed.
cudaError_t launch_backward(int n, const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg, uint64_t n_local,
                            const PathRec* list, const float* T, const uint8_t* status, const float* dX,
                            const float* dL, double* gacc, cudaStream_t stream, int n_sm, uint32_t* rescue_list,
                            unsigned* rescue_count);
// Backward with its scratch in a fixed device array (no allocation): limits below.
constexpr int kNoAllocMaxAcc = 1 << 16;      // 9 n_obj + 3 (n_tx + n_rx) FP64 accumulators
constexpr int kNoAllocMaxSlice = 1 << 20;    // paths of one order in the batch
constexpr int kNoAllocMaxDevices = 64;
// Look up (again) the device address of the fixed scratch array on `device` (current).
cudaError_t noalloc_lookup(int device);
cudaError_t launch_backward_noalloc(int device, const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg,
                                    const PathRec* const* lists, const uint64_t* counts, const float* T,
                                    const uint8_t* status, const float* dX, const float* dL, float* g_tx, float* g_rx,
                                    float* g_vertices, cudaStream_t stream, int n_sm);
// FP64 adjoint over a rescue list (paths of one order slice).
cudaError_t launch_backward_rescue(int n, const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg,
                                   uint64_t n_local, const PathRec* list, const float* T, const uint8_t* status,
                                   const float* dX, const float* dL, double* gacc, cudaStream_t stream, int n_sm,
                                   const uint32_t* rescue_list, const unsigned* rescue_count);
// Gradient by reverse-mode differentiation through `steps` unified solver steps
// (Sec. IV-B's comparison): one path per thread, its per-step state on a tape
// of at most tape_floats floats (fewer resident threads when it is short).
constexpr int kUnrolledMaxRounds = 64;
constexpr int kUnrolledMaxSteps = 4096;
constexpr size_t kUnrolledMaxTape = size_t(16) << 30;  // bytes
size_t unrolled_tape_floats(int n, int steps, uint64_t threads);
cudaError_t launch_unrolled(int n, const SceneDev& S, const BatchDev& B, int steps, int rounds, uint64_t n_local,
                            const PathRec* list, const float* dX, const float* dL, double* gacc, float* tape,
                            size_t tape_floats, float* T_out, uint8_t* status, cudaStream_t stream, int n_sm);
// Obstruction test (k_occlusion.cu): kOcc floats per planar object: origin b (3,
// centred), unit normal (3), dual basis d1 (3) and d2 (3), object id (int bits).
constexpr int kOcc = 13;
// With status and a non-zero mask the selected paths are listed first (sel: n_local uint32, sel_count: one
// counter) and the others get a zero mask.
cudaError_t launch_occlusion(const SceneDev& S, const BatchDev& B, int n, const PathRec* list, uint64_t n_local,
                             const float* T, const uint8_t* status, uint8_t mask, const float* occ, int n_occ,
                             float tol, uint16_t* blocked, uint32_t* sel, unsigned* sel_count, cudaStream_t stream,
                             int n_sm);
// Records from caller-owned device FP32 coordinates (k_scene.cu): endpoints p [n][3] -> kEnd32 FP32 and
// 3 FP64 values each; objects verts [n_obj][3][3] -> FP32, low-part, FP64, aux and occluder records.
// Non-finite or degenerate input sets ERR_BAD_GEOMETRY in *err.
cudaError_t launch_endpoint_records(const float* p, int n, const double* centre, float* rec32, double* rec64,
                                    int* err, cudaStream_t stream);
cudaError_t launch_object_records(int n_obj, const uint8_t* types, const int32_t* occ_slot, const float* verts,
                                  const double* centre, float* rec32, float* reclo, double* rec64, float* aux,
                                  float* occ, int* err, cudaStream_t stream);
cudaError_t launch_backward_finalize(const SceneDev& S, const uint8_t* types, const double* gacc, float* g_tx,
                                     float* g_rx, float* g_vertices, cudaStream_t stream);

// Batch utilities.
cudaError_t launch_enumerate(const BatchDev& B, int32_t* ids, uint8_t* order, int32_t* tx_idx, int32_t* rx_idx,
                             cudaStream_t stream, int n_sm);
// Bucketing of seeded / explicit batches by pattern_key(order, pattern): counts[kPatternKeys].
cudaError_t launch_pattern_histogram(const SceneDev& S, const BatchDev& B, unsigned long long* counts,
                                     cudaStream_t stream, int n_sm);
cudaError_t launch_pattern_scatter(const SceneDev& S, const BatchDev& B, unsigned long long* cursors, PathRec* lists,
                                   cudaStream_t stream, int n_sm);
cudaError_t launch_count_status(const uint8_t* status, uint64_t n, uint8_t mask, unsigned long long* out,
                                cudaStream_t stream, int n_sm);

}  // namespace fpt
