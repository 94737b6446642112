// fpt_api.cu -- host implementation of the C ABI declared in include/fpt.h.
//
// Owns contexts (device, stream, error word, workspace), scenes (object
// records built in FP64 on the host, recentred, split into FP32 hi/lo parts
// and uploaded) and batches (candidate-sequence descriptions; seeded and
// explicit batches are bucketed by order on the device once, so that every
// solver launch is specialised to one order).
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "fpt.h"
#include "fpt_kernels.h"
#include "mlp.h"

using namespace fpt;

// Streams over which the BFGS pattern launches of one order are spread (a
// build-time tuning constant: more streams overlap the launches' tails, but
// co-resident kernels share each SM's instruction cache).
#ifndef FPT_SIDE_STREAMS
#define FPT_SIDE_STREAMS 4
#endif

struct fpt_ctx {
  int device = 0;
  int n_sm = 0;
  cudaStream_t stream = nullptr;
  int* d_err = nullptr;                    // device error word
  double* d_gacc = nullptr;                // backward accumulators (FP64)
  size_t gacc_cap = 0;
  float* d_tape = nullptr;                 // per-step state of fpt_backward_unrolled
  size_t tape_cap = 0;                     // floats
  unsigned long long* d_count = nullptr;   // counters for reductions
  unsigned long long* d_work = nullptr;    // work counters of the lane-refill solver (one per concurrent launch)
  static constexpr int kSide = FPT_SIDE_STREAMS;  // streams for the independent pattern launches of one order
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kSide] = {};
  uint32_t* d_rescue = nullptr;            // path lists: FP64 polish, FP64 adjoint, second polish pass
  float* d_step = nullptr;                 // first Newton steps of the second polish pass's paths
  size_t rescue_cap = 0;
  size_t step_cap = 0;                     // floats of d_step
  unsigned* d_rescue_n = nullptr;          // counters: FP64 polish, FP64 adjoint, selected paths, dropped paths
  fpt_mlp* init_mlp = nullptr;             // network for init_mode = 1
  int acc_flush_tiles = 64;                // backward sums: CTA tiles between flushes of the FP32 partial sums
  int acc_smem = 1;                        // backward sums: 1 = FP32 partial sums per CTA, 0 = straight to FP64
  char msg[512] = "ok";
  // kernel timing
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double prof_ms[FPT_K_COUNT] = {0, 0, 0, 0, 0};
  uint64_t prof_kernels[FPT_K_COUNT] = {0, 0, 0, 0, 0};
};

// Event pair around the launches of one call when timing is on; counts the kernels launched in between.
struct ProfScope {
  fpt_ctx* ctx;
  int cls;
  uint64_t k0 = 0;
  cudaEvent_t a = nullptr, b = nullptr;
  static cudaEvent_t take(fpt_ctx* c) {
    cudaEvent_t e = nullptr;
    if (!c->ev_pool.empty()) {
      e = c->ev_pool.back();
      c->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
    }
    return e;
  }
  ProfScope(fpt_ctx* c, int k) : ctx(c), cls(k) {
    if (!ctx->prof) return;
    k0 = tl_kernel_launches;
    a = take(ctx);
    b = take(ctx);
    if (a) cudaEventRecord(a, ctx->stream);
  }
  ~ProfScope() {
    if (!ctx->prof) return;
    ctx->prof_kernels[cls] += tl_kernel_launches - k0;
    if (!a || !b) return;
    cudaEventRecord(b, ctx->stream);
    ctx->ev_pending.push_back({cls, {a, b}});
  }
};

struct fpt_scene {
  fpt_ctx* ctx = nullptr;
  int n_obj = 0;
  std::vector<uint8_t> types;
  double centre[3] = {0, 0, 0};
  float* d_rec32 = nullptr;
  double* d_rec64 = nullptr;
  float* d_aux = nullptr;
  float* d_reclo = nullptr;
  int n_tx = 0, n_rx = 0;
  float* d_tx32 = nullptr;
  float* d_rx32 = nullptr;
  double* d_tx64 = nullptr;
  double* d_rx64 = nullptr;
  float* d_occ = nullptr;  // planar objects as occluders (kOcc floats each)
  int n_occ = 0;
  uint8_t* d_types = nullptr;      // object types and occluder slots (-1: edge), for records built on the device
  int32_t* d_occ_slot = nullptr;
  int tx_cap = 0, rx_cap = 0;      // endpoints the device buffers hold
  std::vector<int32_t> h_occ_slot;
  // host sources of the asynchronous uploads, kept until the device buffers are freed (cudaFree
  // waits for the device, so no copy from them is still pending when they go)
  std::vector<float> h_rec32, h_aux, h_reclo, h_occ, h_tx32, h_rx32;
  std::vector<double> h_rec64, h_tx64, h_rx64;
};

struct fpt_batch {
  fpt_ctx* ctx = nullptr;
  BatchDev dev{};
  int32_t* d_alphabet = nullptr;
  int32_t* d_type_pos = nullptr;  // alphabet positions of the reflectors, then of the edges
  std::vector<uint8_t> types;     // object types of the scene the batch was built for
  std::vector<int32_t> h_alphabet, h_type_pos;  // host sources of the uploads (as in fpt_scene)
  // (order, pattern) buckets of seeded / explicit batches (built on first use)
  bool bucketed = false;
  PathRec* d_lists = nullptr;
  uint64_t count[kPatternKeys] = {0};
  uint64_t start[kPatternKeys] = {0};
  // per order: the buckets too small for a pattern launch sit together at the end of the order's range
  uint64_t small_start[kMaxOrder + 1] = {0};
  uint64_t small_count[kMaxOrder + 1] = {0};
};

// Smallest bucket worth its own pattern launch: about four paths per resident lane.
static uint64_t min_pattern_bucket(const fpt_ctx* ctx) { return (uint64_t)ctx->n_sm * 4 * 128 * 4; }

static fpt_status fail(fpt_ctx* ctx, fpt_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->msg, sizeof(ctx->msg), fmt, ap);
    va_end(ap);
  }
  return st;
}

#define CUDA_OR_FAIL(ctx, call)                                                                    \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail((ctx), FPT_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

struct fpt_mlp {
  fpt_ctx* ctx = nullptr;
  float scale = 1.f;
  uint64_t seed = 0;
  int64_t step = 0;
  float* d_w = nullptr;          // FP32 master parameters
  float* d_m = nullptr;          // Adam moments
  float* d_v = nullptr;
  float* d_g = nullptr;          // gradient
  __nv_bfloat16* d_wb = nullptr;  // BF16 copy used by the tensor cores
  __nv_bfloat16* d_wt = nullptr;  // BF16 weights pre-tiled for the fused inference kernel
  bool wt_stale = true;
  __nv_bfloat16* d_wtT = nullptr;  // BF16 W^T of layers 2-4 (the backward's dH = dZ W), refreshed when stale
  bool wtT_stale = true;
  float* d_loss = nullptr;
  // fpt_mlp_train: one shuffled mini-batch and the per-epoch mean losses
  __nv_bfloat16* d_Xb = nullptr;
  float *d_Tb = nullptr, *d_Gb = nullptr, *d_hist = nullptr;
  uint64_t train_cap = 0;
  bool xt_ready = false;  // d_Xt already holds the transpose of d_Xb (written by the shuffle gather)
  size_t hist_cap = 0;
  // activations / gradients for a batch of up to cap rows
  uint64_t cap = 0;
  __nv_bfloat16 *d_H1 = nullptr, *d_H2 = nullptr, *d_H3 = nullptr, *d_dZa = nullptr, *d_dZb = nullptr,
                *d_dYb = nullptr, *d_X = nullptr;
  // transposed copies for the weight gradients dW = dZ^T act (K-major operands): act^T, dZ^T, dY^T
  __nv_bfloat16 *d_Ht1 = nullptr, *d_Ht2 = nullptr, *d_Ht3 = nullptr, *d_Xt = nullptr, *d_dZta = nullptr,
                *d_dZtb = nullptr, *d_dYt = nullptr;
  float *d_Z1 = nullptr, *d_Z2 = nullptr, *d_Z3 = nullptr, *d_Y = nullptr, *d_dY = nullptr;
};

static fpt_status mlp_ensure_ws(fpt_ctx* ctx, fpt_mlp* m, uint64_t B, bool train);
static fpt_status mlp_forward_impl(fpt_ctx* ctx, fpt_mlp* m, const __nv_bfloat16* X, uint64_t B, float* Y,
                                   bool train);

static SceneDev scene_dev(const fpt_scene* s) {
  SceneDev d{};
  d.n_obj = s->n_obj;
  d.rec32 = s->d_rec32;
  d.rec64 = s->d_rec64;
  d.aux = s->d_aux;
  d.n_tx = s->n_tx;
  d.n_rx = s->n_rx;
  d.tx32 = s->d_tx32;
  d.rx32 = s->d_rx32;
  d.tx64 = s->d_tx64;
  d.rx64 = s->d_rx64;
  d.reclo = s->d_reclo;
  for (int c = 0; c < 3; ++c) {
    d.centre[c] = s->centre[c];
    d.centre_hi[c] = (float)s->centre[c];
    d.centre_lo[c] = (float)(s->centre[c] - (double)d.centre_hi[c]);
  }
  return d;
}

extern "C" {

void fpt_default_params(fpt_solve_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->max_iters = 64;
  p->fp_iters = 1;
  p->polish = 1;
  p->fixed_iters = 0;
  p->tol_step = 1e-4f;
  p->solved_tol = 1e-5f;
  p->deg_tol = 1e-3f;
  p->cond_fp64 = 1e-4f;
  p->init_mode = 0;
  p->polish_fp64 = 0;
  p->refill = 8;
  p->specialize = 1;
  p->polish_radius = 0.1f;
}

fpt_status fpt_create(fpt_ctx** out, int device, void* cuda_stream) {
  if (!out) return FPT_EINVAL;
  *out = nullptr;
  fpt_ctx* ctx = new (std::nothrow) fpt_ctx();
  if (!ctx) return FPT_ENOMEM;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
  static_assert(kPatternKeys <= 128, "pattern counters");
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_count, 128 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_work, 64 * sizeof(unsigned long long));
  for (int k = 0; k < fpt_ctx::kSide && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join_ev[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_rescue_n, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_rescue_n, 0, 4 * sizeof(unsigned));
  // the fixed array of fpt_backward_noalloc: its address on this device, looked up again for every context
  if (e == cudaSuccess) e = noalloc_lookup(device);
  if (e != cudaSuccess) {
    fpt_destroy(ctx);
    return FPT_ECUDA;
  }
  *out = ctx;
  return FPT_OK;
}

void fpt_destroy(fpt_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (auto& p : ctx->ev_pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_gacc);
  cudaFree(ctx->d_count);
  cudaFree(ctx->d_work);
  for (int k = 0; k < fpt_ctx::kSide; ++k) {
    if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
    if (ctx->join_ev[k]) cudaEventDestroy(ctx->join_ev[k]);
  }
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  cudaFree(ctx->d_rescue);
  cudaFree(ctx->d_step);
  cudaFree(ctx->d_rescue_n);
  cudaFree(ctx->d_tape);
  delete ctx;
}

fpt_status fpt_set_stream(fpt_ctx* ctx, void* cuda_stream) {
  if (!ctx) return FPT_EINVAL;
  // no synchronisation here (the call is legal inside a stream capture): the caller orders the old
  // stream's work, uploads included, before the new stream's
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return FPT_OK;
}

const char* fpt_last_error(const fpt_ctx* ctx) { return ctx ? ctx->msg : "null context"; }

fpt_status fpt_set_accumulation(fpt_ctx* ctx, int32_t flush_tiles, int32_t smem) {
  if (!ctx) return FPT_EINVAL;
  if (flush_tiles < 1 || (smem != 0 && smem != 1))
    return fail(ctx, FPT_EINVAL, "fpt_set_accumulation: flush_tiles must be >= 1 and smem 0 or 1");
  ctx->acc_flush_tiles = flush_tiles;
  ctx->acc_smem = smem;
  return FPT_OK;
}

fpt_status fpt_sync(fpt_ctx* ctx) {
  if (!ctx) return FPT_EINVAL;
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  int err = 0;
  CUDA_OR_FAIL(ctx, cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    CUDA_OR_FAIL(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
    return fail(ctx, FPT_EDEVICE, "device error code %d", err);
  }
  return FPT_OK;
}

// ---------------------------------------------------------------------------
// scene
// ---------------------------------------------------------------------------
static void split(double x, float& hi, float& lo) {
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

fpt_status fpt_scene_upload(fpt_ctx* ctx, const uint8_t* types, const double* verts, int32_t n_obj,
                            fpt_scene** out) {
  if (!ctx || !types || !verts || !out) return fail(ctx, FPT_EINVAL, "null argument");
  *out = nullptr;
  if (n_obj < 1 || n_obj > 65535) return fail(ctx, FPT_EINVAL, "n_obj %d outside [1, 65535]", n_obj);
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = 0; k < n_obj; ++k) {
    if (types[k] != FPT_QUAD && types[k] != FPT_EDGE) return fail(ctx, FPT_EINVAL, "object %d: bad type", k);
    const int nv = types[k] == FPT_QUAD ? 3 : 2;
    for (int v = 0; v < nv; ++v)
      for (int c = 0; c < 3; ++c) {
        double x = verts[9 * k + 3 * v + c];
        if (!std::isfinite(x)) return fail(ctx, FPT_EINVAL, "object %d: non-finite vertex", k);
        lo[c] = x < lo[c] ? x : lo[c];
        hi[c] = x > hi[c] ? x : hi[c];
      }
  }
  fpt_scene* s = new (std::nothrow) fpt_scene();
  if (!s) return FPT_ENOMEM;
  s->ctx = ctx;
  s->n_obj = n_obj;
  s->types.assign(types, types + n_obj);
  for (int c = 0; c < 3; ++c) s->centre[c] = 0.5 * (lo[c] + hi[c]);
  std::vector<float>& rec32 = s->h_rec32;
  std::vector<float>& aux = s->h_aux;
  std::vector<float>& reclo = s->h_reclo;
  std::vector<double>& rec64 = s->h_rec64;
  rec32.assign((size_t)n_obj * kRec32, 0.f);
  aux.assign((size_t)n_obj * kAux, 0.f);
  reclo.assign((size_t)n_obj * kRecLo, 0.f);
  rec64.assign((size_t)n_obj * kRec64, 0.0);
  for (int k = 0; k < n_obj; ++k) {
    const double* v = verts + 9 * k;
    double b[3], a1[3], a2[3];
    for (int c = 0; c < 3; ++c) {
      b[c] = v[c] - s->centre[c];
      a1[c] = v[3 + c] - v[c];
      a2[c] = types[k] == FPT_QUAD ? v[6 + c] - v[c] : 0.0;
    }
    double n1 = std::sqrt(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
    double n2 = std::sqrt(a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2]);
    double cx = a1[1] * a2[2] - a1[2] * a2[1], cy = a1[2] * a2[0] - a1[0] * a2[2], cz = a1[0] * a2[1] - a1[1] * a2[0];
    double area = std::sqrt(cx * cx + cy * cy + cz * cz);
    if (types[k] == FPT_QUAD && area < 1e-9) {
      delete s;
      return fail(ctx, FPT_EINVAL, "object %d: zero-area plane", k);
    }
    if (types[k] == FPT_EDGE && n1 < 1e-9) {
      delete s;
      return fail(ctx, FPT_EINVAL, "object %d: zero-length edge", k);
    }
    for (int c = 0; c < 3; ++c) {
      rec64[kRec64 * k + c] = b[c];
      rec64[kRec64 * k + 3 + c] = a1[c];
      rec64[kRec64 * k + 6 + c] = a2[c];
      split(b[c], rec32[kRec32 * k + c], rec32[kRec32 * k + 3 + c]);
      split(a1[c], rec32[kRec32 * k + 6 + c], reclo[kRecLo * k + c]);
      split(a2[c], rec32[kRec32 * k + 9 + c], reclo[kRecLo * k + 3 + c]);
    }
    // side heights for the boundary distance: distance between the sides t1 = 0, 1 is area/|a2|
    aux[kAux * k + 0] = types[k] == FPT_QUAD ? (float)(area / n2) : (float)n1;
    aux[kAux * k + 1] = types[k] == FPT_QUAD ? (float)(area / n1) : 0.f;
    aux[kAux * k + 2] = types[k] == FPT_EDGE ? 1.f : 0.f;
    aux[kAux * k + 3] = 0.f;
  }
  // occluder records of the planar objects: centred origin, unit normal, dual basis of (a1, a2)
  std::vector<float>& occ = s->h_occ;
  for (int k = 0; k < n_obj; ++k) {
    if (types[k] != FPT_QUAD) continue;
    const double* v = verts + 9 * k;
    double b[3], a1[3], a2[3];
    for (int c = 0; c < 3; ++c) {
      b[c] = v[c] - s->centre[c];
      a1[c] = v[3 + c] - v[c];
      a2[c] = v[6 + c] - v[c];
    }
    double nv[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
    const double nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    const double g11 = a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2];
    const double g12 = a1[0] * a2[0] + a1[1] * a2[1] + a1[2] * a2[2];
    const double g22 = a2[0] * a2[0] + a2[1] * a2[1] + a2[2] * a2[2];
    const double det = g11 * g22 - g12 * g12;
    for (int c = 0; c < 3; ++c) occ.push_back((float)b[c]);
    for (int c = 0; c < 3; ++c) occ.push_back((float)(nv[c] / nn));
    for (int c = 0; c < 3; ++c) occ.push_back((float)((g22 * a1[c] - g12 * a2[c]) / det));
    for (int c = 0; c < 3; ++c) occ.push_back((float)((g11 * a2[c] - g12 * a1[c]) / det));
    int32_t id = k;
    float idf;
    std::memcpy(&idf, &id, sizeof(idf));
    occ.push_back(idf);
  }
  s->n_occ = (int)(occ.size() / kOcc);
  s->h_occ_slot.assign(n_obj, -1);
  for (int k = 0, q = 0; k < n_obj; ++k)
    if (types[k] == FPT_QUAD) s->h_occ_slot[k] = q++;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_types, (size_t)n_obj);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_occ_slot, (size_t)n_obj * sizeof(int32_t));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_types, s->types.data(), (size_t)n_obj, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_occ_slot, s->h_occ_slot.data(), (size_t)n_obj * sizeof(int32_t), cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess && s->n_occ) e = cudaMalloc(&s->d_occ, occ.size() * sizeof(float));
  if (e == cudaSuccess && s->n_occ)
    e = cudaMemcpyAsync(s->d_occ, occ.data(), occ.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_rec32, rec32.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_rec64, rec64.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_aux, aux.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_reclo, reclo.size() * sizeof(float));
  // copies on the context's stream, ordered before every later call on it, with no wait for the
  // device; their host sources live in the scene until it is freed
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_reclo, reclo.data(), reclo.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_rec32, rec32.data(), rec32.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_rec64, rec64.data(), rec64.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_aux, aux.data(), aux.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) {
    fpt_scene_free(s);
    return fail(ctx, FPT_ECUDA, "scene upload: %s", cudaGetErrorString(e));
  }
  *out = s;
  return FPT_OK;
}

fpt_status fpt_scene_upload_device(fpt_ctx* ctx, const uint8_t* types, const float* verts, int32_t n_obj,
                                   const double* centre, fpt_scene** out) {
  if (!ctx || !types || !verts || !out) return fail(ctx, FPT_EINVAL, "null argument");
  *out = nullptr;
  if (n_obj < 1 || n_obj > 65535) return fail(ctx, FPT_EINVAL, "n_obj %d outside [1, 65535]", n_obj);
  for (int k = 0; k < n_obj; ++k)
    if (types[k] != FPT_QUAD && types[k] != FPT_EDGE) return fail(ctx, FPT_EINVAL, "object %d: bad type", k);
  if (centre)
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(centre[c])) return fail(ctx, FPT_EINVAL, "non-finite centre");
  fpt_scene* s = new (std::nothrow) fpt_scene();
  if (!s) return FPT_ENOMEM;
  s->ctx = ctx;
  s->n_obj = n_obj;
  s->types.assign(types, types + n_obj);
  for (int c = 0; c < 3; ++c) s->centre[c] = centre ? centre[c] : 0.0;
  s->h_occ_slot.assign(n_obj, -1);
  int n_occ = 0;
  for (int k = 0; k < n_obj; ++k)
    if (types[k] == FPT_QUAD) s->h_occ_slot[k] = n_occ++;
  s->n_occ = n_occ;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_types, (size_t)n_obj);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_occ_slot, (size_t)n_obj * sizeof(int32_t));
  if (e == cudaSuccess && n_occ) e = cudaMalloc(&s->d_occ, (size_t)n_occ * kOcc * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_rec32, (size_t)n_obj * kRec32 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_rec64, (size_t)n_obj * kRec64 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_aux, (size_t)n_obj * kAux * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_reclo, (size_t)n_obj * kRecLo * sizeof(float));
  // the type tables' host sources stay in the scene until it is freed
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_types, s->types.data(), (size_t)n_obj, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->d_occ_slot, s->h_occ_slot.data(), (size_t)n_obj * sizeof(int32_t), cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess)
    e = launch_object_records(n_obj, s->d_types, s->d_occ_slot, verts, s->centre, s->d_rec32, s->d_reclo, s->d_rec64,
                              s->d_aux, s->d_occ, ctx->d_err, ctx->stream);
  if (e != cudaSuccess) {
    fpt_scene_free(s);
    return fail(ctx, FPT_ECUDA, "device scene upload: %s", cudaGetErrorString(e));
  }
  *out = s;
  return FPT_OK;
}

void fpt_scene_free(fpt_scene* s) {
  if (!s) return;
  cudaFree(s->d_rec32);
  cudaFree(s->d_rec64);
  cudaFree(s->d_aux);
  cudaFree(s->d_reclo);
  cudaFree(s->d_tx32);
  cudaFree(s->d_rx32);
  cudaFree(s->d_tx64);
  cudaFree(s->d_rx64);
  cudaFree(s->d_occ);
  cudaFree(s->d_types);
  cudaFree(s->d_occ_slot);
  delete s;
}

// Upload points (recentred, FP32 pairs and FP64) asynchronously on `stream`.  h32 / h64 hold the host
// sources until the next upload or the scene's release; the old device buffers are freed first
// (cudaFree waits for the device), so no copy from the old sources is pending when they are refilled.
static cudaError_t upload_points(const double* p, int n, const double* centre, float** d32, double** d64,
                                 std::vector<float>& h32, std::vector<double>& h64, cudaStream_t stream) {
  cudaFree(*d32);
  cudaFree(*d64);
  *d32 = nullptr;
  *d64 = nullptr;
  h32.assign((size_t)n * kEnd32, 0.f);
  h64.assign((size_t)n * 3, 0.0);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) {
      double x = p[3 * i + c] - centre[c];
      h64[3 * i + c] = x;
      split(x, h32[kEnd32 * i + c], h32[kEnd32 * i + 3 + c]);
    }
  cudaError_t e = cudaMalloc(d32, h32.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(d64, h64.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(*d32, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(*d64, h64.data(), h64.size() * sizeof(double), cudaMemcpyHostToDevice, stream);
  return e;
}

fpt_status fpt_set_endpoints(fpt_scene* s, const double* tx, int32_t n_tx, const double* rx, int32_t n_rx) {
  if (!s || !tx || !rx) return FPT_EINVAL;
  fpt_ctx* ctx = s->ctx;
  if (n_tx < 1 || n_rx < 1) return fail(ctx, FPT_EINVAL, "need at least one TX and one RX");
  for (int i = 0; i < 3 * n_tx; ++i)
    if (!std::isfinite(tx[i])) return fail(ctx, FPT_EINVAL, "non-finite TX");
  for (int i = 0; i < 3 * n_rx; ++i)
    if (!std::isfinite(rx[i])) return fail(ctx, FPT_EINVAL, "non-finite RX");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, upload_points(tx, n_tx, s->centre, &s->d_tx32, &s->d_tx64, s->h_tx32, s->h_tx64, ctx->stream));
  CUDA_OR_FAIL(ctx, upload_points(rx, n_rx, s->centre, &s->d_rx32, &s->d_rx64, s->h_rx32, s->h_rx64, ctx->stream));
  s->n_tx = s->tx_cap = n_tx;
  s->n_rx = s->rx_cap = n_rx;
  return FPT_OK;
}

// Device buffers for n endpoints: kept when they already hold n, reallocated otherwise (cudaFree waits
// for the device, so a pending copy from an earlier host upload into the old buffer has finished).
static cudaError_t endpoint_buffers(int n, int* cap, float** d32, double** d64) {
  if (n <= *cap && *d32 && *d64) return cudaSuccess;
  cudaFree(*d32);
  cudaFree(*d64);
  *d32 = nullptr;
  *d64 = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(d32, (size_t)n * kEnd32 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(d64, (size_t)n * 3 * sizeof(double));
  if (e == cudaSuccess) *cap = n;
  return e;
}

fpt_status fpt_set_endpoints_device(fpt_scene* s, const float* tx, int32_t n_tx, const float* rx, int32_t n_rx) {
  if (!s || !tx || !rx) return s ? fail(s->ctx, FPT_EINVAL, "null argument") : FPT_EINVAL;
  fpt_ctx* ctx = s->ctx;
  if (n_tx < 1 || n_rx < 1) return fail(ctx, FPT_EINVAL, "need at least one TX and one RX");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, endpoint_buffers(n_tx, &s->tx_cap, &s->d_tx32, &s->d_tx64));
  CUDA_OR_FAIL(ctx, endpoint_buffers(n_rx, &s->rx_cap, &s->d_rx32, &s->d_rx64));
  CUDA_OR_FAIL(ctx, launch_endpoint_records(tx, n_tx, s->centre, s->d_tx32, s->d_tx64, ctx->d_err, ctx->stream));
  CUDA_OR_FAIL(ctx, launch_endpoint_records(rx, n_rx, s->centre, s->d_rx32, s->d_rx64, ctx->d_err, ctx->stream));
  s->n_tx = n_tx;
  s->n_rx = n_rx;
  return FPT_OK;
}

fpt_status fpt_scene_update_vertices(fpt_scene* s, const float* verts) {
  if (!s || !verts) return s ? fail(s->ctx, FPT_EINVAL, "null argument") : FPT_EINVAL;
  fpt_ctx* ctx = s->ctx;
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, launch_object_records(s->n_obj, s->d_types, s->d_occ_slot, verts, s->centre, s->d_rec32,
                                          s->d_reclo, s->d_rec64, s->d_aux, s->d_occ, ctx->d_err, ctx->stream));
  return FPT_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
static fpt_status make_alphabet(fpt_ctx* ctx, const fpt_scene* s, const int32_t* alphabet, int32_t n_alpha,
                                fpt_batch* b) {
  std::vector<int32_t>& a = b->h_alphabet;
  a.clear();
  if (alphabet) {
    if (n_alpha < 1) return fail(ctx, FPT_EINVAL, "empty alphabet");
    a.assign(alphabet, alphabet + n_alpha);
    for (int32_t o : a)
      if (o < 0 || o >= s->n_obj) return fail(ctx, FPT_EINVAL, "alphabet id %d out of range", o);
  } else {
    for (int k = 0; k < s->n_obj; ++k) a.push_back(k);
  }
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, cudaMalloc(&b->d_alphabet, a.size() * sizeof(int32_t)));
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(b->d_alphabet, a.data(), a.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    ctx->stream));
  b->dev.alphabet = b->d_alphabet;
  b->dev.n_alpha = (int)a.size();
  // positions of the reflectors, then of the edges: the exhaustive enumeration by pattern
  std::vector<int32_t>& pos = b->h_type_pos;
  pos.clear();
  for (int pass = 0; pass < 2; ++pass)
    for (size_t k = 0; k < a.size(); ++k)
      if ((s->types[a[k]] == FPT_QUAD) == (pass == 0)) pos.push_back((int32_t)k);
  b->dev.n_alpha_quad = 0;
  for (int32_t o : a) b->dev.n_alpha_quad += s->types[o] == FPT_QUAD;
  CUDA_OR_FAIL(ctx, cudaMalloc(&b->d_type_pos, pos.size() * sizeof(int32_t)));
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(b->d_type_pos, pos.data(), pos.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    ctx->stream));
  b->dev.type_pos = b->d_type_pos;
  b->types = s->types;
  return FPT_OK;
}

// Reciprocals of the exhaustive decoders' divisors (FastDiv).
static void set_reciprocals(BatchDev& d) {
  d.fd_rx = make_fastdiv((uint64_t)d.n_rx);
  d.fd_alpha = make_fastdiv((uint64_t)d.n_alpha);
  d.fd_quad = make_fastdiv((uint64_t)d.n_alpha_quad);
  d.fd_edge = make_fastdiv((uint64_t)(d.n_alpha - d.n_alpha_quad));
  for (int n = 0; n <= kMaxOrder; ++n) d.fd_kpow[n] = make_fastdiv(d.kpow[n]);
  const uint64_t range = d.hi >= d.lo ? (uint64_t)(d.hi - d.lo + 1) : 1u;
  d.fd_alpha1 = make_fastdiv(d.n_alpha > 1 ? (uint64_t)(d.n_alpha - 1) : 1u);
  d.fd_range = make_fastdiv(range);
  d.fd_pp = make_fastdiv(d.per_pair);
  auto t32 = [](uint64_t m) { return m >= 1 && m <= 65535 ? (uint32_t)((1ull << 32) % m) : 0u; };
  d.t32_alpha = t32((uint64_t)d.n_alpha);
  d.t32_alpha1 = t32(d.n_alpha > 1 ? (uint64_t)(d.n_alpha - 1) : 1u);
  d.t32_range = t32(range);
}

static fpt_status check_orders(fpt_ctx* ctx, int lo, int hi) {
  if (lo < 1 || hi > kMaxOrder || lo > hi) return fail(ctx, FPT_EINVAL, "orders [%d, %d] outside [1, %d]", lo, hi, kMaxOrder);
  return FPT_OK;
}

fpt_status fpt_batch_exhaustive(fpt_ctx* ctx, const fpt_scene* s, const int32_t* alphabet, int32_t n_alpha,
                                int32_t lo, int32_t hi, fpt_batch** out) {
  if (!ctx || !s || !out) return fail(ctx, FPT_EINVAL, "null argument");
  *out = nullptr;
  if (s->n_tx < 1 || s->n_rx < 1) return fail(ctx, FPT_EINVAL, "scene has no endpoints");
  fpt_status st = check_orders(ctx, lo, hi);
  if (st != FPT_OK) return st;
  fpt_batch* b = new (std::nothrow) fpt_batch();
  if (!b) return FPT_ENOMEM;
  b->ctx = ctx;
  st = make_alphabet(ctx, s, alphabet, n_alpha, b);
  if (st != FPT_OK) {
    fpt_batch_free(b);
    return st;
  }
  BatchDev& d = b->dev;
  d.mode = BATCH_EXHAUSTIVE;
  d.lo = lo;
  d.hi = hi;
  d.n_max = hi;
  d.n_tx = s->n_tx;
  d.n_rx = s->n_rx;
  // K^n and per-pair offsets; refuse sizes that overflow 64-bit indexing
  const double K = d.n_alpha;
  double total = 0;
  for (int n = lo; n <= hi; ++n) total += std::pow(K, n);
  if (total * (double)s->n_tx * (double)s->n_rx > 9.0e18) {
    fpt_batch_free(b);
    return fail(ctx, FPT_EINVAL, "batch too large for 64-bit path indices");
  }
  d.kpow[0] = 1;
  for (int n = 1; n <= kMaxOrder; ++n) d.kpow[n] = n <= hi ? d.kpow[n - 1] * (uint64_t)d.n_alpha : 0;
  // offset[n] = sum_{m = lo}^{n-1} K^m: first index of order n inside a pair
  uint64_t acc = 0;
  for (int n = 0; n <= kMaxOrder + 1; ++n) {
    d.offset[n] = acc;
    if (n >= lo && n <= hi && n <= kMaxOrder) acc += d.kpow[n];
  }
  d.per_pair = acc;
  d.n_paths = acc * (uint64_t)s->n_tx * (uint64_t)s->n_rx;
  set_reciprocals(d);
  *out = b;
  return FPT_OK;
}

fpt_status fpt_batch_seeded(fpt_ctx* ctx, const fpt_scene* s, const int32_t* alphabet, int32_t n_alpha, uint64_t seed,
                            uint64_t per_pair, int32_t lo, int32_t hi, fpt_batch** out) {
  if (!ctx || !s || !out) return fail(ctx, FPT_EINVAL, "null argument");
  *out = nullptr;
  if (s->n_tx < 1 || s->n_rx < 1) return fail(ctx, FPT_EINVAL, "scene has no endpoints");
  fpt_status st = check_orders(ctx, lo, hi);
  if (st != FPT_OK) return st;
  if (per_pair < 1) return fail(ctx, FPT_EINVAL, "per_pair must be >= 1");
  fpt_batch* b = new (std::nothrow) fpt_batch();
  if (!b) return FPT_ENOMEM;
  b->ctx = ctx;
  st = make_alphabet(ctx, s, alphabet, n_alpha, b);
  if (st == FPT_OK && b->dev.n_alpha < 2 && hi > 1) st = fail(ctx, FPT_EINVAL, "seeded batches need >= 2 objects");
  if (st != FPT_OK) {
    fpt_batch_free(b);
    return st;
  }
  BatchDev& d = b->dev;
  d.mode = BATCH_SEEDED;
  d.lo = lo;
  d.hi = hi;
  d.n_max = hi;
  d.n_tx = s->n_tx;
  d.n_rx = s->n_rx;
  d.seed = seed;
  d.per_pair = per_pair;
  d.n_paths = per_pair * (uint64_t)s->n_tx * (uint64_t)s->n_rx;
  set_reciprocals(b->dev);
  *out = b;
  return FPT_OK;
}

fpt_status fpt_batch_explicit(fpt_ctx* ctx, const fpt_scene* s, const int32_t* ids_dev, const uint8_t* order_dev,
                              const int32_t* tx_idx_dev, const int32_t* rx_idx_dev, uint64_t n, int32_t n_max,
                              fpt_batch** out) {
  // an empty batch (n = 0) is legal and its device arrays may be NULL
  if (!ctx || !s || !out || (n > 0 && (!ids_dev || !order_dev || !tx_idx_dev || !rx_idx_dev)))
    return fail(ctx, FPT_EINVAL, "null argument");
  *out = nullptr;
  if (n_max < 1 || n_max > kMaxOrder) return fail(ctx, FPT_EINVAL, "n_max %d outside [1, %d]", n_max, kMaxOrder);
  if (s->n_tx < 1 || s->n_rx < 1) return fail(ctx, FPT_EINVAL, "scene has no endpoints");
  fpt_batch* b = new (std::nothrow) fpt_batch();
  if (!b) return FPT_ENOMEM;
  b->ctx = ctx;
  BatchDev& d = b->dev;
  d.mode = BATCH_EXPLICIT;
  d.n_alpha = s->n_obj;  // ids are object ids, checked against the object count
  d.lo = 1;
  d.hi = n_max;
  d.n_max = n_max;
  d.n_tx = s->n_tx;
  d.n_rx = s->n_rx;
  d.n_paths = n;
  d.per_pair = 1;
  d.ids = ids_dev;
  d.order = order_dev;
  d.tx_idx = tx_idx_dev;
  d.rx_idx = rx_idx_dev;
  b->types = s->types;
  set_reciprocals(b->dev);
  *out = b;
  return FPT_OK;
}

fpt_status fpt_batch_size(const fpt_batch* b, uint64_t* n_paths, int32_t* n_max) {
  if (!b) return FPT_EINVAL;
  if (n_paths) *n_paths = b->dev.n_paths;
  if (n_max) *n_max = b->dev.n_max;
  return FPT_OK;
}

void fpt_batch_free(fpt_batch* b) {
  if (!b) return;
  cudaFree(b->d_alphabet);
  cudaFree(b->d_type_pos);
  cudaFree(b->d_lists);
  delete b;
}

fpt_status fpt_enumerate(fpt_ctx* ctx, const fpt_batch* b, int32_t* ids, uint8_t* order, int32_t* tx_idx,
                         int32_t* rx_idx) {
  if (!ctx || !b) return fail(ctx, FPT_EINVAL, "null argument");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, launch_enumerate(b->dev, ids, order, tx_idx, rx_idx, ctx->stream, ctx->n_sm));
  return FPT_OK;
}

// Bucket a seeded/explicit batch by (order, pattern) (once per batch; synchronous).
static fpt_status ensure_buckets(fpt_ctx* ctx, fpt_batch* b, const SceneDev& S) {
  if (b->dev.mode == BATCH_EXHAUSTIVE || b->bucketed) return FPT_OK;
  unsigned long long h[kPatternKeys] = {0};
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->d_count, 0, sizeof(h), ctx->stream));
  CUDA_OR_FAIL(ctx, launch_pattern_histogram(S, b->dev, ctx->d_count, ctx->stream, ctx->n_sm));
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(h, ctx->d_count, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  // layout: orders in sequence; inside an order, the buckets large enough for a pattern launch, then the
  // small ones together (the unified kernel takes them in one launch)
  const uint64_t min_bucket = min_pattern_bucket(ctx);
  uint64_t acc = 0;
  unsigned long long cur[kPatternKeys];
  for (int n = 1; n <= kMaxOrder; ++n) {
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1) b->small_start[n] = acc;
      for (unsigned q = 0; q < (unsigned)n_patterns(n); ++q) {
        const int k = pattern_key(n, q);
        if ((h[k] >= min_bucket) != (pass == 0)) continue;
        b->start[k] = acc;
        b->count[k] = h[k];
        cur[k] = acc;
        acc += h[k];
      }
      if (pass == 1) b->small_count[n] = acc - b->small_start[n];
    }
  }
  if (acc != b->dev.n_paths) return fail(ctx, FPT_EDEVICE, "pattern histogram mismatch");
  CUDA_OR_FAIL(ctx, cudaMalloc(&b->d_lists, (acc ? acc : 1) * sizeof(PathRec)));
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(ctx->d_count, cur, sizeof(cur), cudaMemcpyHostToDevice, ctx->stream));
  CUDA_OR_FAIL(ctx, launch_pattern_scatter(S, b->dev, ctx->d_count, b->d_lists, ctx->stream, ctx->n_sm));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  b->bucketed = true;
  return FPT_OK;
}

// Polish scratch for an order slice of n paths of order `order`: three uint32
// lists of n entries and the first Newton steps (2 order floats per path).
static fpt_status ensure_rescue(fpt_ctx* ctx, uint64_t n, int order) {
  if (n > ctx->rescue_cap) {
    cudaFree(ctx->d_rescue);
    ctx->d_rescue = nullptr;
    ctx->rescue_cap = 0;
    CUDA_OR_FAIL(ctx, cudaMalloc(&ctx->d_rescue, 3 * n * sizeof(uint32_t)));
    ctx->rescue_cap = n;
  }
  const size_t step = (size_t)2 * order * n;
  if (step > ctx->step_cap) {
    cudaFree(ctx->d_step);
    ctx->d_step = nullptr;
    ctx->step_cap = 0;
    CUDA_OR_FAIL(ctx, cudaMalloc(&ctx->d_step, step * sizeof(float)));
    ctx->step_cap = step;
  }
  return FPT_OK;
}

// Paths of order n in a batch: count and list (nullptr for exhaustive batches).
static uint64_t order_slice(const fpt_batch* b, int n, const PathRec** list) {
  if (b->dev.mode == BATCH_EXHAUSTIVE) {
    *list = nullptr;
    if (n < b->dev.lo || n > b->dev.hi) return 0;
    return b->dev.kpow[n] * (uint64_t)b->dev.n_tx * (uint64_t)b->dev.n_rx;
  }
  // the buckets of order n are contiguous; the order's range starts at its first bucket in the layout
  uint64_t first = b->small_start[n], c = 0;
  for (unsigned q = 0; q < (unsigned)n_patterns(n); ++q) {
    const int k = pattern_key(n, q);
    c += b->count[k];
    if (b->count[k] && b->start[k] < first) first = b->start[k];
  }
  *list = b->d_lists + first;
  return c;
}

// Paths of order n and interaction-type pattern q: count and list (nullptr for exhaustive batches).
static uint64_t pattern_slice(const fpt_batch* b, int n, unsigned q, const PathRec** list) {
  if (b->dev.mode == BATCH_EXHAUSTIVE) {
    *list = nullptr;
    if (n < b->dev.lo || n > b->dev.hi) return 0;
    uint64_t c = (uint64_t)b->dev.n_tx * (uint64_t)b->dev.n_rx;
    for (int i = 0; i < n; ++i)
      c *= (uint64_t)(((q >> i) & 1u) ? b->dev.n_alpha_quad : b->dev.n_alpha - b->dev.n_alpha_quad);
    return c;
  }
  *list = b->d_lists + b->start[pattern_key(n, q)];
  return b->count[pattern_key(n, q)];
}

static fpt_status check_scene_batch(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* b) {
  if (!ctx || !s || !b) return fail(ctx, FPT_EINVAL, "null argument");
  if (b->dev.n_tx != s->n_tx || b->dev.n_rx != s->n_rx)
    return fail(ctx, FPT_EINVAL, "batch was built for other endpoints");
  if (b->dev.mode == BATCH_EXPLICIT && b->dev.n_alpha != s->n_obj) return fail(ctx, FPT_EINVAL, "batch/scene mismatch");
  if (b->types != s->types) return fail(ctx, FPT_EINVAL, "batch was built for a scene with other object types");
  return FPT_OK;
}

// Solve (and, with grad, the fused backward) of every order of the batch.
static fpt_status solve_impl(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* bc, const fpt_solve_params* prm,
                             float* T, float* X, float* L, uint8_t* status, uint8_t* iters, float* rho,
                             const GradCfg* grad) {
  fpt_status st = check_scene_batch(ctx, s, bc);
  if (st != FPT_OK) return st;
  if (bc->dev.n_paths > 0 && (!T || !status)) return fail(ctx, FPT_EINVAL, "T_out and status_out are required");
  fpt_solve_params p;
  fpt_default_params(&p);
  if (prm) p = *prm;
  if (p.init_mode != 0 && p.init_mode != 1) return fail(ctx, FPT_EINVAL, "init_mode must be 0 or 1");
  if (p.init_mode == 1 && !ctx->init_mlp) return fail(ctx, FPT_EINVAL, "init_mode 1 needs fpt_set_init_mlp");
  if (p.max_iters < 0 || p.fp_iters < 1 || p.polish < 0 || p.polish > 2 || p.specialize < 0 || p.specialize > 2 ||
      !(p.kink_stop >= 0.f) || !(p.polish_radius >= 0.f))
    return fail(ctx, FPT_EINVAL, "bad solver parameters");
  fpt_batch* b = const_cast<fpt_batch*>(bc);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_buckets(ctx, b, scene_dev(s));
  if (st != FPT_OK) return st;
  const SceneDev S = scene_dev(s);
  const float kink = p.kink_stop > 0.f ? p.kink_stop : 0.1f * p.deg_tol;
  SolveCfg sc{p.max_iters, p.fp_iters, p.fixed_iters, p.tol_step * p.tol_step, kink * kink,
              p.refill > 32 ? 32 : p.refill, p.init_mode == 1, kMaxChunk};
  // the polish needs its Newton step only to a modest relative accuracy: 100x looser pivot test than the adjoint
  PolishCfg pc{POLISH_SOLVE, p.polish, p.solved_tol, p.deg_tol, 1e-2f * p.cond_fp64, p.polish_fp64,
               p.polish_radius};
  if (b->dev.n_max > kMaxBfgsOrder) {
    // the kernels of orders 1-5 write the first five slots of a path; clear the rest
    CUDA_OR_FAIL(ctx, cudaMemsetAsync(T, 0, b->dev.n_paths * (uint64_t)b->dev.n_max * 2 * sizeof(float), ctx->stream));
    if (X) CUDA_OR_FAIL(ctx, cudaMemsetAsync(X, 0, b->dev.n_paths * (uint64_t)b->dev.n_max * 3 * sizeof(float), ctx->stream));
  }
  for (int n = 1; n <= kMaxOrder; ++n) {
    const PathRec* list;
    uint64_t cnt = order_slice(b, n, &list);
    if (!cnt) continue;
    if (cnt > 0xFFFFFFFFull) return fail(ctx, FPT_EUNSUPPORTED, "more than 2^32 paths of one order");
    if (p.init_mode == 1) {
      // learned start: fused features -> network -> T on the tensor cores
      fpt_mlp* m = ctx->init_mlp;
      if (m->wt_stale) {
        CUDA_OR_FAIL(ctx, launch_mlp_tile_weights(m->d_wb, m->d_wt, ctx->stream));
        m->wt_stale = false;
      }
      ProfScope ps(ctx, FPT_K_MLP);
      CUDA_OR_FAIL(ctx, launch_mlp_infer(S, b->dev, n, list, cnt, 1.f / m->scale, m->d_wt, m->d_w, T, ctx->d_err,
                                         ctx->stream, ctx->n_sm));
    }
    {
      ProfScope ps(ctx, FPT_K_BFGS);
      // pattern kernels pay off for buckets that fill the GPU several times over.  Seeded and explicit
      // batches keep an order's small buckets together, and the unified kernel takes them in one launch;
      // an exhaustive order with a small pattern runs the unified kernel throughout.
      const bool listed = b->dev.mode != BATCH_EXHAUSTIVE;
      const bool force = p.specialize == 2;
      bool by_pattern = p.specialize && sc.refill > 0 && n <= kMaxBfgsOrder;
      for (unsigned q = 0; by_pattern && !listed && !force && q < (1u << n); ++q) {
        const PathRec* qlist;
        const uint64_t qcnt = pattern_slice(b, n, q, &qlist);
        if (qcnt && qcnt < min_pattern_bucket(ctx)) by_pattern = false;
      }
      if (by_pattern) {
        // the pattern launches of one order are independent: spread them over the side streams so that
        // each launch's tail overlaps the next one; each concurrent launch has its own work counter
        CUDA_OR_FAIL(ctx, cudaEventRecord(ctx->fork_ev, ctx->stream));
        for (int k = 0; k < fpt_ctx::kSide; ++k) CUDA_OR_FAIL(ctx, cudaStreamWaitEvent(ctx->side[k], ctx->fork_ev, 0));
        int used = 0;
        for (unsigned q = 0; q < (1u << n); ++q) {
          const PathRec* qlist;
          const uint64_t qcnt = pattern_slice(b, n, q, &qlist);
          if (!qcnt || (listed && !force && qcnt < min_pattern_bucket(ctx))) continue;
          cudaStream_t sq = ctx->side[used % fpt_ctx::kSide];
          ++used;
          CUDA_OR_FAIL(ctx, launch_bfgs(n, (int)q, S, b->dev, sc, qcnt, qlist, T, status, iters, sq, ctx->n_sm,
                                        ctx->d_work + q));
        }
        if (listed && !force && b->small_count[n]) {
          cudaStream_t sq = ctx->side[used % fpt_ctx::kSide];
          ++used;
          CUDA_OR_FAIL(ctx, launch_bfgs(n, -1, S, b->dev, sc, b->small_count[n], b->d_lists + b->small_start[n], T,
                                        status, iters, sq, ctx->n_sm, ctx->d_work + 32));
        }
        // join every side stream that waited on the fork, used or not (a stream capture must end joined)
        for (int k = 0; k < fpt_ctx::kSide; ++k) {
          CUDA_OR_FAIL(ctx, cudaEventRecord(ctx->join_ev[k], ctx->side[k]));
          CUDA_OR_FAIL(ctx, cudaStreamWaitEvent(ctx->stream, ctx->join_ev[k], 0));
        }
      } else {
        CUDA_OR_FAIL(ctx, launch_bfgs(n, -1, S, b->dev, sc, cnt, list, T, status, iters, ctx->stream, ctx->n_sm,
                                      ctx->d_work));
      }
    }
    st = ensure_rescue(ctx, cnt, n);
    if (st != FPT_OK) return st;
    {
      ProfScope ps(ctx, FPT_K_POLISH);
      GradCfg gc{};
      if (grad) {
        gc = *grad;
        gc.rescue_list = ctx->d_rescue + cnt;
        gc.rescue_count = ctx->d_rescue_n + 1;
      }
      uint32_t* step_list = p.polish_all ? nullptr : ctx->d_rescue + 2 * cnt;
      CUDA_OR_FAIL(ctx, launch_polish(n, S, b->dev, pc, cnt, list, T, X, L, status, rho, nullptr, nullptr, ctx->stream,
                                      ctx->n_sm, ctx->d_rescue, ctx->d_rescue_n, grad ? &gc : nullptr, step_list,
                                      ctx->d_rescue_n + 2, ctx->d_step));
    }
  }
  return FPT_OK;
}

fpt_status fpt_solve(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* bc, const fpt_solve_params* prm, float* T,
                     float* X, float* L, uint8_t* status, uint8_t* iters, float* rho) {
  return solve_impl(ctx, s, bc, prm, T, X, L, status, iters, rho, nullptr);
}

// Context-owned FP64 gradient accumulators, sized for the scene and cleared.
static fpt_status ensure_gacc(fpt_ctx* ctx, const fpt_scene* s) {
  const size_t need = (size_t)(9 * s->n_obj + 3 * (s->n_tx + s->n_rx));
  if (need > ctx->gacc_cap) {
    cudaFree(ctx->d_gacc);
    ctx->d_gacc = nullptr;
    ctx->gacc_cap = 0;
    CUDA_OR_FAIL(ctx, cudaMalloc(&ctx->d_gacc, need * sizeof(double)));
    ctx->gacc_cap = need;
  }
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->d_gacc, 0, need * sizeof(double), ctx->stream));
  return FPT_OK;
}

fpt_status fpt_solve_grad(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* bc, const fpt_solve_params* prm,
                          const float* dX, const float* dL, uint8_t dL_status_mask, float* T, float* X, float* L,
                          uint8_t* status, uint8_t* iters, float* rho, float* g_tx, float* g_rx,
                          float* g_vertices) {
  fpt_status st = check_scene_batch(ctx, s, bc);
  if (st != FPT_OK) return st;
  if (prm && prm->polish_fp64) return fail(ctx, FPT_EUNSUPPORTED, "fpt_solve_grad runs the double-float polish");
  if (prm && prm->polish < 1) return fail(ctx, FPT_EINVAL, "fpt_solve_grad needs polish >= 1");
  if (!status && bc->dev.n_paths > 0) return fail(ctx, FPT_EINVAL, "status_out is required");
  if (!(prm && prm->fuse_adjoint)) {
    // the adjoint kernels after the solve, with the cotangents given here
    st = fpt_solve(ctx, s, bc, prm, T, X, L, status, iters, rho);
    if (st != FPT_OK) return st;
    return fpt_backward(ctx, s, bc, T, status, dX, dL, dL_status_mask, g_tx, g_rx, g_vertices);
  }
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_gacc(ctx, s);
  if (st != FPT_OK) return st;
  fpt_solve_params p;
  fpt_default_params(&p);
  GradCfg gc{};
  gc.dX = dX;
  gc.dL = dL;
  gc.dl_mask = dL ? (uint8_t)0 : dL_status_mask;
  gc.cond_adj = p.cond_fp64;
  gc.deg_tol = prm ? prm->deg_tol : p.deg_tol;
  gc.gacc = ctx->d_gacc;
  gc.flush_tiles = ctx->acc_flush_tiles;
  gc.acc_in_smem = ctx->acc_smem;
  gc.dropped = ctx->d_rescue_n + 3;
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(gc.dropped, 0, sizeof(unsigned), ctx->stream));
  st = solve_impl(ctx, s, bc, prm, T, X, L, status, iters, rho, &gc);
  if (st != FPT_OK) return st;
  const SceneDev S = scene_dev(s);
  ProfScope ps(ctx, FPT_K_OTHER);
  CUDA_OR_FAIL(ctx, launch_backward_finalize(S, nullptr, ctx->d_gacc, g_tx, g_rx, g_vertices, ctx->stream));
  return FPT_OK;
}

fpt_status fpt_validity(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* bc, const float* T, uint8_t* mask,
                        float* bdist, float* rho) {
  fpt_status st = check_scene_batch(ctx, s, bc);
  if (st != FPT_OK) return st;
  if (!T && bc->dev.n_paths > 0) return fail(ctx, FPT_EINVAL, "T is required");
  fpt_batch* b = const_cast<fpt_batch*>(bc);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_buckets(ctx, b, scene_dev(s));
  if (st != FPT_OK) return st;
  fpt_solve_params p;
  fpt_default_params(&p);
  const SceneDev S = scene_dev(s);
  PolishCfg pc{POLISH_VALIDITY, 0, p.solved_tol, p.deg_tol, 1e-2f * p.cond_fp64, 0};
  for (int n = 1; n <= kMaxOrder; ++n) {
    const PathRec* list;
    uint64_t cnt = order_slice(b, n, &list);
    if (!cnt) continue;
    if (cnt > 0xFFFFFFFFull) return fail(ctx, FPT_EUNSUPPORTED, "more than 2^32 paths of one order");
    st = ensure_rescue(ctx, cnt, n);
    if (st != FPT_OK) return st;
    ProfScope ps(ctx, FPT_K_POLISH);
    CUDA_OR_FAIL(ctx, launch_polish(n, S, b->dev, pc, cnt, list, const_cast<float*>(T), nullptr, nullptr, nullptr, rho,
                                    mask, bdist, ctx->stream, ctx->n_sm, ctx->d_rescue, ctx->d_rescue_n));
  }
  return FPT_OK;
}

fpt_status fpt_backward(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* bc, const float* T, const uint8_t* status,
                        const float* dX, const float* dL, uint8_t dL_status_mask, float* g_tx, float* g_rx,
                        float* g_vertices) {
  fpt_status st = check_scene_batch(ctx, s, bc);
  if (st != FPT_OK) return st;
  if (!T && bc->dev.n_paths > 0) return fail(ctx, FPT_EINVAL, "T is required");
  fpt_batch* b = const_cast<fpt_batch*>(bc);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_buckets(ctx, b, scene_dev(s));
  if (st != FPT_OK) return st;
  st = ensure_gacc(ctx, s);
  if (st != FPT_OK) return st;
  const SceneDev S = scene_dev(s);
  fpt_solve_params p;
  fpt_default_params(&p);
  if (!dL && dL_status_mask && !status && bc->dev.n_paths > 0)
    return fail(ctx, FPT_EINVAL, "dL_status_mask needs status");
  BackwardCfg bc_cfg{p.cond_fp64, p.deg_tol, ctx->acc_smem, ctx->acc_flush_tiles, dL ? (uint8_t)0 : dL_status_mask};
  bc_cfg.dropped = ctx->d_rescue_n + 3;
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(bc_cfg.dropped, 0, sizeof(unsigned), ctx->stream));
  for (int n = 1; n <= kMaxOrder; ++n) {
    const PathRec* list;
    uint64_t cnt = order_slice(b, n, &list);
    if (!cnt) continue;
    if (cnt > 0xFFFFFFFFull) return fail(ctx, FPT_EUNSUPPORTED, "more than 2^32 paths of one order");
    st = ensure_rescue(ctx, cnt, n);
    if (st != FPT_OK) return st;
    ProfScope ps(ctx, FPT_K_BACKWARD);
    BackwardCfg cfg_n = bc_cfg;
    cfg_n.sel = ctx->d_rescue + 2 * cnt;  // the third list of the scratch (the polish's, free here)
    cfg_n.sel_count = ctx->d_rescue_n + 2;
    CUDA_OR_FAIL(ctx, launch_backward(n, S, b->dev, cfg_n, cnt, list, T, status, dX, dL, ctx->d_gacc, ctx->stream,
                                      ctx->n_sm, ctx->d_rescue, ctx->d_rescue_n));
  }
  {
    ProfScope ps(ctx, FPT_K_OTHER);
    CUDA_OR_FAIL(ctx, launch_backward_finalize(S, nullptr, ctx->d_gacc, g_tx, g_rx, g_vertices, ctx->stream));
  }
  return FPT_OK;
}

fpt_status fpt_backward_unrolled(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* bc, int32_t steps,
                                 int32_t fp_iters, const float* dX, const float* dL, float* T_out, uint8_t* status_out,
                                 float* g_tx, float* g_rx, float* g_vertices) {
  fpt_status st = check_scene_batch(ctx, s, bc);
  if (st != FPT_OK) return st;
  if (steps < 0 || steps > kUnrolledMaxSteps)
    return fail(ctx, FPT_EINVAL, "steps must be in [0, %d]", kUnrolledMaxSteps);
  if (fp_iters < 1 || fp_iters > kUnrolledMaxRounds) return fail(ctx, FPT_EINVAL, "fp_iters must be in [1, %d]",
                                                                 kUnrolledMaxRounds);
  fpt_batch* b = const_cast<fpt_batch*>(bc);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_buckets(ctx, b, scene_dev(s));
  if (st != FPT_OK) return st;
  st = ensure_gacc(ctx, s);
  if (st != FPT_OK) return st;
  const SceneDev S = scene_dev(s);
  for (int n = 1; n <= kMaxOrder; ++n) {
    const PathRec* list;
    const uint64_t cnt = order_slice(b, n, &list);
    if (!cnt) continue;
    // tape for every resident thread (at most 8 CTAs of kThreads per SM), within kUnrolledMaxTape bytes
    uint64_t threads = ((cnt + kThreads - 1) / kThreads) * kThreads;
    const uint64_t resident = (uint64_t)ctx->n_sm * 8 * kThreads;
    if (threads > resident) threads = resident;
    size_t need = unrolled_tape_floats(n, steps, threads);
    if (need * sizeof(float) > kUnrolledMaxTape) need = kUnrolledMaxTape / sizeof(float);
    if (need > ctx->tape_cap) {
      cudaFree(ctx->d_tape);
      ctx->d_tape = nullptr;
      ctx->tape_cap = 0;
      CUDA_OR_FAIL(ctx, cudaMalloc(&ctx->d_tape, need * sizeof(float)));
      ctx->tape_cap = need;
    }
    ProfScope ps(ctx, FPT_K_BACKWARD);
    CUDA_OR_FAIL(ctx, launch_unrolled(n, S, b->dev, steps, fp_iters, cnt, list, dX, dL, ctx->d_gacc, ctx->d_tape,
                                      ctx->tape_cap, T_out, status_out, ctx->stream, ctx->n_sm));
  }
  {
    ProfScope ps(ctx, FPT_K_OTHER);
    CUDA_OR_FAIL(ctx, launch_backward_finalize(S, nullptr, ctx->d_gacc, g_tx, g_rx, g_vertices, ctx->stream));
  }
  return FPT_OK;
}

fpt_status fpt_occlusion(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* bc, const float* T, const uint8_t* status,
                         uint8_t status_mask, float tol, uint16_t* blocked_out) {
  fpt_status st = check_scene_batch(ctx, s, bc);
  if (st != FPT_OK) return st;
  if (bc->dev.n_paths > 0 && (!T || !blocked_out)) return fail(ctx, FPT_EINVAL, "T and blocked_out are required");
  if (status_mask && !status && bc->dev.n_paths > 0) return fail(ctx, FPT_EINVAL, "status_mask needs status");
  if (!(tol >= 0.f)) return fail(ctx, FPT_EINVAL, "tol must be >= 0");
  if ((size_t)s->n_occ * kOcc * sizeof(float) > kMaxSmemBytes)
    return fail(ctx, FPT_EUNSUPPORTED, "%d planar objects exceed the occluder table", s->n_occ);
  fpt_batch* b = const_cast<fpt_batch*>(bc);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_buckets(ctx, b, scene_dev(s));
  if (st != FPT_OK) return st;
  const SceneDev S = scene_dev(s);
  const float t = tol > 0.f ? tol : 1e-4f;
  for (int n = 1; n <= kMaxOrder; ++n) {
    const PathRec* list;
    const uint64_t cnt = order_slice(b, n, &list);
    if (!cnt) continue;
    if (cnt > 0xFFFFFFFFull) return fail(ctx, FPT_EUNSUPPORTED, "more than 2^32 paths of one order");
    st = ensure_rescue(ctx, cnt, n);
    if (st != FPT_OK) return st;
    ProfScope ps(ctx, FPT_K_OTHER);
    CUDA_OR_FAIL(ctx, launch_occlusion(S, b->dev, n, list, cnt, T, status, status_mask, s->d_occ, s->n_occ, t,
                                       blocked_out, ctx->d_rescue, ctx->d_rescue_n, ctx->stream, ctx->n_sm));
  }
  return FPT_OK;
}

fpt_status fpt_backward_noalloc(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* b, const float* T,
                                const uint8_t* status, const float* dX, const float* dL, uint8_t dL_status_mask,
                                float* g_tx, float* g_rx, float* g_vertices) {
  fpt_status st = check_scene_batch(ctx, s, b);
  if (st != FPT_OK) return st;
  if (!T && b->dev.n_paths > 0) return fail(ctx, FPT_EINVAL, "T is required");
  if (!dL && dL_status_mask && !status && b->dev.n_paths > 0)
    return fail(ctx, FPT_EINVAL, "dL_status_mask needs status");
  const long long need = 9LL * s->n_obj + 3LL * (s->n_tx + s->n_rx);
  if (need > kNoAllocMaxAcc)
    return fail(ctx, FPT_EINVAL, "fpt_backward_noalloc: 9 n_obj + 3 (n_tx + n_rx) = %lld exceeds its limit %d", need,
                kNoAllocMaxAcc);
  if (b->dev.mode != BATCH_EXHAUSTIVE && !b->bucketed)
    return fail(ctx, FPT_EINVAL, "fpt_backward_noalloc: seeded/explicit batch not bucketed yet (solve it first)");
  const PathRec* lists[kMaxOrder + 1] = {nullptr};
  uint64_t counts[kMaxOrder + 1] = {0};
  for (int n = 1; n <= kMaxOrder; ++n) {
    counts[n] = order_slice(b, n, &lists[n]);
    if (counts[n] > (uint64_t)kNoAllocMaxSlice)
      return fail(ctx, FPT_EINVAL, "fpt_backward_noalloc: %llu paths of order %d exceed its limit %d",
                  (unsigned long long)counts[n], n, kNoAllocMaxSlice);
  }
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  fpt_solve_params p;
  fpt_default_params(&p);
  BackwardCfg cfg{p.cond_fp64, p.deg_tol, ctx->acc_smem, ctx->acc_flush_tiles, dL ? (uint8_t)0 : dL_status_mask};
  cfg.dropped = ctx->d_rescue_n + 3;  // context memory, allocated by fpt_create
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(cfg.dropped, 0, sizeof(unsigned), ctx->stream));
  CUDA_OR_FAIL(ctx, launch_backward_noalloc(ctx->device, scene_dev(s), b->dev, cfg, lists, counts, T, status, dX, dL,
                                            g_tx, g_rx, g_vertices, ctx->stream, ctx->n_sm));
  return FPT_OK;
}

fpt_status fpt_backward_dropped(fpt_ctx* ctx, uint64_t* count) {
  if (!ctx || !count) return fail(ctx, FPT_EINVAL, "null argument");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  unsigned h = 0;
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(&h, ctx->d_rescue_n + 3, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  *count = h;
  return FPT_OK;
}

fpt_status fpt_count_status(fpt_ctx* ctx, const uint8_t* status, uint64_t n, uint8_t mask, uint64_t* count) {
  if (!ctx || !count || (!status && n > 0)) return fail(ctx, FPT_EINVAL, "null argument");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  unsigned long long h = 0;
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned long long), ctx->stream));
  CUDA_OR_FAIL(ctx, launch_count_status(status, n, mask, ctx->d_count, ctx->stream, ctx->n_sm));
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(&h, ctx->d_count, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  *count = h;
  return FPT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// learned warm start
// ---------------------------------------------------------------------------
static void mlp_free_ws(fpt_mlp* m) {
  for (void* p : {(void*)m->d_H1, (void*)m->d_H2, (void*)m->d_H3, (void*)m->d_dZa, (void*)m->d_dZb, (void*)m->d_dYb,
                  (void*)m->d_X, (void*)m->d_Z1, (void*)m->d_Z2, (void*)m->d_Z3, (void*)m->d_Y,
                  (void*)m->d_dY, (void*)m->d_Ht1, (void*)m->d_Ht2, (void*)m->d_Ht3, (void*)m->d_Xt, (void*)m->d_dZta,
                  (void*)m->d_dZtb, (void*)m->d_dYt})
    cudaFree(p);
  m->d_H1 = m->d_H2 = m->d_H3 = m->d_dZa = m->d_dZb = m->d_dYb = m->d_X = nullptr;
  m->d_Ht1 = m->d_Ht2 = m->d_Ht3 = m->d_Xt = m->d_dZta = m->d_dZtb = m->d_dYt = nullptr;
  m->d_Z1 = m->d_Z2 = m->d_Z3 = m->d_Y = m->d_dY = nullptr;
  m->cap = 0;
}

static fpt_status mlp_ensure_ws(fpt_ctx* ctx, fpt_mlp* m, uint64_t B, bool train) {
  const uint64_t want = B < 128 ? 128 : B;
  if (want <= m->cap && (!train || m->d_Z1)) return FPT_OK;
  mlp_free_ws(m);
  const size_t H = want * kMlpHidden;
  cudaError_t e = cudaSuccess;
  auto bf = [&](__nv_bfloat16** p, size_t n) { if (e == cudaSuccess) e = cudaMalloc(p, n * sizeof(__nv_bfloat16)); };
  auto f32 = [&](float** p, size_t n) { if (e == cudaSuccess) e = cudaMalloc(p, n * sizeof(float)); };
  bf(&m->d_H1, H);
  bf(&m->d_H2, H);
  bf(&m->d_H3, H);
  bf(&m->d_X, want * kMlpIn);
  f32(&m->d_Y, want * kMlpOut);
  if (train) {
    f32(&m->d_Z1, H);
    f32(&m->d_Z2, H);
    f32(&m->d_Z3, H);
    bf(&m->d_dZa, H);
    bf(&m->d_dZb, H);
    bf(&m->d_dYb, want * kMlpOut);
    f32(&m->d_dY, want * kMlpOut);
    bf(&m->d_Ht1, H);
    bf(&m->d_Ht2, H);
    bf(&m->d_Ht3, H);
    bf(&m->d_Xt, want * kMlpIn);
    bf(&m->d_dZta, H);
    bf(&m->d_dZtb, H);
    bf(&m->d_dYt, want * kMlpOut);
  }
  if (e != cudaSuccess) {
    mlp_free_ws(m);
    return fail(ctx, FPT_ENOMEM, "MLP workspace for %llu rows: %s", (unsigned long long)want, cudaGetErrorString(e));
  }
  m->cap = want;
  return FPT_OK;
}

static GemmArgs gemm_args(int M, int N, int K, const __nv_bfloat16* A, long long sam, long long sak,
                          const __nv_bfloat16* Bm, long long sbn, long long sbk, int op, int* err) {
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = A;
  g.sam = sam;
  g.sak = sak;
  g.B = Bm;
  g.sbn = sbn;
  g.sbk = sbk;
  g.op = op;
  g.err = err;
  return g;
}

// forward pass of B rows of X; with `train`, keeps gelu' at each hidden layer's pre-activation (Z1..Z3)
static fpt_status mlp_forward_impl(fpt_ctx* ctx, fpt_mlp* m, const __nv_bfloat16* X, uint64_t B, float* Y,
                                   bool train) {
  const int Bi = (int)B;
  const __nv_bfloat16* W = m->d_wb;
  const float* P = m->d_w;
  const __nv_bfloat16* in = X;
  __nv_bfloat16* H[3] = {m->d_H1, m->d_H2, m->d_H3};
  float* Z[3] = {m->d_Z1, m->d_Z2, m->d_Z3};
  const int offW[3] = {kOffW1, kOffW2, kOffW3}, offB[3] = {kOffB1, kOffB2, kOffB3};
  for (int l = 0; l < 3; ++l) {
    const int K = l == 0 ? kMlpIn : kMlpHidden;
    GemmArgs g = gemm_args(Bi, kMlpHidden, K, in, K, 1, W + offW[l], K, 1, EPI_BIAS_GELU, ctx->d_err);
    g.bias = P + offB[l];
    g.C = train ? Z[l] : nullptr;
    g.scm = kMlpHidden;
    g.scn = 1;
    g.H = H[l];
    g.shm = kMlpHidden;
    g.shn = 1;
    if (train) {  // H^T [256][B]: the K-major operand of the next layer's weight gradient
      __nv_bfloat16* Ht[3] = {m->d_Ht1, m->d_Ht2, m->d_Ht3};
      g.Ht = Ht[l];
      g.shtm = 1;
      g.shtn = Bi;
    }
    CUDA_OR_FAIL(ctx, launch_gemm(g, 1, ctx->stream));
    in = H[l];
  }
  GemmArgs g = gemm_args(Bi, kMlpOut, kMlpHidden, in, kMlpHidden, 1, W + kOffW4, kMlpHidden, 1, EPI_STORE, ctx->d_err);
  g.bias = P + kOffB4;
  g.C = Y;
  g.scm = kMlpOut;
  g.scn = 1;
  CUDA_OR_FAIL(ctx, launch_gemm(g, 1, ctx->stream));
  return FPT_OK;
}

// loss and gradient (into m->d_g) of a batch; loss accumulated in m->d_loss.  Every GEMM reads K-major
// operands: the weight gradients dW = dZ^T act take the transposed copies written by the epilogues, the
// back-propagation dH = dZ W the transposed BF16 weights.
static int split_k(const fpt_ctx* ctx, int B, int m_tiles) {
  // one (row tile, K split) item per SM (each CTA adds one partial product into the gradient), at least
  // four 64-wide K chunks per split
  int ks = ctx->n_sm / m_tiles;
  const int max_ks = B / 256 > 1 ? B / 256 : 1;
  ks = ks < 1 ? 1 : (ks > max_ks ? max_ks : ks);
  // the GEMM gives each split ceil(B / (ks 64)) chunks of 64: count only the splits that get some
  const int per = (B + ks * 64 - 1) / (ks * 64) * 64;
  return (B + per - 1) / per;
}

static fpt_status mlp_backward_impl(fpt_ctx* ctx, fpt_mlp* m, const __nv_bfloat16* X, const float* T, const float* G,
                                    uint64_t B) {
  const int Bi = (int)B;
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(m->d_g, 0, kMlpParams * sizeof(float), ctx->stream));
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(m->d_loss, 0, sizeof(float), ctx->stream));
  if (m->wtT_stale) {
    CUDA_OR_FAIL(ctx, launch_mlp_transpose_weights(m->d_wb, m->d_wtT, ctx->stream));
    m->wtT_stale = false;
  }
  const __nv_bfloat16* Wt2 = m->d_wtT;
  const __nv_bfloat16* Wt3 = m->d_wtT + 256 * 256;
  const __nv_bfloat16* Wt4 = m->d_wtT + 2 * 256 * 256;
  // weight gradients: K (the batch) split into one slice per SM's item; each slice's partial product is
  // added into m->d_g (zeroed above) by the GEMM's epilogue (TMA reduce-add, else atomics)
  const int ks = split_k(ctx, Bi, 2);
  auto weight_grad = [&](int M, int N, const __nv_bfloat16* At, const __nv_bfloat16* Bt, float* dst, long long scm,
                         long long scn) -> fpt_status {
    GemmArgs g = gemm_args(M, N, Bi, At, Bi, 1, Bt, Bi, 1, EPI_ATOMIC, ctx->d_err);
    g.C = dst;
    g.scm = scm;
    g.scn = scn;
    CUDA_OR_FAIL(ctx, launch_gemm(g, ks, ctx->stream));
    return FPT_OK;
  };
  fpt_status st = mlp_forward_impl(ctx, m, X, B, m->d_Y, true);
  if (st != FPT_OK) return st;
  if (!(m->xt_ready && X == m->d_Xb)) CUDA_OR_FAIL(ctx, launch_bf16_transpose(X, Bi, kMlpIn, m->d_Xt, ctx->stream));
  CUDA_OR_FAIL(ctx, launch_mlp_loss(G, m->d_Y, T, B, m->d_dY, m->d_dYb, m->d_dYt, m->d_loss, ctx->stream));
  // last layer: dW4^T [in][out] = H3^T dY (sum over the batch); db4 = sum_b dY
  st = weight_grad(kMlpHidden, kMlpOut, m->d_Ht3, m->d_dYt, m->d_g + kOffW4, 1, kMlpHidden);
  if (st != FPT_OK) return st;
  CUDA_OR_FAIL(ctx, launch_colsum(m->d_dY, B, kMlpOut, m->d_g + kOffB4, ctx->stream));
  // dZ3 = (dY W4) * gelu'(Z3), its transpose, and db3 = sum_b dZ3 (column sums in the epilogue)
  {
    GemmArgs g = gemm_args(Bi, kMlpHidden, kMlpOut, m->d_dYb, kMlpOut, 1, Wt4, kMlpOut, 1, EPI_GELU_GRAD, ctx->d_err);
    g.Zin = m->d_Z3;
    g.szm = kMlpHidden;
    g.szn = 1;
    g.colsum = m->d_g + kOffB3;
    g.H = m->d_dZa;
    g.shm = kMlpHidden;
    g.shn = 1;
    g.Ht = m->d_dZta;
    g.shtm = 1;
    g.shtn = Bi;
    CUDA_OR_FAIL(ctx, launch_gemm(g, 1, ctx->stream));
  }
  const __nv_bfloat16* acts_t[3] = {m->d_Xt, m->d_Ht1, m->d_Ht2};  // inputs of layers 1..3, transposed
  const __nv_bfloat16* wts[3] = {nullptr, Wt2, Wt3};
  const float* Zs[2] = {m->d_Z1, m->d_Z2};
  const int offW[3] = {kOffW1, kOffW2, kOffW3}, offB[3] = {kOffB1, kOffB2, kOffB3};
  __nv_bfloat16 *dZ = m->d_dZa, *dZn = m->d_dZb, *dZt = m->d_dZta, *dZtn = m->d_dZtb;
  for (int l = 2; l >= 0; --l) {
    const int K_in = l == 0 ? kMlpIn : kMlpHidden;
    // dW_l [out][in] = dZ^T [out][b] act^T [in][b]
    st = weight_grad(kMlpHidden, K_in, dZt, acts_t[l], m->d_g + offW[l], K_in, 1);
    if (st != FPT_OK) return st;
    if (l == 0) break;
    // dZ_{l-1} = (dZ_l W_l) * gelu'(Z_{l-1}) = dZ_l [b][out] (W_l^T)[in][out], its transpose and db_{l-1}
    GemmArgs gd = gemm_args(Bi, kMlpHidden, kMlpHidden, dZ, kMlpHidden, 1, wts[l], kMlpHidden, 1, EPI_GELU_GRAD,
                            ctx->d_err);
    gd.Zin = Zs[l - 1];
    gd.szm = kMlpHidden;
    gd.szn = 1;
    gd.colsum = m->d_g + offB[l - 1];
    gd.H = dZn;
    gd.shm = kMlpHidden;
    gd.shn = 1;
    gd.Ht = dZtn;
    gd.shtm = 1;
    gd.shtn = Bi;
    CUDA_OR_FAIL(ctx, launch_gemm(gd, 1, ctx->stream));
    std::swap(dZ, dZn);
    std::swap(dZt, dZtn);
  }
  return FPT_OK;
}

// splitmix64 stream for the initial weights
static uint64_t sm64_next(uint64_t& state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

extern "C" {

fpt_status fpt_mlp_create(fpt_ctx* ctx, uint64_t seed, float length_scale, fpt_mlp** out) {
  if (!ctx || !out) return fail(ctx, FPT_EINVAL, "null argument");
  *out = nullptr;
  if (!(length_scale > 0.f) || !std::isfinite(length_scale)) return fail(ctx, FPT_EINVAL, "bad length scale");
  fpt_mlp* m = new (std::nothrow) fpt_mlp();
  if (!m) return FPT_ENOMEM;
  m->ctx = ctx;
  m->scale = length_scale;
  m->seed = seed;
  cudaError_t e = cudaSetDevice(ctx->device);
  for (float** p : {&m->d_w, &m->d_m, &m->d_v, &m->d_g})
    if (e == cudaSuccess) e = cudaMalloc(p, kMlpParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_wb, kMlpParams * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_wt, kMlpTiledBytes);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_wtT, kMlpWtElems * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_loss, sizeof(float));
  if (e != cudaSuccess) {
    fpt_mlp_free(m);
    return fail(ctx, FPT_ENOMEM, "MLP parameters: %s", cudaGetErrorString(e));
  }
  std::vector<float> w(kMlpParams, 0.f);
  uint64_t state = seed;
  auto fill = [&](int off, int rows, int cols, int used_rows) {
    const double bound = 1.0 / std::sqrt((double)cols);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) {
        const double u = (double)(sm64_next(state) >> 11) * (1.0 / 9007199254740992.0);
        w[off + r * cols + c] = r < used_rows ? (float)((2.0 * u - 1.0) * bound) : 0.f;
      }
  };
  fill(kOffW1, 256, 64, 256);
  fill(kOffW2, 256, 256, 256);
  fill(kOffW3, 256, 256, 256);
  fill(kOffW4, 16, 256, 8);
  fpt_status st = fpt_mlp_set_params(m, w.data());
  if (st != FPT_OK) {
    fpt_mlp_free(m);
    return st;
  }
  *out = m;
  return FPT_OK;
}

void fpt_mlp_free(fpt_mlp* m) {
  if (!m) return;
  if (m->ctx && m->ctx->init_mlp == m) m->ctx->init_mlp = nullptr;
  mlp_free_ws(m);
  for (void* p : {(void*)m->d_w, (void*)m->d_m, (void*)m->d_v, (void*)m->d_g, (void*)m->d_wb, (void*)m->d_wt,
                  (void*)m->d_loss, (void*)m->d_Xb, (void*)m->d_Tb, (void*)m->d_Gb, (void*)m->d_hist, (void*)m->d_wtT})
    cudaFree(p);
  delete m;
}

fpt_status fpt_mlp_get_params(const fpt_mlp* m, float* host) {
  if (!m || !host) return FPT_EINVAL;
  fpt_ctx* ctx = m->ctx;
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_OR_FAIL(ctx, cudaMemcpy(host, m->d_w, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost));
  return FPT_OK;
}

fpt_status fpt_mlp_set_params(fpt_mlp* m, const float* host) {
  if (!m || !host) return FPT_EINVAL;
  fpt_ctx* ctx = m->ctx;
  for (int i = 0; i < kMlpParams; ++i)
    if (!std::isfinite(host[i])) return fail(ctx, FPT_EINVAL, "non-finite parameter %d", i);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_OR_FAIL(ctx, cudaMemcpy(m->d_w, host, kMlpParams * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_OR_FAIL(ctx, cudaMemset(m->d_m, 0, kMlpParams * sizeof(float)));
  CUDA_OR_FAIL(ctx, cudaMemset(m->d_v, 0, kMlpParams * sizeof(float)));
  CUDA_OR_FAIL(ctx, launch_to_bf16(m->d_w, m->d_wb, kMlpParams, ctx->stream));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  m->step = 0;
  m->wt_stale = true;
  m->wtT_stale = true;
  return FPT_OK;
}

static const char kMlpMagic[8] = {'F', 'P', 'T', 'M', 'L', 'P', '0', '1'};

fpt_status fpt_mlp_save(const fpt_mlp* m, const char* path) {
  if (!m || !path) return FPT_EINVAL;
  fpt_ctx* ctx = m->ctx;
  std::vector<float> buf(3 * (size_t)kMlpParams);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_OR_FAIL(ctx, cudaMemcpy(buf.data(), m->d_w, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost));
  CUDA_OR_FAIL(ctx, cudaMemcpy(buf.data() + kMlpParams, m->d_m, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost));
  CUDA_OR_FAIL(ctx, cudaMemcpy(buf.data() + 2 * kMlpParams, m->d_v, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ctx, FPT_EINVAL, "cannot write %s", path);
  const int32_t n = kMlpParams;
  bool ok = fwrite(kMlpMagic, 1, 8, f) == 8 && fwrite(&n, 4, 1, f) == 1 && fwrite(&m->scale, 4, 1, f) == 1 &&
            fwrite(&m->seed, 8, 1, f) == 1 && fwrite(&m->step, 8, 1, f) == 1 &&
            fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? FPT_OK : fail(ctx, FPT_EINVAL, "short write to %s", path);
}

fpt_status fpt_mlp_load(fpt_ctx* ctx, const char* path, fpt_mlp** out) {
  if (!ctx || !path || !out) return fail(ctx, FPT_EINVAL, "null argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(ctx, FPT_EINVAL, "cannot read %s", path);
  char magic[8];
  int32_t n = 0;
  float scale = 0.f;
  uint64_t seed = 0;
  int64_t step = 0;
  std::vector<float> buf(3 * (size_t)kMlpParams);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMlpMagic, 8) == 0 && fread(&n, 4, 1, f) == 1 &&
            n == kMlpParams && fread(&scale, 4, 1, f) == 1 && fread(&seed, 8, 1, f) == 1 &&
            fread(&step, 8, 1, f) == 1 && fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  fclose(f);
  if (!ok) return fail(ctx, FPT_EINVAL, "%s is not a network file of this version", path);
  fpt_mlp* m = nullptr;
  fpt_status st = fpt_mlp_create(ctx, seed, scale, &m);
  if (st != FPT_OK) return st;
  st = fpt_mlp_set_params(m, buf.data());
  if (st == FPT_OK) {
    cudaError_t e = cudaMemcpy(m->d_m, buf.data() + kMlpParams, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(m->d_v, buf.data() + 2 * kMlpParams, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = fail(ctx, FPT_ECUDA, "%s", cudaGetErrorString(e));
  }
  if (st != FPT_OK) {
    fpt_mlp_free(m);
    return st;
  }
  m->step = step;
  *out = m;
  return FPT_OK;
}

fpt_status fpt_mlp_features(fpt_ctx* ctx, const fpt_mlp* m, const fpt_scene* s, const fpt_batch* b, void* X,
                            float* G) {
  fpt_status st = check_scene_batch(ctx, s, b);
  if (st != FPT_OK) return st;
  if (!m || !X) return fail(ctx, FPT_EINVAL, "null argument");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  ProfScope ps(ctx, FPT_K_OTHER);
  CUDA_OR_FAIL(ctx, launch_mlp_features(scene_dev(s), b->dev, 0, nullptr, 0, b->dev.n_paths, 1.f / m->scale,
                                        static_cast<__nv_bfloat16*>(X), G, ctx->stream));
  return FPT_OK;
}

fpt_status fpt_mlp_forward(fpt_ctx* ctx, fpt_mlp* m, const void* X, uint64_t B, float* Y) {
  if (!ctx || !m || !X || !Y) return fail(ctx, FPT_EINVAL, "null argument");
  if (B < 1 || B > (1ull << 30)) return fail(ctx, FPT_EINVAL, "bad batch size");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  fpt_status st = mlp_ensure_ws(ctx, m, B, false);
  if (st != FPT_OK) return st;
  ProfScope ps(ctx, FPT_K_OTHER);
  return mlp_forward_impl(ctx, m, static_cast<const __nv_bfloat16*>(X), B, Y, false);
}

fpt_status fpt_mlp_loss_grad(fpt_ctx* ctx, fpt_mlp* m, const void* X, const float* T, const float* G, uint64_t B,
                             float* loss, float* grad_out) {
  if (!ctx || !m || !X || !T || !G) return fail(ctx, FPT_EINVAL, "null argument");
  if (B < 1 || B > (1ull << 30)) return fail(ctx, FPT_EINVAL, "bad batch size");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  fpt_status st = mlp_ensure_ws(ctx, m, B, true);
  if (st != FPT_OK) return st;
  st = mlp_backward_impl(ctx, m, static_cast<const __nv_bfloat16*>(X), T, G, B);
  if (st != FPT_OK) return st;
  if (grad_out)
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(grad_out, m->d_g, kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  if (loss) {
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return FPT_OK;
}

fpt_status fpt_mlp_train_step(fpt_ctx* ctx, fpt_mlp* m, const void* X, const float* T, const float* G, uint64_t B,
                              float lr, float* loss) {
  if (!(lr > 0.f)) return fail(ctx, FPT_EINVAL, "learning rate must be positive");
  fpt_status st = fpt_mlp_loss_grad(ctx, m, X, T, G, B, nullptr, nullptr);
  if (st != FPT_OK) return st;
  m->step += 1;
  const float c1 = 1.f - std::pow(0.9f, (float)m->step), c2 = 1.f - std::pow(0.999f, (float)m->step);
  CUDA_OR_FAIL(ctx, launch_adam(m->d_w, m->d_m, m->d_v, m->d_g, kMlpParams, lr, c1, c2, m->d_wb, ctx->stream));
  m->wt_stale = true;
  m->wtT_stale = true;
  if (loss) {
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return FPT_OK;
}

fpt_status fpt_mlp_train(fpt_ctx* ctx, fpt_mlp* m, const void* X, const float* T, const float* G, uint64_t n,
                         const fpt_train_params* prm, float* loss_per_epoch) {
  if (!ctx || !m || !prm) return fail(ctx, FPT_EINVAL, "null argument");
  if (m->ctx != ctx) return fail(ctx, FPT_EINVAL, "network belongs to another context");
  const fpt_train_params p = *prm;
  if (p.epochs < 1 || p.batch < 128 || !(p.lr > 0.f) || !(p.lr_decay > 0.f))
    return fail(ctx, FPT_EINVAL, "fpt_mlp_train: epochs >= 1, batch >= 128, lr > 0 and lr_decay > 0 required");
  if ((uint64_t)p.batch > n) return fail(ctx, FPT_EINVAL, "fpt_mlp_train: fewer samples (%llu) than one batch",
                                         (unsigned long long)n);
  if (!X || !T || !G) return fail(ctx, FPT_EINVAL, "fpt_mlp_train: X, T and G are required");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  const uint64_t B = (uint64_t)p.batch;
  fpt_status st = mlp_ensure_ws(ctx, m, B, true);
  if (st != FPT_OK) return st;
  if (B > m->train_cap || (size_t)p.epochs > m->hist_cap) {
    cudaFree(m->d_Xb);
    cudaFree(m->d_Tb);
    cudaFree(m->d_Gb);
    cudaFree(m->d_hist);
    m->d_Xb = nullptr;
    m->d_Tb = m->d_Gb = m->d_hist = nullptr;
    m->train_cap = m->hist_cap = 0;
    cudaError_t e = cudaMalloc(&m->d_Xb, B * kMlpIn * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_Tb, B * 8 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_Gb, B * 12 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_hist, (size_t)p.epochs * sizeof(float));
    if (e != cudaSuccess) return fail(ctx, FPT_ENOMEM, "fpt_mlp_train: batch buffers: %s", cudaGetErrorString(e));
    m->train_cap = B;
    m->hist_cap = (size_t)p.epochs;
  }
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(m->d_hist, 0, (size_t)p.epochs * sizeof(float), ctx->stream));
  const uint64_t steps = n / B;  // the last partial batch of every epoch is left out
  const __nv_bfloat16* Xs = static_cast<const __nv_bfloat16*>(X);
  float lr = p.lr;
  for (int ep = 0; ep < p.epochs; ++ep) {
    // a new seeded order of the samples every epoch (splitmix64 of seed and epoch)
    uint64_t s0 = p.seed + 0x9E3779B97F4A7C15ULL * (uint64_t)(ep + 1);
    const uint64_t key = sm64_next(s0);
    for (uint64_t k = 0; k < steps; ++k) {
      CUDA_OR_FAIL(ctx, launch_mlp_gather(Xs, T, G, n, k * B, B, key, m->d_Xb, m->d_Tb, m->d_Gb, m->d_Xt,
                                          ctx->stream));
      m->xt_ready = true;
      st = fpt_mlp_train_step(ctx, m, m->d_Xb, m->d_Tb, m->d_Gb, B, lr, nullptr);
      m->xt_ready = false;
      if (st != FPT_OK) return st;
      CUDA_OR_FAIL(ctx, launch_mlp_accumulate(m->d_hist + ep, m->d_loss, 1.f / (float)steps, ctx->stream));
    }
    lr *= p.lr_decay;
  }
  if (loss_per_epoch) {
    CUDA_OR_FAIL(ctx, cudaMemcpyAsync(loss_per_epoch, m->d_hist, (size_t)p.epochs * sizeof(float),
                                      cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return FPT_OK;
}

fpt_status fpt_mlp_infer(fpt_ctx* ctx, fpt_mlp* m, const fpt_scene* s, const fpt_batch* bc, float* T) {
  fpt_status st = check_scene_batch(ctx, s, bc);
  if (st != FPT_OK) return st;
  if (!m) return fail(ctx, FPT_EINVAL, "null network");
  if (m->ctx != ctx) return fail(ctx, FPT_EINVAL, "network belongs to another context");
  if (!T && bc->dev.n_paths > 0) return fail(ctx, FPT_EINVAL, "T_out is required");
  fpt_batch* b = const_cast<fpt_batch*>(bc);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_buckets(ctx, b, scene_dev(s));
  if (st != FPT_OK) return st;
  const SceneDev S = scene_dev(s);
  if (b->dev.n_paths == 0) return FPT_OK;
  // slots past a path's order stay zero
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(T, 0, b->dev.n_paths * (uint64_t)b->dev.n_max * 2 * sizeof(float), ctx->stream));
  if (m->wt_stale) {
    CUDA_OR_FAIL(ctx, launch_mlp_tile_weights(m->d_wb, m->d_wt, ctx->stream));
    m->wt_stale = false;
  }
  for (int n = 1; n <= kMaxOrder; ++n) {
    const PathRec* list;
    const uint64_t cnt = order_slice(b, n, &list);
    if (!cnt) continue;
    ProfScope ps(ctx, FPT_K_MLP);
    CUDA_OR_FAIL(ctx, launch_mlp_infer(S, b->dev, n, list, cnt, 1.f / m->scale, m->d_wt, m->d_w, T, ctx->d_err,
                                       ctx->stream, ctx->n_sm));
  }
  return FPT_OK;
}

fpt_status fpt_set_init_mlp(fpt_ctx* ctx, fpt_mlp* m) {
  if (!ctx) return FPT_EINVAL;
  if (m && m->ctx != ctx) return fail(ctx, FPT_EINVAL, "network belongs to another context");
  ctx->init_mlp = m;
  return FPT_OK;
}

fpt_status fpt_tc_gemm_bf16(fpt_ctx* ctx, int32_t M, int32_t N, int32_t K, const void* A, const void* W,
                            const float* bias, float* C) {
  if (!ctx || !A || !W || !C) return fail(ctx, FPT_EINVAL, "null argument");
  if (M < 1 || K < 1 || N < 1 || N > 256) return fail(ctx, FPT_EINVAL, "bad GEMM shape %d x %d x %d", M, N, K);
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.A = static_cast<const __nv_bfloat16*>(A);
  g.sam = K;
  g.sak = 1;
  g.B = static_cast<const __nv_bfloat16*>(W);
  g.sbn = K;
  g.sbk = 1;
  g.op = EPI_STORE;
  g.bias = bias;
  g.C = C;
  g.scm = N;
  g.scn = 1;
  g.err = ctx->d_err;
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  ProfScope ps(ctx, FPT_K_OTHER);
  CUDA_OR_FAIL(ctx, launch_gemm(g, 1, ctx->stream));
  return FPT_OK;
}

fpt_status fpt_check_bounded_wait(fpt_ctx* ctx, uint32_t limit_us, int arrive, uint64_t* elapsed_ns) {
  if (!ctx) return FPT_EINVAL;
  if (limit_us < 1 || limit_us > 1000000u) return fail(ctx, FPT_EINVAL, "limit %u us outside [1, 10^6]", limit_us);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  unsigned long long* d_ns = nullptr;
  if (elapsed_ns) CUDA_OR_FAIL(ctx, cudaMalloc(&d_ns, sizeof(unsigned long long)));
  cudaError_t e;
  {
    ProfScope ps(ctx, FPT_K_OTHER);
    e = launch_bounded_wait_check(limit_us * 1000u, arrive, ctx->d_err, d_ns, ctx->stream);
  }
  unsigned long long h = 0;
  if (e == cudaSuccess && elapsed_ns) {
    e = cudaMemcpyAsync(&h, d_ns, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  if (d_ns) cudaFree(d_ns);
  CUDA_OR_FAIL(ctx, e);
  if (elapsed_ns) *elapsed_ns = h;
  return FPT_OK;
}

fpt_status fpt_profile_enable(fpt_ctx* ctx, int on) {
  if (!ctx) return FPT_EINVAL;
  ctx->prof = on != 0;
  return FPT_OK;
}

fpt_status fpt_profile_read(fpt_ctx* ctx, double* ms, uint64_t* launches, int reset) {
  if (!ctx) return FPT_EINVAL;
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto& p : ctx->ev_pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.second.first, p.second.second) == cudaSuccess) ctx->prof_ms[p.first] += t;
    ctx->ev_pool.push_back(p.second.first);
    ctx->ev_pool.push_back(p.second.second);
  }
  ctx->ev_pending.clear();
  for (int k = 0; k < FPT_K_COUNT; ++k) {
    if (ms) ms[k] = ctx->prof_ms[k];
    if (launches) launches[k] = ctx->prof_kernels[k];
    if (reset) {
      ctx->prof_ms[k] = 0;
      ctx->prof_kernels[k] = 0;
    }
  }
  return FPT_OK;
}

}  // extern "C"
