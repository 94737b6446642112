// fpt_api.cu -- host implementation of the C ABI declared in include/fpt.h.
//
// Owns contexts (device, stream, error word, workspace), scenes (object
// records built in FP64 on the host, recentred, split into FP32 hi/lo parts
// and uploaded) and batches (candidate-sequence descriptions; seeded and
// explicit batches are bucketed by order on the device once, so that every
// solver launch is specialised to one order).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fpt.h"
#include "fpt_kernels.h"
#include "mlp.h"

using namespace fpt;

struct fpt_ctx {
  int device = 0;
  int n_sm = 0;
  cudaStream_t stream = nullptr;
  int* d_err = nullptr;                    // device error word
  double* d_gacc = nullptr;                // backward accumulators (FP64)
  size_t gacc_cap = 0;
  unsigned long long* d_count = nullptr;   // counters for reductions
  unsigned long long* d_work = nullptr;    // work counter of the lane-refill solver
  uint32_t* d_rescue = nullptr;            // paths whose FP32 Hessian pivots failed (polish scratch)
  size_t rescue_cap = 0;
  unsigned* d_rescue_n = nullptr;
  char msg[512] = "ok";
  // kernel timing
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double prof_ms[FPT_K_COUNT] = {0, 0, 0, 0};
  uint64_t prof_n[FPT_K_COUNT] = {0, 0, 0, 0};
};

// Event pair around one launch when timing is on.
struct ProfScope {
  fpt_ctx* ctx;
  int cls;
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
    a = take(ctx);
    b = take(ctx);
    if (a) cudaEventRecord(a, ctx->stream);
  }
  ~ProfScope() {
    if (!ctx->prof || !a || !b) return;
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
};

struct fpt_batch {
  fpt_ctx* ctx = nullptr;
  BatchDev dev{};
  int32_t* d_alphabet = nullptr;
  // order buckets of seeded / explicit batches (built on first use)
  bool bucketed = false;
  uint64_t* d_lists = nullptr;
  uint64_t count[kMaxOrder + 1] = {0};
  uint64_t start[kMaxOrder + 1] = {0};
};

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
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_count, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_work, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_rescue_n, sizeof(unsigned));
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
  cudaFree(ctx->d_rescue);
  cudaFree(ctx->d_rescue_n);
  delete ctx;
}

fpt_status fpt_set_stream(fpt_ctx* ctx, void* cuda_stream) {
  if (!ctx) return FPT_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return FPT_OK;
}

const char* fpt_last_error(const fpt_ctx* ctx) { return ctx ? ctx->msg : "null context"; }

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
  std::vector<float> rec32((size_t)n_obj * kRec32), aux((size_t)n_obj * kAux), reclo((size_t)n_obj * kRecLo);
  std::vector<double> rec64((size_t)n_obj * kRec64);
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
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_rec32, rec32.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_rec64, rec64.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_aux, aux.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_reclo, reclo.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(s->d_reclo, reclo.data(), reclo.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_rec32, rec32.data(), rec32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_rec64, rec64.data(), rec64.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_aux, aux.data(), aux.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    fpt_scene_free(s);
    return fail(ctx, FPT_ECUDA, "scene upload: %s", cudaGetErrorString(e));
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
  delete s;
}

static cudaError_t upload_points(const double* p, int n, const double* centre, float** d32, double** d64) {
  std::vector<float> h32((size_t)n * kEnd32);
  std::vector<double> h64((size_t)n * 3);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) {
      double x = p[3 * i + c] - centre[c];
      h64[3 * i + c] = x;
      split(x, h32[kEnd32 * i + c], h32[kEnd32 * i + 3 + c]);
    }
  cudaFree(*d32);
  cudaFree(*d64);
  *d32 = nullptr;
  *d64 = nullptr;
  cudaError_t e = cudaMalloc(d32, h32.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(d64, h64.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(*d32, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(*d64, h64.data(), h64.size() * sizeof(double), cudaMemcpyHostToDevice);
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
  CUDA_OR_FAIL(ctx, upload_points(tx, n_tx, s->centre, &s->d_tx32, &s->d_tx64));
  CUDA_OR_FAIL(ctx, upload_points(rx, n_rx, s->centre, &s->d_rx32, &s->d_rx64));
  s->n_tx = n_tx;
  s->n_rx = n_rx;
  return FPT_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
static fpt_status make_alphabet(fpt_ctx* ctx, const fpt_scene* s, const int32_t* alphabet, int32_t n_alpha,
                                fpt_batch* b) {
  std::vector<int32_t> a;
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
  CUDA_OR_FAIL(ctx, cudaMemcpy(b->d_alphabet, a.data(), a.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  b->dev.alphabet = b->d_alphabet;
  b->dev.n_alpha = (int)a.size();
  return FPT_OK;
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
  *out = b;
  return FPT_OK;
}

fpt_status fpt_batch_explicit(fpt_ctx* ctx, const fpt_scene* s, const int32_t* ids_dev, const uint8_t* order_dev,
                              const int32_t* tx_idx_dev, const int32_t* rx_idx_dev, uint64_t n, int32_t n_max,
                              fpt_batch** out) {
  if (!ctx || !s || !out || !ids_dev || !order_dev || !tx_idx_dev || !rx_idx_dev)
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

// Bucket a seeded/explicit batch by order (once per batch; synchronous).
static fpt_status ensure_buckets(fpt_ctx* ctx, fpt_batch* b) {
  if (b->dev.mode == BATCH_EXHAUSTIVE || b->bucketed) return FPT_OK;
  unsigned long long h[kMaxOrder + 1] = {0};
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->d_count, 0, 8 * sizeof(unsigned long long), ctx->stream));
  CUDA_OR_FAIL(ctx, launch_order_histogram(b->dev, ctx->d_count, ctx->stream, ctx->n_sm));
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(h, ctx->d_count, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  uint64_t acc = 0;
  unsigned long long cur[kMaxOrder + 1];
  for (int n = 0; n <= kMaxOrder; ++n) {
    b->start[n] = acc;
    b->count[n] = h[n];
    cur[n] = acc;
    acc += h[n];
  }
  if (acc != b->dev.n_paths) return fail(ctx, FPT_EDEVICE, "order histogram mismatch");
  CUDA_OR_FAIL(ctx, cudaMalloc(&b->d_lists, (acc ? acc : 1) * sizeof(uint64_t)));
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(ctx->d_count, cur, sizeof(cur), cudaMemcpyHostToDevice, ctx->stream));
  CUDA_OR_FAIL(ctx, launch_order_scatter(b->dev, ctx->d_count, b->d_lists, ctx->stream, ctx->n_sm));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  b->bucketed = true;
  return FPT_OK;
}

// Polish scratch: one uint32 per path of the largest order slice.
static fpt_status ensure_rescue(fpt_ctx* ctx, uint64_t n) {
  if (n <= ctx->rescue_cap) return FPT_OK;
  cudaFree(ctx->d_rescue);
  ctx->d_rescue = nullptr;
  ctx->rescue_cap = 0;
  CUDA_OR_FAIL(ctx, cudaMalloc(&ctx->d_rescue, n * sizeof(uint32_t)));
  ctx->rescue_cap = n;
  return FPT_OK;
}

// Paths of order n in a batch: count and list (nullptr for exhaustive batches).
static uint64_t order_slice(const fpt_batch* b, int n, const uint64_t** list) {
  if (b->dev.mode == BATCH_EXHAUSTIVE) {
    *list = nullptr;
    if (n < b->dev.lo || n > b->dev.hi) return 0;
    return b->dev.kpow[n] * (uint64_t)b->dev.n_tx * (uint64_t)b->dev.n_rx;
  }
  *list = b->d_lists + b->start[n];
  return b->count[n];
}

static fpt_status check_scene_batch(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* b) {
  if (!ctx || !s || !b) return fail(ctx, FPT_EINVAL, "null argument");
  if (b->dev.n_tx != s->n_tx || b->dev.n_rx != s->n_rx)
    return fail(ctx, FPT_EINVAL, "batch was built for other endpoints");
  if (b->dev.mode == BATCH_EXPLICIT && b->dev.n_alpha != s->n_obj) return fail(ctx, FPT_EINVAL, "batch/scene mismatch");
  return FPT_OK;
}

fpt_status fpt_solve(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* bc, const fpt_solve_params* prm, float* T,
                     float* X, float* L, uint8_t* status, uint8_t* iters, float* rho) {
  fpt_status st = check_scene_batch(ctx, s, bc);
  if (st != FPT_OK) return st;
  if (!T || !status) return fail(ctx, FPT_EINVAL, "T_out and status_out are required");
  fpt_solve_params p;
  fpt_default_params(&p);
  if (prm) p = *prm;
  if (p.init_mode != 0) return fail(ctx, FPT_EUNSUPPORTED, "learned init is not available in this build");
  if (p.max_iters < 0 || p.fp_iters < 1 || p.polish < 0 || p.polish > 2)
    return fail(ctx, FPT_EINVAL, "bad solver parameters");
  fpt_batch* b = const_cast<fpt_batch*>(bc);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_buckets(ctx, b);
  if (st != FPT_OK) return st;
  const SceneDev S = scene_dev(s);
  SolveCfg sc{p.max_iters, p.fp_iters, p.fixed_iters, p.tol_step * p.tol_step, 0.01f * p.deg_tol * p.deg_tol,
              p.refill > 32 ? 32 : p.refill};
  PolishCfg pc{POLISH_SOLVE, p.polish, p.solved_tol, p.deg_tol, p.cond_fp64, p.polish_fp64};
  for (int n = 1; n <= kMaxOrder; ++n) {
    const uint64_t* list;
    uint64_t cnt = order_slice(b, n, &list);
    if (!cnt) continue;
    {
      ProfScope ps(ctx, FPT_K_BFGS);
      CUDA_OR_FAIL(ctx, launch_bfgs(n, S, b->dev, sc, cnt, list, T, status, iters, ctx->stream, ctx->n_sm, ctx->d_work));
    }
    if (cnt > 0xFFFFFFFFull) return fail(ctx, FPT_EUNSUPPORTED, "more than 2^32 paths of one order");
    st = ensure_rescue(ctx, cnt);
    if (st != FPT_OK) return st;
    {
      ProfScope ps(ctx, FPT_K_POLISH);
      CUDA_OR_FAIL(ctx, launch_polish(n, S, b->dev, pc, cnt, list, T, X, L, status, rho, nullptr, nullptr, ctx->stream,
                                      ctx->n_sm, ctx->d_rescue, ctx->d_rescue_n));
    }
  }
  return FPT_OK;
}

fpt_status fpt_validity(fpt_ctx* ctx, const fpt_scene* s, const fpt_batch* bc, const float* T, uint8_t* mask,
                        float* bdist, float* rho) {
  fpt_status st = check_scene_batch(ctx, s, bc);
  if (st != FPT_OK) return st;
  if (!T) return fail(ctx, FPT_EINVAL, "T is required");
  fpt_batch* b = const_cast<fpt_batch*>(bc);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_buckets(ctx, b);
  if (st != FPT_OK) return st;
  fpt_solve_params p;
  fpt_default_params(&p);
  const SceneDev S = scene_dev(s);
  PolishCfg pc{POLISH_VALIDITY, 0, p.solved_tol, p.deg_tol, p.cond_fp64, 0};
  for (int n = 1; n <= kMaxOrder; ++n) {
    const uint64_t* list;
    uint64_t cnt = order_slice(b, n, &list);
    if (!cnt) continue;
    if (cnt > 0xFFFFFFFFull) return fail(ctx, FPT_EUNSUPPORTED, "more than 2^32 paths of one order");
    st = ensure_rescue(ctx, cnt);
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
  if (!T) return fail(ctx, FPT_EINVAL, "T is required");
  fpt_batch* b = const_cast<fpt_batch*>(bc);
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  st = ensure_buckets(ctx, b);
  if (st != FPT_OK) return st;
  const size_t need = (size_t)(9 * s->n_obj + 3 * (s->n_tx + s->n_rx));
  if (need > ctx->gacc_cap) {
    cudaFree(ctx->d_gacc);
    ctx->d_gacc = nullptr;
    ctx->gacc_cap = 0;
    CUDA_OR_FAIL(ctx, cudaMalloc(&ctx->d_gacc, need * sizeof(double)));
    ctx->gacc_cap = need;
  }
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->d_gacc, 0, need * sizeof(double), ctx->stream));
  const SceneDev S = scene_dev(s);
  fpt_solve_params p;
  fpt_default_params(&p);
  if (!dL && dL_status_mask && !status) return fail(ctx, FPT_EINVAL, "dL_status_mask needs status");
  BackwardCfg bc_cfg{p.cond_fp64, p.deg_tol, 1, 64, dL ? (uint8_t)0 : dL_status_mask};
  for (int n = 1; n <= kMaxOrder; ++n) {
    const uint64_t* list;
    uint64_t cnt = order_slice(b, n, &list);
    if (!cnt) continue;
    if (cnt > 0xFFFFFFFFull) return fail(ctx, FPT_EUNSUPPORTED, "more than 2^32 paths of one order");
    st = ensure_rescue(ctx, cnt);
    if (st != FPT_OK) return st;
    ProfScope ps(ctx, FPT_K_BACKWARD);
    CUDA_OR_FAIL(ctx, launch_backward(n, S, b->dev, bc_cfg, cnt, list, T, status, dX, dL, ctx->d_gacc, ctx->stream,
                                      ctx->n_sm, ctx->d_rescue, ctx->d_rescue_n));
  }
  {
    ProfScope ps(ctx, FPT_K_OTHER);
    CUDA_OR_FAIL(ctx, launch_backward_finalize(S, nullptr, ctx->d_gacc, g_tx, g_rx, g_vertices, ctx->stream));
  }
  return FPT_OK;
}

fpt_status fpt_count_status(fpt_ctx* ctx, const uint8_t* status, uint64_t n, uint8_t mask, uint64_t* count) {
  if (!ctx || !status || !count) return fail(ctx, FPT_EINVAL, "null argument");
  CUDA_OR_FAIL(ctx, cudaSetDevice(ctx->device));
  unsigned long long h = 0;
  CUDA_OR_FAIL(ctx, cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned long long), ctx->stream));
  CUDA_OR_FAIL(ctx, launch_count_status(status, n, mask, ctx->d_count, ctx->stream, ctx->n_sm));
  CUDA_OR_FAIL(ctx, cudaMemcpyAsync(&h, ctx->d_count, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_OR_FAIL(ctx, cudaStreamSynchronize(ctx->stream));
  *count = h;
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
    if (cudaEventElapsedTime(&t, p.second.first, p.second.second) == cudaSuccess) {
      ctx->prof_ms[p.first] += t;
      ctx->prof_n[p.first] += 1;
    }
    ctx->ev_pool.push_back(p.second.first);
    ctx->ev_pool.push_back(p.second.second);
  }
  ctx->ev_pending.clear();
  for (int k = 0; k < FPT_K_COUNT; ++k) {
    if (ms) ms[k] = ctx->prof_ms[k];
    if (launches) launches[k] = ctx->prof_n[k];
    if (reset) {
      ctx->prof_ms[k] = 0;
      ctx->prof_n[k] = 0;
    }
  }
  return FPT_OK;
}

}  // extern "C"
