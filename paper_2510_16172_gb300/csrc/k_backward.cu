// k_backward.cu -- backward launch dispatch by order, the vertex chain rule, and the
// backward without allocation.  The per-path kernels are in backward.cuh; orders
// above the BFGS orders are instantiated in k_high.cu.
#include <mutex>

#include "backward.cuh"

namespace fpt {

extern template struct BackwardOrder<6>;
extern template struct BackwardOrder<7>;
extern template struct BackwardOrder<8>;
extern template struct BackwardOrder<9>;
extern template struct BackwardOrder<10>;

// Vertex chain rule and FP64 -> FP32.
__global__ void backward_finalize_kernel(int n_obj, int n_tx, int n_rx, const float* __restrict__ aux,
                                         const double* __restrict__ gacc, float* g_tx, float* g_rx, float* g_vert) {
  const int total = n_obj + n_tx + n_rx;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    if (k < n_obj) {
      if (!g_vert) continue;
      const double* s = gacc + 9 * k;
      const bool edge = aux[kAux * k + 2] != 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double gbv = s[c], ga1 = s[3 + c], ga2 = edge ? 0.0 : s[6 + c];
        g_vert[9 * k + c] = (float)(gbv - ga1 - ga2);
        g_vert[9 * k + 3 + c] = (float)ga1;
        g_vert[9 * k + 6 + c] = (float)ga2;
      }
    } else if (k < n_obj + n_tx) {
      const int i = k - n_obj;
      if (g_tx)
        for (int c = 0; c < 3; ++c) g_tx[3 * i + c] = (float)gacc[9 * n_obj + 3 * i + c];
    } else {
      const int i = k - n_obj - n_tx;
      if (g_rx)
        for (int c = 0; c < 3; ++c) g_rx[3 * i + c] = (float)gacc[9 * n_obj + 3 * n_tx + 3 * i + c];
    }
  }
}


cudaError_t launch_backward_rescue(int n, const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg,
                                   uint64_t n_local, const PathRec* list, const float* T, const uint8_t* status,
                                   const float* dX, const float* dL, double* gacc, cudaStream_t stream, int n_sm,
                                   const uint32_t* rescue_list, const unsigned* rescue_count) {
  switch (n) {
#define FPT_RESCUE_CASE(K) \
  case K:                  \
    return BackwardOrder<K>::rescue(S, B, cfg, n_local, list, T, status, dX, dL, gacc, stream, n_sm, rescue_list, rescue_count);
    FPT_RESCUE_CASE(1)
    FPT_RESCUE_CASE(2)
    FPT_RESCUE_CASE(3)
    FPT_RESCUE_CASE(4)
    FPT_RESCUE_CASE(5)
    FPT_RESCUE_CASE(6)
    FPT_RESCUE_CASE(7)
    FPT_RESCUE_CASE(8)
    FPT_RESCUE_CASE(9)
    FPT_RESCUE_CASE(10)
#undef FPT_RESCUE_CASE
    default: return cudaErrorInvalidValue;
  }
}


cudaError_t launch_backward(int n, const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg, uint64_t n_local,
                            const PathRec* list, const float* T, const uint8_t* status, const float* dX,
                            const float* dL, double* gacc, cudaStream_t stream, int n_sm, uint32_t* rescue_list,
                            unsigned* rescue_count) {
  switch (n) {
#define FPT_BWD_CASE(K)                                                                                    \
  case K:                                                                                                  \
    return BackwardOrder<K>::launch(S, B, cfg, n_local, list, T, status, dX, dL, gacc, stream, n_sm, rescue_list, \
                                    rescue_count);
    FPT_BWD_CASE(1)
    FPT_BWD_CASE(2)
    FPT_BWD_CASE(3)
    FPT_BWD_CASE(4)
    FPT_BWD_CASE(5)
    FPT_BWD_CASE(6)
    FPT_BWD_CASE(7)
    FPT_BWD_CASE(8)
    FPT_BWD_CASE(9)
    FPT_BWD_CASE(10)
#undef FPT_BWD_CASE
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Fixed scratch for callers that cannot allocate device memory.
//
// One file-scope array holds the FP64 gradient accumulators, the counter and
// the list of the FP64 pass.  It exists once per GPU that loads the library
// and lives until the process exits.  Host code must not pass the symbol
// itself to a kernel (on the host it names a host-side stand-in): its device
// address is looked up with cudaGetSymbolAddress, with that device current,
// whenever a context is created on the device (noalloc_lookup), and cached; a
// device reset can move the array, and the next context looks it up again.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocAccBytes = (size_t)kNoAllocMaxAcc * sizeof(double);
constexpr size_t kNoAllocCountBytes = 256;
constexpr size_t kNoAllocBytes = kNoAllocAccBytes + kNoAllocCountBytes + (size_t)kNoAllocMaxSlice * sizeof(uint32_t);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// The calling thread has `device` current.
cudaError_t noalloc_lookup(int device) {
  if (device < 0 || device >= kNoAllocMaxDevices) return cudaSuccess;  // such devices cannot use the array
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_noalloc_addr[device] = p;
  return cudaSuccess;
}

static cudaError_t noalloc_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_addr[device]) {
      *out = static_cast<unsigned char*>(g_noalloc_addr[device]);
      return cudaSuccess;
    }
  }
  cudaError_t e = noalloc_lookup(device);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  *out = static_cast<unsigned char*>(g_noalloc_addr[device]);
  return cudaSuccess;
}

cudaError_t launch_backward_noalloc(int device, const SceneDev& S, const BatchDev& B, const BackwardCfg& cfg,
                                    const PathRec* const* lists, const uint64_t* counts, const float* T,
                                    const uint8_t* status, const float* dX, const float* dL, float* g_tx, float* g_rx,
                                    float* g_vertices, cudaStream_t stream, int n_sm) {
  unsigned char* base = nullptr;
  cudaError_t e = noalloc_scratch(device, &base);
  if (e != cudaSuccess) return e;
  double* acc = reinterpret_cast<double*>(base);
  unsigned* count = reinterpret_cast<unsigned*>(base + kNoAllocAccBytes);
  uint32_t* list = reinterpret_cast<uint32_t*>(base + kNoAllocAccBytes + kNoAllocCountBytes);
  const size_t need = (size_t)(9 * S.n_obj + 3 * (S.n_tx + S.n_rx));
  // the array keeps the previous call's sums: clear them
  e = cudaMemsetAsync(acc, 0, need * sizeof(double), stream);
  if (e != cudaSuccess) return e;
  for (int n = 1; n <= kMaxOrder; ++n) {
    if (!counts[n]) continue;
    e = launch_backward(n, S, B, cfg, counts[n], lists[n], T, status, dX, dL, acc, stream, n_sm, list, count);
    if (e != cudaSuccess) return e;
  }
  return launch_backward_finalize(S, nullptr, acc, g_tx, g_rx, g_vertices, stream);
}

cudaError_t launch_backward_finalize(const SceneDev& S, const uint8_t* types, const double* gacc, float* g_tx,
                                     float* g_rx, float* g_vertices, cudaStream_t stream) {
  (void)types;
  const int total = S.n_obj + S.n_tx + S.n_rx;
  const int grid = (total + 255) / 256;
  backward_finalize_kernel<<<grid, 256, 0, stream>>>(S.n_obj, S.n_tx, S.n_rx, S.aux, gacc, g_tx, g_rx, g_vertices);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fpt
