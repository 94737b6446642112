// k_misc.cu -- sequence enumeration (Sec. III), bucketing by order and pattern, status counts.
#include "fpt_kernels.h"

namespace fpt {

thread_local uint64_t tl_kernel_launches = 0;

static unsigned grid_for(uint64_t n, int threads, int n_sm, int per_sm) {
  uint64_t want = (n + threads - 1) / threads;
  uint64_t cap = (uint64_t)n_sm * per_sm;
  return (unsigned)(want < cap ? want : cap);
}

// Write the decoded sequence of every path (bit-exact integer indexing).
__global__ void enumerate_kernel(BatchDev B, int32_t* ids, uint8_t* order, int32_t* tx_idx, int32_t* rx_idx) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < B.n_paths; g += stride) {
    PathDesc d;
    decode_global(B, g, d);
    if (ids)
      for (int j = 0; j < B.n_max; ++j) ids[g * (uint64_t)B.n_max + j] = j < d.n ? d.ids[j] : -1;
    if (order) order[g] = (uint8_t)d.n;
    if (tx_idx) tx_idx[g] = d.tx;
    if (rx_idx) rx_idx[g] = d.rx;
  }
}

// Pattern of a decoded sequence from the scene's object types.
__device__ __forceinline__ int path_key(const SceneDev& S, const PathDesc& d) {
  unsigned q = 0;
  for (int i = 0; i < d.n; ++i)
    if (S.aux[kAux * d.ids[i] + 2] == 0.f) q |= 1u << i;
  return pattern_key(d.n, q);
}

// Histogram of (order, pattern) keys (seeded and explicit batches are solved per bucket).
__global__ void pattern_hist_kernel(SceneDev S, BatchDev B, unsigned long long* counts) {
  __shared__ unsigned long long s[kPatternKeys];
  for (int k = threadIdx.x; k < kPatternKeys; k += blockDim.x) s[k] = 0;
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < B.n_paths; g += stride) {
    PathDesc d;
    decode_global(B, g, d);
    atomicAdd(&s[path_key(S, d)], 1ULL);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kPatternKeys; k += blockDim.x)
    if (s[k]) atomicAdd(&counts[k], s[k]);
}

// cursors[key] starts at the first slot of that bucket in `lists`; each slot receives the decoded path.
// A block takes tiles of 256 x kScatterPerThread paths: it counts the tile's paths per bucket in shared
// memory (each path's rank within its bucket, its packed record kept in registers), reserves each
// bucket's range with one global atomic, then writes the records.  One global atomic per (tile, bucket)
// instead of one per path: with ~60 buckets, per-path atomics on the same few cursors serialised the kernel.
constexpr int kScatterPerThread = 8;
__global__ void pattern_scatter_kernel(SceneDev S, BatchDev B, unsigned long long* cursors, PathRec* lists) {
  __shared__ unsigned s_cnt[kPatternKeys];
  __shared__ unsigned long long s_base[kPatternKeys];
  const uint64_t tile = (uint64_t)blockDim.x * kScatterPerThread;
  for (uint64_t t0 = (uint64_t)blockIdx.x * tile; t0 < B.n_paths; t0 += (uint64_t)gridDim.x * tile) {
    for (int k = threadIdx.x; k < kPatternKeys; k += blockDim.x) s_cnt[k] = 0u;
    __syncthreads();
    int key[kScatterPerThread];
    unsigned rank[kScatterPerThread];
    uint4 rec_a[kScatterPerThread], rec_b[kScatterPerThread];
#pragma unroll
    for (int i = 0; i < kScatterPerThread; ++i) {
      const uint64_t g = t0 + (uint64_t)i * blockDim.x + threadIdx.x;
      key[i] = -1;
      rank[i] = 0u;
      rec_a[i] = rec_b[i] = make_uint4(0u, 0u, 0u, 0u);
      if (g < B.n_paths) {
        PathDesc d;
        decode_global(B, g, d);
        key[i] = path_key(S, d);
        rank[i] = atomicAdd(&s_cnt[key[i]], 1u);
        pack_rec(d, rec_a[i], rec_b[i]);
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kPatternKeys; k += blockDim.x)
      if (s_cnt[k]) s_base[k] = atomicAdd(&cursors[k], (unsigned long long)s_cnt[k]);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScatterPerThread; ++i) {
      if (key[i] < 0) continue;
      uint4* p = reinterpret_cast<uint4*>(lists + s_base[key[i]] + rank[i]);
      p[0] = rec_a[i];
      p[1] = rec_b[i];
    }
    __syncthreads();  // s_cnt and s_base are reused by the next tile
  }
}

__global__ void count_status_kernel(const uint8_t* __restrict__ st, uint64_t n, uint8_t mask,
                                    unsigned long long* out) {
  unsigned long long c = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * 16;
  for (uint64_t base = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16; base < n; base += stride) {
    if (base + 16 <= n && ((reinterpret_cast<uintptr_t>(st + base) & 15) == 0)) {
      uint4 v = *reinterpret_cast<const uint4*>(st + base);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int b = 0; b < 4; ++b) c += (((w[k] >> (8 * b)) & mask) == mask);
    } else {
      for (uint64_t i = base; i < n && i < base + 16; ++i) c += ((st[i] & mask) == mask);
    }
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

cudaError_t launch_enumerate(const BatchDev& B, int32_t* ids, uint8_t* order, int32_t* tx_idx, int32_t* rx_idx,
                             cudaStream_t stream, int n_sm) {
  unsigned grid = grid_for(B.n_paths, 256, n_sm, 8);
  if (grid == 0) return cudaSuccess;
  enumerate_kernel<<<grid, 256, 0, stream>>>(B, ids, order, tx_idx, rx_idx);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pattern_histogram(const SceneDev& S, const BatchDev& B, unsigned long long* counts,
                                     cudaStream_t stream, int n_sm) {
  unsigned grid = grid_for(B.n_paths, 256, n_sm, 8);
  if (grid == 0) return cudaSuccess;
  pattern_hist_kernel<<<grid, 256, 0, stream>>>(S, B, counts);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pattern_scatter(const SceneDev& S, const BatchDev& B, unsigned long long* cursors, PathRec* lists,
                                   cudaStream_t stream, int n_sm) {
  unsigned grid = grid_for((B.n_paths + kScatterPerThread - 1) / kScatterPerThread, 256, n_sm, 8);
  if (grid == 0) return cudaSuccess;
  pattern_scatter_kernel<<<grid, 256, 0, stream>>>(S, B, cursors, lists);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_count_status(const uint8_t* status, uint64_t n, uint8_t mask, unsigned long long* out,
                                cudaStream_t stream, int n_sm) {
  unsigned grid = grid_for((n + 15) / 16, 256, n_sm, 8);
  if (grid == 0) return cudaSuccess;
  count_status_kernel<<<grid, 256, 0, stream>>>(status, n, mask, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fpt
