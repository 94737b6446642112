// k_occlusion.cu -- obstruction test of solved paths against the scene's planar objects.
//
// Sec. I: a candidate ray is discarded when it is obstructed, as well as when an
// interaction point falls outside its object (the validity bit).  For segment j
// of a path of order n, from x_j to x_{j+1} (x_0 = TX, x_{n+1} = RX), every
// planar object other than the objects at the segment's two ends is tested: the
// segment is blocked when its ends lie on opposite sides of the object's plane,
// each more than `tol` metres from it, and the crossing point lies in the closed
// parallelogram.  Edges (lines) block nothing.  One thread per path; the
// occluders' records (centred origin, unit normal and the dual basis that gives
// the in-plane coordinates u = d1 . (h - b), v = d2 . (h - b)) are staged in
// shared memory and every thread of a warp walks them in the same order.  When
// only paths with given status bits are tested (typically the few per cent
// that are valid and solved), a first kernel lists them and writes zero for
// the rest, so that the test kernel's warps run full.
#include "fpt_kernels.h"

namespace fpt {

// List the paths of a slice that hold the status bits (local indices); zero the others' masks.  A CTA
// takes kOccSelPer consecutive local indices per thread and appends its chunk in index order with a
// single atomic on the list counter, which one atomic per warp would turn into a serial hot spot.
constexpr int kOccSelThreads = 256, kOccSelPer = 16, kOccSelChunk = kOccSelThreads * kOccSelPer;
__global__ void __launch_bounds__(kOccSelThreads) occlusion_select_kernel(BatchDev B, int n, const PathRec* list,
                                                                          uint64_t n_local,
                                                                          const uint8_t* __restrict__ status,
                                                                          uint8_t mask, uint16_t* __restrict__ blocked,
                                                                          uint32_t* __restrict__ sel,
                                                                          unsigned* __restrict__ sel_count) {
  for (uint64_t c0 = (uint64_t)blockIdx.x * kOccSelChunk; c0 < n_local; c0 += (uint64_t)gridDim.x * kOccSelChunk) {
    const uint64_t j0 = c0 + (uint64_t)threadIdx.x * kOccSelPer;
    unsigned bits = 0;
    SliceWalk walk;
#pragma unroll 4
    for (int k = 0; k < kOccSelPer; ++k) {
      const uint64_t j = j0 + k;
      if (j >= n_local) break;
      // the solver wrote the sequence's REPEAT / INVALID_INPUT bits into its status
      const uint64_t g = list != nullptr ? slice_global(B, n, list, j) : walk.next(B, n, j);
      const uint8_t st = status[g];
      const bool take = !(st & ST_SKIP) && (st & mask) == mask;
      if (!take) blocked[g] = 0;
      bits |= (take ? 1u : 0u) << k;
    }
    cta_append_ordered<kOccSelThreads>(bits, j0, sel, sel_count);
  }
}

// Test the paths of a slice (sel == nullptr) or the listed ones.
__global__ void __launch_bounds__(kThreads) occlusion_kernel(SceneDev S, BatchDev B, int n, const PathRec* list,
                                                             uint64_t n_local, const float* __restrict__ T,
                                                             const uint32_t* __restrict__ sel,
                                                             const unsigned* __restrict__ sel_count,
                                                             const float* __restrict__ occ, int n_occ, float tol,
                                                             uint16_t* __restrict__ blocked) {
  extern __shared__ __align__(16) float s_occ[];
  for (int k = threadIdx.x; k < n_occ * kOcc; k += blockDim.x) s_occ[k] = occ[k];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n_iter = sel ? (uint64_t)*sel_count : n_local;
  for (uint64_t k0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k0 < n_iter; k0 += stride) {
    const uint64_t j = sel ? (uint64_t)sel[k0] : k0;
    PathDesc d;
    fetch_path(B, n, list, j, d);
    uint16_t bits = 0;
    if (!(d.flags & ST_SKIP)) {
      // the points x_0 .. x_{n+1}, relative to the scene centre
      const float2* Tp = reinterpret_cast<const float2*>(T) + d.g * (uint64_t)B.n_max;
      float P[3];
      for (int c = 0; c < 3; ++c) P[c] = S.tx32[kEnd32 * d.tx + c] + S.tx32[kEnd32 * d.tx + 3 + c];
      for (int seg = 0; seg <= n; ++seg) {
        float Q[3];
        if (seg < n) {
          const float* r = S.rec32 + kRec32 * d.ids[seg];
          const float2 t = Tp[seg];
          for (int c = 0; c < 3; ++c) Q[c] = fmaf(r[9 + c], t.y, fmaf(r[6 + c], t.x, r[c] + r[3 + c]));
        } else {
          for (int c = 0; c < 3; ++c) Q[c] = S.rx32[kEnd32 * d.rx + c] + S.rx32[kEnd32 * d.rx + 3 + c];
        }
        const int own0 = seg > 0 ? d.ids[seg - 1] : -1;
        const int own1 = seg < n ? d.ids[seg] : -1;
        for (int k = 0; k < n_occ; ++k) {
          const float* o = s_occ + kOcc * k;
          const int id = __float_as_int(o[12]);
          if (id == own0 || id == own1) continue;
          const float pb0 = P[0] - o[0], pb1 = P[1] - o[1], pb2 = P[2] - o[2];
          const float qb0 = Q[0] - o[0], qb1 = Q[1] - o[1], qb2 = Q[2] - o[2];
          const float dP = fmaf(o[5], pb2, fmaf(o[4], pb1, o[3] * pb0));
          const float dQ = fmaf(o[5], qb2, fmaf(o[4], qb1, o[3] * qb0));
          if (!((dP > tol && dQ < -tol) || (dP < -tol && dQ > tol))) continue;
          const float s = dP / (dP - dQ);
          const float h0 = fmaf(s, qb0 - pb0, pb0), h1 = fmaf(s, qb1 - pb1, pb1), h2 = fmaf(s, qb2 - pb2, pb2);
          const float u = fmaf(o[8], h2, fmaf(o[7], h1, o[6] * h0));
          const float v = fmaf(o[11], h2, fmaf(o[10], h1, o[9] * h0));
          if (u >= 0.f && u <= 1.f && v >= 0.f && v <= 1.f) {
            bits |= (uint16_t)(1u << seg);
            break;
          }
        }
        for (int c = 0; c < 3; ++c) P[c] = Q[c];
      }
    }
    blocked[d.g] = bits;
  }
}

cudaError_t launch_occlusion(const SceneDev& S, const BatchDev& B, int n, const PathRec* list, uint64_t n_local,
                             const float* T, const uint8_t* status, uint8_t mask, const float* occ, int n_occ,
                             float tol, uint16_t* blocked, uint32_t* sel, unsigned* sel_count, cudaStream_t stream,
                             int n_sm) {
  const bool listed = status != nullptr && mask != 0;
  if (listed) {
    if (!sel || !sel_count) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(sel_count, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    const uint64_t want = (n_local + kOccSelChunk - 1) / kOccSelChunk;
    const unsigned g = (unsigned)(want < (uint64_t)n_sm * 8 ? want : (uint64_t)n_sm * 8);
    if (g == 0) return cudaSuccess;
    occlusion_select_kernel<<<g, kOccSelThreads, 0, stream>>>(B, n, list, n_local, status, mask, blocked, sel,
                                                              sel_count);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = (size_t)n_occ * kOcc * sizeof(float);
  if (smem > kMaxSmemBytes) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(occlusion_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, occlusion_kernel, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  // a listed launch strides over the list; a full grid covers the largest list
  const uint64_t want = (n_local + kThreads - 1) / kThreads;
  const uint64_t cap = (uint64_t)n_sm * (uint64_t)per_sm;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  if (grid == 0) return cudaSuccess;
  occlusion_kernel<<<grid, kThreads, smem, stream>>>(S, B, n, list, n_local, T, listed ? sel : nullptr,
                                                     listed ? sel_count : nullptr, occ, n_occ, tol, blocked);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fpt
