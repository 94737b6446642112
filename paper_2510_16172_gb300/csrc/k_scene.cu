// k_scene.cu -- object and endpoint records built on the device from caller-owned
// device FP32 coordinates, so that geometry that lives on the GPU (an optimisation
// loop over TX, RX or vertices driven by the gradients of Sec. III-D) never passes
// through host memory and no call waits for the device.
//
// The records are those the host upload builds (Sec. III-B, Eq. 3: x = A t + b
// with b = v0 and A = [v1 - v0, v3 - v0] for a plane, [e1 - e0, 0] for an edge),
// relative to the scene centre fixed at upload: FP64 b, a1, a2; FP32 hi + lo
// parts of b and the low parts of a1, a2 for the double-float polish; the side
// heights of the boundary distance; the occluder record of each plane.  The
// double arithmetic is written with explicit round-to-nearest operations so that
// no product is fused into an FMA: the records equal the host's bit for bit for
// the same coordinates (the host compiler does not fuse either).
#include "fpt_kernels.h"

namespace fpt {

__device__ __forceinline__ void split_dev(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(__dsub_rn(x, (double)hi));
}

__device__ __forceinline__ double dot3(const double (&a)[3], const double (&b)[3]) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a[0], b[0]), __dmul_rn(a[1], b[1])), __dmul_rn(a[2], b[2]));
}

// p [n][3] FP32 -> rec32 [n][kEnd32] (hi, lo of p - centre) and rec64 [n][3].
__global__ void endpoint_records_kernel(const float* __restrict__ p, int n, double c0, double c1, double c2,
                                        float* __restrict__ rec32, double* __restrict__ rec64, int* err) {
  const double centre[3] = {c0, c1, c2};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x = __dsub_rn((double)p[3 * i + c], centre[c]);
      if (!isfinite(x) && err) atomicCAS(err, 0, ERR_BAD_GEOMETRY);
      rec64[3 * i + c] = x;
      split_dev(x, rec32[kEnd32 * i + c], rec32[kEnd32 * i + 3 + c]);
    }
  }
}

// verts [n_obj][3][3] FP32 (plane: v0, v1, v3; edge: e0, e1, unused) -> every record of the objects.
__global__ void object_records_kernel(int n_obj, const uint8_t* __restrict__ types,
                                      const int32_t* __restrict__ occ_slot, const float* __restrict__ verts,
                                      double c0, double c1, double c2, float* __restrict__ rec32,
                                      float* __restrict__ reclo, double* __restrict__ rec64, float* __restrict__ aux,
                                      float* __restrict__ occ, int* err) {
  const double centre[3] = {c0, c1, c2};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_obj; k += gridDim.x * blockDim.x) {
    const bool quad = types[k] == 0;
    double v[3][3];
    bool finite = true;
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v[q][c] = (double)verts[9 * k + 3 * q + c];
        if (q < 2 || quad) finite = finite && isfinite(v[q][c]);
      }
    double b[3], a1[3], a2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      b[c] = __dsub_rn(v[0][c], centre[c]);
      a1[c] = __dsub_rn(v[1][c], v[0][c]);
      a2[c] = quad ? __dsub_rn(v[2][c], v[0][c]) : 0.0;
    }
    const double n1 = sqrt(dot3(a1, a1)), n2 = sqrt(dot3(a2, a2));
    const double nv[3] = {__dsub_rn(__dmul_rn(a1[1], a2[2]), __dmul_rn(a1[2], a2[1])),
                          __dsub_rn(__dmul_rn(a1[2], a2[0]), __dmul_rn(a1[0], a2[2])),
                          __dsub_rn(__dmul_rn(a1[0], a2[1]), __dmul_rn(a1[1], a2[0]))};
    const double area = sqrt(dot3(nv, nv));
    // the host upload refuses these; here the context's error word reports them (FPT_EDEVICE at fpt_sync)
    if (!finite || (quad && !(area >= 1e-9)) || (!quad && !(n1 >= 1e-9))) {
      if (err) atomicCAS(err, 0, ERR_BAD_GEOMETRY);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rec64[kRec64 * k + c] = b[c];
      rec64[kRec64 * k + 3 + c] = a1[c];
      rec64[kRec64 * k + 6 + c] = a2[c];
      split_dev(b[c], rec32[kRec32 * k + c], rec32[kRec32 * k + 3 + c]);
      split_dev(a1[c], rec32[kRec32 * k + 6 + c], reclo[kRecLo * k + c]);
      split_dev(a2[c], rec32[kRec32 * k + 9 + c], reclo[kRecLo * k + 3 + c]);
    }
    aux[kAux * k + 0] = quad ? __double2float_rn(__ddiv_rn(area, n2)) : __double2float_rn(n1);
    aux[kAux * k + 1] = quad ? __double2float_rn(__ddiv_rn(area, n1)) : 0.f;
    aux[kAux * k + 2] = quad ? 0.f : 1.f;
    aux[kAux * k + 3] = 0.f;
    const int s = occ_slot ? occ_slot[k] : -1;
    if (quad && s >= 0 && occ) {
      const double g11 = dot3(a1, a1), g12 = dot3(a1, a2), g22 = dot3(a2, a2);
      const double det = __dsub_rn(__dmul_rn(g11, g22), __dmul_rn(g12, g12));
      float* o = occ + (size_t)kOcc * s;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[c] = __double2float_rn(b[c]);
        o[3 + c] = __double2float_rn(__ddiv_rn(nv[c], area));
        o[6 + c] = __double2float_rn(__ddiv_rn(__dsub_rn(__dmul_rn(g22, a1[c]), __dmul_rn(g12, a2[c])), det));
        o[9 + c] = __double2float_rn(__ddiv_rn(__dsub_rn(__dmul_rn(g11, a2[c]), __dmul_rn(g12, a1[c])), det));
      }
      o[12] = __int_as_float(k);
    }
  }
}

cudaError_t launch_endpoint_records(const float* p, int n, const double* centre, float* rec32, double* rec64,
                                    int* err, cudaStream_t stream) {
  if (n < 1) return cudaSuccess;
  const int grid = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  endpoint_records_kernel<<<grid, 256, 0, stream>>>(p, n, centre[0], centre[1], centre[2], rec32, rec64, err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_object_records(int n_obj, const uint8_t* types, const int32_t* occ_slot, const float* verts,
                                  const double* centre, float* rec32, float* reclo, double* rec64, float* aux,
                                  float* occ, int* err, cudaStream_t stream) {
  if (n_obj < 1) return cudaSuccess;
  const int grid = (n_obj + 127) / 128;
  object_records_kernel<<<grid, 128, 0, stream>>>(n_obj, types, occ_slot, verts, centre[0], centre[1], centre[2],
                                                   rec32, reclo, rec64, aux, occ, err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace fpt
