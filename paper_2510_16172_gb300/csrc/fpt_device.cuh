// fpt_device.cuh -- device-side data layout and helpers shared by the kernels.
//
// Scene records live in HBM as flat arrays and are staged into shared memory
// per CTA (a scene of K objects costs K * 48 B in FP32 and K * 72 B in FP64).
// Coordinates are relative to the scene centre, which keeps FP32 ulps small.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fpt {

constexpr int kMaxOrder = 10;       // longest sequence solved on the GPU
constexpr int kMaxBfgsOrder = 5;    // longest sequence whose BFGS state fits in registers (pattern kernels, 32-byte records)
constexpr int kRec32 = 12;          // floats per FP32 object record: b_hi[3], b_lo[3], a1[3], a2[3]
constexpr int kRec64 = 9;           // doubles per FP64 object record: b[3], a1[3], a2[3]
constexpr int kAux = 4;             // floats per object: side heights h1, h2 (metres), type, pad
constexpr int kRecLo = 6;           // floats per object: low parts of a1[3], a2[3] (double-float polish)
constexpr int kEnd32 = 6;           // floats per endpoint: hi[3], lo[3]

// status bits (same values as the public header)
constexpr uint8_t ST_VALID = 1, ST_CONVERGED = 2, ST_SOLVED = 4, ST_FP64 = 8, ST_DEGENERATE = 16,
                  ST_REPEAT = 32, ST_NONFINITE = 64, ST_INVALID = 128;
constexpr uint8_t ST_SKIP = ST_REPEAT | ST_INVALID;  // never solved

// device error word codes
constexpr int ERR_NONE = 0, ERR_BAD_ORDER = 1, ERR_SMEM = 2;
// (3: a tensor-core wait ran out, k_mlp.cu)  4: non-finite or degenerate device-side geometry
constexpr int ERR_BAD_GEOMETRY = 4;

struct SceneDev {
  int n_obj;
  const float* rec32;    // [n_obj][12]
  const double* rec64;   // [n_obj][9]
  const float* aux;      // [n_obj][4]
  int n_tx, n_rx;
  const float* tx32;     // [n_tx][6]
  const float* rx32;     // [n_rx][6]
  const double* tx64;    // [n_tx][3]
  const double* rx64;    // [n_rx][3]
  const float* reclo;    // [n_obj][6]
  double centre[3];
  float centre_hi[3], centre_lo[3];
};

enum BatchMode { BATCH_EXHAUSTIVE = 0, BATCH_SEEDED = 1, BATCH_EXPLICIT = 2 };

// Division of 32-bit values by a divisor fixed per batch or launch, through a precomputed 64-bit
// reciprocal m = ceil(2^64 / d): floor(x / d) = floor(x m / 2^64) for every x < 2^32 and 2 <= d < 2^32,
// since x m / 2^64 exceeds x / d by less than x / 2^64 < 2^-32 <= 1 / d and so never reaches the next
// integer.  A multiply-high replaces the long instruction sequence of an integer division.
struct FastDiv {
  uint64_t m;  // ceil(2^64 / d) (0 when d <= 1)
  uint32_t d;
};
__host__ __device__ inline FastDiv make_fastdiv(uint64_t d) {
  FastDiv f;
  f.d = d > 0xFFFFFFFFull ? 0u : (uint32_t)d;  // divisors of 2^32 or more are never used on the fast path
  f.m = f.d <= 1 ? 0ull : ~0ull / f.d + 1ull;
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return f.d <= 1 ? x : (uint32_t)__umul64hi((unsigned long long)x, (unsigned long long)f.m);
}
// r mod d for a 64-bit r and 1 <= d <= 65535, with t32 = 2^32 mod d: r = 2^32 hi + lo, so
// r mod d = ((hi mod d) t32 + lo mod d) mod d, every term below 2^32 (d^2 + d < 2^32).
__device__ __forceinline__ uint32_t fmod64(uint64_t r, const FastDiv& f, uint32_t t32) {
  const uint32_t hi = (uint32_t)(r >> 32), lo = (uint32_t)r;
  const uint32_t a = hi - fdiv(hi, f) * f.d, b = lo - fdiv(lo, f) * f.d;
  const uint32_t c = a * t32 + b;
  return c - fdiv(c, f) * f.d;
}

struct BatchDev {
  int mode;
  int n_alpha;
  const int32_t* alphabet;  // device [n_alpha]
  int lo, hi, n_max;
  int n_tx, n_rx;
  uint64_t per_pair;        // sequences per (tx, rx) pair (exhaustive, seeded)
  uint64_t n_paths;
  uint64_t seed;
  uint64_t kpow[kMaxOrder + 1];    // n_alpha^n
  uint64_t offset[kMaxOrder + 2];  // exhaustive: first r of order n inside a pair
  const int32_t* ids;       // explicit [n][n_max]
  const uint8_t* order;     // explicit [n]
  const int32_t* tx_idx;    // explicit [n]
  const int32_t* rx_idx;    // explicit [n]
  const int32_t* type_pos;  // exhaustive: alphabet positions of the reflectors, then of the edges (ascending)
  int n_alpha_quad;         // exhaustive: reflectors in the alphabet
  // reciprocals for the exhaustive decoders: n_rx, n_alpha, the alphabet's reflectors and edges, K^n
  FastDiv fd_rx, fd_alpha, fd_quad, fd_edge;
  FastDiv fd_kpow[kMaxOrder + 1];
  FastDiv fd_pat;  // set per pattern launch: sequences of the launch's pattern per (tx, rx) pair
  // seeded batches: K - 1, the number of orders and the sequences per pair (divisors of 2^16 or more, or 0,
  // take the 64-bit operators), with 2^32 mod each of the first two
  FastDiv fd_alpha1, fd_range, fd_pp;
  uint32_t t32_alpha, t32_alpha1, t32_range;
};

// Interaction-type pattern of a sequence of order n: bit i set = slot i is a
// planar reflector, clear = an edge.  Seeded and explicit batches are bucketed
// by (order, pattern) up to the BFGS orders, key(n, Q) = 2^n - 2 + Q, and by
// order alone above them (one bucket, Q = 0); keys follow the orders, so the
// buckets of one order form one contiguous range.
constexpr int kPatternKeys = (2 << kMaxBfgsOrder) - 2 + (kMaxOrder - kMaxBfgsOrder);  // 62 + 5
__host__ __device__ constexpr int n_patterns(int n) { return n <= kMaxBfgsOrder ? 1 << n : 1; }
__host__ __device__ constexpr int pattern_key(int n, unsigned q) {
  return n <= kMaxBfgsOrder ? (1 << n) - 2 + (int)q : (2 << kMaxBfgsOrder) - 2 + (n - kMaxBfgsOrder - 1);
}

// One candidate sequence, decoded.
struct PathDesc {
  uint64_t g;
  int n;
  int ids[kMaxOrder];
  int tx, rx;
  uint8_t flags;  // ST_REPEAT / ST_INVALID
};

// A path of a seeded or explicit batch, decoded once when the batch is bucketed
// (32 bytes, two 16-byte loads): words 0-1 g, 2 tx, 3 rx, 4-5 ids[0..3] as
// 16-bit pairs, 6 ids[4] | n << 16 | flags << 24, 7 unused.  Object ids fit in
// 16 bits (a scene holds at most 65535 objects).  Records of sequences longer
// than kMaxBfgsOrder keep g, tx, rx, n and flags; their kernels decode the
// ids from g again (decode_global).
struct __align__(16) PathRec {
  uint32_t w[8];
};

__device__ __forceinline__ void load_rec(const PathRec* list, uint64_t j, PathDesc& d) {
  const uint4* p = reinterpret_cast<const uint4*>(list + j);
  const uint4 a = __ldg(p), b = __ldg(p + 1);
  d.g = (uint64_t)a.x | ((uint64_t)a.y << 32);
  d.tx = (int)a.z;
  d.rx = (int)a.w;
  d.ids[0] = (int)(b.x & 0xFFFFu);
  d.ids[1] = (int)(b.x >> 16);
  d.ids[2] = (int)(b.y & 0xFFFFu);
  d.ids[3] = (int)(b.y >> 16);
  d.ids[4] = (int)(b.z & 0xFFFFu);
  d.n = (int)((b.z >> 16) & 0xFFu);
  d.flags = (uint8_t)(b.z >> 24);
}

// The record of a decoded path as two 16-byte words.
__device__ __forceinline__ void pack_rec(const PathDesc& d, uint4& a, uint4& b) {
  uint32_t id[kMaxBfgsOrder];
#pragma unroll
  for (int i = 0; i < kMaxBfgsOrder; ++i) id[i] = i < d.n && d.n <= kMaxBfgsOrder ? (uint32_t)d.ids[i] & 0xFFFFu : 0u;
  a = make_uint4((uint32_t)d.g, (uint32_t)(d.g >> 32), (uint32_t)d.tx, (uint32_t)d.rx);
  b = make_uint4(id[0] | (id[1] << 16), id[2] | (id[3] << 16), id[4] | ((uint32_t)d.n << 16) | ((uint32_t)d.flags << 24),
                 0u);
}
__device__ __forceinline__ void store_rec(PathRec* list, uint64_t slot, const PathDesc& d) {
  uint4 a, b;
  pack_rec(d, a, b);
  uint4* p = reinterpret_cast<uint4*>(list + slot);
  p[0] = a;
  p[1] = b;
}

// splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// counter-based draw s of sequence g: state number 8 g + s + 1 of a splitmix64 stream
__device__ __forceinline__ uint64_t seeded_draw(uint64_t seed, uint64_t g, int s) {
  return sm64_mix(seed + 0x9E3779B97F4A7C15ULL * (8ULL * g + (uint64_t)s + 1ULL));
}

// kExact: the order d.n is the compile-time kN.  Otherwise it is known only at
// run time and at most kN (kMaxOrder when kN = 0): the slot loop runs over
// compile-time indices guarded by the order, so that the descriptor still stays
// in registers (as in decode_global).
template <int kN = 0, bool kExact = false>
__device__ __forceinline__ void finish_desc(const BatchDev& B, const int* digits, PathDesc& d) {
  constexpr int kSlotsMax = kN > 0 ? kN : kMaxOrder;
  d.flags = 0;
  if constexpr (kExact) {
    for (int j = 0; j < d.n; ++j) {
      int o = B.alphabet[digits[j]];
      d.ids[j] = o;
      if (j > 0 && d.ids[j - 1] == o) d.flags |= ST_REPEAT;
    }
  } else {
#pragma unroll
    for (int j = 0; j < kSlotsMax; ++j)
      if (j < d.n) {
        int o = B.alphabet[digits[j]];
        d.ids[j] = o;
        if (j > 0 && d.ids[j - 1] == o) d.flags |= ST_REPEAT;
      }
  }
}

// Exhaustive batch, order n known: local index j over n_pairs * K^n paths (kN as in finish_desc).
template <int kN = 0>
__device__ __forceinline__ void decode_exhaustive_order(const BatchDev& B, int n, uint64_t j, PathDesc& d) {
  uint64_t kn = B.kpow[n];
  uint64_t pair, r;
  if (j <= 0xFFFFFFFFull && kn <= 0xFFFFFFFFull) {  // one order holds at most 2^32 paths: the usual case
    const uint32_t p32 = fdiv((uint32_t)j, B.fd_kpow[n]);
    pair = p32;
    r = (uint32_t)j - p32 * (uint32_t)kn;
    d.tx = (int)fdiv(p32, B.fd_rx);
  } else {
    pair = j / kn;
    r = j - pair * kn;
    d.tx = (int)(pair / (uint64_t)B.n_rx);
  }
  d.g = pair * B.per_pair + B.offset[n] + r;
  d.n = n;
  d.rx = (int)(pair - (uint64_t)d.tx * (uint64_t)B.n_rx);
  int digits[kMaxOrder];
  const uint64_t K = (uint64_t)B.n_alpha;
  if (kn <= 0xFFFFFFFFull) {  // 32-bit digit extraction
    uint32_t r32 = (uint32_t)r, K32 = (uint32_t)K;
#pragma unroll
    for (int q = kMaxOrder - 1; q >= 0; --q)
      if (q < n) {
        uint32_t qq = fdiv(r32, B.fd_alpha);
        digits[q] = (int)(r32 - qq * K32);
        r32 = qq;
      }
  } else {
#pragma unroll
    for (int q = kMaxOrder - 1; q >= 0; --q)
      if (q < n) {
        uint64_t qq = r / K;
        digits[q] = (int)(r - qq * K);
        r = qq;
      }
  }
  finish_desc<kN, (kN > 0)>(B, digits, d);
}

// Any batch: decode global index g.  kN > 0: the caller knows that the order is
// at most kN (a kernel compiled for order kN over a bucket of that order), so
// the slot loops stop there; kN = 0: any order up to kMaxOrder.
template <int kN = 0>
__device__ __forceinline__ void decode_global(const BatchDev& B, uint64_t g, PathDesc& d) {
  constexpr int kSlotsMax = kN > 0 ? kN : kMaxOrder;
  d.g = g;
  if (B.mode == BATCH_EXPLICIT) {
    int n = B.order[g];
    d.n = n;
    d.tx = B.tx_idx[g];
    d.rx = B.rx_idx[g];
    d.flags = 0;
    if (n < 1 || n > B.n_max || n > kMaxOrder || d.tx < 0 || d.tx >= B.n_tx || d.rx < 0 || d.rx >= B.n_rx) {
      d.flags = ST_INVALID;
      const int cap = B.n_max < kMaxOrder ? B.n_max : kMaxOrder;
      d.n = n < 1 ? 1 : (n > cap ? cap : n);
#pragma unroll
      for (int j = 0; j < kMaxOrder; ++j) d.ids[j] = 0;
      if (d.tx < 0 || d.tx >= B.n_tx) d.tx = 0;
      if (d.rx < 0 || d.rx >= B.n_rx) d.rx = 0;
      return;
    }
#pragma unroll
    for (int j = 0; j < kSlotsMax; ++j)
      if (j < n) {
        int o = B.ids[g * (uint64_t)B.n_max + j];
        d.ids[j] = o;
        if (o < 0 || o >= B.n_alpha) {  // for explicit batches n_alpha holds the object count
          d.flags |= ST_INVALID;
          d.ids[j] = 0;
        }
        if (j > 0 && d.ids[j - 1] == o) d.flags |= ST_REPEAT;
      }
    return;
  }
  uint64_t pair, r;
  if (g <= 0xFFFFFFFFull && B.fd_pp.d > 1) {  // reciprocal multiplies: exact for 32-bit operands
    pair = fdiv((uint32_t)g, B.fd_pp);
    r = g - pair * B.per_pair;
    d.tx = (int)fdiv((uint32_t)pair, B.fd_rx);
  } else {
    pair = g / B.per_pair;
    r = g - pair * B.per_pair;
    d.tx = (int)(pair / (uint64_t)B.n_rx);
  }
  d.rx = (int)(pair - (uint64_t)d.tx * (uint64_t)B.n_rx);
  int digits[kMaxOrder];
  const uint64_t K = (uint64_t)B.n_alpha;
  if (B.mode == BATCH_SEEDED) {
    // the draws of the seeded sampler, reduced with reciprocal multiplies when the divisors are below 2^16
    const bool fast = K >= 2 && K <= 65535 && B.hi - B.lo + 1 <= 65535 && B.fd_alpha.d == (uint32_t)K &&
                      B.fd_range.d == (uint32_t)(B.hi - B.lo + 1);
    const uint64_t r0 = seeded_draw(B.seed, g, 0), r1 = seeded_draw(B.seed, g, 1);
    int n = B.lo + (int)(fast ? fmod64(r0, B.fd_range, B.t32_range) : r0 % (uint64_t)(B.hi - B.lo + 1));
    d.n = n;
    digits[0] = (int)(fast ? fmod64(r1, B.fd_alpha, B.t32_alpha) : r1 % K);
#pragma unroll
    for (int j = 1; j < kSlotsMax; ++j)
      if (j < n) {
        const uint64_t rj = seeded_draw(B.seed, g, j + 1);
        if (fast) {
          const uint32_t v = (uint32_t)digits[j - 1] + 1u + fmod64(rj, B.fd_alpha1, B.t32_alpha1);  // < 2 K
          digits[j] = (int)(v >= (uint32_t)K ? v - (uint32_t)K : v);
        } else {
          digits[j] = (int)(((uint64_t)digits[j - 1] + 1ULL + rj % (K - 1)) % K);
        }
      }
  } else {
    int n = B.lo;
    while (n < B.hi && r >= B.offset[n + 1]) ++n;
    d.n = n;
    r -= B.offset[n];
#pragma unroll
    for (int q = kSlotsMax - 1; q >= 0; --q)
      if (q < n) {
        uint64_t qq = r / K;
        digits[q] = (int)(r - qq * K);
        r = qq;
      }
  }
  finish_desc<kN>(B, digits, d);
}

// Ordered list append of one CTA of kT threads: thread x flags local indices j0_x + k (bit k of
// `bits`), with j0_x ascending in x; the flagged indices are written to sel in index order, after
// the entries earlier CTAs claimed, with one atomic on sel_count for the whole CTA.  Every thread
// of the CTA must call it (it synchronises the CTA).
template <int kT>
__device__ __forceinline__ void cta_append_ordered(unsigned bits, uint64_t j0, uint32_t* __restrict__ sel,
                                                   unsigned* __restrict__ sel_count) {
  __shared__ unsigned s_warp[kT / 32];
  __shared__ unsigned s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned cnt = (unsigned)__popc(bits);
  unsigned incl = cnt;  // inclusive prefix over the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
#pragma unroll
    for (int w = 0; w < kT / 32; ++w) {
      const unsigned c = s_warp[w];
      s_warp[w] = run;
      run += c;
    }
    s_base = run ? atomicAdd(sel_count, run) : 0u;
  }
  __syncthreads();
  unsigned pos = s_base + s_warp[warp] + incl - cnt;
  while (bits) {
    const int k = __ffs(bits) - 1;
    bits &= bits - 1u;
    sel[pos++] = (uint32_t)(j0 + (uint64_t)k);
  }
  __syncthreads();  // s_warp and s_base are rewritten by the next call
}

// Global indices of an exhaustive order-n slice, counted up from local index j: consecutive local
// indices of one TX/RX pair have consecutive global indices, so g is derived once per pair.
struct SliceWalk {
  uint64_t g = 0, left = 0;
  __device__ __forceinline__ uint64_t next(const BatchDev& B, int n, uint64_t j) {
    if (left == 0) {
      const uint64_t kn = B.kpow[n];
      uint64_t pair, r;
      if (j <= 0xFFFFFFFFull && kn <= 0xFFFFFFFFull) {
        const uint32_t p32 = fdiv((uint32_t)j, B.fd_kpow[n]);
        pair = p32;
        r = (uint32_t)j - p32 * (uint32_t)kn;
      } else {
        pair = j / kn;
        r = j - pair * kn;
      }
      g = pair * B.per_pair + B.offset[n] + r;
      left = kn - r;  // paths of this pair from j on
    }
    --left;
    return g++;
  }
};

// Global index g of local index j of an order-n slice, without decoding the
// sequence (the same g as decode_exhaustive_order / the record's).
__device__ __forceinline__ uint64_t slice_global(const BatchDev& B, int n, const PathRec* list, uint64_t j) {
  if (list != nullptr) {
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(list + j));
    return (uint64_t)w.x | ((uint64_t)w.y << 32);
  }
  const uint64_t kn = B.kpow[n];
  if (j <= 0xFFFFFFFFull && kn <= 0xFFFFFFFFull) {  // the usual case: a 32-bit reciprocal multiply
    const uint32_t p32 = fdiv((uint32_t)j, B.fd_kpow[n]);
    return (uint64_t)p32 * B.per_pair + B.offset[n] + ((uint32_t)j - p32 * (uint32_t)kn);
  }
  const uint64_t pair = j / kn;
  return pair * B.per_pair + B.offset[n] + (j - pair * kn);
}

// Path source for one per-order launch: exhaustive batches need no list; other
// batches pass their bucket of decoded path records.
__device__ __forceinline__ void fetch_path(const BatchDev& B, int n, const PathRec* list, uint64_t j,
                                           PathDesc& d) {
  if (list == nullptr) {
    decode_exhaustive_order(B, n, j, d);
  } else {
    load_rec(list, j, d);
    if (n > kMaxBfgsOrder) decode_global(B, d.g, d);
  }
}

// Path source of a kernel compiled for order N: the bucket of records, else the
// exhaustive enumeration of order N (both keep the descriptor in registers).
template <int N>
__device__ __forceinline__ void fetch_path_n(const BatchDev& B, const PathRec* list, uint64_t j, PathDesc& d) {
  if (list != nullptr) {
    load_rec(list, j, d);
    if constexpr (N > kMaxBfgsOrder) decode_global<N>(B, d.g, d);
  } else {
    decode_exhaustive_order<N>(B, N, j, d);
  }
}

// Stage `count` elements of T from global to shared memory (whole CTA).
template <typename T>
__device__ __forceinline__ void stage(T* dst, const T* src, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = src[i];
}

__device__ __forceinline__ void raise_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

}  // namespace fpt
