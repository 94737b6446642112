// k_unrolled.cu -- dispatch of the reverse-mode gradient through the solver's
// iterations by order (the kernel is in unrolled.cuh; orders 6-10 are
// instantiated in k_high.cu).
#include "unrolled.cuh"

namespace fpt {

extern template struct UnrolledOrder<6>;
extern template struct UnrolledOrder<7>;
extern template struct UnrolledOrder<8>;
extern template struct UnrolledOrder<9>;
extern template struct UnrolledOrder<10>;

size_t unrolled_tape_floats(int n, int steps, uint64_t threads) {
  const int M = 2 * n;
  return (size_t)threads * (size_t)steps * (size_t)(M + M * (M + 1) / 2);
}

cudaError_t launch_unrolled(int n, const SceneDev& S, const BatchDev& B, int steps, int rounds, uint64_t n_local,
                            const PathRec* list, const float* dX, const float* dL, double* gacc, float* tape,
                            size_t tape_floats, float* T_out, uint8_t* status, cudaStream_t stream, int n_sm) {
  const float dl_all = 0.f;
  if (rounds < 1 || rounds > kUnrolledMaxRounds || steps < 0) return cudaErrorInvalidValue;
  switch (n) {
#define FPT_UNROLLED_CASE(K)                                                                                     \
  case K:                                                                                                        \
    return UnrolledOrder<K>::launch(S, B, steps, rounds, n_local, list, dX, dL, dl_all, gacc, tape, tape_floats, \
                                    T_out, status, stream, n_sm);
    FPT_UNROLLED_CASE(1)
    FPT_UNROLLED_CASE(2)
    FPT_UNROLLED_CASE(3)
    FPT_UNROLLED_CASE(4)
    FPT_UNROLLED_CASE(5)
    FPT_UNROLLED_CASE(6)
    FPT_UNROLLED_CASE(7)
    FPT_UNROLLED_CASE(8)
    FPT_UNROLLED_CASE(9)
    FPT_UNROLLED_CASE(10)
#undef FPT_UNROLLED_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpt
