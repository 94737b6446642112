// k_polish.cu -- polish launch dispatch by order (the kernels are in polish.cuh;
// orders above the BFGS orders are instantiated in k_high.cu).
#include "polish.cuh"

namespace fpt {

extern template struct PolishOrder<6>;
extern template struct PolishOrder<7>;
extern template struct PolishOrder<8>;
extern template struct PolishOrder<9>;
extern template struct PolishOrder<10>;

cudaError_t launch_polish(int n, const SceneDev& S, const BatchDev& B, const PolishCfg& cfg, uint64_t n_local,
                          const PathRec* list, float* T, float* X, float* L, uint8_t* status, float* rho,
                          uint8_t* mask, float* bdist, cudaStream_t stream, int n_sm, uint32_t* rescue_list,
                          unsigned* rescue_count, const GradCfg* grad, uint32_t* step_list, unsigned* step_count,
                          float* step_delta) {
  switch (n) {
#define FPT_POLISH_CASE(K)                                                                                     \
  case K:                                                                                                      \
    return PolishOrder<K>::launch(S, B, cfg, n_local, list, T, X, L, status, rho, mask, bdist, stream, n_sm, \
                                  rescue_list, rescue_count, grad, step_list, step_count, step_delta);
    FPT_POLISH_CASE(1)
    FPT_POLISH_CASE(2)
    FPT_POLISH_CASE(3)
    FPT_POLISH_CASE(4)
    FPT_POLISH_CASE(5)
    FPT_POLISH_CASE(6)
    FPT_POLISH_CASE(7)
    FPT_POLISH_CASE(8)
    FPT_POLISH_CASE(9)
    FPT_POLISH_CASE(10)
#undef FPT_POLISH_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fpt
