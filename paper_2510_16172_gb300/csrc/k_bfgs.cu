// k_bfgs.cu -- BFGS launch dispatch and the unified kernels of orders 1-5.
// The interaction-type pattern kernels are instantiated in k_bfgs_pat.cu,
// compiled once per entry of FPT_BFGS_RANGES; the unified kernels of orders
// 6-10 (inverse Hessian in shared memory) in k_high.cu, once per order.
#include "bfgs.cuh"

namespace fpt {

extern template struct BfgsOrder<6>;
extern template struct BfgsOrder<7>;
extern template struct BfgsOrder<8>;
extern template struct BfgsOrder<9>;
extern template struct BfgsOrder<10>;

#define FPT_BFGS_EXTERN(n, q0, qn) extern template cudaError_t launch_bfgs_range<n, q0, qn>(unsigned, const BfgsLaunch&);
FPT_BFGS_RANGES(FPT_BFGS_EXTERN)
#undef FPT_BFGS_EXTERN

cudaError_t launch_bfgs(int n, int pattern, const SceneDev& S, const BatchDev& B, const SolveCfg& cfg,
                        uint64_t n_local, const PathRec* list, float* T, uint8_t* status, uint8_t* iters,
                        cudaStream_t stream, int n_sm, unsigned long long* work) {
  const BfgsLaunch a{S, B, cfg, n_local, list, T, status, iters, stream, n_sm, work};
  if (pattern < 0 || n > kMaxBfgsOrder) {
    switch (n) {
      case 1: return BfgsOrder<1>::launch(a);
      case 2: return BfgsOrder<2>::launch(a);
      case 3: return BfgsOrder<3>::launch(a);
      case 4: return BfgsOrder<4>::launch(a);
      case 5: return BfgsOrder<5>::launch(a);
      case 6: return BfgsOrder<6>::launch(a);  // orders 6-10: the inverse Hessian in shared memory
      case 7: return BfgsOrder<7>::launch(a);
      case 8: return BfgsOrder<8>::launch(a);
      case 9: return BfgsOrder<9>::launch(a);
      case 10: return BfgsOrder<10>::launch(a);
      default: return cudaErrorInvalidValue;
    }
  }
  const unsigned q = (unsigned)pattern;
#define FPT_BFGS_CASE(n_, q0, qn) \
  if (n == n_ && q >= q0 && q < q0 + qn) return launch_bfgs_range<n_, q0, qn>(q, a);
  FPT_BFGS_RANGES(FPT_BFGS_CASE)
#undef FPT_BFGS_CASE
  return cudaErrorInvalidValue;
}

}  // namespace fpt
