// k_bfgs.cu -- solver launch dispatch and the unified BFGS kernels of every BFGS
// order.  The interaction-type pattern kernels are instantiated in
// k_bfgs_pat.cu, compiled once per entry of FPT_BFGS_RANGES; the Newton
// kernels of the longer sequences in k_high.cu, once per order.
#include "bfgs.cuh"
#include "newton.cuh"

namespace fpt {

extern template struct NewtonOrder<6>;
extern template struct NewtonOrder<7>;
extern template struct NewtonOrder<8>;
extern template struct NewtonOrder<9>;
extern template struct NewtonOrder<10>;

#define FPT_BFGS_EXTERN(n, q0, qn) extern template cudaError_t launch_bfgs_range<n, q0, qn>(unsigned, const BfgsLaunch&);
FPT_BFGS_RANGES(FPT_BFGS_EXTERN)
#undef FPT_BFGS_EXTERN

template <int N>
static cudaError_t launch_unified(const BfgsLaunch& a) {
  if (a.list != nullptr) return launch_bfgs_nq<N, kAllQuads<N>, SRC_LIST>(a);
  return launch_bfgs_nq<N, kAllQuads<N>, SRC_ORDER>(a);
}

cudaError_t launch_bfgs(int n, int pattern, const SceneDev& S, const BatchDev& B, const SolveCfg& cfg,
                        uint64_t n_local, const PathRec* list, float* T, uint8_t* status, uint8_t* iters,
                        cudaStream_t stream, int n_sm, unsigned long long* work) {
  const BfgsLaunch a{S, B, cfg, n_local, list, T, status, iters, stream, n_sm, work};
  switch (n) {  // longer sequences: the Newton solver (newton.cuh), one kernel per order
    case 6: return NewtonOrder<6>::launch(a);
    case 7: return NewtonOrder<7>::launch(a);
    case 8: return NewtonOrder<8>::launch(a);
    case 9: return NewtonOrder<9>::launch(a);
    case 10: return NewtonOrder<10>::launch(a);
    default: break;
  }
  if (pattern < 0) {
    switch (n) {
      case 1: return launch_unified<1>(a);
      case 2: return launch_unified<2>(a);
      case 3: return launch_unified<3>(a);
      case 4: return launch_unified<4>(a);
      case 5: return launch_unified<5>(a);
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
