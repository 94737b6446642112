// k_bfgs_pat.cu -- one range of interaction-type pattern kernels: order
// FPT_BFGS_ORDER, patterns FPT_BFGS_Q0 .. FPT_BFGS_Q0 + FPT_BFGS_QN - 1.  The
// build compiles this file once per entry of FPT_BFGS_RANGES (bfgs.cuh).
#include "bfgs.cuh"

#if !defined(FPT_BFGS_ORDER) || !defined(FPT_BFGS_Q0) || !defined(FPT_BFGS_QN)
#error "k_bfgs_pat.cu is compiled once per pattern range: define FPT_BFGS_ORDER, FPT_BFGS_Q0 and FPT_BFGS_QN"
#endif

namespace fpt {

template cudaError_t launch_bfgs_range<FPT_BFGS_ORDER, FPT_BFGS_Q0, FPT_BFGS_QN>(unsigned, const BfgsLaunch&);

}  // namespace fpt
