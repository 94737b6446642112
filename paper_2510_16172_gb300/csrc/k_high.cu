// k_high.cu -- the per-order kernels of one sequence order above 5 (BFGS with
// the inverse Hessian in shared memory, polish, backward, the unrolled-AD
// backward) for order
// FPT_HIGH_ORDER.  The build compiles this file once per order 6..10, in
// parallel.
#include "backward.cuh"
#include "bfgs.cuh"
#include "polish.cuh"
#include "unrolled.cuh"

#if !defined(FPT_HIGH_ORDER)
#error "k_high.cu is compiled once per order: define FPT_HIGH_ORDER"
#endif

namespace fpt {

static_assert(FPT_HIGH_ORDER > kMaxBfgsOrder && FPT_HIGH_ORDER <= kMaxOrder, "order outside 6..10");

template struct BfgsOrder<FPT_HIGH_ORDER>;
template struct PolishOrder<FPT_HIGH_ORDER>;
template struct BackwardOrder<FPT_HIGH_ORDER>;
template struct UnrolledOrder<FPT_HIGH_ORDER>;

}  // namespace fpt
