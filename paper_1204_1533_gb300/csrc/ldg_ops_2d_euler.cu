// Jacobian / matvec / preconditioner kernels for D = 2, EQ_EULER.
#include "ldg_ops_impl.cuh"

namespace ldg {
template struct Ops<2, EQ_EULER>;
}  // namespace ldg
