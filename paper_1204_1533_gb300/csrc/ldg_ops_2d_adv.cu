// Jacobian / matvec / preconditioner kernels for D = 2, EQ_ADV.
#include "ldg_ops_impl.cuh"

namespace ldg {
template struct Ops<2, EQ_ADV>;
}  // namespace ldg
