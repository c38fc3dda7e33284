// Jacobian / matvec / preconditioner kernels for D = 3, EQ_NS.
#include "ldg_ops_impl.cuh"

namespace ldg {
template struct Ops<3, EQ_NS>;
}  // namespace ldg
