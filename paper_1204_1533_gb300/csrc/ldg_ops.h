// Per-(dimension, equation) operation table of the Jacobian / Krylov path.
// Each instantiation lives in its own translation unit so the kernels for
// all degrees compile in parallel.
#pragma once
#include "ldg_internal.h"

namespace ldg {

template <int D, int EQ>
struct Ops {
  static bool supported(int p);
  static cudaError_t jacobian(const ldg_handle* h, const double* U, const double* Q, ldg_jac* J,
                              cudaStream_t st);
  static cudaError_t k21(const ldg_handle* h, ldg_jac* J, cudaStream_t st);
  // part 0: y = shift x + scale (K11 x + K12 K21 x) (g: workspace); part 1:
  // g = K21 x only; part 2: y from x and the given g
  static cudaError_t jacvec(const ldg_handle* h, const ldg_jac* J, double shift, double scale,
                            const void* x, void* y, int vprec, cudaStream_t st, void* g = nullptr, int part = 0);
  static cudaError_t precond(const ldg_handle* h, const ldg_jac* J, double shift, double scale,
                             ldg_pc* P, cudaStream_t st);
  static cudaError_t apply(const ldg_handle* h, const ldg_pc* P, const void* r, void* z, int vprec,
                           cudaStream_t st);
};

}  // namespace ldg
