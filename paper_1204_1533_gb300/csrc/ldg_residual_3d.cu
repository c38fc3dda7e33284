// Instantiations of the FP64 gradient/residual kernels for D = 3.
#include "ldg_residual_impl.cuh"

namespace ldg {

#define LDG_RES_CASE(EQ, P) \
  case P:                   \
    return run_residual<3, P, EQ>(h, U, Q, R, st);
#define LDG_GRAD_CASE(NC, P) \
  case P:                    \
    return run_gradient<3, P, NC>(h, U, Qs, Q, st);

cudaError_t residual_3d(const ldg_handle* h, const double* U, const double* Q, double* R,
                        cudaStream_t st) {
  switch (h->kind) {
    case LDG_EQ_POISSON:
      switch (h->p) { LDG_RES_CASE(EQ_POISSON, 1) LDG_RES_CASE(EQ_POISSON, 2) LDG_RES_CASE(EQ_POISSON, 3) LDG_RES_CASE(EQ_POISSON, 4) }
      break;
    case LDG_EQ_EULER:
      switch (h->p) { LDG_RES_CASE(EQ_EULER, 1) LDG_RES_CASE(EQ_EULER, 2) LDG_RES_CASE(EQ_EULER, 3) LDG_RES_CASE(EQ_EULER, 4) }
      break;
    case LDG_EQ_NAVIER_STOKES:
      switch (h->p) { LDG_RES_CASE(EQ_NS, 1) LDG_RES_CASE(EQ_NS, 2) LDG_RES_CASE(EQ_NS, 3) LDG_RES_CASE(EQ_NS, 4) }
      break;

    default:
      break;
  }
  return cudaErrorInvalidValue;
}

cudaError_t gradient_3d(const ldg_handle* h, const double* U, const double* Qs, double* Q, cudaStream_t st) {
  if (h->nc == 1) {
    switch (h->p) { LDG_GRAD_CASE(1, 1) LDG_GRAD_CASE(1, 2) LDG_GRAD_CASE(1, 3) LDG_GRAD_CASE(1, 4) }
  } else if (h->nc == 5) {
    switch (h->p) { LDG_GRAD_CASE(5, 1) LDG_GRAD_CASE(5, 2) LDG_GRAD_CASE(5, 3) LDG_GRAD_CASE(5, 4) }
  }
  return cudaErrorInvalidValue;
}

}  // namespace ldg
