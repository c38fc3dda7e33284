// C-ABI entry points of the Jacobian, split matvec and preconditioner.
#include <cstring>
#include <vector>

#include "ldg_ops.h"

namespace ldg {

#define LDG_DISPATCH(h, CALL)                              \
  do {                                                     \
    if ((h)->D == 2) {                                     \
      switch ((h)->kind) {                                 \
        case LDG_EQ_POISSON: return Ops<2, 0>::CALL;       \
        case LDG_EQ_EULER: return Ops<2, 1>::CALL;         \
        case LDG_EQ_NAVIER_STOKES: return Ops<2, 2>::CALL; \
        case LDG_EQ_ADVECTION: return Ops<2, 3>::CALL;     \
      }                                                    \
    } else if ((h)->D == 3) {                              \
      switch ((h)->kind) {                                 \
        case LDG_EQ_EULER: return Ops<3, 1>::CALL;         \
        case LDG_EQ_NAVIER_STOKES: return Ops<3, 2>::CALL; \
      }                                                    \
    }                                                      \
  } while (0)

bool ops_supported(const ldg_handle* h) {
  if (h->p < 1 || h->p > 4) return false;
  if (h->phys.C22 != 0.0) return false;  // coupled (U, Q) system: ldg_coupled_solve
  if (h->has_wall && h->kind != LDG_EQ_EULER && h->kind != LDG_EQ_NAVIER_STOKES) return false;
  if (h->D == 2) return true;
  return h->kind == LDG_EQ_EULER || h->kind == LDG_EQ_NAVIER_STOKES;
}

cudaError_t launch_jacobian(const ldg_handle* h, const double* U, const double* Q, ldg_jac* J,
                            cudaStream_t st) {
  LDG_DISPATCH(h, jacobian(h, U, Q, J, st));
  return cudaErrorInvalidValue;
}
cudaError_t launch_k21(const ldg_handle* h, ldg_jac* J, cudaStream_t st) {
  LDG_DISPATCH(h, k21(h, J, st));
  return cudaErrorInvalidValue;
}
// algorithmic operations of the kernel timer: one multiply-add per stored
// matrix entry (K11, K12 and each K21 entry once per component) and
// y = shift x + scale s per unknown; ILU(0) apply: one multiply-add per
// factor entry (the forward and backward sweeps and D^-1 together read each
// stored block once)
static double jacvec_flops(const ldg_handle* h) {
  return 2.0 * (double)h->nlines() * (h->nk11() + h->nk12() + (double)h->nk21() * h->nc) + 3.0 * h->ndof;
}
static double apply_flops(const ldg_handle* h) {
  return 2.0 * (double)h->E * h->npe * h->pat_w() * h->nc * h->nc;
}
cudaError_t launch_jacvec(const ldg_handle* h, const ldg_jac* J, double shift, double scale,
                          const void* x, void* y, int vprec, cudaStream_t st) {
  const double esz = J->prec == LDG_PREC_FP32 ? 4.0 : 8.0, vsz = vprec == LDG_PREC_FP32 ? 4.0 : 8.0;
  TimedScope tl(KT_JACVEC, vprec, st,
                (double)h->ntiles() * 32.0 * (h->nk11() + h->nk12()) * esz + 2.0 * h->ndof * vsz, jacvec_flops(h));
  LDG_DISPATCH(h, jacvec(h, J, shift, scale, x, y, vprec, st));
  return cudaErrorInvalidValue;
}
// the two launches of the split product apart (part 1: g = K21 x; part 2: y
// from x and g), for partitioned runs that exchange g's face traces between
static cudaError_t launch_jacvec_part(const ldg_handle* h, const ldg_jac* J, double shift, double scale,
                                      const void* x, void* g, void* y, int vprec, int part, cudaStream_t st) {
  LDG_DISPATCH(h, jacvec(h, J, shift, scale, x, y, vprec, st, g, part));
  return cudaErrorInvalidValue;
}
cudaError_t launch_precond(const ldg_handle* h, const ldg_jac* J, double shift, double scale,
                           ldg_pc* P, cudaStream_t st) {
  LDG_DISPATCH(h, precond(h, J, shift, scale, P, st));
  return cudaErrorInvalidValue;
}
cudaError_t launch_precond_apply(const ldg_handle* h, const ldg_pc* P, const void* r, void* z,
                                 int vprec, cudaStream_t st) {
  const double esz = P->prec == LDG_PREC_FP32 ? 4.0 : 8.0, vsz = vprec == LDG_PREC_FP32 ? 4.0 : 8.0;
  TimedScope tl(KT_APPLY, vprec, st,
                (double)h->E * h->npe * h->pat_w() * h->nc * h->nc * esz + 2.0 * h->ndof * vsz, apply_flops(h));
  LDG_DISPATCH(h, apply(h, P, r, z, vprec, st));
  return cudaErrorInvalidValue;
}

}  // namespace ldg

using namespace ldg;

static size_t esize(int prec) { return prec == LDG_PREC_FP32 ? 4 : 8; }

extern "C" int ldg_jac_destroy(ldg_jac_t* J) {
  if (!J) return LDG_OK;
  cudaFree(J->K11);
  cudaFree(J->K12);
  cudaFree(J->K21);
  cudaFree(J->Kw);
  cudaFree(J->gbuf);
  cudaFree(J->ucvt);
  cudaFree(J->geof);
  delete J;
  return LDG_OK;
}

static int jacobian_impl(ldg_handle_t* h, const double* U, const double* Qin, int prec, ldg_jac_t** Jp,
                         void* stream) {
  if (!h || !U || !Jp || (prec != LDG_PREC_FP32 && prec != LDG_PREC_FP64)) return LDG_ERR_ARG;
  if (!ops_supported(h)) return LDG_ERR_UNSUPPORTED;
  ldg_jac* J = *Jp;
  if (J && (J->h != h || J->prec != prec)) return LDG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!J) {
    J = new ldg_jac();
    J->h = h;
    J->prec = prec;
    const size_t rows = (size_t)h->ntiles() * 32;
    cudaError_t err = cudaMalloc(&J->K11, rows * h->nk11() * esize(prec));
    if (err == cudaSuccess) err = cudaMemset(J->K11, 0, rows * h->nk11() * esize(prec));
    if (err == cudaSuccess && h->viscous()) {
      err = cudaMalloc(&J->K12, rows * h->nk12() * esize(prec));
      if (err == cudaSuccess) err = cudaMemset(J->K12, 0, rows * h->nk12() * esize(prec));
      if (err == cudaSuccess) err = cudaMalloc(&J->K21, rows * h->nk21() * esize(prec));
      if (err == cudaSuccess) err = cudaMemset(J->K21, 0, rows * h->nk21() * esize(prec));
      if (err == cudaSuccess) err = cudaMalloc(&J->gbuf, (size_t)h->ndof * h->D * sizeof(double));
      if (err == cudaSuccess && h->has_wall) err = cudaMalloc(&J->Kw, rows * 2 * h->nc * esize(prec));
    }
    if (err == cudaSuccess && prec == LDG_PREC_FP32)
      err = cudaMalloc(&J->ucvt, (size_t)h->ndof * (h->viscous() ? 1 + h->D : 1) * sizeof(float));
    if (err == cudaSuccess && prec == LDG_PREC_FP32)
      err = cudaMalloc(&J->geof, ((size_t)h->nlines() * (h->nq + 2) * h->D + (size_t)h->E * h->npe) * sizeof(float));
    if (err != cudaSuccess) {
      ldg_jac_destroy(J);
      return LDG_ERR_CUDA;
    }
  }
  const double* Q = Qin;
  if (h->viscous() && !Q) {
    if (launch_gradient(h, U, h->Qbuf, st) != cudaSuccess) return LDG_ERR_CUDA;
    Q = h->Qbuf;
  }
  if (launch_jacobian(h, U, Q, J, st) != cudaSuccess) return LDG_ERR_CUDA;
  if (h->viscous() && !J->k21_built) {
    if (launch_k21(h, J, st) != cudaSuccess) return LDG_ERR_CUDA;
    J->k21_built = true;
  }
  J->built = true;
  *Jp = J;
  return LDG_OK;
}

extern "C" int ldg_jacobian(ldg_handle_t* h, const double* U, int prec, ldg_jac_t** Jp, void* stream) {
  return jacobian_impl(h, U, nullptr, prec, Jp, stream);
}

extern "C" int ldg_jacobian_uq(ldg_handle_t* h, const double* U, const double* Q, int prec, ldg_jac_t** Jp,
                               void* stream) {
  if (h && h->viscous() && !Q) return LDG_ERR_ARG;
  return jacobian_impl(h, U, h && h->viscous() ? Q : nullptr, prec, Jp, stream);
}

extern "C" int ldg_jac_export(const ldg_jac_t* J, void* K11, void* K12, void* K21) {
  if (!J || !J->built) return LDG_ERR_NOT_BUILT;
  const ldg_handle* h = J->h;
  const size_t es = esize(J->prec);
  const int64_t NL = h->nlines(), rows = h->ntiles() * 32;
  auto untile = [&](const void* dev, void* host, int nk) -> int {
    std::vector<unsigned char> tmp((size_t)rows * nk * es);
    if (cudaMemcpy(tmp.data(), dev, tmp.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return LDG_ERR_CUDA;
    unsigned char* out = (unsigned char*)host;
    for (int64_t L = 0; L < NL; ++L)
      for (int k = 0; k < nk; ++k)
        std::memcpy(out + ((size_t)k * NL + L) * es, tmp.data() + (((L >> 5) * nk + k) * 32 + (L & 31)) * es, es);
    return LDG_OK;
  };
  int rc = LDG_OK;
  if (K11) rc = untile(J->K11, K11, h->nk11());
  if (rc == LDG_OK && K12 && h->viscous()) rc = untile(J->K12, K12, h->nk12());
  if (rc == LDG_OK && K21 && h->viscous()) rc = untile(J->K21, K21, h->nk21());
  return rc;
}

extern "C" int ldg_jacvec(ldg_handle_t* h, const ldg_jac_t* J, double shift, double scale, const void* x,
                          void* y, int prec, void* stream) {
  if (!h || !J || !x || !y || J->h != h) return LDG_ERR_ARG;
  if (!J->built) return LDG_ERR_NOT_BUILT;
  if (prec != LDG_PREC_FP32 && prec != LDG_PREC_FP64) return LDG_ERR_ARG;
  if (J->prec == LDG_PREC_FP64 && prec == LDG_PREC_FP32) return LDG_ERR_UNSUPPORTED;
  return launch_jacvec(h, J, shift, scale, x, y, prec, (cudaStream_t)stream) == cudaSuccess ? LDG_OK
                                                                                          : LDG_ERR_CUDA;
}

static int jacvec_args(ldg_handle_t* h, const ldg_jac_t* J, int prec) {
  if (!h || !J || J->h != h) return LDG_ERR_ARG;
  if (!J->built) return LDG_ERR_NOT_BUILT;
  if (prec != LDG_PREC_FP32 && prec != LDG_PREC_FP64) return LDG_ERR_ARG;
  if (J->prec == LDG_PREC_FP64 && prec == LDG_PREC_FP32) return LDG_ERR_UNSUPPORTED;
  return LDG_OK;
}

extern "C" int ldg_k21_apply(ldg_handle_t* h, const ldg_jac_t* J, const void* x, void* g, int prec, void* stream) {
  int rc = jacvec_args(h, J, prec);
  if (rc) return rc;
  if (!x || !g) return LDG_ERR_ARG;
  if (!h->viscous()) return LDG_ERR_UNSUPPORTED;
  return launch_jacvec_part(h, J, 0.0, 0.0, x, g, nullptr, prec, 1, (cudaStream_t)stream) == cudaSuccess
             ? LDG_OK
             : LDG_ERR_CUDA;
}

extern "C" int ldg_jacvec_g(ldg_handle_t* h, const ldg_jac_t* J, double shift, double scale, const void* x,
                            const void* g, void* y, int prec, void* stream) {
  int rc = jacvec_args(h, J, prec);
  if (rc) return rc;
  if (!x || !y || (h->viscous() && !g)) return LDG_ERR_ARG;
  const double esz = J->prec == LDG_PREC_FP32 ? 4.0 : 8.0, vsz = prec == LDG_PREC_FP32 ? 4.0 : 8.0;
  TimedScope tl(KT_JACVEC, prec, (cudaStream_t)stream,
                (double)h->ntiles() * 32.0 * (h->nk11() + h->nk12()) * esz + 2.0 * h->ndof * vsz,
                jacvec_flops(h) - 2.0 * (double)h->nlines() * h->nk21() * h->nc);
  return launch_jacvec_part(h, J, shift, scale, x, const_cast<void*>(g), y, prec, 2, (cudaStream_t)stream) ==
                 cudaSuccess
             ? LDG_OK
             : LDG_ERR_CUDA;
}

extern "C" int ldg_pc_destroy(ldg_pc_t* P) {
  if (!P) return LDG_OK;
  cudaFree(P->F);
  cudaFree(P->Udiag);
  delete P;
  return LDG_OK;
}

extern "C" int ldg_precond(ldg_handle_t* h, const ldg_jac_t* J, double shift, double scale, ldg_pc_t** Pp,
                           void* stream) {
  if (!h || !J || !Pp || J->h != h) return LDG_ERR_ARG;
  if (!J->built) return LDG_ERR_NOT_BUILT;
  ldg_pc* P = *Pp;
  if (P && (P->h != h || P->prec != J->prec)) return LDG_ERR_ARG;
  if (!P) {
    P = new ldg_pc();
    P->h = h;
    P->prec = J->prec;
    const size_t bb = (size_t)h->nc * h->nc;
    cudaError_t err = cudaMalloc(&P->F, (size_t)h->E * h->npe * h->pat_w() * bb * esize(J->prec));
    if (err == cudaSuccess) err = cudaMalloc(&P->Udiag, (size_t)h->E * h->npe * bb * esize(J->prec));
    if (err != cudaSuccess) {
      ldg_pc_destroy(P);
      return LDG_ERR_CUDA;
    }
  }
  if (launch_precond(h, J, shift, scale, P, (cudaStream_t)stream) != cudaSuccess) return LDG_ERR_CUDA;
  P->built = true;
  *Pp = P;
  return LDG_OK;
}

extern "C" int ldg_precond_apply(ldg_handle_t* h, const ldg_pc_t* P, const void* r, void* z, int prec,
                                 void* stream) {
  if (!h || !P || !r || !z || P->h != h) return LDG_ERR_ARG;
  if (!P->built) return LDG_ERR_NOT_BUILT;
  if (prec != P->prec) return LDG_ERR_UNSUPPORTED;
  return launch_precond_apply(h, P, r, z, prec, (cudaStream_t)stream) == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}

extern "C" int ldg_pc_export(const ldg_pc_t* P, void* factors) {
  if (!P || !factors) return LDG_ERR_ARG;
  if (!P->built) return LDG_ERR_NOT_BUILT;
  const ldg_handle* h = P->h;
  const size_t bb = (size_t)h->nc * h->nc, W = h->pat_w(), es = esize(P->prec);
  const size_t bytes = (size_t)h->E * h->npe * W * bb * es;
  const int N = h->p + 1;
  if (cudaMemcpy(factors, P->F, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
    return LDG_ERR_CUDA;
  }
  // the device keeps D_i^-1 in each row's diagonal slot and U_ii aside:
  // put U_ii back (the factors as ILU(0) defines them)
  std::vector<char> ud((size_t)h->E * h->npe * bb * es);
  if (cudaMemcpy(ud.data(), P->Udiag, ud.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return LDG_ERR_CUDA;
  for (int64_t e = 0; e < h->E; ++e)
    for (int i = 0; i < h->npe; ++i) {
      const int dg = i % N + (i / N) % N + (h->D == 3 ? i / (N * N) : 0);  // slots of lower columns
      std::memcpy((char*)factors + (((size_t)e * h->npe + i) * W + dg) * bb * es,
                  ud.data() + ((size_t)e * h->npe + i) * bb * es, bb * es);
    }
  return LDG_OK;
}
