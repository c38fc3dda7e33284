// Definitions of Ops<D, EQ>: runtime degree -> templated launchers.
#pragma once
#include "ldg_linalg_impl.cuh"
#include "ldg_ops.h"

namespace ldg {

#define LDG_FOR_P(F) \
  switch (h->p) {    \
    case 1:          \
      F(1);          \
    case 2:          \
      F(2);          \
    case 3:          \
      F(3);          \
    case 4:          \
      F(4);          \
    default:         \
      break;         \
  }

template <int D, int EQ>
bool Ops<D, EQ>::supported(int p) {
  return p >= 1 && p <= 4;
}

template <int D, int EQ>
cudaError_t Ops<D, EQ>::jacobian(const ldg_handle* h, const double* U, const double* Q, ldg_jac* J,
                                 cudaStream_t st) {
  if (J->prec == LDG_PREC_FP32) {
    // FP32 copies of U (and Q): one conversion per value instead of one per use
    float* uf = (float*)J->ucvt;
    float* qf = h->viscous() ? uf + h->ndof : nullptr;
    const int64_t nconv = h->ndof * (h->viscous() ? 1 + h->D : 1);
    if (!uf) return cudaErrorInvalidValue;
    k_to_float<<<(unsigned)((h->ndof + 255) / 256 < 4096 ? (h->ndof + 255) / 256 : 4096), 256, 0, st>>>(uf, U,
                                                                                                    h->ndof);
    count_launch();
    if (qf) {
      k_to_float<<<(unsigned)((nconv - h->ndof + 255) / 256 < 4096 ? (nconv - h->ndof + 255) / 256 : 4096), 256, 0,
                   st>>>(qf, Q, nconv - h->ndof);
      count_launch();
    }
    const float* gf = (const float*)J->geof;
    if (!gf) return cudaErrorInvalidValue;
    const int64_t nng = h->nlines() * h->nq * h->D, nnend = h->nlines() * 2 * h->D;
    if (!J->geof_ready) {
      // the metric terms in FP32, once per Jacobian object (they do not change)
      const double* src[3] = {h->ng, h->nend, h->invJ};
      const int64_t len[3] = {nng, nnend, h->E * h->npe};
      float* dst = (float*)J->geof;
      for (int a = 0; a < 3; ++a) {
        k_to_float<<<(unsigned)((len[a] + 255) / 256 < 4096 ? (len[a] + 255) / 256 : 4096), 256, 0, st>>>(dst, src[a],
                                                                                                    len[a]);
        count_launch();
        dst += len[a];
      }
      J->geof_ready = true;
    }
    const GeoR<float> gr{gf, gf + nng, gf + nng + nnend};
#define F(P) return run_jacobian<D, P, EQ, float>(h, uf, qf, (float*)J->K11, (float*)J->K12, (float*)J->Kw, gr, st)
    LDG_FOR_P(F)
#undef F
  } else {
    const GeoR<double> gr{h->ng, h->nend, h->invJ};
#define F(P) \
  return run_jacobian<D, P, EQ, double>(h, U, Q, (double*)J->K11, (double*)J->K12, (double*)J->Kw, gr, st)
    LDG_FOR_P(F)
#undef F
  }
  return cudaErrorInvalidValue;
}

template <int D, int EQ>
cudaError_t Ops<D, EQ>::k21(const ldg_handle* h, ldg_jac* J, cudaStream_t st) {
  if (J->prec == LDG_PREC_FP32) {
#define F(P) return run_k21<D, P, float>(h, (float*)J->K21, st)
    LDG_FOR_P(F)
#undef F
  } else {
#define F(P) return run_k21<D, P, double>(h, (double*)J->K21, st)
    LDG_FOR_P(F)
#undef F
  }
  return cudaErrorInvalidValue;
}

template <int D, int EQ>
cudaError_t Ops<D, EQ>::jacvec(const ldg_handle* h, const ldg_jac* J, double shift, double scale,
                               const void* x, void* y, int vprec, cudaStream_t st, void* g, int part) {
  void* gb = g ? g : J->gbuf;
  if (J->prec == LDG_PREC_FP32 && vprec == LDG_PREC_FP32) {
#define F(P)                                                                                      \
  return run_jacvec<D, P, EQ, float, float>(h, (const float*)J->K11, (const float*)J->K12,         \
                                            (const float*)J->K21, (const float*)J->Kw,            \
                                            (float*)gb, shift, scale, (const float*)x, (float*)y, st, part)
    LDG_FOR_P(F)
#undef F
  } else if (J->prec == LDG_PREC_FP32) {
#define F(P)                                                                                        \
  return run_jacvec<D, P, EQ, float, double>(h, (const float*)J->K11, (const float*)J->K12,          \
                                             (const float*)J->K21, (const float*)J->Kw,             \
                                             (double*)gb, shift, scale, (const double*)x, (double*)y, st, part)
    LDG_FOR_P(F)
#undef F
  } else if (vprec == LDG_PREC_FP64) {
#define F(P)                                                                                          \
  return run_jacvec<D, P, EQ, double, double>(h, (const double*)J->K11, (const double*)J->K12,         \
                                              (const double*)J->K21, (const double*)J->Kw,              \
                                              (double*)gb, shift, scale, (const double*)x, (double*)y, st, part)
    LDG_FOR_P(F)
#undef F
  }
  return cudaErrorInvalidValue;
}

template <int D, int EQ>
cudaError_t Ops<D, EQ>::precond(const ldg_handle* h, const ldg_jac* J, double shift, double scale,
                                ldg_pc* P, cudaStream_t st) {
  if (J->prec == LDG_PREC_FP32) {
#define F(PP)                                                                                   \
  return run_precond<D, PP, EQ, float>(h, (const float*)J->K11, (const float*)J->K12,           \
                                       (const float*)J->K21, (const float*)J->Kw, (float*)P->F,    \
                                       (float*)P->Udiag, shift, scale, st)
    LDG_FOR_P(F)
#undef F
  } else {
#define F(PP)                                                                                       \
  return run_precond<D, PP, EQ, double>(h, (const double*)J->K11, (const double*)J->K12,            \
                                        (const double*)J->K21, (const double*)J->Kw, (double*)P->F,    \
                                        (double*)P->Udiag, shift, scale, st)
    LDG_FOR_P(F)
#undef F
  }
  return cudaErrorInvalidValue;
}

template <int D, int EQ>
cudaError_t Ops<D, EQ>::apply(const ldg_handle* h, const ldg_pc* P, const void* r, void* z, int vprec,
                              cudaStream_t st) {
  if (P->prec == LDG_PREC_FP32 && vprec == LDG_PREC_FP32) {
#define F(PP)                                                                                     \
  return run_precond_apply<D, PP, EQ, float, float>(h, (const float*)P->F, \
                                                    (const float*)r, (float*)z, st)
    LDG_FOR_P(F)
#undef F
  } else if (P->prec == LDG_PREC_FP64 && vprec == LDG_PREC_FP64) {
#define F(PP)                                                                                        \
  return run_precond_apply<D, PP, EQ, double, double>(h, (const double*)P->F, \
                                                      (const double*)r, (double*)z, st)
    LDG_FOR_P(F)
#undef F
  }
  return cudaErrorInvalidValue;
}

#undef LDG_FOR_P
}  // namespace ldg
