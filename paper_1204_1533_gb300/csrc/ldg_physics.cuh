// Pointwise physics of the Line-DG scheme for device code.
//
// Every function is a template over the scalar type T so that the same
// source yields the FP64 residual (T = double) and forward-mode derivatives
// for the Jacobian (T = Dual<float, N> or Dual<double, N>). Normals are plain
// reals (metric terms do not depend on the state).
//
// Fluxes (Sec. 5.2 Eqs. 44-48, Sec. 5.1 Eq. 42):
//   Euler    F.n = (rho v.n, rho v v.n + p n, (rho E + p) v.n)
//   NS       F^vis.n with tau = mu (grad v + grad v^T - 2/3 div v I) and heat
//            flux -(mu gamma / Pr) grad e, q = grad of conserved variables;
//            the viscous flux is part of F in du/dt + div F = 0
//   Poisson  F = -q
// Numerical fluxes take (u_out, u_in, n) with n the outward, non-normalised
// normal (Eqs. 5-7); a unit-normal flux is scaled by |n| (Eq. 13).
#pragma once
#include <math.h>

#include "ldg_dual.cuh"

namespace ldg {

enum { EQ_POISSON = 0, EQ_EULER = 1, EQ_NS = 2, EQ_ADV = 3 };
enum { FLUX_ROE = 0, FLUX_LF = 1 };
enum { BC_DIRICHLET = 0, BC_WALL = 1, BC_NEUMANN = 2 };

// physical constants at the precision R of the flux arithmetic (converted
// once per thread: on this part an FP64 -> FP32 conversion costs as much as an
// FP64 multiply-add, so FP32 derivative code must not convert per call)
template <typename R>
struct Phys {
  R gamma, mu, Pr, C11, C11b;
  R adv[3];
  int flux;
  template <typename A>
  __device__ __forceinline__ void set(const A& ph) {
    gamma = R(ph.gamma);
    mu = R(ph.mu);
    Pr = R(ph.Pr);
    C11 = R(ph.C11);
    C11b = R(ph.C11b);
    adv[0] = R(ph.adv[0]);
    adv[1] = R(ph.adv[1]);
    adv[2] = R(ph.adv[2]);
    flux = ph.flux;
  }
};

template <int EQ, int D>
struct NComp {
  static constexpr int value = (EQ == EQ_EULER || EQ == EQ_NS) ? D + 2 : 1;
};

template <int EQ>
struct IsViscous {
  static constexpr bool value = (EQ == EQ_NS || EQ == EQ_POISSON);
};

// ---------------------------------------------------------------------------
// Euler flux dotted with n
// ---------------------------------------------------------------------------
template <int D, typename T, typename R>
__device__ __forceinline__ void euler_flux_n(const T* u, const R* n, R gm1, T* f) {
  T rinv = T(1.0) / u[0];
  T vn = u[1] * n[0];
#pragma unroll
  for (int a = 1; a < D; ++a) vn = vn + u[1 + a] * n[a];
  vn = vn * rinv;  // v.n
  T m2 = u[1] * u[1];
#pragma unroll
  for (int a = 1; a < D; ++a) m2 = m2 + u[1 + a] * u[1 + a];
  T pr = gm1 * (u[D + 1] - R(0.5) * m2 * rinv);
  f[0] = u[0] * vn;
#pragma unroll
  for (int a = 0; a < D; ++a) f[1 + a] = u[1 + a] * vn + pr * n[a];
  f[D + 1] = (u[D + 1] + pr) * vn;
}

// ---------------------------------------------------------------------------
// Roe's approximate Riemann solver with Harten's entropy fix
// ---------------------------------------------------------------------------
template <typename T, typename R>
__device__ __forceinline__ T entropy_fixed_abs(const T& lam, const T& delta) {
  T al = dabs(lam);
  if (val(al) < val(delta)) return (lam * lam + delta * delta) / (R(2.0) * delta);
  return al;
}

template <int D, typename T, typename R>
__device__ __forceinline__ void roe_flux(const T* uo, const T* ui, const R* n, R gamma, T* f) {
  const R gm1 = gamma - R(1.0);
  R nn = n[0] * n[0];
#pragma unroll
  for (int a = 1; a < D; ++a) nn += n[a] * n[a];
  nn = sqrt(nn);
  R nb[D];
#pragma unroll
  for (int a = 0; a < D; ++a) nb[a] = n[a] / nn;
  // left = inside, right = outside
  T ril = T(1.0) / ui[0], rir = T(1.0) / uo[0];
  T vl[D], vr[D];
  T kl = T(0.0), kr = T(0.0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    vl[a] = ui[1 + a] * ril;
    vr[a] = uo[1 + a] * rir;
    kl = kl + ui[1 + a] * vl[a];
    kr = kr + uo[1 + a] * vr[a];
  }
  T pl = gm1 * (ui[D + 1] - R(0.5) * kl);
  T pr = gm1 * (uo[D + 1] - R(0.5) * kr);
  T Hl = (ui[D + 1] + pl) * ril;
  T Hr = (uo[D + 1] + pr) * rir;
  T sl = sqrt(ui[0]), sr = sqrt(uo[0]);
  T ws = T(1.0) / (sl + sr);
  T rt = sl * sr;
  T vt[D];
  T q2 = T(0.0), vnt = T(0.0), dvn = T(0.0), vdv = T(0.0);
  T dv[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    vt[a] = (sl * vl[a] + sr * vr[a]) * ws;
    dv[a] = vr[a] - vl[a];
    q2 = q2 + vt[a] * vt[a];
    vnt = vnt + vt[a] * nb[a];
    dvn = dvn + dv[a] * nb[a];
    vdv = vdv + vt[a] * dv[a];
  }
  T Ht = (sl * Hl + sr * Hr) * ws;
  T c2 = gm1 * (Ht - R(0.5) * q2);
  T ct = sqrt(c2);
  T c2inv = T(1.0) / c2;
  T drho = uo[0] - ui[0];
  T dp = pr - pl;
  T delta = R(0.1) * ct;
  T l1 = entropy_fixed_abs<T, R>(vnt - ct, delta);
  T l2 = entropy_fixed_abs<T, R>(vnt, delta);
  T l5 = entropy_fixed_abs<T, R>(vnt + ct, delta);
  T rcd = rt * ct * dvn;
  T a1 = R(0.5) * (dp - rcd) * c2inv;
  T a2 = drho - dp * c2inv;
  T a5 = R(0.5) * (dp + rcd) * c2inv;
  T w1 = l1 * a1, w2 = l2 * a2, w5 = l5 * a5, ws2 = l2 * rt;
  // dissipation |A| (u_out - u_in)
  T dis[D + 2];
  dis[0] = w1 + w2 + w5;
#pragma unroll
  for (int a = 0; a < D; ++a)
    dis[1 + a] = w1 * (vt[a] - ct * nb[a]) + w2 * vt[a] + ws2 * (dv[a] - dvn * nb[a]) +
                 w5 * (vt[a] + ct * nb[a]);
  dis[D + 1] = w1 * (Ht - ct * vnt) + w2 * (R(0.5) * q2) + ws2 * (vdv - vnt * dvn) +
               w5 * (Ht + ct * vnt);
  // central part with the raw (non-unit) normal: |n| F(u).nbar = F(u).n
  T vnl = vl[0] * n[0], vnr = vr[0] * n[0];
#pragma unroll
  for (int a = 1; a < D; ++a) {
    vnl = vnl + vl[a] * n[a];
    vnr = vnr + vr[a] * n[a];
  }
  const R hn = R(0.5) * nn;
  f[0] = R(0.5) * (ui[0] * vnl + uo[0] * vnr) - hn * dis[0];
#pragma unroll
  for (int a = 0; a < D; ++a)
    f[1 + a] = R(0.5) * (ui[1 + a] * vnl + uo[1 + a] * vnr + (pl + pr) * n[a]) - hn * dis[1 + a];
  f[D + 1] = R(0.5) * ((ui[D + 1] + pl) * vnl + (uo[D + 1] + pr) * vnr) - hn * dis[D + 1];
}

// local Lax-Friedrichs
template <int D, typename T, typename R>
__device__ __forceinline__ void lf_flux(const T* uo, const T* ui, const R* n, R gamma, T* f) {
  R nn = n[0] * n[0];
#pragma unroll
  for (int a = 1; a < D; ++a) nn += n[a] * n[a];
  nn = sqrt(nn);
  const R gm1 = gamma - R(1.0);
  T fl[D + 2], fr[D + 2];
  euler_flux_n<D, T, R>(ui, n, gm1, fl);
  euler_flux_n<D, T, R>(uo, n, gm1, fr);
  T ril = T(1.0) / ui[0], rir = T(1.0) / uo[0];
  T kl = T(0.0), kr = T(0.0), vnl = T(0.0), vnr = T(0.0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    kl = kl + ui[1 + a] * ui[1 + a];
    kr = kr + uo[1 + a] * uo[1 + a];
    vnl = vnl + ui[1 + a] * n[a];
    vnr = vnr + uo[1 + a] * n[a];
  }
  T pl = gm1 * (ui[D + 1] - R(0.5) * kl * ril);
  T pr = gm1 * (uo[D + 1] - R(0.5) * kr * rir);
  T cl = sqrt(gamma * pl * ril), cr = sqrt(gamma * pr * rir);
  T sl = dabs(vnl * ril) / nn + cl;
  T sr = dabs(vnr * rir) / nn + cr;
  T lam = (val(sl) >= val(sr)) ? sl : sr;
  T s = R(0.5) * nn * lam;
#pragma unroll
  for (int c = 0; c < D + 2; ++c) f[c] = R(0.5) * (fl[c] + fr[c]) - s * (uo[c] - ui[c]);
}

// ---------------------------------------------------------------------------
// Navier-Stokes viscous flux . n; q[c * D + b] = d u_c / d x_b
// ---------------------------------------------------------------------------
template <int D, typename T, typename R>
__device__ __forceinline__ void ns_visc_flux_n(const T* u, const T* q, const R* n, R gamma, R mu,
                                               R Pr, T* f) {
  T rinv = T(1.0) / u[0];
  T v[D];
#pragma unroll
  for (int a = 0; a < D; ++a) v[a] = u[1 + a] * rinv;
  T Et = u[D + 1] * rinv;
  T gv[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) gv[a][b] = (q[(1 + a) * D + b] - v[a] * q[b]) * rinv;
  T dv = gv[0][0];
#pragma unroll
  for (int a = 1; a < D; ++a) dv = dv + gv[a][a];
  const R kh = -mu * gamma / Pr;
  const R c23 = R(2.0) / R(3.0);
  // tau . n (row a) and (heat - v.tau) . n
  T en = T(0.0);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    T ge = (q[(D + 1) * D + b] - Et * q[b]) * rinv;
#pragma unroll
    for (int a = 0; a < D; ++a) ge = ge - v[a] * gv[a][b];
    en = en + kh * ge * n[b];
  }
  f[0] = T(0.0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    T tn = T(0.0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      T tab = gv[a][b] + gv[b][a];
      if (a == b) tab = tab - c23 * dv;
      tn = tn + tab * n[b];
    }
    tn = mu * tn;
    f[1 + a] = -tn;
    en = en - v[a] * tn;
  }
  f[D + 1] = en;
}

// inviscid part of F . n for the equation set
template <int EQ, int D, typename T, typename R>
__device__ __forceinline__ void inviscid_flux_n(const T* u, const R* n, const Phys<R>& ph, T* f) {
  if constexpr (EQ == EQ_EULER || EQ == EQ_NS) {
    euler_flux_n<D, T, R>(u, n, ph.gamma - R(1.0), f);
  } else if constexpr (EQ == EQ_ADV) {
    R an = ph.adv[0] * n[0];
#pragma unroll
    for (int b = 1; b < D; ++b) an += ph.adv[b] * n[b];
    f[0] = an * u[0];
  } else {
    f[0] = T(0.0);
  }
}

template <int EQ, int D, typename T, typename R>
__device__ __forceinline__ void inviscid_numflux(const T* uo, const T* ui, const R* n,
                                                 const Phys<R>& ph, T* f) {
  if constexpr (EQ == EQ_EULER || EQ == EQ_NS) {
    if (ph.flux == FLUX_ROE)
      roe_flux<D, T, R>(uo, ui, n, ph.gamma, f);
    else
      lf_flux<D, T, R>(uo, ui, n, ph.gamma, f);
  } else if constexpr (EQ == EQ_ADV) {
    R an = ph.adv[0] * n[0];
#pragma unroll
    for (int b = 1; b < D; ++b) an += ph.adv[b] * n[b];
    f[0] = (an >= R(0.0)) ? an * ui[0] : an * uo[0];
  } else {
    f[0] = T(0.0);
  }
}

template <int EQ, int D, typename T, typename R>
__device__ __forceinline__ void viscous_flux_n(const T* u, const T* q, const R* n, const Phys<R>& ph,
                                               T* f) {
  if constexpr (EQ == EQ_NS) {
    ns_visc_flux_n<D, T, R>(u, q, n, ph.gamma, ph.mu, ph.Pr, f);
  } else if constexpr (EQ == EQ_POISSON) {
    T s = q[0] * n[0];
#pragma unroll
    for (int b = 1; b < D; ++b) s = s + q[b] * n[b];
    f[0] = -s;
  }
}

// no-slip adiabatic wall state: zero momentum, internal energy kept
template <int D, typename T, typename R>
__device__ __forceinline__ void wall_state(const T* ui, T* ub) {
  T m2 = ui[1] * ui[1];
#pragma unroll
  for (int a = 1; a < D; ++a) m2 = m2 + ui[1 + a] * ui[1 + a];
  ub[0] = ui[0];
#pragma unroll
  for (int a = 0; a < D; ++a) ub[1 + a] = T(0.0);
  ub[D + 1] = ui[D + 1] - R(0.5) * m2 / ui[0];
}

}  // namespace ldg
