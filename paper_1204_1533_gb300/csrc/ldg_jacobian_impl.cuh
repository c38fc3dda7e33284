// Line-sparse Jacobian assembly (Sec. 4.1 Eq. 35: K11 = dR/dU, K12 = dR/dQ,
// K21 = dD/dU; Sec. 2.3 sparsity).
//
// For a line of direction d, R_i = -(1/J_i) r_i with r from Eq. 7, so
//   dr_i/du_j     = -sum_q Kd_iq (dF.n/du)(xi_q) phi_j(xi_q)
//                   + L1_i dF^+/du_in [j = p] + L0_i dF^-/du_in [j = 0]
//   dr_i/du_out,e = L_e,i dF^e/du_out                      (face block)
// and likewise for q. The pointwise derivative matrices are evaluated once
// per Gauss point and line end (forward-mode dual numbers over all n_c
// components; the viscous flux is linear in q, so its q-derivatives are
// flux evaluations with unit q vectors) and contracted with the 1-D tables
// row by row (k_jacobian below). Values are computed at precision R (float:
// the mixed path, from FP32 copies of the FP64 state; double: the all-FP64
// path) and stored entry-major in 32-line tiles so each warp's stores are
// coalesced.
#pragma once
#include "ldg_residual_impl.cuh"

namespace ldg {

template <typename R>
struct D1 {
  using T = Dual<R, 1>;
  __device__ __forceinline__ static T seed(R v, bool on) {
    T x(0.0);
    x.v = v;
    x.d[0] = on ? R(1) : R(0);
    return x;
  }
  __device__ __forceinline__ static T cst(R v) {
    T x(0.0);
    x.v = v;
    return x;
  }
};

// 1-D tables at the precision of the derivative arithmetic
template <typename R>
__device__ __forceinline__ R tphi(const Tab& t, int q, int j);
template <>
__device__ __forceinline__ float tphi<float>(const Tab& t, int q, int j) { return t.Phif[q][j]; }
template <>
__device__ __forceinline__ double tphi<double>(const Tab& t, int q, int j) { return t.Phi[q][j]; }
template <typename R>
__device__ __forceinline__ R tlift(const Tab& t, int end, int i);
template <>
__device__ __forceinline__ float tlift<float>(const Tab& t, int end, int i) { return end ? t.L1f[i] : t.L0f[i]; }
template <>
__device__ __forceinline__ double tlift<double>(const Tab& t, int end, int i) { return end ? t.L1[i] : t.L0[i]; }

// weight Kd_iq phi_j(xi_q) of a Gauss-point flux derivative in the in-line
// block, formed in the precision of the derivative arithmetic (an FP64
// product converted to FP32 would put two FP64-pipe operations into every
// FP32 multiply-add of the assembly)
template <typename R>
__device__ __forceinline__ R kdphi(const Tab& t, int i, int q, int j);
template <>
__device__ __forceinline__ float kdphi<float>(const Tab& t, int i, int q, int j) {
  return t.Kdf[i][q] * t.Phif[q][j];
}
template <>
__device__ __forceinline__ double kdphi<double>(const Tab& t, int i, int q, int j) {
  return t.Kd[i][q] * t.Phi[q][j];
}

__device__ __forceinline__ int64_t tile_index(int64_t L, int64_t nk, int64_t k) {
  return ((L >> 5) * nk + k) * 32 + (L & 31);
}

// ---------------------------------------------------------------------------
// Tiled assembly: one block per 32-line tile of the K storage, two rounds
// (K11, then K12 for second-order equations), each in two phases.
//   Phase A, one thread per (line, Gauss point q) and (line, end): the
//   pointwise derivative matrices, written to shared memory lane-minor:
//     K11 round: A_q = d(F.n_q)/du (forward mode, all n_c directions in one
//                evaluation), B_end,side = dF^_end/du_inside / du_outside
//     K12 round: A_q = d(F^vis.n_q)/dq (F^vis is linear in q: one real
//                evaluation per unit q vector), C_end = the line end's
//                viscous-flux derivative when it enters the in-line block,
//                Cf = the face block's (the end whose switch takes the
//                viscous flux from outside)
//   Phase B, one thread per (line, row i, block column): the contraction
//     dr_i/du_j = -sum_q Kd_iq phi_j(xi_q) A_q + L_end,i B_end,in [j = end]
//   and the store; a warp covers the 32 lines of the tile for one entry, so
//   every store is one 128-byte (FP32) segment.
// The state, gradient and metric terms arrive at the arithmetic precision R
// (FP32 copies for the FP32 Jacobian), so the assembly is pure R.
// ---------------------------------------------------------------------------
template <typename R, int M>
__device__ __forceinline__ Dual<R, M> dseed(R v, int k) {
  Dual<R, M> x(0.0);
  x.v = v;
#pragma unroll
  for (int i = 0; i < M; ++i) x.d[i] = (i == k) ? R(1) : R(0);
  return x;
}
template <typename R, int M>
__device__ __forceinline__ Dual<R, M> dconst(R v) {
  Dual<R, M> x(0.0);
  x.v = v;
  return x;
}

// metric terms at the arithmetic precision R (FP32 copies made once per
// FP32 Jacobian object; the FP64 arrays themselves for R = double)
template <typename R>
struct GeoR {
  const R* ng;    // [E][D][nl][nq][D]
  const R* nend;  // [E][D][nl][2][D]
  const R* invJ;  // [E][npe]
};

template <int D, int P, int NC, int EQ, typename R>
struct JacTile {
  using S = Shape<D, P>;
  static constexpr int N = S::N, NQ = S::NQ, NPE = S::NPE, NL = S::NL, NCD = NC * D;
  static constexpr bool VISC = IsViscous<EQ>::value;
  // phase-A item kinds per line: K11 round: the four (end, side) face-flux
  // derivatives first (the heaviest items, one per warp of the block), then
  // the Gauss points; K12 round: the Gauss points and the two ends
  static constexpr int KINDS11 = 4 + NQ;
  static constexpr int KINDS12 = NQ + 2;
  // four warps per block and two blocks per SM: the derivative arithmetic
  // needs up to 255 registers a thread, and two blocks with their own
  // barriers let one block's stores overlap the other's arithmetic
  // K12 (ROUND 2) needs no dual numbers: eight warps per block
  template <int ROUND>
  static constexpr int threads() { return ROUND == 1 ? 128 : 256; }
  static constexpr int MINB = 2;
  static constexpr int SZ11 = (NQ * NC * NC + 4 * NC * NC) * 32;
  static constexpr int SZ12 = VISC ? (NQ * NC * NCD + 3 * NC * NCD) * 32 : 0;
  static constexpr int SMEM11 = SZ11 * (int)sizeof(R);
  static constexpr int SMEM12 = SZ12 * (int)sizeof(R) + 32 * (int)sizeof(int);
  static constexpr int64_t NK11 = (N * N + 2 * N) * NC * NC;
  static constexpr int64_t NK12 = VISC ? (N * N + N) * NC * NCD : 1;
  static constexpr int OFF11 = N * N * NC * NC;
  static constexpr int OFF12 = N * N * NC * NCD;
};

// line L -> (element, direction, first node, node stride)
template <int D, int P>
struct LineAt {
  int64_t e;
  int d, b0, st;
  __device__ __forceinline__ LineAt(int64_t L) {
    using S = Shape<D, P>;
    e = L / (D * S::NL);
    d = (int)((L / S::NL) % D);
    const int l = (int)(L % S::NL);
    st = S::stride(d);
    b0 = S::base(d, l);
  }
};

// d(F^.n)/du at one line end, seeded on the inside (SIDE 0) or outside
// (SIDE 1) trace: the interior, Neumann, no-slip wall and Dirichlet fluxes of
// the residual (Eqs. 25-30, the wall flux of the builder's wall reading)
template <int D, int NC, int EQ, typename R, int SIDE>
__device__ __forceinline__ void end_flux_derivative(const R* uin, const R* uo, const R* qin, const R* qo,
                                                    const R* nv, R nn, int nb, int swv, bool wall, bool neu,
                                                    const Phys<R>& pp, R* out /* [NC][NC] */) {
  using T = Dual<R, NC>;
  constexpr bool VISC = IsViscous<EQ>::value;
  constexpr int NCD = NC * D;
  T ui[NC], ux[NC], F[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    ui[c] = SIDE == 0 ? dseed<R, NC>(uin[c], c) : dconst<R, NC>(uin[c]);
    ux[c] = SIDE == 1 ? dseed<R, NC>(uo[c], c) : dconst<R, NC>(uo[c]);
    F[c] = dconst<R, NC>(R(0));
  }
  if (nb >= 0) {
    inviscid_numflux<EQ, D, T, R>(ux, ui, nv, pp, F);
    if constexpr (VISC) {
      // the viscous flux takes the trace of one side only: its derivative
      // with respect to the other side is zero and is not evaluated
      const bool from_out = swv == 1;
      if (from_out == (SIDE == 1)) {
        T qq[NCD], fv[NC];
#pragma unroll
        for (int cb = 0; cb < NCD; ++cb) qq[cb] = dconst<R, NC>(from_out ? qo[cb] : qin[cb]);
        viscous_flux_n<EQ, D, T, R>(SIDE == 1 ? ux : ui, qq, nv, pp, fv);
#pragma unroll
        for (int c = 0; c < NC; ++c) F[c] = F[c] + fv[c];
      }
      const R pen = pp.C11;  // per unit reference length
#pragma unroll
      for (int c = 0; c < NC; ++c) F[c] = F[c] + pen * (ui[c] - ux[c]);
    }
  } else if (neu || SIDE == 1) {
    // Neumann: the prescribed flux does not depend on the state; walls and
    // Dirichlet data have no outside trace
  } else if (wall) {
    if constexpr (NC == D + 2) {
      T m2 = ui[1] * ui[1];
#pragma unroll
      for (int a = 1; a < D; ++a) m2 = m2 + ui[1 + a] * ui[1 + a];
      const T pr = (pp.gamma - R(1)) * (ui[D + 1] - R(0.5) * m2 / ui[0]);
#pragma unroll
      for (int a = 0; a < D; ++a) F[1 + a] = pr * nv[a];
      if constexpr (VISC) {
        T ub[NC], qq[NCD], fv[NC];
        wall_state<D, T, R>(ui, ub);
#pragma unroll
        for (int cb = 0; cb < NCD; ++cb) qq[cb] = dconst<R, NC>(qin[cb]);
        viscous_flux_n<EQ, D, T, R>(ub, qq, nv, pp, fv);
        const R pen = pp.C11b * nn;
#pragma unroll
        for (int a = 0; a < D; ++a) F[1 + a] = F[1 + a] + fv[1 + a] + pen * (ui[1 + a] - ub[1 + a]);
      }
    }
  } else {
    // Dirichlet data g_D as the outside trace (constant)
    inviscid_numflux<EQ, D, T, R>(ux, ui, nv, pp, F);
    if constexpr (VISC) {
      T qq[NCD], fv[NC];
#pragma unroll
      for (int cb = 0; cb < NCD; ++cb) qq[cb] = dconst<R, NC>(qin[cb]);
      viscous_flux_n<EQ, D, T, R>(ui, qq, nv, pp, fv);
      const R pen = pp.C11b * nn;
#pragma unroll
      for (int c = 0; c < NC; ++c) F[c] = F[c] + fv[c] + pen * (ui[c] - ux[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int cp = 0; cp < NC; ++cp) out[c * NC + cp] = F[c].d[cp];
}

// ROUND 1 assembles K11 (and the wall rows Kw), ROUND 2 K12: two kernels,
// so each holds only its own code and shared memory
template <int D, int P, int NC, int EQ, typename R, int ROUND>
__global__ void __launch_bounds__(JacTile<D, P, NC, EQ, R>::template threads<ROUND>(), (JacTile<D, P, NC, EQ, R>::MINB))
    k_jacobian(const R* __restrict__ Ur, const R* __restrict__ Qr, R* __restrict__ K11, R* __restrict__ K12,
               R* __restrict__ Kw, Geo g, GeoR<R> gr, Tab tab, PhysArgs ph, int64_t nlines) {
  using JT = JacTile<D, P, NC, EQ, R>;
  using S = Shape<D, P>;
  constexpr int N = JT::N, NQ = JT::NQ, NPE = JT::NPE, NCD = JT::NCD;
  constexpr bool VISC = JT::VISC;
  extern __shared__ unsigned char smraw[];
  R* const sm = reinterpret_cast<R*>(smraw);
  int* const fend = reinterpret_cast<int*>(smraw + (JT::SMEM12 - 32 * (int)sizeof(int)));
  Phys<R> pp;
  pp.set(ph);
  const int64_t tile0 = (int64_t)blockIdx.x * 32;

  // ======================= K11 round =======================================
  if constexpr (ROUND == 1) {
  R* A = sm;                         // [NQ][NC][NC][32]
  R* B = sm + NQ * NC * NC * 32;     // [end][side][NC][NC][32]
  for (int it = threadIdx.x; it < 32 * JT::KINDS11; it += JT::template threads<ROUND>()) {
    const int lane = it & 31, kind = it >> 5;
    const int64_t L = tile0 + lane;
    if (L >= nlines) continue;
    const LineAt<D, P> ln(L);
    const R* ue = Ur + ln.e * NC * NPE;
    if (kind >= 4) {
      const int q = kind - 4;
      R n[D];
#pragma unroll
      for (int a = 0; a < D; ++a) n[a] = gr.ng[(L * NQ + q) * D + a];
      using T = Dual<R, NC>;
      T uq[NC], f[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        R s = 0;
#pragma unroll
        for (int t = 0; t < N; ++t) s += tphi<R>(tab, q, t) * ue[c * NPE + ln.b0 + t * ln.st];
        uq[c] = dseed<R, NC>(s, c);
      }
      inviscid_flux_n<EQ, D, T, R>(uq, n, pp, f);
      if constexpr (VISC) {
        const R* qe = Qr + ln.e * NCD * NPE;
        T qq[NCD], fv[NC];
#pragma unroll
        for (int cb = 0; cb < NCD; ++cb) {
          R s = 0;
#pragma unroll
          for (int t = 0; t < N; ++t) s += tphi<R>(tab, q, t) * qe[cb * NPE + ln.b0 + t * ln.st];
          qq[cb] = dconst<R, NC>(s);
        }
        viscous_flux_n<EQ, D, T, R>(uq, qq, n, pp, fv);
#pragma unroll
        for (int c = 0; c < NC; ++c) f[c] = f[c] + fv[c];
      }
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int cp = 0; cp < NC; ++cp) A[((q * NC + c) * NC + cp) * 32 + lane] = f[c].d[cp];
    } else {
      const int end = kind >> 1, side = kind & 1;
      const int aend = ln.b0 + end * P * ln.st;
      const int nb = g.nbr[L * 2 + end];
      const int swv = g.sw[(ln.e * D + ln.d) * 2 + end];
      const bool wall = nb < 0 && ph.bck[-1 - nb] == BC_WALL;
      const bool neu = nb < 0 && ph.bck[-1 - nb] == BC_NEUMANN;
      R nv[D], nn = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        nv[a] = gr.nend[(L * 2 + end) * D + a];
        nn += nv[a] * nv[a];
      }
      nn = sqrt(nn);
      R uin[NC], uo[NC], qin[VISC ? NCD : 1], qo[VISC ? NCD : 1];
#pragma unroll
      for (int c = 0; c < NC; ++c) uin[c] = ue[c * NPE + aend];
      if constexpr (VISC) {
#pragma unroll
        for (int cb = 0; cb < NCD; ++cb) qin[cb] = Qr[(ln.e * NCD + cb) * NPE + aend];
      }
      if (nb >= 0) {
        const int64_t eo = nb / NPE;
        const int ao = nb % NPE;
#pragma unroll
        for (int c = 0; c < NC; ++c) uo[c] = Ur[(eo * NC + c) * NPE + ao];
        if constexpr (VISC) {
#pragma unroll
          for (int cb = 0; cb < NCD; ++cb) qo[cb] = Qr[(eo * NCD + cb) * NPE + ao];
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) uo[c] = g.gD ? (R)g.gD[(ln.e * NC + c) * NPE + aend] : R(0);
        if constexpr (VISC) {
#pragma unroll
          for (int cb = 0; cb < NCD; ++cb) qo[cb] = R(0);
        }
      }
      // the gradient's trace at a no-slip wall is the wall state of the
      // inside trace: identity on rho, zero on momentum and the energy row
      // w = (|m|^2 / (2 rho^2), -m / rho, 1), stored per line end for the
      // K21 part of the split product
      if constexpr (VISC && NC == D + 2) {
        if (Kw && side == 0) {
          R w[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) w[c] = R(0);
          if (wall) {
            const R rho = uin[0];
            R m2 = R(0);
#pragma unroll
            for (int a = 0; a < D; ++a) m2 += uin[1 + a] * uin[1 + a];
            w[0] = m2 / (R(2) * rho * rho);
#pragma unroll
            for (int a = 0; a < D; ++a) w[1 + a] = -uin[1 + a] / rho;
            w[NC - 1] = R(1);
          }
#pragma unroll
          for (int c = 0; c < NC; ++c) Kw[tile_index(L, 2 * NC, end * NC + c)] = w[c];
        }
      }
      R dF[NC * NC];
      if (side == 0)
        end_flux_derivative<D, NC, EQ, R, 0>(uin, uo, qin, qo, nv, nn, nb, swv, wall, neu, pp, dF);
      else
        end_flux_derivative<D, NC, EQ, R, 1>(uin, uo, qin, qo, nv, nn, nb, swv, wall, neu, pp, dF);
#pragma unroll
      for (int k = 0; k < NC * NC; ++k) B[((end * 2 + side) * NC * NC + k) * 32 + lane] = dF[k];
    }
  }
  __syncthreads();
  // phase B: warp w takes the entries k = w, w + warps, ... of each row i;
  // per entry it reads the NQ + 4 pointwise values once and writes the N
  // in-line blocks and the two face blocks of the row (32 lines: one
  // 128-byte FP32 segment per store)
  {
    constexpr int NW = JT::template threads<ROUND>() / 32;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t L = tile0 + lane;
    const bool live = L < nlines;
    const LineAt<D, P> ln(live ? L : tile0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      R w[NQ][N];
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int j = 0; j < N; ++j) w[q][j] = kdphi<R>(tab, i, q, j);
      const R l0 = tlift<R>(tab, 0, i), l1 = tlift<R>(tab, 1, i);
      const R ij = live ? gr.invJ[ln.e * NPE + ln.b0 + i * ln.st] : R(0);
      for (int k = wp; k < NC * NC; k += NW) {
        R a[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) a[q] = A[(q * NC * NC + k) * 32 + lane];
        const R b00 = B[((0 * 2 + 0) * NC * NC + k) * 32 + lane], b10 = B[((1 * 2 + 0) * NC * NC + k) * 32 + lane];
        const R b01 = B[((0 * 2 + 1) * NC * NC + k) * 32 + lane], b11 = B[((1 * 2 + 1) * NC * NC + k) * 32 + lane];
        if (!live) continue;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          R s = (j == 0 ? l0 * b00 : R(0)) + (j == P ? l1 * b10 : R(0));
#pragma unroll
          for (int q = 0; q < NQ; ++q) s -= w[q][j] * a[q];
          K11[tile_index(L, JT::NK11, (i * N + j) * NC * NC + k)] = -ij * s;
        }
        K11[tile_index(L, JT::NK11, JT::OFF11 + (0 * N + i) * NC * NC + k)] = -ij * l0 * b01;
        K11[tile_index(L, JT::NK11, JT::OFF11 + (1 * N + i) * NC * NC + k)] = -ij * l1 * b11;
      }
    }
  }

  }  // ROUND == 1
  // ======================= K12 round: F^vis is linear in q ================
  if constexpr (VISC && ROUND == 2) {
    R* A2 = sm;                            // [NQ][NC][NCD][32]
    R* C2 = sm + NQ * NC * NCD * 32;       // [end][NC][NCD][32] in-line end terms
    R* Cf = C2 + 2 * NC * NCD * 32;        // [NC][NCD][32] face block
    for (int it = threadIdx.x; it < 32 * JT::KINDS12; it += JT::template threads<ROUND>()) {
      const int lane = it & 31, kind = it >> 5;
      const int64_t L = tile0 + lane;
      if (L >= nlines) continue;
      const LineAt<D, P> ln(L);
      const R* ue = Ur + ln.e * NC * NPE;
      if (kind < NQ) {
        const int q = kind;
        R n[D], uq[NC];
#pragma unroll
        for (int a = 0; a < D; ++a) n[a] = gr.ng[(L * NQ + q) * D + a];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          R s = 0;
#pragma unroll
          for (int t = 0; t < N; ++t) s += tphi<R>(tab, q, t) * ue[c * NPE + ln.b0 + t * ln.st];
          uq[c] = s;
        }
#pragma unroll 1
        for (int cb = 0; cb < NCD; ++cb) {
          R unit[NCD], fv[NC];
#pragma unroll
          for (int k = 0; k < NCD; ++k) unit[k] = (k == cb) ? R(1) : R(0);
          viscous_flux_n<EQ, D, R, R>(uq, unit, n, pp, fv);
#pragma unroll
          for (int c = 0; c < NC; ++c) A2[((q * NC + c) * NCD + cb) * 32 + lane] = fv[c];
        }
      } else {
        const int end = kind - NQ;
        const int aend = ln.b0 + end * P * ln.st;
        const int nb = g.nbr[L * 2 + end];
        const int swv = g.sw[(ln.e * D + ln.d) * 2 + end];
        const bool wall = nb < 0 && ph.bck[-1 - nb] == BC_WALL;
        const bool neu = nb < 0 && ph.bck[-1 - nb] == BC_NEUMANN;
        const bool outside = nb >= 0 && swv == 1;
        R nv[D], ut[NC];
#pragma unroll
        for (int a = 0; a < D; ++a) nv[a] = gr.nend[(L * 2 + end) * D + a];
        if (outside) {
          const int64_t eo = nb / NPE;
          const int ao = nb % NPE;
#pragma unroll
          for (int c = 0; c < NC; ++c) ut[c] = Ur[(eo * NC + c) * NPE + ao];
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c) ut[c] = ue[c * NPE + aend];
        }
        bool walled = false;
        if constexpr (NC == D + 2) {
          if (wall) {
            // the wall's viscous flux: wall state, momentum components only
            R ub[NC];
            wall_state<D, R, R>(ut, ub);
#pragma unroll
            for (int c = 0; c < NC; ++c) ut[c] = ub[c];
            walled = true;
          }
        }
        if (swv == 1) fend[lane] = end;
#pragma unroll 1
        for (int cb = 0; cb < NCD; ++cb) {
          R unit[NCD], fv[NC];
#pragma unroll
          for (int k = 0; k < NCD; ++k) unit[k] = (k == cb) ? R(1) : R(0);
          viscous_flux_n<EQ, D, R, R>(ut, unit, nv, pp, fv);
          if (walled) {
            fv[0] = R(0);
            fv[NC - 1] = R(0);
          }
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            C2[((end * NC + c) * NCD + cb) * 32 + lane] = (!outside && !neu) ? fv[c] : R(0);
            if (swv == 1) Cf[(c * NCD + cb) * 32 + lane] = outside ? fv[c] : R(0);
          }
        }
      }
    }
    __syncthreads();
    // phase B: as in the K11 round, warp w takes entries k = w, w + warps,
    // ... of each row i: NQ + 3 reads, N + 1 stores
    {
      constexpr int NW = JT::template threads<ROUND>() / 32;
      const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
      const int64_t L = tile0 + lane;
      const bool live = L < nlines;
      const LineAt<D, P> ln(live ? L : tile0);
      const int fe = live ? fend[lane] : 0;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        R w[NQ][N];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int j = 0; j < N; ++j) w[q][j] = kdphi<R>(tab, i, q, j);
        const R l0 = tlift<R>(tab, 0, i), l1 = tlift<R>(tab, 1, i), li = tlift<R>(tab, fe, i);
        const R ij = live ? gr.invJ[ln.e * NPE + ln.b0 + i * ln.st] : R(0);
        for (int k = wp; k < NC * NCD; k += NW) {
          R a[NQ];
#pragma unroll
          for (int q = 0; q < NQ; ++q) a[q] = A2[(q * NC * NCD + k) * 32 + lane];
          const R c0 = C2[(0 * NC * NCD + k) * 32 + lane], c1 = C2[(1 * NC * NCD + k) * 32 + lane];
          const R cf = Cf[k * 32 + lane];
          if (!live) continue;
#pragma unroll
          for (int j = 0; j < N; ++j) {
            R s = (j == 0 ? l0 * c0 : R(0)) + (j == P ? l1 * c1 : R(0));
#pragma unroll
            for (int q = 0; q < NQ; ++q) s -= w[q][j] * a[q];
            K12[tile_index(L, JT::NK12, (i * N + j) * NC * NCD + k)] = -ij * s;
          }
          K12[tile_index(L, JT::NK12, JT::OFF12 + i * NC * NCD + k)] = -ij * li * cf;
        }
      }
    }
  }
}

template <int D, int P, int EQ, typename R>
cudaError_t run_jacobian(const ldg_handle* h, const R* Ur, const R* Qr, R* K11, R* K12, R* Kw, GeoR<R> gr,
                         cudaStream_t st) {
  constexpr int NC = NComp<EQ, D>::value;
  using JT = JacTile<D, P, NC, EQ, R>;
  constexpr bool VISC = IsViscous<EQ>::value;
  for (int round = 1; round <= (VISC ? 2 : 1); ++round) {
    auto kern = round == 1 ? k_jacobian<D, P, NC, EQ, R, 1> : k_jacobian<D, P, NC, EQ, R, 2>;
    const int smem = round == 1 ? JT::SMEM11 : JT::SMEM12;
    cudaError_t err = set_smem_once(kern, smem);
    if (err != cudaSuccess) return err;
    // shared memory before L1: several blocks per SM need several tile buffers
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)h->ntiles(), round == 1 ? JT::template threads<1>() : JT::template threads<2>(), smem, st>>>(
        Ur, Qr, K11, K12, Kw, h->geo(), gr, h->tab, h->phys, h->nlines());
    count_launch();
  }
  return cudaGetLastError();
}

// FP32 copy of an FP64 array (the state and gradient of an FP32 Jacobian:
// converted once, so the assembly spends no FP64 operations)
static __global__ void k_to_float(float* __restrict__ out, const double* __restrict__ in, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// K21 = dQ/dU, scalar and component-independent (Sec. 4.2), built in FP64:
//   in-line [(i N + j) D + b] = (1/J_i) (-sum_q Kd_iq n_d,b(xi_q) phi_j(xi_q)
//                               + L_e,i n_e,b [j = end node, interior with
//                                 S_e = +1, or a Neumann boundary end])
//   face    [N^2 D + i D + b] = (1/J_i) L_e,i n_e,b for the interior end with S_e = -1
template <int D, int P, typename R>
__global__ void k_build_k21(R* __restrict__ K21, Geo g, Tab tab, PhysArgs ph, int64_t NL) {
  using S = Shape<D, P>;
  constexpr int N = S::N, NPE = S::NPE, NQ = S::NQ;
  constexpr int64_t NK = (N * N + N) * D;
  const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= NL) return;
  const int64_t e = L / (D * S::NL);
  const int d = (int)((L / S::NL) % D), l = (int)(L % S::NL);
  const int st = S::stride(d), b0 = S::base(d, l);
  double nq[NQ][D], nv[2][D];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int a = 0; a < D; ++a) nq[q][a] = g.ng[(L * NQ + q) * D + a];
#pragma unroll
  for (int end = 0; end < 2; ++end)
#pragma unroll
    for (int a = 0; a < D; ++a) nv[end][a] = g.nend[(L * 2 + end) * D + a];
  int nb[2], swv[2];
  bool own[2];  // the end's trace u^ is this line's own end node
#pragma unroll
  for (int end = 0; end < 2; ++end) {
    nb[end] = g.nbr[L * 2 + end];
    swv[end] = g.sw[(e * D + d) * 2 + end];
    own[end] = nb[end] >= 0 ? swv[end] == 1 : ph.bck[-1 - nb[end]] == BC_NEUMANN;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double ij = g.invJ[e * NPE + b0 + i * st];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) s -= tab.Kd[i][q] * nq[q][b] * tab.Phi[q][j];
#pragma unroll
        for (int end = 0; end < 2; ++end)
          if (j == end * P && own[end]) s += (end ? tab.L1[i] : tab.L0[i]) * nv[end][b];
        K21[tile_index(L, NK, (i * N + j) * D + b)] = (R)(ij * s);
      }
#pragma unroll
    for (int b = 0; b < D; ++b) {
      double s = 0.0;
#pragma unroll
      for (int end = 0; end < 2; ++end)
        if (nb[end] >= 0 && swv[end] == -1) s += (end ? tab.L1[i] : tab.L0[i]) * nv[end][b];
      K21[tile_index(L, NK, N * N * D + i * D + b)] = (R)(ij * s);
    }
  }
}

template <int D, int P, typename R>
cudaError_t run_k21(const ldg_handle* h, R* K21, cudaStream_t st) {
  const int64_t NL = h->nlines();
  k_build_k21<D, P, R><<<(unsigned)((NL + 127) / 128), 128, 0, st>>>(K21, h->geo(), h->tab, h->phys, NL);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ldg
