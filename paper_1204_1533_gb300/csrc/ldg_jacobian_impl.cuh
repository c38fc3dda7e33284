// Line-sparse Jacobian assembly (Sec. 4.1 Eq. 35: K11 = dR/dU, K12 = dR/dQ,
// K21 = dD/dU; Sec. 2.3 sparsity).
//
// For a line of direction d, R_i = -(1/J_i) r_i with r from Eq. 7, so
//   dr_i/du_j     = -sum_q Kd_iq (dF.n/du)(xi_q) phi_j(xi_q)
//                   + L1_i dF^+/du_in [j = p] + L0_i dF^-/du_in [j = 0]
//   dr_i/du_out,e = L_e,i dF^e/du_out                      (face block)
// and likewise for q. One thread per line; columns are produced one at a
// time by forward-mode derivatives seeded on a single component (Dual<R,1>),
// which keeps the (p+1)^2 n_c accumulators of a column in registers. The
// viscous flux is linear in q, so K12's columns are flux evaluations with
// unit q vectors. Values are computed at precision R (float: the mixed
// path, FP32 values from the FP64 state; double: the all-FP64 path) and
// stored entry-major in 32-line tiles so each warp's stores are coalesced.
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

template <int D, int P, int NC, int EQ, typename R>
__global__ void __launch_bounds__(Shape<D, P>::THREADS)
    k_jacobian(const double* __restrict__ U, const double* __restrict__ Q, R* __restrict__ K11,
               R* __restrict__ K12, R* __restrict__ Kw, Geo g, Tab tab, PhysArgs ph) {
  using S = Shape<D, P>;
  using T = Dual<R, 1>;
  constexpr int N = S::N, NPE = S::NPE, NQ = S::NQ, NCD = NC * D;
  constexpr bool VISC = IsViscous<EQ>::value;
  constexpr int tile = NC * NPE;
  constexpr int qtile = VISC ? NCD * NPE : 0;
  constexpr int64_t NK11 = (N * N + 2 * N) * NC * NC;
  constexpr int64_t NK12 = VISC ? (N * N + N) * NC * NCD : 1;
  constexpr int OFF11 = N * N * NC * NC;
  constexpr int OFF12 = N * N * NC * NCD;
  extern __shared__ unsigned char smraw[];
  R* sU = reinterpret_cast<R*>(smraw);
  R* sQ = sU + S::EPB * tile;
  const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
  const int ne = (int)min((int64_t)S::EPB, g.E - e0);
  for (int k = threadIdx.x; k < ne * tile; k += blockDim.x) sU[k] = (R)U[e0 * tile + k];
  if constexpr (VISC)
    for (int k = threadIdx.x; k < ne * qtile; k += blockDim.x) sQ[k] = (R)Q[e0 * qtile + k];
  __syncthreads();
  const int le = threadIdx.x / S::TPE, rr = threadIdx.x % S::TPE;
  if (le >= ne) return;
  const int d = rr / S::NL, l = rr % S::NL;
  const int64_t e = e0 + le;
  const int64_t L = (e * D + d) * S::NL + l;
  const int st = S::stride(d), b0 = S::base(d, l);
  const R* uel = sU + le * tile;
  const R* qel = sQ + le * qtile;
  // this line's normals at its Gauss points, converted once into a
  // per-thread shared slot ([k][thread]: conflict-free)
  R* sN = sQ + S::EPB * qtile;
#pragma unroll
  for (int k = 0; k < NQ * D; ++k) sN[k * S::THREADS + threadIdx.x] = (R)g.ng[L * NQ * D + k];
  Phys<R> pp;
  pp.set(ph);
  R ij[N];
#pragma unroll
  for (int i = 0; i < N; ++i) ij[i] = (R)g.invJ[e * NPE + b0 + i * st];
  // end data
  int32_t nb[2];
  int swv[2];
  bool wall[2], neu[2];
  R nv[2][D], nn[2], uin[2][NC], uo[2][NC];
  R qin[2][VISC ? NCD : 1], qo[2][VISC ? NCD : 1];
#pragma unroll
  for (int end = 0; end < 2; ++end) {
    const int aend = b0 + end * P * st;
    nb[end] = g.nbr[L * 2 + end];
    swv[end] = g.sw[(e * D + d) * 2 + end];
    wall[end] = nb[end] < 0 && ph.bck[-1 - nb[end]] == BC_WALL;
    neu[end] = nb[end] < 0 && ph.bck[-1 - nb[end]] == BC_NEUMANN;
    R s = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      nv[end][a] = (R)g.nend[(L * 2 + end) * D + a];
      s += nv[end][a] * nv[end][a];
    }
    nn[end] = sqrt(s);
#pragma unroll
    for (int c = 0; c < NC; ++c) uin[end][c] = uel[c * NPE + aend];
    if constexpr (VISC) {
#pragma unroll
      for (int cb = 0; cb < NCD; ++cb) qin[end][cb] = qel[cb * NPE + aend];
    }
    if (nb[end] >= 0) {
      const int64_t eo = nb[end] / NPE;
      const int ao = nb[end] % NPE;
#pragma unroll
      for (int c = 0; c < NC; ++c) uo[end][c] = (R)U[eo * tile + c * NPE + ao];
      if constexpr (VISC) {
#pragma unroll
        for (int cb = 0; cb < NCD; ++cb) qo[end][cb] = (R)Q[(eo * NCD + cb) * NPE + ao];
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) uo[end][c] = g.gD ? (R)g.gD[e * tile + c * NPE + aend] : R(0);
      if constexpr (VISC) {
#pragma unroll
        for (int cb = 0; cb < NCD; ++cb) qo[end][cb] = R(0);
      }
    }
  }

  // the gradient's trace at a no-slip wall is the wall state of the inside
  // trace: its derivative is the identity on rho, zero on momentum, and the
  // energy row w = (|m|^2 / (2 rho^2), -m / rho, 1); w is stored per line end
  // (zero at other ends) for the K21 part of the split product
  if constexpr (VISC && NC == D + 2) {
    if (Kw) {
#pragma unroll
      for (int end = 0; end < 2; ++end) {
        R w[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) w[c] = R(0);
        if (wall[end]) {
          const R rho = uin[end][0];
          R m2 = R(0);
#pragma unroll
          for (int a = 0; a < D; ++a) m2 += uin[end][1 + a] * uin[end][1 + a];
          w[0] = m2 / (R(2) * rho * rho);
#pragma unroll
          for (int a = 0; a < D; ++a) w[1 + a] = -uin[end][1 + a] / rho;
          w[NC - 1] = R(1);
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) Kw[tile_index(L, 2 * NC, end * NC + c)] = w[c];
      }
    }
  }

  // ---------------- K11: one column (component cp of u) at a time ---------
#pragma unroll 1
  for (int cp = 0; cp < NC; ++cp) {
    R acc[N][N][NC];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[i][j][c] = R(0);
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      R n[D];
#pragma unroll
      for (int a = 0; a < D; ++a) n[a] = sN[(q * D + a) * S::THREADS + threadIdx.x];
      T uq[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        R s = 0;
#pragma unroll
        for (int t = 0; t < N; ++t) s += tphi<R>(tab, q, t) * uel[c * NPE + b0 + t * st];
        uq[c] = D1<R>::seed(s, c == cp);
      }
      T f[NC];
      inviscid_flux_n<EQ, D, T, R>(uq, n, pp, f);
      if constexpr (VISC) {
        T qq[NCD], fv[NC];
#pragma unroll
        for (int cb = 0; cb < NCD; ++cb) {
          R s = 0;
#pragma unroll
          for (int t = 0; t < N; ++t) s += tphi<R>(tab, q, t) * qel[cb * NPE + b0 + t * st];
          qq[cb] = D1<R>::cst(s);
        }
        viscous_flux_n<EQ, D, T, R>(uq, qq, n, pp, fv);
#pragma unroll
        for (int c = 0; c < NC; ++c) f[c] = f[c] + fv[c];
      }
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const R w = kdphi<R>(tab, i, q, j);
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[i][j][c] -= w * f[c].d[0];
        }
    }
#pragma unroll
    for (int end = 0; end < 2; ++end) {
      const int jn = end * P;
      // derivative w.r.t. the inside trace (column of the in-line block at jn)
      // and w.r.t. the outside trace (face block)
#pragma unroll 1
      for (int side = 0; side < 2; ++side) {
        T ui[NC], ux[NC], F[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          ui[c] = D1<R>::seed(uin[end][c], side == 0 && c == cp);
          ux[c] = D1<R>::seed(uo[end][c], side == 1 && c == cp);
        }
        if (nb[end] >= 0) {
          inviscid_numflux<EQ, D, T, R>(ux, ui, nv[end], pp, F);
          if constexpr (VISC) {
            T qq[NCD], fv[NC];
            if (swv[end] == 1) {
#pragma unroll
              for (int cb = 0; cb < NCD; ++cb) qq[cb] = D1<R>::cst(qo[end][cb]);
              viscous_flux_n<EQ, D, T, R>(ux, qq, nv[end], pp, fv);
            } else {
#pragma unroll
              for (int cb = 0; cb < NCD; ++cb) qq[cb] = D1<R>::cst(qin[end][cb]);
              viscous_flux_n<EQ, D, T, R>(ui, qq, nv[end], pp, fv);
            }
            const R pen = pp.C11 * nn[end];
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c] = F[c] + fv[c] + pen * (ui[c] - ux[c]);
          }
        } else if (neu[end]) {
          // Neumann: the prescribed flux does not depend on the state
#pragma unroll
          for (int c = 0; c < NC; ++c) F[c] = D1<R>::cst(R(0));
        } else if (wall[end]) {
          // no-slip adiabatic wall: pressure flux, viscous momentum flux of
          // the wall state, momentum penalty; no outside trace
          if (side == 1) {
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c] = D1<R>::cst(R(0));
          } else if constexpr (NC != D + 2) {
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c] = D1<R>::cst(R(0));
          } else {
            T m2 = ui[1] * ui[1];
#pragma unroll
            for (int a = 1; a < D; ++a) m2 = m2 + ui[1 + a] * ui[1 + a];
            const T pr = (pp.gamma - R(1)) * (ui[D + 1] - R(0.5) * m2 / ui[0]);
            F[0] = D1<R>::cst(R(0));
#pragma unroll
            for (int a = 0; a < D; ++a) F[1 + a] = pr * nv[end][a];
            F[D + 1] = D1<R>::cst(R(0));
            if constexpr (VISC) {
              T ub[NC], qq[NCD], fv[NC];
              wall_state<D, T, R>(ui, ub);
#pragma unroll
              for (int cb = 0; cb < NCD; ++cb) qq[cb] = D1<R>::cst(qin[end][cb]);
              viscous_flux_n<EQ, D, T, R>(ub, qq, nv[end], pp, fv);
              const R pen = pp.C11b * nn[end];
#pragma unroll
              for (int a = 0; a < D; ++a) F[1 + a] = F[1 + a] + fv[1 + a] + pen * (ui[1 + a] - ub[1 + a]);
            }
          }
        } else {
          // Dirichlet data: the outside trace is g_D, constant
          if (side == 1) {
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c] = D1<R>::cst(R(0));
          } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) ux[c] = D1<R>::cst(uo[end][c]);
            inviscid_numflux<EQ, D, T, R>(ux, ui, nv[end], pp, F);
            if constexpr (VISC) {
              T qq[NCD], fv[NC];
#pragma unroll
              for (int cb = 0; cb < NCD; ++cb) qq[cb] = D1<R>::cst(qin[end][cb]);
              viscous_flux_n<EQ, D, T, R>(ui, qq, nv[end], pp, fv);
              const R pen = pp.C11b * nn[end];
#pragma unroll
              for (int c = 0; c < NC; ++c) F[c] = F[c] + fv[c] + pen * (ui[c] - ux[c]);
            }
          }
        }
        if (side == 0) {
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const R li = tlift<R>(tab, end, i);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[i][jn][c] += li * F[c].d[0];
          }
        } else {
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const R li = tlift<R>(tab, end, i);
#pragma unroll
            for (int c = 0; c < NC; ++c)
              K11[tile_index(L, NK11, OFF11 + ((end * N + i) * NC + c) * NC + cp)] = -ij[i] * li * F[c].d[0];
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j)
#pragma unroll
        for (int c = 0; c < NC; ++c)
          K11[tile_index(L, NK11, ((i * N + j) * NC + c) * NC + cp)] = -ij[i] * acc[i][j][c];
  }

  // ---------------- K12: the viscous flux is linear in q -----------------
  if constexpr (VISC) {
#pragma unroll 1
    for (int cb = 0; cb < NCD; ++cb) {
      R unit[NCD];
#pragma unroll
      for (int k = 0; k < NCD; ++k) unit[k] = (k == cb) ? R(1) : R(0);
      R acc[N][N][NC];
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[i][j][c] = R(0);
#pragma unroll 1
      for (int q = 0; q < NQ; ++q) {
        R n[D], uq[NC], fv[NC];
#pragma unroll
        for (int a = 0; a < D; ++a) n[a] = sN[(q * D + a) * S::THREADS + threadIdx.x];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          R s = 0;
#pragma unroll
          for (int t = 0; t < N; ++t) s += tphi<R>(tab, q, t) * uel[c * NPE + b0 + t * st];
          uq[c] = s;
        }
        viscous_flux_n<EQ, D, R, R>(uq, unit, n, pp, fv);
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
          for (int j = 0; j < N; ++j) {
            const R w = kdphi<R>(tab, i, q, j);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[i][j][c] -= w * fv[c];
          }
      }
#pragma unroll
      for (int end = 0; end < 2; ++end) {
        const int jn = end * P;
        const bool outside = nb[end] >= 0 && swv[end] == 1;
        R fv[NC];
        bool walled = false;
        if constexpr (NC == D + 2) {
          if (wall[end]) {
            // the wall's viscous flux: wall state, momentum components only
            R ub[NC];
            wall_state<D, R, R>(uin[end], ub);
            viscous_flux_n<EQ, D, R, R>(ub, unit, nv[end], pp, fv);
            fv[0] = R(0);
            fv[NC - 1] = R(0);
            walled = true;
          }
        }
        if (!walled) viscous_flux_n<EQ, D, R, R>(outside ? uo[end] : uin[end], unit, nv[end], pp, fv);
        if (!outside && !neu[end]) {
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const R li = tlift<R>(tab, end, i);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[i][jn][c] += li * fv[c];
          }
        }
        if (swv[end] == 1) {  // the face block belongs to the S = +1 end
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const R li = tlift<R>(tab, end, i);
#pragma unroll
            for (int c = 0; c < NC; ++c)
              K12[tile_index(L, NK12, OFF12 + (i * NC + c) * NCD + cb)] =
                  outside ? -ij[i] * li * fv[c] : R(0);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
          for (int c = 0; c < NC; ++c)
            K12[tile_index(L, NK12, ((i * N + j) * NC + c) * NCD + cb)] = -ij[i] * acc[i][j][c];
    }
  }
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

template <int D, int P, int EQ, typename R>
cudaError_t run_jacobian(const ldg_handle* h, const double* U, const double* Q, R* K11, R* K12, R* Kw,
                         cudaStream_t st) {
  using S = Shape<D, P>;
  constexpr int NC = NComp<EQ, D>::value;
  constexpr bool VISC = IsViscous<EQ>::value;
  const size_t smem = ((size_t)S::EPB * (NC * S::NPE + (VISC ? NC * D * S::NPE : 0)) +
                       (size_t)S::THREADS * S::NQ * D) * sizeof(R);
  auto kern = k_jacobian<D, P, NC, EQ, R>;
  cudaError_t err = set_smem_once(kern, smem);
  if (err != cudaSuccess) return err;
  const int64_t blocks = (h->E + S::EPB - 1) / S::EPB;
  kern<<<(unsigned)blocks, S::THREADS, smem, st>>>(U, Q, K11, K12, Kw, h->geo(), h->tab, h->phys);
  count_launch();
  return cudaGetLastError();
}

template <int D, int P, typename R>
cudaError_t run_k21(const ldg_handle* h, R* K21, cudaStream_t st) {
  const int64_t NL = h->nlines();
  k_build_k21<D, P, R><<<(unsigned)((NL + 127) / 128), 128, 0, st>>>(K21, h->geo(), h->tab, h->phys, NL);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ldg
