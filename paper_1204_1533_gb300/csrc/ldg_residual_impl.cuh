// FP64 LDG gradient and residual kernels (Sec. 2.1 Eq. 7, Sec. 3 Eqs. 19-32).
//
// Work decomposition: one thread per coordinate line (element e, direction
// d, line l); a block holds EPB whole elements so that the element tile of
// U (and Q) is staged once in shared memory with coalesced loads, every line
// reads its nodes from there, and the D directional results r^(d) of an
// element are summed in shared memory before one coalesced store of
// R = -(1/J) sum_d r^(d) + S. Neighbour traces are single-node gathers.
// FP64 is the binding resource on GB300 (about 1 TFLOP/s against 70 TFLOP/s
// FP32), so every geometric quantity (n_d at Gauss points, n^+- at line
// ends, 1/J) is precomputed and the kernels spend FP64 only on the scheme.
#pragma once
#include "ldg_internal.h"
#include "ldg_physics.cuh"

namespace ldg {

// elements per block: whole 32-line tiles when a block of at most 512
// threads can cover them (so tiled Jacobian accesses of a block never share
// a 128-byte line with another block), otherwise about 128 threads
__host__ __device__ constexpr int elems_per_block(int tpe) {
  int best = 0;
  for (int e = 1; e <= 64 && e * tpe <= 512; ++e)
    if ((e * tpe) % 32 == 0 && (best == 0 || (e * tpe >= 64 && best * tpe < 64))) best = e;
  if (best) return best;
  return tpe >= 128 ? 1 : 128 / tpe;
}

template <int D, int P>
struct Shape {
  static constexpr int N = P + 1;
  static constexpr int NPE = (D == 2) ? N * N : N * N * N;
  static constexpr int NL = (D == 2) ? N : N * N;
  static constexpr int NQ = (3 * P + 2) / 2;
  static constexpr int TPE = D * NL;
  static constexpr int EPB = elems_per_block(TPE);
  static constexpr int THREADS = EPB * TPE;
  __device__ __forceinline__ static int stride(int d) { return d == 0 ? 1 : (d == 1 ? N : N * N); }
  __device__ __forceinline__ static int base(int d, int l) {
    const int s = stride(d);
    return (l % s) + (l / s) * s * N;
  }
};

// ---------------------------------------------------------------------------
// Q = D(U): per line d^(d)_i = L1_i u^+ n^+ + L0_i u^- n^- - sum_q Kd_iq u(xi_q) n_d(xi_q)
// With Qs (scalar Poisson, C22 != 0) the trace at interior ends adds
// C22 (F.n^(in) - F.n^(out)) with F = -q and the unit normal, and at Neumann
// ends C22 (F.n^(in) - G.n): D(U, Q) of the stabilised scheme (Eqs. 26, 30).
// ---------------------------------------------------------------------------
template <int D, int P, int NC>
__global__ void __launch_bounds__(Shape<D, P>::THREADS)
    k_gradient(const double* __restrict__ U, const double* __restrict__ Qs, double* __restrict__ Q, Geo g,
               Tab tab, PhysArgs ph) {
  using S = Shape<D, P>;
  constexpr int N = S::N, NPE = S::NPE, NQ = S::NQ;
  constexpr int tile = NC * NPE;
  extern __shared__ double sm[];
  double* sU = sm;
  double* sG = sm + S::EPB * tile;  // [EPB][D dir][NC][D a][NPE]
  const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
  const int ne = (int)min((int64_t)S::EPB, g.E - e0);
  for (int k = threadIdx.x; k < ne * tile; k += blockDim.x) sU[k] = U[e0 * tile + k];
  __syncthreads();
  const int le = threadIdx.x / S::TPE, r = threadIdx.x % S::TPE;
  if (le < ne) {
    const int d = r / S::NL, l = r % S::NL;
    const int64_t e = e0 + le;
    const int64_t L = (e * D + d) * S::NL + l;
    const int st = S::stride(d), b0 = S::base(d, l);
    const double* uel = sU + le * tile;
    double nq[NQ][D], nv[2][D];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int a = 0; a < D; ++a) nq[q][a] = g.ng[(L * NQ + q) * D + a];
#pragma unroll
    for (int end = 0; end < 2; ++end)
#pragma unroll
      for (int a = 0; a < D; ++a) nv[end][a] = g.nend[(L * 2 + end) * D + a];
    // trace u^ at both ends (Eq. 26; Eq. 28 at Dirichlet faces, Eq. 30 at
    // Neumann faces)
    double uh[2][NC];
#pragma unroll
    for (int end = 0; end < 2; ++end) {
      const int aend = b0 + end * P * st;
      const int32_t nb = g.nbr[L * 2 + end];
      double uin[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) uin[c] = uel[c * NPE + aend];
      // stabilised scheme: unit-normal flux F.n/|n| = -q.n/|n| of the inside trace
      double fin = 0.0, nrm = 1.0;
      const bool stab = NC == 1 && Qs != nullptr;
      if (stab) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) s += nv[end][a] * nv[end][a];
        nrm = sqrt(s);
#pragma unroll
        for (int a = 0; a < D; ++a) fin -= Qs[(e * D + a) * NPE + aend] * nv[end][a];
        fin /= nrm;
      }
      if (nb >= 0) {
        const int64_t eo = nb / NPE;
        const int ao = nb % NPE;
        if (g.sw[(e * D + d) * 2 + end] == 1) {
#pragma unroll
          for (int c = 0; c < NC; ++c) uh[end][c] = uin[c];
        } else {
#pragma unroll
          for (int c = 0; c < NC; ++c) uh[end][c] = U[eo * tile + c * NPE + ao];
        }
        if (stab) {
          double fout = 0.0;
#pragma unroll
          for (int a = 0; a < D; ++a) fout -= Qs[(eo * D + a) * NPE + ao] * nv[end][a];
          uh[end][0] += ph.C22 * (fin - fout / nrm);
        }
      } else {
        const int kind = ph.bck[-1 - nb];
        if (kind == BC_NEUMANN) {
#pragma unroll
          for (int c = 0; c < NC; ++c) uh[end][c] = uin[c];
          if (stab) {
            double gn = 0.0;
            if (g.gN)
#pragma unroll
              for (int a = 0; a < D; ++a) gn += g.gN[(e * D + a) * NPE + aend] * nv[end][a];
            uh[end][0] += ph.C22 * (fin - gn / nrm);
          }
          continue;
        }
        if constexpr (NC == D + 2) {
          if (kind == BC_WALL) {
            wall_state<D, double, double>(uin, uh[end]);
            continue;
          }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) uh[end][c] = g.gD ? g.gD[e * tile + c * NPE + aend] : 0.0;
      }
    }
    double* gout = sG + (size_t)(le * D + d) * NC * D * NPE;
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
      double ul[N];
#pragma unroll
      for (int t = 0; t < N; ++t) ul[t] = uel[c * NPE + b0 + t * st];
      double acc[N][D];
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int a = 0; a < D; ++a)
          acc[i][a] = tab.L1[i] * uh[1][c] * nv[1][a] + tab.L0[i] * uh[0][c] * nv[0][a];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        double uq = tab.Phi[q][0] * ul[0];
#pragma unroll
        for (int t = 1; t < N; ++t) uq = fma(tab.Phi[q][t], ul[t], uq);
#pragma unroll
        for (int a = 0; a < D; ++a) {
          const double w = uq * nq[q][a];
#pragma unroll
          for (int i = 0; i < N; ++i) acc[i][a] = fma(-tab.Kd[i][q], w, acc[i][a]);
        }
      }
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int i = 0; i < N; ++i) gout[(c * D + a) * NPE + b0 + i * st] = acc[i][a];
    }
  }
  __syncthreads();
  constexpr int qt = NC * D * NPE;
  for (int k = threadIdx.x; k < ne * qt; k += blockDim.x) {
    const int le2 = k / qt, rem = k % qt, node = rem % NPE;
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) s += sG[(size_t)(le2 * D + d) * qt + rem];
    Q[e0 * qt + k] = s * g.invJ[(e0 + le2) * NPE + node];
  }
}

// ---------------------------------------------------------------------------
// R = -(1/J) sum_d r^(d) + S with r^(d) from Eq. 7 along every line
// ---------------------------------------------------------------------------
template <int D, int P, int NC, int EQ>
__global__ void __launch_bounds__(Shape<D, P>::THREADS)
    k_residual(const double* __restrict__ U, const double* __restrict__ Q, double* __restrict__ R,
               Geo g, Tab tab, PhysArgs ph) {
  using S = Shape<D, P>;
  constexpr int N = S::N, NPE = S::NPE, NQ = S::NQ;
  constexpr bool VISC = IsViscous<EQ>::value;
  constexpr int tile = NC * NPE;
  constexpr int qtile = VISC ? NC * D * NPE : 0;
  extern __shared__ double sm[];
  double* sU = sm;
  double* sQ = sm + S::EPB * tile;
  double* sR = sQ + S::EPB * qtile;  // [EPB][D][NC][NPE]
  const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
  const int ne = (int)min((int64_t)S::EPB, g.E - e0);
  for (int k = threadIdx.x; k < ne * tile; k += blockDim.x) sU[k] = U[e0 * tile + k];
  if constexpr (VISC)
    for (int k = threadIdx.x; k < ne * qtile; k += blockDim.x) sQ[k] = Q[e0 * qtile + k];
  __syncthreads();
  Phys<double> pp;
  pp.set(ph);
  const int le = threadIdx.x / S::TPE, rr = threadIdx.x % S::TPE;
  if (le < ne) {
    const int d = rr / S::NL, l = rr % S::NL;
    const int64_t e = e0 + le;
    const int64_t L = (e * D + d) * S::NL + l;
    const int st = S::stride(d), b0 = S::base(d, l);
    const double* uel = sU + le * tile;
    const double* qel = sQ + le * qtile;
    double r[N][NC];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < NC; ++c) r[i][c] = 0.0;
    // volume term: - sum_q Kd_iq F(u(xi_q)) . n_d(xi_q)
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      double nv[D];
#pragma unroll
      for (int a = 0; a < D; ++a) nv[a] = g.ng[(L * NQ + q) * D + a];
      double uq[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double s = tab.Phi[q][0] * uel[c * NPE + b0];
#pragma unroll
        for (int t = 1; t < N; ++t) s = fma(tab.Phi[q][t], uel[c * NPE + b0 + t * st], s);
        uq[c] = s;
      }
      double f[NC];
      inviscid_flux_n<EQ, D, double, double>(uq, nv, pp, f);
      if constexpr (VISC) {
        double qq[NC * D];
#pragma unroll
        for (int cb = 0; cb < NC * D; ++cb) {
          double s = tab.Phi[q][0] * qel[cb * NPE + b0];
#pragma unroll
          for (int t = 1; t < N; ++t) s = fma(tab.Phi[q][t], qel[cb * NPE + b0 + t * st], s);
          qq[cb] = s;
        }
        double fv[NC];
        viscous_flux_n<EQ, D, double, double>(uq, qq, nv, pp, fv);
#pragma unroll
        for (int c = 0; c < NC; ++c) f[c] += fv[c];
      }
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int c = 0; c < NC; ++c) r[i][c] = fma(-tab.Kd[i][q], f[c], r[i][c]);
    }
    // end fluxes F^.n^+(u^+(1), u(1)) and F^.n^-(u^-(0), u(0)), lifted by L1 / L0
#pragma unroll 1
    for (int end = 0; end < 2; ++end) {
      const int aend = b0 + end * P * st;
      double nv[D];
#pragma unroll
      for (int a = 0; a < D; ++a) nv[a] = g.nend[(L * 2 + end) * D + a];
      const int32_t nb = g.nbr[L * 2 + end];
      double uin[NC], F[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) uin[c] = uel[c * NPE + aend];
      double qin[VISC ? NC * D : 1];
      if constexpr (VISC) {
#pragma unroll
        for (int cb = 0; cb < NC * D; ++cb) qin[cb] = qel[cb * NPE + aend];
      }
      double nn = nv[0] * nv[0];
#pragma unroll
      for (int a = 1; a < D; ++a) nn += nv[a] * nv[a];
      nn = sqrt(nn);
      if (nb >= 0) {
        const int64_t eo = nb / NPE;
        const int ao = nb % NPE;
        double uout[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) uout[c] = U[eo * tile + c * NPE + ao];
        inviscid_numflux<EQ, D, double, double>(uout, uin, nv, pp, F);
        if constexpr (VISC) {
          double fv[NC];
          if (g.sw[(e * D + d) * 2 + end] == 1) {
            double qout[NC * D];
#pragma unroll
            for (int cb = 0; cb < NC * D; ++cb) qout[cb] = Q[(eo * NC * D + cb) * NPE + ao];
            viscous_flux_n<EQ, D, double, double>(uout, qout, nv, pp, fv);
          } else {
            viscous_flux_n<EQ, D, double, double>(uin, qin, nv, pp, fv);
          }
          const double pen = ph.C11;  // per unit reference length: C11 / h physically
#pragma unroll
          for (int c = 0; c < NC; ++c) F[c] += fv[c] + pen * (uin[c] - uout[c]);
        }
      } else {
        const int kind = ph.bck[-1 - nb];
        bool done = false;
        if (kind == BC_NEUMANN) {  // Eq. 29: F^.n = G.n from the prescribed flux
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            double s = 0.0;
            if (g.gN)
#pragma unroll
              for (int a = 0; a < D; ++a) s = fma(g.gN[((e * NC + c) * D + a) * NPE + aend], nv[a], s);
            F[c] = s;
          }
          done = true;
        }
        if constexpr (NC == D + 2) {
          if (kind == BC_WALL) {
            // no-slip adiabatic wall: pressure flux, viscous flux of the wall
            // state without heat flux, momentum penalty
            double m2 = 0.0;
#pragma unroll
            for (int a = 0; a < D; ++a) m2 += uin[1 + a] * uin[1 + a];
            const double pr = (ph.gamma - 1.0) * (uin[D + 1] - 0.5 * m2 / uin[0]);
            F[0] = 0.0;
#pragma unroll
            for (int a = 0; a < D; ++a) F[1 + a] = pr * nv[a];
            F[D + 1] = 0.0;
            if constexpr (VISC) {
              double ub[NC], fv[NC];
              wall_state<D, double, double>(uin, ub);
              viscous_flux_n<EQ, D, double, double>(ub, qin, nv, pp, fv);
              const double pen = ph.C11b * nn;
#pragma unroll
              for (int a = 0; a < D; ++a) F[1 + a] += fv[1 + a] + pen * (uin[1 + a] - ub[1 + a]);
            }
            done = true;
          }
        }
        if (!done) {
          double gd[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) gd[c] = g.gD ? g.gD[e * tile + c * NPE + aend] : 0.0;
          inviscid_numflux<EQ, D, double, double>(gd, uin, nv, pp, F);
          if constexpr (VISC) {
            double fv[NC];
            viscous_flux_n<EQ, D, double, double>(uin, qin, nv, pp, fv);
            const double pen = ph.C11b * nn;
#pragma unroll
            for (int c = 0; c < NC; ++c) F[c] += fv[c] + pen * (uin[c] - gd[c]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const double li = end ? tab.L1[i] : tab.L0[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) r[i][c] = fma(li, F[c], r[i][c]);
      }
    }
    double* ro = sR + (size_t)(le * D + d) * tile;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < NC; ++c) ro[c * NPE + b0 + i * st] = r[i][c];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ne * tile; k += blockDim.x) {
    const int le2 = k / tile, rem = k % tile, node = rem % NPE;
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) s += sR[(size_t)(le2 * D + d) * tile + rem];
    double v = -s * g.invJ[(e0 + le2) * NPE + node];
    if (g.src) v += g.src[e0 * tile + k];
    R[e0 * tile + k] = v;
  }
}

template <int D, int P, int NC>
cudaError_t run_gradient(const ldg_handle* h, const double* U, const double* Qs, double* Q, cudaStream_t st) {
  using S = Shape<D, P>;
  const size_t smem = (size_t)S::EPB * (NC * S::NPE + D * NC * D * S::NPE) * sizeof(double);
  auto kern = k_gradient<D, P, NC>;
  cudaError_t err = set_smem_once(kern, smem);
  if (err != cudaSuccess) return err;
  const int64_t blocks = (h->E + S::EPB - 1) / S::EPB;
  kern<<<(unsigned)blocks, S::THREADS, smem, st>>>(U, Qs, Q, h->geo(), h->tab, h->phys);
  count_launch();
  return cudaGetLastError();
}

template <int D, int P, int EQ>
cudaError_t run_residual(const ldg_handle* h, const double* U, const double* Q, double* R,
                         cudaStream_t st) {
  using S = Shape<D, P>;
  constexpr int NC = NComp<EQ, D>::value;
  constexpr bool VISC = IsViscous<EQ>::value;
  const size_t smem =
      (size_t)S::EPB * (NC * S::NPE + (VISC ? NC * D * S::NPE : 0) + D * NC * S::NPE) * sizeof(double);
  auto kern = k_residual<D, P, NC, EQ>;
  cudaError_t err = set_smem_once(kern, smem);
  if (err != cudaSuccess) return err;
  const int64_t blocks = (h->E + S::EPB - 1) / S::EPB;
  kern<<<(unsigned)blocks, S::THREADS, smem, st>>>(U, Q, R, h->geo(), h->tab, h->phys);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ldg
