// Split Jacobian-vector product and element-block ILU(0) preconditioner
// (Sec. 4.2, Eq. 41 and the block-Jacobi preconditioner A~).
//
//   g = K21 x                        (k_k21_apply; the discrete gradient of x)
//   y = shift x + scale (K11 x + K12 g)       (k_jacvec)
//   A~_e = shift I + scale mask_e(K11 + K12 K21), block ILU(0)   (k_precond)
//   z = (L U)^-1 r                   (k_precond_apply_lv: FP32, 3-D up to p = 3; else k_precond_apply)
// Matrices are read at their stored precision R, vectors are V (float for
// the mixed path, double for the FP64 path and the FP64 refinement residual),
// sums in V. Every kernel processes whole elements per block so a line's
// D-directional contributions are summed in shared memory before one
// coalesced store.
#pragma once
#include "ldg_jacobian_impl.cuh"

namespace ldg {

template <int D, int P, int NC, typename R, typename V>
__global__ void __launch_bounds__(Shape<D, P>::THREADS)
    k_k21_apply(const R* __restrict__ K21, const R* __restrict__ Kw, const V* __restrict__ x,
                V* __restrict__ gout, Geo g, Tab tab) {
  using S = Shape<D, P>;
  constexpr int N = S::N, NPE = S::NPE;
  constexpr int tile = NC * NPE, gt = NC * D * NPE;
  constexpr int64_t NK = (N * N + N) * D;
  extern __shared__ unsigned char smraw[];
  V* sx = reinterpret_cast<V*>(smraw);
  V* sg = sx + S::EPB * tile;  // [EPB][D dir][NC][D b][NPE]
  const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
  const int ne = (int)min((int64_t)S::EPB, g.E - e0);
  for (int k = threadIdx.x; k < ne * tile; k += blockDim.x) sx[k] = x[e0 * tile + k];
  __syncthreads();
  const int le = threadIdx.x / S::TPE, rr = threadIdx.x % S::TPE;
  if (le < ne) {
    const int d = rr / S::NL, l = rr % S::NL;
    const int64_t e = e0 + le;
    const int64_t L = (e * D + d) * S::NL + l;
    const int st = S::stride(d), b0 = S::base(d, l);
    // the end whose trace u^ comes from outside (interior, S = -1)
    int oend = -1;
    int32_t onb = -1;
#pragma unroll
    for (int end = 0; end < 2; ++end) {
      const int32_t nb = g.nbr[L * 2 + end];
      if (nb >= 0 && g.sw[(e * D + d) * 2 + end] == -1) {
        oend = end;
        onb = nb;
      }
    }
    R kin[N][N][D], kf[N][D];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int b = 0; b < D; ++b) {
#pragma unroll
        for (int j = 0; j < N; ++j) kin[i][j][b] = K21[tile_index(L, NK, (i * N + j) * D + b)];
        kf[i][b] = K21[tile_index(L, NK, N * N * D + i * D + b)];
      }
    V* go = sg + (size_t)(le * D + d) * NC * D * NPE;
#pragma unroll 1
    for (int c = 0; c < NC; ++c) {
      V xl[N];
#pragma unroll
      for (int t = 0; t < N; ++t) xl[t] = sx[le * tile + c * NPE + b0 + t * st];
      V xo = (oend >= 0) ? x[(int64_t)(onb / NPE) * tile + c * NPE + onb % NPE] : V(0);
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int b = 0; b < D; ++b) {
          V s = (V)kf[i][b] * xo;
#pragma unroll
          for (int j = 0; j < N; ++j) s += (V)kin[i][j][b] * xl[j];
          go[(c * D + b) * NPE + b0 + i * st] = s;
        }
    }
    // no-slip wall ends: the trace is the wall state of the end node, whose
    // derivative keeps rho, drops the momentum and maps to the energy row w
    if (Kw) {
#pragma unroll
      for (int end = 0; end < 2; ++end) {
        if (g.nbr[L * 2 + end] >= 0) continue;
        R w[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) w[c] = Kw[tile_index(L, 2 * NC, end * NC + c)];
        if (w[NC - 1] == R(0)) continue;  // a Dirichlet end
        const int aend = b0 + end * P * st;
        V xa[NC], sE = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          xa[c] = sx[le * tile + c * NPE + aend];
          sE += (V)w[c] * xa[c];
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const V li = (V)(g.invJ[e * NPE + b0 + i * st] * (end ? tab.L1[i] : tab.L0[i]));
#pragma unroll
          for (int b = 0; b < D; ++b) {
            const V cf = li * (V)g.nend[(L * 2 + end) * D + b];
            go[(0 * D + b) * NPE + b0 + i * st] += cf * xa[0];
            go[((NC - 1) * D + b) * NPE + b0 + i * st] += cf * sE;
          }
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ne * gt; k += blockDim.x) {
    const int le2 = k / gt, rem = k % gt;
    V s = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) s += sg[(size_t)(le2 * D + d) * gt + rem];
    gout[e0 * gt + k] = s;
  }
}

// One thread per (line, row i): the block's lines are tile aligned and the
// row index is the slowest thread index, so a warp reads one matrix entry of
// 32 consecutive lines (one 128-byte segment in FP32) per load, and the
// (p+1)-fold split gives enough loads in flight to stream K11/K12 from HBM
// even when the mesh has few elements.
template <int D, int P>
struct JvShape {
  static constexpr int THREADS = Shape<D, P>::N * Shape<D, P>::THREADS;
};

template <int D, int P, int NC, int EQ, typename R, typename V>
__global__ void __launch_bounds__(JvShape<D, P>::THREADS)
    k_jacvec(const R* __restrict__ K11, const R* __restrict__ K12, const V* __restrict__ x,
             const V* __restrict__ gx, V* __restrict__ y, double shift, double scale, Geo g) {
  using S = Shape<D, P>;
  constexpr int N = S::N, NPE = S::NPE, NCD = NC * D, NLB = S::THREADS;
  constexpr bool VISC = IsViscous<EQ>::value;
  constexpr int tile = NC * NPE, gt = VISC ? NCD * NPE : 0;
  constexpr int64_t NK11 = (N * N + 2 * N) * NC * NC;
  constexpr int64_t NK12 = VISC ? (N * N + N) * NC * NCD : 1;
  constexpr int OFF11 = N * N * NC * NC, OFF12 = N * N * NC * NCD;
  extern __shared__ unsigned char smraw[];
  V* sx = reinterpret_cast<V*>(smraw);
  V* sgx = sx + S::EPB * tile;
  V* sy = sgx + S::EPB * gt;  // [EPB][D][NC][NPE]
  const int64_t e0 = (int64_t)blockIdx.x * S::EPB;
  const int ne = (int)min((int64_t)S::EPB, g.E - e0);
  for (int k = threadIdx.x; k < ne * tile; k += blockDim.x) sx[k] = x[e0 * tile + k];
  if constexpr (VISC)
    for (int k = threadIdx.x; k < ne * gt; k += blockDim.x) sgx[k] = gx[e0 * gt + k];
  __syncthreads();
  const int i = threadIdx.x / NLB, lloc = threadIdx.x % NLB;
  const int le = lloc / S::TPE, rr = lloc % S::TPE;
  if (le < ne) {
    const int d = rr / S::NL, l = rr % S::NL;
    const int64_t e = e0 + le;
    const int64_t L = (e * D + d) * S::NL + l;
    const int st = S::stride(d), b0 = S::base(d, l);
    V acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = V(0);
    // K11 in-line block, row i
#pragma unroll
    for (int j = 0; j < N; ++j) {
      V xj[NC];
#pragma unroll
      for (int cp = 0; cp < NC; ++cp) xj[cp] = sx[le * tile + cp * NPE + b0 + j * st];
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int cp = 0; cp < NC; ++cp)
          acc[c] += (V)K11[tile_index(L, NK11, ((i * N + j) * NC + c) * NC + cp)] * xj[cp];
    }
    // K11 face blocks: outside traces of both ends
#pragma unroll
    for (int end = 0; end < 2; ++end) {
      const int32_t nb = g.nbr[L * 2 + end];
      if (nb < 0) continue;
      V xo[NC];
#pragma unroll
      for (int cp = 0; cp < NC; ++cp) xo[cp] = x[(int64_t)(nb / NPE) * tile + cp * NPE + nb % NPE];
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int cp = 0; cp < NC; ++cp)
          acc[c] += (V)K11[tile_index(L, NK11, OFF11 + ((end * N + i) * NC + c) * NC + cp)] * xo[cp];
    }
    if constexpr (VISC) {
#pragma unroll 1
      for (int j = 0; j < N; ++j) {
#pragma unroll
        for (int cb = 0; cb < NCD; ++cb) {
          const V gj = sgx[le * gt + cb * NPE + b0 + j * st];
#pragma unroll
          for (int c = 0; c < NC; ++c)
            acc[c] += (V)K12[tile_index(L, NK12, ((i * N + j) * NC + c) * NCD + cb)] * gj;
        }
      }
#pragma unroll
      for (int end = 0; end < 2; ++end) {
        const int32_t nb = g.nbr[L * 2 + end];
        if (g.sw[(e * D + d) * 2 + end] != 1 || nb < 0) continue;
#pragma unroll
        for (int cb = 0; cb < NCD; ++cb) {
          const V go = gx[((int64_t)(nb / NPE) * NCD + cb) * NPE + nb % NPE];
#pragma unroll
          for (int c = 0; c < NC; ++c)
            acc[c] += (V)K12[tile_index(L, NK12, OFF12 + (i * NC + c) * NCD + cb)] * go;
        }
      }
    }
    V* yo = sy + (size_t)(le * D + d) * tile;
#pragma unroll
    for (int c = 0; c < NC; ++c) yo[c * NPE + b0 + i * st] = acc[c];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ne * tile; k += blockDim.x) {
    const int le2 = k / tile, rem = k % tile;
    V s = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) s += sy[(size_t)(le2 * D + d) * tile + rem];
    y[e0 * tile + k] = (V)shift * sx[k] + (V)scale * s;
  }
}

// ---------------------------------------------------------------------------
// Preconditioner: one block per element, A~_e and its ILU(0) in shared memory
// ---------------------------------------------------------------------------
template <typename R, int NC>
__device__ void invert_block(const R* a, R* inv) {
  // Gauss-Jordan with partial pivoting on an NC x NC block (one thread)
  R m[NC][2 * NC];
  for (int r = 0; r < NC; ++r)
    for (int c = 0; c < NC; ++c) {
      m[r][c] = a[r * NC + c];
      m[r][NC + c] = (r == c) ? R(1) : R(0);
    }
  for (int c = 0; c < NC; ++c) {
    int piv = c;
    for (int r = c + 1; r < NC; ++r)
      if (fabs((double)m[r][c]) > fabs((double)m[piv][c])) piv = r;
    if (piv != c)
      for (int k = 0; k < 2 * NC; ++k) {
        R t = m[c][k];
        m[c][k] = m[piv][k];
        m[piv][k] = t;
      }
    const R ip = R(1) / m[c][c];
    for (int k = 0; k < 2 * NC; ++k) m[c][k] *= ip;
    for (int r = 0; r < NC; ++r)
      if (r != c) {
        const R f = m[r][c];
        for (int k = 0; k < 2 * NC; ++k) m[r][k] -= f * m[c][k];
      }
  }
  for (int r = 0; r < NC; ++r)
    for (int c = 0; c < NC; ++c) inv[r * NC + c] = m[r][NC + c];
}

// Gauss-Jordan with partial pivoting on an NC x NC block by one warp: lane
// t < 2 NC holds column t of the augmented matrix [a | I]; pivot columns
// are broadcast by shuffles. Same operations per entry as invert_block.
template <typename R, int NC>
__device__ void invert_block_warp(const R* a, R* inv, int lane) {
  R col[NC];
#pragma unroll
  for (int r = 0; r < NC; ++r)
    col[r] = lane < NC ? a[r * NC + lane] : (lane < 2 * NC ? (r == lane - NC ? R(1) : R(0)) : R(0));
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    R pc[NC];  // column c, broadcast
#pragma unroll
    for (int r = 0; r < NC; ++r) pc[r] = __shfl_sync(0xffffffffu, col[r], c);
    int piv = c;
#pragma unroll
    for (int r = c + 1; r < NC; ++r)
      if (fabs((double)pc[r]) > fabs((double)pc[piv])) piv = r;
    // swap rows c and piv (in this lane's column and in the broadcast copy)
#pragma unroll
    for (int r = c + 1; r < NC; ++r)
      if (r == piv) {
        R t = col[r];
        col[r] = col[c];
        col[c] = t;
        t = pc[r];
        pc[r] = pc[c];
        pc[c] = t;
      }
    const R ip = R(1) / pc[c];
    col[c] *= ip;
#pragma unroll
    for (int r = 0; r < NC; ++r)
      if (r != c) col[r] -= pc[r] * col[c];
  }
  if (lane >= NC && lane < 2 * NC)
#pragma unroll
    for (int r = 0; r < NC; ++r) inv[r * NC + lane - NC] = col[r];
}

struct PcTables {
  const int16_t* pat;   // [NPE][W]
  const int8_t* slot;   // [NPE][NPE]
  const int8_t* nbf;    // [E][2D]
  const int16_t* lvl;   // [NPE]
  const int32_t* lptr;  // [levels + 1]
};

// INPLACE: the element block is assembled and factored directly in its
// slice of F / Ud in global memory (L2-resident while the block works on
// it) when it does not fit in shared memory (FP64 at 3-D, p = 4).
template <int D, int P, int NC, bool VISC, typename R, bool INPLACE>
__global__ void __launch_bounds__(256)
    k_precond(const R* __restrict__ K11, const R* __restrict__ K12, const R* __restrict__ K21,
              const R* __restrict__ Kw, R* F, R* Ud, Geo g, Tab tab, PcTables pt, double shift,
              double scale) {
  using S = Shape<D, P>;
  constexpr int N = S::N, NPE = S::NPE, NL = S::NL, W = D * P + 1, NCD = NC * D, BB = NC * NC;
  constexpr int64_t NK11 = (N * N + 2 * N) * NC * NC;
  constexpr int64_t NK12 = VISC ? (N * N + N) * NC * NCD : 1;
  constexpr int64_t NK21 = (N * N + N) * D;
  constexpr int OFF12 = N * N * NC * NCD;
  extern __shared__ unsigned char smraw[];
  R* const sm = reinterpret_cast<R*>(smraw);
  R* A = INPLACE ? F + (int64_t)blockIdx.x * NPE * W * BB : sm + NPE * W * D;  // [NPE][W][NC][NC]
  R* Di = INPLACE ? Ud + (int64_t)blockIdx.x * NPE * BB : A + NPE * W * BB;   // [NPE][NC][NC] inverses
  R* K21e = sm;                                    // [NPE][W][D] element part of K21
  __shared__ int16_t pat_s[NPE * W];
  __shared__ int8_t slot_s[NPE * NPE];
  __shared__ int16_t lvl_s[NPE];
  __shared__ int32_t lptr_s[D * P + 2];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const R sc = (R)scale;
  for (int k = tid; k < NPE * W; k += nt) pat_s[k] = pt.pat[k];
  for (int k = tid; k < NPE * NPE; k += nt) slot_s[k] = pt.slot[k];
  for (int k = tid; k < NPE; k += nt) lvl_s[k] = pt.lvl[k];
  for (int k = tid; k < D * P + 2; k += nt) lptr_s[k] = pt.lptr[k];
  for (int k = tid; k < NPE * W * BB; k += nt) {
    const int i = k / (W * BB), s = (k / BB) % W, cc = k % BB;
    A[k] = (pt.pat[i * W + s] == i && cc / NC == cc % NC) ? (R)shift : R(0);
  }
  if constexpr (VISC)
    for (int k = tid; k < NPE * W * D; k += nt) K21e[k] = R(0);
  __syncthreads();
  // K11 (and the element part of K21) line by line; directions in turn so
  // that the diagonal block, shared by the D lines of a node, has one writer
#pragma unroll 1
  for (int d = 0; d < D; ++d) {
    const int st = S::stride(d);
    for (int k = tid; k < NL * N * N * BB; k += nt) {
      const int l = k / (N * N * BB), i = (k / (N * BB)) % N, j = (k / BB) % N, cc = k % BB;
      const int b0 = S::base(d, l);
      const int ni = b0 + i * st, nj = b0 + j * st;
      const int64_t L = (e * D + d) * NL + l;
      const int s = slot_s[ni * NPE + nj];
      A[(ni * W + s) * BB + cc] += sc * K11[tile_index(L, NK11, ((i * N + j) * NC + cc / NC) * NC + cc % NC)];
    }
    if constexpr (VISC)
      for (int k = tid; k < NL * N * N * D; k += nt) {
        const int l = k / (N * N * D), i = (k / (N * D)) % N, j = (k / D) % N, b = k % D;
        const int b0 = S::base(d, l);
        const int ni = b0 + i * st, nj = b0 + j * st;
        const int64_t L = (e * D + d) * NL + l;
        K21e[(ni * W + slot_s[ni * NPE + nj]) * D + b] += K21[tile_index(L, NK21, (i * N + j) * D + b)];
      }
    __syncthreads();
  }
  // K12 K21 restricted to the pattern: one thread per (row, c, c')
  if constexpr (VISC) {
    for (int k = tid; k < NPE * BB; k += nt) {
      const int ni = k / BB, c = (k / NC) % NC, cp = k % NC;
      int idx[3] = {ni % N, (ni / N) % N, ni / (N * N)};
      R accs[W];
#pragma unroll
      for (int s = 0; s < W; ++s) accs[s] = R(0);
#pragma unroll 1
      for (int d = 0; d < D; ++d) {
        const int st = S::stride(d);
        const int i = idx[d];
        const int b0 = ni - i * st;
        const int l = (b0 % st) + (b0 / (st * N)) * st;
        const int64_t L = (e * D + d) * NL + l;
        // in-element paths: row i of line L to node g = b0 + t st, then K21 row g
#pragma unroll 1
        for (int t = 0; t < N; ++t) {
          const int ng = b0 + t * st;
          R kb[D];
#pragma unroll
          for (int b = 0; b < D; ++b) kb[b] = K12[tile_index(L, NK12, ((i * N + t) * NC + c) * NCD + cp * D + b)];
          for (int s2 = 0; s2 < W; ++s2) {
            const int nj = pat_s[ng * W + s2];
            const int s = slot_s[ni * NPE + nj];
            if (s < 0) continue;
            R v = 0;
#pragma unroll
            for (int b = 0; b < D; ++b) v += kb[b] * K21e[(ng * W + s2) * D + b];
            accs[s] += v;
          }
        }
        // cross-face path: the S = +1 end's outside gradient depends, through
        // the neighbour's K21 face entry, on this element's end node
#pragma unroll 1
        for (int end = 0; end < 2; ++end) {
          const int32_t nb = g.nbr[L * 2 + end];
          if (nb < 0 || g.sw[(e * D + d) * 2 + end] != 1) continue;
          const int64_t eo = nb / NPE;
          const int ao = nb % NPE;
          const int fn = pt.nbf[e * 2 * D + 2 * d + end];
          const int dn = fn / 2, endn = fn % 2;
          const int sto = S::stride(dn);
          const int bo = ao - (endn * P) * sto;
          const int lo = (bo % sto) + (bo / (sto * N)) * sto;
          const int64_t Lo = (eo * D + dn) * NL + lo;
          const int tpos = endn * P;
          R v = 0;
#pragma unroll
          for (int b = 0; b < D; ++b)
            v += K12[tile_index(L, NK12, OFF12 + (i * NC + c) * NCD + cp * D + b)] *
                 K21[tile_index(Lo, NK21, N * N * D + tpos * D + b)];
          const int nk = b0 + end * P * st;
          accs[slot_s[ni * NPE + nk]] += v;
        }
      }
      // paths through a no-slip wall end: row i -> q at node t of one of its
      // lines (K12) -> the wall trace of the end node aw of t's line in a
      // direction with a wall end (rho kept, energy row w of the wall state)
      if (Kw) {
#pragma unroll 1
        for (int d = 0; d < D; ++d) {
          const int st = S::stride(d);
          const int i = idx[d];
          const int b0 = ni - i * st;
          const int l = (b0 % st) + (b0 / (st * N)) * st;
          const int64_t L = (e * D + d) * NL + l;
#pragma unroll 1
          for (int t = 0; t < N; ++t) {
            const int ng = b0 + t * st;
            R kr[D], ke[D];
#pragma unroll
            for (int b = 0; b < D; ++b) {
              kr[b] = K12[tile_index(L, NK12, ((i * N + t) * NC + c) * NCD + 0 * D + b)];
              ke[b] = K12[tile_index(L, NK12, ((i * N + t) * NC + c) * NCD + (NC - 1) * D + b)];
            }
            const int gi[3] = {ng % N, (ng / N) % N, ng / (N * N)};
#pragma unroll 1
            for (int dw = 0; dw < D; ++dw) {
              const int stw = S::stride(dw), pw = gi[dw];
              const int b0w = ng - pw * stw;
              const int lw = (b0w % stw) + (b0w / (stw * N)) * stw;
              const int64_t Lw = (e * D + dw) * NL + lw;
#pragma unroll 1
              for (int endw = 0; endw < 2; ++endw) {
                if (g.nbr[Lw * 2 + endw] >= 0) continue;
                if (Kw[tile_index(Lw, 2 * NC, endw * NC + NC - 1)] == R(0)) continue;  // Dirichlet end
                const int aw = b0w + endw * P * stw;
                const int s = slot_s[ni * NPE + aw];
                if (s < 0) continue;
                const R wc = Kw[tile_index(Lw, 2 * NC, endw * NC + cp)];
                const R li = (R)(g.invJ[e * NPE + ng] * (endw ? tab.L1[pw] : tab.L0[pw]));
                R v = 0;
#pragma unroll
                for (int b = 0; b < D; ++b) {
                  const R cf = li * (R)g.nend[(Lw * 2 + endw) * D + b];
                  v += ((cp == 0 ? kr[b] : R(0)) + ke[b] * wc) * cf;
                }
                accs[s] += v;
              }
            }
          }
        }
      }
#pragma unroll
      for (int s = 0; s < W; ++s) A[(ni * W + s) * BB + c * NC + cp] += sc * accs[s];
    }
    __syncthreads();
  }
  // block ILU(0), IKJ order inside each row, in the pattern. Rows of one
  // wavefront level (ix + iy + iz) never appear in each other's pattern, so
  // they are factored concurrently, one warp per row; the row's updates use
  // only rows of earlier levels.
  {
    const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
#pragma unroll 1
    for (int lv = 0; lv < D * P + 1; ++lv) {
#pragma unroll 1
      for (int rr = lptr_s[lv] + warp; rr < lptr_s[lv + 1]; rr += nwarps) {
        const int i = lvl_s[rr];
#pragma unroll 1
        for (int s = 0; s < W; ++s) {
          const int k = pat_s[i * W + s];
          if (k >= i) break;
          // A_ik <- A_ik Dinv_k
          R tmp = 0;
          if (lane < BB) {
            const int c = lane / NC, cp = lane % NC;
#pragma unroll
            for (int m = 0; m < NC; ++m) tmp += A[(i * W + s) * BB + c * NC + m] * Di[k * BB + m * NC + cp];
          }
          __syncwarp();
          if (lane < BB) A[(i * W + s) * BB + lane] = tmp;
          __syncwarp();
          // A_ij -= A_ik A_kj for j > k in both patterns
          for (int q = lane; q < W * BB; q += 32) {
            const int s2 = q / BB, c = (q / NC) % NC, cp = q % NC;
            const int j = pat_s[i * W + s2];
            if (j <= k) continue;
            const int sk = slot_s[k * NPE + j];
            if (sk < 0) continue;
            R v = 0;
#pragma unroll
            for (int m = 0; m < NC; ++m) v += A[(i * W + s) * BB + c * NC + m] * A[(k * W + sk) * BB + m * NC + cp];
            A[(i * W + s2) * BB + c * NC + cp] -= v;
          }
          __syncwarp();
        }
        invert_block_warp<R, NC>(A + (i * W + slot_s[i * NPE + i]) * BB, Di + i * BB, lane);
        __syncwarp();
      }
      __syncthreads();
    }
  }
  // stored for the apply: each row's diagonal slot holds D_i^-1 (the only
  // diagonal quantity the triangular solves use), so a row's factors are one
  // contiguous run with no unread block between them; U_ii goes to Ud (read
  // only by the export)
  if constexpr (!INPLACE) {
    for (int k = tid; k < NPE * W * BB; k += nt) {
      const int i = k / (W * BB), sl = (k / BB) % W;
      F[e * NPE * W * BB + k] = (pat_s[i * W + sl] == i) ? Di[i * BB + k % BB] : A[k];
    }
    for (int k = tid; k < NPE * BB; k += nt) {
      const int i = k / BB;
      Ud[e * NPE * BB + k] = A[(i * W + slot_s[i * NPE + i]) * BB + k % BB];
    }
  } else {
    for (int k = tid; k < NPE * BB; k += nt) {
      const int i = k / BB;
      R* a = A + (i * W + slot_s[i * NPE + i]) * BB + k % BB;
      const R u = *a;
      *a = Di[k];
      Di[k] = u;
    }
  }
}

// ---------------------------------------------------------------------------
// ILU(0) apply z = (L U)^-1 r. A warp holds 32 / (n_c G) elements; lane
// (c, g) of an element owns component c of every row and the n_c / G block
// columns m in [g n_c / G, (g + 1) n_c / G). Rows are processed in order
// (forward 1 .. npe-1, then backward npe-1 .. 0): lane (c, g) accumulates
// F[i][s][c][m] y[col(s)][m] over the row's pattern slots and its m range,
// the G lanes of component c sum their parts, and lane (c, 0) stores the
// result in the warp's y slice (shared memory). This row-chain form serves
// the FP64 apply, bound by the FP64 pipe (G = 1 leaves no reduction at all;
// G = 2 doubles the warps of a small mesh), the FP32 apply of 2-D elements
// with G = n_c (the most lanes per element) and of 3-D p = 4 elements with
// G = 1; 3-D FP32 elements up to p = 3 run by wavefronts
// (k_precond_apply_lv below).
//
// Row i = ix + N iy + N^2 iz couples to the nodes of its D lines; its
// pattern slots in ascending column order are: lower z, lower y, lower x,
// the diagonal (slot ix + iy + iz), upper x, upper y, upper z. The loops
// are unrolled at compile time, so slot counts and columns are constants,
// and the factors of the row PD steps ahead are loaded into registers while
// the current row is reduced: the serial row chain never waits on memory.
// (Element shapes too large to unroll run the same loop rolled, loading
// each row's factors when it is processed.)
template <int D, int P, int NC, int G, typename R, typename V>
struct ApplyLanes {
  static constexpr int N = P + 1, NPE = D == 2 ? N * N : N * N * N, W = D * P + 1, BB = NC * NC;
  static constexpr int MPL = NC / G;            // block columns per lane
  static constexpr int LPE = NC * G;            // lanes per element
  static constexpr int EPW = 32 / LPE;          // elements per warp
  static constexpr int MAXS = D * (N - 1);      // slots of one triangle in a row
  static constexpr int TASKS = 2 * NPE - 1;     // forward rows 1.., backward rows ..0
  static constexpr size_t YB = (size_t)EPW * NC * NPE * sizeof(V);
  // small blocks spread a small mesh evenly over the SMs: one warp per block
  // when a warp holds several elements, else two
  static constexpr int WPB = EPW >= 4 ? 1 : (YB * 2 <= 40960 ? 2 : 1);
  static constexpr int THREADS = 32 * WPB;
  static constexpr int REGS_PER_ROW = MAXS * MPL * (int)(sizeof(R) / 4);
  // the task loop is unrolled (and prefetched PD rows ahead) only while the
  // unrolled body stays small enough for the compiler to keep fb in registers
  static constexpr bool UNROLL = TASKS * MAXS * MPL <= 2000;
  static constexpr int UNROLL_N = UNROLL ? TASKS : 1;
  static constexpr int PD = !UNROLL ? 0 : (REGS_PER_ROW * 8 <= 72 ? 8 : (REGS_PER_ROW * 4 <= 72 ? 4 : 2));
  static_assert(NC % G == 0, "G must divide n_c");
};

// sum of v over the G lanes of one component group (G consecutive lanes)
template <int G, typename V>
__device__ __forceinline__ V group_sum(V v, V* scratch, int lane) {
  if constexpr (G == 1) {
    return v;
  } else if constexpr ((G & (G - 1)) == 0) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  } else {
    // gather the G values of the group by shuffles (idle lanes past the last
    // full group read wrapped lanes; their result is not used)
    (void)scratch;
    const int g0 = lane - lane % G;
    V s = 0;
#pragma unroll
    for (int k = 0; k < G; ++k) s += __shfl_sync(0xffffffffu, v, (g0 + k) & 31);
    return s;
  }
}

// MPL consecutive factor values (vector loads where the block layout keeps
// them aligned: the offsets are multiples of MPL elements inside 16-byte
// aligned n_c x n_c blocks)
template <int MPL, typename R>
__device__ __forceinline__ void load_run(const R* p, R (&out)[MPL]) {
  if constexpr (sizeof(R) == 8 && MPL % 2 == 0 && (MPL * 8) % 16 == 0) {
#pragma unroll
    for (int k = 0; k < MPL; k += 2) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(p + k));
      out[k] = v.x;
      out[k + 1] = v.y;
    }
  } else if constexpr (sizeof(R) == 4 && MPL % 4 == 0) {
#pragma unroll
    for (int k = 0; k < MPL; k += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p + k));
      out[k] = v.x;
      out[k + 1] = v.y;
      out[k + 2] = v.z;
      out[k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < MPL; ++k) out[k] = __ldg(p + k);
  }
}

template <int D, int N>
struct RowPos {
  int i, ix, iy, iz, dg;
  __device__ __forceinline__ constexpr RowPos(int r)
      : i(r), ix(r % N), iy((r / N) % N), iz(D == 3 ? r / (N * N) : 0), dg(r % N + (r / N) % N + (D == 3 ? r / (N * N) : 0)) {}
  // column of lower slot k (0 <= k < dg) and upper slot k (slot dg + 1 + k)
  __device__ __forceinline__ constexpr int lower_col(int k) const {
    return k < iz ? i - (iz - k) * N * N : (k < iz + iy ? i - (iy - (k - iz)) * N : i - (ix - (k - iz - iy)));
  }
  __device__ __forceinline__ constexpr int upper_col(int k) const {
    return k < N - 1 - ix ? i + (k + 1)
                          : (k < 2 * N - 2 - ix - iy ? i + (k - (N - 1 - ix) + 1) * N
                                                     : i + (k - (2 * N - 2 - ix - iy) + 1) * N * N);
  }
};

template <int D, int P, int NC, int G, typename R, typename V>
__global__ void __launch_bounds__(ApplyLanes<D, P, NC, G, R, V>::THREADS)
    k_precond_apply(const R* __restrict__ F, const V* __restrict__ r,
                    V* __restrict__ z, int64_t E) {
  using A = ApplyLanes<D, P, NC, G, R, V>;
  constexpr int N = A::N, NPE = A::NPE, W = A::W, BB = A::BB, EPW = A::EPW, MPL = A::MPL;
  constexpr int MAXS = A::MAXS, TASKS = A::TASKS, PD = A::PD, UN = A::UNROLL_N, tile = NC * NPE;
  using Pos = RowPos<D, N>;
  __shared__ V ys[A::WPB][EPW][tile];
  __shared__ V tb[A::WPB][EPW][NC];
  __shared__ V scr[A::WPB][32 + G];  // padded: idle lanes of a partial group read past lane 31
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int el = lane / A::LPE, q = lane % A::LPE, c = q / G, g = q % G, m0 = g * MPL;
  const int64_t e = ((int64_t)blockIdx.x * A::WPB + warp) * EPW + el;
  const bool act = el < EPW && e < E;
  V* y = ys[warp][act ? el : 0];
  V* tbuf = tb[warp][act ? el : 0];
  V* sc = scr[warp];
  if (act)
    for (int k = q; k < tile; k += A::LPE) y[k] = r[e * tile + k];
  const R* Fe = F + (act ? e : 0) * (int64_t)NPE * W * BB + c * NC + m0;

  R fb[PD + 1][MAXS][MPL];
  R db[PD + 1][MPL];
  // factors of task t: forward row t + 1 (lower slots) or backward row
  // 2 npe - 2 - t (upper slots and the inverted diagonal block)
  auto fetch = [&](int t) {
    const bool fwd = t < NPE - 1;
    const Pos ps(fwd ? t + 1 : 2 * NPE - 2 - t);
    const int ns = fwd ? ps.dg : MAXS - ps.dg, s0 = fwd ? 0 : ps.dg + 1, b = t % (PD + 1);
    if (act) {
#pragma unroll
      for (int k = 0; k < MAXS; ++k)
        if (k < ns) load_run<MPL>(Fe + (ps.i * W + s0 + k) * BB, fb[b][k]);
      if (!fwd) load_run<MPL>(Fe + (ps.i * W + ps.dg) * BB, db[b]);  // D_i^-1 in the diagonal slot
    }
  };
#pragma unroll
  for (int t = 0; t < PD && t < TASKS; ++t) fetch(t);
  __syncwarp();
#pragma unroll UN
  for (int t = 0; t < TASKS; ++t) {
    if (t + PD < TASKS) fetch(t + PD);
    const bool fwd = t < NPE - 1;
    const Pos ps(fwd ? t + 1 : 2 * NPE - 2 - t);
    const int b = t % (PD + 1);
    V acc[MPL];
#pragma unroll
    for (int mm = 0; mm < MPL; ++mm) acc[mm] = V(0);
    if (act) {
      if (fwd) {
#pragma unroll
        for (int k = 0; k < MAXS; ++k)
          if (k < ps.dg) {
            const int col = ps.lower_col(k);
#pragma unroll
            for (int mm = 0; mm < MPL; ++mm) acc[mm] += (V)fb[b][k][mm] * y[(m0 + mm) * NPE + col];
          }
      } else {
#pragma unroll
        for (int k = 0; k < MAXS; ++k)
          if (k < MAXS - ps.dg) {
            const int col = ps.upper_col(k);
#pragma unroll
            for (int mm = 0; mm < MPL; ++mm) acc[mm] += (V)fb[b][k][mm] * y[(m0 + mm) * NPE + col];
          }
      }
    }
    V pv = 0;
#pragma unroll
    for (int mm = 0; mm < MPL; ++mm) pv += acc[mm];
    const V s = group_sum<G>(pv, sc, lane);
    if (fwd) {
      if (act && g == 0) y[c * NPE + ps.i] -= s;
      __syncwarp();
    } else {
      if (act && g == 0) tbuf[c] = y[c * NPE + ps.i] - s;
      __syncwarp();
      V d = 0;
      if (act) {
#pragma unroll
        for (int mm = 0; mm < MPL; ++mm) d += (V)db[b][mm] * tbuf[m0 + mm];
      }
      const V zi = group_sum<G>(d, sc, lane);
      if (act && g == 0) y[c * NPE + ps.i] = zi;
      __syncwarp();
    }
  }
  if (act)
    for (int k = q; k < tile; k += A::LPE) z[e * tile + k] = y[k];
}

// ILU(0) apply by wavefronts (FP32): the rows of an element's pattern that
// share the level ix + iy + iz are independent in both triangular solves (a
// row's lower neighbours all lie on lower levels, its upper ones on higher
// levels), so one warp per element takes a whole level at once, one lane
// per (row, component): D p + 1 dependent steps per sweep instead of one per
// row, and every lane's factor loads of a step (its row's lower or upper
// slots, n_c values each) issued together. The backward step finishes with
// the n_c x n_c inverse of the diagonal block, which needs the whole
// component vector of the row: a second pass after the warp's exchange.
template <int D, int P>
constexpr int level_rows_max() {
  constexpr int N = P + 1;
  int best = 0;
  for (int l = 0; l <= D * P; ++l) {
    int cnt = 0;
    for (int i = 0; i < (D == 2 ? N * N : N * N * N); ++i)
      if (i % N + (i / N) % N + (D == 3 ? i / (N * N) : 0) == l) ++cnt;
    best = cnt > best ? cnt : best;
  }
  return best;
}

template <int D, int P, int NC>
struct ApplyLevels {
  static constexpr int N = P + 1, NPE = D == 2 ? N * N : N * N * N, W = D * P + 1, BB = NC * NC;
  static constexpr int LV = D * P + 1;                  // levels 0 .. D p
  static constexpr int MAXS = D * (N - 1);              // slots of one triangle in a row
  static constexpr int MAXR = level_rows_max<D, P>();   // rows of the widest level
  static constexpr int WPB = 4, THREADS = 32 * WPB;     // one element per warp
};

template <int D, int P, int NC, typename R, typename V>
__global__ void __launch_bounds__(ApplyLevels<D, P, NC>::THREADS)
    k_precond_apply_lv(const R* __restrict__ F, const V* __restrict__ r, V* __restrict__ z,
                       const int16_t* __restrict__ lvl, const int32_t* __restrict__ lptr, int64_t E) {
  using A = ApplyLevels<D, P, NC>;
  constexpr int N = A::N, NPE = A::NPE, W = A::W, BB = A::BB, LV = A::LV, MAXS = A::MAXS, tile = NC * NPE;
  using Pos = RowPos<D, N>;
  __shared__ int16_t lvl_s[NPE];
  __shared__ int32_t lptr_s[LV + 1];
  __shared__ V ys[A::WPB][tile];
  __shared__ V tb[A::WPB][A::MAXR * NC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < NPE; k += A::THREADS) lvl_s[k] = lvl[k];
  for (int k = threadIdx.x; k <= LV; k += A::THREADS) lptr_s[k] = lptr[k];
  const int64_t e = (int64_t)blockIdx.x * A::WPB + warp;
  V* y = ys[warp];
  V* t = tb[warp];
  if (e < E)
    for (int k = lane; k < tile; k += 32) y[k] = r[e * tile + k];
  __syncthreads();
  if (e >= E) return;  // no block-wide barrier below
  const R* Fe = F + e * (int64_t)NPE * W * BB;
  // forward: y_i -= sum over lower slots L_is y_col (unit diagonal)
#pragma unroll 1
  for (int l = 1; l < LV; ++l) {
    const int r0 = lptr_s[l], nit = (lptr_s[l + 1] - r0) * NC;
    for (int it = lane; it < nit; it += 32) {
      const int k = it / NC, c = it - k * NC;
      const Pos ps(lvl_s[r0 + k]);
      const R* Fr = Fe + (int64_t)ps.i * W * BB + c * NC;
      V acc = V(0);
#pragma unroll
      for (int s = 0; s < MAXS; ++s)
        if (s < l) {
          const int col = ps.lower_col(s);
#pragma unroll
          for (int m = 0; m < NC; ++m) acc += (V)__ldg(Fr + s * BB + m) * y[m * NPE + col];
        }
      y[c * NPE + ps.i] -= acc;
    }
    __syncwarp();
  }
  // backward: t_i = y_i - sum over upper slots U_is z_col, z_i = D_i^-1 t_i
#pragma unroll 1
  for (int l = LV - 1; l >= 0; --l) {
    const int r0 = lptr_s[l], nit = (lptr_s[l + 1] - r0) * NC, nu = MAXS - l;
    for (int it = lane; it < nit; it += 32) {
      const int k = it / NC, c = it - k * NC;
      const Pos ps(lvl_s[r0 + k]);
      const R* Fr = Fe + ((int64_t)ps.i * W + l + 1) * BB + c * NC;
      V acc = V(0);
#pragma unroll
      for (int s = 0; s < MAXS; ++s)
        if (s < nu) {
          const int col = ps.upper_col(s);
#pragma unroll
          for (int m = 0; m < NC; ++m) acc += (V)__ldg(Fr + s * BB + m) * y[m * NPE + col];
        }
      t[k * NC + c] = y[c * NPE + ps.i] - acc;
    }
    __syncwarp();
    for (int it = lane; it < nit; it += 32) {
      const int k = it / NC, c = it - k * NC;
      const int i = lvl_s[r0 + k];
      const R* Dr = Fe + ((int64_t)i * W + l) * BB + c * NC;  // D_i^-1 in the diagonal slot
      V zc = V(0);
#pragma unroll
      for (int m = 0; m < NC; ++m) zc += (V)__ldg(Dr + m) * t[k * NC + m];
      y[c * NPE + i] = zc;
    }
    __syncwarp();
  }
  for (int k = lane; k < tile; k += 32) z[e * tile + k] = y[k];
}

// The split product y = shift x + scale (K11 x + K12 (K21 x)) as its two
// launches: part 0 both (K21 x into gbuf), part 1 only g = K21 x into gbuf,
// part 2 only y from x and a given g in gbuf (a partitioned part exchanges
// the face traces of g between the two).
template <int D, int P, int EQ, typename R, typename V>
cudaError_t run_jacvec(const ldg_handle* h, const R* K11, const R* K12, const R* K21, const R* Kw, V* gbuf,
                       double shift, double scale, const V* x, V* y, cudaStream_t st, int part = 0) {
  using S = Shape<D, P>;
  constexpr int NC = NComp<EQ, D>::value;
  constexpr bool VISC = IsViscous<EQ>::value;
  const int64_t blocks = (h->E + S::EPB - 1) / S::EPB;
  cudaError_t err;
  if constexpr (VISC) {
    if (part != 2) {
      const size_t sm1 = (size_t)S::EPB * (NC * S::NPE + D * NC * D * S::NPE) * sizeof(V);
      auto k1 = k_k21_apply<D, P, NC, R, V>;
      err = set_smem_once(k1, sm1);
      if (err != cudaSuccess) return err;
      k1<<<(unsigned)blocks, S::THREADS, sm1, st>>>(K21, Kw, x, gbuf, h->geo(), h->tab);
      count_launch();
    }
  }
  if (part == 1) return cudaGetLastError();
  const size_t sm2 = (size_t)S::EPB * (NC * S::NPE + (VISC ? NC * D * S::NPE : 0) + D * NC * S::NPE) * sizeof(V);
  auto k2 = k_jacvec<D, P, NC, EQ, R, V>;
  err = set_smem_once(k2, sm2);
  if (err != cudaSuccess) return err;
  k2<<<(unsigned)blocks, JvShape<D, P>::THREADS, sm2, st>>>(K11, K12, x, gbuf, y, shift, scale, h->geo());
  count_launch();
  return cudaGetLastError();
}

inline PcTables pc_tables(const ldg_handle* h) {
  PcTables t;
  t.pat = h->pat;
  t.slot = h->slot;
  t.nbf = h->nbf;
  t.lvl = h->lvl;
  t.lptr = h->lvl_ptr;
  return t;
}

// dynamic shared memory of the preconditioner build with the element block
// staged on chip, and the static tables it adds
template <int D, int P, int EQ, typename R>
size_t precond_smem() {
  constexpr int NC = NComp<EQ, D>::value;
  using S = Shape<D, P>;
  constexpr int W = D * P + 1;
  return (size_t)(S::NPE * W * NC * NC + S::NPE * NC * NC + S::NPE * W * D) * sizeof(R);
}
template <int D, int P>
constexpr size_t precond_static_smem() {
  using S = Shape<D, P>;
  constexpr int W = D * P + 1;
  return (size_t)S::NPE * W * 2 + (size_t)S::NPE * S::NPE + (size_t)S::NPE * 2 + (D * P + 2) * 4 + 64;
}

template <int D, int P, int EQ, typename R>
cudaError_t run_precond(const ldg_handle* h, const R* K11, const R* K12, const R* K21, const R* Kw, R* F,
                        R* Ud, double shift, double scale, cudaStream_t st) {
  constexpr int NC = NComp<EQ, D>::value;
  constexpr bool VISC = IsViscous<EQ>::value;
  constexpr int W = D * P + 1;
  const size_t smem = precond_smem<D, P, EQ, R>();
  cudaError_t err;
  if (smem + precond_static_smem<D, P>() <= 227 * 1024) {
    auto kern = k_precond<D, P, NC, VISC, R, false>;
    err = set_smem_once(kern, smem);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)h->E, 256, smem, st>>>(K11, K12, K21, Kw, F, Ud, h->geo(), h->tab, pc_tables(h), shift,
                                             scale);
  } else {
    const size_t sm_in = (size_t)Shape<D, P>::NPE * W * D * sizeof(R);
    auto kern = k_precond<D, P, NC, VISC, R, true>;
    err = set_smem_once(kern, sm_in);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)h->E, 256, sm_in, st>>>(K11, K12, K21, Kw, F, Ud, h->geo(), h->tab, pc_tables(h), shift,
                                              scale);
  }
  count_launch();
  return cudaGetLastError();
}

template <int D, int P, int NC, int G, typename R, typename V>
cudaError_t launch_apply_lanes(const ldg_handle* h, const R* F, const V* r, V* z, cudaStream_t st) {
  using A = ApplyLanes<D, P, NC, G, R, V>;
  const int64_t epb = (int64_t)A::EPW * A::WPB;
  const int64_t blocks = (h->E + epb - 1) / epb;
  k_precond_apply<D, P, NC, G, R, V><<<(unsigned)blocks, A::THREADS, 0, st>>>(F, r, z, h->E);
  count_launch();
  return cudaGetLastError();
}

template <int D, int P, int EQ, typename R, typename V>
cudaError_t run_precond_apply(const ldg_handle* h, const R* F, const V* r, V* z,
                              cudaStream_t st) {
  constexpr int NC = NComp<EQ, D>::value;
  // FP32, 3-D elements up to p = 3: by wavefronts (measured 0.59 against
  // 0.68 ms on the 32^3, p = 3 Taylor-Green apply; 0.94 ms for one lane per
  // component). FP32 3-D p = 4: one lane per component along the row chain,
  // rolled (six elements per warp, no group sums; 0.41 against 0.52 ms for
  // one lane per entry on a 32 x 16 x 16 channel; by wavefronts the full
  // channel took 8.0 against 3.3 ms, a level's scattered 4-byte loads of 13
  // slots thrashing L1). FP32 2-D: one
  // lane per block entry (27 against 32 us for one lane per component and
  // 51 us by wavefronts, 64^2 p = 4). FP64: one lane per component along
  // the row chain (no reductions, fewest FP64 operations: the FP64 pipe is
  // the limit) when the mesh gives at least six such warps per SM, else two
  // lanes per component (twice the warps for a few more FP64 additions);
  // element shapes too large to unroll (3-D) run the same lanes rolled
  // (1.55 against 3.55 ms for one lane per entry on the 32^3, p = 3
  // Taylor-Green mesh; 1.49 against 2.06 ms on the 32 x 16 x 16, p = 4
  // channel).
  if constexpr (sizeof(V) == 4 && D == 3 && P <= 3) {
    using A = ApplyLevels<D, P, NC>;
    const int64_t blocks = (h->E + A::WPB - 1) / A::WPB;
    k_precond_apply_lv<D, P, NC, R, V><<<(unsigned)blocks, A::THREADS, 0, st>>>(F, r, z, h->lvl, h->lvl_ptr, h->E);
    count_launch();
    return cudaGetLastError();
  } else if constexpr (sizeof(V) == 4 && D == 3) {
    return launch_apply_lanes<D, P, NC, 1, R, V>(h, F, r, z, st);
  } else if constexpr (sizeof(V) == 8 && ApplyLanes<D, P, NC, 1, R, V>::UNROLL) {
    if constexpr (NC % 2 == 0) {
      const int64_t warps_g1 = (h->E + ApplyLanes<D, P, NC, 1, R, V>::EPW - 1) / ApplyLanes<D, P, NC, 1, R, V>::EPW;
      int dev = 0, sms = 152;
      if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (warps_g1 < 6 * (int64_t)sms) return launch_apply_lanes<D, P, NC, 2, R, V>(h, F, r, z, st);
    }
    return launch_apply_lanes<D, P, NC, 1, R, V>(h, F, r, z, st);
  } else if constexpr (sizeof(V) == 8) {
    return launch_apply_lanes<D, P, NC, 1, R, V>(h, F, r, z, st);
  } else {
    return launch_apply_lanes<D, P, NC, NC, R, V>(h, F, r, z, st);
  }
}

}  // namespace ldg
