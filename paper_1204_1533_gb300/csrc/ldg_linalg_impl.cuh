// Split Jacobian-vector product and element-block ILU(0) preconditioner
// (Sec. 4.2, Eq. 41 and the block-Jacobi preconditioner A~).
//
//   g = K21 x                        (k_k21_apply; the discrete gradient of x)
//   y = shift x + scale (K11 x + K12 g)       (k_jacvec)
//   A~_e = shift I + scale mask_e(K11 + K12 K21), block ILU(0)   (k_precond)
//   z = (L U)^-1 r                   (k_precond_apply)
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
    k_k21_apply(const R* __restrict__ K21, const V* __restrict__ x, V* __restrict__ gout, Geo g) {
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

template <int D, int P, int NC, int EQ, typename R, typename V>
__global__ void __launch_bounds__(Shape<D, P>::THREADS)
    k_jacvec(const R* __restrict__ K11, const R* __restrict__ K12, const V* __restrict__ x,
             const V* __restrict__ gx, V* __restrict__ y, double shift, double scale, Geo g) {
  using S = Shape<D, P>;
  constexpr int N = S::N, NPE = S::NPE, NCD = NC * D;
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
  const int le = threadIdx.x / S::TPE, rr = threadIdx.x % S::TPE;
  if (le < ne) {
    const int d = rr / S::NL, l = rr % S::NL;
    const int64_t e = e0 + le;
    const int64_t L = (e * D + d) * S::NL + l;
    const int st = S::stride(d), b0 = S::base(d, l);
    V acc[N][NC];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[i][c] = V(0);
    // K11 in-line block
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = 0; j < N; ++j) {
        V xj[NC];
#pragma unroll
        for (int cp = 0; cp < NC; ++cp) xj[cp] = sx[le * tile + cp * NPE + b0 + j * st];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int cp = 0; cp < NC; ++cp)
            acc[i][c] += (V)K11[tile_index(L, NK11, ((i * N + j) * NC + c) * NC + cp)] * xj[cp];
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
      for (int i = 0; i < N; ++i)
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int cp = 0; cp < NC; ++cp)
            acc[i][c] += (V)K11[tile_index(L, NK11, OFF11 + ((end * N + i) * NC + c) * NC + cp)] * xo[cp];
    }
    if constexpr (VISC) {
#pragma unroll
      for (int i = 0; i < N; ++i)
#pragma unroll 1
        for (int j = 0; j < N; ++j) {
#pragma unroll
          for (int cb = 0; cb < NCD; ++cb) {
            const V gj = sgx[le * gt + cb * NPE + b0 + j * st];
#pragma unroll
            for (int c = 0; c < NC; ++c)
              acc[i][c] += (V)K12[tile_index(L, NK12, ((i * N + j) * NC + c) * NCD + cb)] * gj;
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
          for (int i = 0; i < N; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c)
              acc[i][c] += (V)K12[tile_index(L, NK12, OFF12 + (i * NC + c) * NCD + cb)] * go;
        }
      }
    }
    V* yo = sy + (size_t)(le * D + d) * tile;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int c = 0; c < NC; ++c) yo[c * NPE + b0 + i * st] = acc[i][c];
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

struct PcTables {
  const int16_t* pat;   // [NPE][W]
  const int8_t* slot;   // [NPE][NPE]
  const int8_t* nbf;    // [E][2D]
  const int16_t* lvl;   // [NPE]
  const int32_t* lptr;  // [levels + 1]
};

template <int D, int P, int NC, bool VISC, typename R>
__global__ void __launch_bounds__(256)
    k_precond(const R* __restrict__ K11, const R* __restrict__ K12, const R* __restrict__ K21,
              R* __restrict__ F, R* __restrict__ Dinv, Geo g, PcTables pt, double shift,
              double scale) {
  using S = Shape<D, P>;
  constexpr int N = S::N, NPE = S::NPE, NL = S::NL, W = D * P + 1, NCD = NC * D, BB = NC * NC;
  constexpr int64_t NK11 = (N * N + 2 * N) * NC * NC;
  constexpr int64_t NK12 = VISC ? (N * N + N) * NC * NCD : 1;
  constexpr int64_t NK21 = (N * N + N) * D;
  constexpr int OFF12 = N * N * NC * NCD;
  extern __shared__ unsigned char smraw[];
  R* A = reinterpret_cast<R*>(smraw);            // [NPE][W][NC][NC]
  R* Di = A + NPE * W * BB;                        // [NPE][NC][NC]
  R* K21e = Di + NPE * BB;                         // [NPE][W][D] element part of K21
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const R sc = (R)scale;
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
      const int s = pt.slot[ni * NPE + nj];
      A[(ni * W + s) * BB + cc] += sc * K11[tile_index(L, NK11, ((i * N + j) * NC + cc / NC) * NC + cc % NC)];
    }
    if constexpr (VISC)
      for (int k = tid; k < NL * N * N * D; k += nt) {
        const int l = k / (N * N * D), i = (k / (N * D)) % N, j = (k / D) % N, b = k % D;
        const int b0 = S::base(d, l);
        const int ni = b0 + i * st, nj = b0 + j * st;
        const int64_t L = (e * D + d) * NL + l;
        K21e[(ni * W + pt.slot[ni * NPE + nj]) * D + b] += K21[tile_index(L, NK21, (i * N + j) * D + b)];
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
            const int nj = pt.pat[ng * W + s2];
            const int s = pt.slot[ni * NPE + nj];
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
          accs[pt.slot[ni * NPE + nk]] += v;
        }
      }
#pragma unroll
      for (int s = 0; s < W; ++s) A[(ni * W + s) * BB + c * NC + cp] += sc * accs[s];
    }
    __syncthreads();
  }
  // block ILU(0), IKJ order, in the pattern
#pragma unroll 1
  for (int i = 0; i < NPE; ++i) {
#pragma unroll 1
    for (int s = 0; s < W; ++s) {
      const int k = pt.pat[i * W + s];
      if (k >= i) break;
      // A_ik <- A_ik Dinv_k
      R tmp = 0;
      if (tid < BB) {
        const int c = tid / NC, cp = tid % NC;
#pragma unroll
        for (int m = 0; m < NC; ++m) tmp += A[(i * W + s) * BB + c * NC + m] * Di[k * BB + m * NC + cp];
      }
      __syncthreads();
      if (tid < BB) A[(i * W + s) * BB + tid] = tmp;
      __syncthreads();
      // A_ij -= A_ik A_kj for j > k in both patterns
      for (int q = tid; q < W * BB; q += nt) {
        const int s2 = q / BB, c = (q / NC) % NC, cp = q % NC;
        const int j = pt.pat[i * W + s2];
        if (j <= k) continue;
        const int sk = pt.slot[k * NPE + j];
        if (sk < 0) continue;
        R v = 0;
#pragma unroll
        for (int m = 0; m < NC; ++m) v += A[(i * W + s) * BB + c * NC + m] * A[(k * W + sk) * BB + m * NC + cp];
        A[(i * W + s2) * BB + c * NC + cp] -= v;
      }
      __syncthreads();
    }
    if (tid == 0) invert_block<R, NC>(A + (i * W + pt.slot[i * NPE + i]) * BB, Di + i * BB);
    __syncthreads();
  }
  for (int k = tid; k < NPE * W * BB; k += nt) F[e * NPE * W * BB + k] = A[k];
  for (int k = tid; k < NPE * BB; k += nt) Dinv[e * NPE * BB + k] = Di[k];
}

template <int D, int P, int NC, typename R, typename V>
__global__ void k_precond_apply(const R* __restrict__ F, const R* __restrict__ Dinv,
                                const V* __restrict__ r, V* __restrict__ z, PcTables pt, int64_t E) {
  using S = Shape<D, P>;
  constexpr int N = S::N, NPE = S::NPE, W = D * P + 1, BB = NC * NC, tile = NC * NPE;
  constexpr int NLEV = D * P + 1;
  __shared__ V y[NPE * NC];
  __shared__ V t[NPE * NC];
  const int64_t e = blockIdx.x;
  const int tid = threadIdx.x;
  const int i = tid / NC, c = tid % NC;
  const bool act = tid < NPE * NC;
  int lev = 0;
  if (act) {
    lev = (i % N) + ((i / N) % N) + (i / (N * N));
    y[c * NPE + i] = r[e * tile + c * NPE + i];
  }
  __syncthreads();
  const R* Fe = F + (size_t)e * NPE * W * BB;
  // forward: y_i -= sum_{k < i} L_ik y_k, level by level
  for (int lv = 1; lv < NLEV; ++lv) {
    V acc = 0;
    if (act && lev == lv) {
      acc = y[c * NPE + i];
      for (int s = 0; s < W; ++s) {
        const int k = pt.pat[i * W + s];
        if (k >= i) break;
#pragma unroll
        for (int m = 0; m < NC; ++m) acc -= (V)Fe[(i * W + s) * BB + c * NC + m] * y[m * NPE + k];
      }
    }
    __syncthreads();
    if (act && lev == lv) y[c * NPE + i] = acc;
    __syncthreads();
  }
  // backward: z_i = Dinv_i (y_i - sum_{j > i} U_ij z_j), levels descending
  for (int lv = NLEV - 1; lv >= 0; --lv) {
    if (act && lev == lv) {
      V acc = y[c * NPE + i];
      for (int s = W - 1; s >= 0; --s) {
        const int j = pt.pat[i * W + s];
        if (j <= i) break;
#pragma unroll
        for (int m = 0; m < NC; ++m) acc -= (V)Fe[(i * W + s) * BB + c * NC + m] * y[m * NPE + j];
      }
      t[c * NPE + i] = acc;
    }
    __syncthreads();
    if (act && lev == lv) {
      V v = 0;
#pragma unroll
      for (int m = 0; m < NC; ++m) v += (V)Dinv[((size_t)e * NPE + i) * BB + c * NC + m] * t[m * NPE + i];
      y[c * NPE + i] = v;
    }
    __syncthreads();
  }
  if (act) z[e * tile + c * NPE + i] = y[c * NPE + i];
}

// ---------------------------------------------------------------------------
template <int D, int P, int EQ, typename R, typename V>
cudaError_t run_jacvec(const ldg_handle* h, const R* K11, const R* K12, const R* K21, V* gbuf,
                       double shift, double scale, const V* x, V* y, cudaStream_t st) {
  using S = Shape<D, P>;
  constexpr int NC = NComp<EQ, D>::value;
  constexpr bool VISC = IsViscous<EQ>::value;
  const int64_t blocks = (h->E + S::EPB - 1) / S::EPB;
  cudaError_t err;
  if constexpr (VISC) {
    const size_t sm1 = (size_t)S::EPB * (NC * S::NPE + D * NC * D * S::NPE) * sizeof(V);
    auto k1 = k_k21_apply<D, P, NC, R, V>;
    err = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (err != cudaSuccess) return err;
    k1<<<(unsigned)blocks, S::THREADS, sm1, st>>>(K21, x, gbuf, h->geo());
    count_launch();
  }
  const size_t sm2 = (size_t)S::EPB * (NC * S::NPE + (VISC ? NC * D * S::NPE : 0) + D * NC * S::NPE) * sizeof(V);
  auto k2 = k_jacvec<D, P, NC, EQ, R, V>;
  err = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  if (err != cudaSuccess) return err;
  k2<<<(unsigned)blocks, S::THREADS, sm2, st>>>(K11, K12, x, gbuf, y, shift, scale, h->geo());
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

template <int D, int P, int EQ, typename R>
size_t precond_smem() {
  constexpr int NC = NComp<EQ, D>::value;
  using S = Shape<D, P>;
  constexpr int W = D * P + 1;
  return (size_t)(S::NPE * W * NC * NC + S::NPE * NC * NC + S::NPE * W * D) * sizeof(R);
}

template <int D, int P, int EQ, typename R>
cudaError_t run_precond(const ldg_handle* h, const R* K11, const R* K12, const R* K21, R* F, R* Dinv,
                        double shift, double scale, cudaStream_t st) {
  constexpr int NC = NComp<EQ, D>::value;
  constexpr bool VISC = IsViscous<EQ>::value;
  const size_t smem = precond_smem<D, P, EQ, R>();
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  auto kern = k_precond<D, P, NC, VISC, R>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  kern<<<(unsigned)h->E, 256, smem, st>>>(K11, K12, K21, F, Dinv, h->geo(), pc_tables(h), shift, scale);
  count_launch();
  return cudaGetLastError();
}

template <int D, int P, int EQ, typename R, typename V>
cudaError_t run_precond_apply(const ldg_handle* h, const R* F, const R* Dinv, const V* r, V* z,
                              cudaStream_t st) {
  constexpr int NC = NComp<EQ, D>::value;
  using S = Shape<D, P>;
  const int threads = ((S::NPE * NC + 31) / 32) * 32;
  k_precond_apply<D, P, NC, R, V><<<(unsigned)h->E, threads, 0, st>>>(F, Dinv, r, z, pc_tables(h), h->E);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ldg
