// Orthogonalisation of one Arnoldi column for GMRES (Sec. 4.2: the linear
// systems of Eq. 39 are solved by preconditioned GMRES): classical
// Gram-Schmidt with one re-orthogonalisation pass (CGS2) as three fused
// sweeps over the basis V_0 .. V_{kv-1}:
//   S1  h1 = V^T w
//   S2  w <- w - V h1,  h2 = V^T w,  nrm2 = ||w||^2
//   S3  w <- (w - V h2) / hn,  hn^2 = nrm2 - ||h2||^2
// The norm of the final vector follows from the second pass (V orthonormal:
// ||w - V h2||^2 = ||w||^2 - ||h2||^2), so S3 needs no reduction and carries
// the normalisation; when the second pass removed almost all of w (the
// difference cancels) the norm is taken explicitly instead. The Hessenberg
// column is h1 + h2 and hn.
//
// Selective variant: the second pass only where one pass may have lost
// orthogonality, by Rutishauser's criterion (re-orthogonalise when the pass
// shrank w by more than a factor K, 10 by default). S1 also returns ||w||^2, so the
// norm after one pass is known before it is made (||w - V h1||^2 =
// ||w||^2 - ||h1||^2, losing at most two digits at the accepted ratios); if
// the ratio passes, one sweep w <- (w - V h1) / hn finishes the column (two
// sweeps, half the multiply-adds of CGS2), otherwise S2 and S3 follow.
//
// FP64 sweeps are bound by the narrow FP64 pipe of this part, so every FP64
// instruction counts: their kernels are instantiated for the exact basis size
// (no predicated-off multiply-adds), read element pairs with 16-byte loads so
// that few threads (one or two blocks per SM) keep enough bytes in flight,
// and reduce the kv + 1 partial sums of a warp by recursive halving (fewer
// threads: fewer partial sums, each reduction step an FP64 addition). FP32
// sweeps are bound by memory and keep a coarser dispatch (basis size rounded
// up to 8, guarded) with two blocks per SM.
#include <cmath>
#include <mutex>
#include <utility>

#include "ldg_internal.h"

namespace ldg {

constexpr int GS_THREADS = 256;
constexpr int GS_WARPS = GS_THREADS / 32;
enum class GsOp { Dots, DotsNorm, UpdateDotsNorm, UpdateScale };

__host__ __device__ constexpr int pow2ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Sweep over kk = KC basis vectors (EXACT) or kk <= KC (guarded). Partial
// sums: row r of `part` ([rows][gridDim.x]) receives block sums of value r:
// the dots (rows 0..kk-1) and, for DotsNorm and UpdateDotsNorm, ||w||^2 of
// the (updated) vector in row kk.
// VEC = 2: each thread takes two consecutive elements per load (16-byte
// loads of FP64 pairs; n even, vectors 16-byte aligned), which doubles the
// bytes in flight per load without more threads (more threads would mean
// more partial sums to reduce, each an FP64 addition).
template <typename V, int VEC>
struct Vec;
template <typename V>
struct Vec<V, 1> {
  using T = V;
  __device__ __forceinline__ static V at(const T& x, int) { return x; }
  __device__ __forceinline__ static void put(T& x, int, V v) { x = v; }
};
template <>
struct Vec<double, 2> {
  using T = double2;
  __device__ __forceinline__ static double at(const T& x, int c) { return c ? x.y : x.x; }
  __device__ __forceinline__ static void put(T& x, int c, double v) {
    if (c)
      x.y = v;
    else
      x.x = v;
  }
};

template <typename V, int VEC, int KC>
constexpr int gs_min_blocks() {
  return sizeof(V) == 4 ? 2 : ((VEC == 2 && KC <= 12) || (VEC == 1 && KC <= 8) ? 2 : 1);
}

template <typename V, GsOp OP, int KC, bool EXACT, int VEC>
__global__ void __launch_bounds__(GS_THREADS, (gs_min_blocks<V, VEC, KC>()))
    k_ortho(const V* __restrict__ Vb, int64_t n, int kk, V* __restrict__ w, const double* __restrict__ h,
            double scale, const double* __restrict__ dsc, double* __restrict__ part) {
  using VT = typename Vec<V, VEC>::T;
  // UpdateScale with a device scale (dsc, written by k_gs_reduce_scale):
  // 0 means the column needs another pass and this sweep does nothing
  V sc = (V)scale;
  if constexpr (OP == GsOp::UpdateScale) {
    if (dsc) {
      const double sd = dsc[0];
      if (sd == 0.0) return;
      sc = (V)sd;
    }
  }
  constexpr bool UPD = OP == GsOp::UpdateDotsNorm || OP == GsOp::UpdateScale;
  constexpr bool DOTS = OP != GsOp::UpdateScale;
  constexpr bool NORM = OP == GsOp::UpdateDotsNorm || OP == GsOp::DotsNorm;
  constexpr int NV = KC + (NORM ? 1 : 0);  // values reduced per thread
  static_assert(NV <= 32, "at most 32 values per warp reduction");
  const int k = EXACT ? KC : kk;
  __shared__ V hs[KC];
  __shared__ double red[GS_WARPS][NV > 0 ? NV : 1];
  if (UPD && threadIdx.x < k) hs[threadIdx.x] = (V)h[threadIdx.x];
  if (UPD) __syncthreads();
  V acc[NV > 0 ? NV : 1];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = V(0);
  const int64_t nv = n / VEC;
  const VT* Vv = reinterpret_cast<const VT*>(Vb);
  VT* wv = reinterpret_cast<VT*>(w);
  for (int64_t i = (int64_t)blockIdx.x * GS_THREADS + threadIdx.x; i < nv; i += (int64_t)gridDim.x * GS_THREADS) {
    VT v[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j)
      if (EXACT || j < k) v[j] = Vv[(int64_t)j * nv + i];
    VT sv = wv[i];
#pragma unroll
    for (int c = 0; c < VEC; ++c) {
      V s = Vec<V, VEC>::at(sv, c);
      if constexpr (UPD) {
        V p[4] = {V(0), V(0), V(0), V(0)};  // four independent chains
#pragma unroll
        for (int j = 0; j < KC; ++j)
          if (EXACT || j < k) p[j & 3] += hs[j] * Vec<V, VEC>::at(v[j], c);
        s -= (p[0] + p[1]) + (p[2] + p[3]);
        if constexpr (OP == GsOp::UpdateScale) s *= sc;
        Vec<V, VEC>::put(sv, c, s);
      }
      if constexpr (DOTS) {
#pragma unroll
        for (int j = 0; j < KC; ++j)
          if (EXACT || j < k) acc[j] += Vec<V, VEC>::at(v[j], c) * s;
        if constexpr (NORM) acc[KC] += s * s;
      }
    }
    if constexpr (UPD) wv[i] = sv;
  }
  if constexpr (DOTS) {
    // warp sums of NV values by recursive halving: each exchange halves the
    // values a lane holds, so lane l ends with the warp total of value
    // l mod KP after KP - 1 + log2(32 / KP) additions (a butterfly per value
    // would take 5 NV)
    constexpr int KP = pow2ceil(NV);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    double x[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) x[j] = j < NV ? (double)acc[j] : 0.0;
#pragma unroll
    for (int half = KP / 2; half >= 1; half >>= 1) {
      const bool up = (lane & half) != 0;
#pragma unroll
      for (int q = 0; q < half; ++q) {
        const double keep = up ? x[half + q] : x[q];
        const double send = up ? x[q] : x[half + q];
        x[q] = keep + __shfl_xor_sync(0xffffffffu, send, half);
      }
    }
    double t = x[0];
#pragma unroll
    for (int o = KP; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane < NV) red[wp][lane] = t;
    __syncthreads();
    if (threadIdx.x < NV) {
      const int j = threadIdx.x;
      const bool live = EXACT || j < k || (NORM && j == KC);
      if (live) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < GS_WARPS; ++q) s += red[q][j];
        const int row = (NORM && j == KC) ? k : j;
        part[(int64_t)row * gridDim.x + blockIdx.x] = s;
      }
    }
  }
}

// Row sums of the block partials: s_r = sum_b part[r][b] for r < rows;
// out[r] = s_r; acc[r] = s_r (mode 1) or acc[r] += s_r (mode 2) for r < nacc,
// and acc[r] = s_r for nacc <= r < rows.
__global__ void k_gs_reduce(const double* __restrict__ part, int nblk, double* __restrict__ out,
                            double* __restrict__ acc, int nacc, int mode) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[(int64_t)blockIdx.x * nblk + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) {
      const int r = blockIdx.x;
      if (out) out[r] = s;
      if (acc) {
        if (r < nacc && mode == 2)
          acc[r] += s;
        else if (mode != 0)
          acc[r] = s;
      }
    }
  }
}

// k_gs_reduce for rows <= 64 in one block, then the column's norm after the
// pass from its rows (V orthonormal: ||w - V h||^2 = ||w||^2 - ||h||^2, with
// h = rows 0..kv-1 and ||w||^2 = row kv): accepted when the difference keeps
// at least 1/thr of ||w||^2; sc[0] = 1/hn (1 when hn = 0) or 0 when not
// accepted, sc[1] = hn.
__global__ void __launch_bounds__(256) k_gs_reduce_scale(const double* __restrict__ part, int nblk, int rows,
                                                         double* __restrict__ out, double* __restrict__ acc,
                                                         int nacc, int mode, int kv, double thr,
                                                         double* __restrict__ sc) {
  __shared__ double val[64];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int r = wp; r < rows; r += 8) {
    double s = 0.0;
    for (int i = lane; i < nblk; i += 32) s += part[(int64_t)r * nblk + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      val[r] = s;
      if (out) out[r] = s;
      if (acc) {
        if (r < nacc && mode == 2)
          acc[r] += s;
        else if (mode != 0)
          acc[r] = s;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ssq = 0.0;
    for (int j = 0; j < kv; ++j) ssq += val[j] * val[j];
    const double ww = val[kv], hn2 = ww - ssq;
    const bool ok = isfinite(ww) && isfinite(ssq) && hn2 >= 0.0 && hn2 * thr >= ww;
    const double hn = ok ? sqrt(hn2) : 0.0;
    sc[0] = ok ? (hn > 0.0 ? 1.0 / hn : 1.0) : 0.0;
    sc[1] = hn;
  }
}

template <typename V>
__global__ void k_gs_scale(V* __restrict__ w, double s, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (V)(s * (double)w[i]);
}

static int sm_count() {
  static std::mutex mu;
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lock(mu);
  if (!cached[dev]) {
    int s = 0;
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s < 1) s = 152;
    cached[dev] = s;
  }
  return cached[dev];
}

template <typename V>
static int gs_blocks() {
  const int b = sm_count() * 2;
  return b < GS_MAX_BLOCKS ? b : GS_MAX_BLOCKS;
}

// ---- dispatch tables -------------------------------------------------------
template <typename V, GsOp OP>
using GsKernel = void (*)(const V*, int64_t, int, V*, const double*, double, const double*, double*);

template <typename V, GsOp OP, int... K>
static GsKernel<V, OP> exact_kernel(int kk, std::integer_sequence<int, K...>) {
  static constexpr GsKernel<V, OP> tab[] = {&k_ortho<V, OP, K + 1, true, 2>...};
  return tab[kk - 1];
}
static constexpr int exact_blocks_tab[] = {2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1,
                                           1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};

// largest basis size of one fused sweep
template <GsOp OP>
constexpr int gs_kmax() { return (OP == GsOp::UpdateDotsNorm || OP == GsOp::DotsNorm) ? GS_KMAX - 1 : GS_KMAX; }

// kernel and blocks per SM for a sweep over kk vectors of length n: FP64 on
// even lengths takes the exact pair kernels, everything else the guarded
// scalar kernels with kk rounded up to 8
template <typename V, GsOp OP>
static GsKernel<V, OP> pick(int kk, int64_t n, const void* a, const void* b, int* per_sm) {
  if constexpr (sizeof(V) == 8) {
    const bool pairs = (n % 2 == 0) && ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0);
    if (pairs) {
      *per_sm = exact_blocks_tab[kk - 1];
      return exact_kernel<V, OP>(kk, std::make_integer_sequence<int, gs_kmax<OP>()>{});
    }
  }
  if (kk <= 8) {
    *per_sm = gs_min_blocks<V, 1, 8>();
    return &k_ortho<V, OP, 8, false, 1>;
  }
  if (kk <= 16) {
    *per_sm = gs_min_blocks<V, 1, 16>();
    return &k_ortho<V, OP, 16, false, 1>;
  }
  if (kk <= 24) {
    *per_sm = gs_min_blocks<V, 1, 24>();
    return &k_ortho<V, OP, 24, false, 1>;
  }
  *per_sm = gs_min_blocks<V, 1, gs_kmax<OP>()>();
  return &k_ortho<V, OP, gs_kmax<OP>(), false, 1>;
}

// One sweep over kk basis vectors; partial sums in part (rows x blocks),
// returns the number of blocks (0 on a launch error).
template <typename V, GsOp OP>
static int sweep(const V* Vb, int kk, int64_t n, V* w, const double* h, double scale, double* part,
                 cudaStream_t st, const double* dsc = nullptr) {
  constexpr bool UPD = OP == GsOp::UpdateDotsNorm || OP == GsOp::UpdateScale;
  const double vsz = sizeof(V), nn = (double)n;
  const double flops = OP == GsOp::Dots       ? 2.0 * kk
                       : OP == GsOp::DotsNorm ? 2.0 * kk + 2.0
                       : (OP == GsOp::UpdateDotsNorm ? 4.0 * kk + 2.0 : 2.0 * kk + 1.0);
  int per_sm = 1;
  const GsKernel<V, OP> kern = pick<V, OP>(kk, n, Vb, w, &per_sm);
  int nb = sm_count() * per_sm;
  if (nb > GS_MAX_BLOCKS) nb = GS_MAX_BLOCKS;
  {
    TimedScope tl(KT_ORTHO, sizeof(V) == 4 ? LDG_PREC_FP32 : LDG_PREC_FP64, st,
                  nn * vsz * (kk + 1 + (UPD ? 1 : 0)), nn * flops);
    kern<<<nb, GS_THREADS, 0, st>>>(Vb, n, kk, w, h, scale, dsc, part);
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? nb : 0;
}

static cudaError_t reduce(const double* part, int nblk, int rows, double* out, double* acc, int nacc, int mode,
                          cudaStream_t st) {
  k_gs_reduce<<<rows, 256, 0, st>>>(part, nblk, out, acc, nacc, mode);
  count_launch();
  return cudaGetLastError();
}
static cudaError_t reduce_scale(const double* part, int nblk, int rows, double* out, double* acc, int nacc, int mode,
                                int kv, double thr, double* sc, cudaStream_t st) {
  k_gs_reduce_scale<<<1, 256, 0, st>>>(part, nblk, rows, out, acc, nacc, mode, kv, thr, sc);
  count_launch();
  return cudaGetLastError();
}

// the column read-back: acc[0..kv] and sc[0..1] to host (pinned when pin is
// given: the copies are queued and the event marks them, so the GPU goes on
// with the update sweep while the host waits), into col[0..kv] and
// col[kv + 1], col[kv + 2]
static cudaError_t read_column(const double* acc, const double* sc, int kv, double* col, double* pin,
                               cudaEvent_t ev, cudaStream_t st) {
  double* dst = pin ? pin : col;
  cudaError_t e = cudaMemcpyAsync(dst, acc, (size_t)(kv + 1) * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst + kv + 1, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev, st);
  return e;
}
static cudaError_t wait_column(int kv, double* col, const double* pin, cudaEvent_t ev, cudaStream_t st) {
  cudaError_t e = ev ? cudaEventSynchronize(ev) : cudaStreamSynchronize(st);
  if (e == cudaSuccess && pin)
    for (int j = 0; j < kv + 3; ++j) col[j] = pin[j];
  return e;
}

template <typename V>
int arnoldi_column(const V* Vb, int kv, int64_t n, V* w, double* part, double* gs, double* col, double reorth_k,
                   int* passes, double* pin, cudaEvent_t ev, cudaStream_t st) {
  double* h1 = gs + 2 * (GS_MAX_BASIS + 2);  // first-pass coefficients
  double* acc = gs;                          // h1 + h2 (kv), then the norm row
  double* h2 = gs + kv + 1;                  // second-pass coefficients
  double* sc = gs + 4 * (GS_MAX_BASIS + 2);  // device scale of the update sweep, hn
  int nb;
  if (passes) *passes = 2;
  if (kv <= gs_kmax<GsOp::UpdateDotsNorm>()) {
    // each pass's reduction also forms the norm after the pass and its
    // scale on the device, so the update + scale sweep is queued before the
    // host reads the column; it does nothing when the pass is not accepted
    if (reorth_k > 0.0) {
      // S1 with ||w||^2; one pass when it keeps more than 1/K of w
      const double K = reorth_k;
      if (!(nb = sweep<V, GsOp::DotsNorm>(Vb, kv, n, w, nullptr, 1.0, part, st))) return LDG_ERR_CUDA;
      LDG_CUDA_TRY(reduce_scale(part, nb, kv + 1, h1, acc, kv, 1, kv, K * K, sc, st));
      LDG_CUDA_TRY(read_column(acc, sc, kv, col, pin, ev, st));
      if (!sweep<V, GsOp::UpdateScale>(Vb, kv, n, w, h1, 1.0, part, st, sc)) return LDG_ERR_CUDA;
      LDG_CUDA_TRY(wait_column(kv, col, pin, ev, st));
      double h1sq = 0.0;
      for (int j = 0; j < kv; ++j) h1sq += col[j] * col[j];
      if (!std::isfinite(col[kv]) || !std::isfinite(h1sq)) return LDG_ERR_NONFINITE;
      if (col[kv + 1] != 0.0) {
        col[kv] = col[kv + 2];
        if (passes) *passes = 1;
        return LDG_OK;
      }
    } else {
      if (!(nb = sweep<V, GsOp::Dots>(Vb, kv, n, w, nullptr, 1.0, part, st))) return LDG_ERR_CUDA;
      LDG_CUDA_TRY(reduce(part, nb, kv, h1, acc, kv, 1, st));
    }
    // second pass; the norm after it from its dots (Pythagoras) unless the
    // pass removed nearly all of w
    const double guard = sizeof(V) == 8 ? 1e-4 : 1e-2;
    if (!(nb = sweep<V, GsOp::UpdateDotsNorm>(Vb, kv, n, w, h1, 1.0, part, st))) return LDG_ERR_CUDA;
    LDG_CUDA_TRY(reduce_scale(part, nb, kv + 1, h2, acc, kv, 2, kv, 1.0 / guard, sc, st));
    LDG_CUDA_TRY(read_column(acc, sc, kv, col, pin, ev, st));
    if (!sweep<V, GsOp::UpdateScale>(Vb, kv, n, w, h2, 1.0, part, st, sc)) return LDG_ERR_CUDA;
    LDG_CUDA_TRY(wait_column(kv, col, pin, ev, st));
    double asq = 0.0;
    for (int j = 0; j < kv; ++j) asq += col[j] * col[j];
    if (!std::isfinite(col[kv]) || !std::isfinite(asq)) return LDG_ERR_NONFINITE;
    if (col[kv + 1] != 0.0) {
      col[kv] = col[kv + 2];
      return LDG_OK;
    }
    // explicit third sweep: w -= V h2 with its norm (its dots are not used)
    double* g3 = gs + 3 * (GS_MAX_BASIS + 2);
    if (!(nb = sweep<V, GsOp::UpdateDotsNorm>(Vb, kv, n, w, h2, 1.0, part, st))) return LDG_ERR_CUDA;
    LDG_CUDA_TRY(reduce(part, nb, kv + 1, nullptr, g3, 0, 1, st));
    double nn2 = 0.0;
    LDG_CUDA_TRY(cudaMemcpyAsync(&nn2, g3 + kv, sizeof(double), cudaMemcpyDeviceToHost, st));
    LDG_CUDA_TRY(cudaStreamSynchronize(st));
    if (!std::isfinite(nn2)) return LDG_ERR_NONFINITE;
    const double hn = std::sqrt(nn2);
    if (hn > 0) {
      k_gs_scale<V><<<gs_blocks<V>(), GS_THREADS, 0, st>>>(w, 1.0 / hn, n);
      count_launch();
      LDG_CUDA_TRY(cudaGetLastError());
    }
    col[kv] = hn;
    return LDG_OK;
  }
  // chunks of GS_KMAX vectors: both passes as dots then update sweeps
  for (int pass = 0; pass < 2; ++pass) {
    double* hp = pass ? h2 : h1;
    for (int j0 = 0; j0 < kv; j0 += GS_KMAX) {
      const int kk = kv - j0 < GS_KMAX ? kv - j0 : GS_KMAX;
      if (!(nb = sweep<V, GsOp::Dots>(Vb + (int64_t)j0 * n, kk, n, w, nullptr, 1.0, part, st))) return LDG_ERR_CUDA;
      LDG_CUDA_TRY(reduce(part, nb, kk, hp + j0, acc + j0, kk, pass ? 2 : 1, st));
    }
    for (int j0 = 0; j0 < kv; j0 += GS_KMAX) {
      const int kk = kv - j0 < GS_KMAX ? kv - j0 : GS_KMAX;
      if (!sweep<V, GsOp::UpdateScale>(Vb + (int64_t)j0 * n, kk, n, w, hp + j0, 1.0, part, st)) return LDG_ERR_CUDA;
    }
  }
  if (!(nb = sweep<V, GsOp::Dots>(w, 1, n, w, nullptr, 1.0, part, st))) return LDG_ERR_CUDA;
  LDG_CUDA_TRY(reduce(part, nb, 1, nullptr, acc + kv, 0, 1, st));
  LDG_CUDA_TRY(cudaMemcpyAsync(col, acc, (size_t)(kv + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  LDG_CUDA_TRY(cudaStreamSynchronize(st));
  const double hn = std::sqrt(col[kv]);
  if (!std::isfinite(hn)) return LDG_ERR_NONFINITE;
  if (hn > 0) {
    k_gs_scale<V><<<gs_blocks<V>(), GS_THREADS, 0, st>>>(w, 1.0 / hn, n);
    count_launch();
    LDG_CUDA_TRY(cudaGetLastError());
  }
  col[kv] = hn;
  return LDG_OK;
}

template int arnoldi_column<float>(const float*, int, int64_t, float*, double*, double*, double*, double, int*,
                                   double*, cudaEvent_t, cudaStream_t);
template int arnoldi_column<double>(const double*, int, int64_t, double*, double*, double*, double*, double, int*,
                                    double*, cudaEvent_t, cudaStream_t);

}  // namespace ldg
