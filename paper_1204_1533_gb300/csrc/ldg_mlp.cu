// Line-local MLP Newton predictor: features, fused forward / backward on
// BF16 tensor cores with FP32 accumulation, Adam, prediction scatter.
// Inference (ldg_mlp_forward, ldg_mlp_predict) runs on the tcgen05 tensor
// cores with tensor-memory accumulators (k_mlp_fwd_tc below); training runs
// the fused forward + backward tile kernel described next.
//
// Network n_in -> 128 -> 128 -> 128 -> n_out with GELU (tanh form of
// Hendrycks and Gimpel), n_in <= 96, n_out <= 32. One block of 4 warps
// processes a tile of 32 lines: the transposed BF16 weights and the
// tile's activations live in shared memory; every matrix product is a
// sequence of m16n8k16 BF16 MMAs with FP32 accumulators, fragments loaded
// with ldmatrix (the .trans form for the transposed operands of the
// backward pass). Training writes one partial gradient per block (no
// atomics); a second kernel sums the partials and applies Adam to the FP32
// master weights, a third re-packs the BF16 copies.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "ldg_internal.h"

namespace ldg {
namespace mlp {

constexpr int HID = 128;
constexpr int INP = 96;   // padded input width
constexpr int OUTP = 32;  // padded output width
constexpr int TR = 32;    // lines per tile
constexpr int LDX = INP + 8;
constexpr int LDH = HID + 8;
constexpr int THREADS = 128;
using bf16 = __nv_bfloat16;

__host__ __device__ constexpr int np_of(int nin, int nout) {
  return nin * HID + HID + 2 * (HID * HID + HID) + HID * nout + nout;
}

struct Dev {
  const bf16* W1t;  // [HID][LDX]   W1t[n][k] = W1[k][n]
  const bf16* W2t;  // [HID][LDH]
  const bf16* W3t;  // [HID][LDH]
  const bf16* W4t;  // [OUTP][LDH]
  const float* b1;  // [HID]
  const float* b2;
  const float* b3;
  const float* b4;  // [OUTP]
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm4(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm4t(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float x) {
  const float c = 0.7978845608028654f;  // sqrt(2/pi)
  return 0.5f * x * (1.f + tanhf(c * (x + 0.044715f * x * x * x)));
}
__device__ __forceinline__ float gelu_d(float x) {
  const float c = 0.7978845608028654f;
  const float t = tanhf(c * (x + 0.044715f * x * x * x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * c * (1.f + 3.f * 0.044715f * x * x);
}

// acc[NT][4] += A[r0..r0+15][0..K) * B, n-tiles n0 + 8j. A row-major in
// shared memory; B either W^T stored [n][k] (BT = false) or a [k][n] array
// read transposed (BT = true).
template <int NT, bool BT>
__device__ __forceinline__ void rows_gemm(float (*acc)[4], const bf16* A, int lda, int r0,
                                          const bf16* B, int ldb, int n0, int K) {
  const int lane = threadIdx.x & 31;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    ldsm4(a, A + (r0 + (lane & 15)) * lda + k0 + (lane >> 4) * 8);
#pragma unroll
    for (int j = 0; j < NT; j += 2) {
      uint32_t b[4];
      if (!BT)
        ldsm4(b, B + (n0 + j * 8 + (lane & 7) + (lane >> 4) * 8) * ldb + k0 + ((lane >> 3) & 1) * 8);
      else
        ldsm4t(b, B + (k0 + (lane & 7) + ((lane >> 3) & 1) * 8) * ldb + n0 + j * 8 + (lane >> 4) * 8);
      mma(acc[j], a, b[0], b[1]);
      mma(acc[j + 1], a, b[2], b[3]);
    }
  }
}

// acc[MT][NT][4] += Hin^T dZ over the tile rows (K = TR): output rows
// m0 + 16 i (input features), columns n0 + 8 j (outputs)
template <int MT, int NT>
__device__ __forceinline__ void wgrad_gemm(float (*acc)[NT][4], const bf16* Hin, int ldh, int m0,
                                           const bf16* dZ, int ldz, int n0) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k0 = 0; k0 < TR; k0 += 16) {
    uint32_t a[MT][4];
#pragma unroll
    for (int i = 0; i < MT; ++i)
      ldsm4t(a[i], Hin + (k0 + (lane & 7) + (lane >> 4) * 8) * ldh + m0 + 16 * i + ((lane >> 3) & 1) * 8);
#pragma unroll
    for (int j = 0; j < NT; j += 2) {
      uint32_t b[4];
      ldsm4t(b, dZ + (k0 + (lane & 7) + ((lane >> 3) & 1) * 8) * ldz + n0 + j * 8 + (lane >> 4) * 8);
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        mma(acc[i][j], a[i], b[0], b[1]);
        mma(acc[i][j + 1], a[i], b[2], b[3]);
      }
    }
  }
}

struct Smem {
  bf16 X[TR * LDX];
  bf16 W1[HID * LDX];
  bf16 W2[HID * LDH];
  bf16 W3[HID * LDH];
  bf16 W4[OUTP * LDH];
  bf16 H1[TR * LDH], H2[TR * LDH], H3[TR * LDH];
  bf16 G1[TR * LDH], G2[TR * LDH], G3[TR * LDH];
  bf16 DA[TR * LDH], DB[TR * LDH];
  float gb[3 * HID + OUTP];
  float loss;
};

__device__ __forceinline__ void copy_bf16(bf16* dst, const bf16* src, int n) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < n / 8; i += blockDim.x) d[i] = s[i];
}

// forward epilogue of a hidden layer: H = gelu(acc + b), G = gelu'(acc + b)
__device__ __forceinline__ void hidden_epilogue(float (*acc)[4], const float* b, bf16* H, bf16* G, int r0, int n0) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = r0 + (lane >> 2) + 8 * h;
      const int col = n0 + 8 * j + (lane & 3) * 2;
      const float z0 = acc[j][2 * h] + b[col], z1 = acc[j][2 * h + 1] + b[col + 1];
      *reinterpret_cast<__nv_bfloat162*>(H + row * LDH + col) = __floats2bfloat162_rn(gelu(z0), gelu(z1));
      if (G)
        *reinterpret_cast<__nv_bfloat162*>(G + row * LDH + col) =
            __floats2bfloat162_rn(gelu_d(z0), gelu_d(z1));
    }
}

// backward epilogue: dZ = acc * G (or acc when G is null); bias gradient
// (sum over rows) accumulated into gb via warp shuffles + shared atomics
__device__ __forceinline__ void back_epilogue(float (*acc)[4], const bf16* G, bf16* DZ, float* gb, int r0, int n0) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = r0 + (lane >> 2) + 8 * h;
      const int col = n0 + 8 * j + (lane & 3) * 2;
      float d0 = acc[j][2 * h], d1 = acc[j][2 * h + 1];
      const __nv_bfloat162 g = *reinterpret_cast<const __nv_bfloat162*>(G + row * LDH + col);
      d0 *= __bfloat162float(g.x);
      d1 *= __bfloat162float(g.y);
      *reinterpret_cast<__nv_bfloat162*>(DZ + row * LDH + col) = __floats2bfloat162_rn(d0, d1);
      s0 += d0;
      s1 += d1;
    }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane < 4) {
      atomicAdd(gb + n0 + 8 * j + lane * 2, s0);
      atomicAdd(gb + n0 + 8 * j + lane * 2 + 1, s1);
    }
  }
}

template <int MT, int NT>
__device__ __forceinline__ void store_wgrad(float (*acc)[NT][4], float* slot, int m0, int n0, int nin_valid,
                                            int nout_valid, int ncols) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + 16 * i + (lane >> 2) + 8 * h;
        const int n = n0 + 8 * j + (lane & 3) * 2;
        if (m < nin_valid) {
          if (n < nout_valid) slot[m * ncols + n] = acc[i][j][2 * h];
          if (n + 1 < nout_valid) slot[m * ncols + n + 1] = acc[i][j][2 * h + 1];
        }
      }
}

// One tile of TR lines: forward; in training also the backward pass and the
// tile's partial gradient (flat order of the oracle: W1 b1 W2 b2 W3 b3 W4 b4)
template <bool TRAIN>
__global__ void __launch_bounds__(THREADS)
    k_mlp(const bf16* __restrict__ X, const float* __restrict__ T, float* __restrict__ Y, Dev w, int nin,
          int nout, int64_t M, float gscale, float* __restrict__ slots, int64_t slot_stride) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem& s = *reinterpret_cast<Smem*>(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * TR;
  copy_bf16(s.W1, w.W1t, HID * LDX);
  copy_bf16(s.W2, w.W2t, HID * LDH);
  copy_bf16(s.W3, w.W3t, HID * LDH);
  copy_bf16(s.W4, w.W4t, OUTP * LDH);
  for (int i = threadIdx.x; i < TR * (INP / 8); i += blockDim.x) {
    const int r = i / (INP / 8), c = i % (INP / 8);
    int4 v = make_int4(0, 0, 0, 0);
    if (row0 + r < M) v = reinterpret_cast<const int4*>(X + (row0 + r) * INP)[c];
    *reinterpret_cast<int4*>(s.X + r * LDX + c * 8) = v;
  }
  if (TRAIN) {
    for (int i = threadIdx.x; i < 3 * HID + OUTP; i += blockDim.x) s.gb[i] = 0.f;
    if (threadIdx.x == 0) s.loss = 0.f;
  }
  __syncthreads();
  const int r0 = 16 * (warp & 1), nh = 64 * (warp >> 1);
  float acc[8][4];
  auto zero = [&]() {
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  };
  // ---------------- forward ----------------
  zero();
  rows_gemm<8, false>(acc, s.X, LDX, r0, s.W1, LDX, nh, INP);
  hidden_epilogue(acc, w.b1, s.H1, TRAIN ? s.G1 : nullptr, r0, nh);
  __syncthreads();
  zero();
  rows_gemm<8, false>(acc, s.H1, LDH, r0, s.W2, LDH, nh, HID);
  hidden_epilogue(acc, w.b2, s.H2, TRAIN ? s.G2 : nullptr, r0, nh);
  __syncthreads();
  zero();
  rows_gemm<8, false>(acc, s.H2, LDH, r0, s.W3, LDH, nh, HID);
  hidden_epilogue(acc, w.b3, s.H3, TRAIN ? s.G3 : nullptr, r0, nh);
  __syncthreads();
  const int no = 16 * (warp >> 1);
  float ya[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  rows_gemm<2, false>(ya, s.H3, LDH, r0, s.W4, LDH, no, HID);
  float lsum = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float c0 = 0.f, c1 = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = r0 + (lane >> 2) + 8 * h;
      const int col = no + 8 * j + (lane & 3) * 2;
      const int64_t gr = row0 + r;
      float y0 = ya[j][2 * h] + w.b4[col], y1 = ya[j][2 * h + 1] + w.b4[col + 1];
      if (!TRAIN) {
        if (gr < M) {
          if (col < nout) Y[gr * nout + col] = y0;
          if (col + 1 < nout) Y[gr * nout + col + 1] = y1;
        }
      } else {
        float d0 = 0.f, d1 = 0.f;
        if (gr < M && col < nout) d0 = y0 - T[gr * nout + col];
        if (gr < M && col + 1 < nout) d1 = y1 - T[gr * nout + col + 1];
        lsum += d0 * d0 + d1 * d1;
        d0 *= gscale;
        d1 *= gscale;
        *reinterpret_cast<__nv_bfloat162*>(s.DA + r * LDH + col) = __floats2bfloat162_rn(d0, d1);
        c0 += d0;
        c1 += d1;
      }
    }
    if (TRAIN) {
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        c0 += __shfl_xor_sync(0xffffffffu, c0, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
      }
      if (lane < 4) {
        atomicAdd(s.gb + 3 * HID + no + 8 * j + lane * 2, c0);
        atomicAdd(s.gb + 3 * HID + no + 8 * j + lane * 2 + 1, c1);
      }
    }
  }
  if (!TRAIN) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) atomicAdd(&s.loss, lsum);
  __syncthreads();
  float* slot = slots + blockIdx.x * slot_stride;
  const int oW1 = 0, ob1 = nin * HID, oW2 = ob1 + HID, ob2 = oW2 + HID * HID, oW3 = ob2 + HID,
            ob3 = oW3 + HID * HID, oW4 = ob3 + HID, ob4 = oW4 + HID * nout;
  // ---------------- layer 4 gradients ----------------
  {
    float g4[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) g4[i][j][0] = g4[i][j][1] = g4[i][j][2] = g4[i][j][3] = 0.f;
    wgrad_gemm<2, 4>(g4, s.H3, LDH, 32 * warp, s.DA, LDH, 0);
    store_wgrad<2, 4>(g4, slot + oW4, 32 * warp, 0, HID, nout, nout);
  }
  zero();
  rows_gemm<8, true>(acc, s.DA, LDH, r0, s.W4, LDH, nh, OUTP);  // dH3 = dZ4 W4^T
  back_epilogue(acc, s.G3, s.DB, s.gb + 2 * HID, r0, nh);
  __syncthreads();
  // ---------------- layer 3 ----------------
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    float g[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) g[i][j][0] = g[i][j][1] = g[i][j][2] = g[i][j][3] = 0.f;
    wgrad_gemm<2, 8>(g, s.H2, LDH, 32 * warp, s.DB, LDH, 64 * half);
    store_wgrad<2, 8>(g, slot + oW3, 32 * warp, 64 * half, HID, HID, HID);
  }
  zero();
  rows_gemm<8, true>(acc, s.DB, LDH, r0, s.W3, LDH, nh, HID);  // dH2 = dZ3 W3^T
  back_epilogue(acc, s.G2, s.DA, s.gb + HID, r0, nh);
  __syncthreads();
  // ---------------- layer 2 ----------------
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    float g[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) g[i][j][0] = g[i][j][1] = g[i][j][2] = g[i][j][3] = 0.f;
    wgrad_gemm<2, 8>(g, s.H1, LDH, 32 * warp, s.DA, LDH, 64 * half);
    store_wgrad<2, 8>(g, slot + oW2, 32 * warp, 64 * half, HID, HID, HID);
  }
  zero();
  rows_gemm<8, true>(acc, s.DA, LDH, r0, s.W2, LDH, nh, HID);  // dH1 = dZ2 W2^T
  back_epilogue(acc, s.G1, s.DB, s.gb, r0, nh);
  __syncthreads();
  // ---------------- layer 1: dW1 = X^T dZ1, input rows in 16-row tiles ----------------
#pragma unroll 1
  for (int mt = warp; mt < INP / 16; mt += 4) {
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
      float g[1][8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) g[0][j][0] = g[0][j][1] = g[0][j][2] = g[0][j][3] = 0.f;
      wgrad_gemm<1, 8>(g, s.X, LDX, 16 * mt, s.DB, LDH, 64 * half);
      store_wgrad<1, 8>(g, slot + oW1, 16 * mt, 64 * half, nin, HID, HID);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < HID; i += blockDim.x) {
    slot[ob1 + i] = s.gb[i];
    slot[ob2 + i] = s.gb[HID + i];
    slot[ob3 + i] = s.gb[2 * HID + i];
  }
  for (int i = threadIdx.x; i < nout; i += blockDim.x) slot[ob4 + i] = s.gb[3 * HID + i];
  if (threadIdx.x == 0) slot[ob4 + nout] = s.loss;
}

// sum of the block partials (+ Adam on the FP32 master weights)
__global__ void k_reduce_adam(const float* __restrict__ slots, int nslots, int64_t stride, int np,
                              float* __restrict__ grad, float* __restrict__ theta, float* __restrict__ m,
                              float* __restrict__ v, float lr, float b1, float b2, float eps, float c1,
                              float c2, int do_adam, float* __restrict__ loss, float lscale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > np) return;
  float g = 0.f;
  for (int s = 0; s < nslots; ++s) g += slots[s * stride + i];
  if (i == np) {
    if (loss) *loss = g * lscale;
    return;
  }
  if (grad) grad[i] = g;
  if (do_adam) {
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 transposed, padded copies of the FP32 master weights
__global__ void k_pack(const float* __restrict__ theta, int nin, int nout, bf16* W1t, bf16* W2t, bf16* W3t,
                       bf16* W4t, float* b1, float* b2, float* b3, float* b4) {
  const int oW1 = 0, ob1 = nin * HID, oW2 = ob1 + HID, ob2 = oW2 + HID * HID, oW3 = ob2 + HID,
            ob3 = oW3 + HID * HID, oW4 = ob3 + HID, ob4 = oW4 + HID * nout;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < HID * LDX) {
    const int n = t / LDX, k = t % LDX;
    W1t[t] = __float2bfloat16(k < nin ? theta[oW1 + k * HID + n] : 0.f);
  }
  if (t < HID * LDH) {
    const int n = t / LDH, k = t % LDH;
    W2t[t] = __float2bfloat16(k < HID ? theta[oW2 + k * HID + n] : 0.f);
    W3t[t] = __float2bfloat16(k < HID ? theta[oW3 + k * HID + n] : 0.f);
  }
  if (t < OUTP * LDH) {
    const int n = t / LDH, k = t % LDH;
    W4t[t] = __float2bfloat16(k < HID && n < nout ? theta[oW4 + k * nout + n] : 0.f);
  }
  if (t < HID) {
    b1[t] = theta[ob1 + t];
    b2[t] = theta[ob2 + t];
    b3[t] = theta[ob3 + t];
  }
  if (t < OUTP) b4[t] = t < nout ? theta[ob4 + t] : 0.f;
}

// ---------------------------------------------------------------------------
// Forward pass on the fifth-generation tensor cores (tcgen05): one CTA of 4
// warps per tile of 128 lines (the MMA's M), persistent over the tiles. The
// four weight matrices are packed once (k_pack) in the canonical K-major
// layout without swizzling -- core matrices of 8 rows x 16 bytes, element
// (r, k) of an R x K operand at byte ((r/8)(K/8) + k/8) 128 + (r%8) 16 +
// (k%8) 2 -- and copied to shared memory by bulk asynchronous copies (TMA)
// completing on an mbarrier. Each layer is a chain of
// tcgen05.mma.cta_group::1.kind::f16 (BF16 operands from shared memory, FP32
// accumulator of 128 lanes x N columns in tensor memory, K = 16 per
// instruction) issued by one thread and committed to an mbarrier; every
// thread then reads its row of the accumulator (tcgen05.ld, warp w owns
// lanes 32w .. 32w + 31), adds the bias, applies GELU and writes the BF16
// activation in the same canonical layout as the next layer's A operand.
// Every wait is bounded: on a timeout the tile's outputs are NaN and the
// error flag is set; tensor memory is released in every case.
// ---------------------------------------------------------------------------
namespace tc {

constexpr int TM = 128;          // lines per tile (the MMA's M)
constexpr int TTHREADS = 128;    // one thread per row of the tile
constexpr int TMEM_COLS = 128;   // the accumulator: 128 lanes x 128 FP32 columns
constexpr long WAIT_LIMIT = 1L << 22;

__host__ __device__ constexpr int coff(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

struct __align__(1024) Smem {
  unsigned char W1[HID * INP * 2];    // B of layer 1: [128][96]
  unsigned char W2[HID * HID * 2];    // [128][128]
  unsigned char W3[HID * HID * 2];
  unsigned char W4[OUTP * HID * 2];   // [32][128]
  unsigned char A0[TM * HID * 2];     // X (K = 96), then H2 (K = 128)
  unsigned char A1[TM * HID * 2];     // H1, H3 (K = 128)
  float bias[3 * HID + OUTP];
  unsigned long long bar_w, bar_mma;
  uint32_t taddr;
};
constexpr uint32_t WBYTES = HID * INP * 2 + 2 * HID * HID * 2 + OUTP * HID * 2;

// shared-memory matrix descriptor: start address, leading byte offset
// (between core matrices along K: 128), stride byte offset (between 8-row
// groups: K/8 core matrices of 128 bytes), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(const void* p, int K) {
  const uint64_t a = smem_u32(p), lbo = 128, sbo = (uint64_t)(K / 8) * 128;
  return ((a >> 4) & 0x3FFFull) | (((lbo >> 4) & 0x3FFFull) << 16) | (((sbo >> 4) & 0x3FFFull) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id, int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(id), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait on the phase with the given parity; false after WAIT_LIMIT polls
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long i = 0; i < WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// bulk asynchronous global -> shared copy (16-byte aligned, size a multiple
// of 16) completing `bytes` transactions on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's accumulator lane, waited on
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// one layer: D [128 x N] = A [128 x K] B^T, B stored [N][K]; K / 16 MMAs,
// each advancing both descriptors by two core matrices (256 bytes) along K
__device__ __forceinline__ void layer_mma(uint32_t tmem, const unsigned char* A, const unsigned char* B, int K,
                                          int N) {
  const uint32_t id = idesc_bf16(N);
  for (int k = 0; k < K / 16; ++k) mma_bf16(tmem, sdesc(A + k * 256, K), sdesc(B + k * 256, K), id, k > 0);
}

// bias + GELU of the accumulator row of this thread into the next layer's A
// operand (K = 128, canonical layout)
__device__ __forceinline__ void hidden_rows(uint32_t trow, const float* b, unsigned char* An, int r) {
#pragma unroll 1
  for (int c0 = 0; c0 < HID; c0 += 32) {
    float v[32];
    tmem_ld32(trow + (uint32_t)c0, v);
#pragma unroll
    for (int j8 = 0; j8 < 4; ++j8) {
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = c0 + 8 * j8 + 2 * q;
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(gelu(v[8 * j8 + 2 * q] + b[c]), gelu(v[8 * j8 + 2 * q + 1] + b[c + 1]));
        pk[q] = *reinterpret_cast<const uint32_t*>(&h2);
      }
      *reinterpret_cast<uint4*>(An + coff(r, c0 + 8 * j8, HID)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  }
}

__global__ void __launch_bounds__(TTHREADS, 1)
    k_mlp_fwd_tc(const bf16* __restrict__ X, float* __restrict__ Y, const unsigned char* __restrict__ Wc, Dev w,
                 int nout, int64_t M, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  Smem& s = *reinterpret_cast<Smem*>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.taddr)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&s.bar_w, 1);
    mbar_init(&s.bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < HID; i += TTHREADS) {
    s.bias[i] = w.b1[i];
    s.bias[HID + i] = w.b2[i];
    s.bias[2 * HID + i] = w.b3[i];
  }
  if (tid < OUTP) s.bias[3 * HID + tid] = w.b4[tid];
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s.taddr;
  if (tid == 0) {
    mbar_expect_tx(&s.bar_w, WBYTES);
    bulk_g2s(s.W1, Wc, HID * INP * 2, &s.bar_w);
    bulk_g2s(s.W2, Wc + HID * INP * 2, HID * HID * 2, &s.bar_w);
    bulk_g2s(s.W3, Wc + HID * INP * 2 + HID * HID * 2, HID * HID * 2, &s.bar_w);
    bulk_g2s(s.W4, Wc + HID * INP * 2 + 2 * HID * HID * 2, OUTP * HID * 2, &s.bar_w);
  }
  bool ok = __syncthreads_and(mbar_wait(&s.bar_w, 0));
  uint32_t phase = 0;
  const int r = warp * 32 + lane;                              // this thread's row of the tile
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);  // its warp's accumulator lanes
  const int64_t ntiles = (M + TM - 1) / TM;
  const unsigned char* Wl[4] = {s.W1, s.W2, s.W3, s.W4};
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t row0 = t * TM;
    for (int i = tid; i < TM * (INP / 8); i += TTHREADS) {
      const int rr = i / (INP / 8), c = i % (INP / 8);
      int4 v = make_int4(0, 0, 0, 0);
      if (row0 + rr < M) v = reinterpret_cast<const int4*>(X + (row0 + rr) * INP)[c];
      *reinterpret_cast<int4*>(s.A0 + coff(rr, 8 * c, INP)) = v;
    }
    fence_async_smem();
    __syncthreads();
#pragma unroll 1
    for (int l = 0; l < 4; ++l) {
      const unsigned char* A = (l & 1) ? s.A1 : s.A0;
      unsigned char* An = (l & 1) ? s.A0 : s.A1;
      if (tid == 0 && ok) {
        fence_after();
        layer_mma(tmem, A, Wl[l], l == 0 ? INP : HID, l == 3 ? OUTP : HID);
        mma_commit(&s.bar_mma);
      }
      const bool done = ok ? mbar_wait(&s.bar_mma, phase) : false;
      phase ^= 1;
      ok = __syncthreads_and(done);
      fence_after();
      if (l < 3) {
        if (ok) hidden_rows(trow, s.bias + l * HID, An, r);
      } else {
        const int64_t gr = row0 + r;
        float v[32];
        if (ok) tmem_ld32(trow, v);
        if (gr < M) {
#pragma unroll
          for (int j = 0; j < OUTP; ++j)
            if (j < nout) Y[gr * nout + j] = ok ? v[j] + s.bias[3 * HID + j] : __int_as_float(0x7fc00000);
        }
      }
      fence_before();
      fence_async_smem();
      __syncthreads();
    }
  }
  if (!ok && tid == 0) *err = 1;
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// the four weight matrices, BF16, transposed ([N][K]), in the canonical
// layout of k_mlp_fwd_tc: W1 [128][96], W2, W3 [128][128], W4 [32][128]
__global__ void k_pack_tc(const float* __restrict__ theta, int nin, int nout, unsigned char* __restrict__ Wc) {
  const int oW2 = nin * HID + HID, oW3 = oW2 + HID * HID + HID, oW4 = oW3 + HID * HID + HID;
  const int n1 = HID * INP, n2 = HID * HID, n4 = OUTP * HID;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n1 + 2 * n2 + n4; t += gridDim.x * blockDim.x) {
    float v;
    unsigned char* dst;
    if (t < n1) {
      const int n = t / INP, k = t % INP;
      v = k < nin ? theta[k * HID + n] : 0.f;
      dst = Wc + coff(n, k, INP);
    } else if (t < n1 + 2 * n2) {
      const int u = (t - n1) % n2, n = u / HID, k = u % HID;
      const bool second = t >= n1 + n2;
      v = theta[(second ? oW3 : oW2) + k * HID + n];
      dst = Wc + n1 * 2 + (second ? n2 * 2 : 0) + coff(n, k, HID);
    } else {
      const int u = t - n1 - 2 * n2, n = u / HID, k = u % HID;
      v = n < nout ? theta[oW4 + k * nout + n] : 0.f;
      dst = Wc + (n1 + 2 * n2) * 2 + coff(n, k, HID);
    }
    *reinterpret_cast<bf16*>(dst) = __float2bfloat16(v);
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// line features / targets / prediction (direction-1 lines)
// ---------------------------------------------------------------------------
__global__ void k_features(const double* __restrict__ Un, const double* __restrict__ Um1,
                           const double* __restrict__ Um2, const float* __restrict__ linemet,
                           const float* __restrict__ mean, const float* __restrict__ rstd, bf16* __restrict__ X,
                           int64_t nlines, int D, int p, int nc, int npe, int nl) {
  const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlines) return;
  const int64_t e = L / nl;
  const int l = (int)(L % nl);
  const int n = p + 1;
  const int base = n * l;  // direction-1 line: node t + (p+1) l
  const int nsf = n * nc;
  bf16* x = X + L * INP;
  int f = 0;
  for (int lev = 0; lev < 3; ++lev)
    for (int t = 0; t < n; ++t)
      for (int c = 0; c < nc; ++c, ++f) {
        const int64_t idx = (e * nc + c) * npe + base + t;
        double v = lev == 0 ? Un[idx] : (lev == 1 ? Un[idx] - Um1[idx] : Um1[idx] - Um2[idx]);
        x[f] = __float2bfloat16((float)(v - mean[f]) * rstd[f]);
      }
  for (int k = 0; k < D * D; ++k, ++f) x[f] = __float2bfloat16((linemet[L * D * D + k] - mean[f]) * rstd[f]);
  for (; f < INP; ++f) x[f] = __float2bfloat16(0.f);
  (void)nsf;
}

__global__ void k_targets(const double* __restrict__ Unext, const double* __restrict__ Un,
                          const double* __restrict__ Um1, const float* __restrict__ oscale, float* __restrict__ T,
                          int64_t nlines, int p, int nc, int npe, int nl) {
  const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlines) return;
  const int64_t e = L / nl;
  const int l = (int)(L % nl), n = p + 1, base = n * l;
  for (int t = 0; t < n; ++t)
    for (int c = 0; c < nc; ++c) {
      const int64_t idx = (e * nc + c) * npe + base + t;
      const double corr = Unext[idx] - (2.0 * Un[idx] - Um1[idx]);
      T[L * (n * nc) + t * nc + c] = (float)(corr / oscale[t * nc + c]);
    }
}

__global__ void k_scatter(const float* __restrict__ Y, const double* __restrict__ Un,
                          const double* __restrict__ Um1, const float* __restrict__ oscale, double* __restrict__ U0,
                          int64_t nlines, int p, int nc, int npe, int nl) {
  const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlines) return;
  const int64_t e = L / nl;
  const int l = (int)(L % nl), n = p + 1, base = n * l;
  for (int t = 0; t < n; ++t)
    for (int c = 0; c < nc; ++c) {
      const int64_t idx = (e * nc + c) * npe + base + t;
      U0[idx] = 2.0 * Un[idx] - Um1[idx] + (double)Y[L * (n * nc) + t * nc + c] * oscale[t * nc + c];
    }
}

}  // namespace mlp
}  // namespace ldg

using namespace ldg;
using namespace ldg::mlp;

struct ldg_mlp {
  int nin = 0, nout = 0, np = 0;
  int step = 0;
  float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  bf16 *W1t = nullptr, *W2t = nullptr, *W3t = nullptr, *W4t = nullptr;
  float *b1 = nullptr, *b2 = nullptr, *b3 = nullptr, *b4 = nullptr;
  float *mean = nullptr, *rstd = nullptr, *oscale = nullptr;
  float* slots = nullptr;
  int64_t slot_cap = 0;
  unsigned char* Wc = nullptr;  // weights in the canonical layout of the tcgen05 forward
  int* err = nullptr;           // set by a forward whose waits ran out (outputs NaN)
  bf16* Xbuf = nullptr;  // prediction workspace
  float* Ybuf = nullptr;
  int64_t pred_cap = 0;
  Dev dev() const {
    Dev d;
    d.W1t = W1t;
    d.W2t = W2t;
    d.W3t = W3t;
    d.W4t = W4t;
    d.b1 = b1;
    d.b2 = b2;
    d.b3 = b3;
    d.b4 = b4;
    return d;
  }
};

static int pack(ldg_mlp_t* m, cudaStream_t st) {
  const int n = HID * LDH > HID * LDX ? HID * LDH : HID * LDX;
  k_pack<<<(n + 255) / 256, 256, 0, st>>>(m->theta, m->nin, m->nout, m->W1t, m->W2t, m->W3t, m->W4t, m->b1,
                                         m->b2, m->b3, m->b4);
  tc::k_pack_tc<<<128, 256, 0, st>>>(m->theta, m->nin, m->nout, m->Wc);
  count_launch(2);
  return cudaGetLastError() == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}

extern "C" int ldg_mlp_destroy(ldg_mlp_t* m) {
  if (!m) return LDG_OK;
  void* ptrs[] = {m->theta, m->m,  m->v,  m->grad, m->W1t, m->W2t,  m->W3t,   m->W4t, m->b1,
                  m->b2,    m->b3, m->b4, m->mean, m->rstd, m->oscale, m->slots, m->Xbuf, m->Ybuf,
                  m->Wc,    m->err};
  for (void* p : ptrs) cudaFree(p);
  delete m;
  return LDG_OK;
}

extern "C" int ldg_mlp_create(int32_t n_in, int32_t n_out, ldg_mlp_t** out) {
  if (!out || n_in < 1 || n_in > INP || n_out < 1 || n_out > OUTP) return LDG_ERR_ARG;
  ldg_mlp_t* m = new ldg_mlp_t();
  m->nin = n_in;
  m->nout = n_out;
  m->np = np_of(n_in, n_out);
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
  };
  al((void**)&m->theta, m->np * 4);
  al((void**)&m->m, m->np * 4);
  al((void**)&m->v, m->np * 4);
  al((void**)&m->grad, m->np * 4);
  al((void**)&m->W1t, HID * LDX * 2);
  al((void**)&m->W2t, HID * LDH * 2);
  al((void**)&m->W3t, HID * LDH * 2);
  al((void**)&m->W4t, OUTP * LDH * 2);
  al((void**)&m->b1, HID * 4);
  al((void**)&m->b2, HID * 4);
  al((void**)&m->b3, HID * 4);
  al((void**)&m->b4, OUTP * 4);
  al((void**)&m->mean, INP * 4);
  al((void**)&m->rstd, INP * 4);
  al((void**)&m->oscale, OUTP * 4);
  al((void**)&m->Wc, tc::WBYTES);
  al((void**)&m->err, sizeof(int));
  if (e != cudaSuccess) {
    ldg_mlp_destroy(m);
    return LDG_ERR_CUDA;
  }
  std::vector<float> ones(INP, 1.f);
  cudaMemcpy(m->rstd, ones.data(), INP * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(m->oscale, ones.data(), OUTP * 4, cudaMemcpyHostToDevice);
  *out = m;
  return LDG_OK;
}

extern "C" int ldg_mlp_params(ldg_mlp_t* m, double* theta, int32_t set) {
  if (!m || !theta) return LDG_ERR_ARG;
  std::vector<float> h(m->np);
  if (set) {
    for (int i = 0; i < m->np; ++i) h[i] = (float)theta[i];
    LDG_CUDA_TRY(cudaMemcpy(m->theta, h.data(), m->np * 4, cudaMemcpyHostToDevice));
    LDG_CUDA_TRY(cudaMemset(m->m, 0, m->np * 4));
    LDG_CUDA_TRY(cudaMemset(m->v, 0, m->np * 4));
    m->step = 0;
    if (pack(m, 0) != LDG_OK) return LDG_ERR_CUDA;
    LDG_CUDA_TRY(cudaDeviceSynchronize());
  } else {
    LDG_CUDA_TRY(cudaMemcpy(h.data(), m->theta, m->np * 4, cudaMemcpyDeviceToHost));
    for (int i = 0; i < m->np; ++i) theta[i] = h[i];
  }
  return LDG_OK;
}

extern "C" int ldg_mlp_set_scaling(ldg_mlp_t* m, const double* in_mean, const double* in_std,
                                   const double* out_scale) {
  if (!m || !in_mean || !in_std || !out_scale) return LDG_ERR_ARG;
  std::vector<float> a(INP, 0.f), b(INP, 1.f), c(OUTP, 1.f);
  for (int i = 0; i < m->nin; ++i) {
    if (!(in_std[i] > 0)) return LDG_ERR_ARG;
    a[i] = (float)in_mean[i];
    b[i] = (float)(1.0 / in_std[i]);
  }
  for (int i = 0; i < m->nout; ++i) c[i] = (float)out_scale[i];
  LDG_CUDA_TRY(cudaMemcpy(m->mean, a.data(), INP * 4, cudaMemcpyHostToDevice));
  LDG_CUDA_TRY(cudaMemcpy(m->rstd, b.data(), INP * 4, cudaMemcpyHostToDevice));
  LDG_CUDA_TRY(cudaMemcpy(m->oscale, c.data(), OUTP * 4, cudaMemcpyHostToDevice));
  return LDG_OK;
}

static cudaError_t smem_attr(const void* kern) {
  return ldg::smem_attr_cached(kern, sizeof(Smem));
}

// inference: the tcgen05 forward, one persistent CTA per SM at most
extern "C" int ldg_mlp_forward(ldg_mlp_t* m, const void* X, int64_t M, float* Y, void* stream) {
  if (!m || !X || !Y || M < 0) return LDG_ERR_ARG;
  if (M == 0) return LDG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (ldg::smem_attr_cached((const void*)tc::k_mlp_fwd_tc, sizeof(tc::Smem)) != cudaSuccess) return LDG_ERR_CUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LDG_ERR_CUDA;
  const int64_t tiles = (M + tc::TM - 1) / tc::TM;
  tc::k_mlp_fwd_tc<<<(unsigned)(tiles < sms ? tiles : sms), tc::TTHREADS, sizeof(tc::Smem), st>>>(
      (const bf16*)X, Y, m->Wc, m->dev(), m->nout, M, m->err);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}

static int grad_impl(ldg_mlp_t* m, const void* X, const float* T, int64_t M, float* grad, float* loss,
                     bool adam, double lr, double b1, double b2, double eps, cudaStream_t st) {
  if (!m || !X || !T || M <= 0) return LDG_ERR_ARG;
  const int64_t tiles = (M + TR - 1) / TR;
  const int64_t stride = ((m->np + 1 + 31) / 32) * 32;
  if (tiles * stride > m->slot_cap) {
    cudaFree(m->slots);
    m->slots = nullptr;
    m->slot_cap = 0;
    if (cudaMalloc((void**)&m->slots, tiles * stride * 4) != cudaSuccess) return LDG_ERR_CUDA;
    m->slot_cap = tiles * stride;
  }
  if (smem_attr((const void*)k_mlp<true>) != cudaSuccess) return LDG_ERR_CUDA;
  const float gscale = 2.0f / (float)((double)M * m->nout);
  k_mlp<true><<<(unsigned)tiles, THREADS, sizeof(Smem), st>>>((const bf16*)X, T, nullptr, m->dev(), m->nin,
                                                             m->nout, M, gscale, m->slots, stride);
  count_launch();
  float c1 = 1.f, c2 = 1.f;
  if (adam) {
    m->step++;
    c1 = (float)(1.0 - std::pow(b1, m->step));
    c2 = (float)(1.0 - std::pow(b2, m->step));
  }
  k_reduce_adam<<<(m->np + 256) / 256, 256, 0, st>>>(m->slots, (int)tiles, stride, m->np, grad ? grad : m->grad,
                                                    m->theta, m->m, m->v, (float)lr, (float)b1, (float)b2,
                                                    (float)eps, c1, c2, adam ? 1 : 0, loss,
                                                    (float)(1.0 / ((double)M * m->nout)));
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return LDG_ERR_CUDA;
  if (adam) return pack(m, st);
  return LDG_OK;
}

extern "C" int ldg_mlp_grad(ldg_mlp_t* m, const void* X, const float* T, int64_t M, float* grad, float* loss,
                            void* stream) {
  if (!grad) return LDG_ERR_ARG;
  return grad_impl(m, X, T, M, grad, loss, false, 0, 0.9, 0.999, 1e-8, (cudaStream_t)stream);
}

extern "C" int ldg_mlp_train_step(ldg_mlp_t* m, const void* X, const float* T, int64_t M, double lr,
                                  float* loss, void* stream) {
  return grad_impl(m, X, T, M, nullptr, loss, true, lr, 0.9, 0.999, 1e-8, (cudaStream_t)stream);
}

static int check_pred(const ldg_handle_t* h, const ldg_mlp_t* m) {
  if (!h || !m) return LDG_ERR_ARG;
  const int nin = 3 * (h->p + 1) * h->nc + h->D * h->D, nout = (h->p + 1) * h->nc;
  if (m->nin != nin || m->nout != nout) return LDG_ERR_ARG;
  return LDG_OK;
}

extern "C" int ldg_line_features(ldg_handle_t* h, const ldg_mlp_t* m, const double* Un, const double* Unm1,
                                 const double* Unm2, void* X, void* stream) {
  int rc = check_pred(h, m);
  if (rc) return rc;
  if (!Un || !Unm1 || !Unm2 || !X) return LDG_ERR_ARG;
  const int64_t nl1 = h->E * h->nl;
  k_features<<<(unsigned)((nl1 + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
      Un, Unm1, Unm2, h->linemet, m->mean, m->rstd, (bf16*)X, nl1, h->D, h->p, h->nc, h->npe, h->nl);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}

extern "C" int ldg_line_targets(ldg_handle_t* h, const ldg_mlp_t* m, const double* Unext, const double* Un,
                                const double* Unm1, float* T, void* stream) {
  int rc = check_pred(h, m);
  if (rc) return rc;
  if (!Unext || !Un || !Unm1 || !T) return LDG_ERR_ARG;
  const int64_t nl1 = h->E * h->nl;
  k_targets<<<(unsigned)((nl1 + 127) / 128), 128, 0, (cudaStream_t)stream>>>(Unext, Un, Unm1, m->oscale, T, nl1,
                                                                             h->p, h->nc, h->npe, h->nl);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}

extern "C" int ldg_mlp_predict(ldg_handle_t* h, ldg_mlp_t* m, const double* Un, const double* Unm1,
                               const double* Unm2, double* U0, void* stream) {
  int rc = check_pred(h, m);
  if (rc) return rc;
  if (!U0) return LDG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nl1 = h->E * h->nl;
  if (nl1 > m->pred_cap) {
    cudaFree(m->Xbuf);
    cudaFree(m->Ybuf);
    m->Xbuf = nullptr;
    m->Ybuf = nullptr;
    m->pred_cap = 0;
    if (cudaMalloc((void**)&m->Xbuf, nl1 * INP * 2) != cudaSuccess) return LDG_ERR_CUDA;
    if (cudaMalloc((void**)&m->Ybuf, nl1 * m->nout * 4) != cudaSuccess) return LDG_ERR_CUDA;
    m->pred_cap = nl1;
  }
  rc = ldg_line_features(h, m, Un, Unm1, Unm2, m->Xbuf, st);
  if (rc) return rc;
  rc = ldg_mlp_forward(m, m->Xbuf, nl1, m->Ybuf, st);
  if (rc) return rc;
  k_scatter<<<(unsigned)((nl1 + 127) / 128), 128, 0, st>>>(m->Ybuf, Un, Unm1, m->oscale, U0, nl1, h->p, h->nc,
                                                           h->npe, h->nl);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}
