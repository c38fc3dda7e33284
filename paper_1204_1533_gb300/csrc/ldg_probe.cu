// FP64 fused multiply-add throughput of the current device (benchmark
// instrumentation; the paper has no counterpart). On this part the FP64 pipe
// is narrow, so the residual, the FP64 ILU(0) apply, the FP64 matvec and the
// FP64 Gram-Schmidt sweeps are bound by FP64 arithmetic, not by memory: their
// roofline needs the FP64 rate the device actually sustains, which this
// kernel measures. Every thread runs PROBE_CHAINS independent chains
// x <- x a + b (no memory traffic inside the loop), four blocks of 256
// threads per SM, and writes one value per block so nothing is dead code.
#include "ldg_internal.h"

namespace ldg {

constexpr int PROBE_CHAINS = 16;
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 4;

__global__ void __launch_bounds__(PROBE_THREADS) k_fp64_fma_probe(int iters, double a, double b,
                                                                  double* __restrict__ sink) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = 1e-3 * (double)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[PROBE_THREADS / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < PROBE_THREADS / 32; ++w) t += ws[w];
    sink[blockIdx.x] = t;
  }
}

}  // namespace ldg

using namespace ldg;

extern "C" int ldg_fp64_fma_probe(int32_t iters, double* sink, int64_t sink_len, double* fmas, void* stream) {
  if (iters < 1 || !sink || !fmas) return LDG_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LDG_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LDG_ERR_CUDA;
  const int64_t blocks = (int64_t)sms * PROBE_BLOCKS_PER_SM;
  if (sink_len < blocks) return LDG_ERR_ARG;
  // a = 1 - 2^-20, b = 2^-30: the chains stay bounded and never denormal
  k_fp64_fma_probe<<<(unsigned)blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(iters, 1.0 - 0x1p-20, 0x1p-30,
                                                                                  sink);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return LDG_ERR_CUDA;
  *fmas = (double)blocks * PROBE_THREADS * PROBE_CHAINS * (double)iters;
  return LDG_OK;
}
