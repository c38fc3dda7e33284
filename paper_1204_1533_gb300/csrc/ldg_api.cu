// C-ABI entry points for the residual path and small device utilities.
#include <cmath>

#include "ldg_internal.h"

#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

namespace ldg {
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches += n; }

namespace {
struct KernelTimer {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;  // reusable events, two per recorded launch
  struct Rec {
    int kind;  // kernel * 2 + (vector precision FP64)
    double bytes, flops;
  };
  std::vector<Rec> recs;
};
KernelTimer g_kt;
}  // namespace

int timer_begin(int kernel, int vprec, cudaStream_t st, double bytes, double flops) {
  std::lock_guard<std::mutex> lock(g_kt.mu);
  if (!g_kt.on) return -1;
  const size_t need = 2 * (g_kt.recs.size() + 1);
  while (g_kt.pool.size() < need) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return -1;
    g_kt.pool.push_back(ev);
  }
  const int slot = (int)g_kt.recs.size();
  g_kt.recs.push_back({kernel * 2 + (vprec == LDG_PREC_FP32 ? 0 : 1), bytes, flops});
  cudaEventRecord(g_kt.pool[2 * slot], st);
  return slot;
}

void timer_end(int slot, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_kt.mu);
  if (slot >= 0 && 2 * (size_t)slot + 1 < g_kt.pool.size()) cudaEventRecord(g_kt.pool[2 * slot + 1], st);
}

// The dynamic shared-memory limit is a per-function, per-device attribute
// (its default leaves 48 KB minus the kernel's static shared memory): set it
// the first time a (kernel, device) pair is launched, and afterwards only
// when a launch asks for more than was set before.
cudaError_t smem_attr_cached(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(fn, dev);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (err == cudaSuccess) done[key] = bytes;
  return err;
}

cudaError_t residual_2d(const ldg_handle* h, const double* U, const double* Q, double* R, cudaStream_t st);
cudaError_t residual_3d(const ldg_handle* h, const double* U, const double* Q, double* R, cudaStream_t st);
cudaError_t gradient_2d(const ldg_handle* h, const double* U, const double* Qs, double* Q, cudaStream_t st);
cudaError_t gradient_3d(const ldg_handle* h, const double* U, const double* Qs, double* Q, cudaStream_t st);

bool residual_supported(int D, int p, int kind) {
  if (p < 1 || p > 4) return false;
  if (D == 2) return kind >= 0 && kind <= 3;
  if (D == 3) return kind >= 0 && kind <= 2;
  return false;
}

cudaError_t launch_gradient(const ldg_handle* h, const double* U, double* Q, cudaStream_t st) {
  return h->D == 2 ? gradient_2d(h, U, nullptr, Q, st) : gradient_3d(h, U, nullptr, Q, st);
}

cudaError_t launch_gradient_uq(const ldg_handle* h, const double* U, const double* Qs, double* Q,
                               cudaStream_t st) {
  return h->D == 2 ? gradient_2d(h, U, Qs, Q, st) : gradient_3d(h, U, Qs, Q, st);
}

cudaError_t launch_residual(const ldg_handle* h, const double* U, const double* Q, double* R,
                            cudaStream_t st) {
  return h->D == 2 ? residual_2d(h, U, Q, R, st) : residual_3d(h, U, Q, R, st);
}

// sum of squares, one partial per block, finished by a single block
__global__ void k_sumsq(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], x[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

__global__ void k_sum_parts(const double* __restrict__ part, int n, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[0] = s;
  }
}

}  // namespace ldg

using namespace ldg;

extern "C" int ldg_gradient(ldg_handle_t* h, const double* U, double* Q, void* stream) {
  if (!h || !U || !Q) return LDG_ERR_ARG;
  if (!h->viscous() || h->phys.C22 != 0.0) return LDG_ERR_UNSUPPORTED;
  return launch_gradient(h, U, Q, (cudaStream_t)stream) == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}

extern "C" int ldg_gradient_uq(ldg_handle_t* h, const double* U, const double* Qs, double* Q, void* stream) {
  if (!h || !U || !Q || (h->phys.C22 != 0.0 && !Qs) || (Qs && Qs == Q)) return LDG_ERR_ARG;
  if (!h->viscous() || (Qs && h->nc != 1)) return LDG_ERR_UNSUPPORTED;
  return launch_gradient_uq(h, U, Qs, Q, (cudaStream_t)stream) == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}

extern "C" int ldg_residual_uq(ldg_handle_t* h, const double* U, const double* Q, double* R,
                               void* stream) {
  if (!h || !U || !R || (h->viscous() && !Q)) return LDG_ERR_ARG;
  return launch_residual(h, U, Q, R, (cudaStream_t)stream) == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}

extern "C" int ldg_residual(ldg_handle_t* h, const double* U, double* R, void* stream) {
  if (!h || !U || !R) return LDG_ERR_ARG;
  if (h->phys.C22 != 0.0) return LDG_ERR_UNSUPPORTED;  // D depends on Q: ldg_coupled_solve
  cudaStream_t st = (cudaStream_t)stream;
  if (h->viscous() && launch_gradient(h, U, h->Qbuf, st) != cudaSuccess) return LDG_ERR_CUDA;
  return launch_residual(h, U, h->viscous() ? h->Qbuf : nullptr, R, st) == cudaSuccess
             ? LDG_OK
             : LDG_ERR_CUDA;
}

extern "C" int ldg_norm2(ldg_handle_t* h, const double* x, int64_t n, double* out, void* stream) {
  if (!h || !x || !out || n < 0) return LDG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = 1024;
  k_sumsq<<<blocks, 256, 0, st>>>(x, n, h->red);
  k_sum_parts<<<1, 1024, 0, st>>>(h->red, blocks, h->red + blocks);
  count_launch(2);
  double s = 0.0;
  LDG_CUDA_TRY(cudaMemcpyAsync(&s, h->red + blocks, sizeof(double), cudaMemcpyDeviceToHost, st));
  LDG_CUDA_TRY(cudaStreamSynchronize(st));
  if (!std::isfinite(s)) return LDG_ERR_NONFINITE;
  *out = std::sqrt(s);
  return LDG_OK;
}

extern "C" int ldg_launch_count(long long* out) {
  if (!out) return LDG_ERR_ARG;
  *out = ldg::g_launches.load();
  return LDG_OK;
}

extern "C" int ldg_kernel_timer(int enable) {
  std::lock_guard<std::mutex> lock(ldg::g_kt.mu);
  ldg::g_kt.on = enable != 0;
  ldg::g_kt.recs.clear();
  return LDG_OK;
}

extern "C" int ldg_kernel_timer_read(int kernel, int prec, long long* launches, double* ms, double* bytes,
                                     double* flops) {
  if (kernel < 0 || kernel >= ldg::KT_COUNT || (prec != LDG_PREC_FP32 && prec != LDG_PREC_FP64) || !launches ||
      !ms)
    return LDG_ERR_ARG;
  std::lock_guard<std::mutex> lock(ldg::g_kt.mu);
  const int want = kernel * 2 + (prec == LDG_PREC_FP32 ? 0 : 1);
  long long n = 0;
  double tot = 0.0, by = 0.0, fl = 0.0;
  for (size_t k = 0; k < ldg::g_kt.recs.size(); ++k) {
    if (ldg::g_kt.recs[k].kind != want) continue;
    cudaEvent_t a = ldg::g_kt.pool[2 * k], b = ldg::g_kt.pool[2 * k + 1];
    if (cudaEventSynchronize(b) != cudaSuccess) return LDG_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, a, b) != cudaSuccess) return LDG_ERR_CUDA;
    tot += t;
    by += ldg::g_kt.recs[k].bytes;
    fl += ldg::g_kt.recs[k].flops;
    ++n;
  }
  *launches = n;
  *ms = tot;
  if (bytes) *bytes = by;
  if (flops) *flops = fl;
  return LDG_OK;
}
