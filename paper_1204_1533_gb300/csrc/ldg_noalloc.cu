// ldg_residual_noalloc: the residual of ldg_residual without any allocation.
//
// For second-order equations the residual needs the LDG gradient Q = D(U)
// as scratch between its two kernels. ldg_residual keeps it in a buffer the
// handle allocated; this entry point keeps it in the file-scope device array
// below instead, so a call never allocates device memory, for callers that
// must not call cudaMalloc after start-up (their device memory is owned by
// another allocator, or their run loop is forbidden to allocate).
//
// The array is part of the library image: every GPU that loads the library
// holds LDG_NOALLOC_MAX_Q doubles (8 MiB) until the process exits. Host code
// may not use the array's name as a device address, so the first call on
// each device looks up its address with cudaGetSymbolAddress (with that
// device current) and caches it. All calls share the array: calls whose
// work overlaps on the GPU (different streams, or different handles on the
// same device) race on it. The gradient kernel writes every entry it later
// reads, so nothing needs clearing between calls.
#include <mutex>

#include "ldg_internal.h"

namespace {

constexpr int kMaxDevices = 64;
__device__ __align__(256) double g_qscratch[LDG_NOALLOC_MAX_Q];
std::mutex g_mutex;
double* g_qaddr[kMaxDevices] = {};

// device address of g_qscratch on the current device (set up once per device)
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LDG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_qaddr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_qscratch) != cudaSuccess || !p) return LDG_ERR_CUDA;
    g_qaddr[dev] = static_cast<double*>(p);
  }
  *out = g_qaddr[dev];
  return LDG_OK;
}

}  // namespace

extern "C" int ldg_residual_noalloc(ldg_handle_t* h, const double* U, double* R, void* stream) {
  if (!h || !U || !R) return LDG_ERR_ARG;
  if (h->phys.C22 != 0.0) return LDG_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  if (!h->viscous())  // first-order equations need no scratch
    return ldg::launch_residual(h, U, nullptr, R, st) == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
  if (h->ndof * h->D > (int64_t)LDG_NOALLOC_MAX_Q) return LDG_ERR_TOO_LARGE;
  double* q = nullptr;
  const int rc = scratch_address(&q);
  if (rc != LDG_OK) return rc;
  if (ldg::launch_gradient(h, U, q, st) != cudaSuccess) return LDG_ERR_CUDA;
  return ldg::launch_residual(h, U, q, R, st) == cudaSuccess ? LDG_OK : LDG_ERR_CUDA;
}
