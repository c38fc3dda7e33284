// Forward-mode dual numbers for the Jacobian kernels: a value and N partial
// derivatives carried through the pointwise flux code. Branches on |x| and
// max() follow the value, as for the non-smooth points of the Roe flux.
#pragma once
#include <math.h>

namespace ldg {

template <typename R, int N>
struct Dual {
  R v;
  R d[N];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(double x) : v(R(x)) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = R(0);
  }
  __device__ __forceinline__ Dual(float x) : v(R(x)) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = R(0);
  }
};

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ float val(float x) { return x; }
template <typename R, int N>
__device__ __forceinline__ R val(const Dual<R, N>& x) { return x.v; }

__device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
__device__ __forceinline__ float sqrt(float x) { return ::sqrtf(x); }
__device__ __forceinline__ double dabs(double x) { return fabs(x); }
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }

#define LDG_DUAL template <typename R, int N> __device__ __forceinline__ Dual<R, N>

LDG_DUAL operator+(const Dual<R, N>& a, const Dual<R, N>& b) {
  Dual<R, N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
LDG_DUAL operator-(const Dual<R, N>& a, const Dual<R, N>& b) {
  Dual<R, N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
LDG_DUAL operator-(const Dual<R, N>& a) {
  Dual<R, N> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
LDG_DUAL operator*(const Dual<R, N>& a, const Dual<R, N>& b) {
  Dual<R, N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.v * b.d[i] + b.v * a.d[i];
  return r;
}
LDG_DUAL operator/(const Dual<R, N>& a, const Dual<R, N>& b) {
  Dual<R, N> r;
  R inv = R(1) / b.v;
  r.v = a.v * inv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
  return r;
}
// mixed with the real type
LDG_DUAL operator+(const Dual<R, N>& a, R b) {
  Dual<R, N> r = a;
  r.v += b;
  return r;
}
LDG_DUAL operator+(R b, const Dual<R, N>& a) { return a + b; }
LDG_DUAL operator-(const Dual<R, N>& a, R b) {
  Dual<R, N> r = a;
  r.v -= b;
  return r;
}
LDG_DUAL operator-(R b, const Dual<R, N>& a) {
  Dual<R, N> r;
  r.v = b - a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
LDG_DUAL operator*(const Dual<R, N>& a, R b) {
  Dual<R, N> r;
  r.v = a.v * b;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
LDG_DUAL operator*(R b, const Dual<R, N>& a) { return a * b; }
LDG_DUAL operator/(const Dual<R, N>& a, R b) {
  R inv = R(1) / b;
  return a * inv;
}
LDG_DUAL sqrt(const Dual<R, N>& a) {
  Dual<R, N> r;
  r.v = sqrt(a.v);
  R h = R(0.5) / r.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * h;
  return r;
}
LDG_DUAL dabs(const Dual<R, N>& a) { return (a.v >= R(0)) ? a : -a; }
#undef LDG_DUAL

}  // namespace ldg
