// Forward-mode dual numbers for the force kernel: a value and K tangent
// components, propagated through every arithmetic operation by the chain
// rule (d(uv) = u dv + v du, d(u/v) = (du - (u/v) dv)/v, d exp(u) = exp(u) du,
// d log|u| = du / u, d sqrt(u) = du / (2 sqrt(u))).  Seeding the nuclear
// coordinates with unit tangents makes every tangent of E_L a derivative
// with respect to a nuclear coordinate.
#pragma once

#include <cmath>

namespace qmc {

// keep the scalar overloads visible next to the dual ones below
using ::exp;
using ::sqrt;

template <int K>
struct Dual {
  double v;
  double d[K];
  __device__ __forceinline__ Dual() : v(0.0) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = 0.0;
  }
  __device__ __forceinline__ Dual(double x) : v(x) {  // NOLINT: constants promote implicitly
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = 0.0;
  }
  __device__ __forceinline__ Dual& operator+=(const Dual& o) {
    v += o.v;
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] += o.d[k];
    return *this;
  }
  __device__ __forceinline__ Dual& operator+=(double o) {  // a constant: the tangents stay
    v += o;
    return *this;
  }
  __device__ __forceinline__ Dual& operator-=(const Dual& o) {
    v -= o.v;
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] -= o.d[k];
    return *this;
  }
  __device__ __forceinline__ Dual& operator*=(const Dual& o) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = d[k] * o.v + v * o.d[k];
    v *= o.v;
    return *this;
  }
};

template <int K>
__device__ __forceinline__ Dual<K> operator+(Dual<K> a, const Dual<K>& b) { return a += b; }
template <int K>
__device__ __forceinline__ Dual<K> operator-(Dual<K> a, const Dual<K>& b) { return a -= b; }
template <int K>
__device__ __forceinline__ Dual<K> operator*(Dual<K> a, const Dual<K>& b) { return a *= b; }
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
// mixed double / Dual operations
template <int K>
__device__ __forceinline__ Dual<K> operator+(const Dual<K>& a, double b) { Dual<K> r = a; r.v += b; return r; }
template <int K>
__device__ __forceinline__ Dual<K> operator+(double b, const Dual<K>& a) { return a + b; }
template <int K>
__device__ __forceinline__ Dual<K> operator-(const Dual<K>& a, double b) { Dual<K> r = a; r.v -= b; return r; }
template <int K>
__device__ __forceinline__ Dual<K> operator-(double b, const Dual<K>& a) { return -(a - b); }
template <int K>
__device__ __forceinline__ Dual<K> operator*(const Dual<K>& a, double b) {
  Dual<K> r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> operator*(double b, const Dual<K>& a) { return a * b; }
template <int K>
__device__ __forceinline__ Dual<K> operator/(const Dual<K>& a, double b) { return a * (1.0 / b); }
template <int K>
__device__ __forceinline__ Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }

template <int K>
__device__ __forceinline__ Dual<K> exp(const Dual<K>& a) {
  Dual<K> r;
  r.v = ::exp(a.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = r.v * a.d[k];
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> sqrt(const Dual<K>& a) {
  Dual<K> r;
  r.v = ::sqrt(a.v);
  const double h = 0.5 / r.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * h;
  return r;
}
template <int K>
__device__ __forceinline__ Dual<K> log_abs(const Dual<K>& a) {
  Dual<K> r;
  r.v = ::log(::fabs(a.v));
  const double ia = 1.0 / a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * ia;
  return r;
}

__device__ __forceinline__ double log_abs(double a) { return ::log(::fabs(a)); }
__device__ __forceinline__ double value_of(double a) { return a; }
template <int K>
__device__ __forceinline__ double value_of(const Dual<K>& a) { return a.v; }

}  // namespace qmc
