// Forward-mode dual numbers in FP32 for the power iteration of the mixed
// path.  Algorithm 5 forms v_new = f(y + q v) - f(y) with q of size ~1e-8
// relative to y, which FP32 cannot resolve; the same quantity to first order
// is q J(y) v, and evaluating f on dual numbers y + eps v gives J(y) v
// exactly up to FP32 rounding.  The power iteration then converges to the
// spectral radius of J(y), the q -> 0 limit of what Algorithm 5 estimates.
#pragma once

#include "models.cuh"

namespace emrkc {

struct Dual {
  float v, d;  // value and tangent
  __device__ __forceinline__ Dual() : v(0.0f), d(0.0f) {}
  __device__ __forceinline__ Dual(double x) : v((float)x), d(0.0f) {}  // constants of the models
  __device__ __forceinline__ Dual(float x, float dx) : v(x), d(dx) {}
};

__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const float r = __frcp_rn(b.v);
  const float q = a.v * r;
  return Dual(q, (a.d - q * b.d) * r);
}
__device__ __forceinline__ bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator<(Dual a, Dual b) { return a.v < b.v; }

template <> struct Math<Dual> {
  static __device__ __forceinline__ Dual ex(Dual x) {
    const float e = __expf(x.v);
    return Dual(e, e * x.d);
  }
  static __device__ __forceinline__ Dual em1(Dual x) { return Dual(Math<float>::em1(x.v), __expf(x.v) * x.d); }
  static __device__ __forceinline__ Dual ln(Dual x) { return Dual(__logf(x.v), x.d / x.v); }
  static __device__ __forceinline__ Dual sq(Dual x) {  // square root
    const float r = sqrtf(x.v);
    return Dual(r, 0.5f * x.d / r);
  }
  static __device__ __forceinline__ Dual dv(Dual a, Dual b) { return a / b; }
  static __device__ __forceinline__ Dual ex_aff(Dual x, double c, double s) { return ex((x - Dual(c)) * Dual(s)); }
  // g(x) = x / (e^x - 1), g'(x) = (e^x - 1 - x e^x) / (e^x - 1)^2 (-1/2 + x/6 near 0)
  static __device__ __forceinline__ Dual x_em1(Dual x) {
    const float g = Math<float>::x_em1(x.v);
    float dg;
    if (fabsf(x.v) < 1e-3f) {
      dg = -0.5f + x.v * (1.0f / 6.0f);
    } else {
      const float em = Math<float>::em1(x.v);
      dg = (em - x.v * (em + 1.0f)) / (em * em);
    }
    return Dual(g, dg * x.d);
  }
};

}  // namespace emrkc
