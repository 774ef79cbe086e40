// Forward-mode derivative scalar for the device code: value + one tangent.
//
// The adjoint kernel evaluates the right-hand side with one derivative
// direction per lane: every lane of a warp runs the same (primal) instruction
// stream, so on GB300, where an FP64 warp instruction costs the same whatever
// its active lanes, the 32 tangents of a warp come at the price of one
// evaluation.  Discrete decisions (contact inclusion, active sets, spline
// branches) are taken on values, so all lanes of a warp stay converged.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace dmx {

struct Dual {
  double v, d;
  __device__ Dual() = default;
  __device__ constexpr Dual(double x) : v(x), d(0.0) {}
  __device__ constexpr Dual(double x, double t) : v(x), d(t) {}
};

// the double versions stay visible next to the Dual overloads below
using ::exp;
using ::fabs;
using ::log1p;
using ::pow;
using ::sincos;
using ::sqrt;

__device__ __forceinline__ double value(double x) { return x; }
__device__ __forceinline__ double value(const Dual& x) { return x.v; }

__device__ __forceinline__ Dual operator+(const Dual& a, const Dual& b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(const Dual& a, const Dual& b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator*(const Dual& a, const Dual& b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(const Dual& a, const Dual& b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator+(const Dual& a, double b) { return Dual(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(double b, const Dual& a) { return Dual(a.v + b, a.d); }
__device__ __forceinline__ Dual operator-(const Dual& a, double b) { return Dual(a.v - b, a.d); }
__device__ __forceinline__ Dual operator-(double b, const Dual& a) { return Dual(b - a.v, -a.d); }
__device__ __forceinline__ Dual operator*(const Dual& a, double b) { return Dual(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator*(double b, const Dual& a) { return Dual(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator/(const Dual& a, double b) { return Dual(a.v / b, a.d / b); }
__device__ __forceinline__ Dual operator/(double b, const Dual& a) { return Dual(b) / a; }
__device__ __forceinline__ Dual& operator+=(Dual& a, const Dual& b) { a.v += b.v; a.d += b.d; return a; }
__device__ __forceinline__ Dual& operator-=(Dual& a, const Dual& b) { a.v -= b.v; a.d -= b.d; return a; }
__device__ __forceinline__ Dual& operator*=(Dual& a, const Dual& b) { a = a * b; return a; }
__device__ __forceinline__ Dual& operator*=(Dual& a, double b) { a.v *= b; a.d *= b; return a; }

__device__ __forceinline__ Dual sqrt(const Dual& a) {
  const double s = ::sqrt(a.v);
  return Dual(s, a.d / (s + s));
}
__device__ __forceinline__ void sincos(const Dual& a, Dual* s, Dual* c) {
  double sv, cv;
  ::sincos(a.v, &sv, &cv);
  *s = Dual(sv, a.d * cv);
  *c = Dual(cv, -a.d * sv);
}
__device__ __forceinline__ Dual exp(const Dual& a) {
  const double e = ::exp(a.v);
  return Dual(e, a.d * e);
}
__device__ __forceinline__ Dual log1p(const Dual& a) { return Dual(::log1p(a.v), a.d / (1.0 + a.v)); }
__device__ __forceinline__ Dual pow(const Dual& a, double p) {
  return Dual(::pow(a.v, p), a.d * (p * ::pow(a.v, p - 1.0)));
}
__device__ __forceinline__ Dual fabs(const Dual& a) { return a.v < 0 ? -a : a; }

// reciprocal square root (CUDA's double rsqrt: one rounding step instead of a
// square root and a division)
__device__ __forceinline__ double rsqrt_t(double x) { return ::rsqrt(x); }
__device__ __forceinline__ Dual rsqrt_t(const Dual& x) {
  const double r = ::rsqrt(x.v);
  return Dual(r, -0.5 * r * r * r * x.d);
}

}  // namespace dmx
