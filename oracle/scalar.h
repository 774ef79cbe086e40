// Scalar types for the CPU oracle.
//
// TEST INFRASTRUCTURE ONLY: the oracle is a plain, slow FP64 restatement of the
// method used to check the CUDA path; no product code may call it.
//
// Every routine of the oracle is written once, templated on its scalar type S:
//   double    -- plain values (rollouts, pins)
//   Dual<T>   -- forward-mode derivative (value + one tangent) used for the
//                Jacobians of the right-hand side and of one integrator step
//   Cnt       -- a double that counts floating-point operations
//                (add/sub/mul/div/sqrt = 1, transcendental = 1) so that the
//                algorithmic work per environment step can be reported.
#pragma once
#include <cmath>
#include <cstdint>

namespace orc {

// ---------------------------------------------------------------- Cnt
extern thread_local std::int64_t g_flops;
// While > 0, operations are not counted (used to leave the constraint solver's
// active-set search out of the algorithmic count; see solve_constraints).
extern thread_local int g_flops_paused;
// While alive, operations are not counted: arithmetic on model constants
// alone (values that a compiled model holds precomputed), which is not
// per-step work of the method.
struct FlopsPaused {
  FlopsPaused() { ++g_flops_paused; }
  ~FlopsPaused() { --g_flops_paused; }
  FlopsPaused(const FlopsPaused&) = delete;
  FlopsPaused& operator=(const FlopsPaused&) = delete;
};
// 1: count the active-set search from the unconstrained acceleration too.
extern thread_local int g_count_search;

struct Cnt {
  double v;
  Cnt() : v(0) {}
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { g_flops += !g_flops_paused; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_flops += !g_flops_paused; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_flops += !g_flops_paused; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_flops += !g_flops_paused; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt sqrt(Cnt a) { g_flops += !g_flops_paused; return Cnt(std::sqrt(a.v)); }
inline Cnt sin(Cnt a) { g_flops += !g_flops_paused; return Cnt(std::sin(a.v)); }
inline Cnt cos(Cnt a) { g_flops += !g_flops_paused; return Cnt(std::cos(a.v)); }
inline Cnt exp(Cnt a) { g_flops += !g_flops_paused; return Cnt(std::exp(a.v)); }
inline Cnt log1p(Cnt a) { g_flops += !g_flops_paused; return Cnt(std::log1p(a.v)); }
inline Cnt pow(Cnt a, double p) { g_flops += !g_flops_paused; return Cnt(std::pow(a.v, p)); }
inline Cnt fabs(Cnt a) { return Cnt(std::fabs(a.v)); }

// ---------------------------------------------------------------- Dual
template <class T>
struct Dual {
  T v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(const T& a, const T& b) : v(a), d(b) {}
};
template <class T> inline Dual<T> operator+(const Dual<T>& a, const Dual<T>& b) { return {a.v + b.v, a.d + b.d}; }
template <class T> inline Dual<T> operator-(const Dual<T>& a, const Dual<T>& b) { return {a.v - b.v, a.d - b.d}; }
template <class T> inline Dual<T> operator*(const Dual<T>& a, const Dual<T>& b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T> inline Dual<T> operator/(const Dual<T>& a, const Dual<T>& b) {
  T q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
template <class T> inline Dual<T> operator-(const Dual<T>& a) { return {-a.v, -a.d}; }
template <class T> inline Dual<T> operator+(const Dual<T>& a, double b) { return {a.v + b, a.d}; }
template <class T> inline Dual<T> operator+(double b, const Dual<T>& a) { return {a.v + b, a.d}; }
template <class T> inline Dual<T> operator-(const Dual<T>& a, double b) { return {a.v - b, a.d}; }
template <class T> inline Dual<T> operator-(double b, const Dual<T>& a) { return {b - a.v, -a.d}; }
template <class T> inline Dual<T> operator*(const Dual<T>& a, double b) { return {a.v * b, a.d * b}; }
template <class T> inline Dual<T> operator*(double b, const Dual<T>& a) { return {a.v * b, a.d * b}; }
template <class T> inline Dual<T> operator/(const Dual<T>& a, double b) { return {a.v / b, a.d / b}; }
template <class T> inline Dual<T> operator/(double b, const Dual<T>& a) { return Dual<T>(b) / a; }
using std::sqrt; using std::sin; using std::cos; using std::exp; using std::log1p; using std::pow; using std::fabs;
template <class T> inline Dual<T> sqrt(const Dual<T>& a) { T s = sqrt(a.v); return {s, a.d / (s + s)}; }
template <class T> inline Dual<T> sin(const Dual<T>& a) { return {sin(a.v), a.d * cos(a.v)}; }
template <class T> inline Dual<T> cos(const Dual<T>& a) { return {cos(a.v), -(a.d * sin(a.v))}; }
template <class T> inline Dual<T> exp(const Dual<T>& a) { T e = exp(a.v); return {e, a.d * e}; }
template <class T> inline Dual<T> log1p(const Dual<T>& a) { return {log1p(a.v), a.d / (T(1.0) + a.v)}; }
template <class T> inline Dual<T> pow(const Dual<T>& a, double p) {
  return {pow(a.v, p), a.d * (p * pow(a.v, p - 1.0))};
}
template <class T> inline Dual<T> fabs(const Dual<T>& a);

// ---------------------------------------------------------------- primal value
inline double val(double x) { return x; }
inline double val(const Cnt& x) { return x.v; }
template <class T> inline double val(const Dual<T>& x) { return val(x.v); }

template <class T> inline Dual<T> fabs(const Dual<T>& a) { return val(a) < 0 ? -a : a; }

// The scalar in which the Newton search (a sequence of discrete decisions) runs:
// the value type for Dual, the type itself otherwise.
template <class S> struct PrimalOf { using type = S; };
template <class T> struct PrimalOf<Dual<T>> { using type = double; };

template <class S> inline S smin(const S& a, const S& b) { return val(a) <= val(b) ? a : b; }
template <class S> inline S smax(const S& a, const S& b) { return val(a) >= val(b) ? a : b; }

}  // namespace orc
