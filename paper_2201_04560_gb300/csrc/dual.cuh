// Forward-mode (tangent-linear) FP64 number for the sensitivity step: value v and the
// derivative d of v with respect to one model parameter (sigma of Eq. S or kappa of Eq. Q).
// Running the fused step on this type advances the state and its tangent together, so
// d(state)/d(parameter) after n steps is exact to rounding (no tape, no checkpoints).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

// The type and its overloads live in their own namespace and are found by argument-dependent
// lookup, so that they never hide the float/double math functions of code that also
// instantiates the step for plain types.
namespace ppl_dual {

struct __align__(16) Dual {
  double v, d;
  Dual() = default;
  __host__ __device__ constexpr Dual(double x) : v(x), d(0.0) {}
  __host__ __device__ constexpr Dual(double x, double dx) : v(x), d(dx) {}
  __host__ __device__ explicit operator double() const { return v; }
};

__host__ __device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__host__ __device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__host__ __device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__host__ __device__ __forceinline__ Dual &operator+=(Dual &a, Dual b) { return a = a + b; }
__host__ __device__ __forceinline__ Dual &operator-=(Dual &a, Dual b) { return a = a - b; }
__host__ __device__ __forceinline__ Dual &operator*=(Dual &a, Dual b) { return a = a * b; }
// comparisons act on values (branches of the step are taken on the primal state)
__host__ __device__ __forceinline__ bool operator<(Dual a, Dual b) { return a.v < b.v; }
__host__ __device__ __forceinline__ bool operator>(Dual a, Dual b) { return a.v > b.v; }
__host__ __device__ __forceinline__ bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
__host__ __device__ __forceinline__ bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
__host__ __device__ __forceinline__ bool operator==(Dual a, Dual b) { return a.v == b.v; }
__host__ __device__ __forceinline__ bool operator!=(Dual a, Dual b) { return a.v != b.v; }

__device__ __forceinline__ Dual sqrt(Dual a) {
  const double r = ::sqrt(a.v);
  return Dual(r, r > 0.0 ? 0.5 * a.d / r : 0.0);
}
__device__ __forceinline__ Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }
__device__ __forceinline__ Dual fmax(Dual a, Dual b) { return a.v >= b.v ? a : b; }
__device__ __forceinline__ Dual fmin(Dual a, Dual b) { return a.v <= b.v ? a : b; }

}  // namespace ppl_dual

namespace ppl_dev {

using ppl_dual::Dual;

template <typename T>
struct is_dual : std::false_type {};
template <>
struct is_dual<Dual> : std::true_type {};

template <typename T>
__host__ __device__ __forceinline__ double value_of(T x) {
  return (double)x;
}
template <typename T>
__host__ __device__ __forceinline__ double tangent_of(T) {
  return 0.0;
}
template <>
__host__ __device__ __forceinline__ double tangent_of<Dual>(Dual x) {
  return x.d;
}

}  // namespace ppl_dev
