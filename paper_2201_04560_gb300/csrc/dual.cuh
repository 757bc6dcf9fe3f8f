// Forward-mode (tangent-linear) numbers for the sensitivity step: value v and the derivative
// d of v with respect to one model parameter (sigma of Eq. S or kappa of Eq. Q). Running the
// fused step on this type advances the state and its tangent together, so
// d(state)/d(parameter) after n steps is exact to rounding (no tape, no checkpoints).
// Dual carries FP64 values and derivatives, DualF FP32 ones (the FP32 step's arithmetic;
// its domain sums stay FP64).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

// The type and its overloads live in their own namespace and are found by argument-dependent
// lookup, so that they never hide the float/double math functions of code that also
// instantiates the step for plain types.
namespace ppl_dual {

template <typename T>
struct alignas(2 * sizeof(T)) DualT {
  T v, d;
  DualT() = default;
  // one constructor from double for both widths: literals and FP64 sums convert without
  // ambiguity, and a float argument passes through double exactly
  __host__ __device__ constexpr DualT(double x) : v(static_cast<T>(x)), d(T(0)) {}
  __host__ __device__ constexpr DualT(double x, double dx) : v(static_cast<T>(x)), d(static_cast<T>(dx)) {}
  __host__ __device__ explicit operator double() const { return (double)v; }
};

using Dual = DualT<double>;
using DualF = DualT<float>;

template <typename T>
__host__ __device__ __forceinline__ DualT<T> make(T v, T d) {
  DualT<T> r;
  r.v = v;
  r.d = d;
  return r;
}

template <typename T>
__host__ __device__ __forceinline__ DualT<T> operator+(DualT<T> a, DualT<T> b) { return make(a.v + b.v, a.d + b.d); }
template <typename T>
__host__ __device__ __forceinline__ DualT<T> operator-(DualT<T> a, DualT<T> b) { return make(a.v - b.v, a.d - b.d); }
template <typename T>
__host__ __device__ __forceinline__ DualT<T> operator-(DualT<T> a) { return make(-a.v, -a.d); }
template <typename T>
__host__ __device__ __forceinline__ DualT<T> operator*(DualT<T> a, DualT<T> b) {
  return make(a.v * b.v, a.d * b.v + a.v * b.d);
}
template <typename T>
__host__ __device__ __forceinline__ DualT<T> operator/(DualT<T> a, DualT<T> b) {
  const T q = a.v / b.v;
  return make(q, (a.d - q * b.d) / b.v);
}
// mixed forms: a plain number is a constant (zero derivative)
#define PPL_DUAL_MIXED(op)                                                                               \
  template <typename T>                                                                                  \
  __host__ __device__ __forceinline__ DualT<T> operator op(DualT<T> a, double b) { return a op DualT<T>(b); } \
  template <typename T>                                                                                  \
  __host__ __device__ __forceinline__ DualT<T> operator op(double a, DualT<T> b) { return DualT<T>(a) op b; }
PPL_DUAL_MIXED(+)
PPL_DUAL_MIXED(-)
PPL_DUAL_MIXED(*)
PPL_DUAL_MIXED(/)
#undef PPL_DUAL_MIXED
template <typename T>
__host__ __device__ __forceinline__ DualT<T> &operator+=(DualT<T> &a, DualT<T> b) { return a = a + b; }
template <typename T>
__host__ __device__ __forceinline__ DualT<T> &operator-=(DualT<T> &a, DualT<T> b) { return a = a - b; }
template <typename T>
__host__ __device__ __forceinline__ DualT<T> &operator*=(DualT<T> &a, DualT<T> b) { return a = a * b; }
// comparisons act on values (branches of the step are taken on the primal state)
template <typename T>
__host__ __device__ __forceinline__ bool operator<(DualT<T> a, DualT<T> b) { return a.v < b.v; }
template <typename T>
__host__ __device__ __forceinline__ bool operator>(DualT<T> a, DualT<T> b) { return a.v > b.v; }
template <typename T>
__host__ __device__ __forceinline__ bool operator<=(DualT<T> a, DualT<T> b) { return a.v <= b.v; }
template <typename T>
__host__ __device__ __forceinline__ bool operator>=(DualT<T> a, DualT<T> b) { return a.v >= b.v; }
template <typename T>
__host__ __device__ __forceinline__ bool operator==(DualT<T> a, DualT<T> b) { return a.v == b.v; }
template <typename T>
__host__ __device__ __forceinline__ bool operator!=(DualT<T> a, DualT<T> b) { return a.v != b.v; }

template <typename T>
__device__ __forceinline__ DualT<T> sqrt(DualT<T> a) {
  const T r = ::sqrt(a.v);
  return make(r, r > T(0) ? T(0.5) * a.d / r : T(0));
}
template <typename T>
__device__ __forceinline__ DualT<T> fabs(DualT<T> a) { return a.v < T(0) ? -a : a; }
template <typename T>
__device__ __forceinline__ DualT<T> fmax(DualT<T> a, DualT<T> b) { return a.v >= b.v ? a : b; }
template <typename T>
__device__ __forceinline__ DualT<T> fmin(DualT<T> a, DualT<T> b) { return a.v <= b.v ? a : b; }

}  // namespace ppl_dual

namespace ppl_dev {

using ppl_dual::Dual;
using ppl_dual::DualF;

template <typename T>
struct is_dual : std::false_type {};
template <typename T>
struct is_dual<ppl_dual::DualT<T>> : std::true_type {};

template <typename T>
__host__ __device__ __forceinline__ double value_of(T x) {
  return (double)x;
}
template <typename T>
__host__ __device__ __forceinline__ double tangent_of(T) {
  return 0.0;
}
template <typename T>
__host__ __device__ __forceinline__ double tangent_of(ppl_dual::DualT<T> x) {
  return (double)x.d;
}

}  // namespace ppl_dev
