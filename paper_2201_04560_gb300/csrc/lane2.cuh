// Two FP32 lanes (two adjacent columns of the row-marching step) computed with the packed
// f32x2 instructions of sm_100+ (one FMA/ADD/MUL instruction for both lanes).
//
// Products are kept pending (Mul2) so that a product followed by an addition becomes one
// fused multiply-add, as the compiler contracts the scalar code. The packed instructions
// take no negated operand, so a difference is one packed subtraction (sub.rn.f32x2, written
// out below) and a product is subtracted after rounding unless its first factor is a
// constant that the compiler negates. Division and square root act lane by lane.
#pragma once

#include <cuda_runtime.h>

// The type and its overloads live in their own namespace and are found by argument-dependent
// lookup, so that they never hide the float math functions of the scalar code.
namespace ppl_lane {

struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ F2(float a) : v(make_float2(a, a)) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit F2(float2 x) : v(x) {}
  __device__ __forceinline__ float lo() const { return v.x; }
  __device__ __forceinline__ float hi() const { return v.y; }
};

struct Mul2 {  // a * b, not yet rounded
  float2 a, b;
  __device__ __forceinline__ operator F2() const { return F2(__fmul2_rn(a, b)); }
};

__device__ __forceinline__ float2 neg2(float2 x) { return make_float2(-x.x, -x.y); }
// a - b in one packed instruction (PTX sub.f32x2, sm_100+)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n sub.rn.f32x2 rd, ra, rb;\n"
      " mov.b64 {%0, %1}, rd;\n}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ F2 ev(F2 x) { return x; }
__device__ __forceinline__ F2 ev(Mul2 m) { return F2(__fmul2_rn(m.a, m.b)); }

// products
__device__ __forceinline__ Mul2 operator*(F2 a, F2 b) { return Mul2{a.v, b.v}; }
__device__ __forceinline__ Mul2 operator*(float s, F2 b) { return Mul2{make_float2(s, s), b.v}; }
__device__ __forceinline__ Mul2 operator*(F2 a, float s) { return Mul2{a.v, make_float2(s, s)}; }
__device__ __forceinline__ Mul2 operator*(Mul2 m, F2 b) { return Mul2{ev(m).v, b.v}; }
__device__ __forceinline__ Mul2 operator*(F2 a, Mul2 m) { return Mul2{a.v, ev(m).v}; }
__device__ __forceinline__ Mul2 operator*(Mul2 m, float s) { return Mul2{ev(m).v, make_float2(s, s)}; }
__device__ __forceinline__ Mul2 operator*(float s, Mul2 m) { return Mul2{make_float2(s, s), ev(m).v}; }
__device__ __forceinline__ Mul2 operator*(Mul2 m, Mul2 n) { return Mul2{ev(m).v, ev(n).v}; }

// sums: a pending product fuses with the other operand
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator+(Mul2 m, F2 c) { return F2(__ffma2_rn(m.a, m.b, c.v)); }
__device__ __forceinline__ F2 operator+(F2 c, Mul2 m) { return F2(__ffma2_rn(m.a, m.b, c.v)); }
__device__ __forceinline__ F2 operator+(Mul2 m, Mul2 n) { return F2(__ffma2_rn(m.a, m.b, ev(n).v)); }
__device__ __forceinline__ F2 operator+(F2 a, float s) { return a + F2(s); }
__device__ __forceinline__ F2 operator+(float s, F2 a) { return a + F2(s); }
__device__ __forceinline__ F2 operator+(Mul2 m, float s) { return m + F2(s); }
__device__ __forceinline__ F2 operator+(float s, Mul2 m) { return m + F2(s); }

__device__ __forceinline__ F2 operator-(F2 a) { return F2(sub2(make_float2(0.0f, 0.0f), a.v)); }
__device__ __forceinline__ Mul2 operator-(Mul2 m) { return Mul2{neg2(m.a), m.b}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(sub2(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(Mul2 m, F2 c) { return F2(sub2(ev(m).v, c.v)); }
__device__ __forceinline__ F2 operator-(F2 c, Mul2 m) { return F2(__ffma2_rn(neg2(m.a), m.b, c.v)); }
__device__ __forceinline__ F2 operator-(Mul2 m, Mul2 n) { return F2(sub2(ev(m).v, ev(n).v)); }
__device__ __forceinline__ F2 operator-(F2 a, float s) { return a - F2(s); }
__device__ __forceinline__ F2 operator-(float s, F2 a) { return F2(s) - a; }
__device__ __forceinline__ F2 operator-(Mul2 m, float s) { return m - F2(s); }
__device__ __forceinline__ F2 operator-(float s, Mul2 m) { return F2(s) - m; }

__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2 &operator+=(F2 &a, Mul2 m) { return a = a + m; }
__device__ __forceinline__ F2 &operator-=(F2 &a, F2 b) { return a = a - b; }

// lane-wise division and square root (the scalar forms of the FP32 build)
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ F2 operator/(Mul2 a, F2 b) { return ev(a) / b; }
__device__ __forceinline__ F2 operator/(F2 a, Mul2 b) { return a / ev(b); }
__device__ __forceinline__ F2 operator/(Mul2 a, Mul2 b) { return ev(a) / ev(b); }
__device__ __forceinline__ F2 operator/(float s, F2 b) { return F2(s / b.v.x, s / b.v.y); }
__device__ __forceinline__ F2 operator/(float s, Mul2 b) { return s / ev(b); }
__device__ __forceinline__ F2 sqrt(F2 a) { return F2(sqrtf(a.v.x), sqrtf(a.v.y)); }
__device__ __forceinline__ F2 sqrt(Mul2 a) { return sqrt(ev(a)); }
__device__ __forceinline__ F2 fmax(F2 a, F2 b) { return F2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }

}  // namespace ppl_lane

namespace ppl_dev {
using ppl_lane::F2;
}  // namespace ppl_dev
