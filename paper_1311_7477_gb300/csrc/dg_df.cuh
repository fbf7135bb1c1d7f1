// Double-float arithmetic on the float32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2: about 48
// bits of significand, with the exponent range of float32.  The operations are built from two
// error-free transformations,
//   TwoSum     s + e = a + b exactly, s = fl(a + b)        (Knuth, TAOCP vol. 2, Sec. 4.2.2)
//   TwoProduct p + e = a * b exactly, p = fl(a * b),
//              e = fma(a, b, -p)                           (Dekker 1971, in its FMA form)
// in the style of Dekker's add2 and mul2 (1971): the sum adds the low parts in plain float32,
// so its ABSOLUTE error is bounded by a few eps32^2 (|a| + |b|) --
// the bound that matters here, where large terms cancel -- while its relative error is not
// bounded under cancellation.  Every step is an explicit round-to-nearest intrinsic or fmaf,
// so no compiler contraction changes the result.
//
// Two symmetries are kept exactly (they give the bracket's J(f, f) = 0 bitwise):
//   a * b == b * a   (the two cross terms are rounded separately and added: commutative)
//   a - b == -(b - a) (round-to-nearest is odd-symmetric and TwoSum is exact)
#pragma once

#include <cuda_runtime.h>

namespace dgk {

// keep CUDA's float and double fma visible next to the double-float overload declared below
using ::fma;

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit df(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ explicit df(int v) : hi(float(v)), lo(0.0f) {}
  // the nearest float and the float nearest to the remainder (exact for |v| within the
  // float32 exponent range and 48 significant bits)
  __host__ __device__ explicit df(double v) : hi(float(v)), lo(float(v - double(float(v)))) {}
  __host__ __device__ explicit operator double() const { return double(hi) + double(lo); }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}

// Renormalisation (Dekker's fast TwoSum): exact when |a| >= |b| or a == 0.
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  const float c = __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi));
  return df_fast_two_sum(p, __fadd_rn(e, c));
}

__device__ __forceinline__ df fma(df a, df b, df c) { return a * b + c; }

// the float nearest to hi + lo
__device__ __forceinline__ float to_float(df a) { return __fadd_rn(a.hi, a.lo); }

}  // namespace dgk
