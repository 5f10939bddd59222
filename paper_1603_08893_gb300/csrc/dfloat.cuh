// Float-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2, about 48 significant bits (rounding
// ~ 2^-47 per operation, relative to the operands).  Built on the error-free transformations
// of Knuth (two-sum), Dekker (fast two-sum, |a| >= |b|) and the FMA
// two-product.  GB300 issues float32 at 64x its float64 rate, so the
// float64-accuracy transforms of the mixed path (residual G:P and the
// projection of dF) run on the float32 pipe in this representation.
#pragma once
#include <type_traits>

#include "common.cuh"

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // rounds d to the nearest float-float (exact for |d| within float range
  // up to the last 5 bits of the double significand)
  __host__ __device__ explicit constexpr dfl(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

template <typename R>
struct is_dfl : std::false_type {};
template <>
struct is_dfl<dfl> : std::true_type {};

// s + e = a + b exactly (Knuth)
RVE_DEV dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker)
RVE_DEV dfl fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

// Sum with an absolute error of a few 2^-48 (|a| + |b|): the high parts are
// added exactly, the low parts in one rounding, then renormalised.  Under
// cancellation the result's relative error can grow, its absolute error does
// not -- the bound that a linear transform (DFT, projection) needs, whose
// error analysis is in absolute terms relative to the input's norm.  About
// half the operations of the variant that also adds the low parts exactly.
RVE_DEV dfl operator+(dfl a, dfl b) {
  const dfl s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

RVE_DEV dfl operator-(dfl a) { return {-a.hi, -a.lo}; }
RVE_DEV dfl operator-(dfl a, dfl b) { return a + (-b); }

// p + e = a.hi b.hi exactly (FMA two-product), plus the cross terms
RVE_DEV dfl operator*(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

RVE_DEV dfl fma(dfl a, dfl b, dfl c) { return a * b + c; }
RVE_DEV dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
RVE_DEV dfl& operator-=(dfl& a, dfl b) { return a = a - b; }
RVE_DEV dfl& operator*=(dfl& a, dfl b) { return a = a * b; }
