// Double-float values: an unevaluated sum h + l of two FP32 numbers with
// |l| <= ulp(h) / 2, about 48 significant bits, evaluated on the FP32 pipes.
// Used by the FP64-accurate path (FMM_FP64DF) for its M2L, whose FP64
// arithmetic would otherwise run at GB300's FP64 rate (1/64 of FP32).
//
// The operations are the classical error-free transformations: Knuth's
// two-sum, the FMA-based exact product (the error of a * b is
// fma(a, b, -a * b)), and Dekker's fast two-sum for renormalisation when the
// first operand dominates.  Addition is the short form (one two-sum of the
// high parts, the low parts added in FP32): its error is bounded by a few
// 2^-48 of |a| + |b|, the scale at which FP64 sums of the same terms are
// accurate too.
#pragma once

#include <cuda_runtime.h>

namespace fmm {
namespace {

struct dff {
  float h, l;
  dff() = default;
  __host__ __device__ constexpr dff(float hi, float lo) : h(hi), l(lo) {}
  // from FP64: the nearest float and the float nearest the remainder (folded
  // at compile time for table constants)
  __host__ __device__ constexpr explicit dff(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
};

// s + e == a + b with |e| <= ulp(s) / 2 when |a| >= |b| (Dekker)
__device__ __forceinline__ dff dff_fast(float a, float b) {
  const float s = a + b;
  return dff(s, b - (s - a));
}

__device__ __forceinline__ dff operator-(dff a) { return dff(-a.h, -a.l); }

__device__ __forceinline__ dff operator+(dff a, dff b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  return dff_fast(s, e);
}

__device__ __forceinline__ dff operator-(dff a, dff b) { return a + (-b); }

__device__ __forceinline__ dff operator*(dff a, dff b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return dff_fast(p, e);
}

// a * b + c with one renormalisation
__device__ __forceinline__ dff fmar(dff a, dff b, dff c) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = p + c.h;
  const float bb = s - p;
  float f = (p - (s - bb)) + (c.h - bb);
  f += e + c.l;
  return dff_fast(s, f);
}

__device__ __forceinline__ double to_double(dff a) { return (double)a.h + (double)a.l; }

}  // namespace
}  // namespace fmm
