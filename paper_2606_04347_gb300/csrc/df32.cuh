// df32.cuh -- double-float arithmetic: a value carried as an unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi)/2 after every operation), about 48 significant bits.
//
// The FP32-mixed form keeps the membrane's spectral state (the carried spectrum phi^ of
// Sec. 3.3 and the stored ETDRK2 partial sum) and the transforms that enter or leave it in
// this format: FP32 roundoff there is white noise of size eps32 * rms(phi) in real space,
// and the recovery U = GU / G divides its effect on G = g(phi) by G near the recovery edge
// (G down to 1e-3, where phi or 1 - phi is about 0.0075).  Every operation runs on the FP32
// pipes (FP64 arithmetic is a small fraction of the FP32 rate on this part).
//
// Building blocks (error-free transformations): the sum a + b = s + e with s = fl(a + b)
// and e recovered exactly by Knuth's two-sum, and the product a * b = p + e with
// e = fma(a, b, -p).  Addition uses the one two-sum form (error about eps32^2 (|a| + |b|),
// the bound an FFT butterfly needs); multiplication keeps the cross terms hi*lo and lo*hi.
// The intrinsics __fadd_rn / __fsub_rn / __fmul_rn / __fmaf_rn are never contracted or
// reassociated by the compiler, which the error-free steps rely on.
#pragma once
#include <cuda_runtime.h>

namespace etd {

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfloat(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ constexpr dfloat(float f) : hi(f), lo(0.0f) {}
  // Split of a double (exact to the 48 bits kept); constant-folded for literals.
  __host__ __device__ constexpr dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

struct __align__(16) dcomplex {
  dfloat x, y;
};

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return dfloat(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float h = __fadd_rn(p, e);
  return dfloat(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// a + b with b a plain FP32 value (an increment already accurate to its own rounding).
__device__ __forceinline__ dfloat add_f(dfloat a, float b) { return a + dfloat(b, 0.0f); }

// The nearest FP32 value of hi + lo.
__device__ __forceinline__ float to_float(dfloat a) { return __fadd_rn(a.hi, a.lo); }

}  // namespace etd
