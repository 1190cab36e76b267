// Double-FP32 ("double-word") arithmetic for FP64-class passes on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two binary32 numbers with
// |lo| <= ulp(hi)/2: about 48 significant bits.  GB300 executes binary64 at
// about 1/57 of the binary32 rate, so an FFT pass in double-word arithmetic
// (roughly 8-12 FP32 instructions per binary64 operation) runs several times
// faster than in binary64, with errors near 1e-14, three orders of magnitude
// inside the 1e-11 parity bar of the dipolar potential.
//
// Building blocks: Knuth's TwoSum and Dekker's Fast2Sum (error-free sums),
// the FMA-based exact product error, the "sloppy" double-word sum and the
// double-word product analysed by Joldes, Muller and Popescu ("Tight and
// rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44, 2017).  The sloppy sum's error is bounded by a
// small multiple of (|a| + |b|) 2^-47: the normwise bound an FFT needs.
// Every step uses the _rn intrinsics, which the compiler never contracts
// into an FMA or reorders (either would break the error-free steps).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace atkm {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // From binary64: constants and host-side set-up (device loads use tor<df>).
  __host__ __device__ constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  // From an integer: exact for |i| < 2^24 (grid indices, frequencies, sizes).
  __host__ __device__ constexpr df(int i) : hi((float)i), lo(0.0f) {}
};

struct __align__(16) cdf {
  df x, y;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// requires |a| >= |b| or a == 0
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df& operator+=(df& a, df b) { a = a + b; return a; }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the leading product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// The sign factors of the small DFTs are +-1 (exact); anything else multiplies.
__device__ __forceinline__ df operator*(int s, df a) { return s == 1 ? a : (s == -1 ? -a : df(s) * a); }
__device__ __forceinline__ df operator/(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = a - b * df(q1, 0.0f);
  return df_fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ bool operator>(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
// The double-word overload must not hide the binary64 ones inside namespace atkm.
using ::fabs;
__device__ __forceinline__ df fabs(df a) { return a.hi < 0.0f ? -a : a; }
// 1/sqrt(v): the binary32 estimate refined by one Newton step in double-word.
__device__ __forceinline__ df df_rsqrt(df v) {
  const df y(rsqrtf(v.hi), 0.0f);
  const df e = df(1.0f, 0.0f) - v * (y * y);
  return y + y * (df(0.5f, 0.0f) * e);
}

// Complex operations, inlined at every butterfly and twiddle of the FFT
// engine.  As out-of-line functions (one copy of their code per kernel) the
// double-word ATKM compiled several times faster but ran at two thirds of
// this speed: the passes are issue-bound and the calls cost instructions.
static __device__ __forceinline__ cdf df_cadd(cdf a, cdf b) {
  cdf r;
  r.x = a.x + b.x;
  r.y = a.y + b.y;
  return r;
}
static __device__ __forceinline__ cdf df_csub(cdf a, cdf b) {
  cdf r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  return r;
}
// a * b (conj_b = false) or a * conj(b) (conj_b = true)
static __device__ __forceinline__ cdf df_cmul(cdf a, cdf b, bool conj_b) {
  const df by = conj_b ? -b.y : b.y;
  cdf r;
  r.x = a.x * b.x - a.y * by;
  r.y = a.x * by + a.y * b.x;
  return r;
}
static __device__ __forceinline__ cdf df_cscl(cdf a, df s) {
  cdf r;
  r.x = a.x * s;
  r.y = a.y * s;
  return r;
}

}  // namespace atkm
