// Double-word FP32 arithmetic ("df": an unevaluated sum hi + lo of two floats,
// |lo| <= ulp(hi)/2), about 48 significant bits, on the FP32 pipes.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, and converts
// between the two on the FP64 pipe as well, so the mixed-precision column
// solve computes in df and converts FP64 inputs with integer operations.
//
// Algorithms (error-free transformations and double-word operations):
//   two_sum       Knuth, TAOCP vol. 2, Sec. 4.2.2 (6 additions, no branch)
//   fast_two_sum  Dekker 1971 (requires |a| >= |b| or a == 0)
//   two_prod      via the fused multiply-add (exact product error)
//   add           "AccurateDWPlusDW", Joldes, Muller & Popescu, ACM TOMS 44
//                 (2017), Alg. 6: relative error below 3u^2 + 13u^3 (u = 2^-24)
//   add_same_sign "SloppyDWPlusDW", ibid. Alg. 5: fewer operations, its error
//                 bound holds when the operands have the same sign (no
//                 cancellation)
//   add (df, float) "DWPlusFP", ibid. Alg. 4
//   mul           "DWTimesDW1", ibid. Alg. 10
//   mul (df, float) "DWTimesFP1", ibid. Alg. 7
//   rcp           one Newton-Raphson step r + r (1 - x r) in df from the
//                 approximate FP32 reciprocal of the leading word (the step
//                 doubles its ~23 correct bits).
// The additions and subtractions use the _rn intrinsics so the compiler never
// fuses them into multiply-adds, which would break the exact error terms.
#pragma once
#include <cuda_runtime.h>

namespace icon {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  const df v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ df add_same_sign(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator+(df a, float b) {
  const df s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(a.lo, s.lo));
}

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  const float t = __fmaf_rn(a.lo, b.hi, __fmul_rn(a.hi, b.lo));
  return fast_two_sum(p, __fadd_rn(e, t));
}

__device__ __forceinline__ df operator*(df a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.hi, b, -p);
  return fast_two_sum(p, __fmaf_rn(a.lo, b, e));
}

__device__ __forceinline__ df rcp(df x) {
  const float r = __fdividef(1.0f, x.hi);
  const df e = (x * (-r)) + 1.0f;  // 1 - x r, small
  return df{r, 0.0f} + e * r;      // r + r (1 - x r)
}

// double -> df with integer operations only: hi keeps the leading 24
// significant bits (truncated), lo the next 29 bits rounded to 24.
// Magnitudes below 2^-74 keep only hi, below 2^-126 become (signed) zero, at
// or above 2^128 infinity; NaN stays NaN.
__device__ __forceinline__ df to_df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const int e = (int)((h >> 20) & 0x7FFu);  // biased FP64 exponent
  const unsigned sign = h & 0x80000000u;
  if (e <= 896) return {__uint_as_float(sign), 0.0f};  // zero or below the FP32 normal range
  if (e >= 1151) {  // beyond the FP32 range (or infinity, NaN)
    const bool nan = e == 2047 && ((h & 0xFFFFFu) | l) != 0u;
    return {__uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u)), 0.0f};
  }
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29));
  const unsigned r = l & 0x1FFFFFFFu;  // the 29 bits below hi's last place, weight 2^(e - 1075)
  float lo = 0.0f;
  if (r != 0u && e - 1075 + 127 >= 1) {
    lo = __fmul_rn(__uint2float_rn(r), __uint_as_float((unsigned)(e - 1075 + 127) << 23));
    if (sign) lo = -lo;
  }
  return {hi, lo};
}

__device__ __forceinline__ df to_df(float x) { return {x, 0.0f}; }

// float -> double by exponent re-bias (exact; FP32 subnormals read as zero)
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  if (e == 0u) return __longlong_as_double((long long)sign);
  if (e == 255u) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | m));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) | m));
}

// one FP64 addition; both words convert exactly with integer operations
__device__ __forceinline__ double to_double(df a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }

// leading-word value (FP32 mirrors)
__device__ __forceinline__ float to_float(df a) { return __fadd_rn(a.hi, a.lo); }

// Double-word values whose additions and subtractions use "SloppyDWPlusDW"
// (Joldes, Muller & Popescu, Alg. 5): 11 operations instead of 20.  Its error
// is bounded in absolute terms, about 2u^2 (|a| + |b|), so the relative error
// of a sum grows with the cancellation (|a| + |b|) / |a + b|.  For a
// computation whose accuracy is set at FP32 level elsewhere (the column solve
// of the mixed-precision step, fed by FP32 stencils), this is still many
// orders of magnitude below that level.  Products and reciprocals as df.
struct dws {
  float hi, lo;
};

__device__ __forceinline__ dws to_dws(df x) { return {x.hi, x.lo}; }
__device__ __forceinline__ df to_df(dws x) { return {x.hi, x.lo}; }

__device__ __forceinline__ dws operator+(dws a, dws b) {
  const df s = two_sum(a.hi, b.hi);
  return to_dws(fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))));
}
__device__ __forceinline__ dws operator-(dws a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dws operator-(dws a, dws b) { return a + (-b); }
__device__ __forceinline__ dws operator+(dws a, float b) { return to_dws(to_df(a) + b); }
__device__ __forceinline__ dws operator*(dws a, dws b) { return to_dws(to_df(a) * to_df(b)); }
__device__ __forceinline__ dws operator*(dws a, float b) { return to_dws(to_df(a) * b); }
__device__ __forceinline__ dws rcp(dws x) { return to_dws(rcp(to_df(x))); }
__device__ __forceinline__ double to_double(dws a) { return to_double(to_df(a)); }
__device__ __forceinline__ float to_float(dws a) { return to_float(to_df(a)); }

}  // namespace icon
