// Pair-of-FP32 ("double-float") arithmetic for the outer CG operators of the mixed solver.
// A value is the unevaluated sum hi + lo of two floats (about 48 significant bits): Dekker's
// error-free TwoSum / FastTwoSum and the FMA-based TwoProd.  Every add and multiply uses the _rn
// intrinsics so that the compiler cannot contract them into fused operations that would break
// the error terms.  PairNum wraps a pair with operators, so that templates written for float or
// double (the Walsh-Hadamard butterflies of the hex element) compile for pairs unchanged.
#pragma once

#include <cuda_runtime.h>

namespace topo {

struct f2 {
  float h, l;
};

__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ f2 df_neg(f2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ f2 df_sub(f2 a, f2 b) { return df_add(a, df_neg(b)); }

// The sum without the closing renormalisation (8 operations instead of 11): hi = RN(a.h + b.h),
// lo = its rounding error (TwoSum) plus the low parts.  hi + lo keeps about 48 bits relative to
// the operands; after a cancellation lo may exceed half an ulp of hi, which the next products
// (renormalised) and the final conversion to FP64 absorb.  For the short butterflies and node sums
// of the element operators; long accumulations (dot products) keep df_add.
__device__ __forceinline__ f2 df_add_nr(f2 a, f2 b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return {s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ f2 df_sub_nr(f2 a, f2 b) { return df_add_nr(a, df_neg(b)); }

__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return fast_two_sum(p, e);
}
// The product without the closing renormalisation (4 instead of 7 operations): p = a.h b.h
// rounded and e its exact error plus the cross terms, |e| below about 2^-22 |p|.  Like the sums of
// df_add_nr, for values that feed further pair sums and products (the element operators);
// products that end in a dot product keep df_mul.
__device__ __forceinline__ f2 df_mul_nr(f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return {p, e};
}

// double -> float pair with integer operations only: hi = d truncated to 24 significant bits,
// lo = the remaining 29 bits rounded to float.  |d| < 2^-126 gives 0; the finite range of the
// outer operator's inputs is well inside float's.
__device__ __forceinline__ f2 df_from_double(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff);
  const int ef = e - 1023 + 127;
  if (ef <= 0) return {0.0f, 0.0f};
  const unsigned sign = (unsigned)(b >> 63) << 31;
  if (ef >= 255)  // beyond float range, infinities and NaNs: an infinity or a NaN
    return {__uint_as_float(sign | 0x7f800000u | (unsigned)((b >> 29) & 0x7fffffu) |
                            (e == 2047 && (b & 0xfffffffffffffull) ? 1u : 0u)),
            0.0f};
  const float hi = __uint_as_float(sign | ((unsigned)ef << 23) |
                                   (unsigned)((b >> 29) & 0x7fffffu));
  const unsigned rem = (unsigned)(b & ((1ull << 29) - 1));
  // rem * 2^(e - 1075) = rem * 2^-52 * 2^(e - 1023); both factors are normal floats here
  float lo = __fmul_rn(__fmul_rn(__uint2float_rn(rem), 0x1p-52f),
                       __uint_as_float((unsigned)ef << 23));
  return {hi, sign ? -lo : lo};
}

// float -> double exactly, with integer operations (normal floats; zero and subnormals give 0).
__device__ __forceinline__ double double_from_float(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xff;
  if (ef == 0) return 0.0;
  if (ef == 255)  // infinities and NaNs stay what they are (breakdown tests see them)
    return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                            (0x7ffull << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(ef + 896) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

// Conversions between FP64 and FP32 with integer operations, written from the IEEE 754 binary64
// and binary32 formats.  The FP64 pipe of this part issues about two instructions per clock per
// SM and a conversion instruction (F2F) takes one of its slots, so vector kernels that convert
// every entry become FP64-bound; the integer pipe is far wider.  Both give the results of the
// hardware conversions (rounding to nearest, ties to even; subnormals; overflow to infinity;
// a NaN stays a NaN).
__device__ __forceinline__ float float_from_double_rn(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xfffffffffffffull;
  if (e == 2047) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  const int ef = e - 896;  // the binary32 exponent field
  if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
  if (ef >= 1) {  // normal: 23 of the 52 fraction bits, the other 29 decide the rounding
    unsigned u = ((unsigned)ef << 23) | (unsigned)(m >> 29);
    const unsigned rem = (unsigned)(m & 0x1fffffffu);
    if (rem > 0x10000000u || (rem == 0x10000000u && (u & 1u))) ++u;  // (carries into the exponent)
    return __uint_as_float(sign | u);
  }
  // a binary32 subnormal or zero: u 2^-149 with u = M 2^(e - 1075 + 149) = M >> (30 - ef)
  const int sh = 30 - ef;
  if (e == 0 || sh >= 54) return __uint_as_float(sign);
  const unsigned long long M = m | (1ull << 52);
  unsigned u = (unsigned)(M >> sh);
  const unsigned long long rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (u & 1u))) ++u;
  return __uint_as_float(sign | u);
}

__device__ __forceinline__ double double_from_float_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned ef = (u >> 23) & 0xff, mant = u & 0x7fffffu;
  if (ef == 255)
    return __longlong_as_double((long long)(sign | (0x7ffull << 52) | ((unsigned long long)mant << 29)));
  if (ef == 0) {
    if (mant == 0) return __longlong_as_double((long long)sign);
    const int pb = 31 - __clz(mant);  // leading bit: the value is 2^(pb - 149) (1 + frac)
    const unsigned long long frac = (unsigned long long)(mant - (1u << pb)) << (52 - pb);
    return __longlong_as_double((long long)(sign | ((unsigned long long)(pb + 874) << 52) | frac));
  }
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(ef + 896) << 52) | ((unsigned long long)mant << 29)));
}

// Widening and narrowing of a vector entry of precision TV (float or double).
__device__ __forceinline__ double double_of(float f) { return double_from_float_exact(f); }
__device__ __forceinline__ double double_of(double d) { return d; }
template <typename TV>
__device__ __forceinline__ TV tv_from_double(double d) {
  if constexpr (sizeof(TV) == 4) return float_from_double_rn(d);
  else return d;
}

// host: a double constant as a float pair (hi = the nearest float, lo = the rest rounded)
inline f2 df_const(double c) {
  const float h = (float)c;
  return {h, (float)(c - (double)h)};
}

struct PairNum {
  f2 v;
};
__device__ __forceinline__ PairNum operator+(PairNum a, PairNum b) { return {df_add_nr(a.v, b.v)}; }
__device__ __forceinline__ PairNum operator-(PairNum a, PairNum b) { return {df_sub_nr(a.v, b.v)}; }
__device__ __forceinline__ PairNum operator-(PairNum a) { return {df_neg(a.v)}; }
__device__ __forceinline__ PairNum operator*(PairNum a, PairNum b) { return {df_mul_nr(a.v, b.v)}; }
using ::fma;  // (the float and double overloads stay visible next to the pair one)
__device__ __forceinline__ PairNum fma(PairNum a, PairNum b, PairNum c) {
  return {df_add_nr(df_mul_nr(a.v, b.v), c.v)};
}

}  // namespace topo
