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

__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return fast_two_sum(p, e);
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

// host: a double constant as a float pair (hi = the nearest float, lo = the rest rounded)
inline f2 df_const(double c) {
  const float h = (float)c;
  return {h, (float)(c - (double)h)};
}

struct PairNum {
  f2 v;
};
__device__ __forceinline__ PairNum operator+(PairNum a, PairNum b) { return {df_add(a.v, b.v)}; }
__device__ __forceinline__ PairNum operator-(PairNum a, PairNum b) { return {df_sub(a.v, b.v)}; }
__device__ __forceinline__ PairNum operator-(PairNum a) { return {df_neg(a.v)}; }
__device__ __forceinline__ PairNum operator*(PairNum a, PairNum b) { return {df_mul(a.v, b.v)}; }
using ::fma;  // (the float and double overloads stay visible next to the pair one)
__device__ __forceinline__ PairNum fma(PairNum a, PairNum b, PairNum c) {
  return {df_add(df_mul(a.v, b.v), c.v)};
}

}  // namespace topo
