// Exact base-256 digits of FP64 values for the BF16-slice products (oz_gemm.cu, fe_oz.cu).
#pragma once
#include <cstdint>

namespace rchfsi {

// FP64 arithmetic is scarce on this GPU, so the slicing works on the bits: the binary exponent E
// with |x| in [2^(E-1), 2^E) (E = -100000 for 0), and the digits of x 2^(56 - e) in base 256 by
// integer shifts.
__device__ __forceinline__ int exp_of(double x) {
  const long long b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
  if (b == 0) return -100000;
  const int eb = (int)(b >> 52);
  if (eb != 0) return eb - 1022;
  // subnormal: 2^-1074 times the 52-bit fraction
  return -1074 + (64 - __clzll(b));
}

// round(x 2^(56 - e)) as a signed 64-bit integer, for |x| < 2^e (so |result| <= 2^56).
__device__ __forceinline__ long long fixed56(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const long long b = bits & 0x7fffffffffffffffLL;
  if (b == 0) return 0;
  const int eb = (int)(b >> 52);
  long long mant = b & 0x000fffffffffffffLL;
  int ex;  // x = mant 2^ex
  if (eb != 0) {
    mant |= 0x0010000000000000LL;
    ex = eb - 1075;
  } else {
    ex = -1074;
  }
  const int sh = ex + 56 - e;  // <= 4 since |x| < 2^e
  long long f;
  if (sh >= 0) f = mant << sh;
  else if (sh > -63) f = (mant + (1LL << (-sh - 1))) >> (-sh);
  else f = 0;
  return bits < 0 ? -f : f;
}


// Digit s (s = 0 .. 6) of round(x 2^(56 - e)) in place: returns t_s and leaves the remainder in f.
// sum_s t_s 2^(48 - 8 s) = f on entry; |t_0| <= 256, |t_s| <= 128.
__device__ __forceinline__ long long next_digit(long long& f, int s) {
  const int sh = 48 - 8 * s;
  if (sh <= 0) return f;
  const long long t = (f + (1LL << (sh - 1))) >> sh;
  f -= t << sh;
  return t;
}

// x (finite FP32, |x| in the normal range or 0) times 2^p as an FP64 value, by integer arithmetic.
__device__ __forceinline__ double f32_scaled(float x, int p) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t e8 = (b >> 23) & 0xff;
  if (e8 == 0) return 0.0;
  const long long e = (long long)e8 - 127 + 1023 + p;
  if (e <= 0 || e >= 2047) return ldexp((double)x, p);  // out of the normal range: rare, exact path
  const unsigned long long bits = ((unsigned long long)(b >> 31) << 63) | ((unsigned long long)e << 52) |
                                  ((unsigned long long)(b & 0x7fffff) << 29);
  return __longlong_as_double((long long)bits);
}

}  // namespace rchfsi
