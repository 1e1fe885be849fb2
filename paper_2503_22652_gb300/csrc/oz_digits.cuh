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

// round(x 2^q) as a signed 64-bit integer (nearest, ties away from zero), by integer arithmetic,
// for finite x with |x| 2^q < 2^62 and q <= 38 + 150 - (biased exponent of x).  Zero and FP32
// subnormals give 0.  Branch-free: the 24-bit significand is placed at bit 39 and shifted right
// by 39 - (its scale), rounding on the bits shifted out.
__device__ __forceinline__ long long f32_to_fixed(float x, int q) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t e8 = (b >> 23) & 0xffu;
  const int r0 = 189 - (int)e8 - q;  // 39 - (e8 - 150 + q): the right shift
  // |x| 2^q < 1/2 (r0 > 63) rounds to 0, as does a zero or subnormal x
  const uint32_t mant = (e8 != 0u && r0 <= 63) ? ((b & 0x7fffffu) | 0x800000u) : 0u;
  const int r = min(max(r0, 1), 63);
  unsigned long long u = (unsigned long long)mant << 39;
  u = (u + (1ull << (r - 1))) >> r;
  const long long v = (long long)u;
  return (b >> 31) ? -v : v;
}

// v 2^e as an FP64 value, rounded to nearest even, by integer arithmetic (|v| < 2^63).
__device__ __forceinline__ double fixed_to_f64(long long v, int e) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
  unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  a <<= lz;                          // leading one at bit 63
  unsigned long long mant = a >> 11;  // 53 significant bits
  const unsigned long long rem = a & 0x7ffull;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ++mant;
  long long ex = 63 - lz + (long long)e;  // v 2^e = 1.f 2^ex
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  const long long be = ex + 1023;
  if (be <= 0 || be >= 2047) return ldexp((double)v, e);  // out of the normal range: rare
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (mant & 0xfffffffffffffull)));
}

}  // namespace rchfsi
