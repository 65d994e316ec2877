// Exact fixed-point helpers of the refinement residual, integer instructions only (every
// FP64-pipe instruction is scarce on this GPU): conversions between FP64 / FP32 values and
// 64-bit fixed-point integers with a power-of-two scale, and the scaled 64 x 64-bit product.
#pragma once
#include <cstdint>

namespace ts {

// x as a fixed-point integer with the scale 2^(1022 + H - emax), H = 53 + P: the mantissa
// with its implicit bit, pre-shifted left by P, then shifted right by t = emax - e; integer
// instructions only.  Exact when t <= P; otherwise the magnitude is truncated toward zero
// onto the fixed-point grid.  |result| < 2^H whenever e <= emax; zero and subnormals give 0.
__device__ __forceinline__ long long to_fixed(double x, int emax, int P) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF);
  const long long m = ((bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52)) << P;
  int t = emax - e;
  t = (e == 0 || t > 63) ? 63 : t;  // m < 2^63, so a shift by 63 gives 0
  const long long sgn = bits >> 63;  // 0 or -1
  return ((m >> t) ^ sgn) - sgn;
}

// v -> double, rounded to nearest even, with integer instructions only (|v| < 2^63): the
// magnitude is normalised with a count of leading zeros, its top 53 bits kept and rounded on
// the 11 bits below them; a carry out of the mantissa bumps the exponent through the add.
__device__ __forceinline__ double i64_to_f64(long long v) {
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ULL;
  unsigned long long a = v < 0 ? 0ULL - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll(a);
  a <<= (lz & 63);
  unsigned long long m = a >> 11;
  const unsigned rem = (unsigned)a & 0x7FFu;
  m += (rem > 0x400u || (rem == 0x400u && (m & 1ULL))) ? 1ULL : 0ULL;
  const unsigned long long mag = ((unsigned long long)(1023 + 63 - 1 - lz) << 52) + m;
  return __longlong_as_double((long long)(a == 0 ? 0ULL : (sgn | mag)));
}

// v -> float, rounded to nearest even, with 32-bit integer instructions only: the top 23
// fraction bits rounded on the 29 below them, exponent rebased from 1023 to 127.  Results
// below the normal float range are flushed to zero (signed), above it give infinity; NaN
// stays NaN.
__device__ __forceinline__ float f64_to_f32(double v) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const unsigned lo = (unsigned)bits, hi = (unsigned)(bits >> 32);
  const unsigned sgn = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1FFFFFFFu;
  m += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  unsigned f = ((unsigned)(e - 896) << 23) + m;
  f = e <= 896 ? 0u : f;
  f = e >= 1151 ? 0x7F800000u : f;
  f = (e == 2047 && ((hi & 0xFFFFFu) | lo)) ? 0x7FC00000u : f;
  return __uint_as_float(sgn | f);
}

// (Q * U) >> F for 64-bit Q and U with the 128-bit product (floor), 0 < F < 64, for
// results that fit in 64 bits.
__device__ __forceinline__ long long mul_shift(long long q, long long u, int F) {
  const unsigned long long lo = (unsigned long long)q * (unsigned long long)u;
  const long long hi = __mul64hi(q, u);
  return (long long)((unsigned long long)hi << (64 - F)) | (long long)(lo >> F);
}

// v 2^s as a 64-bit integer, rounded to nearest (ties away from zero), for |v 2^s| < 2^62:
// the FP32 mantissa (implicit bit included) shifted left by e - 150 + s, or right with a
// rounding half added first; no branches.  Zero and FP32 subnormals give 0; shifts that
// would overflow are clamped (the caller keeps |v 2^s| in range).
__device__ __forceinline__ long long f32_to_fixed(float v, int s) {
  const uint32_t u = __float_as_uint(v);
  const int e = (int)((u >> 23) & 0xFFu);
  const int sh = e - 150 + s;
  const int shl = min(max(sh, 0), 38);
  const int shr = min(max(-sh, 0), 63);
  const unsigned long long m = (unsigned long long)((u & 0x7FFFFFu) | 0x800000u) << shl;
  const unsigned long long half = (1ull << shr) >> 1;
  const unsigned long long mag = e == 0 ? 0ull : (m + half) >> shr;
  return (u >> 31) ? -(long long)mag : (long long)mag;
}

// v 2^-s as a double, rounded to nearest even, integer instructions only (|v| < 2^63);
// results below the normal range are flushed to zero.
__device__ __forceinline__ double fixed_to_f64(long long v, int s) {
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ULL;
  unsigned long long a = v < 0 ? 0ULL - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll(a);
  a <<= (lz & 63);
  unsigned long long m = a >> 11;
  const unsigned rem = (unsigned)a & 0x7FFu;
  m += (rem > 0x400u || (rem == 0x400u && (m & 1ULL))) ? 1ULL : 0ULL;
  const long long ex = 1023LL + 63 - lz - s;  // biased exponent of the leading bit
  const unsigned long long mag = ((unsigned long long)(ex - 1) << 52) + m;
  return __longlong_as_double((long long)((a == 0 || ex <= 0) ? sgn : (sgn | mag)));
}

// The same rounded toward zero (for a final result whose error budget is far above one
// FP64 ulp): fewer instructions.
__device__ __forceinline__ double fixed_to_f64_rz(long long v, int s) {
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ULL;
  unsigned long long a = v < 0 ? 0ULL - (unsigned long long)v : (unsigned long long)v;
  const int lz = __clzll(a);
  a <<= (lz & 63);
  const long long ex = 1023LL + 63 - lz - s;
  const unsigned long long mag = ((unsigned long long)(ex - 1) << 52) + (a >> 11);
  return __longlong_as_double((long long)((a == 0 || ex <= 0) ? sgn : (sgn | mag)));
}

}  // namespace ts
