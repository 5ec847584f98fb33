// Rounding of exact integer results to IEEE doubles with integer instructions only.
//
// On sm_103a the FP64 pipe issues about 1.6 operations per clock per SM, and conversions
// between 64-bit integers and floating types run at that rate too, while 64-bit integer
// shifts and adds issue about 12 per clock and 32-bit ones several times more.  The
// element-wise kernels of an iteration round exact Ozaki sums (S * 2^c, S an integer) to
// doubles, so they assemble the sign, exponent and significand fields directly: the same
// round-to-nearest-even result as an FP64 conversion, without the FP64 pipe.
#pragma once

#include "frx_internal.cuh"

namespace frx {

typedef __int128 i128;
typedef unsigned __int128 u128;

// leading zeros of a nonzero 64-bit word (host and device)
__host__ __device__ __forceinline__ int clz64(u64 a) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return a ? __builtin_clzll(a) : 64;
#endif
}

__host__ __device__ __forceinline__ int bitlen_u64(u64 a) { return 64 - clz64(a); }

__host__ __device__ __forceinline__ int bitlen_u128(u128 a) {
  u64 hi = (u64)(a >> 64);
  return hi ? 128 - clz64(hi) : 64 - clz64((u64)a);
}

__host__ __device__ __forceinline__ u128 abs_i128(i128 v) { return v < 0 ? (u128)0 - (u128)v : (u128)v; }

// an upper bound on the bit length of |v| (exact for v >= 0, at most one more for v < 0):
// the bit length of v XOR its sign mask, plus one for negatives
__device__ __forceinline__ int bitlen_bound_i128(i128 v) {
  const u64 hi = (u64)(v >> 64), lo = (u64)v, sm = (u64)((i64)hi >> 63);
  const u64 h = hi ^ sm, l = lo ^ sm;
  return (h ? 128 - __clzll((long long)h) : 64 - __clzll((long long)l)) + (int)(sm & 1);
}

// full signed 64 x 64 -> 128-bit product
__device__ __forceinline__ i128 mul_i64(i64 a, i64 b) {
  const u64 lo = (u64)a * (u64)b;
  const u64 hi = (u64)__mul64hi(a, b);
  return (i128)(((u128)hi << 64) | (u128)lo);
}

// Bits of RN-even((-1)^neg * a * 2^c) for a > 0.  False when the result is subnormal or
// overflows (the caller then takes a general path).  Works on the 64-bit halves: the top
// 64 bits of a and a sticky bit for the rest decide the rounding exactly.
__host__ __device__ __forceinline__ bool rn_bits(u128 a, bool neg, int c, u64& bits) {
  const u64 hi = (u64)(a >> 64), lo = (u64)a;
  int E;
  u64 mant;
  if (hi == 0) {
    const int L = bitlen_u64(lo);
    E = L - 1 + c;
    if (L <= 53) {
      mant = lo << (53 - L);
    } else {
      const int sh = L - 53;  // 1..11
      mant = lo >> sh;
      const u64 rest = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
      if (rest > half || (rest == half && (mant & 1))) ++mant;
    }
  } else {
    const int Lh = bitlen_u64(hi);  // 1..64
    E = 63 + Lh + c;
    u64 top;
    bool sticky;
    if (Lh == 64) {
      top = hi;
      sticky = lo != 0;
    } else {
      top = (hi << (64 - Lh)) | (lo >> Lh);
      sticky = (lo << (64 - Lh)) != 0;
    }
    mant = top >> 11;
    const u64 rest = top & 0x7ffull;
    if (rest > 0x400ull || (rest == 0x400ull && (sticky || (mant & 1)))) ++mant;
  }
  if (mant >> 53) {  // rounding carried into a new binade
    mant >>= 1;
    ++E;
  }
  if (E < -1022 || E > 1023) return false;
  bits = (neg ? (1ull << 63) : 0ull) | ((u64)(E + 1023) << 52) | (mant & ((1ull << 52) - 1));
  return true;
}

// out = RN-even(S * 2^c); false (out untouched) for a subnormal or overflowing result.
__host__ __device__ __forceinline__ bool rn_scaled(i128 S, int c, double& out) {
  if (S == 0) {
    out = 0.0;
    return true;
  }
  u64 b;
  if (!rn_bits(abs_i128(S), S < 0, c, b)) return false;
  out = bits_to_double(b);
  return true;
}

// RN(x1 + N 2^c) for the usual update, a correction far below x1 whose sum stays in x1's
// binade: with x1 = P 2^q (P a signed 53-bit integer) and s = q - c >= 1, the sum is
// (P + floor(N / 2^s) + f) 2^q with 0 <= f < 1; bit s - 1 of N and the bits below it (sticky)
// decide round-half-even to an integer R, and R 2^q is the correctly rounded sum when
// 2^52 < |P + floor(N / 2^s)| and |R| < 2^53.  False otherwise (the caller takes the exact
// 128-bit path): x1 zero, subnormal or not finite, s outside [1, 127], or a sum that may leave
// the binade.
__host__ __device__ __forceinline__ bool add_on_grid_rn(double x1, i128 N, int c, double& out) {
  const u64 b = double_to_bits(x1);
  const int be = (int)((b >> 52) & 0x7ff);
  const int s = be - 1075 - c;
  if (be == 0 || be == 0x7ff || s < 1 || s > 127) return false;
  const i128 T2 = N >> (s - 1);                        // floor(N / 2^(s-1))
  const i64 t2 = (i64)T2;
  if ((i128)t2 != T2 || t2 > (1ll << 60) || t2 < -(1ll << 60)) return false;
  const bool sticky = s > 1 && ((u128)N << (129 - s)) != 0;
  const i64 m = (i64)((b & ((1ull << 52) - 1)) | (1ull << 52));
  const i64 F = ((b >> 63) ? -m : m) + (t2 >> 1);        // P + floor(N / 2^s)
  const i64 R = F + ((t2 & 1) && (sticky || (F & 1)) ? 1 : 0);
  const u64 aF = F < 0 ? (u64)0 - (u64)F : (u64)F, aR = R < 0 ? (u64)0 - (u64)R : (u64)R;
  if (aF <= (1ull << 52) || aR >= (1ull << 53)) return false;
  out = bits_to_double((R < 0 ? (1ull << 63) : 0ull) | ((u64)be << 52) | (aR & ((1ull << 52) - 1)));
  return true;
}

// RN(x1 + N 2^c) exactly in 128-bit integers; false when the aligned sum would not fit
// or the result leaves the normal range
__host__ __device__ __forceinline__ bool add_exact_rn(double x1, i128 N, int c, double& out) {
  if (is_zero(x1)) return rn_scaled(N, c, out);
  i64 P;
  int q;
  decompose(x1, P, q);
  const int bn = N == 0 ? 0 : bitlen_u128(abs_i128(N));
  const int d = q - c;
  if (d >= 0) {
    if (d > 72 || bn > 125) return false;
    return rn_scaled(((i128)P << d) + N, c, out);
  }
  if (bn - d > 125) return false;
  return rn_scaled((i128)P + (N << (-d)), q, out);
}

// Single-precision value of D * 2^q truncated to 24 bits (for sums of squares that only
// feed norm estimates).  Zero below the normal float range; false above 2^60.
__device__ __forceinline__ bool f32_scaled(i64 D, int q, float& out) {
  if (D == 0) {
    out = 0.f;
    return true;
  }
  const u64 a = D < 0 ? (u64)0 - (u64)D : (u64)D;
  const int L = bitlen_u64(a);
  const int E = L - 1 + q;
  if (E > 60) return false;
  if (E < -126) {
    out = 0.f;
    return true;
  }
  const unsigned m24 = (unsigned)(L > 24 ? a >> (L - 24) : a << (24 - L));
  out = __int_as_float((int)((D < 0 ? 0x80000000u : 0u) | ((unsigned)(E + 127) << 23) | (m24 & 0x7fffffu)));
  return true;
}

// Single-precision value of the double x * 2^s, truncated; zero for tiny values and false
// above 2^60 (the caller accumulates those in FP64).
__device__ __forceinline__ bool f32_of_double(double x, int s, float& out) {
  const u64 b = (u64)__double_as_longlong(x);
  const int bexp = (int)((b >> 52) & 0x7ff);
  if (bexp == 0) {
    out = 0.f;
    return true;
  }
  const int E = bexp - 1023 + s;
  if (E > 60) return false;
  if (E < -126) {
    out = 0.f;
    return true;
  }
  out = __int_as_float((int)((unsigned)(b >> 32 & 0x80000000u) | ((unsigned)(E + 127) << 23) |
                             (unsigned)((b >> 29) & 0x7fffffu)));
  return true;
}

// floor-toward-zero of |m| * |N| / 2^s with the sign of m * N, for a product known to
// satisfy |m N| < 2^(126 + s) (so the result fits); s may be negative (left shift).
__device__ __forceinline__ i128 mul_shift(i64 m, i128 N, int s) {
  const bool neg = (m < 0) != (N < 0);
  const u64 am = m < 0 ? (u64)0 - (u64)m : (u64)m;
  const u128 aN = abs_i128(N);
  const u128 p0 = (u128)am * (u64)aN;
  const u128 p1 = (u128)am * (u64)(aN >> 64);
  const u128 mid = (p0 >> 64) + (u128)(u64)p1;
  const u64 w0 = (u64)p0, w1 = (u64)mid, w2 = (u64)(p1 >> 64) + (u64)(mid >> 64);
  const u128 lo = ((u128)w1 << 64) | (u128)w0;
  u128 v;
  if (s <= 0) {
    v = lo << (-s);
  } else if (s >= 192) {
    v = 0;
  } else if (s >= 128) {
    v = (u128)(w2 >> (s - 128));
  } else {
    v = (lo >> s) | ((u128)w2 << (128 - s));
  }
  return neg ? -(i128)v : (i128)v;
}

}  // namespace frx
