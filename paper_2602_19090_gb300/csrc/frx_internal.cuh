// Internal helpers shared by the frx CUDA translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/frx.h"

namespace frx {

constexpr int EZERO = -(1 << 30);   // exponent of an all-zero row or column
constexpr int DIGIT_BITS = 8;                        // 8-bit digits: |d| <= 2^7 (exact in bf16)
constexpr int DIGIT_MAX = 1 << (DIGIT_BITS - 1);     // 128
constexpr int PRODUCT_BITS = 2 * (DIGIT_BITS - 1);   // |d_L d_R| <= 2^14
constexpr int MAX_PLANES = 16;                       // digit planes per operand (128 bits)

typedef unsigned long long u64;
typedef long long i64;

#define FRX_CUDA_TRY(expr)                               \
  do {                                                   \
    cudaError_t err__ = (expr);                          \
    if (err__ != cudaSuccess) return FRX_E_CUDA;         \
  } while (0)

#define FRX_TRY(expr)                                    \
  do {                                                   \
    int st__ = (expr);                                   \
    if (st__ < 0) return st__;                           \
  } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------------------
// Exact exponent helpers (ceil(log2 |x|) from the IEEE bits)
// ---------------------------------------------------------------------------
__host__ __device__ inline int ceil_log2_absbits(u64 ab) {
  // ab: bits of a finite positive double
  int bexp = (int)(ab >> 52);
  u64 man = ab & ((1ull << 52) - 1);
  if (bexp == 0) {
    if (man == 0) return EZERO;
#ifdef __CUDA_ARCH__
    int msb = 63 - __clzll((long long)man);
#else
    int msb = 63 - __builtin_clzll(man);
#endif
    // value = man * 2^-1074 in [2^(msb-1074), 2^(msb-1073))
    return (man & (man - 1)) ? msb - 1073 : msb - 1074;
  }
  return man == 0 ? bexp - 1023 : bexp - 1022;
}

__host__ __device__ inline bool nonfinite_absbits(u64 ab) { return (ab >> 52) == 0x7ff; }

__host__ __device__ inline double bits_to_double(u64 b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, 8);
  return d;
#endif
}

__host__ __device__ inline u64 double_to_bits(double x) {
#ifdef __CUDA_ARCH__
  return (u64)__double_as_longlong(x);
#else
  u64 b;
  __builtin_memcpy(&b, &x, 8);
  return b;
#endif
}

// 2^k as a double for k in [-1074, 1023] (exact)
__host__ __device__ inline double pow2(int k) {
  if (k >= -1022) return bits_to_double((u64)(k + 1023) << 52);
  return bits_to_double(1ull << (k + 1074));
}

// ---------------------------------------------------------------------------
// Fixed-grid digit extraction in exact integer arithmetic.
//   x = P * 2^q (P signed, |P| < 2^53).  Plane r has weight 2^(e + 1 - 7r);
//   d_r = RNE(rho_{r-1} / w_r), rho_r = rho_{r-1} - d_r w_r (round half to even),
//   which is the sigma-trick fl((sigma + rho) - sigma) with ulp(sigma) = w_r.
// ---------------------------------------------------------------------------
// x == +-0 tested on its bits (an integer instruction, not a compare on the FP64 pipe)
__host__ __device__ inline bool is_zero(double x) { return (double_to_bits(x) << 1) == 0; }

__host__ __device__ inline void decompose(double x, i64& P, int& q) {
  u64 b = double_to_bits(x);
  int bexp = (int)((b >> 52) & 0x7ff);
  i64 m = (i64)(b & ((1ull << 52) - 1));
  if (bexp == 0) {
    q = -1074;
  } else {
    m |= (1ll << 52);
    q = bexp - 1075;
  }
  P = (b >> 63) ? -m : m;
}

// round-half-even of P / 2^sh, 1 <= sh <= 62
__host__ __device__ inline i64 rne_shift(i64 P, int sh) {
  i64 fl = P >> sh;  // arithmetic shift: floor
  i64 rem = P - (fl << sh);
  i64 half = 1ll << (sh - 1);
  if (rem > half || (rem == half && (fl & 1))) fl += 1;
  return fl;
}

// next digit of the residual (P, q) on the grid 2^wexp; updates P
__host__ __device__ inline int next_digit(i64& P, int q, int wexp) {
  if (P == 0) return 0;
  int sh = wexp - q;
  if (sh <= 0) {
    i64 d = P << (-sh);
    P = 0;
    return (int)d;
  }
  if (sh > 60) return 0;  // |P| < 2^54, so |P / 2^sh| < 1/2
  i64 d = rne_shift(P, sh);
  P -= d << sh;
  return (int)d;
}

__device__ inline __nv_bfloat16 digit_bf16(int d) { return __float2bfloat16_rn((float)d); }

// P 2^q as a double for |P| < 2^53, assembled from its fields with integer instructions
// when the result is normal (ldexp otherwise)
__device__ __forceinline__ double exact_double(i64 P, int q) {
  if (P == 0) return 0.0;
  const u64 a = P < 0 ? (u64)0 - (u64)P : (u64)P;
  const int L = 64 - __clzll((long long)a);
  const int E = L - 1 + q;
  if (L <= 53 && E >= -1022 && E <= 1023)
    return __longlong_as_double((long long)((P < 0 ? (1ull << 63) : 0ull) | ((u64)(E + 1023) << 52) |
                                            ((a << (53 - L)) & ((1ull << 52) - 1))));
  return ldexp((double)P, q);
}

// Digits of x = P 2^q on the fixed grid of exponent e, computed plane by plane instead of
// through the sequential remainder.  With b = DIGIT_BITS: after r round-half-even digits
// the partial sum is the round-half-even multiple Q_r 2^(s_r) of P, s_r = e + 1 - b r - q
// (a tie leaves Q_r even, since Q_r = 2^b Q_(r-1) + d_r with d_r chosen even), so
// d_r = Q_r - 2^b Q_(r-1); as |d_r| <= 2^(b-1) it depends only on Q_r mod 2^(b+1) and
// Q_(r-1) mod 2 (Q_0 = 0 because |x| < 2^e).  The digits of -x are those of x negated.
//
// The value is placed once on the grid one bit below the last plane's LSB:
// A = |P| 2^(q - g), g = e - b K (bits shifted out only set a sticky flag; A < 2^(b K),
// which fits 128 bits for K <= MAX_PLANES).  Plane r = K - j then has its LSB at bit
// p = 1 + b j of A, a constant in the unrolled loop, and its sticky bit is "trailing zeros
// of A < p - 1".  L lanes (values) share e and K; emit(r, d) receives plane r's digits of
// all lanes, from r = 1 down to r = K.
template <int L, class Emit>
__device__ __forceinline__ void for_each_digit(const i64 (&P)[L], const int (&q)[L], int e, int K, Emit emit) {
  unsigned __int128 A[L];
  bool neg[L], sticky0[L];
  int tz[L];
  unsigned par[L];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    neg[l] = P[l] < 0;
    const u64 a = neg[l] ? (u64)0 - (u64)P[l] : (u64)P[l];
    A[l] = 0;
    sticky0[l] = false;
    if (a != 0) {
      const int sh = q[l] - (e - DIGIT_BITS * K);
      if (sh >= 0) {
        // |x| < 2^e bounds bitlen(a) + sh by b K <= 128, so the shift stays in range
        A[l] = sh < 128 ? (unsigned __int128)a << sh : (unsigned __int128)0;
      } else if (sh > -64) {
        A[l] = a >> (-sh);
        sticky0[l] = (a & ((1ull << (-sh)) - 1)) != 0;
      } else {
        sticky0[l] = true;
      }
    }
    const u64 lo = (u64)A[l], hi = (u64)(A[l] >> 64);
    tz[l] = lo ? __ffsll((long long)lo) - 1 : (hi ? 63 + __ffsll((long long)hi) : 128);
    par[l] = 0;
  }
#pragma unroll
  for (int j = MAX_PLANES - 1; j >= 0; --j) {
    if (j < K) {
      const int p = 1 + DIGIT_BITS * j;
      int d[L];
#pragma unroll
      for (int l = 0; l < L; ++l) {
        constexpr unsigned MASK = (2u << DIGIT_BITS) - 1u;   // b + 1 bits: Q_r mod 2^(b+1)
        const unsigned tq = (unsigned)(A[l] >> p) & MASK;
        const unsigned rb = (unsigned)(A[l] >> (p - 1)) & 1u;
        const unsigned st = (sticky0[l] || tz[l] < p - 1) ? 1u : 0u;
        const unsigned qr = (tq + (rb & (st | (tq & 1u)))) & MASK;
        int v = (int)((qr - (par[l] << DIGIT_BITS)) & MASK);
        v = v >= (1 << DIGIT_BITS) ? v - (2 << DIGIT_BITS) : v;
        d[l] = neg[l] ? -v : v;
        par[l] = qr & 1u;
      }
      emit(K - j, d);
    }
  }
}

// ---------------------------------------------------------------------------
// Double-double arithmetic (FMA-based TwoProduct; explicit roundings)
// ---------------------------------------------------------------------------
struct dd {
  double h, l;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
  double x = __dadd_rn(a, b);
  double z = __dsub_rn(x, a);
  double y = __dadd_rn(__dsub_rn(a, __dsub_rn(x, z)), __dsub_rn(b, z));
  return {x, y};
}

__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  double x = __dadd_rn(a, b);
  double y = __dsub_rn(b, __dsub_rn(x, a));
  return {x, y};
}

__device__ __forceinline__ dd two_prod(double a, double b) {
  double p = __dmul_rn(a, b);
  double e = __fma_rn(a, b, -p);
  return {p, e};
}

// accurate double-double addition (same formula as the oracle's dd_add)
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.h, b.h);
  dd t = two_sum(a.l, b.l);
  double se = __dadd_rn(s.l, t.h);
  dd u = fast_two_sum(s.h, se);
  double ue = __dadd_rn(u.l, t.l);
  return fast_two_sum(u.h, ue);
}

__device__ __forceinline__ dd dd_add_d(dd a, double b) {
  dd s = two_sum(a.h, b);
  double se = __dadd_rn(s.l, a.l);
  return fast_two_sum(s.h, se);
}

__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.h, b);
  double pe = __dadd_rn(p.l, __dmul_rn(a.l, b));
  return fast_two_sum(p.h, pe);
}

__device__ __forceinline__ dd dd_div(dd a, dd b) {
  double q1 = __ddiv_rn(a.h, b.h);
  dd p = dd_mul_d(b, q1);
  dd r = dd_add(a, dd{-p.h, -p.l});
  double q2 = __ddiv_rn(r.h, b.h);
  return fast_two_sum(q1, q2);
}

// exact int64 -> double-double, scaled by 2^ex (exact unless it underflows)
__device__ __forceinline__ dd i64_to_dd_scaled(i64 R, int ex) {
  double h = __ll2double_rn(R);
  i64 rest = R - __double2ll_rn(h);
  double l = __ll2double_rn(rest);
  if (ex >= -1022 + 64 && ex <= 1023 - 64) {
    double s = pow2(ex);
    return {__dmul_rn(h, s), __dmul_rn(l, s)};
  }
  return {ldexp(h, ex), ldexp(l, ex)};
}

// warp and block reductions of double-double values
__device__ __forceinline__ dd warp_sum_dd(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    v = dd_add(v, w);
  }
  return v;
}

}  // namespace frx
