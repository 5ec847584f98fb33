// Element-wise and per-column kernels of one refinement iteration (Alg. 1, Sec. 3):
// recombination of the exact slice-product groups into double-double, r and lambda
// (Alg. 1), the residual V - X^(1) diag(lambda) (inside W), the correction E~
// (with the Ogita-Aishima cluster rule) and the update by pair arithmetic
// (Sec. 2.2).
#include "frx_internal.cuh"
#include "grouped.cuh"
#include "intround.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "refine_kernels.cuh"

namespace frx {

// value of entry (i, j) of an Ozaki product from its int64 groups (least significant first),
// as a double-double; general path (any number of groups)
__device__ __forceinline__ int tlast_of(const GroupArgs& ga, int g) {
  int t1 = 2 + (g + 1) * ga.gs - 1;
  return t1 < ga.tmax ? t1 : ga.tmax;
}

// fields of a GroupArgs from its device descriptor (plan-driven products)
__device__ __forceinline__ GroupArgs resolve(GroupArgs g) {
  if (g.dyn) {
    const GemmDesc& d = *g.dyn;
    g.groups = d.active ? d.groups : 0;
    g.gs = d.gs;
    g.tmax = d.tmax;
    g.word32 = d.word32;
    int t0 = 2 + g.gs - 1 < g.tmax ? 2 + g.gs - 1 : g.tmax;
    g.exact128 = g.groups > 0 && (g.word32 ? 31 : 62) + DIGIT_BITS * (g.tmax - t0) + 1 <= 127;
  }
  return g;
}

__device__ __forceinline__ i64 group_word(const GroupArgs& ga, int g, int64_t i, int64_t j) {
  int64_t idx = g * ga.ogs + j * ga.ldo + i;
  return ga.word32 ? (i64) reinterpret_cast<const int32_t*>(ga.out)[idx] : reinterpret_cast<const i64*>(ga.out)[idx];
}

__device__ __forceinline__ dd gather_dd_general(const GroupArgs& ga, int64_t i, int64_t j, int eLi, int eRj) {
  dd acc{0.0, 0.0};
  if (eLi == EZERO || eRj == EZERO) return acc;
  for (int g = ga.groups - 1; g >= 0; --g) {
    i64 R = group_word(ga, g, i, j);
    if (R == 0) continue;
    acc = dd_add(acc, i64_to_dd_scaled(R, eLi + eRj + 2 - DIGIT_BITS * tlast_of(ga, g)));
  }
  return acc;
}

__device__ __forceinline__ int clz128(u128 a) {
  u64 hi = (u64)(a >> 64), lo = (u64)a;
  return hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
}

// round-to-nearest-even of a 128-bit integer to a double
__device__ __forceinline__ double i128_to_double_rn(i128 N) {
  if (N == 0) return 0.0;
  bool neg = N < 0;
  u128 a = neg ? (u128)(-N) : (u128)N;
  double r;
  if ((a >> 63) == 0) {
    r = __ull2double_rn((u64)a);
  } else {
    int sh = (127 - clz128(a)) - 62;                 // keep 63 bits; the rest is a sticky bit
    u64 v = (u64)(a >> sh);
    if ((a & (((u128)1 << sh) - 1)) != 0) v |= 1ull;
    r = __dmul_rn(__ull2double_rn(v), pow2(sh));
  }
  return neg ? -r : r;
}

// integer value of an integer-valued double
__device__ __forceinline__ i128 double_to_i128(double h) {
  u64 b = (u64)__double_as_longlong(h);
  int bexp = (int)((b >> 52) & 0x7ff);
  if (bexp == 0) return 0;
  int e = bexp - 1075;
  u64 m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  u128 v = e >= 0 ? ((u128)m << e) : (u128)(m >> (-e));
  return (b >> 63) ? -(i128)v : (i128)v;
}

// sum_g R_g 2^(b (tlast[G-1] - tlast[g])) (b = DIGIT_BITS), exact (caller checks ga.exact128)
__device__ __forceinline__ i128 combine_groups(const GroupArgs& ga, int64_t i, int64_t j) {
  if (ga.word32 && ga.groups <= 16) {
    // one int32 plane per anti-diagonal: all loads issued first, then Horner with the
    // constant shift b in int64 chunks of four planes (|chunk| < 2^(31 + 3b + 1) <= 2^56),
    // merged in 128 bits
    const int32_t* p = reinterpret_cast<const int32_t*>(ga.out) + j * ga.ldo + i;
    int32_t v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = q < ga.groups ? __ldg(p + q * ga.ogs) : 0;
    i128 N = 0;
#pragma unroll
    for (int g = 0; g < 16; g += 4) {
      if (g >= ga.groups) break;
      int len = ga.groups - g < 4 ? ga.groups - g : 4;
      i64 c = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < len) c = (c << DIGIT_BITS) + (i64)v[g + q];
      N = g ? (N << (DIGIT_BITS * len)) + (i128)c : (i128)c;
    }
    return N;
  }
  if (ga.word32) {
    const int32_t* p = reinterpret_cast<const int32_t*>(ga.out) + j * ga.ldo + i;
    i128 N = 0;
    for (int g = 0; g < ga.groups; ++g) N = (N << DIGIT_BITS) + (i128)p[g * ga.ogs];
    return N;
  }
  i128 N = 0;
  for (int g = 0; g < ga.groups; ++g) {
    if (g) N <<= DIGIT_BITS * (tlast_of(ga, g) - tlast_of(ga, g - 1));
    N += (i128)group_word(ga, g, i, j);
  }
  return N;
}

// int32 planes in chunks of at most W32_CHUNK (|chunk| < 2^(31 + b (W32_CHUNK - 1) + 1) <= 2^120):
// each chunk is exact in 128 bits and converted to a double-double; chunks are added most
// significant first
constexpr int W32_CHUNK = (120 - 32) / DIGIT_BITS + 1;
__device__ __forceinline__ dd gather_dd_w32_chunked(const GroupArgs& ga, int64_t i, int64_t j, int eLi, int eRj) {
  dd acc{0.0, 0.0};
  if (eLi == EZERO || eRj == EZERO) return acc;
  const int32_t* p = reinterpret_cast<const int32_t*>(ga.out) + j * ga.ldo + i;
  int g = 0;
  while (g < ga.groups) {
    int len = ga.groups - g < W32_CHUNK ? ga.groups - g : W32_CHUNK;
    i128 N = 0;
    for (int q = 0; q < len; q += 4) {
      int l4 = len - q < 4 ? len - q : 4;
      i64 c = 0;
      for (int u = 0; u < l4; ++u) c = (c << DIGIT_BITS) + (i64)p[(g + q + u) * ga.ogs];
      N = q ? (N << (DIGIT_BITS * l4)) + (i128)c : (i128)c;
    }
    int ex = eLi + eRj + 2 - DIGIT_BITS * (g + len + 1);   // plane g has t = g + 2
    double h = i128_to_double_rn(N);
    double l = i128_to_double_rn(N - double_to_i128(h));
    dd part = (ex >= -1022 + 130 && ex <= 1023 - 130) ? dd{__dmul_rn(h, pow2(ex)), __dmul_rn(l, pow2(ex))}
                                                       : dd{ldexp(h, ex), ldexp(l, ex)};
    acc = g ? dd_add(acc, part) : part;
    g += len;
  }
  return acc;
}

__device__ __forceinline__ dd gather_dd(const GroupArgs& ga, int64_t i, int64_t j, int eLi, int eRj) {
  if (!ga.exact128)
    return ga.word32 ? gather_dd_w32_chunked(ga, i, j, eLi, eRj) : gather_dd_general(ga, i, j, eLi, eRj);
  if (eLi == EZERO || eRj == EZERO || ga.groups == 0) return dd{0.0, 0.0};
  i128 N = combine_groups(ga, i, j);
  double h = i128_to_double_rn(N);
  double l = i128_to_double_rn(N - double_to_i128(h));
  int ex = eLi + eRj + 2 - DIGIT_BITS * ga.tmax;
  if (ex >= -1022 + 130 && ex <= 1023 - 130) {
    double sc = pow2(ex);
    return {__dmul_rn(h, sc), __dmul_rn(l, sc)};
  }
  return {ldexp(h, ex), ldexp(l, ex)};
}

// RN of the entry as a single double
__device__ __forceinline__ double gather_d(const GroupArgs& ga, int64_t i, int64_t j, int eLi, int eRj) {
  if (!ga.exact128)
    return (ga.word32 ? gather_dd_w32_chunked(ga, i, j, eLi, eRj) : gather_dd_general(ga, i, j, eLi, eRj)).h;
  if (eLi == EZERO || eRj == EZERO || ga.groups == 0) return 0.0;
  double h = i128_to_double_rn(combine_groups(ga, i, j));
  int ex = eLi + eRj + 2 - DIGIT_BITS * ga.tmax;
  if (ex >= -1022 + 130 && ex <= 1023 - 130) return __dmul_rn(h, pow2(ex));
  return ldexp(h, ex);
}

__device__ __forceinline__ int bitlen128(i128 v) {
  u128 a = v < 0 ? (u128)(-v) : (u128)v;
  return a == 0 ? 0 : 128 - clz128(a);
}

// RN(S * 2^ex) for an exact 128-bit S
__device__ __forceinline__ double i128_scaled_rn(i128 S, int ex) {
  double h = i128_to_double_rn(S);
  if (ex >= -1022 + 130 && ex <= 1023 - 130) return __dmul_rn(h, pow2(ex));
  return ldexp(h, ex);
}

// integer m with x = m * 2^G (x on the grid 2^G, |m| < 2^62)
__device__ __forceinline__ i64 grid_mantissa(double x, int G) {
  if (is_zero(x)) return 0;
  i64 P;
  int q;
  decompose(x, P, q);
  return q >= G ? (P << (q - G)) : (P >> (G - q));
}

__device__ __forceinline__ i128 warp_sum_i128(i128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u64 lo = (u64)v, hi = (u64)((u128)v >> 64);
    u64 lo2 = __shfl_xor_sync(0xffffffffu, lo, o), hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
    v += (i128)(((u128)hi2 << 64) | (u128)lo2);
  }
  return v;
}

// Minimum resident blocks per SM requested from the register allocator by the element-wise
// kernels; tuning constants, measured on GB300.
#ifndef FRX_MINB_RESIDUAL
#define FRX_MINB_RESIDUAL 3
#endif
#ifndef FRX_MINB_CORRECTION
#define FRX_MINB_CORRECTION 3
#endif
#ifndef FRX_MINB_UPDATE
#define FRX_MINB_UPDATE 3
#endif
constexpr int RPT = 2;   // launch sizing: threads cover n / RPT rows (at most ELEM_THREADS)
constexpr int ELEM_THREADS = 256;

__host__ __device__ inline int elem_threads(int64_t n) {
  int64_t t = (n + RPT - 1) / RPT;
  t = (t + 31) / 32 * 32;
  return (int)(t < 32 ? 32 : (t > ELEM_THREADS ? ELEM_THREADS : t));
}

// the int32 anti-diagonal planes of entry (i, j) (at most MP; zero beyond groups)
template <int MP>
__device__ __forceinline__ void load_planes(const GroupArgs& g, int64_t i, int64_t j, bool valid, int32_t (&v)[MP]) {
  const int32_t* p = reinterpret_cast<const int32_t*>(g.out) + j * g.ldo + i;
#pragma unroll
  for (int q = 0; q < MP; ++q) v[q] = (valid && q < g.groups) ? __ldg(p + q * g.ogs) : 0;
}

// Per-thread asynchronous copies into shared memory (cp.async): the element-wise kernels keep
// the loads of the next PIPE - 1 row trips in flight while they work on the current one.  Each
// thread reads back only what it copied, so a wait on its own copy groups is all the ordering
// needed.  A copy with ok = false reads nothing and fills zeros (src must still be a valid
// address).
constexpr int PIPE = 3;

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// sum_q v_q 2^(b (groups - 1 - q)) exactly (b = DIGIT_BITS; |result| < 2^127 when the product's
// exact128 flag holds): Horner in int64 chunks of four planes, merged in 128 bits
template <int MP>
__device__ __forceinline__ i128 horner(const int32_t (&v)[MP], int groups) {
  i128 N = 0;
#pragma unroll
  for (int g = 0; g < MP; g += 4) {
    if (g < groups) {
      const int len = groups - g < 4 ? groups - g : 4;
      i64 c = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < len && g + q < MP) c = (c << DIGIT_BITS) + (i64)v[g + q];
      N = g ? (N << (DIGIT_BITS * len)) + (i128)c : (i128)c;
    }
  }
  return N;
}

constexpr int MP_RESIDUAL = 16;   // planes kept in registers by the fast paths
constexpr int MP_UPDATE = 12;

// N 2^ex as a double-double (h = RN(N 2^ex), l = RN of the rest) on the integer pipes;
// false when a part would be subnormal or overflow
__device__ __forceinline__ bool dd_from_i128(i128 N, int ex, dd& out) {
  double h;
  if (!rn_scaled(N, ex, h)) return false;
  if (is_zero(h)) {
    out = dd{0.0, 0.0};
    return true;
  }
  i64 P;
  int q;
  decompose(h, P, q);
  const i128 R = q >= ex ? N - ((i128)P << (q - ex)) : (i128)0;
  double l;
  if (!rn_scaled(R, ex, l)) return false;
  out = dd{h, l};
  return true;
}

__global__ void __launch_bounds__(256) k_groups_to_dd(GroupArgs ga, const int32_t* __restrict__ eL,
                                                      const int32_t* __restrict__ eR, int64_t M, int64_t N,
                                                      double* __restrict__ Ch, int64_t ldh, double* __restrict__ Cl,
                                                      int64_t ldl) {
  int64_t i = (int64_t)blockIdx.y * 256 + threadIdx.x;
  int64_t j = blockIdx.x;   // columns on x: N may exceed 65535
  if (i >= M) return;
  ga = resolve(ga);
  const int ei = eL[i], ej = eR[j];
  dd v{0.0, 0.0};
  bool done = ei == EZERO || ej == EZERO || ga.groups == 0;
  if (!done && ga.word32 && ga.exact128 && ga.groups <= 16) {
    int32_t pl[16];
    load_planes<16>(ga, i, j, true, pl);
    const i128 S = horner<16>(pl, ga.groups);
    const int ex = ei + ej + 2 - DIGIT_BITS * ga.tmax;
    done = Cl ? dd_from_i128(S, ex, v) : rn_scaled(S, ex, v.h);   // the low word only when asked
  }
  if (!done) v = gather_dd(ga, i, j, ei, ej);
  Ch[i + j * ldh] = v.h;
  if (Cl) Cl[i + j * ldl] = v.l;
}

__device__ dd block_sum_dd(dd v, dd* red) {
  v = warp_sum_dd(v);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    v = lane < nw ? red[lane] : dd{0.0, 0.0};
    v = warp_sum_dd(v);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  dd r = red[0];
  __syncthreads();
  return r;
}

__device__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    v = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

__device__ u64 block_max_u64(u64 v, u64* red) {
  for (int o = 16; o > 0; o >>= 1) {
    u64 w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    v = lane < nw ? red[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) {
      u64 x = __shfl_xor_sync(0xffffffffu, v, o);
      v = x > v ? x : v;
    }
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  u64 r = red[0];
  __syncthreads();
  return r;
}

// ---- r, lambda, Res (inner part): one block per column j --------------------------------
// smem: n double-doubles (V column).  x^T x is exact in integers (X1 lies on the grid
// 2^(f_j + beta - 53)); x^T v is accumulated with TwoProduct/TwoSum (Dot2 form).
__device__ __noinline__ void residual_general(ResidualArgs a, int64_t jcol) {
  extern __shared__ __align__(16) dd vcol[];
  __shared__ dd redd[32];
  __shared__ u64 redu[32];
  __shared__ i128 redi[32];
  const int64_t j = jcol;
  const int64_t n = a.n;
  const int fj = a.f[j];
  const int gj = fj + a.beta - 53;
  const double* x = a.X1 + j * a.ld1;
  const bool exact = a.V.exact128 != 0;
  i128* ncol = reinterpret_cast<i128*>(vcol);   // exact V entries when exact128
  i128 nn_int = 0;
  double s = 0.0, err = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    dd v;
    int ei = a.eA[i];
    if (exact) {
      i128 N = (ei == EZERO || a.V.groups == 0) ? (i128)0 : combine_groups(a.V, i, j);
      ncol[i] = N;
      int ex = ei + fj + 2 - DIGIT_BITS * a.V.tmax;
      double h = i128_to_double_rn(N);
      double l = i128_to_double_rn(N - double_to_i128(h));
      if (ex >= -1022 + 130 && ex <= 1023 - 130) {
        double sc = pow2(ex);
        v = {__dmul_rn(h, sc), __dmul_rn(l, sc)};
      } else {
        v = {ldexp(h, ex), ldexp(l, ex)};
      }
    } else {
      v = gather_dd(a.V, i, j, ei, fj);
      vcol[i] = v;
    }
    if (a.Vh) a.Vh[i + j * n] = v.h;
    if (a.Vl) a.Vl[i + j * n] = v.l;
    double xi = x[i];
    i64 m = grid_mantissa(xi, gj);
    nn_int += (i128)m * (i128)m;
    dd p = two_prod(xi, v.h);
    dd t = two_sum(s, p.h);
    s = t.h;
    err = __dadd_rn(err, __dadd_rn(t.l, __dadd_rn(p.l, __dmul_rn(xi, v.l))));
  }
  // block reductions
  nn_int = warp_sum_i128(nn_int);
  {
    dd w{s, err};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double s2 = __shfl_xor_sync(0xffffffffu, w.h, o), e2 = __shfl_xor_sync(0xffffffffu, w.l, o);
      dd t = two_sum(w.h, s2);
      w = {t.h, __dadd_rn(__dadd_rn(w.l, e2), t.l)};
    }
    int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
      redi[wi] = nn_int;
      redd[wi] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int nw = blockDim.x >> 5;
      i128 tot = 0;
      dd acc{0.0, 0.0};
      for (int k = 0; k < nw; ++k) {
        tot += redi[k];
        dd t = two_sum(acc.h, redd[k].h);
        acc = {t.h, __dadd_rn(__dadd_rn(acc.l, redd[k].l), t.l)};
      }
      redi[0] = tot;
      redd[0] = fast_two_sum(acc.h, acc.l);
    }
    __syncthreads();
  }
  const i128 nt = redi[0];
  const dd dv = redd[0];
  double nh = i128_to_double_rn(nt);
  double nl = i128_to_double_rn(nt - double_to_i128(nh));
  const double sc = pow2(2 * gj);
  const dd nn{__dmul_rn(nh, sc), __dmul_rn(nl, sc)};
  const double lam = dd_div(dv, nn).h;
  const double r = dd_add_d(dd{-nn.h, -nn.l}, 1.0).h;
  if (threadIdx.x == 0) {
    a.lam[j] = lam;
    a.r[j] = r;
  }
  i64 L = 0;
  int qL = 0;
  if (!is_zero(lam)) decompose(lam, L, qL);
  u64 mx = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double xi = x[i];
    double res;
    bool done = false;
    if (exact) {
      // Res = N 2^c - (m L) 2^(gj + qL), exact in 128 bits after alignment
      int ei = a.eA[i];
      i128 N = ncol[i];
      i128 ML = (i128)grid_mantissa(xi, gj) * (i128)L;
      int c = ei + fj + 2 - DIGIT_BITS * a.V.tmax;
      int d = (gj + qL) - c;
      if (ei == EZERO) {
        N = 0;
        d = 0;
        c = gj + qL;
      }
      if (d >= 0 && bitlen128(ML) + d <= 125 && bitlen128(N) <= 125) {
        res = i128_scaled_rn(N - (ML << d), c);
        done = true;
      } else if (d < 0 && bitlen128(N) - d <= 125 && bitlen128(ML) <= 125) {
        res = i128_scaled_rn((N << (-d)) - ML, gj + qL);
        done = true;
      }
    }
    if (!done) {
      dd v = exact ? gather_dd_general(a.V, i, j, a.eA[i], fj) : vcol[i];
      dd p = two_prod(xi, lam);
      dd t = two_sum(v.h, -p.h);
      res = __dadd_rn(t.h, __dadd_rn(t.l, __dsub_rn(v.l, p.l)));
    }
    a.Res[i + j * a.ldr] = res;
    u64 ab = double_to_bits(res) & 0x7fffffffffffffffull;
    mx = ab > mx ? ab : mx;
  }
  mx = block_max_u64(mx, redu);
  if (threadIdx.x == 0) a.h[j] = mx == 0 ? EZERO : ceil_log2_absbits(mx);
}

// Integer fast path of r, lambda, Res for int32 planes (at most 16) that combine exactly in 128
// bits.  One pass over the rows forms each V entry N_i 2^(c_i) (kept in shared memory), x^T x
// exactly, and x^T v on a fixed grid: each warp keeps an anchor T_w, the largest bound 2^T_w on
// its terms so far, and accumulates every term truncated once on the grid 2^(T_w + log2 n - 126)
// (when T_w grows, the partial sums move to the coarser grid, truncated once more).  With T the
// final largest bound, the sum's error stays below 2^(T + 2 log2 n - 125), and every partial sum
// fits 128 bits.  A second pass rounds Res = V - x lambda once from its exact integer value.
__device__ __forceinline__ i128 shift_down(i128 v, int d) { return d >= 127 ? (i128)0 : (v >> d); }

// The residual's first pass streams x_i, eA_i and the planes through a two-stage copy
// pipeline placed after the V column in dynamic shared memory (the second pass streams x_i and
// eA_i through it again); blocks of 256 threads while the column and the stages fit, else 128.
constexpr int PIPE_R = 2;
constexpr size_t RES_SMEM_MAX = RESIDUAL_SMEM_MAX;

__host__ __device__ inline size_t residual_pipe_smem(int threads) {
  return (size_t)PIPE_R * threads * (sizeof(double) + (1 + MP_RESIDUAL) * sizeof(int32_t));
}
__host__ __device__ inline int residual_threads(int64_t n) {
  const int t = elem_threads(n);
  return sizeof(dd) * (size_t)n + residual_pipe_smem(t) <= RES_SMEM_MAX ? t : 128;
}
__host__ __device__ inline size_t residual_smem(int64_t n, int threads) {
  return sizeof(dd) * (size_t)n + residual_pipe_smem(threads);
}

// debug copies of V = N 2^ex as double-doubles
__device__ __noinline__ void write_v_copies(const ResidualArgs& a, i128 N, int ex, int64_t at) {
  const double h = i128_to_double_rn(N), l = i128_to_double_rn(N - double_to_i128(h));
  const dd vd = (ex >= -1022 + 130 && ex <= 1023 - 130) ? dd{__dmul_rn(h, pow2(ex)), __dmul_rn(l, pow2(ex))}
                                                        : dd{ldexp(h, ex), ldexp(l, ex)};
  if (a.Vh) a.Vh[at] = vd.h;
  if (a.Vl) a.Vl[at] = vd.l;
}

__device__ __forceinline__ void residual_body(ResidualArgs a, unsigned bx, unsigned) {
  if (a.done && *a.done) return;
  a.V = resolve(a.V);
  if (a.beta_dyn) a.beta = *a.beta_dyn;
  if (!(a.V.word32 && a.V.exact128 && a.V.groups <= MP_RESIDUAL)) {
    residual_general(a, bx);
    return;
  }
  extern __shared__ __align__(16) dd vcol[];
  i128* ncol = reinterpret_cast<i128*>(vcol);
  __shared__ u64 redu[32];
  __shared__ i128 redi[32];
  __shared__ int redt[32];
  __shared__ int redb[32][4];
  const int64_t j = bx;
  const int64_t n = a.n;
  const int fj = a.f[j];
  const int gj = fj + a.beta - 53;
  const int cbase = fj + 2 - DIGIT_BITS * a.V.tmax;   // c_i = eA_i + cbase
  const double* x = a.X1 + j * a.ld1;
  const int nb = a.V.groups;
  int lg = 0;
  while (((int64_t)1 << lg) < n) ++lg;
  u128 nn = 0;
  i128 acc = 0;                 // x^T v in units of 2^(aw + lg - 126 + gj)
  int aw = -(1 << 30);          // the warp's anchor (warp-uniform)
  int tb = -(1 << 30);
  int bmmax = 0, bnmax = 0, emin = 1 << 30, emax = -(1 << 30);   // bounds for pass 2
  // pass 1 (block-uniform trips: the anchor is a warp maximum)
  const int B = blockDim.x, tid = threadIdx.x;
  double* sx = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(vcol) + sizeof(dd) * n);   // [PIPE_R][B]
  int32_t* si = reinterpret_cast<int32_t*>(sx + PIPE_R * B);              // [PIPE_R][1 + MP_RESIDUAL][B]
  const int32_t* pcol = reinterpret_cast<const int32_t*>(a.V.out) + j * a.V.ldo;
  const int64_t ogs = a.V.ogs;
  auto issue = [&](int64_t i, int st) {
    const bool ok = i < n;
    const int64_t ic = ok ? i : 0;
    cp_async8(sx + st * B + tid, x + ic, ok);
    int32_t* d = si + st * (1 + MP_RESIDUAL) * B + tid;
    cp_async4(d, a.eA + ic, ok);
    const int32_t* p = pcol + ic;
#pragma unroll
    for (int q = 0; q < MP_RESIDUAL; ++q) {
      if (q >= nb) break;
      d += B;
      cp_async4(d, p, ok);
      p += ogs;
    }
    cp_async_commit();
  };
#pragma unroll
  for (int st = 0; st < PIPE_R - 1; ++st) issue(tid + (int64_t)st * B, st);
  int st = 0, sti = PIPE_R - 1;   // stage of the current trip, stage the next copies go to
  for (int64_t i = tid, i0 = 0; i0 < n; i += B, i0 += B) {
    issue(i + (int64_t)(PIPE_R - 1) * B, sti);
    sti = sti == PIPE_R - 1 ? 0 : sti + 1;
    cp_async_wait<PIPE_R - 1>();
    const int cur = st;
    st = st == PIPE_R - 1 ? 0 : st + 1;
    const bool ok = i < n;
    const int32_t* d = si + cur * (1 + MP_RESIDUAL) * B + tid;
    const double xv = ok ? sx[cur * B + tid] : 0.0;
    const int ei = ok ? d[0] : EZERO;
    int32_t v[MP_RESIDUAL];
#pragma unroll
    for (int q = 0; q < MP_RESIDUAL; ++q) v[q] = q < nb ? d[(1 + q) * B] : 0;
    i128 N = 0;
    i64 m = 0;
    int t = -(1 << 30);
    if (ok) {
      N = ei == EZERO ? (i128)0 : horner<MP_RESIDUAL>(v, nb);
      ncol[i] = N;
      if (a.Vh || a.Vl) write_v_copies(a, N, ei + cbase, i + j * n);
      m = grid_mantissa(xv, gj);
      const u64 am = m < 0 ? (u64)0 - (u64)m : (u64)m;
      nn += (u128)am * am;
      const int bm = am ? bitlen_u64(am) : 0;
      const int bn = N != 0 ? bitlen_bound_i128(N) : 0;
      bmmax = bm > bmmax ? bm : bmmax;
      bnmax = bn > bnmax ? bn : bnmax;
      if (ei != EZERO) {
        emin = ei < emin ? ei : emin;
        emax = ei > emax ? ei : emax;
      }
      if (N != 0 && m != 0) {
        t = bm + bn + ei + cbase;
        tb = t > tb ? t : tb;
      }
    }
    int tw = t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tw = max(tw, __shfl_xor_sync(0xffffffffu, tw, o));
    if (tw > aw) {
      acc = aw > -(1 << 29) ? shift_down(acc, tw - aw) : (i128)0;
      aw = tw;
    }
    if (t > -(1 << 29)) acc += mul_shift(m, N, aw + lg - 126 - (ei + cbase));
  }
  cp_async_wait<0>();
  // block reductions: x^T x (exact) and the term bound
  {
    u64 lo = (u64)nn, hi = (u64)(nn >> 64);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const u64 lo2 = __shfl_xor_sync(0xffffffffu, lo, o), hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
      const u128 sum = (((u128)hi << 64) | lo) + (((u128)hi2 << 64) | lo2);
      lo = (u64)sum;
      hi = (u64)(sum >> 64);
      tb = max(tb, __shfl_xor_sync(0xffffffffu, tb, o));
      bmmax = max(bmmax, __shfl_xor_sync(0xffffffffu, bmmax, o));
      bnmax = max(bnmax, __shfl_xor_sync(0xffffffffu, bnmax, o));
      emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
      redi[wi] = (i128)(((u128)hi << 64) | lo);
      redt[wi] = tb;
      redb[wi][0] = bmmax;
      redb[wi][1] = bnmax;
      redb[wi][2] = emin;
      redb[wi][3] = emax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      u128 tot = 0;
      int tm = -(1 << 30), b0 = 0, b1 = 0, e0 = 1 << 30, e1 = -(1 << 30);
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        tot += (u128)redi[k];
        tm = max(tm, redt[k]);
        b0 = max(b0, redb[k][0]);
        b1 = max(b1, redb[k][1]);
        e0 = min(e0, redb[k][2]);
        e1 = max(e1, redb[k][3]);
      }
      redi[0] = (i128)tot;
      redt[0] = tm;
      redb[0][0] = b0;
      redb[0][1] = b1;
      redb[0][2] = e0;
      redb[0][3] = e1;
    }
    __syncthreads();
  }
  const u128 nn_tot = (u128)redi[0];
  const int T = redt[0];
  bmmax = redb[0][0];
  bnmax = redb[0][1];
  emin = redb[0][2];
  emax = redb[0][3];
  __syncthreads();
  // x^T v: every warp's partial sums moved to the grid of the final bound T
  const int lsb = T + lg - 126;
  acc = aw > -(1 << 29) ? shift_down(acc, T - aw) : (i128)0;
  acc = warp_sum_i128(acc);
  {
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) redi[wi] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      i128 tot = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += redi[k];
      redi[0] = tot;
      // lambda_j = x^T v / x^T x and r_j = 1 - x^T x (double-double, once per column)
      const i128 nt = (i128)nn_tot;
      const double nh = i128_to_double_rn(nt);
      const double nl = i128_to_double_rn(nt - double_to_i128(nh));
      const double sc = pow2(2 * gj);
      const dd nnd{__dmul_rn(nh, sc), __dmul_rn(nl, sc)};
      const double dh = i128_to_double_rn(tot);
      const double dl = i128_to_double_rn(tot - double_to_i128(dh));
      const int ex = lsb + gj;
      const dd dv = (ex >= -1022 + 130 && ex <= 1023 - 130) ? dd{__dmul_rn(dh, pow2(ex)), __dmul_rn(dl, pow2(ex))}
                                                            : dd{ldexp(dh, ex), ldexp(dl, ex)};
      const double lam = T > -(1 << 29) ? dd_div(dv, nnd).h : 0.0;
      a.lam[j] = lam;
      a.r[j] = dd_add_d(dd{-nnd.h, -nnd.l}, 1.0).h;
      redu[0] = (u64)__double_as_longlong(lam);
    }
    __syncthreads();
  }
  const double lam = __longlong_as_double((long long)redu[0]);
  __syncthreads();
  // pass 2: Res = N 2^c - (m L) 2^(gj + qL), rounded once.  The aligned difference fits
  // 128 bits for every row when the block-wide bounds say so; otherwise per row.
  i64 L = 0;
  int qL = 0;
  if (!is_zero(lam)) decompose(lam, L, qL);
  const int bL = L ? bitlen_u64(L < 0 ? (u64)0 - (u64)L : (u64)L) : 0;
  const int gq = gj + qL;
  const int dmax = emax > -(1 << 29) ? gq - (emin + cbase) : 0, dmin = emax > -(1 << 29) ? gq - (emax + cbase) : 0;
  const bool safe = dmin >= -60 && dmax <= 60 && bmmax + bL + (dmax > 0 ? dmax : 0) <= 125 &&
                    bnmax + (dmin < 0 ? -dmin : 0) <= 125 && bnmax <= 125 && bmmax + bL <= 125;
  u64 mx = 0;
  // x_i and eA_i come through the first pass's stages again, one trip ahead
  auto issue2 = [&](int64_t i, int st2) {
    const bool ok = i < n;
    const int64_t ic = ok ? i : 0;
    cp_async8(sx + st2 * B + tid, x + ic, ok);
    cp_async4(si + st2 * (1 + MP_RESIDUAL) * B + tid, a.eA + ic, ok);
    cp_async_commit();
  };
#pragma unroll
  for (int q = 0; q < PIPE_R - 1; ++q) issue2(tid + (int64_t)q * B, q);
  int sc = 0, sci = PIPE_R - 1;   // stage of the current trip, stage the next copies go to
  for (int64_t i = tid, i0 = 0; i0 < n; i += B, i0 += B) {
    issue2(i + (int64_t)(PIPE_R - 1) * B, sci);
    sci = sci == PIPE_R - 1 ? 0 : sci + 1;
    cp_async_wait<PIPE_R - 1>();
    const int cur = sc;
    sc = sc == PIPE_R - 1 ? 0 : sc + 1;
    if (i >= n) continue;
    const double xi = sx[cur * B + tid];
    const int ei = si[cur * (1 + MP_RESIDUAL) * B + tid];
    const i128 N = ncol[i];
    const i128 ML = mul_i64(grid_mantissa(xi, gj), L);
    const int c = ei == EZERO ? gq : ei + cbase;
    const int d = gq - c;
    double res;
    bool done = false;
    if (safe || (d >= 0 ? (bitlen_u128(abs_i128(ML)) + d <= 125 && bitlen_u128(abs_i128(N)) <= 125)
                        : (bitlen_u128(abs_i128(N)) - d <= 125 && bitlen_u128(abs_i128(ML)) <= 125))) {
      done = d >= 0 ? rn_scaled(N - (ML << d), c, res) : rn_scaled((N << (-d)) - ML, gq, res);
    }
    if (!done) {
      const dd v = gather_dd_general(a.V, i, j, ei, fj);
      const dd p = two_prod(xi, lam);
      const dd t = two_sum(v.h, -p.h);
      res = __dadd_rn(t.h, __dadd_rn(t.l, __dsub_rn(v.l, p.l)));
    }
    a.Res[i + j * a.ldr] = res;
    const u64 ab = double_to_bits(res) & 0x7fffffffffffffffull;
    mx = ab > mx ? ab : mx;
  }
  cp_async_wait<0>();
  mx = block_max_u64(mx, redu);
  if (threadIdx.x == 0) a.h[j] = mx == 0 ? EZERO : ceil_log2_absbits(mx);
}

// ---- ||off-diagonal W||_F^2 (for the automatic cluster threshold) ------------------
__device__ __forceinline__ void w_offdiag_body(CorrectionArgs a, unsigned bx, unsigned) {
  if (a.done && *a.done) return;
  a.W = resolve(a.W);
  const int64_t j = bx;
  if (a.W.groups == 0) {
    if (threadIdx.x == 0) a.norms[a.n + j] = 0.0;
    return;
  }
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < a.n; i += blockDim.x) {
    if (i == j) continue;
    double w = gather_d(a.W, i, j, a.f[i], a.h[j]);
    s += w * w;
  }
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) a.norms[a.n + j] = s;
}

// ---- the correction: E~ column j, its exponent, ||E~||_F^2 -----------------------------------
// e_ij = w_ij / (lambda_j - lambda_i) (one IEEE division), e_jj = r_j / 2, and the
// Ogita-Aishima rule e_ij = r_ij / 2 inside clusters (|lambda_j - lambda_i| <= omega, with
// r_ij = -x_i^T x_j in double-double).  w_ij is the exact W entry rounded once on the
// integer pipes; ||E~||_F^2 (an estimate only) is accumulated in single precision.
constexpr int MP_CORRECTION = 12;

__device__ __noinline__ double gather_d_general(GroupArgs g, int64_t i, int64_t j, int eLi, int eRj) {
  return gather_d(g, i, j, eLi, eRj);
}

__device__ __forceinline__ void correction_body(CorrectionArgs a, unsigned bx, unsigned) {
  if (a.done && *a.done) return;
  a.W = resolve(a.W);
  if (a.omega_dyn) a.omega = *a.omega_dyn;
  __shared__ double red[32];
  __shared__ u64 redu[32];
  __shared__ dd redd[32];
  __shared__ int clist[64];
  __shared__ int ccount;
  const int64_t j = bx;
  const int64_t n = a.n;
  const double lj = a.lam[j];
  // |diff| <= omega compared on the bit patterns (exact for non-negative doubles; a negative
  // omega marks no cluster), which keeps the FP64 pipe for the division
  const bool any_cluster = a.omega >= 0.0;
  const u64 omega_bits = any_cluster ? double_to_bits(a.omega) : 0ull;
  const int hj = a.h[j];
  const bool have_w = a.W.groups > 0 && hj != EZERO;
  const bool fast = a.W.word32 && a.W.exact128 && a.W.groups <= MP_CORRECTION;
  const int cbase = hj + 2 - DIGIT_BITS * a.W.tmax;   // c_i = f_i + cbase
  if (threadIdx.x == 0) ccount = 0;
  __syncthreads();
  // copy slots per stage: lambda_i (double), then f_i and the planes (int32), [slot][thread]
  extern __shared__ __align__(16) unsigned char cpipe[];
  const int B = blockDim.x, tid = threadIdx.x;
  double* sl = reinterpret_cast<double*>(cpipe);                          // [PIPE][B]
  int32_t* si = reinterpret_cast<int32_t*>(sl + PIPE * B);                // [PIPE][1 + MP_CORRECTION][B]
  const int np = have_w && fast ? a.W.groups : 0;                        // planes copied per row
  const int32_t* pcol = reinterpret_cast<const int32_t*>(a.W.out) + j * a.W.ldo;
  const int64_t ogs = a.W.ogs;
  auto issue = [&](int64_t i, int st) {
    const bool ok = i < n;
    const int64_t ic = ok ? i : 0;
    cp_async8(sl + st * B + tid, a.lam + ic, ok);
    int32_t* d = si + st * (1 + MP_CORRECTION) * B + tid;
    cp_async4(d, a.f + ic, ok);
    const int32_t* p = pcol + ic;
#pragma unroll
    for (int q = 0; q < MP_CORRECTION; ++q) {
      if (q >= np) break;
      d += B;
      cp_async4(d, p, ok);
      p += ogs;
    }
    cp_async_commit();
  };
#pragma unroll
  for (int st = 0; st < PIPE - 1; ++st) issue(tid + (int64_t)st * B, st);
  float s2f = 0.f;
  double s2d = 0.0;
  u64 mx = 0;
  int st = 0, sti = PIPE - 1;   // stage of the current trip, stage the next copies go to
  for (int64_t i = tid, i0 = 0; i0 < n; i += B, i0 += B) {   // block-uniform trips
    issue(i + (int64_t)(PIPE - 1) * B, sti);
    sti = sti == PIPE - 1 ? 0 : sti + 1;
    cp_async_wait<PIPE - 1>();
    const int cur = st;
    st = st == PIPE - 1 ? 0 : st + 1;
    if (i >= n) continue;
    const double li = sl[cur * B + tid];
    const int32_t* d = si + cur * (1 + MP_CORRECTION) * B + tid;
    const int fi = d[0];
    double w = 0.0;
    if (have_w && fi != EZERO) {
      bool ok = false;
      if (fast) {
        int32_t v[MP_CORRECTION];
#pragma unroll
        for (int q = 0; q < MP_CORRECTION; ++q) v[q] = q < np ? d[(1 + q) * B] : 0;
        ok = rn_scaled(horner<MP_CORRECTION>(v, np), fi + cbase, w);
      }
      if (!ok) w = gather_d_general(a.W, i, j, fi, hj);
    }
    if (a.Wout) a.Wout[i + j * n] = w;
    double e;
    if (i == j) {
      e = a.r[j] * 0.5;
    } else {
      const double diff = __dsub_rn(lj, li);
      if (any_cluster && (double_to_bits(diff) & 0x7fffffffffffffffull) <= omega_bits) {
        const int slot = atomicAdd(&ccount, 1);
        if (slot < 64) clist[slot] = (int)i;
        else atomicOr(a.flags, FLAG_RANGE);
        e = 0.0;
      } else {
        e = __ddiv_rn(w, diff);
      }
    }
    a.E[i + j * a.lde] = e;
    float f;
    if (f32_of_double(e, 32, f)) s2f = __fmaf_rn(f, f, s2f);
    else s2d = __fma_rn(e, e, s2d);
    const u64 ab = double_to_bits(e) & 0x7fffffffffffffffull;
    mx = ab > mx ? ab : mx;
  }
  cp_async_wait<0>();
  __syncthreads();
  const int nc = ccount < 64 ? ccount : 64;
  const double* xj = a.X1 + j * a.ld1;
  for (int c = 0; c < nc; ++c) {
    const int i = clist[c];
    const double* xi = a.X1 + (int64_t)i * a.ld1;
    dd acc{0.0, 0.0};
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) acc = dd_add(acc, two_prod(xi[k], xj[k]));
    acc = block_sum_dd(acc, redd);
    if (threadIdx.x == 0) {
      const double e = -acc.h * 0.5;   // r_ij / 2
      a.E[i + j * a.lde] = e;
      s2d = __fma_rn(e, e, s2d);
      const u64 ab = double_to_bits(e) & 0x7fffffffffffffffull;
      mx = ab > mx ? ab : mx;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && nc) atomicAdd(a.ccount, nc);
  const double s2 = block_sum_d(__fma_rn((double)s2f, 0x1p-64, s2d), red);
  mx = block_max_u64(mx, redu);
  if (threadIdx.x == 0) {
    a.norms[j] = s2;
    a.eta[j] = mx == 0 ? EZERO : ceil_log2_absbits(mx);
  }
}

// dynamic shared memory of the correction's copy pipeline for blocks of `threads`
__host__ __device__ inline size_t correction_pipe_smem(int threads) {
  return (size_t)PIPE * threads * (sizeof(double) + (1 + MP_CORRECTION) * sizeof(int32_t));
}

// ---- the update: X <- RN(X1 + X1 E~) (pair arithmetic), ||X_new - X_old||_F^2 ----------------
// RN(x1 + N 2^c) for int64 N with |N 2^c| well below |x1|: x1 = P 2^q (53-bit P) and the
// sum is rounded on x1's grid with round-half-even on the combined integer.  Returns false
// when the result leaves x1's binade (then the caller takes the general path).
__device__ __forceinline__ bool add_small_rn(double x1, i64 N, int c, double& out) {
  if (is_zero(x1)) return false;
  i64 P;
  int q;
  decompose(x1, P, q);
  if (P > -(1ll << 52) && P < (1ll << 52)) return false;   // subnormal x1
  int sh = q - c;   // N 2^c = (N / 2^sh) ulps of x1
  i64 T;
  if (sh <= 0) {
    return false;     // U is not below x1's grid: general path
  } else if (sh >= 63) {
    // |N| < 2^63 <= 2^sh: |N / 2^sh| < 1; below half an ulp whenever |N| < 2^(sh - 1)
    if (sh == 63 && (N >= (1ll << 62) || N <= -(1ll << 62))) return false;
    T = P;
  } else {
    i64 fl = N >> sh;
    i64 rem = N - (fl << sh);
    i64 half = 1ll << (sh - 1);
    T = P + fl;
    if (rem > half || (rem == half && (T & 1))) T += 1;
  }
  if (T >= (1ll << 53) || T <= -(1ll << 53) || (T > -(1ll << 52) && T < (1ll << 52))) return false;
  out = __dmul_rn(__ll2double_rn(T), pow2(q));
  return true;
}

// general per-element path of the update (int64 groups, > 16 planes, wide exponent gaps,
// subnormal results): RN(x1 + U) through int64/int128 sums, else double-double
__device__ __noinline__ double update_general(const UpdateArgs& a, double x1, int64_t i, int64_t j, int ri, int ej) {
  int c = ri + ej + 2 - DIGIT_BITS * a.U.tmax;
  double xn;
  if (a.U.word32 && a.U.groups <= (62 - 31) / DIGIT_BITS + 1) {
    // the anti-diagonal planes combine exactly in int64 (31 + 8 (groups - 1) + 1 <= 63 bits)
    const int32_t* p = reinterpret_cast<const int32_t*>(a.U.out) + j * a.U.ldo + i;
    i64 N = 0;
    for (int q = 0; q < a.U.groups; ++q) N = (N << DIGIT_BITS) + (i64)p[q * a.U.ogs];
    if (add_small_rn(x1, N, c, xn)) return xn;
  }
  if (a.U.exact128) {
    i128 N = combine_groups(a.U, i, j);
    const int G = a.f[j] + a.beta - 53;
    i128 m = (i128)grid_mantissa(x1, G);
    int d = G - c;
    if (d >= 0 && bitlen128(m) + d <= 124 && bitlen128(N) <= 124) return i128_scaled_rn((m << d) + N, c);
    if (d < 0 && bitlen128(N) - d <= 124) return i128_scaled_rn(m + (N << (-d)), G);
  }
  dd u = gather_dd(a.U, i, j, ri, ej);
  dd c2 = two_sum(x1, u.h);
  double cl = __dadd_rn(u.l, c2.l);
  return __dadd_rn(c2.h, cl);
}

// (xn - xo)^2 into a single-precision partial (scaled by 2^64) when the two exponents are
// close, else into an FP64 partial; only the norm estimate of the stopping test reads it
__device__ __forceinline__ void accumulate_dx2(double xn, double xo, float& d2f, double& d2d) {
  i64 Pn, Po;
  int qn, qo;
  decompose(xn, Pn, qn);
  decompose(xo, Po, qo);
  const int dq = qn - qo;
  if (dq >= -9 && dq <= 9) {
    const i64 D = dq >= 0 ? (Pn << dq) - Po : Pn - (Po << (-dq));
    float f;
    if (f32_scaled(D, (dq >= 0 ? qo : qn) + 32, f)) {
      d2f = __fmaf_rn(f, f, d2f);
      return;
    }
  }
  const double dx = __dsub_rn(xn, xo);
  d2d = __fma_rn(dx, dx, d2d);
}

// X(:, j) <- RN(X1(:, j) + U(:, j)) (Alg. 1's update, one rounding); ||X_new - X_old||_F^2
// partial per column.  One block per column; exact sums and their rounding run on the
// integer pipes.
__device__ __forceinline__ void update_body(UpdateArgs a, unsigned bx, unsigned) {
  if (a.done && *a.done) return;
  a.U = resolve(a.U);
  if (a.beta_dyn) a.beta = *a.beta_dyn;
  __shared__ double red[32];
  // copy slots per stage: x1, x_old (doubles), then rho and the planes (int32), [slot][thread]
  extern __shared__ __align__(16) unsigned char upipe[];
  const int B = blockDim.x, tid = threadIdx.x;
  double* sx = reinterpret_cast<double*>(upipe);                          // [PIPE][2][B]
  int32_t* si = reinterpret_cast<int32_t*>(sx + PIPE * 2 * B);            // [PIPE][1 + MP_UPDATE][B]
  const int64_t j = bx;
  const int ej = a.eta[j];
  const bool none = a.U.groups == 0 || ej == EZERO;
  const bool fast = a.U.word32 && a.U.exact128 && a.U.groups <= MP_UPDATE;
  const int np = fast && !none ? a.U.groups : 0;                          // planes copied per row
  const double* x1c = a.X1 + j * a.ld1;
  double* xc = a.X + j * a.ldx;
  const int32_t* pcol = reinterpret_cast<const int32_t*>(a.U.out) + j * a.U.ldo;
  const int64_t ogs = a.U.ogs;
  const int64_t n = a.n;
  const int cshift = ej + 2 - DIGIT_BITS * a.U.tmax;                      // c = rho_i + cshift
  auto issue = [&](int64_t i, int st) {
    const bool ok = i < n;
    const int64_t ic = ok ? i : 0;
    cp_async8(sx + (st * 2 + 0) * B + tid, x1c + ic, ok);
    cp_async8(sx + (st * 2 + 1) * B + tid, xc + ic, ok);
    int32_t* d = si + st * (1 + MP_UPDATE) * B + tid;
    cp_async4(d, a.rho + ic, ok);
    const int32_t* p = pcol + ic;
#pragma unroll
    for (int q = 0; q < MP_UPDATE; ++q) {
      if (q >= np) break;
      d += B;
      cp_async4(d, p, ok);
      p += ogs;
    }
    cp_async_commit();
  };
#pragma unroll
  for (int st = 0; st < PIPE - 1; ++st) issue(tid + (int64_t)st * B, st);
  float d2f = 0.f;
  double d2d = 0.0;
  int st = 0, sti = PIPE - 1;   // stage of the current trip, stage the next copies go to
  for (int64_t i = tid, i0 = 0; i0 < n; i += B, i0 += B) {   // block-uniform trips
    issue(i + (int64_t)(PIPE - 1) * B, sti);
    sti = sti == PIPE - 1 ? 0 : sti + 1;
    cp_async_wait<PIPE - 1>();
    const int cur = st;
    st = st == PIPE - 1 ? 0 : st + 1;
    if (i >= n) continue;
    const double x1 = sx[(cur * 2 + 0) * B + tid], xo = sx[(cur * 2 + 1) * B + tid];
    const int32_t* d = si + cur * (1 + MP_UPDATE) * B + tid;
    const int ri = d[0];
    double xn = x1;
    if (!none && ri != EZERO) {
      bool done = false;
      if (fast) {
        int32_t v[MP_UPDATE];
#pragma unroll
        for (int q = 0; q < MP_UPDATE; ++q) v[q] = q < np ? d[(1 + q) * B] : 0;
        const i128 N = horner<MP_UPDATE>(v, np);
        const int c = ri + cshift;
        done = add_on_grid_rn(x1, N, c, xn) || add_exact_rn(x1, N, c, xn);
      }
      if (!done) xn = update_general(a, x1, i, j, ri, ej);
    }
    xc[i] = xn;
    accumulate_dx2(xn, xo, d2f, d2d);
  }
  cp_async_wait<0>();
  const double d2 = block_sum_d(__fma_rn((double)d2f, 0x1p-64, d2d), red);
  if (threadIdx.x == 0) a.norms[2 * a.n + j] = d2;
}

// dynamic shared memory of the update's copy pipeline for blocks of `threads`
__host__ __device__ inline size_t update_pipe_smem(int threads) {
  return (size_t)PIPE * threads * (2 * sizeof(double) + (1 + MP_UPDATE) * sizeof(int32_t));
}

// ---- single-problem kernels (one block per column) ---------------------------------
__global__ void __launch_bounds__(ELEM_THREADS, FRX_MINB_RESIDUAL) k_residual(ResidualArgs a) {
  residual_body(a, blockIdx.x, 0);
}
__global__ void __launch_bounds__(256) k_w_offdiag_norm2(CorrectionArgs a) { w_offdiag_body(a, blockIdx.x, 0); }
__global__ void __launch_bounds__(ELEM_THREADS, FRX_MINB_CORRECTION) k_correction(CorrectionArgs a) {
  correction_body(a, blockIdx.x, 0);
}
__global__ void __launch_bounds__(ELEM_THREADS, FRX_MINB_UPDATE) k_update(UpdateArgs a) {
  update_body(a, blockIdx.x, 0);
}

// ---------------------------------------------------------------------------
GroupArgs group_args(const PlaneGemm& g) {
  GroupArgs ga;
  ga.out = g.out;
  ga.ogs = g.ogs;
  ga.ldo = g.ldo;
  ga.dyn = g.dyn;
  ga.groups = g.d.active ? g.d.groups : 0;
  ga.gs = g.d.gs;
  ga.tmax = g.d.tmax;
  ga.word32 = g.d.word32;
  // |R_g| < 2^31 (int32 planes) or 2^62 (int64 groups); the combination spans
  // DIGIT_BITS (tmax - t_last(0)) more bits and must stay below 2^127
  int t0 = 2 + g.d.gs - 1 < g.d.tmax ? 2 + g.d.gs - 1 : g.d.tmax;
  ga.exact128 = ga.groups > 0 && (g.d.word32 ? 31 : 62) + DIGIT_BITS * (g.d.tmax - t0) + 1 <= 127;
  return ga;
}

int launch_groups_to_dd(const PlaneGemm& g, const int32_t* eL, const int32_t* eR, double* Ch, int64_t ldh,
                        double* Cl, int64_t ldl, cudaStream_t s) {
  if (g.M == 0 || g.N == 0) return FRX_OK;
  dim3 grid((unsigned)g.N, (unsigned)((g.M + 255) / 256));
  k_groups_to_dd<<<grid, 256, 0, s>>>(group_args(g), eL, eR, g.M, g.N, Ch, ldh, Cl, ldl);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

size_t residual_launch_smem(int64_t n, int threads) { return residual_smem(n, threads); }

int set_refine_kernel_attributes() {
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RES_SMEM_MAX));
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_grouped<ResidualArgs, residual_body, ELEM_THREADS, FRX_MINB_RESIDUAL>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RES_SMEM_MAX));
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_correction, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)correction_pipe_smem(ELEM_THREADS)));
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_grouped<CorrectionArgs, correction_body, ELEM_THREADS, FRX_MINB_CORRECTION>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)correction_pipe_smem(ELEM_THREADS)));
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)update_pipe_smem(ELEM_THREADS)));
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_grouped<UpdateArgs, update_body, ELEM_THREADS, FRX_MINB_UPDATE>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)update_pipe_smem(ELEM_THREADS)));
  return FRX_OK;
}

int launch_residual(const ResidualArgs& a0, cudaStream_t s) {
  ResidualArgs a = a0;
  a.gx = (unsigned)a.n;
  const int threads = residual_threads(a.n);
  const size_t smem = residual_smem(a.n, threads);
  if (record_launch(LK_RESIDUAL, a, a.n, threads, smem)) return FRX_OK;
  k_residual<<<(unsigned)a.n, threads, smem, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_w_offdiag_norm2(const CorrectionArgs& a0, cudaStream_t s) {
  CorrectionArgs a = a0;
  a.gx = (unsigned)a.n;
  if (record_launch(LK_W_OFFDIAG, a, a.n, 256, 0)) return FRX_OK;
  k_w_offdiag_norm2<<<(unsigned)a.n, 256, 0, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_correction(const CorrectionArgs& a0, cudaStream_t s) {
  CorrectionArgs a = a0;
  a.gx = (unsigned)a.n;
  const int threads = elem_threads(a.n);
  const size_t smem = correction_pipe_smem(threads);
  if (record_launch(LK_CORRECTION, a, a.n, threads, smem)) return FRX_OK;
  k_correction<<<(unsigned)a.n, threads, smem, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_update(const UpdateArgs& a0, cudaStream_t s) {
  UpdateArgs a = a0;
  a.gx = (unsigned)a.n;
  const int threads = elem_threads(a.n);
  const size_t smem = update_pipe_smem(threads);
  if (record_launch(LK_UPDATE, a, a.n, threads, smem)) return FRX_OK;
  k_update<<<(unsigned)a.n, threads, smem, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}


int launch_grouped_refine(int kind, const void* tab, const long long* start, int count, long long blocks,
                          int threads, size_t smem, cudaStream_t s) {
  if (blocks <= 0) return FRX_OK;
  const unsigned grid = (unsigned)blocks;
  threads = threads < 32 ? 32 : (threads > ELEM_THREADS ? ELEM_THREADS : threads);
  switch (kind) {
    case LK_RESIDUAL:
      k_grouped<ResidualArgs, residual_body, ELEM_THREADS, FRX_MINB_RESIDUAL>
          <<<grid, threads, smem, s>>>((const ResidualArgs*)tab, start, count);
      break;
    case LK_W_OFFDIAG:
      k_grouped<CorrectionArgs, w_offdiag_body, 256, 1><<<grid, 256, 0, s>>>((const CorrectionArgs*)tab, start, count);
      break;
    case LK_CORRECTION:
      k_grouped<CorrectionArgs, correction_body, ELEM_THREADS, FRX_MINB_CORRECTION>
          <<<grid, threads, correction_pipe_smem(threads), s>>>((const CorrectionArgs*)tab, start, count);
      break;
    case LK_UPDATE:
      k_grouped<UpdateArgs, update_body, ELEM_THREADS, FRX_MINB_UPDATE>
          <<<grid, threads, update_pipe_smem(threads), s>>>((const UpdateArgs*)tab, start, count);
      break;
    default:
      return FRX_E_UNSUPPORTED;
  }
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

}  // namespace frx
