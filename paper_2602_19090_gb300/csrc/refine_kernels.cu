// Element-wise and per-column kernels of one refinement iteration (Alg. 1, Sec. 3):
// recombination of the exact slice-product groups into double-double, r and lambda
// (lines 2-3), the residual V - X^(1) diag(lambda) (line 4), the correction E~
// (line 5, with the Ogita-Aishima cluster rule) and the update by pair arithmetic
// (line 6, Sec. 2.2).
#include "frx_internal.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "refine_kernels.cuh"

namespace frx {

typedef __int128 i128;
typedef unsigned __int128 u128;

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

// sum_g R_g 2^(7 (tlast[G-1] - tlast[g])), exact (caller checks ga.exact128)
__device__ __forceinline__ i128 combine_groups(const GroupArgs& ga, int64_t i, int64_t j) {
  if (ga.word32 && ga.groups <= 16) {
    // one int32 plane per anti-diagonal: all loads issued first, then Horner with the
    // constant shift 7 in int64 chunks of four planes (|chunk| < 2^(31 + 21)), merged in 128 bits
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
        if (q < len) c = (c << 7) + (i64)v[g + q];
      N = g ? (N << (7 * len)) + (i128)c : (i128)c;
    }
    return N;
  }
  if (ga.word32) {
    const int32_t* p = reinterpret_cast<const int32_t*>(ga.out) + j * ga.ldo + i;
    i128 N = 0;
    for (int g = 0; g < ga.groups; ++g) N = (N << 7) + (i128)p[g * ga.ogs];
    return N;
  }
  i128 N = 0;
  for (int g = 0; g < ga.groups; ++g) {
    if (g) N <<= DIGIT_BITS * (tlast_of(ga, g) - tlast_of(ga, g - 1));
    N += (i128)group_word(ga, g, i, j);
  }
  return N;
}

// int32 planes in chunks of at most 13 (|chunk| < 2^(31 + 84)): each chunk is exact in 128
// bits and converted to a double-double; chunks are added most significant first
__device__ __forceinline__ dd gather_dd_w32_chunked(const GroupArgs& ga, int64_t i, int64_t j, int eLi, int eRj) {
  dd acc{0.0, 0.0};
  if (eLi == EZERO || eRj == EZERO) return acc;
  const int32_t* p = reinterpret_cast<const int32_t*>(ga.out) + j * ga.ldo + i;
  int g = 0;
  while (g < ga.groups) {
    int len = ga.groups - g < 13 ? ga.groups - g : 13;
    i128 N = 0;
    for (int q = 0; q < len; q += 4) {
      int l4 = len - q < 4 ? len - q : 4;
      i64 c = 0;
      for (int u = 0; u < l4; ++u) c = (c << 7) + (i64)p[(g + q + u) * ga.ogs];
      N = q ? (N << (7 * l4)) + (i128)c : (i128)c;
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
  if (x == 0.0) return 0;
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

__global__ void __launch_bounds__(256) k_groups_to_dd(GroupArgs ga, const int32_t* __restrict__ eL,
                                                      const int32_t* __restrict__ eR, int64_t M, int64_t N,
                                                      double* __restrict__ Ch, int64_t ldh, double* __restrict__ Cl,
                                                      int64_t ldl) {
  int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  int64_t j = blockIdx.y;
  if (i >= M) return;
  ga = resolve(ga);
  dd v = gather_dd(ga, i, j, eL[i], eR[j]);
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

// ---- lines 2-4 (inner part): one block per column j --------------------------------
// smem: n double-doubles (V column).  x^T x is exact in integers (X1 lies on the grid
// 2^(f_j + beta - 53)); x^T v is accumulated with TwoProduct/TwoSum (Dot2 form).
__global__ void __launch_bounds__(256) k_residual(ResidualArgs a) {
  if (a.done && *a.done) return;
  a.V = resolve(a.V);
  if (a.beta_dyn) a.beta = *a.beta_dyn;
  extern __shared__ dd vcol[];
  __shared__ dd redd[32];
  __shared__ u64 redu[32];
  __shared__ i128 redi[32];
  const int64_t j = blockIdx.x;
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
  if (lam != 0.0) decompose(lam, L, qL);
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

// ---- ||off-diagonal W||_F^2 (for the automatic cluster threshold) ------------------
__global__ void __launch_bounds__(256) k_w_offdiag_norm2(CorrectionArgs a) {
  if (a.done && *a.done) return;
  a.W = resolve(a.W);
  if (a.W.groups == 0) return;
  __shared__ double red[32];
  const int64_t j = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < a.n; i += blockDim.x) {
    if (i == j) continue;
    double w = gather_d(a.W, i, j, a.f[i], a.h[j]);
    s += w * w;
  }
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) atomicAdd(a.norms + 1, s);
}

// ---- line 5: E~ column j, its exponent, ||E~||_F^2 -----------------------------------
__global__ void __launch_bounds__(256) k_correction(CorrectionArgs a) {
  if (a.done && *a.done) return;
  a.W = resolve(a.W);
  if (a.omega_dyn) a.omega = *a.omega_dyn;
  __shared__ double red[32];
  __shared__ u64 redu[32];
  __shared__ dd redd[32];
  __shared__ int clist[64];
  __shared__ int ccount;
  const int64_t j = blockIdx.x;
  const int64_t n = a.n;
  const double lj = a.lam[j];
  const int hj = a.h[j];
  if (threadIdx.x == 0) ccount = 0;
  __syncthreads();
  double s2 = 0.0;
  u64 mx = 0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double e;
    double w = (a.W.groups > 0) ? gather_d(a.W, i, j, a.f[i], hj) : 0.0;
    if (a.Wout) a.Wout[i + j * n] = w;
    if (i == j) {
      e = a.r[j] * 0.5;
    } else {
      double diff = __dsub_rn(lj, a.lam[i]);
      if (fabs(diff) <= a.omega) {
        int slot = atomicAdd(&ccount, 1);
        if (slot < 64) clist[slot] = (int)i;
        else atomicOr(a.flags, FLAG_RANGE);
        e = 0.0;
      } else {
        e = __ddiv_rn(w, diff);
      }
    }
    a.E[i + j * a.lde] = e;
  }
  __syncthreads();
  int nc = ccount < 64 ? ccount : 64;
  const double* xj = a.X1 + j * a.ld1;
  for (int c = 0; c < nc; ++c) {
    int i = clist[c];
    const double* xi = a.X1 + (int64_t)i * a.ld1;
    dd acc{0.0, 0.0};
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) acc = dd_add(acc, two_prod(xi[k], xj[k]));
    acc = block_sum_dd(acc, redd);
    if (threadIdx.x == 0) a.E[i + j * a.lde] = -acc.h * 0.5;   // r_ij / 2
    __syncthreads();
  }
  if (threadIdx.x == 0 && nc) atomicAdd(a.ccount, nc);
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double e = a.E[i + j * a.lde];
    s2 += e * e;
    u64 ab = double_to_bits(e) & 0x7fffffffffffffffull;
    mx = ab > mx ? ab : mx;
  }
  s2 = block_sum_d(s2, red);
  mx = block_max_u64(mx, redu);
  if (threadIdx.x == 0) {
    atomicAdd(a.norms + 0, s2);
    a.eta[j] = mx == 0 ? EZERO : ceil_log2_absbits(mx);
  }
}

// ---- line 6: X <- RN(X1 + X1 E~) (pair arithmetic), ||X_new - X_old||_F^2 ----------------
// RN(x1 + N 2^c) for int64 N with |N 2^c| well below |x1|: x1 = P 2^q (53-bit P) and the
// sum is rounded on x1's grid with round-half-even on the combined integer.  Returns false
// when the result leaves x1's binade (then the caller takes the general path).
__device__ __forceinline__ bool add_small_rn(double x1, i64 N, int c, double& out) {
  if (x1 == 0.0) return false;
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

// one block per column: X(:, j) <- RN(X1(:, j) + U(:, j)); one atomic per column for ||dX||_F^2
__global__ void __launch_bounds__(1024) k_update(UpdateArgs a) {
  if (a.done && *a.done) return;
  a.U = resolve(a.U);
  if (a.beta_dyn) a.beta = *a.beta_dyn;
  __shared__ double red[32];
  const int64_t j = blockIdx.x;
  const int ej = a.eta[j];
  double d2 = 0.0;
  for (int64_t i = threadIdx.x; i < a.n; i += blockDim.x) {
    double x1 = a.X1[i + j * a.ld1];
    double xn = x1;
    if (a.U.groups > 0) {
      bool done = false;
      int ri = a.rho[i];
      if (ri != EZERO && ej != EZERO) {
        int c = ri + ej + 2 - DIGIT_BITS * a.U.tmax;
        if (a.U.word32 && a.U.groups <= 5) {
          // the anti-diagonal planes combine exactly in int64 (31 + 28 bits)
          const int32_t* p = reinterpret_cast<const int32_t*>(a.U.out) + j * a.U.ldo + i;
          int32_t v[5];
#pragma unroll
          for (int q = 0; q < 5; ++q) v[q] = q < a.U.groups ? __ldg(p + q * a.U.ogs) : 0;
          i64 N = 0;
#pragma unroll
          for (int q = 0; q < 5; ++q)
            if (q < a.U.groups) N = (N << 7) + (i64)v[q];
          done = add_small_rn(x1, N, c, xn);
        }
        if (!done && a.U.exact128) {
          i128 N = combine_groups(a.U, i, j);
          const int G = a.f[j] + a.beta - 53;
          i128 m = (i128)grid_mantissa(x1, G);
          int d = G - c;
          if (d >= 0 && bitlen128(m) + d <= 124 && bitlen128(N) <= 124) {
            xn = i128_scaled_rn((m << d) + N, c);
            done = true;
          } else if (d < 0 && bitlen128(N) - d <= 124) {
            xn = i128_scaled_rn(m + (N << (-d)), G);
            done = true;
          }
        }
      }
      if (!done) {
        dd u = gather_dd(a.U, i, j, ri, ej);
        dd c2 = two_sum(x1, u.h);
        double cl = __dadd_rn(u.l, c2.l);
        xn = __dadd_rn(c2.h, cl);
      }
    }
    double xo = a.X[i + j * a.ldx];
    double dx = __dsub_rn(xn, xo);
    d2 = __fma_rn(dx, dx, d2);
    a.X[i + j * a.ldx] = xn;
  }
  d2 = block_sum_d(d2, red);
  if (threadIdx.x == 0) atomicAdd(a.norms + 2, d2);
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
  // 7 (tmax - t_last(0)) more bits and must stay below 2^127
  int t0 = 2 + g.d.gs - 1 < g.d.tmax ? 2 + g.d.gs - 1 : g.d.tmax;
  ga.exact128 = ga.groups > 0 && (g.d.word32 ? 31 : 62) + DIGIT_BITS * (g.d.tmax - t0) + 1 <= 127;
  return ga;
}

int launch_groups_to_dd(const PlaneGemm& g, const int32_t* eL, const int32_t* eR, double* Ch, int64_t ldh,
                        double* Cl, int64_t ldl, cudaStream_t s) {
  if (g.M == 0 || g.N == 0) return FRX_OK;
  dim3 grid((unsigned)((g.M + 255) / 256), (unsigned)g.N);
  k_groups_to_dd<<<grid, 256, 0, s>>>(group_args(g), eL, eR, g.M, g.N, Ch, ldh, Cl, ldl);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int set_refine_kernel_attributes() {
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_residual, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(dd) * (size_t)FRX_MAX_N)));
  return FRX_OK;
}

int launch_residual(const ResidualArgs& a, cudaStream_t s) {
  size_t smem = sizeof(dd) * (size_t)a.n;
  k_residual<<<(unsigned)a.n, 256, smem, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_w_offdiag_norm2(const CorrectionArgs& a, cudaStream_t s) {
  k_w_offdiag_norm2<<<(unsigned)a.n, 256, 0, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_correction(const CorrectionArgs& a, cudaStream_t s) {
  k_correction<<<(unsigned)a.n, 256, 0, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_update(const UpdateArgs& a, cudaStream_t s) {
  k_update<<<(unsigned)a.n, 1024, 0, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

}  // namespace frx
