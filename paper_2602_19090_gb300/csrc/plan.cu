// Device-side plan of each refinement iteration: the Sec. 4.1 choice of beta and alpha,
// the slice counts of the three Ozaki products, the cluster threshold and the stopping
// test, computed by single-block kernels so that an iteration needs no host round-trip.
// Every decision uses the same IEEE operations, in the same order, as the CPU oracle.
#include "frx_internal.cuh"
#include "kernels.cuh"
#include "plan.cuh"
#include "profile.cuh"
#include "grouped.cuh"
#include "plan_launch.cuh"

namespace frx {

constexpr int PT = 1024;  // threads of the plan kernels
constexpr double U53 = 1.1102230246251565e-16;

__device__ int dfloor_log2(double x) {
  int ex;
  frexp(x, &ex);
  return ex - 1;
}

__device__ int dceil_log2(double x) {
  int ex;
  double fr = frexp(x, &ex);
  return fr == 0.5 ? ex - 1 : ex;
}

__device__ int dceil_log2_sqrt(int64_t n) {
  int bl = 0;
  for (uint64_t v = (uint64_t)(n - 1); v; v >>= 1) ++bl;
  return (bl + 1) / 2;
}

__device__ int dceil_log2_int(int64_t n) {
  int bl = 0;
  for (uint64_t v = (uint64_t)(n - 1); v; v >>= 1) ++bl;
  return bl;
}

// Slice count of an Ozaki product: the smallest k >= 1 with 16 n 2^(eL + eR - b k) <= tau
// (b = DIGIT_BITS), evaluated exactly as 2^(b k - eL - eR - 4) tau >= n; capped; 0 if an operand
// is zero.  The dropped part's entries are sums over n terms of digit tails below
// 2^(eL + eR - b k); such sums grow like sqrt(n) (the reading Sec. 4.1 makes when it replaces
// log2 n by ceil(log2 sqrt n)) and the 2-norm of the n x n error like sqrt(n) times its entries;
// 16 is the calibrated margin.
constexpr int SLICE_MARGIN_LOG2 = 4;
__device__ int dslices_for(int64_t n, int eL, int eR, double tau, int kcap) {
  if (eL == EZERO || eR == EZERO) return 0;
  for (int k = 1; k <= kcap; ++k)
    if (ldexp(tau, DIGIT_BITS * k - eL - eR - SLICE_MARGIN_LOG2) >= (double)n) return k;
  return kcap;
}

// ---- block reductions (PT threads) ----
__device__ int bmax_int(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (PT >> 5) ? red[threadIdx.x] : INT32_MIN;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

__device__ int bmin_int(int v, int* red) { return -bmax_int(-v, red); }

__device__ double bmax_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (PT >> 5) ? red[threadIdx.x] : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

__device__ double bmin_d(double v, double* red) { return -bmax_d(-v, red); }

__device__ double bsum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (PT >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

// Order-preserving integer keys of doubles (non-NaN): the bitonic sort compares integers,
// since one SM's FP64 pipe would take ~0.1 ms for the ~78 compare stages at n = 4096.
__device__ __forceinline__ u64 order_key(double v) {
  const u64 b = double_to_bits(v);
  return (b >> 63) ? ~b : (b | (1ull << 63));
}

__device__ __forceinline__ double key_value(u64 k) {
  return bits_to_double((k >> 63) ? (k & ~(1ull << 63)) : ~k);
}

// Smallest adjacent gap of the sorted estimates exceeding omega (Lam if none) and max |lam|.
// s: dynamic smem of next_pow2(n) doubles.  With `rank` (each estimate's position in ascending
// order, from k_rank_keys) the keys are placed by rank; without, this block sorts them (bitonic
// network on their integer keys).
__device__ void gap_of(const double* lam, int64_t n, double omega, double* s, double* red, double& g,
                       double& Lam, const uint32_t* rank) {
  u64* key = reinterpret_cast<u64*>(s);
  int64_t m = 1;
  while (m < n) m <<= 1;
  u64 amax = 0;
  for (int64_t i = threadIdx.x; i < (rank ? n : m); i += PT) {
    const double v = i < n ? lam[i] : INFINITY;
    key[rank ? (int64_t)rank[i] : i] = order_key(v);
    if (i < n) {
      const u64 ab = double_to_bits(v) & 0x7fffffffffffffffull;
      amax = ab > amax ? ab : amax;
    }
  }
  __syncthreads();
  for (int64_t k = 2; !rank && k <= m; k <<= 1) {
    for (int64_t jj = k >> 1; jj > 0; jj >>= 1) {
      for (int64_t i = threadIdx.x; i < m; i += PT) {
        const int64_t l = i ^ jj;
        if (l > i) {
          const u64 a = key[i], b = key[l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            key[i] = b;
            key[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  double gmin = INFINITY;
  for (int64_t i = 1 + threadIdx.x; i < n; i += PT) {
    const double d = __dsub_rn(key_value(key[i]), key_value(key[i - 1]));
    if (d > omega) gmin = fmin(gmin, d);
  }
  gmin = bmin_d(gmin, red);
  Lam = bmax_d(bits_to_double(amax), red);
  g = isinf(gmin) ? Lam : gmin;
}

__device__ void raise(DevPlan* p, int st) {
  if (threadIdx.x == 0) {
    p->status = st;
    p->done = 1;
    p->V.active = p->W.active = p->U.active = 0;
  }
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ void plan_init_impl(DevPlan* p, const int32_t* eA, const double* D,
                                                  double* lam_prev, PlanOpts o, double omega_prev,
                                                  const uint32_t* rank) {
  extern __shared__ double sbuf[];
  __shared__ int redi[32];
  __shared__ double redd[32];
  bool bad = false;
  int emax = EZERO;
  for (int64_t i = threadIdx.x; i < o.n; i += PT) {
    double v = D[i];
    bad |= !isfinite(v);
    lam_prev[i] = v;
    emax = max(emax, eA[i]);
  }
  emax = bmax_int(emax, redi);
  int anybad = bmax_int(bad ? 1 : 0, redi);
  double g, Lam;
  gap_of(D, o.n, omega_prev, sbuf, redd, g, Lam, rank);
  if (threadIdx.x == 0) {
    p->iter = 0;
    p->done = 0;
    p->status = FRX_MAX_ITER;
    p->eAmax = emax;
    p->sliced_kA = 0;
    p->products = 0;
    p->omega = omega_prev;
    p->have_prev_step = 0;
    p->noncontract = 0;
    p->prev_step = 0.0;
    p->g = g;
    p->Lam = Lam;
    p->est = INFINITY;
    p->clustered = 0;
    p->ccount = 0;
    for (int k = 0; k < 4; ++k) p->norms[k] = 0.0;
    p->V.active = p->W.active = p->U.active = 0;
    if (p->flags & FLAG_NONFINITE) anybad = 1;
  }
  __syncthreads();
  if (anybad) raise(p, FRX_E_NONFINITE);
}

// beta, alpha, s_X, k_V and the V product (Alg. 1 with Sec. 3 and Sec. 4.1)
__device__ __forceinline__ void plan_v_impl(DevPlan* p, const int32_t* f, PlanOpts o) {
  __shared__ int redi[32];
  __shared__ double redd[32];
  __shared__ unsigned long long s2lo[32], s2hi[32];
  if (p->done) return;
  int fmx = EZERO, fmn = INT32_MAX, zero = 0;
  for (int64_t i = threadIdx.x; i < o.n; i += PT) {
    int e = f[i];
    if (e == EZERO) {
      zero = 1;
    } else {
      fmx = max(fmx, e);
      fmn = min(fmn, e);
    }
  }
  fmx = bmax_int(fmx, redi);
  fmn = bmin_int(fmn, redi);
  zero = bmax_int(zero, redi);
  if (zero || (p->flags & FLAG_NONFINITE)) {
    raise(p, zero ? FRX_E_ARG : FRX_E_NONFINITE);
    return;
  }
  // S2 = sum_j 2^(2 f_j), exactly rounded (integer accumulation relative to the smallest term)
  double S2 = 0.0;
  if (fmx - fmn <= 45) {
    unsigned __int128 acc = 0;
    for (int64_t i = threadIdx.x; i < o.n; i += PT) acc += (unsigned __int128)1 << (2 * (f[i] - fmn));
    unsigned long long lo = (unsigned long long)acc, hi = (unsigned long long)(acc >> 64);
    // warp + block sum of 128-bit values
    for (int off = 16; off > 0; off >>= 1) {
      unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, off), hi2 = __shfl_xor_sync(0xffffffffu, hi, off);
      unsigned long long nl = lo + lo2;
      hi = hi + hi2 + (nl < lo ? 1ull : 0ull);
      lo = nl;
    }
    if ((threadIdx.x & 31) == 0) {
      s2lo[threadIdx.x >> 5] = lo;
      s2hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned __int128 tot = 0;
      for (int w = 0; w < PT / 32; ++w) tot += ((unsigned __int128)s2hi[w] << 64) | s2lo[w];
      // round to nearest even: keep 63 bits and a sticky bit (the value is below 2^(90 + 14))
      double r;
      if ((tot >> 63) == 0) {
        r = __ull2double_rn((unsigned long long)tot);
      } else {
        int bl = 0;
        for (unsigned __int128 v = tot; v; v >>= 1) ++bl;
        int sh = bl - 63;
        unsigned long long v = (unsigned long long)(tot >> sh);
        if ((tot & (((unsigned __int128)1 << sh) - 1)) != 0) v |= 1ull;
        r = ldexp(__ull2double_rn(v), sh);
      }
      redd[0] = ldexp(r, 2 * fmn);
    }
    __syncthreads();
    S2 = redd[0];
  } else if (threadIdx.x == 0) {
    // ascending sequential sum (the exponent spread is beyond the integer accumulator)
    for (int e = fmn; e <= fmx; ++e)
      for (int64_t i = 0; i < o.n; ++i)
        if (f[i] == e) S2 = __dadd_rn(S2, ldexp(1.0, 2 * e));
  }
  if (threadIdx.x != 0) return;
  const int64_t n = o.n;
  double g = p->g, Lam = p->Lam;
  int beta;
  if (o.x_planes > 0) {
    beta = 54 - DIGIT_BITS * o.x_planes;   // X kept at x_planes planes (previous-study form)
  } else if (o.beta_override >= 0) {
    beta = min(max(o.beta_override, 3), 47);
  } else if (g <= 0.0 || Lam <= 0.0 || S2 <= 0.0) {
    beta = 3;
  } else {
    // Sec. 4.1 uses xi = n; the sparse-matrix rule of Sec. 4 has min(k, sqrt n)^2
    const double kk = (double)(p->rownnz > 0 ? p->rownnz : 1);
    double xi = o.sparse_rule ? (kk * kk < (double)n ? kk * kk : (double)n) : (o.xi > 0 ? o.xi : (double)n);
    double q = __ddiv_rn(__dsqrt_rn(__ddiv_rn(__dmul_rn(__dmul_rn(xi, o.delta), g), __dmul_rn(Lam, S2))),
                         0.75 * U53);
    int b = o.beta_ceil ? dceil_log2(q) : dfloor_log2(q);
    beta = min(max(b, 3), 47);
  }
  p->iter += 1;
  p->beta = beta;
  p->alpha = o.sparse_rule ? 53 - beta + dceil_log2_int(p->rownnz > 0 ? p->rownnz : 1)
            : (o.theory_alpha ? 53 - beta + dceil_log2_int(n) : 53 - beta + dceil_log2_sqrt(n));
  p->sX = (54 - beta + DIGIT_BITS - 1) / DIGIT_BITS;
  p->fmax = fmx;
  p->S2 = S2;
  int kV = o.slices_A > 0 ? o.slices_A : dslices_for(n, p->eAmax, fmx, __dmul_rn(o.delta, g), o.k_cap);
  if (kV < 1) kV = 1;
  p->kV = kV;
  GemmDesc d;
  d.kL = kV;
  d.kR = p->sX;
  d.T = kV + 1;
  if (gemm_desc_layout(d, n, 64) != FRX_OK || !d.word32) {
    raise(p, FRX_E_UNSUPPORTED);
    return;
  }
  gemm_desc_schedule(d, n, n, 256);
  p->V = d;
  p->products += desc_pairs(d);
  for (int k = 0; k < 4; ++k) p->norms[k] = 0.0;
  p->ccount = 0;
}

// after the A planes for this iteration are written
__device__ __forceinline__ void plan_mark_sliced_impl(DevPlan* p) {
  if (threadIdx.x == 0 && !p->done && p->kV > p->sliced_kA) p->sliced_kA = p->kV;
}

// k_W and the W product (Alg. 1)
__device__ __forceinline__ void plan_w_impl(DevPlan* p, const int32_t* h, PlanOpts o) {
  __shared__ int redi[32];
  if (p->done) return;
  int hm = EZERO;
  for (int64_t i = threadIdx.x; i < o.n; i += PT) hm = max(hm, h[i]);
  hm = bmax_int(hm, redi);
  if (threadIdx.x != 0) return;
  int kW = dslices_for(o.n, p->fmax, hm, __dmul_rn(o.delta, p->g), o.k_cap);
  p->kW = kW;
  GemmDesc d;
  d.kL = min(p->sX, kW);
  d.kR = kW;
  d.T = kW + 1;
  if (kW > 0) {
    if (gemm_desc_layout(d, o.n, 64) != FRX_OK || !d.word32) {
      raise(p, FRX_E_UNSUPPORTED);
      return;
    }
  } else {
    d.active = 0;
    d.groups = 0;
    d.tmax = 0;
    d.gs = 1;
    d.word32 = 1;
  }
  gemm_desc_schedule(d, o.n, o.n, 256);
  p->W = d;
  p->products += desc_pairs(d);
}

// cluster threshold omega (fixed, or the Ogita-Aishima form from ||W_off||_F and ||diag R||_2)
// sum of n per-column partials in a fixed order (strided per thread, then a fixed tree), so
// that the norms and the decisions taken from them repeat bit for bit from run to run
__device__ __forceinline__ double sum_columns(const double* c, int64_t n, double* redd) {
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += PT) s = __dadd_rn(s, c[i]);
  return bsum_d(s, redd);
}

// colsq: per-column squared norms [3][n] written by the correction, off-diagonal-W and
// update kernels (E~, W_off, X_new - X_old)
__device__ __forceinline__ void plan_omega_impl(DevPlan* p, const double* r, const double* colsq, PlanOpts o) {
  __shared__ double redd[32];
  if (p->done) return;
  if (o.cluster_omega >= 0) {
    if (threadIdx.x == 0) p->omega = o.cluster_omega;
    return;
  }
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < o.n; i += PT) s = __fma_rn(r[i], r[i], s);
  s = bsum_d(s, redd);
  const double w2 = sum_columns(colsq + o.n, o.n, redd);
  if (threadIdx.x == 0) {
    p->norms[1] = w2;
    p->omega = 2.0 * (__dsqrt_rn(w2) + p->Lam * __dsqrt_rn(s));
  }
}

// k_U and the update product (Alg. 1)
__device__ __forceinline__ void plan_u_impl(DevPlan* p, const int32_t* rho, const int32_t* eta, PlanOpts o) {
  __shared__ int redi[32];
  if (p->done) return;
  int rm = EZERO, em = EZERO;
  for (int64_t i = threadIdx.x; i < o.n; i += PT) {
    rm = max(rm, rho[i]);
    em = max(em, eta[i]);
  }
  rm = bmax_int(rm, redi);
  em = bmax_int(em, redi);
  if (threadIdx.x != 0) return;
  // the exact int32 sums need kU n 2^14 < 2^31 (up to kU pairs per anti-diagonal)
  const int cap = (int)(((1ll << 31) - 1) / ((long long)o.n << PRODUCT_BITS));
  int kU = dslices_for(o.n, rm, em, o.delta, o.k_cap);
  kU = kU < cap ? kU : cap;
  p->kU = kU;
  GemmDesc d;
  d.kL = kU;
  d.kR = kU;
  d.T = kU + 1;
  if (kU > 0) {
    if (gemm_desc_layout(d, o.n, 64) != FRX_OK || !d.word32) {
      raise(p, FRX_E_UNSUPPORTED);
      return;
    }
  } else {
    d.active = 0;
    d.groups = 0;
    d.tmax = 0;
    d.gs = 1;
    d.word32 = 1;
  }
  gemm_desc_schedule(d, o.n, o.n, 256);
  p->U = d;
  p->products += desc_pairs(d);
}

// stopping test (reading R7): est = step^2 max|lam| / (xi_stop gap) <= delta
__device__ __forceinline__ void plan_end_impl(DevPlan* p, const double* lam_new, double* lam_prev,
                                              const double* colsq, PlanOpts o, const uint32_t* rank) {
  extern __shared__ double sbuf[];
  __shared__ double redd[32];
  if (p->done) return;
  const double omega = p->omega;
  double g, Lam;
  gap_of(lam_new, o.n, omega, sbuf, redd, g, Lam, rank);
  for (int64_t i = threadIdx.x; i < o.n; i += PT) lam_prev[i] = lam_new[i];
  const double e2 = sum_columns(colsq, o.n, redd);
  __syncthreads();
  const double dx2 = sum_columns(colsq + 2 * o.n, o.n, redd);
  if (threadIdx.x != 0) return;
  p->norms[0] = e2;
  p->norms[2] = dx2;
  if (p->flags & FLAG_NONFINITE) {
    raise(p, FRX_E_NONFINITE);
    return;
  }
  if (p->flags & (FLAG_TIMEOUT | FLAG_RANGE | FLAG_CONFIG)) {
    raise(p, (p->flags & FLAG_TIMEOUT) ? FRX_E_TIMEOUT : (p->flags & FLAG_RANGE) ? FRX_E_RANGE : FRX_E_UNSUPPORTED);
    return;
  }
  double step = __dsqrt_rn(p->norms[2]);
  double xs = o.xi_stop > 0 ? o.xi_stop : (double)o.n;
  double est = g > 0 ? __ddiv_rn(__dmul_rn(__dmul_rn(step, step), Lam), __dmul_rn(xs, g)) : INFINITY;
  p->step = step;
  p->est = est;
  p->g = g;
  p->Lam = Lam;
  p->normE = __dsqrt_rn(p->norms[0]);
  p->clustered = p->ccount / 2;
  // stagnation: two consecutive steps that failed to halve (a single one is expected when
  // the start lies outside Theorem 1's basin and the next step repairs the first)
  p->noncontract = (p->have_prev_step && step > 0.5 * p->prev_step) ? p->noncontract + 1 : 0;
  if (est <= o.delta) {
    p->status = FRX_OK;
    p->done = 1;
  } else if (p->noncontract >= 2) {
    p->status = FRX_STAGNATED;
    p->done = 1;
  } else if (p->iter >= o.max_iter) {
    p->status = FRX_MAX_ITER;
    p->done = 1;
  }
  p->prev_step = step;
  p->have_prev_step = 1;
}

// ---------------------------------------------------------------------------
static size_t sort_smem(int64_t n) {
  int64_t m = 1;
  while (m < n) m <<= 1;
  return (size_t)m * sizeof(double);
}


// ---- kernels: single problem (one block) and grouped bodies ----------------------------
struct PlanArgs {
  DevPlan* p;
  const int32_t* e0;     // eA (init), f (v), h (w), rho (u)
  const int32_t* e1;     // eta (u)
  const double* d0;      // D (init), r (omega), lam_new (end)
  double* d1;            // lam_prev (init, end)
  PlanOpts o;
  double omega_prev;
  unsigned gx;
  const double* colsq;   // per-column squared norms (omega, end)
};

__global__ void __launch_bounds__(PT) k_plan_init(DevPlan* p, const int32_t* eA, const double* D, double* lam_prev,
                                                  PlanOpts o, double omega_prev, const uint32_t* rank) {
  plan_init_impl(p, eA, D, lam_prev, o, omega_prev, rank);
}
__global__ void __launch_bounds__(PT) k_plan_v(DevPlan* p, const int32_t* f, PlanOpts o) { plan_v_impl(p, f, o); }
__global__ void k_plan_mark_sliced(DevPlan* p) { plan_mark_sliced_impl(p); }
__global__ void __launch_bounds__(PT) k_plan_w(DevPlan* p, const int32_t* h, PlanOpts o) { plan_w_impl(p, h, o); }
__global__ void __launch_bounds__(PT) k_plan_omega(DevPlan* p, const double* r, const double* colsq, PlanOpts o) {
  plan_omega_impl(p, r, colsq, o);
}
__global__ void __launch_bounds__(PT) k_plan_u(DevPlan* p, const int32_t* rho, const int32_t* eta, PlanOpts o) {
  plan_u_impl(p, rho, eta, o);
}
__global__ void __launch_bounds__(PT) k_plan_end(DevPlan* p, const double* lam_new, double* lam_prev,
                                                 const double* colsq, PlanOpts o, const uint32_t* rank) {
  plan_end_impl(p, lam_new, lam_prev, colsq, o, rank);
}

// Position of every estimate in ascending order of its integer key, ties by index:
// rank_i = #{j : k_j < k_i} + #{j < i : k_j = k_i}, a permutation of 0..n-1 (the order the
// bitonic network of gap_of produces).  Blocks cover 256 estimates i by a slice of the j; their
// counts are added to rank (zeroed first).  Skipped, like the plan kernel after it, once the
// refinement has finished.
constexpr int RANK_TILE = 1024;

__global__ void __launch_bounds__(256) k_rank_keys(const DevPlan* p, const double* lam, int64_t n, int64_t per,
                                                   uint32_t* rank) {
  __shared__ u64 kj[RANK_TILE];
  if (p && p->done) return;
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const u64 ki = i < n ? order_key(lam[i]) : 0ull;
  const int64_t j0 = (int64_t)blockIdx.y * per, j1 = min(n, j0 + per);
  uint32_t cnt = 0;
  for (int64_t t0 = j0; t0 < j1; t0 += RANK_TILE) {
    const int m = (int)min((int64_t)RANK_TILE, j1 - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < m; q += 256) kj[q] = order_key(lam[t0 + q]);
    __syncthreads();
    const int64_t below = i - t0;   // kj[q] comes before k_i on ties when q < below
    for (int q = 0; q < m; ++q) {
      const u64 k = kj[q];
      cnt += (k < ki || (k == ki && q < below)) ? 1u : 0u;
    }
  }
  if (i < n && cnt) atomicAdd(&rank[i], cnt);
}

// ranks of lam[0..n) into `rank` (n words of scratch), on stream s
static int launch_rank_keys(const DevPlan* p, const double* lam, int64_t n, uint32_t* rank, cudaStream_t s) {
  FRX_CUDA_TRY(cudaMemsetAsync(rank, 0, sizeof(uint32_t) * (size_t)n, s));
  const int64_t bx = (n + 255) / 256;
  int64_t by = (4 * 152 + bx - 1) / bx;                 // about four blocks per SM in all
  by = by < 1 ? 1 : (by > (n + 255) / 256 ? (n + 255) / 256 : by);
  const int64_t per = (n + by - 1) / by;
  k_rank_keys<<<dim3((unsigned)bx, (unsigned)by), 256, 0, s>>>(p, lam, n, per, rank);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

__device__ __forceinline__ void plan_init_body(PlanArgs a, unsigned, unsigned) {
  plan_init_impl(a.p, a.e0, a.d0, a.d1, a.o, a.omega_prev, nullptr);
}
__device__ __forceinline__ void plan_v_body(PlanArgs a, unsigned, unsigned) { plan_v_impl(a.p, a.e0, a.o); }
__device__ __forceinline__ void plan_mark_sliced_body(PlanArgs a, unsigned, unsigned) { plan_mark_sliced_impl(a.p); }
__device__ __forceinline__ void plan_w_body(PlanArgs a, unsigned, unsigned) { plan_w_impl(a.p, a.e0, a.o); }
__device__ __forceinline__ void plan_omega_body(PlanArgs a, unsigned, unsigned) {
  plan_omega_impl(a.p, a.d0, a.colsq, a.o);
}
__device__ __forceinline__ void plan_u_body(PlanArgs a, unsigned, unsigned) { plan_u_impl(a.p, a.e0, a.e1, a.o); }
__device__ __forceinline__ void plan_end_body(PlanArgs a, unsigned, unsigned) {
  plan_end_impl(a.p, a.d0, a.d1, a.colsq, a.o, nullptr);
}

int launch_plan_init(DevPlan* p, const int32_t* eA, const double* D, double* lam_prev, const PlanOpts& o,
                     double omega_prev, uint32_t* rank, cudaStream_t s) {
  size_t sm = sort_smem(o.n);
  if (record_launch(LK_PLAN_INIT, PlanArgs{p, eA, nullptr, D, lam_prev, o, omega_prev, 1u}, 1, PT, sm)) return FRX_OK;
  if (rank) FRX_TRY(launch_rank_keys(nullptr, D, o.n, rank, s));   // the plan is reset below: no done test
  k_plan_init<<<1, PT, sm, s>>>(p, eA, D, lam_prev, o, omega_prev, rank);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_plan_v(DevPlan* p, const int32_t* f, const PlanOpts& o, cudaStream_t s) {
  if (record_launch(LK_PLAN_V, PlanArgs{p, f, nullptr, nullptr, nullptr, o, 0.0, 1u}, 1, PT, 0)) return FRX_OK;
  k_plan_v<<<1, PT, 0, s>>>(p, f, o);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_plan_mark_sliced(DevPlan* p, cudaStream_t s) {
  PlanOpts none{};
  if (record_launch(LK_PLAN_MARK_SLICED, PlanArgs{p, nullptr, nullptr, nullptr, nullptr, none, 0.0, 1u}, 1, 32, 0))
    return FRX_OK;
  k_plan_mark_sliced<<<1, 32, 0, s>>>(p);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_plan_w(DevPlan* p, const int32_t* h, const PlanOpts& o, cudaStream_t s) {
  if (record_launch(LK_PLAN_W, PlanArgs{p, h, nullptr, nullptr, nullptr, o, 0.0, 1u}, 1, PT, 0)) return FRX_OK;
  k_plan_w<<<1, PT, 0, s>>>(p, h, o);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_plan_omega(DevPlan* p, const double* r, const double* colsq, const PlanOpts& o, cudaStream_t s) {
  if (record_launch(LK_PLAN_OMEGA, PlanArgs{p, nullptr, nullptr, r, nullptr, o, 0.0, 1u, colsq}, 1, PT, 0))
    return FRX_OK;
  k_plan_omega<<<1, PT, 0, s>>>(p, r, colsq, o);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_plan_u(DevPlan* p, const int32_t* rho, const int32_t* eta, const PlanOpts& o, cudaStream_t s) {
  if (record_launch(LK_PLAN_U, PlanArgs{p, rho, eta, nullptr, nullptr, o, 0.0, 1u}, 1, PT, 0)) return FRX_OK;
  k_plan_u<<<1, PT, 0, s>>>(p, rho, eta, o);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_plan_end(DevPlan* p, const double* lam_new, double* lam_prev, const double* colsq, const PlanOpts& o,
                    uint32_t* rank, cudaStream_t s) {
  size_t sm = sort_smem(o.n);
  if (record_launch(LK_PLAN_END, PlanArgs{p, nullptr, nullptr, lam_new, lam_prev, o, 0.0, 1u, colsq}, 1, PT, sm))
    return FRX_OK;
  if (rank) FRX_TRY(launch_rank_keys(p, lam_new, o.n, rank, s));
  k_plan_end<<<1, PT, sm, s>>>(p, lam_new, lam_prev, colsq, o, rank);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

__global__ void k_collect_done(DevPlan* const* plans, int count, int* done) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < count) done[b] = plans[b]->done;
}

__global__ void k_gather_plans(DevPlan* const* plans, int count, DevPlan* out) {
  int b = blockIdx.x;
  if (b >= count) return;
  const int* src = reinterpret_cast<const int*>(plans[b]);
  int* dst = reinterpret_cast<int*>(out + b);
  for (int k = threadIdx.x; k < (int)(sizeof(DevPlan) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
}

int launch_collect_done(DevPlan* const* plans, int count, int* done, cudaStream_t s) {
  k_collect_done<<<(count + 255) / 256, 256, 0, s>>>(plans, count, done);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_gather_plans(DevPlan* const* plans, int count, DevPlan* out, cudaStream_t s) {
  k_gather_plans<<<count, 128, 0, s>>>(plans, count, out);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}


int launch_grouped_plan(int kind, const void* tab, const long long* start, int count, long long blocks, int threads,
                        size_t smem, cudaStream_t s) {
  if (blocks <= 0) return FRX_OK;
  const unsigned grid = (unsigned)blocks;
  const PlanArgs* t = (const PlanArgs*)tab;
  switch (kind) {
    case LK_PLAN_INIT: k_grouped<PlanArgs, plan_init_body, PT, 1><<<grid, PT, smem, s>>>(t, start, count); break;
    case LK_PLAN_V: k_grouped<PlanArgs, plan_v_body, PT, 1><<<grid, PT, 0, s>>>(t, start, count); break;
    case LK_PLAN_MARK_SLICED:
      k_grouped<PlanArgs, plan_mark_sliced_body, 32, 1><<<grid, 32, 0, s>>>(t, start, count);
      break;
    case LK_PLAN_W: k_grouped<PlanArgs, plan_w_body, PT, 1><<<grid, PT, 0, s>>>(t, start, count); break;
    case LK_PLAN_OMEGA: k_grouped<PlanArgs, plan_omega_body, PT, 1><<<grid, PT, 0, s>>>(t, start, count); break;
    case LK_PLAN_U: k_grouped<PlanArgs, plan_u_body, PT, 1><<<grid, PT, 0, s>>>(t, start, count); break;
    case LK_PLAN_END: k_grouped<PlanArgs, plan_end_body, PT, 1><<<grid, PT, smem, s>>>(t, start, count); break;
    default: return FRX_E_UNSUPPORTED;
  }
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}


int set_plan_kernel_attributes() {
  int bytes = (int)sort_smem(FRX_MAX_N);
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_plan_init, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_plan_end, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_grouped<PlanArgs, plan_init_body, PT, 1>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_grouped<PlanArgs, plan_end_body, PT, 1>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  return FRX_OK;
}

}  // namespace frx
