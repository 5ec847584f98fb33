// Device-side plan of one refinement iteration (Sec. 3.3 / Sec. 4.1) and the descriptors
// the kernels of that iteration read, so an iteration runs without host round-trips.
#pragma once

#include "frx_internal.cuh"

namespace frx {

constexpr int MAX_GROUPS = 40;   // anti-diagonal groups of one product (2 * MAX_PLANES - 1 fit)

// One Ozaki product: plane counts, pair bound, layout of the exact sums and the
// persistent schedule (units = ntm * ntn * groups, groups ordered by decreasing work).
struct GemmDesc {
  int active;       // 0: no product this iteration (kernels return at once)
  int kL, kR, T;
  int tmax, gs, groups, word32;
  int ntm, ntn, units;
  int gorder[MAX_GROUPS];
};

// host/device: fill tmax, gs, groups, word32 (same rule as plan_plane_gemm); returns FRX_OK or
// FRX_E_UNSUPPORTED.  out_bytes_per_elem = 0 keeps int64 groups of any count.
__host__ __device__ inline int gemm_desc_layout(GemmDesc& d, int64_t K, int out_bytes_per_elem) {
  d.tmax = d.T < d.kL + d.kR ? d.T : d.kL + d.kR;
  d.word32 = 0;
  if (d.kL <= 0 || d.kR <= 0 || d.tmax < 2) {
    d.groups = 0;
    d.gs = 1;
    d.active = 0;
    return FRX_OK;
  }
  d.active = 1;
  if (K >= (1 << 19)) return FRX_E_UNSUPPORTED;
  int pmax = 0;
  for (int t = 2; t <= d.tmax; ++t) {
    int lo = t - d.kR > 1 ? t - d.kR : 1;
    int hi = d.kL < t - 1 ? d.kL : t - 1;
    int c = hi - lo + 1;
    pmax = c > pmax ? c : pmax;
  }
  unsigned long long smax = (unsigned long long)pmax * (unsigned long long)K << PRODUCT_BITS;
  int bs = 0;
  for (unsigned long long v = smax; v; v >>= 1) ++bs;  // smax < 2^bs
  if (bs > 61) return FRX_E_UNSUPPORTED;
  if (out_bytes_per_elem > 0 && smax < (1ull << 31) && (d.tmax - 1) * 4 <= out_bytes_per_elem &&
      d.tmax - 1 <= MAX_GROUPS) {
    d.word32 = 1;
    d.gs = 1;
    d.groups = d.tmax - 1;
    return FRX_OK;
  }
  d.gs = (61 - bs) / DIGIT_BITS + 1;
  d.groups = (d.tmax - 1 + d.gs - 1) / d.gs;
  if (d.groups > MAX_GROUPS) return FRX_E_UNSUPPORTED;
  if (out_bytes_per_elem > 0 && d.groups * 8 > out_bytes_per_elem) return FRX_E_UNSUPPORTED;
  return FRX_OK;
}

// host/device: persistent schedule for tiles of 128 x bn over an M x N output
__host__ __device__ inline void gemm_desc_schedule(GemmDesc& d, int64_t M, int64_t N, int bn) {
  d.ntm = (int)((M + 127) / 128);
  d.ntn = (int)((N + bn - 1) / bn);
  d.units = d.active ? d.ntm * d.ntn * d.groups : 0;
  int work[MAX_GROUPS];
  for (int q = 0; q < d.groups && q < MAX_GROUPS; ++q) {
    int t0 = 2 + q * d.gs, t1 = t0 + d.gs - 1 < d.tmax ? t0 + d.gs - 1 : d.tmax, w = 0;
    for (int t = t0; t <= t1; ++t) {
      int lo = t - d.kR > 1 ? t - d.kR : 1, hi = d.kL < t - 1 ? d.kL : t - 1;
      w += hi - lo + 1;
    }
    work[q] = w;
    d.gorder[q] = q;
  }
  // stable insertion sort by decreasing work
  for (int a = 1; a < d.groups && a < MAX_GROUPS; ++a) {
    int x = d.gorder[a], b = a - 1;
    while (b >= 0 && work[d.gorder[b]] < work[x]) {
      d.gorder[b + 1] = d.gorder[b];
      --b;
    }
    d.gorder[b + 1] = x;
  }
}

__host__ __device__ inline int desc_pairs(const GemmDesc& d) {
  int c = 0;
  for (int t = 2; t <= d.tmax && d.active; ++t) {
    int lo = t - d.kR > 1 ? t - d.kR : 1, hi = d.kL < t - 1 ? d.kL : t - 1;
    if (hi >= lo) c += hi - lo + 1;
  }
  return c;
}

struct PlanOpts {
  int slices_A;
  double xi;
  int beta_ceil, theory_alpha, beta_override, k_cap, max_iter;
  double xi_stop, cluster_omega;
  int x_planes;
  int sparse_rule;
  double delta;
  int64_t n;
};

// Iteration state kept on the device (one per matrix)
struct DevPlan {
  int iter, done, status;
  int beta, alpha, sX, kV, kW, kU, sliced_kA, eAmax, fmax;
  int clustered, have_prev_step;
  int noncontract;  // consecutive iterations whose step exceeded half the previous one
  int rownnz;       // largest number of nonzeros in a row of A (atomic max of the A scan)
  long long products;
  double g, Lam, S2, omega, step, prev_step, est, normE;
  double norms[4];  // [0] ||E~||_F^2, [1] ||W_off||_F^2, [2] ||dX||_F^2
  int flags;        // FLAG_* raised by kernels
  int ccount;       // cluster pairs counted by the correction kernel
  GemmDesc V, W, U;
};

}  // namespace frx
