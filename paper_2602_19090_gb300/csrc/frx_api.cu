// C ABI of frx: argument checks, workspace layout, the host-side plan of each
// iteration (Sec. 3.3 / Sec. 4.1) and the refinement driver (Algorithm 1 iterated).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "frx_internal.cuh"
#include "kernels.cuh"
#include "refine_kernels.cuh"

using namespace frx;

namespace {

constexpr double U53 = 1.1102230246251565e-16;  // 2^-53

// ---------------------------------------------------------------------------
// workspace carving
// ---------------------------------------------------------------------------
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) / 256 * 256;
    T* p = base ? (T*)(base + off) : nullptr;
    off += sizeof(T) * count;
    return p;
  }
};

struct RefineWs {
  int* flags;      // [0] flags, [1] cluster count
  double* norms;   // [0] ||E||^2, [1] ||W_off||^2, [2] ||dX||^2
  int32_t *eA, *f, *h, *eta, *rho;
  u64* rowmax;
  double *lam, *r;
  double *X1, *Res, *E;
  __nv_bfloat16 *Ap, *Xp, *Rp, *X1rp;
  i64* groups;
  int64_t pitch, ps;
  size_t bytes;
};

RefineWs carve_refine(void* work, int64_t n, int kcap) {
  RefineWs w;
  Carver c(work);
  w.pitch = round_up(n, 64);
  w.ps = n * w.pitch;
  w.flags = c.take<int>(4);
  w.norms = c.take<double>(4);
  w.eA = c.take<int32_t>(n);
  w.f = c.take<int32_t>(n);
  w.h = c.take<int32_t>(n);
  w.eta = c.take<int32_t>(n);
  w.rho = c.take<int32_t>(n);
  w.rowmax = c.take<u64>(n);
  w.lam = c.take<double>(n);
  w.r = c.take<double>(n);
  w.X1 = c.take<double>(n * n);
  w.Res = c.take<double>(n * n);
  w.E = c.take<double>(n * n);
  w.Ap = c.take<__nv_bfloat16>((size_t)kcap * w.ps);
  w.Xp = c.take<__nv_bfloat16>((size_t)8 * w.ps);
  w.Rp = c.take<__nv_bfloat16>((size_t)kcap * w.ps);
  w.X1rp = c.take<__nv_bfloat16>((size_t)kcap * w.ps);
  w.groups = c.take<i64>((size_t)8 * n * n);   // 64 bytes per entry: 8 int64 groups or 16 int32 planes
  w.bytes = c.off + 256;
  return w;
}

struct GemmWs {
  int* flags;
  int32_t *eA, *eB;
  u64* rowmax;
  __nv_bfloat16 *Ap, *Bp;
  i64* groups;
  int64_t pitch;
  size_t bytes;
};

GemmWs carve_gemm(void* work, int64_t m, int64_t n, int64_t k, int slices) {
  GemmWs w;
  Carver c(work);
  w.pitch = round_up(k, 64);
  w.flags = c.take<int>(4);
  w.eA = c.take<int32_t>(m);
  w.eB = c.take<int32_t>(n);
  w.rowmax = c.take<u64>(m);
  w.Ap = c.take<__nv_bfloat16>((size_t)slices * m * w.pitch);
  w.Bp = c.take<__nv_bfloat16>((size_t)slices * n * w.pitch);
  w.groups = c.take<i64>((size_t)8 * m * n);
  w.bytes = c.off + 256;
  return w;
}

bool aligned256(const void* p) { return ((uintptr_t)p & 255) == 0; }

// ---------------------------------------------------------------------------
// host plan (same FP64 formulas, in the same order, as the CPU oracle)
// ---------------------------------------------------------------------------
int floor_log2d(double x) {
  int ex;
  frexp(x, &ex);
  return ex - 1;
}

int ceil_log2d(double x) {
  int ex;
  double fr = frexp(x, &ex);
  return fr == 0.5 ? ex - 1 : ex;
}

int ceil_log2_sqrt_int(int64_t n) {
  int bl = 0;
  for (uint64_t v = (uint64_t)(n - 1); v; v >>= 1) ++bl;
  return (bl + 1) / 2;
}

int ceil_log2_int(int64_t n) {
  int bl = 0;
  for (uint64_t v = (uint64_t)(n - 1); v; v >>= 1) ++bl;
  return bl;
}

// smallest adjacent gap of the sorted estimates exceeding omega; Lam = max |lam|
double min_gap(const std::vector<double>& lam, double omega, double* Lam) {
  double L = 0.0;
  for (double v : lam) L = fabs(v) > L ? fabs(v) : L;
  *Lam = L;
  std::vector<double> s(lam);
  std::sort(s.begin(), s.end());
  double g = INFINITY;
  bool any = false;
  for (size_t i = 1; i < s.size(); ++i) {
    double d = s[i] - s[i - 1];
    if (d > omega) {
      g = d < g ? d : g;
      any = true;
    }
  }
  return any ? g : L;
}

// sum_j 2^(2 f_j), exactly rounded (integer accumulation relative to the smallest term)
double sum_pow4(const std::vector<int32_t>& f) {
  int emin = INT32_MAX, emax = INT32_MIN;
  for (int32_t e : f)
    if (e != EZERO) {
      emin = e < emin ? e : emin;
      emax = e > emax ? e : emax;
    }
  if (emin == INT32_MAX) return 0.0;
  if (emax - emin <= 45) {
    unsigned __int128 acc = 0;
    for (int32_t e : f)
      if (e != EZERO) acc += (unsigned __int128)1 << (2 * (e - emin));
    return ldexp((double)acc, 2 * emin);
  }
  std::vector<int32_t> s;
  for (int32_t e : f)
    if (e != EZERO) s.push_back(e);
  std::sort(s.begin(), s.end());
  double acc = 0.0;
  for (int32_t e : s) acc += ldexp(1.0, 2 * e);
  return acc;
}

int beta_rule(int64_t n, double delta, double g, double Lam, double S2, const frx_opts& o) {
  if (o.beta_override >= 0) return std::min(std::max(o.beta_override, 3), 47);
  double xi = o.xi > 0 ? o.xi : (double)n;
  if (g <= 0.0 || Lam <= 0.0 || S2 <= 0.0) return 3;
  double q = sqrt((xi * delta * g) / (Lam * S2)) / (0.75 * U53);
  int b = o.beta_ceil ? ceil_log2d(q) : floor_log2d(q);
  return std::min(std::max(b, 3), 47);
}

int alpha_rule(int64_t n, int beta, const frx_opts& o) {
  return o.theory_alpha ? 53 - beta + ceil_log2_int(n) : 53 - beta + ceil_log2_sqrt_int(n);
}

// smallest k >= 1 with (2^(7k - eL - eR - 6) tau)^2 >= n^3, capped at k_cap; 0 if an operand is zero
int slices_for(int64_t n, int eL, int eR, double tau, int kcap) {
  if (eL == EZERO || eR == EZERO) return 0;
  double n3 = (double)n * (double)n * (double)n;
  for (int k = 1; k <= kcap; ++k) {
    double v = ldexp(tau, 7 * k - eL - eR - 6);
    if (v * v >= n3) return k;
  }
  return kcap;
}

int vmax(const std::vector<int32_t>& v) {
  int m = EZERO;
  for (int32_t e : v) m = e > m ? e : m;
  return m;
}

template <class T>
int to_host(std::vector<T>& h, const T* d, int64_t n, cudaStream_t s) {
  h.resize((size_t)n);
  FRX_CUDA_TRY(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
  FRX_CUDA_TRY(cudaStreamSynchronize(s));
  return FRX_OK;
}

int check_flags(const int* dflags, cudaStream_t s) {
  int f = 0;
  FRX_CUDA_TRY(cudaMemcpyAsync(&f, dflags, sizeof(int), cudaMemcpyDeviceToHost, s));
  FRX_CUDA_TRY(cudaStreamSynchronize(s));
  if (f & FLAG_NONFINITE) return FRX_E_NONFINITE;
  if (f & FLAG_TIMEOUT) return FRX_E_TIMEOUT;
  if (f & FLAG_RANGE) return FRX_E_RANGE;
  return FRX_OK;
}

PlaneGemm make_gemm(const __nv_bfloat16* L, int64_t Lps, const __nv_bfloat16* R, int64_t Rps, int64_t pitch,
                    int64_t M, int64_t N, int64_t K, int kL, int kR, int T, i64* out) {
  PlaneGemm g;
  g.L = L;
  g.Lps = Lps;
  g.R = R;
  g.Rps = Rps;
  g.pitch = pitch;
  g.M = M;
  g.N = N;
  g.K = K;
  g.kL = kL;
  g.kR = kR;
  g.T = T;
  g.out = out;
  g.ogs = M * N;
  g.ldo = M;
  g.flags = nullptr;
  g.word32 = 0;
  g.out_bytes_per_elem = 64;
  g.tmax = g.gs = g.groups = 0;
  return g;
}

struct DebugOut {
  double *X1, *Vh, *Vl, *Res, *W, *E, *r;
};

int validate_opts(const frx_opts& o) {
  if (o.k_cap < 1 || o.k_cap > MAX_PLANES || o.max_iter < 1 || o.slices_A < 0 || o.slices_A > o.k_cap)
    return FRX_E_ARG;
  return FRX_OK;
}

// one iteration; lam_prev (host) in, lam_new (device ws.lam) out
int refine_iteration(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, double delta,
                     const frx_opts& o, RefineWs& ws, const std::vector<int32_t>& eA_h, int& sliced_kA,
                     const std::vector<double>& lam_prev, double omega_prev, frx_info& info, double& step,
                     double& omega_out, std::vector<double>& lam_new, const DebugOut* dbg, cudaStream_t s) {
  // S1: column exponents of X (eq. tau's w_j)
  FRX_TRY(launch_col_exponents(X, ldx, n, n, ws.f, ws.flags, s));
  std::vector<int32_t> f_h;
  FRX_TRY(to_host(f_h, ws.f, n, s));
  FRX_TRY(check_flags(ws.flags, s));
  for (int32_t e : f_h)
    if (e == EZERO) return FRX_E_ARG;  // a zero column is not an eigenvector approximation

  // S2: plan (Sec. 4.1), using the previous eigenvalue estimates
  double Lam;
  double g = min_gap(lam_prev, omega_prev, &Lam);
  double S2 = sum_pow4(f_h);
  int beta = beta_rule(n, delta, g, Lam, S2, o);
  int alpha = alpha_rule(n, beta, o);
  int sX = (54 - beta + 6) / 7;
  int eAmax = vmax(eA_h), fmax = vmax(f_h);
  int kV = o.slices_A > 0 ? o.slices_A : slices_for(n, eAmax, fmax, delta * g, o.k_cap);
  if (kV < 1) kV = 1;

  // S3: digit planes of A (rows of A = columns of A by symmetry); kept across iterations
  if (kV > sliced_kA) {
    FRX_TRY(launch_slice_cols(A, lda, n, n, ws.eA, kV, ws.Ap, ws.ps, ws.pitch, s));
    sliced_kA = kV;
  }
  // S4: X^(1) (eq. tau, eq. x) and its column planes
  FRX_TRY(launch_truncate_slice_x(X, ldx, n, ws.f, beta, sX, ws.X1, n, ws.Xp, ws.ps, ws.pitch, s));

  // S5/S6: V = A X^(1) (Alg. 1 line 1 with eq. mat_mul), pairs r + s <= k_V + 1
  PlaneGemm gv = make_gemm(ws.Ap, ws.ps, ws.Xp, ws.ps, ws.pitch, n, n, n, kV, sX, kV + 1, ws.groups);
  gv.flags = ws.flags;
  FRX_TRY(plan_plane_gemm(gv));
  FRX_TRY(launch_plane_gemm(gv, s));

  // S7/S8: r, lambda, Res (lines 2-4)
  ResidualArgs ra;
  ra.n = n;
  ra.V = group_args(gv);
  ra.eA = ws.eA;
  ra.f = ws.f;
  ra.X1 = ws.X1;
  ra.ld1 = n;
  ra.lam = ws.lam;
  ra.r = ws.r;
  ra.Res = ws.Res;
  ra.ldr = n;
  ra.h = ws.h;
  ra.beta = beta;
  ra.Vh = dbg ? dbg->Vh : nullptr;
  ra.Vl = dbg ? dbg->Vl : nullptr;
  FRX_TRY(launch_residual(ra, s));
  std::vector<int32_t> h_h;
  FRX_TRY(to_host(h_h, ws.h, n, s));

  // S9: W = X^(1)^T Res
  int hmax = vmax(h_h);
  int kW = slices_for(n, fmax, hmax, delta * g, o.k_cap);
  PlaneGemm gw = make_gemm(ws.Xp, ws.ps, ws.Rp, ws.ps, ws.pitch, n, n, n, std::min(sX, kW), kW, kW + 1,
                           ws.groups);
  gw.flags = ws.flags;
  if (kW > 0) {
    FRX_TRY(launch_slice_cols(ws.Res, n, n, n, ws.h, kW, ws.Rp, ws.ps, ws.pitch, s));
    FRX_TRY(plan_plane_gemm(gw));
    FRX_TRY(launch_plane_gemm(gw, s));
  } else {
    gw.groups = 0;
  }

  // S10: E~ (line 5) with the cluster threshold
  FRX_CUDA_TRY(cudaMemsetAsync(ws.norms, 0, 4 * sizeof(double), s));
  FRX_CUDA_TRY(cudaMemsetAsync(ws.flags + 1, 0, sizeof(int), s));
  CorrectionArgs ca;
  ca.n = n;
  ca.W = group_args(gw);
  ca.f = ws.f;
  ca.h = ws.h;
  ca.lam = ws.lam;
  ca.r = ws.r;
  ca.X1 = ws.X1;
  ca.ld1 = n;
  ca.E = ws.E;
  ca.lde = n;
  ca.eta = ws.eta;
  ca.norms = ws.norms;
  ca.ccount = ws.flags + 1;
  ca.flags = ws.flags;
  ca.Wout = dbg ? dbg->W : nullptr;
  double omega = o.cluster_omega;
  if (omega < 0) {
    double w2 = 0.0;
    if (gw.groups > 0) {
      FRX_TRY(launch_w_offdiag_norm2(ca, s));
      std::vector<double> nh;
      FRX_TRY(to_host(nh, ws.norms, 4, s));
      w2 = nh[1];
    }
    std::vector<double> rh;
    FRX_TRY(to_host(rh, ws.r, n, s));
    double rn = 0.0;
    for (double v : rh) rn += v * v;
    omega = 2.0 * (sqrt(w2) + Lam * sqrt(rn));
  }
  ca.omega = omega;
  FRX_TRY(launch_correction(ca, s));

  // S11: U = X^(1) E~ (rows of X^(1), columns of E~), X <- RN(X^(1) + U)
  FRX_TRY(launch_row_exponents(ws.X1, n, n, n, ws.rho, ws.rowmax, ws.flags, s));
  std::vector<int32_t> eta_h, rho_h;
  FRX_TRY(to_host(eta_h, ws.eta, n, s));
  FRX_TRY(to_host(rho_h, ws.rho, n, s));
  int kU = slices_for(n, vmax(rho_h), vmax(eta_h), delta, o.k_cap);
  PlaneGemm gu = make_gemm(ws.X1rp, ws.ps, ws.Rp, ws.ps, ws.pitch, n, n, n, kU, kU, kU + 1, ws.groups);
  gu.flags = ws.flags;
  if (kU > 0) {
    FRX_TRY(launch_slice_rows(ws.X1, n, n, n, ws.rho, kU, ws.X1rp, ws.ps, ws.pitch, s));
    FRX_TRY(launch_slice_cols(ws.E, n, n, n, ws.eta, kU, ws.Rp, ws.ps, ws.pitch, s));
    FRX_TRY(plan_plane_gemm(gu));
    FRX_TRY(launch_plane_gemm(gu, s));
  } else {
    gu.groups = 0;
  }
  if (dbg) {
    if (dbg->X1) FRX_CUDA_TRY(cudaMemcpyAsync(dbg->X1, ws.X1, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
    if (dbg->Res)
      FRX_CUDA_TRY(cudaMemcpyAsync(dbg->Res, ws.Res, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
    if (dbg->E) FRX_CUDA_TRY(cudaMemcpyAsync(dbg->E, ws.E, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
    if (dbg->r) FRX_CUDA_TRY(cudaMemcpyAsync(dbg->r, ws.r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  UpdateArgs ua;
  ua.n = n;
  ua.U = group_args(gu);
  ua.rho = ws.rho;
  ua.eta = ws.eta;
  ua.f = ws.f;
  ua.beta = beta;
  ua.X1 = ws.X1;
  ua.ld1 = n;
  ua.X = X;
  ua.ldx = ldx;
  ua.norms = ws.norms;
  FRX_TRY(launch_update(ua, s));

  std::vector<double> nh;
  FRX_TRY(to_host(nh, ws.norms, 4, s));
  FRX_TRY(to_host(lam_new, ws.lam, n, s));
  int cc = 0;
  FRX_CUDA_TRY(cudaMemcpyAsync(&cc, ws.flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  FRX_TRY(check_flags(ws.flags, s));

  step = sqrt(nh[2]);
  omega_out = omega;
  double Lam_new;
  double g_new = min_gap(lam_new, omega, &Lam_new);
  double xs = o.xi_stop > 0 ? o.xi_stop : (double)n;
  info.err_est = g_new > 0 ? step * step * Lam_new / (xs * g_new) : INFINITY;
  info.step = step;
  info.min_gap = g_new;
  info.max_lambda = Lam_new;
  info.beta = beta;
  info.alpha = alpha;
  info.s_X = sX;
  info.k_V = kV;
  info.k_W = kW;
  info.k_U = kU;
  info.omega = omega;
  info.clustered_pairs = cc / 2;
  info.products += pairs_in(kV, sX, kV + 1) + (kW > 0 ? pairs_in(std::min(sX, kW), kW, kW + 1) : 0) +
                   (kU > 0 ? pairs_in(kU, kU, kU + 1) : 0);
  return FRX_OK;
}

int refine_common(const double* A, int64_t lda, double* X, int64_t ldx, double* D, int64_t n, double delta,
                  const frx_opts* popts, double omega_prev, void* work, size_t work_bytes, frx_info* pinfo,
                  const DebugOut* dbg, bool single, void* stream) {
  frx_opts o;
  frx_default_opts(&o);
  if (popts) o = *popts;
  frx_info info;
  memset(&info, 0, sizeof(info));
  int st = FRX_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (!A || !X || !D || n < 1 || lda < n || ldx < n) st = FRX_E_ARG;
  else if (n > FRX_MAX_N) st = FRX_E_UNSUPPORTED;
  else if (!(delta > U53)) st = FRX_E_DELTA;
  else if (validate_opts(o) < 0) st = FRX_E_ARG;
  RefineWs ws = carve_refine(nullptr, n, o.k_cap);
  if (st == FRX_OK && (!work || !aligned256(work) || work_bytes < ws.bytes)) st = FRX_E_WORKSPACE;
  if (st == FRX_OK) {
    ws = carve_refine(work, n, o.k_cap);
    st = [&]() -> int {
      FRX_CUDA_TRY(cudaMemsetAsync(ws.flags, 0, 4 * sizeof(int), s));
      FRX_TRY(launch_col_exponents(A, lda, n, n, ws.eA, ws.flags, s));
      std::vector<int32_t> eA_h;
      FRX_TRY(to_host(eA_h, ws.eA, n, s));
      FRX_TRY(check_flags(ws.flags, s));
      std::vector<double> lam(n), lam_new;
      FRX_CUDA_TRY(cudaMemcpyAsync(lam.data(), D, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
      FRX_CUDA_TRY(cudaStreamSynchronize(s));
      for (double v : lam)
        if (!isfinite(v)) return FRX_E_NONFINITE;
      int sliced = 0;
      double omega = omega_prev, prev_step = -1.0;
      int status = FRX_MAX_ITER;
      int iters = single ? 1 : o.max_iter;
      for (int it = 1; it <= iters; ++it) {
        double step = 0.0, om = 0.0;
        FRX_TRY(refine_iteration(A, lda, X, ldx, n, delta, o, ws, eA_h, sliced, lam, omega, info, step, om,
                                 lam_new, dbg, s));
        info.iters = it;
        lam = lam_new;
        omega = om;
        if (info.err_est <= delta) {
          status = FRX_OK;
          break;
        }
        if (prev_step >= 0 && step > 0.5 * prev_step) {
          status = FRX_STAGNATED;
          break;
        }
        prev_step = step;
      }
      FRX_CUDA_TRY(cudaMemcpyAsync(D, lam.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
      FRX_CUDA_TRY(cudaStreamSynchronize(s));
      return status;
    }();
  }
  info.status = st;
  if (pinfo) *pinfo = info;
  return st;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void frx_default_opts(frx_opts* o) {
  if (!o) return;
  o->slices_A = 0;
  o->xi = 0.0;
  o->beta_ceil = 0;
  o->theory_alpha = 0;
  o->beta_override = -1;
  o->k_cap = 16;
  o->max_iter = 10;
  o->xi_stop = 0.0;
  o->cluster_omega = 0.0;
}

const char* frx_status_string(int st) {
  switch (st) {
    case FRX_OK: return "converged";
    case FRX_MAX_ITER: return "iteration limit reached";
    case FRX_STAGNATED: return "stagnated before reaching delta";
    case FRX_E_ARG: return "invalid argument";
    case FRX_E_NONFINITE: return "input contains Inf or NaN";
    case FRX_E_DELTA: return "delta must exceed 2^-53";
    case FRX_E_CUDA: return "CUDA error";
    case FRX_E_WORKSPACE: return "workspace missing, misaligned or too small";
    case FRX_E_TIMEOUT: return "device wait timed out";
    case FRX_E_UNSUPPORTED: return "size not supported";
    case FRX_E_RANGE: return "value range outside the digit grid";
    default: return "unknown status";
  }
}

size_t frx_refine_workspace_bytes(int64_t n, const frx_opts* opts) {
  if (n < 1 || n > FRX_MAX_N) return 0;
  int kcap = opts ? opts->k_cap : 16;
  if (kcap < 1 || kcap > MAX_PLANES) return 0;
  return carve_refine(nullptr, n, kcap).bytes;
}

int frx_refine(const double* A, int64_t lda, double* X, int64_t ldx, double* D, int64_t n, double delta,
               const frx_opts* opts, void* work, size_t work_bytes, frx_info* info, void* stream) {
  return refine_common(A, lda, X, ldx, D, n, delta, opts, 0.0, work, work_bytes, info, nullptr, false, stream);
}

int frx_refine_step(const double* A, int64_t lda, double* X, int64_t ldx, double* D, int64_t n, double delta,
                    const frx_opts* opts, double omega_prev, void* work, size_t work_bytes, frx_info* info,
                    double* X1, double* Vh, double* Vl, double* Res, double* W, double* E, double* r_out,
                    void* stream) {
  DebugOut d{X1, Vh, Vl, Res, W, E, r_out};
  int st = refine_common(A, lda, X, ldx, D, n, delta, opts, omega_prev, work, work_bytes, info, &d, true, stream);
  // a single step reports soft statuses as-is; FRX_MAX_ITER only means "not yet converged"
  return st;
}

size_t frx_ozaki_gemm_workspace_bytes(int64_t m, int64_t n, int64_t k, int slices) {
  if (m < 1 || n < 1 || k < 1 || slices < 1 || slices > MAX_PLANES) return 0;
  return carve_gemm(nullptr, m, n, k, slices).bytes;
}

int frx_ozaki_gemm(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                   double* C_lo, int64_t m, int64_t n, int64_t k, int slices, int mode, void* work,
                   size_t work_bytes, void* stream) {
  if (!A || !B || !C || m < 1 || n < 1 || k < 1 || lda < m || ldb < k || ldc < m) return FRX_E_ARG;
  if (slices < 1 || slices > MAX_PLANES || (mode != FRX_MODE_FULL && mode != FRX_MODE_TRIANGULAR)) return FRX_E_ARG;
  if (m > (1 << 20) || n > (1 << 20) || k > 65536) return FRX_E_UNSUPPORTED;
  GemmWs ws = carve_gemm(nullptr, m, n, k, slices);
  if (!work || !aligned256(work) || work_bytes < ws.bytes) return FRX_E_WORKSPACE;
  ws = carve_gemm(work, m, n, k, slices);
  cudaStream_t s = (cudaStream_t)stream;
  FRX_CUDA_TRY(cudaMemsetAsync(ws.flags, 0, 4 * sizeof(int), s));
  FRX_TRY(launch_row_exponents(A, lda, m, k, ws.eA, ws.rowmax, ws.flags, s));
  FRX_TRY(launch_col_exponents(B, ldb, k, n, ws.eB, ws.flags, s));
  FRX_TRY(launch_slice_rows(A, lda, m, k, ws.eA, slices, ws.Ap, m * ws.pitch, ws.pitch, s));
  FRX_TRY(launch_slice_cols(B, ldb, k, n, ws.eB, slices, ws.Bp, n * ws.pitch, ws.pitch, s));
  int T = mode == FRX_MODE_FULL ? 2 * slices : slices + 1;
  PlaneGemm g = make_gemm(ws.Ap, m * ws.pitch, ws.Bp, n * ws.pitch, ws.pitch, m, n, k, slices, slices, T, ws.groups);
  g.flags = ws.flags;
  FRX_TRY(plan_plane_gemm(g));
  FRX_TRY(launch_plane_gemm(g, s));
  FRX_TRY(launch_groups_to_dd(g, ws.eA, ws.eB, C, ldc, C_lo, ldc, s));
  return check_flags(ws.flags, s);
}

size_t frx_exponents_workspace_bytes(int64_t rows) {
  if (rows < 1) return 0;
  return 256 + (size_t)round_up(8 * rows, 256);
}

int frx_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int axis, int32_t* e, void* work,
                  size_t work_bytes, void* stream) {
  if (!M || !e || rows < 1 || cols < 1 || ld < rows || (axis != 0 && axis != 1)) return FRX_E_ARG;
  if (!work || !aligned256(work) || work_bytes < frx_exponents_workspace_bytes(rows)) return FRX_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  int* flags = (int*)work;
  u64* scratch = (u64*)((char*)work + 256);
  FRX_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
  if (axis == 0) {
    FRX_TRY(launch_row_exponents(M, ld, rows, cols, e, scratch, flags, s));
  } else {
    FRX_TRY(launch_col_exponents(M, ld, rows, cols, e, flags, s));
  }
  return check_flags(flags, s);
}

int frx_slice_planes(const double* M, int64_t ld, int64_t rows, int64_t cols, int axis, const int32_t* e, int k,
                     uint16_t* planes, int64_t plane_stride, int64_t pitch, void* stream) {
  if (!M || !e || !planes || rows < 1 || cols < 1 || ld < rows || k < 1 || k > MAX_PLANES) return FRX_E_ARG;
  if (pitch % 8 || pitch < (axis == 0 ? cols : rows)) return FRX_E_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(planes);
  if (axis == 0) return launch_slice_rows(M, ld, rows, cols, e, k, p, plane_stride, pitch, s);
  if (axis == 1) return launch_slice_cols(M, ld, rows, cols, e, k, p, plane_stride, pitch, s);
  return FRX_E_ARG;
}

int frx_group_size(int kL, int kR, int T, int64_t K) {
  PlaneGemm g = make_gemm(nullptr, 0, nullptr, 0, 8, 1, 1, K, kL, kR, T, nullptr);
  g.out_bytes_per_elem = 0;  // int64 groups only (any count): the documented format
  int st = plan_plane_gemm(g);
  return st < 0 ? st : g.gs;
}

int frx_plane_products(const uint16_t* L, int64_t L_plane_stride, const uint16_t* R, int64_t R_plane_stride,
                       int64_t pitch, int64_t m, int64_t n, int64_t K, int kL, int kR, int T, int64_t* out,
                       void* stream) {
  if (!L || !R || !out || m < 1 || n < 1 || K < 1 || pitch < K || pitch % 8 || kL < 1 || kR < 1) return FRX_E_ARG;
  PlaneGemm g = make_gemm(reinterpret_cast<const __nv_bfloat16*>(L), L_plane_stride,
                          reinterpret_cast<const __nv_bfloat16*>(R), R_plane_stride, pitch, m, n, K, kL, kR, T,
                          reinterpret_cast<i64*>(out));
  g.out_bytes_per_elem = 0;
  FRX_TRY(plan_plane_gemm(g));
  return launch_plane_gemm(g, (cudaStream_t)stream);
}

}  // extern "C"
