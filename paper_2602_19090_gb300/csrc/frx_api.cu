// C ABI of frx: argument checks, workspace layout, the host-side plan of each
// iteration (Sec. 3.3 / Sec. 4.1) and the refinement loop (Algorithm 1 iterated).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <vector>

#include "frx_internal.cuh"
#include "grouped.cuh"
#include "kernels.cuh"
#include "refine_kernels.cuh"
#include "plan_launch.cuh"
#include "profile.cuh"

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
  DevPlan* plan;
  double* lam_prev;
  int* flags;      // [0] flags, [1] cluster count
  double* colsq;   // per-column squared norms [3][n]: E~, off-diagonal W, X_new - X_old
  int32_t *eA, *f, *h, *eta, *rho;
  u64* rowmax;
  double *lam, *r;
  double *X1, *Res, *E;
  __nv_bfloat16 *Ap, *Xp, *Rp, *X1rp;
  i64* groups;
  int32_t* ell;    // nonzero columns of A's rows (sparse V product), ELL_MAX per row
  uint32_t* rank;  // positions of the eigenvalue estimates in ascending order (plan kernels)
  int64_t pitch, ps;
  size_t bytes;
  int tile;        // tile configuration of the slice products (set by the autotuner)
  int sparse_v;    // > 0: V = A X^(1) over A's nonzeros, at most sparse_v of them per row
};

RefineWs carve_refine(void* work, int64_t n, int kcap) {
  RefineWs w;
  Carver c(work);
  w.pitch = round_up(n, 64);
  w.ps = n * w.pitch;
  w.plan = c.take<DevPlan>(1);
  w.lam_prev = c.take<double>(n);
  w.flags = c.take<int>(4);
  w.eA = c.take<int32_t>(n);
  w.f = c.take<int32_t>(n);
  w.h = c.take<int32_t>(n);
  w.eta = c.take<int32_t>(n);
  w.rho = c.take<int32_t>(n);
  w.rowmax = c.take<u64>(n);
  w.colsq = c.take<double>(3 * n);
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
  w.ell = c.take<int32_t>((size_t)ELL_MAX * n);
  w.rank = c.take<uint32_t>(n);
  w.bytes = c.off + 256;
  w.tile = TILE_128x256;
  w.sparse_v = 0;
  return w;
}

struct GemmWs {
  int* flags;
  int32_t *eA, *eB;
  u64* rowmax;
  __nv_bfloat16 *Ap, *Bp;
  i64* groups;
  int out_bytes;   // bytes per product entry of the exact-sum buffer
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
  // exact sums: one int32 plane per anti-diagonal (at most 2 slices - 1 of them, full set),
  // at least 64 bytes per entry for the int64 grouping used beyond the int32 bound
  w.out_bytes = 4 * (2 * slices - 1) > 64 ? 4 * (2 * slices - 1) : 64;
  w.groups = c.take<i64>((size_t)((w.out_bytes + 7) / 8) * m * n);
  w.bytes = c.off + 256;
  return w;
}

bool aligned256(const void* p) { return ((uintptr_t)p & 255) == 0; }

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
  if (f & FLAG_CONFIG) return FRX_E_UNSUPPORTED;
  return FRX_OK;
}

PlaneGemm make_gemm(const __nv_bfloat16* L, int64_t Lps, const __nv_bfloat16* R, int64_t Rps, int64_t pitch,
                    int64_t M, int64_t N, int64_t K, int kL, int kR, int T, i64* out) {
  PlaneGemm g;
  memset(&g, 0, sizeof(g));
  g.L = L;
  g.Lps = Lps;
  g.R = R;
  g.Rps = Rps;
  g.pitch = pitch;
  g.M = M;
  g.N = N;
  g.K = K;
  g.d.kL = kL;
  g.d.kR = kR;
  g.d.T = T;
  g.out = out;
  g.ogs = M * N;
  g.ldo = M;
  g.flags = nullptr;
  g.dyn = nullptr;
  g.done = nullptr;
  g.out_bytes_per_elem = 64;
  return g;
}

struct DebugOut {
  double *X1, *Vh, *Vl, *Res, *W, *E, *r;
};

// Choice of the V product under the sparse rule: FRX_SPARSE_V=0 keeps the dense product,
// FRX_SPARSE_V=1 takes the sparse one whenever the pattern fits the ELL layout (cross-checks and
// measurements), otherwise the sparse one is taken when its CUDA-core work (nnz per row) stays
// below the dense tensor-core work (n per row): nnz * 160 <= n.  Measured on GB300 at n = 2048
// and 4096, the two take equal time near nnz * 136 = n; the factor 160 keeps a margin.
int sparse_v_mode() {
  const char* env = getenv("FRX_SPARSE_V");
  if (env && env[0] == '0') return 0;
  if (env && env[0] == '1') return 2;
  return 1;
}

int validate_opts(const frx_opts& o) {
  if (o.k_cap < 1 || o.k_cap > MAX_PLANES || o.max_iter < 1 || o.slices_A < 0 || o.slices_A > o.k_cap)
    return FRX_E_ARG;
  // x_planes digit planes of X: at most ceil(56 / DIGIT_BITS), the full FP64 width
  if (o.x_planes < 0 || o.x_planes > (56 + DIGIT_BITS - 1) / DIGIT_BITS) return FRX_E_ARG;
  if (o.sparse_rule != 0 && o.sparse_rule != 1) return FRX_E_ARG;
  return FRX_OK;
}

PlanOpts plan_opts(const frx_opts& o, double delta, int64_t n, int max_iter) {
  PlanOpts p;
  p.slices_A = o.slices_A;
  p.xi = o.xi;
  p.beta_ceil = o.beta_ceil;
  p.theory_alpha = o.theory_alpha;
  p.beta_override = o.beta_override;
  p.k_cap = o.k_cap;
  p.max_iter = max_iter;
  p.xi_stop = o.xi_stop;
  p.cluster_omega = o.cluster_omega;
  p.x_planes = o.x_planes;
  p.sparse_rule = o.sparse_rule;
  p.delta = delta;
  p.n = n;
  return p;
}

// a plan-driven product: d carries the plane capacities (tensor maps) and the kernel variant
PlaneGemm dyn_gemm(const __nv_bfloat16* L, int capL, const __nv_bfloat16* R, int capR, const RefineWs& ws,
                   int64_t n, const GemmDesc* dyn) {
  PlaneGemm g = make_gemm(L, ws.ps, R, ws.ps, ws.pitch, n, n, n, capL, capR, capL + capR, ws.groups);
  g.d.active = 1;
  g.d.word32 = 1;
  g.d.groups = 1;
  g.dyn = dyn;
  g.done = &ws.plan->done;
  g.flags = &ws.plan->flags;
  g.tile = ws.tile;
  return g;
}

// the representative product the autotuner times for a refinement of order n: 8 planes of
// A (fewer when k_cap is smaller) against 5 planes of X^(1), the triangular set r + s <= kL + 1
PlaneGemm tuning_gemm(const RefineWs& ws, int64_t n, int kcap) {
  const int kL = kcap < 8 ? kcap : 8, kR = 5;
  PlaneGemm g = make_gemm(ws.Ap, ws.ps, ws.Xp, ws.ps, ws.pitch, n, n, n, kL, kR, kL + 1, ws.groups);
  g.out_bytes_per_elem = 64;
  g.flags = &ws.plan->flags;
  return g;
}

// One iteration of Algorithm 1 (Sec. 3 form), entirely on the stream: every decision is
// taken by the plan kernels and read back by the kernels that follow.
int enqueue_iteration(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, const frx_opts& o,
                      const PlanOpts& po, const RefineWs& ws, const DebugOut* dbg, cudaStream_t s) {
  DevPlan* P = ws.plan;
  const int* done = &P->done;
  int* flags = &P->flags;
  const int kcap = o.k_cap;
  // S1 / S2: column exponents of X (eq. tau's w_j), then beta, alpha, s_X, k_V
  FRX_TRY(launch_col_exponents(X, ldx, n, n, ws.f, flags, s, done));
  FRX_TRY(launch_plan_v(P, ws.f, po, s));
  // S3: digit planes of A (rows of A = columns of A by symmetry), extended when k_V grows
  SliceDyn da;
  da.nplanes = &P->kV;
  da.from = &P->sliced_kA;
  da.done = done;
  FRX_TRY(launch_slice_cols(A, lda, n, n, ws.eA, 0, ws.Ap, ws.ps, ws.pitch, s, da));
  FRX_TRY(launch_plan_mark_sliced(P, s));
  // S4: X^(1) (eq. tau, eq. x) and its column planes
  SliceDyn dx;
  dx.nplanes = &P->sX;
  dx.beta = &P->beta;
  dx.done = done;
  FRX_TRY(launch_truncate_slice_x(X, ldx, n, ws.f, 0, 0, ws.X1, n, ws.Xp, ws.ps, ws.pitch, s, dx));
  // S5/S6: V = A X^(1), pairs r + s <= k_V + 1
  PlaneGemm gv = dyn_gemm(ws.Ap, kcap, ws.Xp, 8, ws, n, &P->V);
  if (ws.sparse_v)
    FRX_TRY(launch_sparse_v(ws.Ap, ws.Xp, ws.ps, ws.pitch, ws.ell, ws.sparse_v, n, &P->V, done, flags, gv.out32(),
                            gv.ogs, s));
  else
    FRX_TRY(launch_plane_gemm(gv, s));
  // S7/S8: r, lambda, Res (Alg. 1)
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
  ra.beta = 0;
  ra.beta_dyn = &P->beta;
  ra.done = done;
  ra.Vh = dbg ? dbg->Vh : nullptr;
  ra.Vl = dbg ? dbg->Vl : nullptr;
  FRX_TRY(launch_residual(ra, s));
  // S9: W = X^(1)^T Res
  FRX_TRY(launch_plan_w(P, ws.h, po, s));
  SliceDyn dr;
  dr.nplanes = &P->kW;
  dr.done = done;
  FRX_TRY(launch_slice_cols(ws.Res, n, n, n, ws.h, 0, ws.Rp, ws.ps, ws.pitch, s, dr));
  PlaneGemm gw = dyn_gemm(ws.Xp, 8, ws.Rp, kcap, ws, n, &P->W);
  FRX_TRY(launch_plane_gemm(gw, s));
  // S10: E~ (Alg. 1) with the cluster threshold
  CorrectionArgs ca;
  ca.n = n;
  ca.W = group_args(gw);
  ca.f = ws.f;
  ca.h = ws.h;
  ca.lam = ws.lam;
  ca.r = ws.r;
  ca.X1 = ws.X1;
  ca.ld1 = n;
  ca.omega = 0.0;
  ca.omega_dyn = &P->omega;
  ca.done = done;
  ca.E = ws.E;
  ca.lde = n;
  ca.eta = ws.eta;
  ca.norms = ws.colsq;
  ca.ccount = &P->ccount;
  ca.flags = flags;
  ca.Wout = dbg ? dbg->W : nullptr;
  if (o.cluster_omega < 0) FRX_TRY(launch_w_offdiag_norm2(ca, s));
  FRX_TRY(launch_plan_omega(P, ws.r, ws.colsq, po, s));
  FRX_TRY(launch_correction(ca, s));
  // S11: U = X^(1) E~ (rows of X^(1), columns of E~), X <- RN(X^(1) + U)
  FRX_TRY(launch_row_exponents(ws.X1, n, n, n, ws.rho, ws.rowmax, flags, s, done));
  FRX_TRY(launch_plan_u(P, ws.rho, ws.eta, po, s));
  SliceDyn du;
  du.nplanes = &P->kU;
  du.done = done;
  FRX_TRY(launch_slice_rows(ws.X1, n, n, n, ws.rho, 0, ws.X1rp, ws.ps, ws.pitch, s, du));
  FRX_TRY(launch_slice_cols(ws.E, n, n, n, ws.eta, 0, ws.Rp, ws.ps, ws.pitch, s, du));
  PlaneGemm gu = dyn_gemm(ws.X1rp, kcap, ws.Rp, kcap, ws, n, &P->U);
  FRX_TRY(launch_plane_gemm(gu, s));
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
  ua.beta = 0;
  ua.beta_dyn = &P->beta;
  ua.done = done;
  ua.X1 = ws.X1;
  ua.ld1 = n;
  ua.X = X;
  ua.ldx = ldx;
  ua.norms = ws.colsq;
  FRX_TRY(launch_update(ua, s));
  // S12: stopping test
  FRX_TRY(launch_plan_end(P, ws.lam, ws.lam_prev, ws.colsq, po, ws.rank, s));
  return FRX_OK;
}

// dynamic shared memory limits of the refinement kernels, set once per device before any
// launch or capture
int ensure_attributes() {
  static PerDevice pd;
  return once_per_device(pd, [](int) {
    int st = set_refine_kernel_attributes();
    if (st == FRX_OK) st = set_plan_kernel_attributes();
    if (st == FRX_OK) st = set_sparse_v_attributes();
    if (st == FRX_OK) st = prepare_plane_gemm_grouped();
    return st;
  });
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
  DevPlan hp;
  memset(&hp, 0, sizeof(hp));
  if (st == FRX_OK) {
    ws = carve_refine(work, n, o.k_cap);
    const int max_iter = single ? 1 : o.max_iter;
    const PlanOpts po = plan_opts(o, delta, n, max_iter);
    st = [&]() -> int {
      FRX_TRY(ensure_attributes());
      FRX_CUDA_TRY(cudaMemsetAsync(ws.plan, 0, sizeof(DevPlan), s));
      FRX_CUDA_TRY(cudaMemsetAsync(ws.rowmax, 0, sizeof(u64) * n, s));
      PlaneGemm rep = tuning_gemm(ws, n, o.k_cap);
      FRX_TRY(plan_plane_gemm(rep));
      FRX_TRY(tune_tile_refine(rep, s, ws.tile));
      FRX_TRY(launch_col_exponents(A, lda, n, n, ws.eA, &ws.plan->flags, s, nullptr, &ws.plan->rownnz));
      const int svm = o.sparse_rule ? sparse_v_mode() : 0;
      if (svm) {
        // the sparse-matrix setting: V over A's nonzeros when every row holds at most ELL_MAX of
        // them and (unless forced) nnz * 160 <= n (one read of the count)
        int nz = 0;
        FRX_CUDA_TRY(cudaMemcpyAsync(&nz, &ws.plan->rownnz, sizeof(int), cudaMemcpyDeviceToHost, s));
        FRX_CUDA_TRY(cudaStreamSynchronize(s));
        if (nz >= 1 && nz <= ELL_MAX && (svm == 2 || (int64_t)nz * 160 <= n)) {
          FRX_TRY(launch_build_ell(A, lda, n, ws.ell, s));
          ws.sparse_v = nz;
        }
      }
      FRX_TRY(launch_plan_init(ws.plan, ws.eA, D, ws.lam_prev, po, omega_prev, ws.rank, s));
      for (int it = 1; it <= max_iter; ++it) {
        FRX_TRY(enqueue_iteration(A, lda, X, ldx, n, o, po, ws, dbg, s));
        int done = 0;
        FRX_CUDA_TRY(cudaMemcpyAsync(&done, &ws.plan->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        FRX_CUDA_TRY(cudaStreamSynchronize(s));
        if (done) break;
      }
      FRX_CUDA_TRY(cudaMemcpyAsync(&hp, ws.plan, sizeof(DevPlan), cudaMemcpyDeviceToHost, s));
      FRX_CUDA_TRY(cudaStreamSynchronize(s));
      if (hp.status >= 0 && hp.iter > 0)
        FRX_CUDA_TRY(cudaMemcpyAsync(D, ws.lam_prev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      FRX_CUDA_TRY(cudaStreamSynchronize(s));
      profile_add_gemm_work(2.0 * (double)n * (double)n * (double)n * (double)hp.products);
      return hp.status;
    }();
  }
  info.status = st;
  info.iters = hp.iter;
  info.beta = hp.beta;
  info.alpha = hp.alpha;
  info.s_X = hp.sX;
  info.k_V = hp.kV;
  info.k_W = hp.kW;
  info.k_U = hp.kU;
  info.products = hp.products;
  info.err_est = hp.est;
  info.step = hp.step;
  info.min_gap = hp.g;
  info.max_lambda = hp.Lam;
  info.omega = hp.omega;
  info.clustered_pairs = hp.clustered;
  if (pinfo) *pinfo = info;
  return st;
}

// ---------------------------------------------------------------------------
// batched refinement: every stage of an iteration is one grouped launch over all problems
// ---------------------------------------------------------------------------
// The launch sequence of one iteration is recorded once per problem (the same kernels in
// the same order, with each problem's arguments); stage k of every problem then runs as one
// launch whose blocks are the union of the problems' blocks, and the slice products of a
// stage run in one persistent tensor-core launch.  An iteration is one captured CUDA graph.
constexpr int BATCH_CHUNK = 2048;                      // problems per grouped launch
// Threads per column block of the residual, correction and update stages when every problem
// has n <= 512 (at most 8 rows per thread): on a batch of 256 matrices of n in [32, 511],
// 64 threads took 23.5 ms per batch against 25.3 (128) and 23.9 (32), the smaller block
// reductions and fewer idle threads outweighing the lower parallelism per column.
#ifndef FRX_BATCH_SMALL_THREADS
#define FRX_BATCH_SMALL_THREADS 64
#endif
constexpr size_t TABLE_BYTES_PER_PROBLEM = 16 * 1024;  // argument tables of all stages

struct BatchLayout {
  std::vector<size_t> off;
  size_t plans_off, done_off, gather_off, tables_off, tables_bytes, bytes;
};

BatchLayout batch_layout(const int64_t* n, int count, int kcap) {
  BatchLayout L;
  size_t off = 0;
  for (int b = 0; b < count; ++b) {
    L.off.push_back(off);
    off += round_up((int64_t)carve_refine(nullptr, n[b], kcap).bytes, 256);
  }
  const int chunk = count < BATCH_CHUNK ? count : BATCH_CHUNK;
  L.plans_off = off;
  off += round_up(sizeof(DevPlan*) * (size_t)chunk, 256);
  L.done_off = off;
  off += round_up(sizeof(int) * (size_t)chunk, 256);
  L.gather_off = off;
  off += round_up(sizeof(DevPlan) * (size_t)chunk, 256);
  L.tables_off = off;
  L.tables_bytes = TABLE_BYTES_PER_PROBLEM * (size_t)chunk + 65536;
  off += round_up((int64_t)L.tables_bytes, 256);
  L.bytes = off + 256;
  return L;
}

struct Stage {
  int kind;
  size_t tab_off, start_off;
  long long blocks;
  int threads;
  size_t smem;
  int variant;   // slice products: output tile width
};

// stage k of a phase groups record k of every problem (same kind and argument size); the
// slice-product stages list the problems in `gemm_order` (largest first, so that the
// persistent kernel's units come roughly in decreasing order of work), the others in batch order
int build_stages(const std::vector<std::vector<LaunchRecord>>& recs, const std::vector<int>& gemm_order,
                 std::vector<unsigned char>& blob, std::vector<Stage>& stages) {
  const int count = (int)recs.size();
  const size_t K = recs[0].size();
  for (int b = 1; b < count; ++b)
    if (recs[b].size() != K) return FRX_E_UNSUPPORTED;
  for (size_t k = 0; k < K; ++k) {
    Stage st;
    st.kind = recs[0][k].kind;
    const size_t sz = recs[0][k].args.size();
    st.blocks = 0;
    st.threads = 0;
    st.smem = 0;
    st.variant = recs[0][k].variant;
    st.tab_off = (blob.size() + 63) / 64 * 64;
    blob.resize(st.tab_off + sz * (size_t)count);
    for (int b = 0; b < count; ++b) {
      const int src = st.kind == LK_GEMM ? gemm_order[b] : b;
      const LaunchRecord& r = recs[src][k];
      if (r.kind != st.kind || r.args.size() != sz || r.variant != st.variant) return FRX_E_UNSUPPORTED;
      memcpy(blob.data() + st.tab_off + sz * b, r.args.data(), sz);
    }
    st.start_off = (blob.size() + 7) / 8 * 8;
    blob.resize(st.start_off + sizeof(long long) * (size_t)(count + 1));
    long long* start = reinterpret_cast<long long*>(blob.data() + st.start_off);
    for (int b = 0; b < count; ++b) {
      const LaunchRecord& r = recs[b][k];
      start[b] = st.blocks;
      st.blocks += r.blocks;
      st.threads = r.threads > st.threads ? r.threads : st.threads;
      st.smem = r.smem > st.smem ? r.smem : st.smem;
    }
    start[count] = st.blocks;
    if (st.kind == LK_RESIDUAL || st.kind == LK_CORRECTION || st.kind == LK_UPDATE) {
      // one block per column: with every problem at n <= 1024 columns are short, and 128
      // threads per block (up to 8 rows each) keep fewer threads idle at the same occupancy
      long long most = 0;
      for (int b = 0; b < count; ++b) most = recs[b][k].blocks > most ? recs[b][k].blocks : most;
      if (most <= 1024) st.threads = 128;
      if (most <= 512) st.threads = FRX_BATCH_SMALL_THREADS;
      // the residual's copy stages follow its V column and grow with the block
      if (st.kind == LK_RESIDUAL) {
        if (residual_launch_smem(most, st.threads) > RESIDUAL_SMEM_MAX) st.threads = 128;
        st.smem = residual_launch_smem(most, st.threads);
      }
    }
    stages.push_back(st);
  }
  return FRX_OK;
}

int launch_stage(const Stage& st, char* tables, int count, cudaStream_t s) {
  const void* tab = tables + st.tab_off;
  const long long* start = reinterpret_cast<const long long*>(tables + st.start_off);
  switch (st.kind) {
    case LK_GEMM:
      return launch_plane_gemm_grouped(tab, count, st.variant, s);
    case LK_COL_EXPONENTS:
    case LK_ROW_MAXBITS:
    case LK_MAXBITS_TO_EXPONENTS:
    case LK_SLICE_COLS:
    case LK_SLICE_ROWS:
    case LK_TRUNCATE_SLICE_X:
    case LK_ZERO:
    case LK_COPY:
      return launch_grouped_scan(st.kind, tab, start, count, st.blocks, st.threads, st.smem, s);
    case LK_RESIDUAL:
    case LK_W_OFFDIAG:
    case LK_CORRECTION:
    case LK_UPDATE:
      return launch_grouped_refine(st.kind, tab, start, count, st.blocks, st.threads, st.smem, s);
    default:
      return launch_grouped_plan(st.kind, tab, start, count, st.blocks, st.threads, st.smem, s);
  }
}

// the library's own stream for the batched path (captures cannot use the legacy stream),
// bridged to the caller's stream with events
// Launch plan of one batched chunk: its recorded stages, their argument tables (pinned host
// copy, uploaded into the caller's scratch on every call) and the instantiated iteration graph.
// A later call with the same key (pointers, leading dimensions, orders, options, delta, scratch,
// tile policy) reuses it and skips the recording, the tensor-map encoding and the capture.
struct BatchPlan {
  std::vector<unsigned char> key;
  unsigned char* blob = nullptr;   // pinned
  size_t blob_bytes = 0;
  std::vector<DevPlan*> hplans;
  std::vector<Stage> stages[3];
  cudaGraphExec_t exec = nullptr;
  long long last_use = 0;
};

#ifndef FRX_BATCH_PLAN_CACHE
#define FRX_BATCH_PLAN_CACHE 4   // plans kept per device (0: none)
#endif

// One per device.  `busy` serialises batched calls on the device: they share the stream,
// its events, the graph capture on it and the plan cache, which concurrent callers would
// interleave.
struct BatchStream {
  cudaStream_t s = nullptr;
  cudaEvent_t enter = nullptr, leave = nullptr;
  std::mutex busy;
  std::vector<BatchPlan*> plans;
  long long uses = 0;
};

int batch_stream(BatchStream** out) {
  static std::mutex mu;
  static BatchStream streams[64];
  int dev = 0;
  FRX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return FRX_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  BatchStream& b = streams[dev];
  if (!b.s) {
    FRX_CUDA_TRY(cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking));
    FRX_CUDA_TRY(cudaEventCreateWithFlags(&b.enter, cudaEventDisableTiming));
    FRX_CUDA_TRY(cudaEventCreateWithFlags(&b.leave, cudaEventDisableTiming));
  }
  *out = &b;
  return FRX_OK;
}

// record the three phases of every problem: setup, one iteration, finish
int record_phases(const double* const* A, const int64_t* lda, double* const* X, const int64_t* ldx,
                  double* const* D, const int64_t* n, int count, const frx_opts& o, const std::vector<PlanOpts>& po,
                  const std::vector<RefineWs>& ws, int tile, std::vector<std::vector<LaunchRecord>> (&rec)[3]) {
  LaunchRecorder R;
  R.tile = tile;
  LaunchRecorder*& active = active_recorder();
  active = &R;
  cudaStream_t none = nullptr;   // nothing is launched while recording
  int st = [&]() -> int {
    for (int b = 0; b < count; ++b) {
      R.recs.clear();
      FRX_TRY(record_bytes(ws[b].plan, nullptr, sizeof(DevPlan)));
      FRX_TRY(record_bytes(ws[b].rowmax, nullptr, sizeof(u64) * (size_t)n[b]));
      FRX_TRY(launch_col_exponents(A[b], lda[b], n[b], n[b], ws[b].eA, &ws[b].plan->flags, none, nullptr,
                                    &ws[b].plan->rownnz));
      FRX_TRY(launch_plan_init(ws[b].plan, ws[b].eA, D[b], ws[b].lam_prev, po[b], 0.0, nullptr, none));
      rec[0][b] = std::move(R.recs);
      R.recs.clear();
      FRX_TRY(enqueue_iteration(A[b], lda[b], X[b], ldx[b], n[b], o, po[b], ws[b], nullptr, none));
      rec[1][b] = std::move(R.recs);
      R.recs.clear();
      FRX_TRY(record_bytes(D[b], ws[b].lam_prev, sizeof(double) * (size_t)n[b]));
      rec[2][b] = std::move(R.recs);
    }
    return FRX_OK;
  }();
  active = nullptr;
  return st;
}

template <class T>
void key_append(std::vector<unsigned char>& k, const T& v) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
  k.insert(k.end(), p, p + sizeof(T));
}

// record, tune, build the argument tables and capture the iteration graph of a chunk
int build_batch_plan(const double* const* A, const int64_t* lda, double* const* X, const int64_t* ldx,
                     double* const* D, const int64_t* n, int count, double delta, const frx_opts& o, char* base,
                     const BatchLayout& L, const size_t* off, cudaStream_t s, BatchPlan& plan) {
  std::vector<RefineWs> ws(count);
  std::vector<PlanOpts> po(count);
  plan.hplans.resize(count);
  for (int b = 0; b < count; ++b) {
    ws[b] = carve_refine(base + off[b], n[b], o.k_cap);
    plan.hplans[b] = ws[b].plan;
    po[b] = plan_opts(o, delta, n[b], o.max_iter);
  }
  // tile configuration of the grouped slice products: cached per batch signature (the sorted orders),
  // else timed on representative products over the problems' plane buffers
  int tile = TILE_128x256;
  {
    std::vector<PlaneGemm> reps(count);
    std::vector<long long> key = {3, count, o.k_cap};
    std::vector<int64_t> sorted(n, n + count);
    std::sort(sorted.begin(), sorted.end());
    key.insert(key.end(), sorted.begin(), sorted.end());
    for (int b = 0; b < count; ++b) {
      reps[b] = tuning_gemm(ws[b], n[b], o.k_cap);
      FRX_TRY(plan_plane_gemm(reps[b]));
    }
    FRX_TRY(tune_tile_grouped(reps, key, base + L.tables_off, s, tile));
  }
  for (int b = 0; b < count; ++b) ws[b].tile = tile;
  std::vector<std::vector<LaunchRecord>> rec[3];
  for (int q = 0; q < 3; ++q) rec[q].resize(count);
  FRX_TRY(record_phases(A, lda, X, ldx, D, n, count, o, po, ws, tile, rec));
  std::vector<int> gemm_order(count);
  for (int b = 0; b < count; ++b) gemm_order[b] = b;
  std::stable_sort(gemm_order.begin(), gemm_order.end(), [&](int x, int y) { return n[x] > n[y]; });
  std::vector<unsigned char> blob;
  for (int q = 0; q < 3; ++q) FRX_TRY(build_stages(rec[q], gemm_order, blob, plan.stages[q]));
  if (blob.size() > L.tables_bytes) return FRX_E_UNSUPPORTED;
  FRX_CUDA_TRY(cudaHostAlloc((void**)&plan.blob, blob.size() ? blob.size() : 1, cudaHostAllocDefault));
  memcpy(plan.blob, blob.data(), blob.size());
  plan.blob_bytes = blob.size();
  // the iteration, captured once: every stage of it plus the collection of the finish flags
  char* tables = base + L.tables_off;
  DevPlan** dplans = (DevPlan**)(base + L.plans_off);
  int* ddone = (int*)(base + L.done_off);
  cudaGraph_t graph = nullptr;
  FRX_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int cst = [&]() -> int {
    for (const Stage& st : plan.stages[1]) FRX_TRY(launch_stage(st, tables, count, s));
    return launch_collect_done(dplans, count, ddone, s);
  }();
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (cst != FRX_OK) {
    if (graph) cudaGraphDestroy(graph);
    return cst;
  }
  if (e != cudaSuccess) return FRX_E_CUDA;
  e = cudaGraphInstantiate(&plan.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return FRX_E_CUDA;
  count_launches(-(int)(plan.stages[1].size() + 1));   // captured, not launched: counted per replay
  return FRX_OK;
}

void free_batch_plan(BatchPlan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->blob) cudaFreeHost(p->blob);
  delete p;
}

int refine_batched_chunk(const double* const* A, const int64_t* lda, double* const* X, const int64_t* ldx,
                         double* const* D, const int64_t* n, int count, double delta, const frx_opts& o, char* base,
                         const BatchLayout& L, const size_t* off, frx_info* infos, BatchStream& bs) {
  cudaStream_t s = bs.s;
  // the plan's key: everything the recorded launches depend on
  std::vector<unsigned char> key;
  key_append(key, count);
  key_append(key, base);
  key_append(key, delta);
  // the options field by field (the struct's padding bytes are not part of the key)
  key_append(key, o.slices_A);
  key_append(key, o.xi);
  key_append(key, o.beta_ceil);
  key_append(key, o.theory_alpha);
  key_append(key, o.beta_override);
  key_append(key, o.k_cap);
  key_append(key, o.max_iter);
  key_append(key, o.xi_stop);
  key_append(key, o.cluster_omega);
  key_append(key, o.x_planes);
  key_append(key, o.sparse_rule);
  key_append(key, tile_policy());
  for (int b = 0; b < count; ++b) {
    key_append(key, A[b]);
    key_append(key, lda[b]);
    key_append(key, X[b]);
    key_append(key, ldx[b]);
    key_append(key, D[b]);
    key_append(key, n[b]);
    key_append(key, off[b]);
  }
  BatchPlan* plan = nullptr;
  for (BatchPlan* p : bs.plans)
    if (p->key == key) plan = p;
  bool owned = false;   // a plan not kept in the cache is freed at the end of the call
  if (!plan) {
    plan = new BatchPlan();
    plan->key = key;
    const int st = build_batch_plan(A, lda, X, ldx, D, n, count, delta, o, base, L, off, s, *plan);
    if (st != FRX_OK) {
      free_batch_plan(plan);
      return st;
    }
    if (FRX_BATCH_PLAN_CACHE > 0) {
      if ((int)bs.plans.size() >= FRX_BATCH_PLAN_CACHE) {
        auto lru = std::min_element(bs.plans.begin(), bs.plans.end(),
                                    [](BatchPlan* x, BatchPlan* y) { return x->last_use < y->last_use; });
        free_batch_plan(*lru);
        bs.plans.erase(lru);
      }
      bs.plans.push_back(plan);
    } else {
      owned = true;
    }
  }
  plan->last_use = ++bs.uses;
  char* tables = base + L.tables_off;
  DevPlan** dplans = (DevPlan**)(base + L.plans_off);
  int* ddone = (int*)(base + L.done_off);
  DevPlan* gathered = (DevPlan*)(base + L.gather_off);
  int st = [&]() -> int {
    // the argument tables live in the caller's scratch, which may have been reused since
    FRX_CUDA_TRY(cudaMemcpyAsync(tables, plan->blob, plan->blob_bytes, cudaMemcpyHostToDevice, s));
    FRX_CUDA_TRY(
        cudaMemcpyAsync(dplans, plan->hplans.data(), sizeof(DevPlan*) * count, cudaMemcpyHostToDevice, s));
    for (const Stage& sg : plan->stages[0]) FRX_TRY(launch_stage(sg, tables, count, s));
    std::vector<int> done(count);
    for (int it = 1; it <= o.max_iter; ++it) {
      FRX_CUDA_TRY(cudaGraphLaunch(plan->exec, s));
      count_launches((long long)plan->stages[1].size() + 1);   // the graph's kernels, per replay
      FRX_CUDA_TRY(cudaMemcpyAsync(done.data(), ddone, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
      FRX_CUDA_TRY(cudaStreamSynchronize(s));
      bool all = true;
      for (int b = 0; b < count; ++b) all &= done[b] != 0;
      if (all) break;
    }
    for (const Stage& sg : plan->stages[2]) FRX_TRY(launch_stage(sg, tables, count, s));
    FRX_TRY(launch_gather_plans(dplans, count, gathered, s));
    std::vector<DevPlan> hp(count);
    FRX_CUDA_TRY(cudaMemcpyAsync(hp.data(), gathered, sizeof(DevPlan) * count, cudaMemcpyDeviceToHost, s));
    FRX_CUDA_TRY(cudaStreamSynchronize(s));
    int worst = FRX_OK;
    double ops = 0.0;
    for (int b = 0; b < count; ++b) {
      const DevPlan& P = hp[b];
      ops += 2.0 * (double)n[b] * (double)n[b] * (double)n[b] * (double)P.products;
      if (infos) {
        frx_info& I = infos[b];
        memset(&I, 0, sizeof(I));
        I.status = P.status;
        I.iters = P.iter;
        I.beta = P.beta;
        I.alpha = P.alpha;
        I.s_X = P.sX;
        I.k_V = P.kV;
        I.k_W = P.kW;
        I.k_U = P.kU;
        I.products = P.products;
        I.err_est = P.est;
        I.step = P.step;
        I.min_gap = P.g;
        I.max_lambda = P.Lam;
        I.omega = P.omega;
        I.clustered_pairs = P.clustered;
      }
      if (P.status < 0) {
        if (worst >= 0) worst = P.status;
      } else if (worst >= 0 && P.status > worst) {
        worst = P.status;
      }
    }
    profile_add_gemm_work(ops);
    return worst;
  }();
  if (owned) free_batch_plan(plan);
  return st;
}

int refine_batched_impl(const double* const* A, const int64_t* lda, double* const* X, const int64_t* ldx,
                        double* const* D, const int64_t* n, int count, double delta, const frx_opts& o, void* work,
                        size_t work_bytes, frx_info* infos, cudaStream_t caller) {
  BatchLayout L = batch_layout(n, count, o.k_cap);
  if (!work || !aligned256(work) || work_bytes < L.bytes) return FRX_E_WORKSPACE;
  FRX_TRY(ensure_attributes());
  BatchStream* bs = nullptr;
  FRX_TRY(batch_stream(&bs));
  std::lock_guard<std::mutex> serial(bs->busy);
  cudaStream_t s = bs->s;
  FRX_CUDA_TRY(cudaEventRecord(bs->enter, caller));
  FRX_CUDA_TRY(cudaStreamWaitEvent(s, bs->enter, 0));
  int worst = FRX_OK;
  for (int c0 = 0; c0 < count; c0 += BATCH_CHUNK) {
    const int c = count - c0 < BATCH_CHUNK ? count - c0 : BATCH_CHUNK;
    int st = refine_batched_chunk(A + c0, lda + c0, X + c0, ldx + c0, D + c0, n + c0, c, delta, o, (char*)work, L,
                                  L.off.data() + c0, infos ? infos + c0 : nullptr, *bs);
    if (st < 0) {
      worst = st;
      break;
    }
    if (worst >= 0 && st > worst) worst = st;
  }
  if (cudaEventRecord(bs->leave, s) != cudaSuccess || cudaStreamWaitEvent(caller, bs->leave, 0) != cudaSuccess)
    return FRX_E_CUDA;
  return worst;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void frx_default_opts(frx_opts* o) {
  if (!o) return;
  o->slices_A = 0;
  o->xi = 1.0;
  o->beta_ceil = 0;
  o->theory_alpha = 0;
  o->beta_override = -1;
  o->k_cap = 16;
  o->max_iter = 10;
  o->xi_stop = 0.0;
  o->cluster_omega = 0.0;
  o->x_planes = 0;
  o->sparse_rule = 0;
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

size_t frx_refine_batched_workspace_bytes(const int64_t* n, int count, const frx_opts* opts) {
  if (!n || count < 1) return 0;
  int kcap = opts ? opts->k_cap : 16;
  if (kcap < 1 || kcap > MAX_PLANES) return 0;
  for (int b = 0; b < count; ++b)
    if (n[b] < 1 || n[b] > FRX_MAX_N) return 0;
  return batch_layout(n, count, kcap).bytes;
}

int frx_refine_batched(const double* const* A, const int64_t* lda, double* const* X, const int64_t* ldx,
                       double* const* D, const int64_t* n, int count, double delta, const frx_opts* opts, void* work,
                       size_t work_bytes, frx_info* infos, void* stream) {
  frx_opts o;
  frx_default_opts(&o);
  if (opts) o = *opts;
  if (!A || !lda || !X || !ldx || !D || !n || count < 1) return FRX_E_ARG;
  if (!(delta > U53)) return FRX_E_DELTA;
  if (validate_opts(o) < 0) return FRX_E_ARG;
  for (int b = 0; b < count; ++b) {
    if (!A[b] || !X[b] || !D[b] || n[b] < 1 || lda[b] < n[b] || ldx[b] < n[b]) return FRX_E_ARG;
    if (n[b] > FRX_MAX_N) return FRX_E_UNSUPPORTED;
  }
  // the scratch is checked before any device call, as in frx_refine
  if (!work || !aligned256(work) || work_bytes < batch_layout(n, count, o.k_cap).bytes) return FRX_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FRX_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return FRX_E_ARG;
  return refine_batched_impl(A, lda, X, ldx, D, n, count, delta, o, work, work_bytes, infos, s);
}

int frx_check_wait_timeout(void* work, size_t work_bytes, void* stream) {
  if (!work || !aligned256(work) || work_bytes < 256) return FRX_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  int* flags = (int*)work;
  FRX_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
  FRX_TRY(launch_wait_timeout(flags, s));
  return check_flags(flags, s);
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
  FRX_CUDA_TRY(cudaMemsetAsync(ws.rowmax, 0, sizeof(u64) * m, s));
  FRX_TRY(launch_row_exponents(A, lda, m, k, ws.eA, ws.rowmax, ws.flags, s));
  FRX_TRY(launch_col_exponents(B, ldb, k, n, ws.eB, ws.flags, s));
  FRX_TRY(launch_slice_rows(A, lda, m, k, ws.eA, slices, ws.Ap, m * ws.pitch, ws.pitch, s));
  FRX_TRY(launch_slice_cols(B, ldb, k, n, ws.eB, slices, ws.Bp, n * ws.pitch, ws.pitch, s));
  int T = mode == FRX_MODE_FULL ? 2 * slices : slices + 1;
  PlaneGemm g = make_gemm(ws.Ap, m * ws.pitch, ws.Bp, n * ws.pitch, ws.pitch, m, n, k, slices, slices, T, ws.groups);
  g.out_bytes_per_elem = ws.out_bytes;
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
  FRX_CUDA_TRY(cudaMemsetAsync(work, 0, frx_exponents_workspace_bytes(rows), s));
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
  return st < 0 ? st : g.d.gs;
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
