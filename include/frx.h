/*
 * frx: forward-error-oriented eigenvector refinement with Ozaki-scheme products
 * on GB300 (sm_103a).  C ABI.
 *
 * Method: Terao & Ozaki, "Forward Error-Oriented Iterative Refinement for
 * Eigenvectors of a Real Symmetric Matrix": Algorithm 1 (Ogita-Aishima step) with
 * the Sec. 3 modification (X^ is replaced by its beta-truncated first slice X^(1),
 * eq. tau / eq. x, and A X^(1) is formed by n_A error-free slice products,
 * eq. mat_mul) and the Sec. 4.1 choice of alpha and beta.  The error-free slices
 * of Sec. 2.3 (eq. sigma, eq. a) are taken on a fixed 8-bit digit grid so that
 * every slice is an integer digit in [-128, 128] (exact in bfloat16): slice r of a row
 * (or column) whose maximum magnitude v satisfies 2^(e-1) < v <= 2^e has weight
 * 2^(e + 1 - 8r).  Slice products run on the tensor cores with exact integer
 * accumulation and are recombined in double-double.
 *
 * Conventions for every call below:
 *  - Matrices are FP64, column-major, with a leading dimension ld >= rows
 *    (element (i, j) at p[i + j * ld]).  All matrix and vector pointers are
 *    DEVICE pointers unless a parameter says "host".
 *  - `stream` is a cudaStream_t passed as void* (NULL: the legacy default stream).
 *    Work is enqueued on it; calls that return information to the host
 *    (frx_refine's info, the status word) synchronise that stream.
 *  - `work` is caller-owned device scratch of at least the bytes the matching
 *    *_workspace_bytes call returns, 256-byte aligned.  The library allocates no
 *    device memory.  Scratch contents are undefined after a call.
 *  - The caller owns every buffer.  The library keeps no pointer after a call.
 *  - Return value: an frx_status.  Negative values are hard errors; outputs are
 *    then unspecified.  No C++ exception crosses this boundary.
 */
#ifndef FRX_H
#define FRX_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FRX_API __attribute__((visibility("default")))
#else
#define FRX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FRX_OK = 0,              /* converged: error estimate <= delta                       */
  FRX_MAX_ITER = 1,        /* soft: max_iter reached, info->err_est filled              */
  FRX_STAGNATED = 2,       /* soft: the step stopped halving before convergence          */
  FRX_E_ARG = -1,          /* bad size, leading dimension, pointer, option or alignment   */
  FRX_E_NONFINITE = -2,    /* an input entry is Inf or NaN                                */
  FRX_E_DELTA = -3,        /* delta <= u = 2^-53 (Sec. 3.1 requires delta > u)            */
  FRX_E_CUDA = -4,         /* a CUDA runtime call or kernel launch failed                  */
  FRX_E_WORKSPACE = -5,    /* work is NULL, misaligned or smaller than required            */
  FRX_E_TIMEOUT = -6,      /* a bounded device-side wait gave up                           */
  FRX_E_UNSUPPORTED = -7,  /* size outside the supported range                            */
  FRX_E_RANGE = -8         /* exponent range too wide for the fixed digit grid            */
} frx_status;

/* Product set of an Ozaki product: all (r, s) with r <= kL, s <= kR. */
#define FRX_MODE_FULL 0
/* Triangular set r + s <= k + 1: k(k+1)/2 products (cited after eq. alp_beta). */
#define FRX_MODE_TRIANGULAR 1

/* Options of frx_refine.  Fill with frx_default_opts, then override. */
typedef struct {
  int slices_A;          /* 0: automatic number of A slices k_V; > 0: fixed (e.g. 8)        */
  double xi;             /* > 0: eq. proposed_beta with this xi (default 1); <= 0: xi = n, the
                            "n delta" form of the Sec. 4.1 experiments                          */
  int beta_ceil;         /* 0: floor (Sec. 4.1); 1: ceil (eq. proposed_beta)                  */
  int theory_alpha;      /* 0: alpha = 53 - beta + ceil(log2 sqrt n) (Sec. 4.1);
                            1: alpha = 53 - beta + ceil(log2 n) (eq. proposed_beta)           */
  int beta_override;     /* < 0: use the rule; else a fixed beta (clamped to [3, 47])          */
  int k_cap;             /* largest number of digit planes per operand, 1..16                  */
  int max_iter;          /* iteration limit (>= 1)                                           */
  double xi_stop;        /* <= 0: n.  Stop when step^2 * max|lam| / (xi_stop * gap) <= delta  */
  double cluster_omega;  /* >= 0: |lam_j - lam_i| <= omega is a cluster pair (0: only equal
                            estimates); < 0: Ogita-Aishima threshold
                            2 (||W||_F + max|lam| ||diag R||_2) each iteration              */
  int x_planes;          /* 0: X^(1) from the Sec. 3 truncation (beta rule).  1..7: X is kept at
                            x_planes digit planes (rounded to the last plane's grid, beta =
                            54 - 8 x_planes) with no truncation rule: the "previous study"
                            form of Sec. 4 (both operands sliced; 7 planes = full FP64 width) */
  int sparse_rule;       /* 0: the dense Sec. 4.1 beta rule.  1: the sparse-matrix rule of Sec. 4
                            (xi = min(k, sqrt n)^2, alpha = 53 - beta + ceil(log2 k)) with k the
                            largest number of nonzeros in a row of A, counted on the device   */
} frx_opts;

/* Per-call report of frx_refine (host struct). */
typedef struct {
  int status;            /* same as the return value                                      */
  int iters;             /* iterations performed                                          */
  int beta, alpha;       /* last iteration's beta (eq. tau) and alpha (Sec. 4.1)           */
  int s_X;               /* digit planes of X^(1) = ceil((54 - beta) / 8)                 */
  int k_V, k_W, k_U;     /* slice counts of the three products of the last iteration      */
  long long products;    /* slice-pair products executed over all iterations              */
  double err_est;        /* est = step^2 * max|lam| / (xi_stop * gap), last iteration      */
  double step;           /* ||X_k - X_{k-1}||_F of the last iteration                      */
  double min_gap;        /* smallest gap of the final eigenvalue estimates (clusters excluded) */
  double max_lambda;     /* max |lam| of the final estimates                              */
  double omega;          /* cluster threshold used in the last iteration                  */
  int clustered_pairs;   /* cluster pairs treated by the r_ij / 2 rule in the last iteration */
} frx_info;

/* Default options: automatic slices, eq. proposed_beta with xi = 1 and floor rounding (Sec. 4.1),
 * k_cap 16, max_iter 10. */
FRX_API void frx_default_opts(frx_opts* opts);

/* Text for a status code (static storage). */
FRX_API const char* frx_status_string(int status);

/* Scratch bytes frx_refine needs for order n (independent of the options' values
 * except k_cap).  Returns 0 for n outside [1, FRX_MAX_N]. */
FRX_API size_t frx_refine_workspace_bytes(int64_t n, const frx_opts* opts);

#define FRX_MAX_N 12288

/*
 * Refine approximate eigenpairs of the symmetric matrix A (n x n) until the
 * forward-error estimate reaches delta (Algorithm 1 iterated, Sec. 3 and 4.1).
 *   A     (in)      n x n, lda >= n.  Must be exactly symmetric; both triangles are read.
 *   X     (in/out)  n x n, ldx >= n: approximate eigenvectors X^ on entry, refined X^ on
 *                   exit (the column order and signs are kept).
 *   D     (in/out)  n: eigenvalue estimates; on entry they set the first iteration's
 *                   beta and slice counts (the estimates of iteration k-1 are used in
 *                   iteration k); on exit the estimates lam_i = x_i^T v_i / (1 - r_i)
 *                   of the last iteration (the estimates of Alg. 1).
 *   delta (in)      target forward error, delta > 2^-53.
 *   opts  (in,host) options, or NULL for the defaults.
 *   info  (out,host) may be NULL.
 * Errors: FRX_E_ARG (also for n < 1: an empty problem is refused, not refined), FRX_E_DELTA,
 * FRX_E_NONFINITE, FRX_E_WORKSPACE, FRX_E_UNSUPPORTED (n > FRX_MAX_N), FRX_E_RANGE,
 * FRX_E_TIMEOUT, FRX_E_CUDA.  The plan of each iteration
 * (beta, alpha, plane counts, the stopping test) is computed on the device; the host
 * synchronises `stream` once per iteration to read the finish flag, and once more at the end
 * to read the report.  The first call for a new n may time the tile configurations of the
 * slice products (see frx_set_tile).
 */
FRX_API int frx_refine(const double* A, int64_t lda, double* X, int64_t ldx, double* D, int64_t n,
               double delta, const frx_opts* opts, void* work, size_t work_bytes,
               frx_info* info, void* stream);

/*
 * One iteration of Algorithm 1 (Sec. 3 form) with optional copies of its
 * intermediates, for inspection and testing.  Same arguments as frx_refine;
 * `D` holds the previous estimates on entry and the new ones on exit; `omega_prev`
 * is the cluster threshold of the previous iteration (0 on the first).  Each
 * optional output (NULL to skip) is an n x n column-major FP64 matrix with ld = n:
 *   X1  the truncated slice X^(1) (eq. tau, eq. x)
 *   Vh, Vl  V = A X^(1) as a double-double (Alg. 1, eq. mat_mul)
 *   Res     V - X^(1) diag(lam), rounded to FP64 (inside W, Alg. 1)
 *   W       X^(1)^T Res (Alg. 1)
 *   E       the correction E~ (Alg. 1)
 * `r_out` (n, device, optional) receives r_i = 1 - x_i^T x_i (Alg. 1).
 * info->err_est/step refer to this single step.
 */
FRX_API int frx_refine_step(const double* A, int64_t lda, double* X, int64_t ldx, double* D, int64_t n,
                    double delta, const frx_opts* opts, double omega_prev,
                    void* work, size_t work_bytes, frx_info* info,
                    double* X1, double* Vh, double* Vl, double* Res, double* W, double* E,
                    double* r_out, void* stream);

/*
 * Batched refinement of `count` independent symmetric problems of possibly different
 * orders (each as in frx_refine, with the same delta and options).  A, X, D, lda, ldx and
 * n are HOST arrays of length `count` holding device pointers and sizes.  Every stage of
 * an iteration runs as one grouped launch over all problems (the slice products as one
 * persistent tensor-core launch); the iteration is captured once into a CUDA graph and
 * replayed until every problem has converged, stagnated or reached max_iter.  Each
 * problem's plan lives on the device, so the host reads only an array of finish flags per
 * iteration.  Problems are processed in chunks of 2048.  The refined X and D, the
 * iteration and product counts equal those of frx_refine on each problem, bit for bit (the
 * reported norms may differ in their last bits: columns are summed with another block
 * size).  `infos` (host, `count` entries) may be NULL.  Batched calls on one device from
 * several host threads run one after another (they share the library's stream for the
 * device).  Launch plans: the library keeps, per device, the launch plans of the last 4
 * distinct batched calls (recorded stages, a pinned host copy of their argument tables, the
 * instantiated iteration graph) and reuses one when a call has the same pointers, leading
 * dimensions, orders, options, delta and scratch; the tables are uploaded into the scratch
 * on every call and all device work is redone.
 * Returns FRX_OK if every problem converged, else the largest soft status (1, 2), or the
 * first hard error (< 0; the per-problem statuses are then in infos when it is not NULL).
 * Argument errors, checked before any device work: count < 1, a NULL array or pointer, an
 * order below 1 or a leading dimension below it (FRX_E_ARG), delta <= u (FRX_E_DELTA), an
 * order above FRX_MAX_N (FRX_E_UNSUPPORTED), scratch NULL, not 256-byte aligned or below
 * frx_refine_batched_workspace_bytes (FRX_E_WORKSPACE).
 * The call must not be made while `stream` is being captured.
 */
FRX_API size_t frx_refine_batched_workspace_bytes(const int64_t* n, int count, const frx_opts* opts);
FRX_API int frx_refine_batched(const double* const* A, const int64_t* lda, double* const* X,
                               const int64_t* ldx, double* const* D, const int64_t* n, int count,
                               double delta, const frx_opts* opts, void* work, size_t work_bytes,
                               frx_info* infos, void* stream);

/* Scratch bytes of frx_ozaki_gemm for these sizes and k. */
FRX_API size_t frx_ozaki_gemm_workspace_bytes(int64_t m, int64_t n, int64_t k, int slices);

/*
 * C = A B by the Ozaki scheme (Sec. 2.3): A (m x k) is split by rows and B (k x n)
 * by columns into `slices` digit planes each (eq. sigma/tau, eq. a/x on the fixed
 * 8-bit grid); the products of the selected plane pairs (FRX_MODE_FULL: all
 * slices^2; FRX_MODE_TRIANGULAR: r + s <= slices + 1) are exact integer matrices,
 * recombined exactly per anti-diagonal and rounded: C = RN(C_hi + C_lo).
 *   C_lo (out, optional) receives the low word of the double-double result
 *   (ld = ldc).  When the planes hold A and B exactly and mode is FULL, C_hi + C_lo
 *   equals the exact product to about 2^-104 relative.
 * slices in [1, 16]; m, n, k in [1, 2^20] with k <= 65536; A, B finite.  The exact sums
 * are int32 planes while (pairs per anti-diagonal) * k * 2^14 < 2^31, int64 groups beyond
 * (slower).
 */
FRX_API int frx_ozaki_gemm(const double* A, int64_t lda, const double* B, int64_t ldb,
                   double* C, int64_t ldc, double* C_lo, int64_t m, int64_t n, int64_t k,
                   int slices, int mode, void* work, size_t work_bytes, void* stream);

/*
 * frx_ozaki_gemm without caller scratch, for callers that cannot allocate device
 * memory (for example a plugin inside a framework that has reserved the whole device
 * memory for its own allocator, or code that is given a stream but no allocator).
 * The paper has no counterpart: this is a library convenience around frx_ozaki_gemm.
 * Same arguments and results as frx_ozaki_gemm, minus `work`/`work_bytes`.
 *   Limits: m, n, k <= 512 and slices <= 8; larger sizes return FRX_E_UNSUPPORTED
 *   before any device work.
 *   Scratch: a fixed 24 MiB + 64 KiB array of device memory inside this library.  It is
 *   reserved on a device when the library's code for this call is loaded there: with
 *   CUDA's default lazy module loading at the first call on that device (with
 *   CUDA_MODULE_LOADING=EAGER when the library is loaded), and it is held until the process
 *   exits.  A caller whose framework later takes all free device memory must therefore make
 *   one call on each device first.  The call allocates nothing.  Every call looks up the
 *   array's device address on the current device (a host-side query).  Call with the device
 *   that owns `stream` current.  Like frx_ozaki_gemm, every call synchronises `stream` to
 *   read back its status word, so no call may be made while `stream` is being captured.
 *   Sharing: every call uses the same array and leaves its contents behind (each call
 *   clears what it needs).  Calls whose GPU work overlaps (different streams or host
 *   threads without ordering) race on the array: order them, e.g. on one stream.
 */
FRX_API int frx_ozaki_gemm_static(const double* A, int64_t lda, const double* B, int64_t ldb,
                                  double* C, int64_t ldc, double* C_lo, int64_t m, int64_t n,
                                  int64_t k, int slices, int mode, void* stream);

/*
 * Digit planes of the slice products, for bit-exact checks of the integer path.
 *   frx_exponents: e[i] = ceil(log2 max |row i|) (axis 0) or of column j (axis 1) of an
 *     rows x cols matrix; -2^30 for an all-zero line.  Returns FRX_E_NONFINITE on Inf/NaN.
 *     Needs frx_exponents_workspace_bytes(rows) bytes of scratch; synchronises `stream`.
 *   frx_slice_planes: bfloat16 digit planes (as uint16 bit patterns) of the matrix,
 *     split by rows (axis 0) or columns (axis 1) with the exponents e; plane r is
 *     stored at planes + r * plane_stride as `lines x pitch` (line = row for axis 0,
 *     column for axis 1; pitch >= the other dimension, multiple of 8; the pad is zero).
 *   frx_plane_products: the exact anti-diagonal sums of the slice products grouped
 *     into int64 words: out[g * n * m + j * m + i] = sum over t in group g of
 *     2^(8 (t_last(g) - t)) * sum_{r + s = t, r <= kL, s <= kR, t <= T} (L_r R_s)_ij,
 *     groups of `frx_group_size(...)` consecutive t starting at t = 2.
 */
FRX_API size_t frx_exponents_workspace_bytes(int64_t rows);
FRX_API int frx_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int axis,
                  int32_t* e, void* work, size_t work_bytes, void* stream);
FRX_API int frx_slice_planes(const double* M, int64_t ld, int64_t rows, int64_t cols, int axis,
                     const int32_t* e, int k, uint16_t* planes, int64_t plane_stride,
                     int64_t pitch, void* stream);
FRX_API int frx_group_size(int kL, int kR, int T, int64_t K);
FRX_API int frx_plane_products(const uint16_t* L, int64_t L_plane_stride, const uint16_t* R,
                       int64_t R_plane_stride, int64_t pitch, int64_t m, int64_t n, int64_t K,
                       int kL, int kR, int T, int64_t* out, void* stream);

/*
 * Launch accounting and kernel timing (native tracing).
 *   kernel_launches  kernels this library launched since the last reset
 *   gemm_launches    slice-product GEMM launches among them
 *   gemm_ms          summed CUDA-event time of those GEMM launches, measured on the
 *                    stream they were launched on (only while profiling is on)
 *   gemm_ops         algorithmic operations of those launches: 2 m n K per slice pair
 *   gemm_bytes       algorithmic bytes: every digit plane read once (2 bytes per
 *                    digit) plus every int64 group word written once
 *   simt_launches    slice-product launches among gemm_launches that ran on the CUDA cores
 *                    instead of the tensor cores (about 100 times slower): the driver lacks
 *                    the tensor-map encoder, an operand of frx_plane_products is not 16-byte
 *                    aligned or its plane stride or pitch is not a multiple of 8 digits, or
 *                    FRX_GEMM=simt is set.  The library's own products never take it.
 * frx_profile_enable(1) starts timing every GEMM launch with a pair of CUDA events;
 * frx_profile_read waits for the recorded events, fills `out` (host) and, if `reset`
 * is nonzero, clears the counters.  Thread-safe; the counters are process-wide.
 */
typedef struct {
  long long kernel_launches;
  long long gemm_launches;
  double gemm_ms;
  double gemm_ops;
  double gemm_bytes;
  long long simt_launches;
} frx_profile;

FRX_API void frx_profile_enable(int on);
FRX_API int frx_profile_read(frx_profile* out, int reset);

/*
 * Self-test of the bounded device waits.  Every wait of the tensor-core kernels on an
 * mbarrier gives up after 2 s (by the global timer), raises a flag and returns, so that a call
 * whose device work stalls reports FRX_E_TIMEOUT instead of hanging.  This call runs one such
 * wait on a barrier that nothing completes and returns what a stalled call returns:
 * FRX_E_TIMEOUT, after about 2 s.  `work`: at least 256 bytes of device scratch, 256-byte
 * aligned.  Synchronises `stream`; the context stays usable afterwards.
 */
FRX_API int frx_check_wait_timeout(void* work, size_t work_bytes, void* stream);

/*
 * Tile autotuner of the slice products (no counterpart in the paper; it changes the time of
 * a product, never its result: every tile sum is exact).
 *   The tensor-core kernel covers a product's m x n output with one of two tile
 *   configurations, one CTA per tile: FRX_TILE_128x128 or FRX_TILE_128x256.
 *   The first time a product shape is seen (frx_ozaki_gemm: m, n, k, planes and pair bound;
 *   frx_refine: n and the plane capacities; frx_refine_batched: the sorted orders of the
 *   batch), a cost model settles it when 128 x 256 tiles cover the output with under 3%
 *   padding and leave at least 4 units per SM; otherwise every offered configuration is
 *   timed with CUDA events on the call's stream (4 launches each, one stream
 *   synchronisation) and the fastest is cached for the shape, process-wide.  On a stream
 *   under capture nothing is timed or cached: the model's estimate is used.
 *   frx_set_tile(t): FRX_TILE_AUTO (0, default) autotunes; another FRX_TILE_* forces that
 *     configuration (int64 exact sums always use 128 x 128 tiles).  Returns the previous
 *     setting, or FRX_E_ARG for another value.  Process-wide.
 *   frx_last_tile(): the configuration of the last slice-product launch made by the calling
 *     host thread (FRX_TILE_AUTO before any).
 *   frx_tune_stats: decisions taken by timing and by the model, and cache hits, since the
 *     last clear (clear != 0 also empties the cache).  Any pointer may be NULL.
 */
#define FRX_TILE_AUTO 0
#define FRX_TILE_128x128 1
#define FRX_TILE_128x256 2
FRX_API int frx_set_tile(int tile);
FRX_API int frx_last_tile(void);
FRX_API int frx_tune_stats(long long* measured, long long* modelled, long long* hits, int clear);

#ifdef __cplusplus
}
#endif
#endif /* FRX_H */
