// Exponent scans and fixed-grid digit slicing (Sec. 2.3, eq. sigma/tau, eq. a/x;
// eq. tau with s = 1 for the truncation X^(1) of Sec. 3).
//
// Every kernel is a body over its block coordinates (bx, by): launched on its own with
// blockIdx, or grouped over many problems (grouped.cuh) for the batched refinement.
#include "frx_internal.cuh"
#include "grouped.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace frx {

struct ColExpArgs {
  const double* M;
  int64_t ld, rows, cols;
  int32_t* e;
  int* flags;
  const int* done;
  int* nnz_max;   // optional: atomic max of the columns' nonzero counts
  unsigned gx;
};

struct RowMaxArgs {
  const double* M;
  int64_t ld, rows, cols;
  u64* rowmax;
  int* flags;
  const int* done;
  unsigned gx;
};

struct MaxToExpArgs {
  u64* mx;
  int64_t n;
  int32_t* e;
  const int* done;
  unsigned gx;
};

struct SliceArgs {   // slice_cols (rows = K, lines = N) and slice_rows (rows = M rows, K = columns)
  const double* M;
  int64_t ld, K, lines;
  const int32_t* e;
  int nplanes;
  __nv_bfloat16* planes;
  int64_t ps, pitch;
  SliceDyn dyn;
  unsigned gx;
};

struct TruncArgs {
  const double* X;
  int64_t ldx, n;
  const int32_t* f;
  int beta, nplanes;
  double* X1;
  int64_t ld1;
  __nv_bfloat16* planes;
  int64_t ps, pitch;
  SliceDyn dyn;
  unsigned gx;
};

struct BytesArgs {   // zero (src == nullptr) or copy `words` 8-byte words
  u64* dst;
  const u64* src;
  int64_t words;
  unsigned gx;
};

// ---- S1: exponent of every column (one block per column) ------------------
__device__ __forceinline__ void col_exponents_body(ColExpArgs a, unsigned bx, unsigned) {
  if (a.done && *a.done) return;
  const int64_t j = bx;
  const double* col = a.M + j * a.ld;
  u64 mx = 0;
  bool bad = false;
  int nz = 0;
  for (int64_t i = threadIdx.x; i < a.rows; i += blockDim.x) {
    u64 ab = double_to_bits(col[i]) & 0x7fffffffffffffffull;
    bad |= nonfinite_absbits(ab);
    nz += ab != 0;
    mx = ab > mx ? ab : mx;
  }

  for (int o = 16; o > 0; o >>= 1) {
    u64 other = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = other > mx ? other : mx;
  }
  __shared__ u64 red[8];
  __shared__ int sbad, snz;
  if (threadIdx.x == 0) sbad = snz = 0;
  __syncthreads();
  if (bad) atomicOr(&sbad, 1);
  if (a.nnz_max) {
    for (int o = 16; o > 0; o >>= 1) nz += __shfl_xor_sync(0xffffffffu, nz, o);
    if ((threadIdx.x & 31) == 0 && nz) atomicAdd(&snz, nz);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = red[w] > mx ? red[w] : mx;
    mx = red[0] > mx ? red[0] : mx;
    a.e[j] = sbad ? EZERO : (mx == 0 ? EZERO : ceil_log2_absbits(mx));
    if (sbad) atomicOr(a.flags, FLAG_NONFINITE);
    if (a.nnz_max && snz) atomicMax(a.nnz_max, snz);
  }
}

// ---- S1: exponent of every row of a column-major matrix --------------------
// blocks (ceil(rows / 256), ceil(cols / 64)); rowmax must be zeroed first.
__device__ __forceinline__ void row_maxbits_body(RowMaxArgs a, unsigned bx, unsigned by) {
  if (a.done && *a.done) return;
  int64_t i = (int64_t)bx * 256 + threadIdx.x;
  if (i >= a.rows) return;
  int64_t j0 = (int64_t)by * 64;
  int64_t j1 = j0 + 64 < a.cols ? j0 + 64 : a.cols;
  u64 mx = 0;
  bool bad = false;
  for (int64_t j = j0; j < j1; ++j) {
    u64 ab = double_to_bits(a.M[i + j * a.ld]) & 0x7fffffffffffffffull;
    bad |= nonfinite_absbits(ab);
    mx = ab > mx ? ab : mx;
  }
  if (bad) atomicOr(a.flags, FLAG_NONFINITE);
  if (mx) atomicMax(a.rowmax + i, mx);
}

__device__ __forceinline__ void maxbits_to_exponents_body(MaxToExpArgs a, unsigned bx, unsigned) {
  if (a.done && *a.done) return;
  int64_t i = (int64_t)bx * blockDim.x + threadIdx.x;
  if (i < a.n) {
    a.e[i] = a.mx[i] == 0 ? EZERO : ceil_log2_absbits(a.mx[i]);
    a.mx[i] = 0;  // ready for the next scan
  }
}

__device__ __forceinline__ void bytes_body(BytesArgs a, unsigned bx, unsigned) {
  for (int64_t w = (int64_t)bx * blockDim.x + threadIdx.x; w < a.words; w += (int64_t)a.gx * blockDim.x)
    a.dst[w] = a.src ? a.src[w] : 0ull;
}
// Two consecutive entries per thread: their digits of one plane are stored as one bf16x2
// word when the plane layout allows it (4-byte aligned base, even strides).
__device__ __forceinline__ bool pair_stores_ok(const __nv_bfloat16* planes, int64_t ps, int64_t pitch) {
  return ((uintptr_t)planes & 3) == 0 && (ps & 1) == 0 && (pitch & 1) == 0;
}

__device__ __forceinline__ void store_digit_pair(__nv_bfloat16* out, bool pair, bool second, int d0, int d1) {
  if (pair) {
    *reinterpret_cast<__nv_bfloat162*>(out) = __halves2bfloat162(digit_bf16(d0), digit_bf16(d1));
  } else {
    out[0] = digit_bf16(d0);
    if (second) out[1] = digit_bf16(d1);
  }
}

// ---- S3/S4: digit planes along columns (no transpose) ---------------------
// planes[r * ps + j * pitch + k] = digit r of M[k, j] (column exponent e[j]); pad k in [K, pitch) = 0.
// planes [from, nplanes) are written; nplanes / from may come from the device plan
__device__ __forceinline__ void slice_cols_body(SliceArgs a, unsigned bx, unsigned by) {
  const double* __restrict__ M = a.M;
  const int64_t ld = a.ld, K = a.K, pitch = a.pitch, ps = a.ps;
  const int32_t* __restrict__ e = a.e;
  __nv_bfloat16* __restrict__ planes = a.planes;
  const SliceDyn dyn = a.dyn;
  int nplanes = a.nplanes;
  if (dyn.done && *dyn.done) return;
  if (dyn.nplanes) nplanes = *dyn.nplanes;
  const int from = dyn.from ? *dyn.from : 0;
  if (from >= nplanes) return;
  const int64_t k = 2 * ((int64_t)by * 256 + threadIdx.x);
  const int64_t j = bx;   // columns on x: N may exceed 65535
  if (k >= pitch) return;
  __nv_bfloat16* out = planes + j * pitch + k;
  const int ej = e[j];
  const bool live = ej != EZERO;
  i64 P[2];
  int q[2];
  decompose(live && k < K ? M[k + j * ld] : 0.0, P[0], q[0]);
  decompose(live && k + 1 < K ? M[k + 1 + j * ld] : 0.0, P[1], q[1]);
  const bool pair = pair_stores_ok(planes, ps, pitch) && k + 1 < pitch;
  const bool second = k + 1 < pitch;
  for_each_digit<2>(P, q, live ? ej : 0, nplanes, [&](int r, const int (&d)[2]) {
    if (r > from) store_digit_pair(out + (int64_t)(r - 1) * ps, pair, second, d[0], d[1]);
  });
}

// ---- digit planes along rows of a column-major matrix (transpose through smem) ----
// planes[r * ps + i * pitch + k] = digit r of M[i, k] (row exponent e[i]); tile 8 rows x 64
// columns; each thread takes one row and two consecutive k (paired stores).
__device__ __forceinline__ void slice_rows_body(SliceArgs a, unsigned bx, unsigned by) {
  const double* __restrict__ M = a.M;
  const int64_t ld = a.ld, rows = a.lines, K = a.K, pitch = a.pitch, ps = a.ps;
  const int32_t* __restrict__ e = a.e;
  __nv_bfloat16* __restrict__ planes = a.planes;
  const SliceDyn dyn = a.dyn;
  int nplanes = a.nplanes;
  if (dyn.done && *dyn.done) return;
  if (dyn.nplanes) nplanes = *dyn.nplanes;
  if (nplanes <= 0) return;
  __shared__ double tile[8][65];
  const int64_t i0 = (int64_t)bx * 8, k0 = (int64_t)by * 64;   // rows may reach 2^20
  {
    const int ii = threadIdx.x & 7, kk = threadIdx.x >> 3;  // 8 rows x 32 columns per pass
    for (int pass = 0; pass < 2; ++pass) {
      const int c = kk + 32 * pass;
      const int64_t i = i0 + ii, k = k0 + c;
      tile[ii][c] = (i < rows && k < K) ? M[i + k * ld] : 0.0;
    }
  }
  __syncthreads();
  const int ii = threadIdx.x >> 5, kp = threadIdx.x & 31;
  const int64_t i = i0 + ii, k = k0 + 2 * kp;
  if (i >= rows || k >= pitch) return;
  __nv_bfloat16* out = planes + i * pitch + k;
  const int ei = e[i];
  const bool live = ei != EZERO;
  i64 P[2];
  int q[2];
  decompose(live && k < K ? tile[ii][2 * kp] : 0.0, P[0], q[0]);
  decompose(live && k + 1 < K ? tile[ii][2 * kp + 1] : 0.0, P[1], q[1]);
  const bool second = k + 1 < pitch;
  const bool pair = pair_stores_ok(planes, ps, pitch) && second;
  for_each_digit<2>(P, q, live ? ei : 0, nplanes, [&](int r, const int (&d)[2]) {
    store_digit_pair(out + (int64_t)(r - 1) * ps, pair, second, d[0], d[1]);
  });
}

// ---- Sec. 3: X^(1) = fl((tau_j + x) - tau_j) with tau_j = 0.75 * 2^(f_j + beta),
//      i.e. round-half-even of x to the grid 2^(f_j + beta - 53); then its sX column planes.
//      Two consecutive rows per thread.
__device__ __forceinline__ void truncate_to_grid(double x, int gexp, i64& P, int& q) {
  decompose(x, P, q);
  const int sh = gexp - q;
  if (sh > 0 && P != 0) {
    if (sh > 60) {
      P = 0;
    } else {
      P = rne_shift(P, sh);
      q = gexp;
    }
  }
}

__device__ __forceinline__ void truncate_slice_x_body(TruncArgs a, unsigned bx, unsigned by) {
  const double* __restrict__ X = a.X;
  const int64_t ldx = a.ldx, n = a.n, ld1 = a.ld1, pitch = a.pitch, ps = a.ps;
  const int32_t* __restrict__ f = a.f;
  double* __restrict__ X1 = a.X1;
  __nv_bfloat16* __restrict__ planes = a.planes;
  const SliceDyn dyn = a.dyn;
  int nplanes = a.nplanes, beta = a.beta;
  if (dyn.done && *dyn.done) return;
  if (dyn.nplanes) nplanes = *dyn.nplanes;
  if (dyn.beta) beta = *dyn.beta;
  const int64_t k = 2 * ((int64_t)by * 256 + threadIdx.x);
  const int64_t j = bx;
  if (k >= pitch) return;
  __nv_bfloat16* out = planes + j * pitch + k;
  const int fj = f[j];
  const bool live = fj != EZERO;
  const int gexp = fj + beta - 53;
  i64 P[2];
  int q[2];
  truncate_to_grid(live && k < n ? X[k + j * ldx] : 0.0, gexp, P[0], q[0]);
  truncate_to_grid(live && k + 1 < n ? X[k + 1 + j * ldx] : 0.0, gexp, P[1], q[1]);
  if (k < n) X1[k + j * ld1] = exact_double(P[0], q[0]);
  if (k + 1 < n) X1[k + 1 + j * ld1] = exact_double(P[1], q[1]);
  const bool pair = pair_stores_ok(planes, ps, pitch) && k + 1 < pitch;
  const bool second = k + 1 < pitch;
  for_each_digit<2>(P, q, live ? fj : 0, nplanes, [&](int r, const int (&d)[2]) {
    store_digit_pair(out + (int64_t)(r - 1) * ps, pair, second, d[0], d[1]);
  });
}


// ---- single-problem kernels ------------------------------------------------
__global__ void __launch_bounds__(256) k_col_exponents(ColExpArgs a) { col_exponents_body(a, blockIdx.x, 0); }
__global__ void __launch_bounds__(256) k_row_maxbits(RowMaxArgs a) { row_maxbits_body(a, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(256) k_maxbits_to_exponents(MaxToExpArgs a) {
  maxbits_to_exponents_body(a, blockIdx.x, 0);
}
__global__ void __launch_bounds__(256) k_slice_cols(SliceArgs a) { slice_cols_body(a, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(256) k_slice_rows(SliceArgs a) { slice_rows_body(a, blockIdx.x, blockIdx.y); }
__global__ void __launch_bounds__(256) k_truncate_slice_x(TruncArgs a) {
  truncate_slice_x_body(a, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// host launchers (each records its launch instead while a recorder is active)
// ---------------------------------------------------------------------------
int launch_col_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int32_t* e, int* flags,
                         cudaStream_t s, const int* done, int* nnz_max) {
  if (cols == 0) return FRX_OK;
  ColExpArgs a{M, ld, rows, cols, e, flags, done, nnz_max, (unsigned)cols};
  if (record_launch(LK_COL_EXPONENTS, a, cols, 256, 0)) return FRX_OK;
  k_col_exponents<<<(unsigned)cols, 256, 0, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

// scratch must be zero on entry; it is left zero (k_maxbits_to_exponents clears it)
int launch_row_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int32_t* e, u64* scratch,
                         int* flags, cudaStream_t s, const int* done) {
  if (rows == 0) return FRX_OK;
  const unsigned gx = (unsigned)((rows + 255) / 256), gy = (unsigned)((cols + 63) / 64);
  RowMaxArgs a{M, ld, rows, cols, scratch, flags, done, gx};
  MaxToExpArgs b{scratch, rows, e, done, gx};
  if (record_launch(LK_ROW_MAXBITS, a, (long long)gx * gy, 256, 0)) {
    record_launch(LK_MAXBITS_TO_EXPONENTS, b, gx, 256, 0);
    return FRX_OK;
  }
  k_row_maxbits<<<dim3(gx, gy), 256, 0, s>>>(a);
  count_launches(1);
  k_maxbits_to_exponents<<<gx, 256, 0, s>>>(b);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_slice_cols(const double* M, int64_t ld, int64_t K, int64_t N, const int32_t* e, int nplanes,
                      __nv_bfloat16* planes, int64_t ps, int64_t pitch, cudaStream_t s, SliceDyn dyn) {
  if (N == 0 || (nplanes == 0 && !dyn.nplanes)) return FRX_OK;
  const unsigned gx = (unsigned)N, gy = (unsigned)((pitch + 511) / 512);
  SliceArgs a{M, ld, K, N, e, nplanes, planes, ps, pitch, dyn, gx};
  if (record_launch(LK_SLICE_COLS, a, (long long)gx * gy, 256, 0)) return FRX_OK;
  k_slice_cols<<<dim3(gx, gy), 256, 0, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_slice_rows(const double* M, int64_t ld, int64_t rows, int64_t K, const int32_t* e, int nplanes,
                      __nv_bfloat16* planes, int64_t ps, int64_t pitch, cudaStream_t s, SliceDyn dyn) {
  if (rows == 0 || (nplanes == 0 && !dyn.nplanes)) return FRX_OK;
  const unsigned gx = (unsigned)((rows + 7) / 8), gy = (unsigned)((pitch + 63) / 64);
  SliceArgs a{M, ld, K, rows, e, nplanes, planes, ps, pitch, dyn, gx};
  if (record_launch(LK_SLICE_ROWS, a, (long long)gx * gy, 256, 0)) return FRX_OK;
  k_slice_rows<<<dim3(gx, gy), 256, 0, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_truncate_slice_x(const double* X, int64_t ldx, int64_t n, const int32_t* f, int beta, int nplanes,
                            double* X1, int64_t ld1, __nv_bfloat16* planes, int64_t ps, int64_t pitch,
                            cudaStream_t s, SliceDyn dyn) {
  const unsigned gx = (unsigned)n, gy = (unsigned)((pitch + 511) / 512);
  TruncArgs a{X, ldx, n, f, beta, nplanes, X1, ld1, planes, ps, pitch, dyn, gx};
  if (record_launch(LK_TRUNCATE_SLICE_X, a, (long long)gx * gy, 256, 0)) return FRX_OK;
  k_truncate_slice_x<<<dim3(gx, gy), 256, 0, s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

// zero (src == nullptr) or copy 8-byte words, as a recorded launch (batched refinement)
int record_bytes(void* dst, const void* src, size_t bytes) {
  if (bytes % 8 || ((uintptr_t)dst & 7) || ((uintptr_t)src & 7)) return FRX_E_ARG;
  const int64_t words = (int64_t)(bytes / 8);
  const unsigned gx = (unsigned)((words + 255) / 256 < 64 ? (words + 255) / 256 : 64);
  BytesArgs a{(u64*)dst, (const u64*)src, words, gx ? gx : 1};
  return record_launch(src ? LK_COPY : LK_ZERO, a, a.gx, 256, 0) ? FRX_OK : FRX_E_ARG;
}

int launch_grouped_scan(int kind, const void* tab, const long long* start, int count, long long blocks, int threads,
                        size_t smem, cudaStream_t s) {
  if (blocks <= 0) return FRX_OK;
  const unsigned grid = (unsigned)blocks;
  switch (kind) {
    case LK_COL_EXPONENTS:
      k_grouped<ColExpArgs, col_exponents_body, 256, 1><<<grid, 256, 0, s>>>((const ColExpArgs*)tab, start, count);
      break;
    case LK_ROW_MAXBITS:
      k_grouped<RowMaxArgs, row_maxbits_body, 256, 1><<<grid, 256, 0, s>>>((const RowMaxArgs*)tab, start, count);
      break;
    case LK_MAXBITS_TO_EXPONENTS:
      k_grouped<MaxToExpArgs, maxbits_to_exponents_body, 256, 1>
          <<<grid, 256, 0, s>>>((const MaxToExpArgs*)tab, start, count);
      break;
    case LK_SLICE_COLS:
      k_grouped<SliceArgs, slice_cols_body, 256, 1><<<grid, 256, 0, s>>>((const SliceArgs*)tab, start, count);
      break;
    case LK_SLICE_ROWS:
      k_grouped<SliceArgs, slice_rows_body, 256, 1><<<grid, 256, 0, s>>>((const SliceArgs*)tab, start, count);
      break;
    case LK_TRUNCATE_SLICE_X:
      k_grouped<TruncArgs, truncate_slice_x_body, 256, 1><<<grid, 256, 0, s>>>((const TruncArgs*)tab, start, count);
      break;
    case LK_ZERO:
    case LK_COPY:
      k_grouped<BytesArgs, bytes_body, 256, 1><<<grid, 256, 0, s>>>((const BytesArgs*)tab, start, count);
      break;
    default:
      return FRX_E_UNSUPPORTED;
  }
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

}  // namespace frx
