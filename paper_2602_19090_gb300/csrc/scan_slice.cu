// Exponent scans and fixed-grid digit slicing (Sec. 2.3, eq. sigma/tau, eq. a/x;
// eq. tau with s = 1 for the truncation X^(1) of Sec. 3).
#include "frx_internal.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace frx {

// ---- S1: exponent of every column (one block per column) ------------------
__global__ void __launch_bounds__(256) k_col_exponents(const double* __restrict__ M, int64_t ld,
                                                       int64_t rows, int64_t cols, int32_t* __restrict__ e,
                                                       int* __restrict__ flags, const int* done) {
  if (done && *done) return;
  int64_t j = blockIdx.x;
  const double* col = M + j * ld;
  u64 mx = 0;
  bool bad = false;
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
    u64 ab = double_to_bits(col[i]) & 0x7fffffffffffffffull;
    bad |= nonfinite_absbits(ab);
    mx = ab > mx ? ab : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    u64 other = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = other > mx ? other : mx;
  }
  __shared__ u64 red[8];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  if (bad) atomicOr(&sbad, 1);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = red[w] > mx ? red[w] : mx;
    mx = red[0] > mx ? red[0] : mx;
    e[j] = sbad ? EZERO : (mx == 0 ? EZERO : ceil_log2_absbits(mx));
    if (sbad) atomicOr(flags, FLAG_NONFINITE);
  }
}

// ---- S1: exponent of every row of a column-major matrix --------------------
// grid (ceil(rows / 256), ceil(cols / 64)); rowmax must be zeroed first.
__global__ void __launch_bounds__(256) k_row_maxbits(const double* __restrict__ M, int64_t ld,
                                                     int64_t rows, int64_t cols, u64* __restrict__ rowmax,
                                                     int* __restrict__ flags, const int* done) {
  if (done && *done) return;
  int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= rows) return;
  int64_t j0 = (int64_t)blockIdx.y * 64;
  int64_t j1 = j0 + 64 < cols ? j0 + 64 : cols;
  u64 mx = 0;
  bool bad = false;
  for (int64_t j = j0; j < j1; ++j) {
    u64 ab = double_to_bits(M[i + j * ld]) & 0x7fffffffffffffffull;
    bad |= nonfinite_absbits(ab);
    mx = ab > mx ? ab : mx;
  }
  if (bad) atomicOr(flags, FLAG_NONFINITE);
  if (mx) atomicMax(rowmax + i, mx);
}

__global__ void k_maxbits_to_exponents(u64* __restrict__ mx, int64_t n, int32_t* __restrict__ e, const int* done) {
  if (done && *done) return;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    e[i] = mx[i] == 0 ? EZERO : ceil_log2_absbits(mx[i]);
    mx[i] = 0;  // ready for the next scan
  }
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
__global__ void __launch_bounds__(256) k_slice_cols(const double* __restrict__ M, int64_t ld, int64_t K,
                                                    int64_t N, const int32_t* __restrict__ e, int nplanes,
                                                    __nv_bfloat16* __restrict__ planes, int64_t ps,
                                                    int64_t pitch, SliceDyn dyn) {
  if (dyn.done && *dyn.done) return;
  if (dyn.nplanes) nplanes = *dyn.nplanes;
  const int from = dyn.from ? *dyn.from : 0;
  if (from >= nplanes) return;
  const int64_t k = 2 * ((int64_t)blockIdx.y * 256 + threadIdx.x);
  const int64_t j = blockIdx.x;   // columns on x: N may exceed 65535
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
__global__ void __launch_bounds__(256) k_slice_rows(const double* __restrict__ M, int64_t ld, int64_t rows,
                                                    int64_t K, const int32_t* __restrict__ e, int nplanes,
                                                    __nv_bfloat16* __restrict__ planes, int64_t ps,
                                                    int64_t pitch, SliceDyn dyn) {
  if (dyn.done && *dyn.done) return;
  if (dyn.nplanes) nplanes = *dyn.nplanes;
  if (nplanes <= 0) return;
  __shared__ double tile[8][65];
  const int64_t i0 = (int64_t)blockIdx.x * 8, k0 = (int64_t)blockIdx.y * 64;   // rows may reach 2^20
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

__global__ void __launch_bounds__(256) k_truncate_slice_x(const double* __restrict__ X, int64_t ldx, int64_t n,
                                                          const int32_t* __restrict__ f, int beta, int nplanes,
                                                          double* __restrict__ X1, int64_t ld1,
                                                          __nv_bfloat16* __restrict__ planes, int64_t ps,
                                                          int64_t pitch, SliceDyn dyn) {
  if (dyn.done && *dyn.done) return;
  if (dyn.nplanes) nplanes = *dyn.nplanes;
  if (dyn.beta) beta = *dyn.beta;
  const int64_t k = 2 * ((int64_t)blockIdx.y * 256 + threadIdx.x);
  const int64_t j = blockIdx.x;
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

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int launch_col_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int32_t* e, int* flags,
                         cudaStream_t s, const int* done) {
  if (cols == 0) return FRX_OK;
  k_col_exponents<<<(unsigned)cols, 256, 0, s>>>(M, ld, rows, cols, e, flags, done);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

// scratch must be zero on entry; it is left zero (k_maxbits_to_exponents clears it)
int launch_row_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int32_t* e, u64* scratch,
                         int* flags, cudaStream_t s, const int* done) {
  if (rows == 0) return FRX_OK;
  dim3 g((unsigned)((rows + 255) / 256), (unsigned)((cols + 63) / 64));
  k_row_maxbits<<<g, 256, 0, s>>>(M, ld, rows, cols, scratch, flags, done);
  count_launches(1);
  k_maxbits_to_exponents<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(scratch, rows, e, done);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_slice_cols(const double* M, int64_t ld, int64_t K, int64_t N, const int32_t* e, int nplanes,
                      __nv_bfloat16* planes, int64_t ps, int64_t pitch, cudaStream_t s, SliceDyn dyn) {
  if (N == 0 || (nplanes == 0 && !dyn.nplanes)) return FRX_OK;
  dim3 g((unsigned)N, (unsigned)((pitch + 511) / 512));
  k_slice_cols<<<g, 256, 0, s>>>(M, ld, K, N, e, nplanes, planes, ps, pitch, dyn);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_slice_rows(const double* M, int64_t ld, int64_t rows, int64_t K, const int32_t* e, int nplanes,
                      __nv_bfloat16* planes, int64_t ps, int64_t pitch, cudaStream_t s, SliceDyn dyn) {
  if (rows == 0 || (nplanes == 0 && !dyn.nplanes)) return FRX_OK;
  dim3 g((unsigned)((rows + 7) / 8), (unsigned)((pitch + 63) / 64));
  k_slice_rows<<<g, 256, 0, s>>>(M, ld, rows, K, e, nplanes, planes, ps, pitch, dyn);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_truncate_slice_x(const double* X, int64_t ldx, int64_t n, const int32_t* f, int beta, int nplanes,
                            double* X1, int64_t ld1, __nv_bfloat16* planes, int64_t ps, int64_t pitch,
                            cudaStream_t s, SliceDyn dyn) {
  dim3 g((unsigned)n, (unsigned)((pitch + 511) / 512));
  k_truncate_slice_x<<<g, 256, 0, s>>>(X, ldx, n, f, beta, nplanes, X1, ld1, planes, ps, pitch, dyn);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

}  // namespace frx
