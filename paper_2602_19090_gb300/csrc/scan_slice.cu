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
  int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x;
  int64_t j = blockIdx.y;
  if (k >= pitch) return;
  __nv_bfloat16* out = planes + j * pitch + k;
  int ej = e[j];
  if (k >= K || ej == EZERO) {
    for (int r = from; r < nplanes; ++r) out[r * ps] = digit_bf16(0);
    return;
  }
  i64 P;
  int q;
  decompose(M[k + j * ld], P, q);
  const DigitSource src = digit_source(P, q);
  unsigned par = from > 0 ? digit_q8(src, ej + 1 - DIGIT_BITS * from) & 1u : 0u;
  for (int r = from + 1; r <= nplanes; ++r) {
    const unsigned q8 = digit_q8(src, ej + 1 - DIGIT_BITS * r);
    out[(r - 1) * ps] = digit_bf16(digit_from_q(src, q8, par));
    par = q8 & 1u;
  }
}

// ---- digit planes along rows of a column-major matrix (transpose through smem) ----
// planes[r * ps + i * pitch + k] = digit r of M[i, k] (row exponent e[i]); tile 32 x 32.
__global__ void __launch_bounds__(256) k_slice_rows(const double* __restrict__ M, int64_t ld, int64_t rows,
                                                    int64_t K, const int32_t* __restrict__ e, int nplanes,
                                                    __nv_bfloat16* __restrict__ planes, int64_t ps,
                                                    int64_t pitch, SliceDyn dyn) {
  if (dyn.done && *dyn.done) return;
  if (dyn.nplanes) nplanes = *dyn.nplanes;
  if (nplanes <= 0) return;
  __shared__ double tile[32][33];
  int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  int64_t i0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
  for (int yy = ty; yy < 32; yy += 8) {
    int64_t i = i0 + tx, k = k0 + yy;
    tile[yy][tx] = (i < rows && k < K) ? M[i + k * ld] : 0.0;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    int64_t i = i0 + yy, k = k0 + tx;
    if (i >= rows || k >= pitch) continue;
    __nv_bfloat16* out = planes + i * pitch + k;
    int ei = e[i];
    if (k >= K || ei == EZERO) {
      for (int r = 0; r < nplanes; ++r) out[r * ps] = digit_bf16(0);
      continue;
    }
    i64 P;
    int q;
    decompose(tile[tx][yy], P, q);
    const DigitSource src = digit_source(P, q);
    unsigned par = 0;
    for (int r = 1; r <= nplanes; ++r) {
      const unsigned q8 = digit_q8(src, ei + 1 - DIGIT_BITS * r);
      out[(r - 1) * ps] = digit_bf16(digit_from_q(src, q8, par));
      par = q8 & 1u;
    }
  }
}

// ---- Sec. 3: X^(1) = fl((tau_j + x) - tau_j) with tau_j = 0.75 * 2^(f_j + beta),
//      i.e. round-half-even of x to the grid 2^(f_j + beta - 53); then its sX column planes.
__global__ void __launch_bounds__(256) k_truncate_slice_x(const double* __restrict__ X, int64_t ldx, int64_t n,
                                                          const int32_t* __restrict__ f, int beta, int nplanes,
                                                          double* __restrict__ X1, int64_t ld1,
                                                          __nv_bfloat16* __restrict__ planes, int64_t ps,
                                                          int64_t pitch, SliceDyn dyn) {
  if (dyn.done && *dyn.done) return;
  if (dyn.nplanes) nplanes = *dyn.nplanes;
  if (dyn.beta) beta = *dyn.beta;
  int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x;
  int64_t j = blockIdx.y;
  if (k >= pitch) return;
  __nv_bfloat16* out = planes + j * pitch + k;
  int fj = f[j];
  if (k >= n || fj == EZERO) {
    for (int r = 0; r < nplanes; ++r) out[r * ps] = digit_bf16(0);
    if (k < n) X1[k + j * ld1] = 0.0;
    return;
  }
  i64 P;
  int q;
  decompose(X[k + j * ldx], P, q);
  int gexp = fj + beta - 53;
  int sh = gexp - q;
  if (sh > 0 && P != 0) {
    if (sh > 60) {
      P = 0;
    } else {
      P = rne_shift(P, sh);
      q = gexp;
    }
  }
  X1[k + j * ld1] = exact_double(P, q);
  const DigitSource src = digit_source(P, q);
  unsigned par = 0;
  for (int r = 1; r <= nplanes; ++r) {
    const unsigned q8 = digit_q8(src, fj + 1 - DIGIT_BITS * r);
    out[(r - 1) * ps] = digit_bf16(digit_from_q(src, q8, par));
    par = q8 & 1u;
  }
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
  dim3 g((unsigned)((pitch + 255) / 256), (unsigned)N);
  k_slice_cols<<<g, 256, 0, s>>>(M, ld, K, N, e, nplanes, planes, ps, pitch, dyn);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_slice_rows(const double* M, int64_t ld, int64_t rows, int64_t K, const int32_t* e, int nplanes,
                      __nv_bfloat16* planes, int64_t ps, int64_t pitch, cudaStream_t s, SliceDyn dyn) {
  if (rows == 0 || (nplanes == 0 && !dyn.nplanes)) return FRX_OK;
  dim3 g((unsigned)((pitch + 31) / 32), (unsigned)((rows + 31) / 32));
  k_slice_rows<<<g, 256, 0, s>>>(M, ld, rows, K, e, nplanes, planes, ps, pitch, dyn);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int launch_truncate_slice_x(const double* X, int64_t ldx, int64_t n, const int32_t* f, int beta, int nplanes,
                            double* X1, int64_t ld1, __nv_bfloat16* planes, int64_t ps, int64_t pitch,
                            cudaStream_t s, SliceDyn dyn) {
  dim3 g((unsigned)((pitch + 255) / 256), (unsigned)n);
  k_truncate_slice_x<<<g, 256, 0, s>>>(X, ldx, n, f, beta, nplanes, X1, ld1, planes, ps, pitch, dyn);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

}  // namespace frx
