// V = A X^(1) over the nonzeros of a sparse A (the sparse-matrix setting of Sec. 4).
//
// The dense path forms V's exact anti-diagonal sums S_t = sum_{r + s = t} A^(r) X^(s) on the
// tensor cores over all n columns of A.  When A has few nonzeros per row, the same exact
// integer sums come from the nonzeros alone: S_t(i, j) = sum_{l : a_il != 0} sum_{r + s = t}
// dA_r(i, l) dX_s(l, j), with the same digits (read from the same digit planes).  Integer sums
// do not depend on the order of their terms, so the int32 planes written here are bit for bit
// those of the tensor-core product, and every later step of the iteration reads them
// unchanged.
//
// ELL layout of A's nonzero pattern: ell[i * ELL_MAX + q] is the column of the q-th nonzero of
// row i (ascending), -1 after the last.  A is symmetric, so row i is column i of the
// column-major input, read contiguously.
#include "frx_internal.cuh"
#include "kernels.cuh"
#include "plan.cuh"
#include "profile.cuh"

namespace frx {
namespace {

constexpr int SPV_ROWS = 32;      // rows of a block (threadIdx.x)
constexpr int SPV_COLS = 8;       // columns per pass (threadIdx.y)
constexpr int SPV_COLIT = 8;      // passes: a block covers 32 rows x 64 columns
constexpr int SPV_MAXL = MAX_PLANES;   // planes of A
constexpr int SPV_MAXR = 8;       // planes of X^(1) (at most 7: 56 bits)
constexpr int SPV_MAXT = SPV_MAXL + SPV_MAXR - 1;

// bf16 bits of an integer digit (|d| <= 128) to the integer: adding 1.5 * 2^23 to an integer-valued
// float below 2^22 in magnitude is exact and leaves the integer in the low mantissa bits, so one
// float add and one integer subtract replace the slower float-to-int conversion
__device__ __forceinline__ int bf16_digit(unsigned short b) {
  return __float_as_int(__fadd_rn(__uint_as_float((unsigned)b << 16), 12582912.0f)) - 0x4B400000;
}

// one warp per row i: the columns of its nonzeros, in ascending order
__global__ void __launch_bounds__(256) k_build_ell(const double* __restrict__ A, int64_t lda, int64_t n,
                                                   int32_t* __restrict__ ell) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= n) return;
  const double* col = A + i * lda;
  int32_t* out = ell + i * ELL_MAX;
  int count = 0;
  for (int64_t l0 = 0; l0 < n && count < ELL_MAX; l0 += 32) {
    const int64_t l = l0 + lane;
    const bool nz = l < n && col[l] != 0.0;
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    const int pos = count + __popc(m & ((1u << lane) - 1u));
    if (nz && pos < ELL_MAX) out[pos] = (int32_t)l;
    count += __popc(m);
  }
  for (int q = (count < ELL_MAX ? count : ELL_MAX) + lane; q < ELL_MAX; q += 32) out[q] = -1;
}

struct SparseVArgs {
  const unsigned short* Ap;   // digit planes of A: plane r at Ap + r ps, line i (= row i) at i pitch
  const unsigned short* Xp;   // column planes of X^(1): plane s at Xp + s ps, column j at j pitch
  int64_t ps, pitch, n, ogs;
  const int32_t* ell;
  int nzcap;                  // largest number of nonzeros in a row (<= ELL_MAX): shared-memory slots
  const GemmDesc* dV;         // the plan's V product: kL = k_V, kR = s_X, T, tmax
  const int* done;
  int* flags;
  int32_t* out;               // int32 plane of anti-diagonal t at out + (t - 2) ogs, column-major
};

// The (i, j) sums of one block's rows over its 8 passes of 8 columns.  SX (= s_X) is a template
// argument so the inner loop is fully unrolled without tests; the k_V loop stops at the plan's
// k_V by a warp-uniform break.  Pairs with r + s + 2 > T are not skipped: they only reach S_t with
// t > T >= tmax, which are not stored.
template <int SX>
__device__ __forceinline__ void sparse_v_rows(const SparseVArgs& a, const int* sidx, const short* sa, int nnz,
                                              int kV, int tmax, int64_t i) {
  constexpr int NT = SPV_MAXL + SX - 1;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int jj = 0; jj < SPV_COLIT; ++jj) {
    const int64_t j = ((int64_t)blockIdx.y * SPV_COLIT + jj) * SPV_COLS + ty;
    if (j >= a.n) break;
    int S[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) S[t] = 0;
    const unsigned short* xj = a.Xp + j * a.pitch;
    // the X digits of the next nonzero are loaded while the current one is multiplied
    unsigned short xn[SX];
    if (nnz > 0) {
      const int l0 = sidx[tx];
#pragma unroll
      for (int s = 0; s < SX; ++s) xn[s] = xj[s * a.ps + l0];
    }
    for (int q = 0; q < nnz; ++q) {
      int xs[SX];
#pragma unroll
      for (int s = 0; s < SX; ++s) xs[s] = bf16_digit(xn[s]);
      if (q + 1 < nnz) {
        const int l1 = sidx[(q + 1) * SPV_ROWS + tx];
#pragma unroll
        for (int s = 0; s < SX; ++s) xn[s] = xj[s * a.ps + l1];
      }
#pragma unroll
      for (int r = 0; r < SPV_MAXL; ++r) {
        if (r >= kV) break;
        const int ar = sa[(q * SPV_MAXL + r) * SPV_ROWS + tx];
#pragma unroll
        for (int s = 0; s < SX; ++s) S[r + s] += ar * xs[s];
      }
    }
    int32_t* o = a.out + j * a.n + i;
#pragma unroll
    for (int t = 0; t < NT; ++t)
      if (t + 2 <= tmax) o[t * a.ogs] = S[t];
  }
}

__global__ void __launch_bounds__(SPV_ROWS * SPV_COLS) k_sparse_v(SparseVArgs a) {
  if (a.done && *a.done) return;
  const GemmDesc* D = a.dV;
  if (!D->active) return;
  const int kV = D->kL, sX = D->kR, tmax = D->tmax;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (kV > SPV_MAXL || sX < 1 || sX > SPV_MAXR || tmax > SPV_MAXT + 1) {
    if (tx == 0 && ty == 0 && blockIdx.x == 0 && blockIdx.y == 0) atomicOr(a.flags, FLAG_CONFIG);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  const int nzcap = a.nzcap;
  int* sidx = reinterpret_cast<int*>(smem);                                     // [nzcap][32]
  short* sa = reinterpret_cast<short*>(smem + sizeof(int) * nzcap * SPV_ROWS);  // [nzcap][16][32]
  const int64_t i = (int64_t)blockIdx.x * SPV_ROWS + tx;
  // the block's rows: their nonzero columns and the digits of A there
  for (int q = ty; q < nzcap; q += SPV_COLS) {
    const int l = i < a.n ? a.ell[i * ELL_MAX + q] : -1;
    sidx[q * SPV_ROWS + tx] = l;
    for (int r = 0; r < kV; ++r)
      sa[(q * SPV_MAXL + r) * SPV_ROWS + tx] = l >= 0 ? (short)bf16_digit(a.Ap[r * a.ps + i * a.pitch + l]) : 0;
  }
  __syncthreads();
  if (i >= a.n) return;
  int nnz = 0;
  while (nnz < nzcap && sidx[nnz * SPV_ROWS + tx] >= 0) ++nnz;
  switch (sX) {
    case 1: sparse_v_rows<1>(a, sidx, sa, nnz, kV, tmax, i); break;
    case 2: sparse_v_rows<2>(a, sidx, sa, nnz, kV, tmax, i); break;
    case 3: sparse_v_rows<3>(a, sidx, sa, nnz, kV, tmax, i); break;
    case 4: sparse_v_rows<4>(a, sidx, sa, nnz, kV, tmax, i); break;
    case 5: sparse_v_rows<5>(a, sidx, sa, nnz, kV, tmax, i); break;
    case 6: sparse_v_rows<6>(a, sidx, sa, nnz, kV, tmax, i); break;
    case 7: sparse_v_rows<7>(a, sidx, sa, nnz, kV, tmax, i); break;
    default: sparse_v_rows<8>(a, sidx, sa, nnz, kV, tmax, i); break;
  }
}

size_t sparse_v_smem(int nzcap) {
  return sizeof(int) * (size_t)nzcap * SPV_ROWS + sizeof(short) * (size_t)nzcap * SPV_MAXL * SPV_ROWS;
}

}  // namespace

int launch_build_ell(const double* A, int64_t lda, int64_t n, int32_t* ell, cudaStream_t s) {
  k_build_ell<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(A, lda, n, ell);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

int set_sparse_v_attributes() {
  FRX_CUDA_TRY(
      cudaFuncSetAttribute(k_sparse_v, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sparse_v_smem(ELL_MAX)));
  return FRX_OK;
}

int launch_sparse_v(const __nv_bfloat16* Ap, const __nv_bfloat16* Xp, int64_t ps, int64_t pitch, const int32_t* ell,
                    int nzcap, int64_t n, const GemmDesc* dV, const int* done, int* flags, int32_t* out,
                    int64_t ogs, cudaStream_t s) {
  if (nzcap < 1 || nzcap > ELL_MAX) return FRX_E_ARG;
  SparseVArgs a;
  a.Ap = reinterpret_cast<const unsigned short*>(Ap);
  a.Xp = reinterpret_cast<const unsigned short*>(Xp);
  a.ps = ps;
  a.pitch = pitch;
  a.n = n;
  a.ogs = ogs;
  a.ell = ell;
  a.nzcap = nzcap;
  a.dV = dV;
  a.done = done;
  a.flags = flags;
  a.out = out;
  dim3 grid((unsigned)((n + SPV_ROWS - 1) / SPV_ROWS), (unsigned)((n + SPV_COLS * SPV_COLIT - 1) / (SPV_COLS * SPV_COLIT)));
  k_sparse_v<<<grid, dim3(SPV_ROWS, SPV_COLS), sparse_v_smem(nzcap), s>>>(a);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

}  // namespace frx
