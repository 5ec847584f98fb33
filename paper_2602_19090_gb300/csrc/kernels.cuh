// Launchers of the frx kernels (host-side declarations).
#pragma once

#include "frx_internal.cuh"

namespace frx {

enum : int { FLAG_NONFINITE = 1, FLAG_TIMEOUT = 2, FLAG_RANGE = 4 };

// scan_slice.cu
int launch_col_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int32_t* e, int* flags,
                         cudaStream_t s);
int launch_row_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int32_t* e, u64* scratch,
                         int* flags, cudaStream_t s);
int launch_slice_cols(const double* M, int64_t ld, int64_t K, int64_t N, const int32_t* e, int nplanes,
                      __nv_bfloat16* planes, int64_t ps, int64_t pitch, cudaStream_t s);
int launch_slice_rows(const double* M, int64_t ld, int64_t rows, int64_t K, const int32_t* e, int nplanes,
                      __nv_bfloat16* planes, int64_t ps, int64_t pitch, cudaStream_t s);
int launch_truncate_slice_x(const double* X, int64_t ldx, int64_t n, const int32_t* f, int beta, int nplanes,
                            double* X1, int64_t ld1, __nv_bfloat16* planes, int64_t ps, int64_t pitch,
                            cudaStream_t s);

// Description of one Ozaki product on digit planes:
//   L: kL planes of an M x K left operand, row-major per plane (row i at L + r*Lps + i*pitch)
//   R: kR planes of a K x N right operand, column-major per plane (column j at R + s*Rps + j*pitch)
//   pairs (r, s) with r + s <= T; anti-diagonals t = 2 .. tmax grouped by `gs`;
//   out[g * ogs + j * ldo + i] = sum_{t in group g} 2^(7 (t_last(g) - t)) S_t[i, j]  (exact int64)
struct PlaneGemm {
  const __nv_bfloat16* L;
  int64_t Lps;
  const __nv_bfloat16* R;
  int64_t Rps;
  int64_t pitch;
  int64_t M, N, K;
  int kL, kR, T;
  int tmax, gs, groups;
  i64* out;     // int64 groups (word32 == 0) ...
  int64_t ogs, ldo;
  int* flags;   // device status word (timeouts), may be null
  // int32 per-anti-diagonal planes: plane t - 2 at (int32_t*)out + (t - 2) * ogs (gs = 1).
  // Chosen by plan_plane_gemm when every S_t fits int32 and `out_bytes_per_elem` holds them.
  int word32;
  int out_bytes_per_elem;
  __host__ __device__ int32_t* out32() const { return reinterpret_cast<int32_t*>(out); }
};

// host: fill tmax / gs / groups; returns FRX_E_UNSUPPORTED if exactness cannot be guaranteed
int plan_plane_gemm(PlaneGemm& g);
int pairs_in(int kL, int kR, int T);
inline int group_last_t(const PlaneGemm& g, int grp) {
  int t1 = 2 + (grp + 1) * g.gs - 1;
  return t1 < g.tmax ? t1 : g.tmax;
}

// gemm_simt.cu / gemm_tc.cu
int launch_plane_gemm(const PlaneGemm& g, cudaStream_t s);
int launch_plane_gemm_simt(const PlaneGemm& g, cudaStream_t s);
int launch_plane_gemm_tc(const PlaneGemm& g, int* flags, cudaStream_t s);
bool plane_gemm_tc_supported(const PlaneGemm& g);

// refine_kernels.cu
int launch_groups_to_dd(const PlaneGemm& g, const int32_t* eL, const int32_t* eR, double* Ch, int64_t ldh,
                        double* Cl, int64_t ldl, cudaStream_t s);

}  // namespace frx
