// Launchers of the frx kernels (host-side declarations).
#pragma once

#include <mutex>
#include <vector>

#include "frx_internal.cuh"
#include "plan.cuh"

namespace frx {

enum : int { FLAG_NONFINITE = 1, FLAG_TIMEOUT = 2, FLAG_RANGE = 4, FLAG_CONFIG = 8 };

// One-time setup per CUDA device: kernel attributes and occupancy figures belong to a device,
// so a process that drives several devices sets them on each.  f() runs once per device and
// its status is returned for the current device on every call.
constexpr int FRX_MAX_DEVICES = 64;
struct PerDevice {
  std::once_flag once[FRX_MAX_DEVICES];
  int status[FRX_MAX_DEVICES] = {};
};

template <class F>
int once_per_device(PerDevice& pd, F f) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FRX_E_CUDA;
  if (dev < 0 || dev >= FRX_MAX_DEVICES) return FRX_E_UNSUPPORTED;
  std::call_once(pd.once[dev], [&]() { pd.status[dev] = f(dev); });
  return pd.status[dev];
}

// Output tile configurations of the tensor-core products (the values of frx_set_tile):
// 128 x 128 or 128 x 256 tiles per CTA
enum : int { TILE_AUTO = 0, TILE_128x128 = 1, TILE_128x256 = 2, TILE_LAST = TILE_128x256 };
inline int tile_bn(int cfg) { return cfg == TILE_128x128 ? 128 : 256; }

// optional device-side parameters of the slicing kernels (null: use the launch arguments)
struct SliceDyn {
  const int* nplanes = nullptr;  // planes to produce
  const int* from = nullptr;     // first plane to write (earlier planes are kept)
  const int* beta = nullptr;     // beta of the truncation (k_truncate_slice_x)
  const int* done = nullptr;     // nonzero: the refinement has finished, do nothing
};

// scan_slice.cu
// nnz_max (optional): atomic max of the columns' nonzero counts
int launch_col_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int32_t* e, int* flags,
                         cudaStream_t s, const int* done = nullptr, int* nnz_max = nullptr);
int launch_row_exponents(const double* M, int64_t ld, int64_t rows, int64_t cols, int32_t* e, u64* scratch,
                         int* flags, cudaStream_t s, const int* done = nullptr);
int launch_slice_cols(const double* M, int64_t ld, int64_t K, int64_t N, const int32_t* e, int nplanes,
                      __nv_bfloat16* planes, int64_t ps, int64_t pitch, cudaStream_t s, SliceDyn dyn = SliceDyn());
int launch_slice_rows(const double* M, int64_t ld, int64_t rows, int64_t K, const int32_t* e, int nplanes,
                      __nv_bfloat16* planes, int64_t ps, int64_t pitch, cudaStream_t s, SliceDyn dyn = SliceDyn());
int launch_truncate_slice_x(const double* X, int64_t ldx, int64_t n, const int32_t* f, int beta, int nplanes,
                            double* X1, int64_t ld1, __nv_bfloat16* planes, int64_t ps, int64_t pitch,
                            cudaStream_t s, SliceDyn dyn = SliceDyn());

// Description of one Ozaki product on digit planes:
//   L: planes of an M x K left operand, row-major per plane (row i at L + r*Lps + i*pitch)
//   R: planes of a K x N right operand, column-major per plane (column j at R + s*Rps + j*pitch)
//   d: plane counts kL, kR, pair bound T (r + s <= T), layout of the exact sums (int64 groups
//      of gs anti-diagonals, or one int32 plane per anti-diagonal) and the persistent schedule;
//      out[g * ogs + j * ldo + i].  When `dyn` is set the kernels read d from device memory
//      (written by the device plan) and `done` lets them return when the refinement finished.
struct PlaneGemm {
  const __nv_bfloat16* L;
  int64_t Lps;
  const __nv_bfloat16* R;
  int64_t Rps;
  int64_t pitch;
  int64_t M, N, K;
  GemmDesc d;
  const GemmDesc* dyn;
  const int* done;
  i64* out;
  int64_t ogs, ldo;
  int* flags;   // device status word (timeouts), may be null
  int out_bytes_per_elem;
  int tile;     // output tile configuration of the tensor-core kernel (TILE_AUTO: the autotuner decides)
  __host__ __device__ int32_t* out32() const { return reinterpret_cast<int32_t*>(out); }
};

// host: fill the layout and schedule of g.d; FRX_E_UNSUPPORTED if exactness cannot be guaranteed
int plan_plane_gemm(PlaneGemm& g);
int pairs_in(int kL, int kR, int T);

// sparse_v.cu: V = A X^(1) over the nonzeros of A (ELL pattern of at most ELL_MAX per row)
constexpr int ELL_MAX = 64;
int launch_build_ell(const double* A, int64_t lda, int64_t n, int32_t* ell, cudaStream_t s);
int set_sparse_v_attributes();
int launch_sparse_v(const __nv_bfloat16* Ap, const __nv_bfloat16* Xp, int64_t ps, int64_t pitch, const int32_t* ell,
                    int nzcap, int64_t n, const GemmDesc* dV, const int* done, int* flags, int32_t* out,
                    int64_t ogs, cudaStream_t s);

// gemm_simt.cu / gemm_tc.cu
int launch_plane_gemm(const PlaneGemm& g, cudaStream_t s);
int launch_plane_gemm_simt(const PlaneGemm& g, cudaStream_t s);
int launch_plane_gemm_tc(const PlaneGemm& g, int* flags, int tile, cudaStream_t s);
bool plane_gemm_tc_supported(const PlaneGemm& g);
// grouped slice products: a device table of per-problem entries (tensor maps + arguments,
// 64-byte aligned, tc_problem_bytes() each) run in one persistent launch
size_t tc_problem_bytes();
int tc_problem_fill(const PlaneGemm& g, int* flags, void* host_entry, int tile);
int launch_plane_gemm_grouped(const void* table, int count, int tile, cudaStream_t s);
int prepare_plane_gemm_grouped();
// a device wait that nothing completes (self-test of the bounded waits)
int launch_wait_timeout(int* dflags, cudaStream_t s);
// a zero (src == nullptr) or copy of 8-byte words recorded as a grouped-launch entry
int record_bytes(void* dst, const void* src, size_t bytes);

// autotune.cu: output tile configuration (TILE_*) of the tensor-core products
int tile_policy();
int tune_tile_single(const PlaneGemm& g, int kind, cudaStream_t s, int& tile);
int tune_tile_refine(const PlaneGemm& rep, cudaStream_t s, int& tile);
int tune_tile_grouped(const std::vector<PlaneGemm>& gs, const std::vector<long long>& key, void* table,
                      cudaStream_t s, int& tile);
int& last_tile();

// refine_kernels.cu
int launch_groups_to_dd(const PlaneGemm& g, const int32_t* eL, const int32_t* eR, double* Ch, int64_t ldh,
                        double* Cl, int64_t ldl, cudaStream_t s);

}  // namespace frx
