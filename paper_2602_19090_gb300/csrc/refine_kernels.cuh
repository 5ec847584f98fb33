// Argument blocks of the per-iteration kernels.
#pragma once

#include "kernels.cuh"

namespace frx {

struct GroupArgs {  // exact anti-diagonal sums of one Ozaki product (int64 groups or int32 planes)
  const void* out;
  int64_t ogs, ldo;
  int groups, gs, tmax;
  int word32;
  int exact128;            // all groups combine exactly in 128 bits
  const GemmDesc* dyn;     // when set, the fields above are read from it at kernel entry
};

struct ResidualArgs {
  int64_t n;
  GroupArgs V;           // V = A X^(1): left exponents eA (rows of A), right f (columns of X)
  const int32_t* eA;
  const int32_t* f;
  const double* X1;
  int64_t ld1;
  double* lam;           // out: lambda_j (Alg. 1)
  double* r;             // out: r_j (Alg. 1)
  double* Res;           // out: V - X1 diag(lambda) rounded to FP64
  int64_t ldr;
  int32_t* h;            // out: column exponents of Res
  int beta;              // X1 lies on the grid 2^(f_j + beta - 53)
  const int* beta_dyn;   // device beta (overrides beta)
  const int* done;
  double* Vh;            // optional debug copies (ld = n)
  double* Vl;
  unsigned gx;           // blocks of the single launch (one per column)
};

struct CorrectionArgs {
  int64_t n;
  GroupArgs W;           // W = X1^T Res: left exponents f, right h
  const int32_t* f;
  const int32_t* h;
  const double* lam;
  const double* r;
  const double* X1;
  int64_t ld1;
  double omega;          // cluster threshold
  const double* omega_dyn;
  const int* done;
  double* E;             // out: E~
  int64_t lde;
  int32_t* eta;          // out: column exponents of E~
  double* norms;         // per-column squared norms [3][n]: E~(:, j), W_offdiag(:, j) (this kernel writes [0], [1])
  int* ccount;           // out: cluster pairs found
  int* flags;
  double* Wout;          // optional debug copy (ld = n)
  unsigned gx;
};

struct UpdateArgs {
  int64_t n;
  GroupArgs U;           // U = X1 E~: left exponents rho (rows of X1), right eta
  const int32_t* rho;
  const int32_t* eta;
  const int32_t* f;      // X1 lies on the grid 2^(f_j + beta - 53)
  int beta;
  const int* beta_dyn;
  const int* done;
  const double* X1;
  int64_t ld1;
  double* X;             // in: X_old, out: X_new
  int64_t ldx;
  double* norms;         // per-column squared norms [3][n]: this kernel writes [2] (X_new - X_old)(:, j)
  unsigned gx;
};

GroupArgs group_args(const PlaneGemm& g);
int set_refine_kernel_attributes();
// dynamic shared memory of a residual launch over columns of order at most n with blocks of
// `threads` (the V column, then the first pass's copy stages), and its ceiling: 220 KB, which
// leaves room for the kernel's static shared memory within the 227 KB a block may hold
size_t residual_launch_smem(int64_t n, int threads);
constexpr size_t RESIDUAL_SMEM_MAX = 220 * 1024;
int launch_residual(const ResidualArgs& a, cudaStream_t s);
int launch_w_offdiag_norm2(const CorrectionArgs& a, cudaStream_t s);
int launch_correction(const CorrectionArgs& a, cudaStream_t s);
int launch_update(const UpdateArgs& a, cudaStream_t s);

}  // namespace frx
