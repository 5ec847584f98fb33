// Exact digit-plane products on the CUDA cores, grouped by anti-diagonal.
// Sec. 2.3: every slice product A^(r) X^(s) is exact; here the slices are 8-bit
// integer digits (|d| <= 128), so the products are exact integer matrices (int32 per pair:
// |sum| <= K 2^14 < 2^31 for K <= 2^16; int64 per anti-diagonal group).  Used where the
// tensor-core kernel's alignment rules are not met and as the cross-check of the
// tensor-core path.
#include <stdlib.h>

#include "frx_internal.cuh"
#include "grouped.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace frx {

int pairs_in(int kL, int kR, int T) {
  int c = 0;
  for (int r = 1; r <= kL; ++r)
    for (int s = 1; s <= kR; ++s)
      if (r + s <= T) ++c;
  return c;
}

int plan_plane_gemm(PlaneGemm& g) {
  int st = gemm_desc_layout(g.d, g.K, g.out_bytes_per_elem);
  if (st != FRX_OK) return st;
  gemm_desc_schedule(g.d, g.M, g.N, g.d.word32 ? 256 : 128);
  return FRX_OK;
}

namespace {

constexpr int BM = 64, BN = 64, BK = 32;

__device__ __forceinline__ int bf16_digit(unsigned short b) {
  return (int)__uint_as_float((unsigned)b << 16);
}

__global__ void __launch_bounds__(256) k_plane_gemm_simt(PlaneGemm g) {
  if (g.done && *g.done) return;
  const GemmDesc& d = g.dyn ? *g.dyn : g.d;
  if (!d.active) return;
  const int kL = d.kL, kR = d.kR, tmax = d.tmax, gs = d.gs, groups = d.groups, word32 = d.word32;
  __shared__ __align__(16) int As[BK][BM];
  __shared__ __align__(16) int Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
  const int lrow = tid >> 2, lk = (tid & 3) * 8;
  const int64_t Kloop = (g.K + BK - 1) / BK * BK;
  const unsigned short* L = reinterpret_cast<const unsigned short*>(g.L);
  const unsigned short* R = reinterpret_cast<const unsigned short*>(g.R);

  for (int grp = 0; grp < groups; ++grp) {
    const int t0 = 2 + grp * gs;
    const int t1 = t0 + gs - 1 < tmax ? t0 + gs - 1 : tmax;
    i64 racc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) racc[a][b] = 0;
    for (int t = t0; t <= t1; ++t) {
      i64 tacc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) tacc[a][b] = 0;
      const int rlo = t - kR > 1 ? t - kR : 1;
      const int rhi = kL < t - 1 ? kL : t - 1;
      for (int r = rlo; r <= rhi; ++r) {
        const unsigned short* Lp = L + (int64_t)(r - 1) * g.Lps;
        const unsigned short* Rp = R + (int64_t)(t - r - 1) * g.Rps;
        int acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0;
        for (int64_t k0 = 0; k0 < Kloop; k0 += BK) {
          uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
          if (i0 + lrow < g.M && k0 + lk < g.pitch)
            va = *reinterpret_cast<const uint4*>(Lp + (i0 + lrow) * g.pitch + k0 + lk);
          if (j0 + lrow < g.N && k0 + lk < g.pitch)
            vb = *reinterpret_cast<const uint4*>(Rp + (j0 + lrow) * g.pitch + k0 + lk);
          unsigned short ha[8], hb[8];
          memcpy(ha, &va, 16);
          memcpy(hb, &vb, 16);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            As[lk + q][lrow] = bf16_digit(ha[q]);
            Bs[lk + q][lrow] = bf16_digit(hb[q]);
          }
          __syncthreads();
#pragma unroll 8
          for (int kk = 0; kk < BK; ++kk) {
            const int4 av = *reinterpret_cast<const int4*>(&As[kk][ty * 4]);
            const int4 bv = *reinterpret_cast<const int4*>(&Bs[kk][tx * 4]);
            const int ar[4] = {av.x, av.y, av.z, av.w};
            const int br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) acc[a][b] += ar[a] * br[b];
          }
          __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) tacc[a][b] += acc[a][b];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) racc[a][b] = racc[a][b] * (1 << DIGIT_BITS) + tacc[a][b];
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int64_t j = j0 + tx * 4 + b;
      if (j >= g.N) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        int64_t i = i0 + ty * 4 + a;
        if (i >= g.M) continue;
        if (word32)
          g.out32()[grp * g.ogs + j * g.ldo + i] = (int32_t)racc[a][b];
        else
          g.out[grp * g.ogs + j * g.ldo + i] = racc[a][b];
      }
    }
  }
}

}  // namespace

int launch_plane_gemm_simt(const PlaneGemm& g, cudaStream_t s) {
  if ((!g.dyn && g.d.groups == 0) || g.M == 0 || g.N == 0) return FRX_OK;
  if (g.pitch % 8) return FRX_E_ARG;
  dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM));
  k_plane_gemm_simt<<<grid, 256, 0, s>>>(g);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

// Tensor-core kernel when the operands allow it; FRX_GEMM=simt selects the CUDA-core
// kernel (used to cross-check the two implementations bit for bit).
int launch_plane_gemm(const PlaneGemm& g, cudaStream_t s) {
  if ((!g.dyn && g.d.groups == 0) || g.M == 0 || g.N == 0) return FRX_OK;
  if (active_recorder()) {
    // batched refinement: the product becomes one entry of a grouped tensor-core launch
    std::vector<unsigned char> entry(tc_problem_bytes());
    const int tile = active_recorder()->tile;
    FRX_TRY(tc_problem_fill(g, g.flags, entry.data(), tile));
    LaunchRecord r;
    r.kind = LK_GEMM;
    r.args = std::move(entry);
    r.blocks = 0;
    r.threads = 0;
    r.smem = 0;
    r.variant = tile;
    active_recorder()->recs.push_back(std::move(r));
    return FRX_OK;
  }
  const char* env = getenv("FRX_GEMM");
  bool simt = env && env[0] == 's';
  if (!simt && plane_gemm_tc_supported(g)) {
    int tile = g.tile;
    if (tile == TILE_AUTO) FRX_TRY(tune_tile_single(g, 1, s, tile));
    GemmTimer timer(g, s);
    return launch_plane_gemm_tc(g, g.flags, tile, s);
  }
  GemmTimer timer(g, s);
  count_simt_launch();
  return launch_plane_gemm_simt(g, s);
}

}  // namespace frx
