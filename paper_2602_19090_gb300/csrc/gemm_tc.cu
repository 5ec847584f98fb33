// Exact digit-plane products on the 5th-generation tensor cores (sm_103a).
//
// Sec. 2.3 multiplies error-free slices so that every slice product is exact.  The
// slices here are integer digits in [-128, 128] stored as bfloat16 (exact: its 8-bit
// significand holds every integer up to 256), multiplied by tcgen05.mma (.kind::f16,
// bf16 x bf16 -> f32 in TMEM).  Every product is an integer of magnitude <= 2^14, so an
// FP32 accumulator holds exact integers as long as the accumulated count stays <= 2^10
// terms per lane (|sum| <= 2^24); the accumulator is therefore drained into integer
// registers every CHUNK_KB k-blocks (and at the end of every anti-diagonal t).  With int32
// planes each anti-diagonal's exact sum S_t is stored as one plane (while
// pairs * K * 2^14 < 2^31).  Beyond that the sums are int64 Horner groups
// R_g = sum_{t in g} 2^(8 (t_last - t)) S_t, formed by split-K: the inner dimension is cut into
// chunks short enough for every chunk's S_t to be exact in int32 registers, and each unit adds
// its chunk's 2^(8 (t_last - t)) S_t to the zeroed group word with a 64-bit atomic (integer
// addition: exact and independent of the order the chunks land in).  A BN = 128 kernel that
// accumulates the Horner groups in int64 registers remains for FRX_SPLITK=0.
//
// Tile configurations (int32 planes): 128 x 128 or 128 x 256 output tiles per CTA.  The
// configuration changes no result; the autotuner picks it.  Every CTA loads its own operand
// tiles from this GPU's memory (no cluster launch).
//
// Persistent: one CTA per SM walks the units (output tile, anti-diagonal group)
// in rounds (serpentine when there are few), groups ordered by decreasing work and tiles in
// bands of TILE_BAND tile rows.  A grouped variant walks the units of many problems (the
// batched refinement).
// Warp roles:
//   warp 0       TMA producer (3-D tensor maps over the plane stacks, 128B swizzle)
//   warp 1       TMEM allocator and single-thread MMA issuer
//   warps 2..9   epilogue: tcgen05.ld of the FP32 accumulator, exact integer sums
// Pipeline: 4-6 smem stages (A 16 KB + B BN * 128 bytes), two TMEM accumulators of BN
// columns each.  Every mbarrier wait is bounded by the global timer; on expiry the
// CTA raises FLAG_TIMEOUT, drains what it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "frx_internal.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace frx {
namespace {

constexpr int BM = 128, BK = 64;   // BK bf16 = 128 bytes = one swizzle row
constexpr int MAX_STAGES = 6;
constexpr int CHUNK_KB = (1 << (24 - PRODUCT_BITS)) / BK;   // 16 * 64 = 1024 products: |sum| <= 2^24
static_assert(CHUNK_KB >= 1, "a k-block of products must stay exact in FP32");
constexpr int NUM_EPI_WARPS = 8;
constexpr int NUM_THREADS = 32 * (2 + NUM_EPI_WARPS);
constexpr uint32_t STAGE_A_BYTES = BM * BK * 2;
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // 2 s

struct Smem {
  // tiles first (1024-byte aligned by the dynamic smem base adjustment)
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: false on timeout or when another role has aborted
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* flags) {
  uint32_t addr = smem_u32(bar);
  if (mbar_try(addr, parity)) return true;
  unsigned long long t0 = gtimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(addr, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort) return false;
      if (gtimer() - t0 > WAIT_LIMIT_NS) {
        *abort = 1;
        if (flags) atomicOr(flags, FLAG_TIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// K-major operand, 128-byte swizzle: 8-row groups 1024 bytes apart (SBO), version 1
__device__ __forceinline__ uint64_t smem_desc(const void* tile) {
  uint64_t addr = smem_u32(tile);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3fff;
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

// kind::f16, A = B = bf16, D = f32, both K-major, M = 128, N = bn
__host__ __device__ constexpr uint32_t idesc_for(int bn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
  int64_t M, N;
  int nkb;       // k-blocks of 64
  int nsplit;    // split-K chunks (1: none); each unit covers k-blocks [c kcb, (c + 1) kcb)
  int kcb;
  void* out;     // int64 groups, or int32 per-t planes when W32
  int64_t ogs, ldo;
  int* flags;
  // product description (d, or *dyn when set): plane counts, groups and the persistent
  // schedule: unit u = (group gorder[u / tiles], tile u % tiles), tiles = ntm * ntn, groups
  // ordered by decreasing work so a static round-robin over CTAs stays balanced
  GemmDesc d;
  const GemmDesc* dyn;
  const int* done;
  int bn;        // tile width the right operand's tensor map was encoded for
};

// one problem of a grouped launch: its tensor maps and arguments (device table entry)
struct TcProblem {
  CUtensorMap mapL;
  CUtensorMap mapR;
  TcArgs a;
};

// per-launch scalars read once at kernel entry
struct TcRun {
  int64_t M, N;
  int nkb, kL, kR, tmax, gs, groups, ntm, ntn, units, nsplit, kcb;
  void* out;
  int64_t ogs, ldo;
  int* flags;
};

__device__ __forceinline__ int pair_lo(int t, int kR) { return t - kR > 1 ? t - kR : 1; }
__device__ __forceinline__ int pair_hi(int t, int kL) { return kL < t - 1 ? kL : t - 1; }

// BN_ = 128: int64 Horner groups of gs anti-diagonals, 64 columns per epilogue thread.
// BN_ = 256 (W32): one exact int32 plane per anti-diagonal t (gs = 1), 128 columns per thread.
// Tile t of a group in banded raster order: bands of TILE_BAND tile rows, each walked
// column by column, so the units in flight at one time (consecutive t) share A panels
// across a band's width and B panels across its TILE_BAND rows, instead of sweeping whole
// tile rows (where every B panel is re-read once per few rows).
#ifndef FRX_TILE_BAND
#define FRX_TILE_BAND 16
#endif
constexpr int TILE_BAND = FRX_TILE_BAND;

__device__ __forceinline__ void tile_origin(int t, int ntm, int ntn, int bm, int bn, int& i0, int& j0) {
  const int band = t / (TILE_BAND * ntn);
  const int rows = min(TILE_BAND, ntm - band * TILE_BAND);
  const int local = t - band * TILE_BAND * ntn;
  i0 = (band * TILE_BAND + local % rows) * bm;
  j0 = (local / rows) * bn;
}

// The unit this CTA takes in round r of the persistent loop.  With few rounds, rounds
// alternate direction (serpentine): units come in decreasing order of work, so a CTA that took
// one of the longest units of a round takes one of the shortest of the next, which evens out
// the CTAs' totals where plain round-robin would give the first CTAs the longest unit of every
// round.  With many rounds the imbalance is confined to the short units of the tail, and plain
// round-robin keeps the units in flight a contiguous window (better L2 reuse of the panels).
constexpr int SERPENTINE_MAX_ROUNDS = 16;

__device__ __forceinline__ int unit_of_round(int r, bool serp) {
  const int P = (int)gridDim.x, c = (int)blockIdx.x;
  return (serp && (r & 1)) ? (r + 1) * P - 1 - c : r * P + c;
}

// the product description of a launch's problem, resolved from its arguments; the tiling
// (128 x BN tiles, units = tiles x groups x split-K chunks) belongs to the kernel variant, not
// to the plan.  W32: int32 accumulation in registers; SPLIT: int64 Horner groups accumulated
// by atomics over K-chunks (W32 without SPLIT writes one int32 plane per anti-diagonal).
template <int BN, bool W32, bool SPLIT>
__device__ __forceinline__ bool tc_run_of(const TcArgs& a0, TcRun& a, const int*& gorder) {
  if (a0.done && *a0.done) return false;
  const GemmDesc* D = a0.dyn ? a0.dyn : &a0.d;
  if (!D->active || D->groups <= 0) return false;
  if (a0.bn != BN || D->word32 != ((W32 && !SPLIT) ? 1 : 0) ||
      (SPLIT && (a0.nsplit < 1 || a0.kcb < 1 || (long long)a0.nsplit * a0.kcb < a0.nkb))) {
    // the tensor map's box or the exact-sum layout does not fit this variant: no product
    if (a0.flags) atomicOr(a0.flags, FLAG_CONFIG);
    return false;
  }
  a.M = a0.M;
  a.N = a0.N;
  a.nkb = a0.nkb;
  a.kL = D->kL;
  a.kR = D->kR;
  a.tmax = D->tmax;
  a.gs = D->gs;
  a.groups = D->groups;
  a.ntm = (int)((a0.M + BM - 1) / BM);
  a.ntn = (int)((a0.N + BN - 1) / BN);
  a.nsplit = SPLIT ? a0.nsplit : 1;
  a.kcb = SPLIT ? a0.kcb : a0.nkb;
  a.units = a.ntm * a.ntn * D->groups * a.nsplit;
  a.out = a0.out;
  a.ogs = a0.ogs;
  a.ldo = a0.ldo;
  a.flags = a0.flags;
  gorder = D->gorder;
  return true;
}

// Unit sources of the kernel body.  A unit is (output tile, anti-diagonal group) of one
// problem; unit(u, lu) makes `run`, `gorder` and the tensor maps describe the problem that
// global unit u belongs to and sets lu to its index within that problem.
struct SingleSrc {
  TcRun run;
  const int* gorder;
  const CUtensorMap* mapL;
  const CUtensorMap* mapR;
  int* flags0;
  int rnd, P;
  bool serp;
  __device__ void begin() {
    P = (int)gridDim.x;
    serp = run.units <= SERPENTINE_MAX_ROUNDS * P;
    rnd = 0;
  }
  __device__ void prefetch_next() {}
  // the next unit of this CTA in round order
  __device__ bool next(int& lu) {
    while ((long long)rnd * P < run.units) {
      const int u = unit_of_round(rnd++, serp);
      if (u < run.units) {
        lu = u;
        return true;
      }
    }
    return false;
  }
};


constexpr int MAX_GROUPED = 2048;   // problems of one grouped launch

// Units of a grouped launch: problem-major (problems listed largest first), then groups by
// decreasing work, then tiles, dealt round-robin over the CTAs.  (Giving each CTA a contiguous
// run of units with an equal share of the slice-pair work was measured slower on a batch of
// 256 matrices of n in [32, 512]: 37.9 against 26.5 ms, since the small problems' many short
// units carry a fixed epilogue cost that the work measure leaves out.)
// The per-unit fields of one problem of a grouped launch, kept in shared memory so that a CTA
// moving to another problem's unit (most units, for small problems) reads them there instead
// of following the problem's argument and plan pointers through global memory.
struct RunRec {
  int M, N;
  void* out;
  int64_t ogs, ldo;
  int* flags;
  const int* gorder;
  int nkb, kL, kR, tmax, gs, groups, ntm, ntn, units;
};
constexpr int RUN_CACHE = 256;   // problems whose records fit beside the stages

__device__ __forceinline__ void rec_of(const TcRun& r, const int* g, RunRec& c) {
  c.M = (int)r.M;
  c.N = (int)r.N;
  c.out = r.out;
  c.ogs = r.ogs;
  c.ldo = r.ldo;
  c.flags = r.flags;
  c.gorder = g;
  c.nkb = r.nkb;
  c.kL = r.kL;
  c.kR = r.kR;
  c.tmax = r.tmax;
  c.gs = r.gs;
  c.groups = r.groups;
  c.ntm = r.ntm;
  c.ntn = r.ntn;
  c.units = r.units;
}

__device__ __forceinline__ void run_of_rec(const RunRec& c, TcRun& r, const int*& g) {
  r.M = c.M;
  r.N = c.N;
  r.nkb = c.nkb;
  r.kL = c.kL;
  r.kR = c.kR;
  r.tmax = c.tmax;
  r.gs = c.gs;
  r.groups = c.groups;
  r.ntm = c.ntm;
  r.ntn = c.ntn;
  r.units = c.units;
  r.nsplit = 1;
  r.kcb = c.nkb;
  r.out = c.out;
  r.ogs = c.ogs;
  r.ldo = c.ldo;
  r.flags = c.flags;
  g = c.gorder;
}

template <int BN, bool W32>
struct GroupedSrc {
  const TcProblem* probs;
  const int* prefix;   // shared: units of problems 0..m-1
  const RunRec* recs;  // shared records of every problem, or nullptr (more than RUN_CACHE)
  int count;
  int cur;             // problem `run` currently describes
  TcRun run;
  const int* gorder;
  const CUtensorMap* mapL;
  const CUtensorMap* mapR;
  int* flags0;
  int rnd;
  __device__ void begin() { rnd = 0; }
  // problem of global unit u (last m with prefix[m] <= u)
  __device__ int problem_of(int u) const {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= u) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
  // the producer asks for the tensor maps of this CTA's next unit ahead of its loads
  __device__ void prefetch_next() {
    const int u = (int)blockIdx.x + rnd * (int)gridDim.x;
    if (u >= prefix[count]) return;
    const int m = problem_of(u);
    if (m == cur) return;
    asm volatile("prefetch.tensormap [%0];" ::"l"(&probs[m].mapL) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&probs[m].mapR) : "memory");
  }
  __device__ bool next(int& lu) {
    const int u = (int)blockIdx.x + rnd++ * (int)gridDim.x;
    if (u >= prefix[count]) return false;
    const int lo = problem_of(u);
    if (lo != cur) {
      cur = lo;
      if (recs) run_of_rec(recs[lo], run, gorder);
      else tc_run_of<BN, W32, false>(probs[lo].a, run, gorder);
      mapL = &probs[lo].mapL;
      mapR = &probs[lo].mapR;
    }
    lu = u - prefix[lo];
    return true;
  }
};

// BN_ = 128: int64 Horner groups of gs anti-diagonals, 64 columns per epilogue thread.
// BN_ = 256 (W32): one exact int32 plane per anti-diagonal t (gs = 1), 128 columns per thread;
// with SPLIT the unit's K-chunk sum of each t is added to its int64 Horner group by atomics.
// A unit's slot q = lu / tiles names its group gorder[q / nsplit] and K-chunk q % nsplit.
template <int BN_, bool W32, bool SPLIT, class Src>
__device__ __forceinline__ void tc_body(Src& src) {
  constexpr int BN = BN_;
  constexpr int STAGES = BN == 256 ? 4 : 6;
  constexpr uint32_t STAGE_B_BYTES = BN * BK * 2;
  constexpr uint32_t STAGE_BYTES = STAGE_A_BYTES + STAGE_B_BYTES;
  constexpr uint32_t TMEM_COLS = 2 * BN;
  constexpr uint32_t IDESC = idesc_for(BN);
  constexpr int NCOL = BN / 2;   // columns per epilogue thread
  typedef typename std::conditional<W32, int, i64>::type Acc;
  extern __shared__ __align__(1024) unsigned char dsmem[];
  unsigned char* base = (unsigned char*)(((uintptr_t)dsmem + 1023) & ~(uintptr_t)1023);
  unsigned char* tiles_smem = base;
  Smem* sm = reinterpret_cast<Smem*>(base + STAGES * STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&sm->full[s], 1);
      mbar_init(&sm->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm->acc_full[b], 1);
      mbar_init(&sm->acc_empty[b], NUM_EPI_WARPS);
    }
    mbar_init(&sm->drain, 1);
    sm->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm->tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm->tmem_base;
  volatile int* abort = &sm->abort;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      long long issued = 0;
      bool ok = !*abort;
      src.begin();
      int lu;
      while (ok && src.next(lu)) {
        src.prefetch_next();
        const TcRun& a = src.run;
        const int* gorder = src.gorder;
        const int tiles = a.ntm * a.ntn;
        const int q = lu / tiles, tile = lu % tiles;
        const int grp = gorder[q / a.nsplit], kb0 = (q % a.nsplit) * a.kcb, kb1 = min(a.nkb, kb0 + a.kcb);
        int i0, j0;
        tile_origin(tile, a.ntm, a.ntn, BM, BN, i0, j0);
        int t0 = 2 + grp * a.gs, t1 = min(t0 + a.gs - 1, a.tmax);
        for (int t = t0; t <= t1 && ok; ++t) {
          for (int r = pair_lo(t, a.kR); r <= pair_hi(t, a.kL) && ok; ++r) {
            int s = t - r;
            for (int kb = kb0; kb < kb1; ++kb) {
              if (!mbar_wait(&sm->empty[stage], phase ^ 1, abort, a.flags)) {
                ok = false;
                break;
              }
              unsigned char* st = tiles_smem + stage * STAGE_BYTES;
              mbar_expect_tx(&sm->full[stage], STAGE_BYTES);
              tma_load_3d(st, src.mapL, kb * BK, i0, r - 1, &sm->full[stage]);
              tma_load_3d(st + STAGE_A_BYTES, src.mapR, kb * BK, j0, s - 1, &sm->full[stage]);
              ++issued;
              if (++stage == STAGES) {
                stage = 0;
                phase ^= 1;
              }
            }
          }
        }
      }
      if (ok) {
        // the MMA has released every stage this CTA's copies filled: no arrival can target
        // this CTA's barriers after it exits
        for (int q = 0; q < STAGES; ++q) {
          if (!mbar_wait(&sm->empty[stage], phase ^ 1, abort, src.flags0)) break;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      } else {
        // let the copies this thread issued land before the CTA exits (bounded)
        unsigned long long t0 = gtimer();
        long long back = issued < STAGES ? issued : STAGES;
        int st2 = stage;
        uint32_t ph2 = phase;
        for (long long q = 0; q < back; ++q) {
          if (--st2 < 0) {
            st2 = STAGES - 1;
            ph2 ^= 1;
          }
          while (!mbar_try(smem_u32(&sm->full[st2]), ph2) && gtimer() - t0 < 10000000ull) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int buf = 0;
      uint32_t acc_phase[2] = {0, 0};
      bool ok = true;
      bool any = false;
      src.begin();
      int lu;
      while (ok && src.next(lu)) {
        const TcRun& a = src.run;
        const int* gorder = src.gorder;
        const int tiles = a.ntm * a.ntn;
        const int q = lu / tiles;
        const int grp = gorder[q / a.nsplit], kb0 = (q % a.nsplit) * a.kcb, kb1 = min(a.nkb, kb0 + a.kcb);
        int t0 = 2 + grp * a.gs, t1 = min(t0 + a.gs - 1, a.tmax);
        for (int t = t0; t <= t1 && ok; ++t) {
          int rlo = pair_lo(t, a.kR), rhi = pair_hi(t, a.kL);
          int total = (rhi - rlo + 1) * (kb1 - kb0);
          int cnt = 0, done = 0;
          for (int r = rlo; r <= rhi && ok; ++r) {
            for (int kb = kb0; kb < kb1; ++kb) {
              if (cnt == 0) {
                if (!mbar_wait(&sm->acc_empty[buf], acc_phase[buf] ^ 1, abort, a.flags)) {
                  ok = false;
                  break;
                }
                fence_after();
              }
              if (!mbar_wait(&sm->full[stage], phase, abort, a.flags)) {
                ok = false;
                break;
              }
              fence_after();
              unsigned char* st = tiles_smem + stage * STAGE_BYTES;
              uint64_t da = smem_desc(st), db = smem_desc(st + STAGE_A_BYTES);
              uint32_t d = tmem + (uint32_t)(buf * BN);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(d, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), IDESC, (cnt > 0 || kk > 0) ? 1u : 0u);
              mma_commit(&sm->empty[stage]);
              any = true;
              if (++stage == STAGES) {
                stage = 0;
                phase ^= 1;
              }
              ++cnt;
              ++done;
              if (cnt == CHUNK_KB || done == total) {
                mma_commit(&sm->acc_full[buf]);
                acc_phase[buf] ^= 1;
                buf ^= 1;
                cnt = 0;
              }
            }
          }
        }
      }
      if (!ok && any) {
        // wait (bounded) for the MMAs already issued before the CTA frees TMEM
        mma_commit(&sm->drain);
        unsigned long long t0 = gtimer();
        while (!mbar_try(smem_u32(&sm->drain), 0) && gtimer() - t0 < 10000000ull) {
        }
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int ew = warp - 2;                 // 0..7
    const int quad = warp & 3;               // TMEM lanes 32*quad .. +31 (warp % 4 rule)
    const int col0 = (ew >> 2) * NCOL;       // columns [col0, col0 + NCOL)
    Acc R[NCOL];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) R[c] = 0;
    int buf = 0;
    uint32_t acc_phase[2] = {0, 0};
    bool ok = true;
    src.begin();
    int lu;
    while (ok && src.next(lu)) {
      const TcRun& a = src.run;
      const int* gorder = src.gorder;
      const int tiles = a.ntm * a.ntn;
      const int q = lu / tiles, tile = lu % tiles;
      const int grp = gorder[q / a.nsplit], kb0 = (q % a.nsplit) * a.kcb, kb1 = min(a.nkb, kb0 + a.kcb);
      int i0, j0;
      tile_origin(tile, a.ntm, a.ntn, BM, BN, i0, j0);
      const int64_t row = (int64_t)i0 + quad * 32 + lane;
      int t0 = 2 + grp * a.gs, t1 = min(t0 + a.gs - 1, a.tmax);
      for (int t = t0; t <= t1 && ok; ++t) {
        int total = (pair_hi(t, a.kL) - pair_lo(t, a.kR) + 1) * (kb1 - kb0);
        int chunks = (total + CHUNK_KB - 1) / CHUNK_KB;
        if constexpr (!W32) {
#pragma unroll
          for (int c = 0; c < NCOL; ++c) R[c] <<= DIGIT_BITS;
        }
        for (int ch = 0; ch < chunks; ++ch) {
          if (!mbar_wait(&sm->acc_full[buf], acc_phase[buf], abort, a.flags)) {
            ok = false;
            break;
          }
          fence_after();
          uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BN + col0);
#pragma unroll
          for (int h = 0; h < NCOL / 32; ++h) {
            uint32_t v[32];
            tmem_ld32(taddr + h * 32, v);
#pragma unroll
            for (int c = 0; c < 32; ++c) R[h * 32 + c] += (Acc)__float2int_rn(__uint_as_float(v[c]));
          }
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sm->acc_empty[buf]);
          acc_phase[buf] ^= 1;
          buf ^= 1;
        }
        if constexpr (SPLIT) {
          // this chunk's exact S_t, weighted for its Horner group, added to the group word
          if (ok && row < a.M) {
            unsigned long long* o = reinterpret_cast<unsigned long long*>(a.out) + grp * a.ogs + row;
            const int sh = DIGIT_BITS * (t1 - t);
#pragma unroll
            for (int c = 0; c < NCOL; ++c) {
              const int64_t j = (int64_t)j0 + col0 + c;
              if (j < a.N && R[c] != 0) atomicAdd(o + j * a.ldo, (unsigned long long)((i64)R[c] << sh));
            }
          }
#pragma unroll
          for (int c = 0; c < NCOL; ++c) R[c] = 0;
        }
      }
      if (!ok) break;
      if (!SPLIT && row < a.M) {
        Acc* o = reinterpret_cast<Acc*>(a.out) + grp * a.ogs + row;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
          int64_t j = (int64_t)j0 + col0 + c;
          if (j < a.N) o[j * a.ldo] = R[c];
        }
      }
#pragma unroll
      for (int c = 0; c < NCOL; ++c) R[c] = 0;
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}


template <int BN_, bool W32, bool SPLIT>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_plane_gemm_tc(const __grid_constant__ CUtensorMap mapL, const __grid_constant__ CUtensorMap mapR,
                    const __grid_constant__ TcArgs a0) {
  SingleSrc src;
  if (!tc_run_of<BN_, W32, SPLIT>(a0, src.run, src.gorder)) return;
  src.mapL = &mapL;
  src.mapR = &mapR;
  src.flags0 = a0.flags;
  if (threadIdx.x == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapL) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&mapR) : "memory");
  }
  tc_body<BN_, W32, SPLIT>(src);
}

// In-place exclusive prefix sum of a[0..count-1] in shared memory, a[count] = the total, by
// all NUM_THREADS threads: each thread sums a contiguous chunk, the chunk totals are scanned
// across the block, and each thread writes its chunk's prefixes.
__device__ __forceinline__ void block_exclusive_scan(int* a, int count, int* warp_tot) {
  const int per = (count + NUM_THREADS - 1) / NUM_THREADS;
  const int lo = min((int)threadIdx.x * per, count), hi = min(lo + per, count);
  int s = 0;
  for (int m = lo; m < hi; ++m) s += a[m];
  // inclusive scan of the thread totals: within warps, then across the warps' totals
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  int before = 0;
  for (int k = 0; k < w; ++k) before += warp_tot[k];
  int run = before + inc - s;   // exclusive prefix of this thread's chunk
  __syncthreads();
  for (int m = lo; m < hi; ++m) {
    const int v = a[m];
    a[m] = run;
    run += v;
  }
  if (threadIdx.x == NUM_THREADS - 1) a[count] = before + inc;
  __syncthreads();
}

// Many problems in one persistent launch (batched refinement): every CTA forms the prefix
// of the problems' unit counts (0 for finished or inactive products; the problems' arguments
// are read by all threads in parallel) and walks the global unit sequence.
template <int BN_, bool W32>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    k_plane_gemm_tc_grouped(const TcProblem* __restrict__ probs, int count) {
  __shared__ int prefix[MAX_GROUPED + 1];
  __shared__ int warp_tot[NUM_THREADS / 32];
  __shared__ RunRec recs[RUN_CACHE];
  const bool cached = count <= RUN_CACHE;
  for (int m = threadIdx.x; m < count; m += NUM_THREADS) {
    TcRun r;
    const int* g;
    const bool live = tc_run_of<BN_, W32, false>(probs[m].a, r, g);
    prefix[m] = live ? r.units : 0;
    if (cached && live) rec_of(r, g, recs[m]);
  }
  __syncthreads();
  block_exclusive_scan(prefix, count, warp_tot);
  if (prefix[count] == 0) return;
  GroupedSrc<BN_, W32> src;
  src.probs = probs;
  src.prefix = prefix;
  src.recs = cached ? recs : nullptr;
  src.count = count;
  src.cur = -1;
  src.gorder = nullptr;
  src.mapL = src.mapR = nullptr;
  src.flags0 = probs[0].a.flags;
  memset(&src.run, 0, sizeof(src.run));
  tc_body<BN_, W32, false>(src);
}

// A wait that nothing completes (no thread ever arrives on the barrier): the bounded wait of
// the slice-product kernels must give up after its limit, raise FLAG_TIMEOUT and return, so
// that the host reads an error status and the context stays usable.
__global__ void k_wait_timeout(int* flags) {
  __shared__ uint64_t bar;
  __shared__ int abort;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, &abort, flags);   // phase 0 never completes
}

// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

bool make_map(CUtensorMap* m, const void* base, int64_t K, int64_t rows, int planes, int64_t pitch,
              int64_t plane_stride, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * 2, (cuuint64_t)plane_stride * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t smem_bytes(int bn) {
  int stages = bn == 256 ? 4 : 6;
  return (size_t)stages * (STAGE_A_BYTES + (size_t)bn * BK * 2) + sizeof(Smem) + 1024;
}

}  // namespace

bool plane_gemm_tc_supported(const PlaneGemm& g) {
  if ((!g.dyn && g.d.groups <= 0) || g.M < 1 || g.N < 1 || g.K < 1) return false;
  if (g.pitch % 8 || g.Lps % 8 || g.Rps % 8) return false;
  if (((uintptr_t)g.L & 15) || ((uintptr_t)g.R & 15)) return false;
  if (g.M > (1 << 24) || g.N > (1 << 24)) return false;
  return get_encode() != nullptr;
}

// the streaming multiprocessors of the current device (persistent grids)
int sm_count(int& sms) {
  int dev = 0;
  FRX_CUDA_TRY(cudaGetDevice(&dev));
  FRX_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return FRX_OK;
}

template <int BN, bool W32, bool SPLIT>
int launch_variant(const PlaneGemm& g, const TcArgs& a, cudaStream_t s) {
  // tensor maps span the allocated planes (g.d.kL, g.d.kR: the capacity when d comes from the
  // device)
  CUtensorMap mL, mR;
  if (!make_map(&mL, g.L, g.K, g.M, g.d.kL, g.pitch, g.Lps, BM)) return FRX_E_CUDA;
  if (!make_map(&mR, g.R, g.K, g.N, g.d.kR, g.pitch, g.Rps, BN)) return FRX_E_CUDA;
  size_t smem = smem_bytes(BN);
  static PerDevice pd;
  FRX_TRY(once_per_device(pd, [&](int) -> int {
    FRX_CUDA_TRY(
        cudaFuncSetAttribute(k_plane_gemm_tc<BN, W32, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem));
    return FRX_OK;
  }));
  int sms = 0;
  FRX_TRY(sm_count(sms));
  const int64_t units = a.dyn ? (int64_t)sms
                              : ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * (int64_t)a.d.groups * a.nsplit;
  const unsigned grid = (unsigned)(units < sms ? units : sms);
  if (grid == 0) return FRX_OK;
  if (SPLIT) {
    // the units add into the group words: start them at zero (groups are ogs apart, each m x n
    // column-major with leading dimension ldo)
    for (int q = 0; q < a.d.groups; ++q)
      FRX_CUDA_TRY(cudaMemset2DAsync(g.out + q * g.ogs, sizeof(i64) * (size_t)g.ldo, 0, sizeof(i64) * (size_t)g.M,
                                     (size_t)g.N, s));
  }
  k_plane_gemm_tc<BN, W32, SPLIT><<<grid, NUM_THREADS, smem, s>>>(mL, mR, a);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

size_t tc_problem_bytes() { return sizeof(TcProblem); }

int launch_wait_timeout(int* dflags, cudaStream_t s) {
  k_wait_timeout<<<1, 32, 0, s>>>(dflags);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  return FRX_OK;
}

// one entry of a grouped launch's table (host memory), for a product with int32 planes and
// one CTA per output tile (TILE_128x128 or TILE_128x256)
int tc_problem_fill(const PlaneGemm& g, int* flags, void* host_entry, int tile) {
  if (!plane_gemm_tc_supported(g) || !g.d.word32 || (tile != TILE_128x128 && tile != TILE_128x256))
    return FRX_E_UNSUPPORTED;
  const int bn = tile_bn(tile);
  TcProblem* e = reinterpret_cast<TcProblem*>(host_entry);
  memset(e, 0, sizeof(TcProblem));
  if (!make_map(&e->mapL, g.L, g.K, g.M, g.d.kL, g.pitch, g.Lps, BM)) return FRX_E_CUDA;
  if (!make_map(&e->mapR, g.R, g.K, g.N, g.d.kR, g.pitch, g.Rps, bn)) return FRX_E_CUDA;
  e->a.M = g.M;
  e->a.N = g.N;
  e->a.nkb = (int)((g.K + BK - 1) / BK);
  e->a.out = (void*)g.out;
  e->a.ogs = g.ogs;
  e->a.ldo = g.ldo;
  e->a.flags = flags;
  e->a.d = g.d;
  e->a.dyn = g.dyn;
  e->a.done = g.done;
  e->a.bn = bn;
  e->a.nsplit = 1;
  e->a.kcb = e->a.nkb;
  return FRX_OK;
}

// shared-memory attributes of the grouped kernels (before any stream capture)
int prepare_plane_gemm_grouped() {
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_plane_gemm_tc_grouped<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_bytes(256)));
  FRX_CUDA_TRY(cudaFuncSetAttribute(k_plane_gemm_tc_grouped<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_bytes(128)));
  return FRX_OK;
}

// all problems of `table` (device memory, `count` entries filled for `tile`) in one
// persistent launch
int launch_plane_gemm_grouped(const void* table, int count, int tile, cudaStream_t s) {
  if (count <= 0) return FRX_OK;
  if (count > MAX_GROUPED || ((uintptr_t)table & 63) || (tile != TILE_128x128 && tile != TILE_128x256))
    return FRX_E_UNSUPPORTED;
  const int bn = tile_bn(tile);
  int sms = 0;
  FRX_TRY(sm_count(sms));
  const TcProblem* tab = reinterpret_cast<const TcProblem*>(table);
  if (bn == 256)
    k_plane_gemm_tc_grouped<256, true><<<(unsigned)sms, NUM_THREADS, smem_bytes(256), s>>>(tab, count);
  else
    k_plane_gemm_tc_grouped<128, true><<<(unsigned)sms, NUM_THREADS, smem_bytes(128), s>>>(tab, count);
  count_launches(1);
  FRX_CUDA_TRY(cudaGetLastError());
  last_tile() = tile;
  return FRX_OK;
}

// Split-K for int64 Horner groups: every K-chunk's anti-diagonal sums must stay exact in int32
// (pmax pairs x kcb k-blocks x 64 x 2^14 < 2^31).  The chunk is as long as that allows; when the
// output leaves SMs idle, more chunks (of at least 8 k-blocks) give them work.
void split_k_of(const PlaneGemm& g, int nkb, int tiles, int sms, int& nsplit, int& kcb) {
  int pmax = 1;
  for (int t = 2; t <= g.d.tmax; ++t) {
    const int lo = t - g.d.kR > 1 ? t - g.d.kR : 1, hi = g.d.kL < t - 1 ? g.d.kL : t - 1;
    pmax = hi - lo + 1 > pmax ? hi - lo + 1 : pmax;
  }
  const long long kmax = (((1ll << 31) - 1) / ((long long)pmax << PRODUCT_BITS)) / BK;   // k-blocks
  kcb = (int)(kmax < nkb ? kmax : nkb);
  nsplit = (nkb + kcb - 1) / kcb;
  kcb = (nkb + nsplit - 1) / nsplit;   // the same count of chunks, balanced (kcb only shrinks)
  // raise the requested chunk count one at a time (the chunk length only shrinks, so every
  // chunk stays exact); stop once the units fill the SMs or a chunk would drop below 8 k-blocks
  const long long base = (long long)tiles * g.d.groups;
  for (int want = nsplit + 1; base * nsplit < sms; ++want) {
    const int k2 = (nkb + want - 1) / want;
    if (k2 < 8) break;
    kcb = k2;
    nsplit = (nkb + kcb - 1) / kcb;
  }
}

bool split_k_enabled() {
  const char* env = getenv("FRX_SPLITK");
  return !(env && env[0] == '0');
}

// tile: TILE_128x128 or TILE_128x256 for int32 planes.  Int64 groups run split-K on 128 x 256
// tiles (FRX_SPLITK=0: the int64-register kernel on 128 x 128 tiles).
int launch_plane_gemm_tc(const PlaneGemm& g, int* flags, int tile, cudaStream_t s) {
  TcArgs a;
  a.M = g.M;
  a.N = g.N;
  a.nkb = (int)((g.K + BK - 1) / BK);
  a.nsplit = 1;
  a.kcb = a.nkb;
  a.out = (void*)g.out;
  a.ogs = g.ogs;
  a.ldo = g.ldo;
  a.flags = flags;
  a.d = g.d;
  a.dyn = g.dyn;
  a.done = g.done;
  if (!g.d.word32) {
    if (!g.dyn && split_k_enabled()) {
      int sms = 0;
      FRX_TRY(sm_count(sms));
      const int tiles = (int)(((g.M + BM - 1) / BM) * ((g.N + 255) / 256));
      split_k_of(g, a.nkb, tiles, sms, a.nsplit, a.kcb);
      a.bn = 256;
      last_tile() = TILE_128x256;
      return launch_variant<256, true, true>(g, a, s);
    }
    a.bn = 128;
    last_tile() = TILE_128x128;
    return launch_variant<128, false, false>(g, a, s);
  }
  last_tile() = tile;
  a.bn = tile_bn(tile);
  switch (tile) {
    case TILE_128x128:
      return launch_variant<128, true, false>(g, a, s);
    case TILE_128x256:
      return launch_variant<256, true, false>(g, a, s);
    default:
      return FRX_E_UNSUPPORTED;
  }
}

}  // namespace frx
