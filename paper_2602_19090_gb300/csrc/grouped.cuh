// Grouped launches: one launch runs the same kernel body over many independent problems
// (the matrices of a batched refinement).  Each problem contributes the blocks of its own
// single-problem launch; a block finds its problem by binary search in the prefix of the
// problems' block counts and takes that problem's argument struct from a device table.
#pragma once

#include <vector>

#include "frx_internal.cuh"

namespace frx {

// problem m of block b: the last m with start[m] <= b (start[count] = total blocks)
__device__ __forceinline__ int group_of(const long long* __restrict__ start, int count, long long b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Body(args, bx, by): the single-problem kernel's work for block (bx, by); Args carries the
// single launch's grid width gx.
template <class Args, void (*Body)(Args, unsigned, unsigned), int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
    k_grouped(const Args* __restrict__ tab, const long long* __restrict__ start, int count) {
  const long long b = blockIdx.x;
  const int m = group_of(start, count, b);
  const long long local = b - start[m];
  const unsigned gx = tab[m].gx;
  Body(tab[m], (unsigned)(local % gx), (unsigned)(local / gx));
}

// Kinds of recorded launches (one per kernel body)
enum LaunchKind {
  LK_COL_EXPONENTS = 1,
  LK_ROW_MAXBITS,
  LK_MAXBITS_TO_EXPONENTS,
  LK_SLICE_COLS,
  LK_SLICE_ROWS,
  LK_TRUNCATE_SLICE_X,
  LK_RESIDUAL,
  LK_W_OFFDIAG,
  LK_CORRECTION,
  LK_UPDATE,
  LK_PLAN_INIT,
  LK_PLAN_V,
  LK_PLAN_MARK_SLICED,
  LK_PLAN_W,
  LK_PLAN_OMEGA,
  LK_PLAN_U,
  LK_PLAN_END,
  LK_GEMM,
  LK_ZERO,
  LK_COPY,
};

// A launch recorded instead of issued: its kind, its argument struct (bytes), its blocks,
// threads per block and dynamic shared memory.
struct LaunchRecord {
  int kind;
  std::vector<unsigned char> args;
  long long blocks;
  int threads;
  size_t smem;
  int variant = 0;   // slice products: the tile configuration the entry was filled for
};

struct LaunchRecorder {
  std::vector<LaunchRecord> recs;
  int tile = 2;      // tile configuration of the slice products recorded (128 x 256)
};

// the calling host thread's active recorder (nullptr: launchers issue their kernels)
LaunchRecorder*& active_recorder();

template <class Args>
bool record_launch(int kind, const Args& a, long long blocks, int threads, size_t smem) {
  LaunchRecorder* R = active_recorder();
  if (!R) return false;
  LaunchRecord r;
  r.kind = kind;
  r.args.assign(reinterpret_cast<const unsigned char*>(&a), reinterpret_cast<const unsigned char*>(&a) + sizeof(Args));
  r.blocks = blocks;
  r.threads = threads;
  r.smem = smem;
  R->recs.push_back(std::move(r));
  return true;
}

// grouped launch of `count` recorded problems of one kind (the table and the block starts
// live in device memory); defined by the translation unit that owns the kind
int launch_grouped_scan(int kind, const void* tab, const long long* start, int count, long long blocks, int threads,
                        size_t smem, cudaStream_t s);
int launch_grouped_refine(int kind, const void* tab, const long long* start, int count, long long blocks,
                          int threads, size_t smem, cudaStream_t s);
int launch_grouped_plan(int kind, const void* tab, const long long* start, int count, long long blocks, int threads,
                        size_t smem, cudaStream_t s);

}  // namespace frx
