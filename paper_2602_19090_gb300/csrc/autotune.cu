// Tile-width autotuner of the slice products.
//
// The persistent tensor-core kernel covers an M x N output of a product with 128 x 256 or
// 128 x 128 tiles (exact int32 planes).  Wide tiles read each A panel once for twice the
// columns; narrow tiles waste less of a small or ragged output and give the SMs more units to
// balance.  The choice changes no bit of the result (every tile sum is exact), only the time.
//
// A product (or a batch of products run as one grouped launch) is described by a key: the
// output shape, inner dimension and plane counts, or for a batch its sorted sizes.  The first
// time a key is seen, a cost model decides at once when the wide tiles cover the output with
// almost no padding and still give every SM several units; otherwise both widths are timed
// with CUDA events on the caller's stream (one warm launch, then TUNE_REPS launches each) and
// the faster one is cached for the key.  A stream that is being captured cannot be timed: the
// model's estimate decides there and nothing is cached.  frx_set_tile_n forces a width.
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "frx_internal.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace frx {
namespace {

constexpr int TUNE_REPS = 3;
constexpr double WIDE_COVER = 0.97;   // padded-area fraction above which wide tiles win outright
constexpr int WIDE_UNITS_PER_SM = 4;

std::atomic<int> g_policy{0};
std::mutex g_mu;
std::map<std::vector<long long>, int> g_cache;
long long g_measured = 0, g_modelled = 0, g_hits = 0;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// output area, padded area at width bn and units (tiles x anti-diagonal groups) of one product
struct Shape {
  double area, padded[2];
  int64_t units[2];
};

void add_shape(Shape& sh, int64_t M, int64_t N, int groups) {
  const int widths[2] = {256, 128};
  sh.area += (double)M * (double)N;
  for (int w = 0; w < 2; ++w) {
    sh.padded[w] += (double)(cdiv(M, 128) * 128) * (double)(cdiv(N, widths[w]) * widths[w]);
    sh.units[w] += cdiv(M, 128) * cdiv(N, widths[w]) * (int64_t)groups;
  }
}

// 256 when wide tiles settle it without timing, 0 when both must be timed
int model_decides(const Shape& sh, int sms) {
  if (sh.area >= WIDE_COVER * sh.padded[0] && sh.units[0] >= (int64_t)WIDE_UNITS_PER_SM * sms) return 256;
  return 0;
}

// the model's estimate when nothing can be timed: waves of units, each unit's cost
// proportional to its tile width
int model_estimate(const Shape& sh, int sms) {
  const double c256 = (double)cdiv(sh.units[0], sms) * 256.0;
  const double c128 = (double)cdiv(sh.units[1], sms) * 128.0;
  return c128 < c256 ? 128 : 256;
}

int sms_of_device(int& sms) {
  int dev = 0;
  FRX_CUDA_TRY(cudaGetDevice(&dev));
  FRX_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return FRX_OK;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return true;
  return cs != cudaStreamCaptureStatusNone;
}

// milliseconds per launch of `launch` (one warm launch first)
template <class F>
int time_launches(F launch, cudaStream_t s, float& ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  FRX_CUDA_TRY(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return FRX_E_CUDA;
  }
  int st = [&]() -> int {
    FRX_TRY(launch());
    FRX_CUDA_TRY(cudaEventRecord(a, s));
    for (int r = 0; r < TUNE_REPS; ++r) FRX_TRY(launch());
    FRX_CUDA_TRY(cudaEventRecord(b, s));
    FRX_CUDA_TRY(cudaEventSynchronize(b));
    FRX_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    ms /= (float)TUNE_REPS;
    return FRX_OK;
  }();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  count_launches(TUNE_REPS + 1);
  return st;
}

bool cached(const std::vector<long long>& key, int& bn) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  bn = it->second;
  ++g_hits;
  return true;
}

void store(const std::vector<long long>& key, int bn, bool measured) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = bn;
  if (measured) ++g_measured;
  else ++g_modelled;
}

// decide for `key` from the model or by timing launch(256) against launch(128); prepare()
// runs once before the first timed launch
template <class P, class F>
int decide(const std::vector<long long>& key, const Shape& sh, P prepare, F launch, cudaStream_t s, int& bn) {
  const int forced = g_policy.load();
  if (forced) {
    bn = forced;
    return FRX_OK;
  }
  if (cached(key, bn)) return FRX_OK;
  int sms = 0;
  FRX_TRY(sms_of_device(sms));
  const int m = model_decides(sh, sms);
  if (m) {
    bn = m;
    store(key, bn, false);
    return FRX_OK;
  }
  if (capturing(s)) {
    bn = model_estimate(sh, sms);
    return FRX_OK;
  }
  float t256 = 0.f, t128 = 0.f;
  FRX_TRY(prepare());
  FRX_TRY(time_launches([&]() { return launch(256); }, s, t256));
  FRX_TRY(time_launches([&]() { return launch(128); }, s, t128));
  bn = t128 < t256 ? 128 : 256;
  store(key, bn, true);
  return FRX_OK;
}

}  // namespace

int tile_policy() { return g_policy.load(); }

// a static product with int32 planes, timed on the product itself: its inputs are in place
// and the timing launches write the exact sums the real launch writes again afterwards.
// For a representative product, prepare() fills its operands first.
template <class P>
int tune_single_impl(const PlaneGemm& g, int kind, P prepare, cudaStream_t s, int& bn) {
  if (!g.d.word32) {
    bn = 128;   // int64 groups: the only variant
    return FRX_OK;
  }
  if (g.dyn) {
    // plan-driven product without a tuned width: nothing to time it on here
    bn = tile_policy() ? tile_policy() : 256;
    return FRX_OK;
  }
  Shape sh = {};
  add_shape(sh, g.M, g.N, g.d.groups);
  std::vector<long long> key = {kind, g.M, g.N, g.K, g.d.kL, g.d.kR, g.d.T};
  return decide(key, sh, prepare, [&](int w) { return launch_plane_gemm_tc(g, g.flags, w, s); }, s, bn);
}

int tune_tile_single(const PlaneGemm& g, int kind, cudaStream_t s, int& bn) {
  return tune_single_impl(g, kind, []() { return (int)FRX_OK; }, s, bn);
}

// zero both operands' planes of a representative product (its timing reads defined digits)
int zero_operands(const PlaneGemm& g, cudaStream_t s) {
  FRX_CUDA_TRY(cudaMemsetAsync((void*)g.L, 0, sizeof(__nv_bfloat16) * (size_t)g.Lps * g.d.kL, s));
  FRX_CUDA_TRY(cudaMemsetAsync((void*)g.R, 0, sizeof(__nv_bfloat16) * (size_t)g.Rps * g.d.kR, s));
  return FRX_OK;
}

// a batch of representative products run as one grouped launch (their operands are zeroed
// before timing); `table` is device scratch of at least 2 * count * tc_problem_bytes()
// bytes, 64-byte aligned
int tune_tile_grouped(const std::vector<PlaneGemm>& gs, const std::vector<long long>& key, void* table,
                      cudaStream_t s, int& bn) {
  bn = 256;
  const int count = (int)gs.size();
  if (count == 0) return FRX_OK;
  Shape sh = {};
  for (const PlaneGemm& g : gs) add_shape(sh, g.M, g.N, g.d.groups);
  const size_t eb = tc_problem_bytes();
  std::vector<unsigned char> host(eb * (size_t)count);
  char* dev[2] = {(char*)table, (char*)table + eb * (size_t)count};
  bool uploaded[2] = {false, false};
  auto launch = [&](int w) -> int {
    const int slot = w == 256 ? 0 : 1;
    if (!uploaded[slot]) {
      for (int b = 0; b < count; ++b) FRX_TRY(tc_problem_fill(gs[b], gs[b].flags, host.data() + eb * b, w));
      FRX_CUDA_TRY(cudaMemcpyAsync(dev[slot], host.data(), host.size(), cudaMemcpyHostToDevice, s));
      FRX_CUDA_TRY(cudaStreamSynchronize(s));
      uploaded[slot] = true;
    }
    return launch_plane_gemm_grouped(dev[slot], count, w, s);
  };
  auto prepare = [&]() -> int {
    for (const PlaneGemm& g : gs) FRX_TRY(zero_operands(g, s));
    return FRX_OK;
  };
  return decide(key, sh, prepare, launch, s, bn);
}

// the width of a refinement's plan-driven products (keyed by n and the representative's
// plane counts), tuned on a representative product over the workspace's plane buffers
int tune_tile_refine(const PlaneGemm& rep, cudaStream_t s, int& bn) {
  return tune_single_impl(rep, 2, [&]() { return zero_operands(rep, s); }, s, bn);
}

int& last_tile_n() {
  static thread_local int w = 0;
  return w;
}

}  // namespace frx

using namespace frx;

extern "C" {

int frx_set_tile_n(int tile_n) {
  if (tile_n != 0 && tile_n != 128 && tile_n != 256) return FRX_E_ARG;
  return g_policy.exchange(tile_n);
}

int frx_last_tile_n(void) { return last_tile_n(); }

int frx_tune_stats(long long* measured, long long* modelled, long long* hits, int clear) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (measured) *measured = g_measured;
  if (modelled) *modelled = g_modelled;
  if (hits) *hits = g_hits;
  if (clear) {
    g_cache.clear();
    g_measured = g_modelled = g_hits = 0;
  }
  return FRX_OK;
}

}  // extern "C"
