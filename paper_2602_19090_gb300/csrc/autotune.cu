// Tile autotuner of the slice products.
//
// The persistent tensor-core kernel covers the M x N output of a product with 128 x 256 or
// 128 x 128 tiles per CTA.  Wide tiles read each A panel once for more columns; narrow tiles
// waste less of a small or ragged output and give the SMs more units to balance.  The choice
// changes no bit of the result (every tile sum is exact), only the time.
//
// A product (or a batch of products run as one grouped launch) is described by a key: the
// output shape, inner dimension and plane counts, or for a batch its sorted sizes.  The first
// time a key is seen, a cost model decides at once when the wide configuration covers the
// output with almost no padding and still gives every SM several units; otherwise every
// candidate is timed with CUDA events on the caller's stream (one warm launch, then TUNE_REPS
// launches each) and the fastest is cached for the key.  A stream that is being captured cannot
// be timed: the model's estimate decides there and nothing is cached.  frx_set_tile forces a
// configuration.
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "frx_internal.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace frx {
namespace {

static_assert(TILE_AUTO == FRX_TILE_AUTO && TILE_128x128 == FRX_TILE_128x128 && TILE_128x256 == FRX_TILE_128x256,
              "tile codes of the C ABI");

constexpr int TUNE_REPS = 3;
constexpr double WIDE_COVER = 0.97;   // padded-area fraction above which the wide tiles win outright
constexpr int WIDE_UNITS_PER_SM = 4;
constexpr int WIDE_SETTLED = TILE_128x256;   // the model's choice for large, tile-aligned products

std::atomic<int> g_policy{TILE_AUTO};
std::mutex g_mu;
std::map<std::vector<long long>, int> g_cache;
long long g_measured = 0, g_modelled = 0, g_hits = 0;

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// output area, and per tile configuration (index cfg - 1) the padded area and the CTA units
// (one CTA's tile-and-anti-diagonal-group work items)
struct Shape {
  double area = 0.0, padded[TILE_LAST] = {};
  int64_t units[TILE_LAST] = {};
};

void add_shape(Shape& sh, int64_t M, int64_t N, int groups) {
  sh.area += (double)M * (double)N;
  for (int c = TILE_128x128; c <= TILE_LAST; ++c) {
    const int bn = tile_bn(c);
    sh.padded[c - 1] += (double)(cdiv(M, 128) * 128) * (double)(cdiv(N, bn) * bn);
    sh.units[c - 1] += cdiv(M, 128) * cdiv(N, bn) * (int64_t)groups;
  }
}

// the settled configuration, or TILE_AUTO when the candidates must be timed
int model_decides(const Shape& sh, int sms) {
  const int w = WIDE_SETTLED - 1;
  if (sh.area >= WIDE_COVER * sh.padded[w] && sh.units[w] >= (int64_t)WIDE_UNITS_PER_SM * sms) return WIDE_SETTLED;
  return TILE_AUTO;
}

// the model's estimate when nothing can be timed: waves of CTA units, each unit's cost
// proportional to its tile width
int model_estimate(const Shape& sh, const std::vector<int>& cands, int sms) {
  int best = cands[0];
  double bc = 1e300;
  for (int c : cands) {
    const double cost = (double)cdiv(sh.units[c - 1], sms) * tile_bn(c);
    if (cost < bc) {
      bc = cost;
      best = c;
    }
  }
  return best;
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

bool cached(const std::vector<long long>& key, int& tile) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  tile = it->second;
  ++g_hits;
  return true;
}

void store(const std::vector<long long>& key, int tile, bool measured) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = tile;
  if (measured) ++g_measured;
  else ++g_modelled;
}

// decide for `key` among `cands` from the model or by timing launch(cfg) for each; prepare()
// runs once before the first timed launch
template <class P, class F>
int decide(const std::vector<long long>& shape_key, const Shape& sh, const std::vector<int>& cands, P prepare,
           F launch, cudaStream_t s, int& tile) {
  // decisions belong to a device (a process may drive devices of different kinds)
  int dev = 0;
  FRX_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<long long> key = shape_key;
  key.push_back(dev);
  const int forced = g_policy.load();
  if (forced != TILE_AUTO) {
    bool offered = false;
    for (int c : cands) offered |= c == forced;
    tile = offered ? forced : TILE_128x256;
    return FRX_OK;
  }
  if (cached(key, tile)) return FRX_OK;
  int sms = 0;
  FRX_TRY(sms_of_device(sms));
  const int m = model_decides(sh, sms);
  bool offered = false;
  for (int c : cands) offered |= c == m;
  if (m != TILE_AUTO && offered) {
    tile = m;
    store(key, tile, false);
    return FRX_OK;
  }
  if (capturing(s)) {
    tile = model_estimate(sh, cands, sms);
    return FRX_OK;
  }
  FRX_TRY(prepare());
  float best = 1e30f;
  for (int c : cands) {
    float ms = 0.f;
    FRX_TRY(time_launches([&]() { return launch(c); }, s, ms));
    if (ms < best) {
      best = ms;
      tile = c;
    }
  }
  store(key, tile, true);
  return FRX_OK;
}

// candidates for one product
std::vector<int> single_candidates() { return {TILE_128x256, TILE_128x128}; }

// zero both operands' planes of a representative product (its timing reads defined digits)
int zero_operands(const PlaneGemm& g, cudaStream_t s) {
  FRX_CUDA_TRY(cudaMemsetAsync((void*)g.L, 0, sizeof(__nv_bfloat16) * (size_t)g.Lps * g.d.kL, s));
  FRX_CUDA_TRY(cudaMemsetAsync((void*)g.R, 0, sizeof(__nv_bfloat16) * (size_t)g.Rps * g.d.kR, s));
  return FRX_OK;
}

// a static product with int32 planes, timed on the product itself: its inputs are in place
// and the timing launches write the exact sums the real launch writes again afterwards.
// For a representative product, prepare() fills its operands first.
template <class P>
int tune_single_impl(const PlaneGemm& g, int kind, P prepare, cudaStream_t s, int& tile) {
  if (!g.d.word32) {
    tile = TILE_128x128;   // int64 groups: the only variant
    return FRX_OK;
  }
  if (g.dyn) {
    // plan-driven product without a tuned configuration: nothing to time it on here
    const int p = tile_policy();
    tile = p != TILE_AUTO ? p : TILE_128x256;
    return FRX_OK;
  }
  Shape sh;
  add_shape(sh, g.M, g.N, g.d.groups);
  std::vector<long long> key = {kind, g.M, g.N, g.K, g.d.kL, g.d.kR, g.d.T};
  return decide(key, sh, single_candidates(), prepare,
                [&](int c) { return launch_plane_gemm_tc(g, g.flags, c, s); }, s, tile);
}

}  // namespace

int tile_policy() { return g_policy.load(); }

int tune_tile_single(const PlaneGemm& g, int kind, cudaStream_t s, int& tile) {
  return tune_single_impl(g, kind, []() { return (int)FRX_OK; }, s, tile);
}

// the configuration of a refinement's plan-driven products (keyed by n and the
// representative's plane counts), tuned on a representative product over the workspace's
// plane buffers
int tune_tile_refine(const PlaneGemm& rep, cudaStream_t s, int& tile) {
  return tune_single_impl(rep, 2, [&]() { return zero_operands(rep, s); }, s, tile);
}

// a batch of representative products run as one grouped launch (their operands are zeroed
// before timing); `table` is device scratch of at least 2 * count * tc_problem_bytes()
// bytes, 64-byte aligned.  Grouped launches use one CTA per tile.
int tune_tile_grouped(const std::vector<PlaneGemm>& gs, const std::vector<long long>& key, void* table,
                      cudaStream_t s, int& tile) {
  tile = TILE_128x256;
  const int count = (int)gs.size();
  if (count == 0) return FRX_OK;
  Shape sh;
  for (const PlaneGemm& g : gs) add_shape(sh, g.M, g.N, g.d.groups);
  const size_t eb = tc_problem_bytes();
  std::vector<unsigned char> host(eb * (size_t)count);
  char* dev[2] = {(char*)table, (char*)table + eb * (size_t)count};
  bool uploaded[2] = {false, false};
  auto launch = [&](int c) -> int {
    const int slot = c == TILE_128x256 ? 0 : 1;
    if (!uploaded[slot]) {
      for (int b = 0; b < count; ++b) FRX_TRY(tc_problem_fill(gs[b], gs[b].flags, host.data() + eb * b, c));
      FRX_CUDA_TRY(cudaMemcpyAsync(dev[slot], host.data(), host.size(), cudaMemcpyHostToDevice, s));
      FRX_CUDA_TRY(cudaStreamSynchronize(s));
      uploaded[slot] = true;
    }
    return launch_plane_gemm_grouped(dev[slot], count, c, s);
  };
  auto prepare = [&]() -> int {
    for (const PlaneGemm& g : gs) FRX_TRY(zero_operands(g, s));
    return FRX_OK;
  };
  return decide(key, sh, std::vector<int>{TILE_128x256, TILE_128x128}, prepare, launch, s, tile);
}

int& last_tile() {
  static thread_local int t = TILE_AUTO;
  return t;
}

}  // namespace frx

using namespace frx;

extern "C" {

int frx_set_tile(int tile) {
  if (tile < TILE_AUTO || tile > TILE_LAST) return FRX_E_ARG;
  return g_policy.exchange(tile);
}

int frx_last_tile(void) { return last_tile(); }

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
