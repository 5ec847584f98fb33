// Launch accounting and CUDA-event timing of the slice-product GEMMs.
#include <mutex>
#include <vector>

#include "frx_internal.cuh"
#include "grouped.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace frx {
namespace {

struct Timed {
  cudaEvent_t a, b;
};

std::mutex mu;
bool enabled = false;
long long launches = 0, gemm_launches = 0, simt_launches = 0;
double gemm_ms = 0.0, gemm_ops = 0.0, gemm_bytes = 0.0;
std::vector<Timed> pending;
std::vector<cudaEvent_t> free_events;

cudaEvent_t get_event() {
  if (!free_events.empty()) {
    cudaEvent_t e = free_events.back();
    free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

void count_launches(int k) {
  std::lock_guard<std::mutex> g(mu);
  launches += k;
}

void count_simt_launch() {
  std::lock_guard<std::mutex> g(mu);
  simt_launches += 1;
}

// operations of plan-driven products, known only once the device plan has run
void profile_add_gemm_work(double ops) {
  std::lock_guard<std::mutex> g(mu);
  gemm_ops += ops;
}

GemmTimer::GemmTimer(const PlaneGemm& g, cudaStream_t s) : s_(s) {
  std::lock_guard<std::mutex> lk(mu);
  gemm_launches += 1;
  launches += 1;
  if (!g.dyn) {
    int pairs = desc_pairs(g.d);
    gemm_ops += 2.0 * (double)g.M * (double)g.N * (double)g.K * pairs;
    gemm_bytes += 2.0 * (double)g.K * ((double)g.M * g.d.kL + (double)g.N * g.d.kR) +
                  (g.d.word32 ? 4.0 : 8.0) * g.d.groups * (double)g.M * g.N;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s_, &cs);
  if (enabled && cs == cudaStreamCaptureStatusNone) {
    a_ = get_event();
    b_ = get_event();
    cudaEventRecord(a_, s_);
  }
}

GemmTimer::~GemmTimer() {
  if (a_) {
    cudaEventRecord(b_, s_);
    std::lock_guard<std::mutex> lk(mu);
    pending.push_back({a_, b_});
  }
}

LaunchRecorder*& active_recorder() {
  static thread_local LaunchRecorder* r = nullptr;
  return r;
}

}  // namespace frx

using namespace frx;

extern "C" {

void frx_profile_enable(int on) {
  std::lock_guard<std::mutex> g(mu);
  enabled = on != 0;
}

int frx_profile_read(frx_profile* out, int reset) {
  std::lock_guard<std::mutex> g(mu);
  for (auto& t : pending) {
    if (cudaEventSynchronize(t.b) != cudaSuccess) return FRX_E_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    gemm_ms += ms;
    free_events.push_back(t.a);
    free_events.push_back(t.b);
  }
  pending.clear();
  if (out) {
    out->kernel_launches = launches;
    out->gemm_launches = gemm_launches;
    out->gemm_ms = gemm_ms;
    out->gemm_ops = gemm_ops;
    out->gemm_bytes = gemm_bytes;
    out->simt_launches = simt_launches;
  }
  if (reset) {
    launches = gemm_launches = simt_launches = 0;
    gemm_ms = gemm_ops = gemm_bytes = 0.0;
  }
  return FRX_OK;
}

}  // extern "C"
