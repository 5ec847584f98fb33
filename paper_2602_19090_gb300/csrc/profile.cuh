// Launch accounting (see frx_profile_* in include/frx.h).
#pragma once

#include "kernels.cuh"

namespace frx {

void count_launches(int k);
void count_simt_launch();   // a slice product that ran on the CUDA cores (see frx_profile)
void profile_add_gemm_work(double ops);

// RAII: counts one GEMM launch and, with profiling on, brackets it with CUDA events
class GemmTimer {
 public:
  GemmTimer(const PlaneGemm& g, cudaStream_t s);
  ~GemmTimer();

 private:
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

}  // namespace frx
