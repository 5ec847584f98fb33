// Launchers of the device-side plan kernels (plan.cu).
#pragma once

#include "plan.cuh"

namespace frx {

// rank: n words of scratch for a many-block ranking of the estimates ahead of the one-block
// plan kernel (nullptr: the plan kernel sorts them itself)
int launch_plan_init(DevPlan* p, const int32_t* eA, const double* D, double* lam_prev, const PlanOpts& o,
                     double omega_prev, uint32_t* rank, cudaStream_t s);
int launch_plan_v(DevPlan* p, const int32_t* f, const PlanOpts& o, cudaStream_t s);
int launch_plan_mark_sliced(DevPlan* p, cudaStream_t s);
int launch_plan_w(DevPlan* p, const int32_t* h, const PlanOpts& o, cudaStream_t s);
int launch_plan_omega(DevPlan* p, const double* r, const double* colsq, const PlanOpts& o, cudaStream_t s);
int launch_plan_u(DevPlan* p, const int32_t* rho, const int32_t* eta, const PlanOpts& o, cudaStream_t s);
int launch_plan_end(DevPlan* p, const double* lam_new, double* lam_prev, const double* colsq, const PlanOpts& o,
                    uint32_t* rank, cudaStream_t s);
int set_plan_kernel_attributes();
int launch_collect_done(DevPlan* const* plans, int count, int* done, cudaStream_t s);
int launch_gather_plans(DevPlan* const* plans, int count, DevPlan* out, cudaStream_t s);

}  // namespace frx
