// Adjoint of the step (reverse mode with checkpoint recomputation) -- internal interface.
#pragma once
#include <cstddef>
#include <cstdint>

#include "cf_internal.cuh"

namespace cf {

// limits of the per-thread articulated step used by the adjoint
constexpr int kG1Body = 24;
constexpr int kG1Geom = 32;
constexpr int kG1Q = 48;
constexpr int kG1V = 48;
constexpr int kG1Tree = 8;
constexpr int kG1Lanes = 64;   // tangent lanes per world (inputs nq + nv + nu <= 128, two passes)

struct GradArgs {
  int T, ckpt, W;
  int64_t total_nq, total_nv, total_nu;
  char* tape;
  const float *dqT, *dvT;
  float *dq0, *dv0, *dtau;
  int num_sms;
  size_t smem;               // dynamic shared memory of the step launch over all worlds
  int variant;               // step-kernel variant of the forward recomputation (launch_step)
};

size_t grad_workspace_bytes(int W, int64_t total_nq, int64_t total_nv, const cf_batch_opts& o);
// checks that every scene fits the per-thread step; returns false with a reason
bool grad_scene_supported(const DScene& s, const char** why);
cudaError_t run_grad(const StepParams& p, const GradArgs& g, int nctrl, cudaStream_t s);

}  // namespace cf
