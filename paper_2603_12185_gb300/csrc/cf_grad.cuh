// Adjoint of the step (reverse mode with checkpoint recomputation) -- internal interface.
#pragma once
#include <cstddef>
#include <cstdint>

#include "cf_internal.cuh"

namespace cf {

struct GradArgs {
  int T, ckpt, W;
  int64_t total_nq, total_nv;
  char* tape;
  const float *dqT, *dvT;
  float *dq0, *dv0, *dtau;
  int num_sms;
};

size_t grad_workspace_bytes(int W, int64_t total_nq, int64_t total_nv, const cf_batch_opts& o);
cudaError_t run_grad(const StepParams& p, const GradArgs& g, int nctrl, cudaStream_t s);

}  // namespace cf
