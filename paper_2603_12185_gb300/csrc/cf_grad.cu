#include "cf_grad.cuh"

namespace cf {
size_t grad_workspace_bytes(int W, int64_t total_nq, int64_t total_nv, const cf_batch_opts& o) {
  (void)W; (void)total_nq; (void)total_nv; (void)o;
  return 256;
}
cudaError_t run_grad(const StepParams&, const GradArgs&, int, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace cf
