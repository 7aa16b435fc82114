// Instantiation of the evaluation kernel for the IV64 value type (node by
// node, in the paper's operation order), for 1 or 2 points per thread.
#include "eval_kernel.cuh"

namespace fp {
cudaError_t launch_eval_iv64(const EvalArgs& a, const OpArgs&, int, cudaStream_t s, int variant, int ppt) {
  if (variant == 1) return cudaErrorInvalidValue;
  if (ppt == 2) return launch_eval_smem<IV64, 2>(a, s);
  return launch_eval_smem<IV64, 1>(a, s);
}
}  // namespace fp
