// Instantiation of the evaluation kernels for the F32C value type.
#include "eval_kernel.cuh"

namespace fp {
cudaError_t launch_eval_f32c(const EvalArgs& a, const OpArgs& o, int scheme, cudaStream_t s, int variant) {
  return launch_eval_fused<F32C, 2, 2>(a, o, scheme, s, variant);
}
}  // namespace fp
