// Instantiation of the evaluation kernels for the F64 value type.
#include "eval_kernel.cuh"

namespace fp {
cudaError_t launch_eval_f64(const EvalArgs& a, const OpArgs& o, int scheme, cudaStream_t s, int variant) {
  return launch_eval_fused<F64, 1, 1>(a, o, scheme, s, variant);
}
}  // namespace fp
