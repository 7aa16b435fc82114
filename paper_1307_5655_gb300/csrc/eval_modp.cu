// Instantiation of the evaluation kernels for the MODP value type.
#include "eval_kernel.cuh"

namespace fp {
cudaError_t launch_eval_modp(const EvalArgs& a, const OpArgs& o, int scheme, cudaStream_t s, int variant) {
  return launch_eval_fused<MODP, 2, 2>(a, o, scheme, s, variant);
}
}  // namespace fp
