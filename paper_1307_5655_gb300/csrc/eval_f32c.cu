// Instantiation of the evaluation kernels for the F32C value type, for every
// points-per-thread count the autotuner may choose (default 2).
#include "eval_kernel.cuh"

namespace fp {
cudaError_t launch_eval_f32c(const EvalArgs& a, const OpArgs& o, int scheme, cudaStream_t s, int variant, int ppt) {
  switch (ppt) {
    case 1: return launch_eval_fused<F32C, 1, 1>(a, o, scheme, s, variant);
    case 2: return launch_eval_fused<F32C, 2, 2>(a, o, scheme, s, variant);
    case 4: return launch_eval_fused<F32C, 4, 4>(a, o, scheme, s, variant);
    default: return launch_eval_fused<F32C, 2, 2>(a, o, scheme, s, variant);
  }
}
}  // namespace fp
