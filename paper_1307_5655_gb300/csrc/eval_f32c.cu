// Instantiation of the evaluation kernel for the F32C value type.
#include "eval_kernel.cuh"

namespace fp {
cudaError_t launch_eval_f32c(const EvalArgs& a, cudaStream_t s) { return launch_eval<F32C, 2>(a, s); }
}  // namespace fp
