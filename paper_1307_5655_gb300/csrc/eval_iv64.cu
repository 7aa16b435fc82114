// Instantiation of the evaluation kernel for the IV64 value type.
#include "eval_kernel.cuh"

namespace fp {
cudaError_t launch_eval_iv64(const EvalArgs& a, cudaStream_t s) { return launch_eval<IV64, 1>(a, s); }
}  // namespace fp
