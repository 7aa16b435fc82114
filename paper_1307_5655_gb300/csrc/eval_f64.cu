// Instantiation of the evaluation kernel for the F64 value type.
#include "eval_kernel.cuh"

namespace fp {
cudaError_t launch_eval_f64(const EvalArgs& a, cudaStream_t s) { return launch_eval<F64, 1>(a, s); }
}  // namespace fp
