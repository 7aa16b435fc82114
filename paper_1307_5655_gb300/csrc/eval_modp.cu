// Instantiation of the evaluation kernel for the MODP value type.
#include "eval_kernel.cuh"

namespace fp {
cudaError_t launch_eval_modp(const EvalArgs& a, cudaStream_t s) { return launch_eval<MODP, 2>(a, s); }
}  // namespace fp
