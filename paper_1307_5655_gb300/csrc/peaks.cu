// Sustained arithmetic rates of the operations the evaluation kernels are
// bound by: the denominators of their rooflines.  Each thread runs kChains
// independent dependent chains of one operation (the library's own
// arithmetic policies, so the rate is that of the code the kernels run);
// only out[thread] is written.
#include <cuda_runtime.h>

#include "eval_kernel.cuh"

namespace fp {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

// Operands come from memory (registers at run time): FP64 instructions with
// constant-bank operands issue slower than with register operands.
struct Params {
  double d[4];
  float f[4];
  uint64_t u[2];
  uint32_t w[2];
};

struct OpDfma {
  using T = double;
  static __device__ T init(const Params& q, int j) { return q.d[0] + j * 1e-3 + threadIdx.x * 1e-9; }
  static __device__ T step(const Params& q, T a) { return fma(a, q.d[1], q.d[2]); }
  static __device__ double out(T a) { return a; }
};
struct OpDaddRd {
  using T = double;
  static __device__ T init(const Params& q, int j) { return q.d[0] + j * 1e-3 + threadIdx.x * 1e-9; }
  static __device__ T step(const Params& q, T a) { return __dadd_rd(a, q.d[3]); }
  static __device__ double out(T a) { return a; }
};
struct OpDmulRu {
  using T = double;
  static __device__ T init(const Params& q, int j) { return q.d[0] + j * 1e-3 + threadIdx.x * 1e-9; }
  static __device__ T step(const Params& q, T a) { return __dmul_ru(a, q.d[1]); }
  static __device__ double out(T a) { return a; }
};
struct OpFfma {
  using T = float;
  static __device__ T init(const Params& q, int j) { return q.f[0] + j * 1e-3f + threadIdx.x * 1e-7f; }
  static __device__ T step(const Params& q, T a) { return fmaf(a, q.f[1], q.f[2]); }
  static __device__ double out(T a) { return a; }
};
struct OpF32cMad {  // the compensated multiply-add in its general form
  using T = float2;
  static __device__ T init(const Params& q, int j) { return make_float2(q.f[0] + j * 1e-3f + threadIdx.x * 1e-7f, 0.0f); }
  static __device__ T step(const Params& q, T a) {
    return F32C::mad(a, make_float2(q.f[1], q.f[3]), make_float2(q.f[2], q.f[3]));
  }
  static __device__ double out(T a) { return (double)a.x + a.y; }
};
struct OpF32cHorner {  // Horner's step: coefficient added, x a loaded FP32 point
  using T = float2;
  static __device__ T init(const Params& q, int j) { return make_float2(q.f[0] + j * 1e-3f + threadIdx.x * 1e-7f, 0.0f); }
  static __device__ T step(const Params& q, T a) {
    return F32C::mad_k<false, true, true>(a, make_float2(q.f[1], 0.0f), make_float2(q.f[2], 0.0f));
  }
  static __device__ double out(T a) { return (double)a.x + a.y; }
};
// one radix-2 butterfly mod p per step, on a pair: (a, b) -> (a + w b, a - w b)
// (the transforms' arithmetic: MODP::reduce, MODP::add, MODP::sub)
struct ModpPair {
  uint64_t a, b;
};
struct OpModpButterfly {
  using T = ModpPair;
  static __device__ T init(const Params& q, int j) { return ModpPair{q.u[0] + j + threadIdx.x, q.u[0] + 7 * j}; }
  static __device__ T step(const Params& q, T v) {
    const uint64_t t = MODP::reduce(v.b * q.u[1], __umul64hi(v.b, q.u[1]));
    return ModpPair{MODP::add(v.a, t), MODP::sub(v.a, t)};
  }
  static __device__ double out(T v) { return (double)(v.a ^ v.b); }
};

struct OpModpMulAdd {
  using T = uint64_t;
  static __device__ T init(const Params& q, int j) { return q.u[0] + j + threadIdx.x; }
  static __device__ T step(const Params& q, T a) { return MODP::mul_add(a, q.u[1], q.u[0]); }
  static __device__ double out(T a) { return (double)a; }
};
struct OpImad {
  using T = uint32_t;
  static __device__ T init(const Params& q, int j) { return q.w[0] + j + threadIdx.x; }
  static __device__ T step(const Params& q, T a) { return a * q.w[0] + q.w[1]; }
  static __device__ double out(T a) { return (double)a; }
};
struct OpImadWide {  // the low half of the previous value times a 32-bit word, plus a 64-bit addend
  using T = uint64_t;
  static __device__ T init(const Params& q, int j) { return q.u[0] + j + threadIdx.x; }
  static __device__ T step(const Params& q, T a) { return (uint64_t)(uint32_t)a * q.w[0] + q.u[1]; }
  static __device__ double out(T a) { return (double)a; }
};

template <class Op>
__global__ void __launch_bounds__(kThreads) k_rate(const Params* prm, double* out, int iters) {
  const Params q = *prm;
  typename Op::T a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = Op::init(q, j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = Op::step(q, a[j]);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += Op::out(a[j]);
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// G chain steps per second: one warm-up launch, then `reps` timed launches
template <class Op>
int time_rate(const Params* prm, double* out, int blocks, int iters, cudaStream_t st, double& gops) {
  const int reps = 3;
  k_rate<Op><<<blocks, kThreads, 0, st>>>(prm, out, iters);
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return FP_E_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return FP_E_CUDA; }
  cudaEventRecord(a, st);
  for (int r = 0; r < reps; ++r) k_rate<Op><<<blocks, kThreads, 0, st>>>(prm, out, iters);
  cudaEventRecord(b, st);
  const cudaError_t e = cudaEventSynchronize(b);
  float ms = 0;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess || ms <= 0) return FP_E_CUDA;
  gops = (double)blocks * kThreads * kChains * iters * reps / (ms * 1e-3) / 1e9;
  return FP_OK;
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" int fp_measure_rates(double* rates, int nrates, void* stream) {
  if (!rates || nrates < 0) return FP_E_BAD_VALUE;
  if (nrates > FP_RATE_COUNT) nrates = FP_RATE_COUNT;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return FP_E_CUDA;
  }
  const int blocks = sms * kBlocksPerSm;
  double* out = nullptr;
  Params* prm = nullptr;
  if (cudaMalloc((void**)&out, (size_t)blocks * kThreads * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&prm, sizeof(Params)) != cudaSuccess) {
    cudaGetLastError();
    if (out) cudaFree(out);
    return FP_E_NOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Params h{};
  h.d[0] = 0.5; h.d[1] = 0.999999; h.d[2] = 1e-7; h.d[3] = 1e-12;
  h.f[0] = 0.5f; h.f[1] = 0.9999f; h.f[2] = 1e-4f; h.f[3] = 1e-9f;
  h.u[0] = 0x9E3779B97F4A7C15ull % 0xFFFFFFFF00000001ull; h.u[1] = 0x1234567890ABCDEull;
  h.w[0] = 0x9E3779B1u; h.w[1] = 0x7F4A7C15u;
  int rc = cudaMemcpy(prm, &h, sizeof(Params), cudaMemcpyHostToDevice) == cudaSuccess ? FP_OK : FP_E_CUDA;
  for (int i = 0; i < nrates && rc == FP_OK; ++i) {
    double g = 0;
    switch (i) {
      case FP_RATE_DFMA: rc = time_rate<OpDfma>(prm, out, blocks, 2048, st, g); break;
      case FP_RATE_DADD_RD: rc = time_rate<OpDaddRd>(prm, out, blocks, 2048, st, g); break;
      case FP_RATE_DMUL_RU: rc = time_rate<OpDmulRu>(prm, out, blocks, 2048, st, g); break;
      case FP_RATE_FFMA: rc = time_rate<OpFfma>(prm, out, blocks, 65536, st, g); break;
      case FP_RATE_F32C_MAD: rc = time_rate<OpF32cMad>(prm, out, blocks, 8192, st, g); break;
      case FP_RATE_F32C_HORNER: rc = time_rate<OpF32cHorner>(prm, out, blocks, 8192, st, g); break;
      case FP_RATE_MODP_MULADD: rc = time_rate<OpModpMulAdd>(prm, out, blocks, 2048, st, g); break;
      case FP_RATE_MODP_BUTTERFLY: rc = time_rate<OpModpButterfly>(prm, out, blocks, 2048, st, g); break;
      case FP_RATE_IMAD: rc = time_rate<OpImad>(prm, out, blocks, 16384, st, g); break;
      case FP_RATE_IMAD_WIDE: rc = time_rate<OpImadWide>(prm, out, blocks, 16384, st, g); break;
      default: break;
    }
    rates[i] = g;
  }
  cudaFree(out);
  cudaFree(prm);
  return rc;
}
