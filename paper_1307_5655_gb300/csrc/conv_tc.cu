// FP64 polynomial products on the tensor cores: the products (S + c) q^d of
// the composition walk (Sec. 2.1 over polynomial values, Sec. 1.2), batched
// over pairs, as split-precision bf16 matrix products (tcgen05, TMEM) with an
// exact integer recombination.
//
// Blocks.  Both operands are cut into blocks of T = 64 coefficients; block u
// of a has the exponent bound alpha_u (every |a_i| < 2^alpha_u), and the
// window of b that output block w meets at step v -- b[64 v - 63 .. 64 v + 63]
// -- has the bound beta_v.  Output block w (coefficients 64 w .. 64 w + 63) is
//     out[64 w + r] = sum_v sum_s a[64 (w - v) + s] b[64 v + r - s],
// so for every v one matrix product D[w][r] = sum_s A[w - v][s] B_v[r][s]
// with A the blocks of a as rows (a window of rows shifted by one per step)
// and B_v the 64 x 64 Toeplitz matrix of the window.  With the block stored
// reversed (k = 63 - s) the second operand is b[64 v - 63 + r + k], a Hankel
// matrix: its 8-element core rows are 16-byte lines W[8 m + rho .. + 7] of
// the window W = b[64 v - 63 ..], m = row group + column group, rho = row in
// the group.  Eight copies of the window, shifted by rho elements and
// interleaved line by line (line m * 8 + rho), are therefore that operand as
// it stands: a K-major descriptor with both core-matrix strides 128 bytes
// reads it (2 KB per slice instead of an 8 KB Toeplitz tile), and the next
// step's copies are built while the tensor cores run this step's.
//
// Slices.  x in a block of bound 2^alpha is rounded to the integer
// X = round(x 2^(6 - alpha + 7 (S - 1))) (|X| <= 2^(7 S - 1)) and written in
// S signed base-128 digits d_0 (most significant, |d_0| <= 64) .. d_{S-1}
// (in [-64, 63]); slice i holds d_i 2^(-7 i) as a bf16 (exact).  The product
// of slices i (of a) and j (of b) is d d' 2^(-7 (i + j)); the pairs with
// i + j <= S - 1 are kept (the dropped ones are below 2^(-7 S) of the block
// products).  Accumulator g (g = i + j = 0..3) sums one group exactly: over
// K = 64 its integer value D_g = sum d d' has |D_g| <= 4 * 64^3 < 2^22 and
// FP32 holds it without rounding.  The groups g >= 4 are summed with FP32
// rounding far below the recombination's resolution, in two accumulators
// (the pairs with i even and odd: two parts of a step that two threads can
// issue side by side).
//
// Recombination.  Each step reads the six accumulators (tcgen05.ld), turns
// each into its integer with one FMA against 1.5 2^23 (exact for |D| < 2^22),
// and forms C = D_0 2^28 + D_1 2^21 + D_2 2^14 + D_3 2^7 (|C| < 2^47) and
// D_4 (the two combined accumulators' integers, each rounded to the unit):
// the step contributes (C + D_4) 2^(alpha_{w-v} + beta_v - 40), rounded to
// the row's unit once.  TMEM holds the four exact accumulators once and the
// combined pair twice (512 columns): step v + 1's combined group is queued
// before step v is read out, and the tensor cores run it during that
// readout; its exact groups follow once step v is read.  Each output row
// keeps a 64-bit fixed-point accumulator with unit 2^F_w, F_w = max over the
// row's steps of alpha + beta - 40 - (15 - hr), hr the bits of the row's step
// count: every contribution stays below 2^(62 - hr) units and their sum
// below 2^62; smaller contributions are rounded to the unit.  No FP64
// arithmetic runs per step (GB300's FP64 rate is 1/64 of its FP32 rate).  The
// result is (double) acc 2^F_w.
//
// Error: |result - a * b|_j <= (S + 2) 2^(-7 S) sum_s 2^(alpha + beta) (the
// slices and dropped pairs, per block product) plus 2^F_w per step (the
// fixed-point rounding) plus one rounding to double: about 2^-52 (S = 8) of
// the largest block products that meet at coefficient j.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/fastpoly.h"

namespace fp {
namespace tc {

constexpr int T = 64;                // coefficients per block: N and K of one step
constexpr int V = 32;                // steps per load of the A window
constexpr int MROWS = 128;           // output blocks per tile (MMA M, TMEM lanes)
constexpr int WROWS = MROWS + V;     // rows of the A window in shared memory
constexpr int STRIP = WROWS * 16;    // bytes of one (slice, 8-column chunk) strip of A
constexpr int HANKEL = 16 * 8 * 16;  // bytes of one slice's shifted window copies (16 lines x 8 shifts)
constexpr int NACC = 5;              // accumulator groups: exact g = 0..3, combined g >= 4
constexpr int NCOMB = 2;             // TMEM accumulators of the combined group
constexpr int READERS = 256;         // warps 0-7 read the accumulators out and build the operands
constexpr int THREADS = READERS + 32;  // warp 8 issues the MMAs
constexpr int ZERO_EXP = -100000;    // exponent bound of an all-zero block
constexpr int TMEM_COLS = 512;       // exact groups 4 x 64, combined group 2 buffers x NCOMB x 64
constexpr int SMEM_MIN = 120 * 1024; // at least half the SM: one tile per SM holds the TMEM

__host__ __device__ constexpr int smem_bytes(int S) { return S * 8 * STRIP + 2 * S * HANKEL + 2 * S * 256; }

// ------------------------------------------------------------------ slicing
// smallest alpha with |x| < 2^alpha (ZERO_EXP for x = 0)
__device__ __forceinline__ int exp_bound(double x) {
  const long long b = __double_as_longlong(x);
  if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) return ZERO_EXP;
  const int e = (int)((b >> 52) & 0x7FF);
  return e == 0 ? -1022 : e - 1022;
}

// X = round(x 2^(6 - alpha + 7 (S - 1))) from the bits of x (|x| < 2^alpha)
template <int S>
__device__ __forceinline__ long long to_fixed(double x, int alpha) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  long long m = b & 0xFFFFFFFFFFFFFll;
  if (e) m |= 1ll << 52;
  const int sh = (e ? e : 1) - 1075 + 6 - alpha + 7 * (S - 1);  // |x| = m 2^(max(e,1) - 1075)
  long long X;
  if (sh >= 0) X = m << sh;  // then m 2^sh < 2^(7 S - 1)
  else if (sh > -64) X = (m + (1ll << (-sh - 1))) >> (-sh);
  else X = 0;
  return b < 0 ? -X : X;
}

// the bf16 bit pattern of d 2^(-7 i) (exact: |d| <= 64)
__device__ __forceinline__ uint32_t bf16_digit(int d, int i) {
  const float f = __int2float_rn(d) * __int_as_float((127 - 7 * i) << 23);
  return __float_as_uint(f) >> 16;
}

// 8 consecutive values of one block row -> S 16-byte chunks (one per slice)
template <int S>
__device__ __forceinline__ void slice8(const double* x, int alpha, uint4* chunk) {
  uint32_t w[S][4];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    long long X = alpha == ZERO_EXP ? 0 : to_fixed<S>(x[e], alpha);
    int d[S];
#pragma unroll
    for (int i = S - 1; i > 0; --i) {
      const int r = (int)((X + 64) & 127) - 64;
      d[i] = r;
      X = (X - r) >> 7;
    }
    d[0] = (int)X;
#pragma unroll
    for (int i = 0; i < S; ++i) {
      const uint32_t h = bf16_digit(d[i], i);
      if (e & 1) w[i][e >> 1] |= h << 16;
      else w[i][e >> 1] = h;
    }
  }
#pragma unroll
  for (int i = 0; i < S; ++i) chunk[i] = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}

// Blocks of a as rows, each reversed: ahat[pair][slice][chunk][u] (16 bytes:
// coefficients 64 u + 63 - 8 chunk down to 64 u + 56 - 8 chunk), alpha[pair][u].
// Eight threads per block row.
template <int S>
__global__ void k_slice_rows(const double* a, int64_t a_pitch, int alen, int nA, int64_t npairs, uint4* ahat,
                             int* alpha) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = gid >> 3;
  const int t = (int)(gid & 7);
  const bool valid = row < npairs * nA;
  const int64_t pr = valid ? row / nA : 0;
  const int u = valid ? (int)(row - pr * nA) : 0;
  double x[8];
  int al = ZERO_EXP;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int idx = 64 * u + 8 * t + e;
    x[e] = (valid && idx < alen) ? a[pr * a_pitch + idx] : 0.0;
    al = max(al, exp_bound(x[e]));
  }
  al = max(al, __shfl_xor_sync(0xffffffffu, al, 1));
  al = max(al, __shfl_xor_sync(0xffffffffu, al, 2));
  al = max(al, __shfl_xor_sync(0xffffffffu, al, 4));
  if (!valid) return;
  double xr[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) xr[e] = x[7 - e];
  uint4 ch[S];
  slice8<S>(xr, al, ch);
#pragma unroll
  for (int i = 0; i < S; ++i) ahat[((pr * S + i) * 8 + (7 - t)) * nA + u] = ch[i];
  if (t == 0) alpha[pr * nA + u] = al;
}

// Windows of b: rhat[pair][v][slice][t] (bf16) holds b[64 v - 63 + t] for
// t < 127 (0 at t = 127 and outside b), beta[pair][v].  Sixteen threads per
// window, eight entries each.
template <int S>
__global__ void k_slice_windows(const double* b, int64_t b_pitch, int blen, int nV, int64_t npairs, uint4* rhat,
                                int* beta) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t win = gid >> 4;
  const int m = (int)(gid & 15);
  const bool valid = win < npairs * nV;
  const int64_t pr = valid ? win / nV : 0;
  const int v = valid ? (int)(win - pr * nV) : 0;
  double x[8];
  int be = ZERO_EXP;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int tp = 8 * m + e;
    const int idx = 64 * v - 63 + tp;
    x[e] = (valid && tp < 127 && idx >= 0 && idx < blen) ? b[pr * b_pitch + idx] : 0.0;
    be = max(be, exp_bound(x[e]));
  }
  be = max(be, __shfl_xor_sync(0xffffffffu, be, 1));
  be = max(be, __shfl_xor_sync(0xffffffffu, be, 2));
  be = max(be, __shfl_xor_sync(0xffffffffu, be, 4));
  be = max(be, __shfl_xor_sync(0xffffffffu, be, 8));
  if (!valid) return;
  uint4 ch[S];
  slice8<S>(x, be, ch);
#pragma unroll
  for (int i = 0; i < S; ++i) rhat[((pr * nV + v) * S + i) * 16 + m] = ch[i];
  if (m == 0) beta[pr * nV + v] = be;
}

// ------------------------------------------------------------------ tcgen05
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, K-major, no swizzle: core matrices of 8
// rows x 16 bytes; lbo = bytes between core matrices along K, sbo = along M/N
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | (uint64_t)((lbo >> 4) & 0x3FFF) << 16 |
         (uint64_t)((sbo >> 4) & 0x3FFF) << 32 | 1ull << 46;
}

// instruction descriptor: bf16 x bf16 -> f32, both K-major, M = 128, N = 64
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(T >> 3) << 17) | ((uint32_t)(MROWS >> 4) << 24);

// COL: what the MMA does with the A collector buffer -- 0 read A from shared
// memory and discard it, 1 read and keep it (fill), 2 reuse the kept A (use),
// 3 reuse it for the last time (lastuse)
template <int COL>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  if constexpr (COL == 0)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
  else if constexpr (COL == 1)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
  else if constexpr (COL == 2)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
  else
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

// The MMAs of one step: PASS 0 the exact groups (i + j < NACC - 1, into
// accumulator i + j at column 64 (i + j) of tmem), PASS 1 and 2 the combined
// group's pairs with i even / odd (into the one accumulator at tmem): slice i
// of the A window times slice j of B_v over K = 64 (four MMAs of K = 16).
// Each accumulator gets its MMAs from one pass, in order (deterministic
// sums), and the first MMA into it overwrites it.  The start-address field of a descriptor holds addr >> 4 (14
// bits, shared memory < 256 KB): adding offset >> 4 moves it.
template <int S, int PASS, int I, int KS, int J>
__device__ __forceinline__ void issue_j(uint32_t tmem, uint64_t dA, uint64_t dB, uint32_t& used) {
  if constexpr (J < S) {
    constexpr bool exact = I + J < NACC - 1;
    constexpr bool keep = I + J <= S - 1 && (PASS == 0 ? exact : (!exact && (I & 1) == PASS - 1));
    if constexpr (keep) {
      constexpr int g = PASS == 0 ? I + J : 0;
      mma<0>(tmem + (uint32_t)(g * T), dA + (uint64_t)(((I * 8 + 2 * KS) * STRIP) >> 4),
             dB + (uint64_t)((J * HANKEL + 2 * KS * 128) >> 4), (used >> g) & 1u);
      used |= 1u << g;
    }
    issue_j<S, PASS, I, KS, J + 1>(tmem, dA, dB, used);
  }
}

template <int S, int PASS, int I, int KS>
__device__ __forceinline__ void issue_iks(uint32_t tmem, uint64_t dA, uint64_t dB, uint32_t& used) {
  if constexpr (I < S) {
    if constexpr (KS < T / 16) {
      issue_j<S, PASS, I, KS, 0>(tmem, dA, dB, used);
      issue_iks<S, PASS, I, KS + 1>(tmem, dA, dB, used);
    } else {
      issue_iks<S, PASS, I + 1, 0>(tmem, dA, dB, used);
    }
  }
}

template <int S, int PASS>
__device__ __forceinline__ void issue_mmas(uint32_t tmem, uint64_t dA, uint64_t dB) {
  uint32_t used = 0;
  issue_iks<S, PASS, 0, 0>(tmem, dA, dB, used);
}

// eight consecutive columns of the warp's 32 TMEM lanes (one lane per thread)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// the reader warps' barrier (named barrier 1; the issuing warp takes no part)
__device__ __forceinline__ void readers_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(READERS) : "memory"); }

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\tselp.b32 %0, 1, 0, P1;\n\t}\n"
      : "=r"(done)
      : "r"(bar), "r"(phase));
  return done != 0;
}

// bounded wait for an mbarrier phase (false: gave up)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try(bar, phase)) return true;
  return false;
}

// One tile: output blocks w0 .. w0 + 127 of one pair, all 64 coefficients.
// Warps 0-7 (the readers) read the accumulators out -- warp i reads TMEM
// lanes 32 (i & 3) .. + 31 and columns 32 (i >> 2) .. + 31 of each
// accumulator: one output block and 32 of its coefficients per thread -- and
// build the operands; lane 0 of warp 8 issues the MMAs.  tcgen05.mma holds
// its thread while the tensor cores' queue is full, so a thread that issued
// and also read out would leave the tensor cores idle during its readout.
//
// Steps k = 0 .. v_hi - v_lo (v = v_lo + k).  The readers read a step's
// exact and combined groups together (one rounding shift per coefficient);
// the issuer queues step k + 1's combined group (its buffer alternates) ahead
// of its exact groups, so the tensor cores run it during step k's readout.
// Barriers (b = parity of the step they concern):
//   full_x     step k's exact groups are in TMEM (commit; phase k)
//   full_y(b)  step k's combined group (commit; phase k >> 1)
//   ops(b)     step k's operands are in shared memory (the readers; the
//              (k >> 1)-th phase of ops(k & 1) for k >= 1 -- step 0 is
//              covered by the prologue's __syncthreads): signalled after
//              step k - 2's readout, when its Hankel operand is built, or
//              after step k - 1's when the A window is reloaded for step k
//   free(b)    step k is read out (the readers; phase k >> 1): step k + 1's
//              exact groups and step k + 2's combined group may overwrite
// Each barrier's next phase needs an MMA that is issued only after its
// waiter passed the current one, so no wait is ever more than one phase
// behind and the parity of the awaited phase identifies it.
template <int S>
__global__ void __launch_bounds__(THREADS, 1)
    k_conv_tc(const uint4* __restrict__ ahat, const int* __restrict__ alpha, int nA, const uint4* __restrict__ rhat,
              const int* __restrict__ beta, int nV, int nW, int rl, int mtiles, double* out, int64_t out_pitch,
              int mode, const double* init, int64_t init_pitch, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[7];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail[3];  // a reader's wait of iteration k gave up (slot k & 1); the issuer's (slot 2)
  unsigned char* sA = smem;                                // A window: S x 8 strips
  unsigned char* sH = smem + S * 8 * STRIP;                // Hankel operand: 2 buffers x S slices
  uint32_t* sW = (uint32_t*)(sH + 2 * S * HANKEL);         // staged windows: 2 buffers x S x 64 words
  const int64_t pr = blockIdx.x / mtiles;
  const int w0 = (int)(blockIdx.x % mtiles) * MROWS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool reader = threadIdx.x < READERS;
  const int q = warp & 3, h = (warp >> 2) & 1;  // TMEM lane quadrant, column half
  const int w = w0 + 32 * q + lane;             // a reader's output block
  const int* al = alpha + pr * nA;
  const int* be = beta + pr * nV;
  const int v_lo = max(0, w0 - nA + 1);
  const int v_hi = min(nV - 1, w0 + MROWS - 1);
  const int nsteps = v_hi - v_lo + 1;  // may be <= 0
  // the row's fixed-point unit 2^F: with n steps meeting the row (hr bits),
  // every contribution |C| 2^E < 2^(47 + 15 - hr) and their sum < 2^62
  int mx = 2 * ZERO_EXP;
  const int v_first = max(0, w - nA + 1), v_last = min(nV - 1, w);
  if (reader && w < nW)
    for (int v = v_first; v <= v_last; ++v) mx = max(mx, __ldg(al + w - v) + __ldg(be + v));
  const int hr = 32 - __clz(max(1, v_last - v_first + 1));
  const int P = 15 - hr;  // C is pre-shifted by P: E <= P
  const int F = mx - 40 - P;
  long long acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = 0;

  const uint32_t full_x = smem_u32(&bar[0]);
  auto full_y = [&](int b) { return smem_u32(&bar[1 + b]); };
  auto ops = [&](int b) { return smem_u32(&bar[3 + b]); };
  auto freed = [&](int b) { return smem_u32(&bar[5 + b]); };
  // the phase of ops(k & 1) that step k's operands complete (k >= 1)
  auto ops_phase = [](int k) { return ((k - 2 + (k & 1)) >> 1) & 1; };
  // step k's A window is loaded after step k - 1's readout (every V steps)
  auto reload = [](int k) { return k > 0 && k % V == 0; };
  if (threadIdx.x == 0) {
    s_fail[0] = s_fail[1] = s_fail[2] = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(full_x), "r"(1));
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(full_y(b)), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(ops(b)), "r"(READERS));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(freed(b)), "r"(READERS));
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // W_v of every slice into staging buffer sb (readers)
  auto stage_window = [&](int v, int sb) {
    if (threadIdx.x < S * 16)
      ((uint4*)(sW + sb * S * 64))[threadIdx.x] = __ldg(rhat + (pr * nV + v) * (S * 16) + threadIdx.x);
  };
  // the shifted copies of staging buffer sb into Hankel buffer hb: line
  // m * 8 + rho of slice j holds W_j[8 m + rho .. + 7] (m < 15: the MMAs read
  // row group + column group <= 14); lines in order, so eight threads store
  // 128 consecutive bytes
  auto build_hankel = [&](int hb, int sb) {
    unsigned char* base = sH + hb * (S * HANKEL);
    const uint32_t* wsrc = sW + sb * S * 64;
    for (int e = threadIdx.x; e < S * 120; e += READERS) {
      const int j = e / 120, line = e - j * 120, m = line >> 3, rho = line & 7;
      const uint32_t* src = wsrc + j * 64 + 4 * m + (rho >> 1);
      const uint32_t sft = 16u * (rho & 1);
      const uint32_t x0 = src[0], x1 = src[1], x2 = src[2], x3 = src[3], x4 = src[4];
      *(uint4*)(base + j * HANKEL + line * 16) = make_uint4(__funnelshift_r(x0, x1, sft), __funnelshift_r(x1, x2, sft),
                                                            __funnelshift_r(x2, x3, sft), __funnelshift_r(x3, x4, sft));
    }
  };
  // A window for the chunk of steps starting at v: block rows ub .. ub +
  // WROWS - 1 (zero outside a), every slice and chunk; step v' reads rows
  // w0 - v' .. w0 - v' + 127
  auto load_window = [&](int v) {
    const int ub = w0 - v - (V - 1);
    for (int e = threadIdx.x; e < S * 8 * WROWS; e += READERS) {
      const int sk = e / WROWS, r = e - sk * WROWS;
      const int u = ub + r;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (u >= 0 && u < nA) val = __ldg(ahat + (pr * (S * 8) + sk) * (int64_t)nA + u);
      *(uint4*)(sA + sk * STRIP + r * 16) = val;
    }
  };

  // Prologue (readers): the operands of steps 0 and 1.
  if (reader && nsteps > 0) {
    stage_window(v_lo, 0);
    if (nsteps > 1) stage_window(v_lo + 1, 1);
    load_window(v_lo);
  }
  if (reader) readers_sync();
  if (reader && nsteps > 0) {
    build_hankel(0, 0);
    if (nsteps > 1) build_hankel(1, 1);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (reader && nsteps > 1) mbar_arrive(ops(1));  // step 1's operands (its Hankel, window 0)

  if (!reader) {
    // The issuer.  Step k: slice i of the A window (row of block w0 - v at
    // window row V - 1 - k % V) times slice j of Hankel buffer k & 1; the
    // combined group's halves into columns 256 + 128 (k & 1) + 0 / 64 (after
    // step k - 2's readout), then the exact groups into columns 0 .. 255
    // (after step k - 1's).
    if (lane == 0) {
      int kx = -1, ky = -1;  // the last steps whose exact / combined groups were issued
      for (int k = 0; k < nsteps; ++k) {
        if (k >= 1 && !mbar_wait(ops(k & 1), ops_phase(k))) break;
        if (k >= 2 && !mbar_wait(freed(k & 1), ((k - 2) >> 1) & 1)) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int roff = (V - 1) - k % V;
        const uint64_t dA = sdesc(smem_u32(sA) + 16u * roff, STRIP, 128);
        const uint64_t dB = sdesc(smem_u32(sH) + (uint32_t)((k & 1) * S * HANKEL), 128, 128);
        const uint32_t tc = tmem + (uint32_t)((NACC - 1) * T + NCOMB * T * (k & 1));
        issue_mmas<S, 1>(tc, dA, dB);
        issue_mmas<S, 2>(tc + T, dA, dB);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(full_y(k & 1)));
        ky = k;
        if (k >= 1 && !mbar_wait(freed((k - 1) & 1), ((k - 1) >> 1) & 1)) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        issue_mmas<S, 0>(tmem, dA, dB);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(full_x));
        kx = k;
      }
      if (kx != nsteps - 1) {
        s_fail[2] = 1;
        // the MMAs in flight (the last commit to each barrier), bounded
        if (kx >= 0) mbar_wait(full_x, kx & 1);
        if (ky >= 0) mbar_wait(full_y(ky & 1), (ky >> 1) & 1);
        if (ky >= 1) mbar_wait(full_y((ky - 1) & 1), ((ky - 1) >> 1) & 1);
      }
    }
    __syncwarp();
  } else {
    for (int k = 0; k < nsteps; ++k) {
      const int v = v_lo + k;
      // this row's step: (C + D) 2^E units of 2^F, E = alpha + beta - 40 - F <= P
      const int u = w - v;
      const int E = (w < nW && u >= 0 && u < nA) ? __ldg(al + u) + __ldg(be + v) - 40 - F : -1000;
      const int sh = min(63, P - E);
      const long long rnd = sh > 0 ? 1ll << (sh - 1) : 0;
      if (!mbar_wait(full_y(k & 1), (k >> 1) & 1)) s_fail[k & 1] = 1;
      if (!mbar_wait(full_x, k & 1)) s_fail[k & 1] = 1;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int qc = 0; qc < 4; ++qc) {
        uint32_t r[NACC - 1 + NCOMB][8];
#pragma unroll
        for (int g = 0; g < NACC - 1; ++g)
          tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(g * T + 32 * h + 8 * qc), r[g]);
#pragma unroll
        for (int kk = 0; kk < NCOMB; ++kk)
          tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) +
                       (uint32_t)((NACC - 1) * T + NCOMB * T * (k & 1) + T * kk + 32 * h + 8 * qc),
                   r[NACC - 1 + kk]);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          int d[NACC - 1];
#pragma unroll
          for (int g = 0; g < NACC - 1; ++g)
            d[g] = __float_as_int(fmaf(__uint_as_float(r[g][c]), __int_as_float((127 + 7 * g) << 23), 12582912.0f)) -
                   0x4B400000;
          int dc = 0;
#pragma unroll
          for (int kk = 0; kk < NCOMB; ++kk)
            dc += __float_as_int(fmaf(__uint_as_float(r[NACC - 1 + kk][c]),
                                      __int_as_float((127 + 7 * (NACC - 1)) << 23), 12582912.0f)) -
                  0x4B400000;
          const long long C = (long long)d[0] * (1ll << 28) + (long long)d[1] * (1ll << 21) +
                              (long long)d[2] * (1ll << 14) + (long long)d[3] * 128 + dc;
          acc[8 * qc + c] += ((C << P) + rnd) >> sh;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      mbar_arrive(freed(k & 1));
      if (k + 1 < nsteps && reload(k + 1)) {
        // the next chunk's window: every MMA reading the current one is done
        load_window(v + 1);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive(ops((k + 1) & 1));
      }
      if (k + 2 < nsteps) stage_window(v + 2, k & 1);
      readers_sync();
      // (a reader past this check may set the next iteration's slot before a
      // slower one reads this one: separate slots keep the decision uniform)
      if (s_fail[k & 1]) break;
      if (k + 2 < nsteps) {
        // step k + 2's Hankel operand into buffer k & 1: step k's MMAs are done
        build_hankel(k & 1, k & 1);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (!reload(k + 2)) mbar_arrive(ops(k & 1));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  const bool failed = s_fail[0] | s_fail[1] | s_fail[2];
  if (failed) {
    if (threadIdx.x == 0) atomicExch(status, 1);
  } else if (reader && w < nW) {
    double* o = out + pr * out_pitch;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const int j = 64 * w + 32 * h + c;
      if (j < rl) {
        double val = ldexp((double)acc[c], F);
        if (mode == 1) val += o[j];
        else if (mode == 2 && j == 0) val += init[pr * init_pitch];
        o[j] = val;
      }
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct Dims {
  int nA, nV, nW;
};
inline Dims dims(int alen, int blen) {
  Dims d;
  d.nA = (int)ceil_div(alen, T);
  d.nV = (blen + 62) / T + 1;
  d.nW = (int)ceil_div((int64_t)alen + blen - 1, T);
  return d;
}
inline size_t r256(size_t b) { return (b + 255) & ~(size_t)255; }

template <int S>
int launch(const double* a, int64_t a_pitch, int alen, const double* b, int64_t b_pitch, int blen, double* out,
           int64_t out_pitch, int mode, const double* init, int64_t init_pitch, int64_t npairs, void* work,
           int* status, cudaStream_t st) {
  const Dims d = dims(alen, blen);
  unsigned char* p = (unsigned char*)work;
  uint4* ahat = (uint4*)p;
  p += r256((size_t)npairs * S * 8 * d.nA * 16);
  int* alpha = (int*)p;
  p += r256((size_t)npairs * d.nA * 4);
  uint4* rhat = (uint4*)p;
  p += r256((size_t)npairs * d.nV * S * 256);
  int* beta = (int*)p;
  const int64_t rows = npairs * d.nA, wins = npairs * d.nV;
  k_slice_rows<S><<<(unsigned)ceil_div(rows * 8, 256), 256, 0, st>>>(a, a_pitch, alen, d.nA, npairs, ahat, alpha);
  k_slice_windows<S><<<(unsigned)ceil_div(wins * 16, 256), 256, 0, st>>>(b, b_pitch, blen, d.nV, npairs, rhat, beta);
  const int smem = smem_bytes(S) > SMEM_MIN ? smem_bytes(S) : SMEM_MIN;
  if (cudaFuncSetAttribute(k_conv_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return FP_E_CUDA;
  const int mtiles = (int)ceil_div(d.nW, MROWS);
  k_conv_tc<S><<<(unsigned)(npairs * mtiles), THREADS, smem, st>>>(ahat, alpha, d.nA, rhat, beta, d.nV, d.nW,
                                                                  alen + blen - 1, mtiles, out, out_pitch, mode,
                                                                  init, init_pitch, status);
  return cudaGetLastError() == cudaSuccess ? FP_OK : FP_E_CUDA;
}

}  // namespace tc

// Work space of conv_tc for these lengths (bytes, 256-byte granules).
size_t conv_tc_workspace(int alen, int blen, int64_t npairs, int slices) {
  const tc::Dims d = tc::dims(alen, blen);
  return tc::r256((size_t)npairs * slices * 8 * d.nA * 16) + tc::r256((size_t)npairs * d.nA * 4) +
         tc::r256((size_t)npairs * d.nV * slices * 256) + tc::r256((size_t)npairs * d.nV * 4);
}

// out[pair][0 .. alen + blen - 1) = a[pair] * b[pair] (mode 0), added into out
// (mode 1), or written with init[pair] added at degree 0 (mode 2); `out` may
// be `a` or `b` (both are sliced before the product is written).  status: a
// device int set to 1 if a tile gave up waiting for its tensor-core work.
int conv_tc(const double* a, int64_t a_pitch, int alen, const double* b, int64_t b_pitch, int blen, double* out,
            int64_t out_pitch, int mode, const double* init, int64_t init_pitch, int64_t npairs, void* work,
            int* status, int slices, cudaStream_t st) {
  if (alen < 1 || blen < 1 || npairs < 1) return FP_E_BAD_VALUE;
  switch (slices) {
    case 6: return tc::launch<6>(a, a_pitch, alen, b, b_pitch, blen, out, out_pitch, mode, init, init_pitch, npairs, work, status, st);
    case 7: return tc::launch<7>(a, a_pitch, alen, b, b_pitch, blen, out, out_pitch, mode, init, init_pitch, npairs, work, status, st);
    case 8: return tc::launch<8>(a, a_pitch, alen, b, b_pitch, blen, out, out_pitch, mode, init, init_pitch, npairs, work, status, st);
  }
  return FP_E_BAD_VALUE;
}

}  // namespace fp
