// Per-point replay of a compiled evaluation tree (the coefficient walk of
// Moroz, Sec. 2.1, with the precomputed powers of Sec. 2.2) on sm_103a.
//
// Parallelisation: points are independent; each thread owns PPT points
// (point index = block base + p * TPB + thread).  The schedule (one control
// word and two coefficients per non-root node) is the same for every point,
// so every lane reads the same address: the loads are warp-uniform and served
// by L1 after the first warp of the SM.  Each thread keeps its accumulators
// m[0..L] and its power table x_v^d in its own column of shared memory
// (stride TPB, conflict-free), so no barrier is ever needed and warps run
// independently.
//
// Accumulator update per non-root node N with parent P, in node index order:
//   fused types (FP64, FP32C, MODP):
//     s   = c_N                 if N is a leaf, else m[lh(N)]
//     init= c_P                 if N is P's first child, else m[lh(P)]
//     m[lh(P)] = s * x^d(N) + init
//   i.e. the coefficient of P is folded in when P's first child arrives, so
//   each node costs one multiply-add (the paper's step adds c_N to the
//   children's sum and then multiplies; the result is the same polynomial).
//   IV64 keeps the paper's order literally (see the interval policy).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tree.hpp"

namespace fp {

constexpr int kTPB = 128;

struct EvalArgs {
  const uint32_t* ctrl;
  const void* ca;
  const void* cb;
  const uint32_t* pow_prog;
  const uint2* pow_dv;  // per power slot: (variable, degree)
  int64_t nsteps;   // non-root nodes
  int npow;
  int nslot;        // max lazy height + 1
  int nvars;
  int root_leaf;
  int root_lh;
  int root_pid;
  uint64_t root_c;  // raw bits of the root coefficient in the type's coefficient format
  const void* points;
  int64_t npts;
  void* out;
};

// ---------------------------------------------------------------- policies
// Each policy defines:
//   coef  coefficient type in the schedule
//   val   accumulator / result value, pw: power-table value
//   load_point(pts, v, idx, npts)   ->  pw  (x_v at point idx)
//   square(a), mulx(a, x)           ->  pw  (power program)
//   node(leaf, first, ca, cb, src*, dst*, xd)   (one schedule step)
//   root(leaf, c, acc*), apply_root_power(r, xd), store(out, idx, npts, r)

struct F64 {
  using coef = double;
  using val = double;
  using pw = double;
  static __device__ __forceinline__ coef coef_from_bits(uint64_t b) { return __longlong_as_double((long long)b); }
  static __device__ __forceinline__ pw load_point(const void* pts, int v, int64_t idx, int64_t npts) {
    return __ldg((const double*)pts + (int64_t)v * npts + idx);
  }
  static __device__ __forceinline__ pw dummy_point() { return 0.5; }
  static __device__ __forceinline__ pw square(pw a) { return __dmul_rn(a, a); }
  static __device__ __forceinline__ pw mulx(pw a, pw x) { return __dmul_rn(a, x); }
  static __device__ __forceinline__ void node(bool leaf, bool first, coef ca, coef cb, const val* src, val* dst, pw xd) {
    const double s = leaf ? ca : *src;
    const double init = first ? cb : *dst;
    *dst = fma(s, xd, init);
  }
  static __device__ __forceinline__ val root(bool leaf, coef c, const val* acc) { return leaf ? c : *acc; }
  static __device__ __forceinline__ val apply_root_power(val r, pw xd) { return __dmul_rn(r, xd); }
  static __device__ __forceinline__ void store(void* out, int64_t idx, int64_t, val r) { ((double*)out)[idx] = r; }
};

// FP32 with error-free transformations (Ogita-Rump-Oishi TwoSum, FMA-based
// TwoProduct; compensated evaluation in the manner of Graillat-Langlois-
// Louvet's compensated Horner).  A value is an unevaluated pair hi + lo where
// lo collects the exact rounding errors of hi's operations (and their
// propagation, to first order).
struct F32C {
  using coef = float;
  using val = float2;
  using pw = float2;
  static __device__ __forceinline__ coef coef_from_bits(uint64_t b) { return __int_as_float((int)(uint32_t)b); }
  static __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }
  static __device__ __forceinline__ float2 renorm(float hi, float lo) {  // |hi| >= |lo|
    const float s = __fadd_rn(hi, lo);
    return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
  }
  static __device__ __forceinline__ pw load_point(const void* pts, int v, int64_t idx, int64_t npts) {
    return make_float2(__ldg((const float*)pts + (int64_t)v * npts + idx), 0.0f);
  }
  static __device__ __forceinline__ pw dummy_point() { return make_float2(0.5f, 0.0f); }
  static __device__ __forceinline__ pw square(pw a) {
    const float p = __fmul_rn(a.x, a.x);
    const float e = __fmaf_rn(a.x, a.x, -p);
    return renorm(p, __fmaf_rn(__fadd_rn(a.x, a.x), a.y, e));
  }
  static __device__ __forceinline__ pw mulx(pw a, pw x) {
    const float p = __fmul_rn(a.x, x.x);
    const float e = __fmaf_rn(a.x, x.x, -p);
    return renorm(p, __fmaf_rn(a.y, x.x, e));
  }
  static __device__ __forceinline__ void node(bool leaf, bool first, coef ca, coef cb, const val* src, val* dst, pw xd) {
    const float2 s = leaf ? make_float2(ca, 0.0f) : *src;
    const float2 init = first ? make_float2(cb, 0.0f) : *dst;
    const float p = __fmul_rn(s.x, xd.x);
    const float pe = __fmaf_rn(s.x, xd.x, -p);
    float h, se;
    two_sum(init.x, p, h, se);
    float lo = __fadd_rn(init.y, __fadd_rn(pe, se));
    lo = __fmaf_rn(s.y, xd.x, lo);
    lo = __fmaf_rn(s.x, xd.y, lo);
    *dst = make_float2(h, lo);
  }
  static __device__ __forceinline__ val root(bool leaf, coef c, const val* acc) { return leaf ? make_float2(c, 0.0f) : *acc; }
  static __device__ __forceinline__ val apply_root_power(val r, pw xd) {
    const float p = __fmul_rn(r.x, xd.x);
    const float pe = __fmaf_rn(r.x, xd.x, -p);
    float lo = __fmaf_rn(r.y, xd.x, pe);
    lo = __fmaf_rn(r.x, xd.y, lo);
    return make_float2(p, lo);
  }
  static __device__ __forceinline__ void store(void* out, int64_t idx, int64_t npts, val r) {
    float s, e;
    two_sum(r.x, r.y, s, e);
    ((float*)out)[idx] = s;
    ((float*)out)[npts + idx] = e;
  }
};

// Integers modulo p = 2^64 - 2^32 + 1.  128-bit products, reduced with
// 2^64 = 2^32 - 1 and 2^96 = -1 (mod p).
struct MODP {
  using coef = uint64_t;
  using val = uint64_t;
  using pw = uint64_t;
  static constexpr uint64_t P = 0xFFFFFFFF00000001ull;
  static __device__ __forceinline__ coef coef_from_bits(uint64_t b) { return b; }
  static __device__ __forceinline__ uint64_t reduce(uint64_t lo, uint64_t hi) {
    const uint64_t hh = hi >> 32, hl = hi & 0xFFFFFFFFull;
    uint64_t t0 = lo - hh;
    if (lo < hh) t0 -= 0xFFFFFFFFull;           // borrow of 2^64 == 2^32 - 1
    const uint64_t t1 = (hl << 32) - hl;        // hl * (2^32 - 1)
    uint64_t r = t0 + t1;
    if (r < t1) r += 0xFFFFFFFFull;             // carry of 2^64
    if (r >= P) r -= P;
    return r;
  }
  static __device__ __forceinline__ uint64_t mul_add(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t lo = a * b;
    uint64_t hi = __umul64hi(a, b);
    lo += c;
    hi += (lo < c) ? 1ull : 0ull;
    return reduce(lo, hi);
  }
  static __device__ __forceinline__ pw load_point(const void* pts, int v, int64_t idx, int64_t npts) {
    const uint64_t x = __ldg((const unsigned long long*)pts + (int64_t)v * npts + idx);
    return x >= P ? x - P : x;
  }
  static __device__ __forceinline__ pw dummy_point() { return 2; }
  static __device__ __forceinline__ pw square(pw a) { return mul_add(a, a, 0); }
  static __device__ __forceinline__ pw mulx(pw a, pw x) { return mul_add(a, x, 0); }
  static __device__ __forceinline__ void node(bool leaf, bool first, coef ca, coef cb, const val* src, val* dst, pw xd) {
    const uint64_t s = leaf ? ca : *src;
    const uint64_t init = first ? cb : *dst;
    *dst = mul_add(s, xd, init);
  }
  static __device__ __forceinline__ val root(bool leaf, coef c, const val* acc) { return leaf ? c : *acc; }
  static __device__ __forceinline__ val apply_root_power(val r, pw xd) { return mul_add(r, xd, 0); }
  static __device__ __forceinline__ void store(void* out, int64_t idx, int64_t, val r) { ((uint64_t*)out)[idx] = r; }
};

// Closed intervals with directed rounding.  The operation order is the
// paper's walk verbatim: p = (m[h] + c) * x^d; m[h] = 0; m[lh(parent)] += p.
// Two shortcuts give bit-identical endpoints: a leaf's m[h] is zero, so
// m[h] + c = [c, c] exactly (coefficients of leaves are non-zero); a first
// child adds into a zero slot, and [+0,+0] + p equals p except that an upper
// bound -0 becomes +0 (round-up of +0 + -0).
struct IV {
  double lo, hi;
};

struct IV64 {
  using coef = double;
  using val = IV;
  using pw = IV;
  static __device__ __forceinline__ coef coef_from_bits(uint64_t b) { return __longlong_as_double((long long)b); }
  static __device__ __forceinline__ int cls(const IV& a) { return a.lo >= 0.0 ? 0 : (a.hi <= 0.0 ? 1 : 2); }
  // Moore's nine sign cases: each bound is the directed rounding of the exact
  // extreme product.
  static __device__ __forceinline__ IV mul(const IV& a, const IV& b) {
    const int ca = cls(a), cb = cls(b);
    IV r;
    if (ca == 0) {
      if (cb == 0) { r.lo = __dmul_rd(a.lo, b.lo); r.hi = __dmul_ru(a.hi, b.hi); }
      else if (cb == 1) { r.lo = __dmul_rd(a.hi, b.lo); r.hi = __dmul_ru(a.lo, b.hi); }
      else { r.lo = __dmul_rd(a.hi, b.lo); r.hi = __dmul_ru(a.hi, b.hi); }
    } else if (ca == 1) {
      if (cb == 0) { r.lo = __dmul_rd(a.lo, b.hi); r.hi = __dmul_ru(a.hi, b.lo); }
      else if (cb == 1) { r.lo = __dmul_rd(a.hi, b.hi); r.hi = __dmul_ru(a.lo, b.lo); }
      else { r.lo = __dmul_rd(a.lo, b.hi); r.hi = __dmul_ru(a.lo, b.lo); }
    } else {
      if (cb == 0) { r.lo = __dmul_rd(a.lo, b.hi); r.hi = __dmul_ru(a.hi, b.hi); }
      else if (cb == 1) { r.lo = __dmul_rd(a.hi, b.lo); r.hi = __dmul_ru(a.lo, b.lo); }
      else {
        const double l1 = __dmul_rd(a.lo, b.hi), l2 = __dmul_rd(a.hi, b.lo);
        const double h1 = __dmul_ru(a.lo, b.lo), h2 = __dmul_ru(a.hi, b.hi);
        r.lo = l1 < l2 ? l1 : l2;
        r.hi = h1 > h2 ? h1 : h2;
      }
    }
    return r;
  }
  static __device__ __forceinline__ pw load_point(const void* pts, int v, int64_t idx, int64_t npts) {
    const double* b = (const double*)pts + (int64_t)(2 * v) * npts;
    IV r;
    r.lo = __ldg(b + idx);
    r.hi = __ldg(b + npts + idx);
    return r;
  }
  static __device__ __forceinline__ pw dummy_point() { IV r; r.lo = 0.5; r.hi = 0.5; return r; }
  static __device__ __forceinline__ pw square(pw a) {
    IV r;
    const int c = cls(a);
    if (c == 0) { r.lo = __dmul_rd(a.lo, a.lo); r.hi = __dmul_ru(a.hi, a.hi); }
    else if (c == 1) { r.lo = __dmul_rd(a.hi, a.hi); r.hi = __dmul_ru(a.lo, a.lo); }
    else {
      const double h1 = __dmul_ru(a.lo, a.lo), h2 = __dmul_ru(a.hi, a.hi);
      r.lo = 0.0;
      r.hi = h1 > h2 ? h1 : h2;
    }
    return r;
  }
  static __device__ __forceinline__ pw mulx(pw a, pw x) { return mul(a, x); }
  static __device__ __forceinline__ void node(bool leaf, bool first, coef ca, coef, const val* src, val* dst, pw xd) {
    IV s;
    if (leaf) { s.lo = ca; s.hi = ca; }
    else { const IV m = *src; s.lo = __dadd_rd(m.lo, ca); s.hi = __dadd_ru(m.hi, ca); }
    const IV p = mul(s, xd);
    if (first) {
      IV r;
      r.lo = p.lo;
      r.hi = (p.hi == 0.0) ? 0.0 : p.hi;
      *dst = r;
    } else {
      const IV m = *dst;
      IV r;
      r.lo = __dadd_rd(m.lo, p.lo);
      r.hi = __dadd_ru(m.hi, p.hi);
      *dst = r;
    }
  }
  static __device__ __forceinline__ val root(bool leaf, coef c, const val* acc) {
    IV r;
    if (leaf) { r.lo = c; r.hi = c; }
    else { const IV m = *acc; r.lo = __dadd_rd(m.lo, c); r.hi = __dadd_ru(m.hi, c); }
    return r;
  }
  static __device__ __forceinline__ val apply_root_power(val r, pw xd) { return mul(r, xd); }
  static __device__ __forceinline__ void store(void* out, int64_t idx, int64_t npts, val r) {
    ((double*)out)[idx] = r.lo;
    ((double*)out)[npts + idx] = r.hi;
  }
};

// ---------------------------------------------------------------- kernel
// x^d by left-to-right binary exponentiation: x^d = (x^floor(d/2))^2 * x^(d mod 2),
// the same sequence as the power program (used when the table does not fit).
template <class A>
__device__ __forceinline__ typename A::pw binexp(typename A::pw x, uint32_t d) {
  typename A::pw r = x;
  for (int b = 30 - __clz(d); b >= 0; --b) {
    r = A::square(r);
    if ((d >> b) & 1u) r = A::mulx(r, x);
  }
  return r;
}

// TABLE = true: pw holds the full power table [npow][PPT][TPB] (Sec. 2.2).
// TABLE = false: pw holds only the points x_v [nvars][PPT][TPB] and every
// node computes its power on the fly (trees with very many distinct powers,
// e.g. the Direct scheme).
template <class A, int PPT, bool TABLE>
__global__ void __launch_bounds__(kTPB) eval_kernel(const EvalArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using V = typename A::val;
  using W = typename A::pw;
  using C = typename A::coef;
  V* acc = reinterpret_cast<V*>(smem_raw);                          // [nslot][PPT][TPB]
  W* pw = reinterpret_cast<W*>(smem_raw + sizeof(V) * (size_t)g.nslot * PPT * kTPB);
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * (kTPB * PPT);

  if (TABLE) {
    // power table: every distinct x_v^d once per point
    for (int k = 0; k < g.npow; ++k) {
      const uint32_t w = __ldg(g.pow_prog + k);
      const uint32_t op = w & 3u, a1 = (w >> 2) & 0x7FFFu, a2 = w >> 17;
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        const int64_t idx = base + p * kTPB + tid;
        W r;
        if (op == kPowLoad) r = idx < g.npts ? A::load_point(g.points, (int)a1, idx, g.npts) : A::dummy_point();
        else if (op == kPowSq) r = A::square(pw[(a1 * PPT + p) * kTPB + tid]);
        else r = A::mulx(pw[(a1 * PPT + p) * kTPB + tid], pw[(a2 * PPT + p) * kTPB + tid]);
        pw[(k * PPT + p) * kTPB + tid] = r;
      }
    }
  } else {
    for (int v = 0; v < g.nvars; ++v) {
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        const int64_t idx = base + p * kTPB + tid;
        pw[(v * PPT + p) * kTPB + tid] = idx < g.npts ? A::load_point(g.points, v, idx, g.npts) : A::dummy_point();
      }
    }
  }

  // coefficient walk (Sec. 2.1) over the non-root nodes
  const C* ca = reinterpret_cast<const C*>(g.ca);
  const C* cb = reinterpret_cast<const C*>(g.cb);
  uint32_t c_next = g.nsteps > 0 ? __ldg(g.ctrl) : 0u;
  C a_next = g.nsteps > 0 ? ca[0] : C(0);
  C b_next = g.nsteps > 0 ? cb[0] : C(0);
  for (int64_t i = 0; i < g.nsteps; ++i) {
    const uint32_t c = c_next;
    const C va = a_next, vb = b_next;
    if (i + 1 < g.nsteps) {
      c_next = __ldg(g.ctrl + i + 1);
      a_next = ca[i + 1];
      b_next = cb[i + 1];
    }
    const int S = (int)((c >> kCtrlS) & 63u), D = (int)((c >> kCtrlD) & 63u);
    const bool leaf = (c >> kCtrlLeaf) & 1u, first = (c >> kCtrlFirst) & 1u;
    const int pid = (int)(c >> kCtrlPid);
    uint32_t dv = 0, dd = 0;
    if (!TABLE) {
      const uint2 q = __ldg(g.pow_dv + pid);
      dv = q.x;
      dd = q.y;
    }
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const W xd = TABLE ? pw[(pid * PPT + p) * kTPB + tid] : binexp<A>(pw[(dv * PPT + p) * kTPB + tid], dd);
      A::node(leaf, first, va, vb, &acc[(S * PPT + p) * kTPB + tid], &acc[(D * PPT + p) * kTPB + tid], xd);
    }
  }

  // root
  const C rc = A::coef_from_bits(g.root_c);
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    const int64_t idx = base + p * kTPB + tid;
    V r = A::root(g.root_leaf, rc, &acc[(g.root_lh * PPT + p) * kTPB + tid]);
    if (g.root_pid >= 0) {
      W xd;
      if (TABLE) xd = pw[(g.root_pid * PPT + p) * kTPB + tid];
      else { const uint2 q = __ldg(g.pow_dv + g.root_pid); xd = binexp<A>(pw[(q.x * PPT + p) * kTPB + tid], q.y); }
      r = A::apply_root_power(r, xd);
    }
    if (idx < g.npts) A::store(g.out, idx, g.npts, r);
  }
}

// Launch helpers (defined per type in eval_<type>.cu).
size_t eval_smem_bytes(fp_dtype dt, int nslot, int npow, int ppt);
int eval_ppt(fp_dtype dt);
cudaError_t launch_eval_f64(const EvalArgs& a, cudaStream_t s);
cudaError_t launch_eval_f32c(const EvalArgs& a, cudaStream_t s);
cudaError_t launch_eval_iv64(const EvalArgs& a, cudaStream_t s);
cudaError_t launch_eval_modp(const EvalArgs& a, cudaStream_t s);

// Shared memory of one block; the power table is used while it leaves room
// for at least two resident blocks per SM.
constexpr size_t kTableSmemCap = 100 * 1024;
constexpr size_t kSmemMax = 227 * 1024;

template <class A, int PPT>
size_t eval_smem(const EvalArgs& a, bool table) {
  return (sizeof(typename A::val) * (size_t)a.nslot +
          sizeof(typename A::pw) * (size_t)(table ? a.npow : a.nvars)) * PPT * kTPB;
}

template <class A, int PPT>
cudaError_t launch_eval(const EvalArgs& a, cudaStream_t s) {
  const bool table = eval_smem<A, PPT>(a, true) <= kTableSmemCap;
  const size_t smem = eval_smem<A, PPT>(a, table);
  if (smem > kSmemMax) return cudaErrorInvalidValue;
  static int configured_dev = -1;  // raise the dynamic shared-memory cap once per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(eval_kernel<A, PPT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(eval_kernel<A, PPT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    if (e != cudaSuccess) return e;
    configured_dev = dev;
  }
  const int64_t per_block = (int64_t)kTPB * PPT;
  const int64_t blocks = (a.npts + per_block - 1) / per_block;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  if (table) eval_kernel<A, PPT, true><<<(unsigned)blocks, kTPB, smem, s>>>(a);
  else eval_kernel<A, PPT, false><<<(unsigned)blocks, kTPB, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fp
