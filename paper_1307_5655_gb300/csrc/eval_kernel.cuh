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
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>
#include <cstring>
#include <type_traits>

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
  static __device__ __forceinline__ val from_coef(coef c) { return c; }
  static constexpr bool kSlotAtEnd = false;
  static constexpr bool kExact = false;
  static constexpr bool kKindRuns = false;
  static __device__ __forceinline__ val mad(val s, pw xd, val init) { return fma(s, xd, init); }
  template <bool SC, bool IC, bool X1>
  static __device__ __forceinline__ val mad_k(val s, pw xd, val init) { return fma(s, xd, init); }
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
  // s * x^d + init with the rounding errors of the product and the sum
  // (exact by TwoProduct / TwoSum) and the first-order terms of the
  // operands' own corrections gathered in lo
  static __device__ __forceinline__ val mad(val s, pw xd, val init) {
    const float p = __fmul_rn(s.x, xd.x);
    const float pe = __fmaf_rn(s.x, xd.x, -p);
    float h, se;
    two_sum(init.x, p, h, se);
    float lo = __fadd_rn(init.y, __fadd_rn(pe, se));
    lo = __fmaf_rn(s.y, xd.x, lo);
    lo = __fmaf_rn(s.x, xd.y, lo);
    return make_float2(h, lo);
  }
  // mad with operands known to have a zero low part: SC, s is a coefficient;
  // IC, init is a coefficient; X1, the power is x itself (a loaded FP32
  // point).  The terms dropped are exact zeros, so the value is mad's.
  template <bool SC, bool IC, bool X1>
  static __device__ __forceinline__ val mad_k(val s, pw xd, val init) {
    const float p = __fmul_rn(s.x, xd.x);
    const float pe = __fmaf_rn(s.x, xd.x, -p);
    float h, se;
    two_sum(init.x, p, h, se);
    float lo = IC ? __fadd_rn(pe, se) : __fadd_rn(init.y, __fadd_rn(pe, se));
    if constexpr (!SC) lo = __fmaf_rn(s.y, xd.x, lo);
    if constexpr (!X1) lo = __fmaf_rn(s.x, xd.y, lo);
    return make_float2(h, lo);
  }
  static constexpr bool kSlotAtEnd = true;
  static constexpr bool kExact = false;
  static constexpr bool kKindRuns = false;
  // a + b with the rounding error of the leading sum (TwoSum) kept in lo
  static __device__ __forceinline__ val add(val a, val b) {
    float h, e;
    two_sum(a.x, b.x, h, e);
    return make_float2(h, __fadd_rn(__fadd_rn(a.y, b.y), e));
  }
  static __device__ __forceinline__ val from_coef(coef c) { return make_float2(c, 0.0f); }
  static __device__ __forceinline__ void node(bool leaf, bool first, coef ca, coef cb, const val* src, val* dst, pw xd) {
    const float2 s = leaf ? make_float2(ca, 0.0f) : *src;
    const float2 init = first ? make_float2(cb, 0.0f) : *dst;
    *dst = mad(s, xd, init);
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
  // lo + 2^64 hi mod p, hi = h1 2^32 + h0: congruent to lo - h1 + h0 (2^32 - 1)
  // (2^96 = -1, 2^64 = 2^32 - 1), on 32-bit halves with the carry flag:
  //   t = lo - h1, less 2^32 - 1 on a borrow (then t >= 2^32);
  //   u = h0 (2^32 - 1) = h0 2^32 - h0;
  //   r = t + u, plus 2^32 - 1 on a carry (r < (2^32 - 1)^2 there: no second
  //   carry); r + (2^32 - 1) carries out exactly when r >= p, and then equals r - p.
  static __device__ __forceinline__ uint64_t reduce(uint64_t lo, uint64_t hi) {
    uint32_t r0, r1;
    asm("{\n\t"
        ".reg .u32 t0, t1, m, u0, u1, s0, s1, c, v0, v1;\n\t"
        ".reg .pred q;\n\t"
        "sub.cc.u32 t0, %2, %5;\n\t"
        "subc.cc.u32 t1, %3, 0;\n\t"
        "subc.u32 m, 0, 0;\n\t"
        "sub.cc.u32 t0, t0, m;\n\t"
        "subc.u32 t1, t1, 0;\n\t"
        "sub.cc.u32 u0, 0, %4;\n\t"
        "subc.u32 u1, %4, 0;\n\t"
        "add.cc.u32 s0, t0, u0;\n\t"
        "addc.cc.u32 s1, t1, u1;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "neg.s32 m, c;\n\t"
        "add.cc.u32 s0, s0, m;\n\t"
        "addc.u32 s1, s1, 0;\n\t"
        "add.cc.u32 v0, s0, 0xFFFFFFFF;\n\t"
        "addc.cc.u32 v1, s1, 0;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "setp.ne.u32 q, c, 0;\n\t"
        "selp.u32 %0, v0, s0, q;\n\t"
        "selp.u32 %1, v1, s1, q;\n\t"
        "}"
        : "=r"(r0), "=r"(r1)
        : "r"((uint32_t)lo), "r"((uint32_t)(lo >> 32)), "r"((uint32_t)hi), "r"((uint32_t)(hi >> 32)));
    return (uint64_t)r1 << 32 | r0;
  }
  // (a + b) mod p for a, b < p: s = a + b (carry c); s + (2^32 - 1) carries
  // out exactly when s >= p, and then equals s - p; with c set the true sum is
  // s + 2^64, which is congruent to s + 2^32 - 1 < p.
  static __device__ __forceinline__ uint64_t add(uint64_t a, uint64_t b) {
    uint32_t r0, r1;
    asm("{\n\t"
        ".reg .u32 s0, s1, t0, t1, c;\n\t"
        ".reg .pred q;\n\t"
        "add.cc.u32 s0, %2, %4;\n\t"
        "addc.cc.u32 s1, %3, %5;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "add.cc.u32 t0, s0, 0xFFFFFFFF;\n\t"
        "addc.cc.u32 t1, s1, 0;\n\t"
        "addc.u32 c, c, 0;\n\t"
        "setp.ne.u32 q, c, 0;\n\t"
        "selp.u32 %0, t0, s0, q;\n\t"
        "selp.u32 %1, t1, s1, q;\n\t"
        "}"
        : "=r"(r0), "=r"(r1)
        : "r"((uint32_t)a), "r"((uint32_t)(a >> 32)), "r"((uint32_t)b), "r"((uint32_t)(b >> 32)));
    return (uint64_t)r1 << 32 | r0;
  }
  // (a - b) mod p for a, b < p: on a borrow, d = a - b + 2^64 >= 2^32, and
  // a - b + p = d - (2^32 - 1).
  static __device__ __forceinline__ uint64_t sub(uint64_t a, uint64_t b) {
    uint32_t r0, r1;
    asm("{\n\t"
        ".reg .u32 d0, d1, m;\n\t"
        "sub.cc.u32 d0, %2, %4;\n\t"
        "subc.cc.u32 d1, %3, %5;\n\t"
        "subc.u32 m, 0, 0;\n\t"
        "sub.cc.u32 %0, d0, m;\n\t"
        "subc.u32 %1, d1, 0;\n\t"
        "}"
        : "=r"(r0), "=r"(r1)
        : "r"((uint32_t)a), "r"((uint32_t)(a >> 32)), "r"((uint32_t)b), "r"((uint32_t)(b >> 32)));
    return (uint64_t)r1 << 32 | r0;
  }
  // (a b + c) mod p from the 128-bit product (a b + c < 2^128: no overflow)
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
  static __device__ __forceinline__ val from_coef(coef c) { return c; }
  static constexpr bool kSlotAtEnd = false;
  static constexpr bool kExact = true;  // any evaluation order gives the same residue
  static constexpr bool kKindRuns = false;
  static __device__ __forceinline__ val mad(val s, pw xd, val init) { return mul_add(s, xd, init); }
  template <bool SC, bool IC, bool X1>
  static __device__ __forceinline__ val mad_k(val s, pw xd, val init) { return mul_add(s, xd, init); }
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
  // the node walk runs nodes of one kind as a loop (walk_run): a leaf skips
  // the coefficient's additions and a first child the accumulation's
  static constexpr bool kKindRuns = true;
  static __device__ __forceinline__ coef coef_from_bits(uint64_t b) { return __longlong_as_double((long long)b); }
  // Sign tests on the bit patterns (integer pipe; double compares would use
  // the reduced-rate FP64 pipe): x >= 0.0 holds for sign bit clear or -0.0,
  // x <= 0.0 for sign bit set or +0.0 (NaN bounds do not occur).  Bitwise
  // rather than short-circuit logic, so no branches.
  static __device__ __forceinline__ int ge0(double x) {
    const long long b = __double_as_longlong(x);
    return (b >= 0) | (b == (long long)0x8000000000000000ull);
  }
  static __device__ __forceinline__ int le0(double x) { return __double_as_longlong(x) <= 0; }
  static __device__ __forceinline__ int cls(const IV& a) { return ge0(a.lo) ? 0 : (le0(a.hi) ? 1 : 2); }
  // p ? a : b as an integer select.  The FP64 pipe is the walk's bound: as a
  // plain conditional the compiler may instead issue each product twice
  // under complementary predicates, which doubles its FP64 issue slots.
  static __device__ __forceinline__ double sel(int p, double a, double b) {
    double r;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %3, 0;\n\tselp.f64 %0, %1, %2, q;\n\t}"
        : "=d"(r)
        : "d"(a), "d"(b), "r"(p));
    return r;
  }
  // -0.0 -> +0.0, anything else unchanged (integer compare and select)
  static __device__ __forceinline__ double pos_zero(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    asm("{\n\t.reg .pred z;\n\tsetp.eq.u64 z, %1, 0x8000000000000000;\n\tselp.b64 %0, 0, %1, z;\n\t}"
        : "=l"(b)
        : "l"(b));
    return __longlong_as_double((long long)b);
  }
  // Moore's nine sign cases: each bound is the directed rounding of the exact
  // extreme product.  The operands of the two products are selected per lane
  // (lanes hold points of different signs, so branching per case would run
  // several cases' multiplies in every warp); only the case where both
  // intervals straddle zero needs two more products, taken by a branch.
  //   lower bound operands        upper bound operands
  //   P x P  a.lo b.lo            a.hi b.hi
  //   P x N  a.hi b.lo            a.lo b.hi
  //   P x M  a.hi b.lo            a.hi b.hi
  //   N x P  a.lo b.hi            a.hi b.lo
  //   N x N  a.hi b.hi            a.lo b.lo
  //   N x M  a.lo b.hi            a.lo b.lo
  //   M x P  a.lo b.hi            a.hi b.hi
  //   M x N  a.hi b.lo            a.lo b.lo
  //   M x M  min(a.lo b.hi, a.hi b.lo)   max(a.lo b.lo, a.hi b.hi)
  // The four operand choices of case 3 ca + cb, as bits (lower a, lower b,
  // upper a, upper b; 1 = the other bound) of a 4-bit field of kSel.
  static constexpr unsigned long long kSel =
      (0x0ull << 0) | (0x5ull << 4) | (0x1ull << 8) |    // P x P, P x N, P x M
      (0xAull << 12) | (0xFull << 16) | (0xEull << 20) |  // N x P, N x N, N x M
      (0x2ull << 24) | (0xDull << 28) | (0xEull << 32);   // M x P, M x N, M x M
  static __device__ __forceinline__ IV mul(const IV& a, const IV& b) {
    const int ca = cls(a), cb = cls(b);
    const int m = (int)(kSel >> (4 * (3 * ca + cb))) & 0xF;
    IV r;
    r.lo = __dmul_rd(sel(m & 1, a.hi, a.lo), sel(m & 2, b.hi, b.lo));
    r.hi = __dmul_ru(sel(m & 4, a.lo, a.hi), sel(m & 8, b.lo, b.hi));
    if (ca == 2 && cb == 2) {
      const double l2 = __dmul_rd(a.hi, b.lo), h2 = __dmul_ru(a.hi, b.hi);
      r.lo = r.lo < l2 ? r.lo : l2;
      r.hi = r.hi > h2 ? r.hi : h2;
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
  // tight square: non-negative [lo^2, hi^2]; non-positive [hi^2, lo^2];
  // straddling [+0, max(lo^2, hi^2)] (selected per lane as in mul)
  static __device__ __forceinline__ pw square(pw a) {
    IV r;
    const int c = cls(a);
    const double l = sel(c == 1, a.hi, a.lo), h = sel(c == 1, a.lo, a.hi);
    r.lo = __dmul_rd(l, l);
    r.hi = __dmul_ru(h, h);
    if (c == 2) {
      const double h1 = __dmul_ru(a.lo, a.lo);
      r.lo = 0.0;
      r.hi = h1 > r.hi ? h1 : r.hi;
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
      r.hi = pos_zero(p.hi);  // RU(+0 + p.hi): an exact zero sum is +0
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

// The node walk's cursor: the next step's control word and coefficients are
// loaded one step ahead.
template <class C>
struct WalkState {
  int64_t i;
  uint32_t c_next;
  C a_next, b_next;
};

// bit 0: leaf, bit 1: first child
__device__ __forceinline__ int node_kind(uint32_t c) {
  return (int)(((c >> kCtrlLeaf) & 1u) | (((c >> kCtrlFirst) & 1u) << 1));
}

// One node of the walk (at w.i), of kind (leaf, first) -- compile-time
// constants when called from walk_run.
template <class A, int PPT, bool TABLE>
__device__ __forceinline__ void walk_step(const EvalArgs& g, WalkState<typename A::coef>& w, typename A::val* acc,
                                          typename A::pw* pw, int tid, bool leaf, bool first) {
  using W = typename A::pw;
  using C = typename A::coef;
  const C* ca = reinterpret_cast<const C*>(g.ca);
  const C* cb = reinterpret_cast<const C*>(g.cb);
  const uint32_t c = w.c_next;
  const C va = w.a_next, vb = w.b_next;
  ++w.i;
  if (w.i < g.nsteps) {
    w.c_next = __ldg(g.ctrl + w.i);
    w.a_next = ca[w.i];
    w.b_next = cb[w.i];
  }
  const int S = (int)((c >> kCtrlS) & 63u), D = (int)((c >> kCtrlD) & 63u);
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

// the node at w.i, its kind read from its control word
template <class A, int PPT, bool TABLE>
__device__ __forceinline__ void walk_node(const EvalArgs& g, WalkState<typename A::coef>& w, typename A::val* acc,
                                          typename A::pw* pw, int tid) {
  const int k = node_kind(w.c_next);
  walk_step<A, PPT, TABLE>(g, w, acc, pw, tid, k & 1, k & 2);
}

// the nodes from w.i on while they are of kind (LEAF, FIRST); at least one
template <class A, int PPT, bool TABLE, bool LEAF, bool FIRST>
__device__ __forceinline__ void walk_run(const EvalArgs& g, WalkState<typename A::coef>& w, typename A::val* acc,
                                         typename A::pw* pw, int tid) {
  constexpr int kKind = (LEAF ? 1 : 0) | (FIRST ? 2 : 0);
  do {
    walk_step<A, PPT, TABLE>(g, w, acc, pw, tid, LEAF, FIRST);
  } while (w.i < g.nsteps && node_kind(w.c_next) == kKind);
}

// TABLE = true: pw holds the full power table [npow][PPT][TPB] (Sec. 2.2).
// TABLE = false: pw holds only the points x_v [nvars][PPT][TPB] and every
// node computes its power on the fly (trees with very many distinct powers,
// e.g. the Direct scheme).
template <class A, int PPT, bool TABLE>
__device__ __forceinline__ void node_tile(const EvalArgs& g, int64_t base, unsigned char* smem_raw) {
  using V = typename A::val;
  using W = typename A::pw;
  using C = typename A::coef;
  V* acc = reinterpret_cast<V*>(smem_raw);                          // [nslot][PPT][TPB]
  W* pw = reinterpret_cast<W*>(smem_raw + sizeof(V) * (size_t)g.nslot * PPT * kTPB);
  const int tid = threadIdx.x;

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
  WalkState<C> w;
  w.i = 0;
  w.c_next = g.nsteps > 0 ? __ldg(g.ctrl) : 0u;
  w.a_next = g.nsteps > 0 ? ca[0] : C(0);
  w.b_next = g.nsteps > 0 ? cb[0] : C(0);
  if constexpr (A::kKindRuns) {
    // in runs of nodes of one kind (leaf or not, first child or not): each
    // run is a loop whose body is compiled for its kind, so a kind's missing
    // operations are skipped by a branch rather than issued under a false
    // predicate (which still takes their FP64 pipe slots)
    while (w.i < g.nsteps) {
      switch (node_kind(w.c_next)) {
        case 0: walk_run<A, PPT, TABLE, false, false>(g, w, acc, pw, tid); break;
        case 1: walk_run<A, PPT, TABLE, true, false>(g, w, acc, pw, tid); break;
        case 2: walk_run<A, PPT, TABLE, false, true>(g, w, acc, pw, tid); break;
        default: walk_run<A, PPT, TABLE, true, true>(g, w, acc, pw, tid); break;
      }
    }
  } else {
    // one multiply-add per node whatever its kind: the kind only selects
    // operands
    while (w.i < g.nsteps) walk_node<A, PPT, TABLE>(g, w, acc, pw, tid);
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

template <class A, int PPT, bool TABLE>
__global__ void __launch_bounds__(kTPB) eval_kernel(const EvalArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  node_tile<A, PPT, TABLE>(g, (int64_t)blockIdx.x * (kTPB * PPT), smem_raw);
}


// ---------------------------------------------------------------- grouped-op kernel
// The walk grouped into ops (kOpNode / kOpChain / kOpBlock / kOpPartial): the
// fused value types evaluate chains as a register loop and dense runs (whole
// subtrees, or a node with its last children) with a compile-time template
// of the scheme's split -- Horner's rule over the run for exact types -- and
// dispatch once per op.

// The grouped-op kernel's table per point: entries of 8 bytes, the walk's
// powers at [0, nlive), the slots at [nlive, nlive + nslot); the power
// program writes explicit positions (its temporaries above nlive).
struct OpArgs {
  const void* recs;    // OpRec<coef> [nops]
  const void* stream;  // coefficients of chains and blocks
  const uint2* prog;   // [nprog] {op | A1 << 2 | A2 << 17, destination}
  const uint32_t* chain_pid;  // [nsteps] position of each node's edge power
  int64_t nops;
  int nprog, nlive, nslot, entries;
  int root_lh, root_pid;      // root slot, position of the root's power (-1: none)
  int pos_x1;                 // position of x_b (b: the blocks' variable) among the walk's powers (-1: none)
  int pid_pow[kMaxBlock + 1];  // position of x^d for the block templates (-1: absent)
  int ext;                     // Balanced tree with two-part blocks or recomputed edge powers
  int64_t split;               // first op of the root's later children (0: none)
  int ndefer;                  // ops from split on whose edge goes into the root's slot
  const uint2* defer_edges;    // [ndefer] their {PID, z} in walk order
};

// The kernels of a Balanced tree whose schedule has two-part blocks or
// recomputed edge powers (OpArgs::ext) are a template of their own: the code
// for them slows the plain Balanced kernel down even where it never runs.
constexpr int kSchemeBExt = 0x100 | FP_SCHEME_B;

template <int SCHEME>
__host__ __device__ constexpr int scheme_split(int n) {
  if (SCHEME == FP_SCHEME_E) {
    int f = 1;
    while (2 * f <= n) f *= 2;
    return f;
  }
  return (n + 1) / 2;  // FP_SCHEME_B
}

// which powers x^d (d <= kMaxBlock) a block template of the scheme can use
template <int SCHEME>
__host__ __device__ constexpr bool block_uses_power(int d) {
  for (int m = 2; m <= kMaxBlock; ++m)  // sizes of dense runs inside a block
    for (int n = 1; n < m; ++n)
      if (scheme_split<SCHEME>(n) == d) return true;
  return false;
}

// value of the tree T_f over the dense run c[LO..HI] (index order: c[LO] is
// the highest term), relative to the exponent of c[HI]:
//   T(run) = T(b) + T(a) x^f(n),  b = the f(n) lowest terms (Def. 1.2)
// BASE: the run ends at the block's last node, whose value is `base` (its
// coefficient for a block; its slot, which holds c_N plus N's earlier
// children, for a partial block)
template <class A, int SCHEME, int LO, int HI, bool BASE>
__device__ __forceinline__ typename A::val block_eval(const typename A::coef (&c)[kMaxBlock],
                                                      const typename A::pw (&xp)[kMaxBlock + 1],
                                                      const typename A::val& base) {
  if constexpr (LO == HI) {
    if constexpr (BASE) return base;
    else return A::from_coef(c[HI]);
  } else {
    constexpr int n = HI - LO;
    constexpr int f = scheme_split<SCHEME>(n);
    const typename A::val b = block_eval<A, SCHEME, HI - f + 1, HI, BASE>(c, xp, base);
    const typename A::val a = block_eval<A, SCHEME, LO, HI - f, false>(c, xp, base);
    // a single term is a bare coefficient; the base is one when the type
    // adds a partial block's slot after the block (A::kSlotAtEnd)
    constexpr bool a_coef = LO == HI - f;
    constexpr bool b_coef = f == 1 && (!BASE || A::kSlotAtEnd);
    return A::template mad_k<a_coef, b_coef, f == 1>(a, xp[f], b);
  }
}

// coefficients st[off + 4q .. off + 4q + 3] (off is a multiple of 4)
template <class C>
__device__ __forceinline__ void load4(const C* st, int64_t off, int q, C (&c)[4]) {
  if constexpr (sizeof(C) == 8) {
    const ulonglong2* v = reinterpret_cast<const ulonglong2*>(st + off) + 2 * q;
    const ulonglong2 u0 = __ldg(v), u1 = __ldg(v + 1);
    memcpy(&c[0], &u0.x, 8); memcpy(&c[1], &u0.y, 8); memcpy(&c[2], &u1.x, 8); memcpy(&c[3], &u1.y, 8);
  } else {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(st + off) + q);
    memcpy(&c[0], &u.x, 4); memcpy(&c[1], &u.y, 4); memcpy(&c[2], &u.z, 4); memcpy(&c[3], &u.w, 4);
  }
}

// The value of the block's last node N is its coefficient; for a partial
// block it is N's slot (slot[p]).  Types with A::kSlotAtEnd evaluate the run
// with 0 for N and add the slot afterwards (the slot's load then overlaps the
// block's arithmetic; one add more), the others start from the slot.  The
// op's run is loaded before the dispatch, in 4-element vectors (loading per
// length inside each case raised the register use of the kernels that serve
// every scheme -- batch, resident -- into spills).
template <class A, int SCHEME, int PPT>
__device__ __forceinline__ void block_dispatch(int len, bool partial, const typename A::coef* st, int64_t off,
                                               const typename A::pw (&xp)[PPT][kMaxBlock + 1],
                                               const typename A::val (&slot)[PPT], typename A::val (&v)[PPT]) {
  typename A::coef c[kMaxBlock];
#pragma unroll
  for (int q = 0; q < kMaxBlock / 4; ++q) {
    typename A::coef c4[4];
    if (4 * q < len) load4(st, off, q, c4);
    else c4[0] = c4[1] = c4[2] = c4[3] = typename A::coef(0);
#pragma unroll
    for (int r = 0; r < 4; ++r) c[4 * q + r] = c4[r];
  }
#define FP_BLOCK_CASE(L)                                                                      \
  case L:                                                                                     \
    _Pragma("unroll") for (int p = 0; p < PPT; ++p) {                                         \
      if constexpr (A::kSlotAtEnd) {                                                          \
        const typename A::val base = A::from_coef(partial ? typename A::coef(0) : c[L - 1]);  \
        v[p] = block_eval<A, SCHEME, 0, L - 1, true>(c, xp[p], base);                         \
        if (partial) v[p] = A::add(v[p], slot[p]);                                            \
      } else {                                                                                \
        const typename A::val base = partial ? slot[p] : A::from_coef(c[L - 1]);              \
        v[p] = block_eval<A, SCHEME, 0, L - 1, true>(c, xp[p], base);                         \
      }                                                                                       \
    }                                                                                         \
    break;
  switch (len) {
    FP_BLOCK_CASE(1) FP_BLOCK_CASE(2) FP_BLOCK_CASE(3) FP_BLOCK_CASE(4) FP_BLOCK_CASE(5) FP_BLOCK_CASE(6)
    FP_BLOCK_CASE(7) FP_BLOCK_CASE(8) FP_BLOCK_CASE(9) FP_BLOCK_CASE(10) FP_BLOCK_CASE(11)
    FP_BLOCK_CASE(12) FP_BLOCK_CASE(13) FP_BLOCK_CASE(14) FP_BLOCK_CASE(15) FP_BLOCK_CASE(16)
    default: break;
  }
#undef FP_BLOCK_CASE
}

// A Balanced run of L = 17 .. 22 nodes as its two parts in one straight
// piece of code: a, the upper ceil(L / 2) nodes, and b, the lower floor(L / 2)
// (ending at the op's last node), then T(b) + T(a) x^f -- the operations of
// the two-part loop below, in its order, without its second dispatch and part
// moves, and with the two parts' chains independent for the scheduler.
template <class A, int SCHEME, int PPT, int L>
__device__ __forceinline__ void two_part_case(bool partial, const typename A::coef* st, int64_t off,
                                              const typename A::pw (&xp)[PPT][kMaxBlock + 1],
                                              const typename A::val (&slot)[PPT], const typename A::pw (&xf)[PPT],
                                              typename A::val (&v)[PPT]) {
  using C = typename A::coef;
  using V = typename A::val;
  constexpr int LB = L / 2, LA = L - LB;
  const int64_t offb = off + ((LA + kStreamAlign - 1) & ~(kStreamAlign - 1));
  C ca[kMaxBlock], cb[kMaxBlock];
#pragma unroll
  for (int q = 0; q < (LA + 3) / 4; ++q) {
    C c4[4];
    load4(st, off, q, c4);
#pragma unroll
    for (int r = 0; r < 4; ++r) ca[4 * q + r] = c4[r];
  }
#pragma unroll
  for (int q = 0; q < (LB + 3) / 4; ++q) {
    C c4[4];
    load4(st, offb, q, c4);
#pragma unroll
    for (int r = 0; r < 4; ++r) cb[4 * q + r] = c4[r];
  }
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    const V va = block_eval<A, SCHEME, 0, LA - 1, true>(ca, xp[p], A::from_coef(ca[LA - 1]));
    V vb;
    if constexpr (A::kSlotAtEnd) {
      vb = block_eval<A, SCHEME, 0, LB - 1, true>(cb, xp[p], A::from_coef(partial ? C(0) : cb[LB - 1]));
      if (partial) vb = A::add(vb, slot[p]);
    } else {
      vb = block_eval<A, SCHEME, 0, LB - 1, true>(cb, xp[p], partial ? slot[p] : A::from_coef(cb[LB - 1]));
    }
    v[p] = A::mad(va, xf[p], vb);
  }
}

// 128-bit loads of an op record and of coefficient runs (read-only path)
template <class C>
__device__ __forceinline__ void load_rec(const OpRec<C>* r, uint4& h, C& a, C& b) {
  h = __ldg(reinterpret_cast<const uint4*>(r));
  if constexpr (sizeof(C) == 8) {
    const ulonglong2 q = __ldg(reinterpret_cast<const ulonglong2*>(r) + 1);
    memcpy(&a, &q.x, 8);
    memcpy(&b, &q.y, 8);
  } else {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(r) + 2);
    memcpy(&a, &q.x, 4);
    memcpy(&b, &q.y, 4);
  }
}

// TPB: threads per block (the stride of the per-point table); kTPB unless the
// launch chose narrower blocks for a small grid
// The edge power x^d of an op marked kPidRecompute, rebuilt from its record's
// z word: the table entry at its base position (0x7FFF: x itself), then m
// steps of squaring and, where the bit of d is set, multiplying by x -- the
// power program's own steps, so the value is the table's would-be entry.
template <class A>
__device__ __forceinline__ typename A::pw rebuild_power(uint32_t z, const typename A::pw* col, int stride,
                                                        typename A::pw x) {
  const int base = (int)(z & 0x7FFFu), m = (int)((z >> 15) & 15u);
  const uint32_t bits = z >> 19;
  typename A::pw y = base == 0x7FFF ? x : col[base * stride];
  for (int i = m - 1; i >= 0; --i) {
    y = A::square(y);
    if ((bits >> i) & 1u) y = A::mulx(y, x);
  }
  return y;
}

// SPLIT (one point per thread, TPB = 64): the block's two warps evaluate the
// same 32 points, warp 0 the ops [0, o.split) (the root's first child's
// subtree, ending with its edge into the root's slot) and warp 1 the others,
// keeping the values of its edges into the root's slot (marked in w) in its
// own table entries past o.entries; after warp 0 is done warp 1 applies them,
// in walk order, to warp 0's root slot -- the walk's own operations in its own
// order, so the result is that of one warp.  Twice the warps for a grid too
// small to fill the SMs' schedulers evenly.
template <class A, int PPT, int SCHEME, int TPB = kTPB, bool SPLIT = false>
__device__ __forceinline__ void ops_tile(const EvalArgs& g, const OpArgs& o, int64_t base, unsigned char* smem_raw) {
  using V = typename A::val;
  using W = typename A::pw;
  using C = typename A::coef;
  static_assert(sizeof(V) == sizeof(W), "powers and slots share one table");
  W* pw = reinterpret_cast<W*>(smem_raw);                        // [entries][PPT][TPB]
  V* acc = reinterpret_cast<V*>(smem_raw) + (size_t)o.nlive * PPT * TPB;  // slots above the walk's powers
  const int tid = threadIdx.x;
  static_assert(!SPLIT || (PPT == 1 && TPB == 64), "the split runs one point per thread in two warps");
  const int col = SPLIT ? (tid & 31) : tid;  // the thread's point within the block's points
  const int half = SPLIT ? (tid >> 5) : 0;

  for (int k = 0; k < o.nprog; ++k) {
    const uint2 e = __ldg(o.prog + k);
    const uint32_t op = e.x & 3u, a1 = (e.x >> 2) & 0x7FFFu, a2 = e.x >> 17, dst = e.y;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      const int64_t idx = base + p * TPB + col;
      W r;
      if (op == kPowLoad) r = idx < g.npts ? A::load_point(g.points, (int)a1, idx, g.npts) : A::dummy_point();
      else if (op == kPowSq) r = A::square(pw[(a1 * PPT + p) * TPB + tid]);
      else r = A::mulx(pw[(a1 * PPT + p) * TPB + tid], pw[(a2 * PPT + p) * TPB + tid]);
      pw[(dst * PPT + p) * TPB + tid] = r;
    }
  }

  // powers x^d of the block templates: every one is a partial degree of the
  // tree, so it is read from the power table (recomputing them per block
  // would cost FP64 multiplies), before the slots reuse the temporaries' space
  W xp[PPT][kMaxBlock + 1];
  if constexpr (SCHEME != 0) {
#pragma unroll
    for (int d = 1; d <= kMaxBlock; ++d) {
      if (block_uses_power<SCHEME>(d)) {
        const int q = o.pid_pow[d] < 0 ? 0 : o.pid_pow[d];
#pragma unroll
        for (int p = 0; p < PPT; ++p) xp[p][d] = pw[(q * PPT + p) * TPB + tid];
      }
    }
  }

  const OpRec<C>* recs = reinterpret_cast<const OpRec<C>*>(o.recs);
  const C* st = reinterpret_cast<const C*>(o.stream);
  int64_t i_begin = 0, i_end = o.nops;
  V* defer = reinterpret_cast<V*>(smem_raw) + (size_t)o.entries * TPB;  // SPLIT: kept root edges
  int nd = 0;
  if constexpr (SPLIT) {
    if (half == 0) i_end = o.split;
    else i_begin = o.split;
  }
  for (int64_t i = i_begin; i < i_end; ++i) {
    uint4 h;
    C a, b;
    load_rec(recs + i, h, a, b);
    const uint32_t kind = h.x & 3u;
    const int S = (int)((h.x >> kOpS) & 63u), D = (int)((h.x >> kOpD) & 63u);
    const bool leaf = (h.x >> kOpLeaf) & 1u, first = (h.x >> kOpFirst) & 1u;
    const int pid = (int)(h.x >> kOpPid);
    const int len = (int)(h.y & 255u) + 1;
    const int64_t off = (int64_t)(h.w & 0x7FFFFFFFu);
    V v[PPT];
    if (kind == kOpNode) {
#pragma unroll
      for (int p = 0; p < PPT; ++p) v[p] = leaf ? A::from_coef(a) : acc[(S * PPT + p) * TPB + tid];
    } else if (kind == kOpChain) {
      const int64_t j0 = (int64_t)h.z;
      const C* cs = st + off;  // node j0 + t uses cs[t]
#pragma unroll
      for (int p = 0; p < PPT; ++p) v[p] = leaf ? A::from_coef(__ldg(cs)) : acc[(S * PPT + p) * TPB + tid];
      if ((h.x >> kOpUniform) & 1u) {
        const int pc = (int)__ldg(o.chain_pid + j0);
        W xu[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) xu[p] = pw[(pc * PPT + p) * TPB + tid];
        if (pc == o.pos_x1) {  // Horner runs over consecutive exponents
          for (int t = 1; t < len; ++t) {
            const V cj = A::from_coef(__ldg(cs + t));
#pragma unroll
            for (int p = 0; p < PPT; ++p) v[p] = A::template mad_k<false, true, true>(v[p], xu[p], cj);
          }
        } else {
          for (int t = 1; t < len; ++t) {
            const V cj = A::from_coef(__ldg(cs + t));
#pragma unroll
            for (int p = 0; p < PPT; ++p) v[p] = A::template mad_k<false, true, false>(v[p], xu[p], cj);
          }
        }
      } else {
        for (int t = 1; t < len; ++t) {
          const int pc = (int)__ldg(o.chain_pid + j0 + t - 1);
          const V cj = A::from_coef(__ldg(cs + t));
#pragma unroll
          for (int p = 0; p < PPT; ++p)
            v[p] = A::template mad_k<false, true, false>(v[p], pw[(pc * PPT + p) * TPB + tid], cj);
        }
      }
    } else if constexpr (SCHEME != 0 && A::kExact) {
      // exact arithmetic: the run's value does not depend on the order of
      // its operations, so the block is evaluated by Horner's rule over the
      // same run (one short loop instead of an unrolled template per length)
      const C* cs = st + off;
      const bool partial = kind == kOpPartial;
      const V c0 = A::from_coef(__ldg(cs));
#pragma unroll
      for (int p = 0; p < PPT; ++p) v[p] = c0;
      for (int t = 1; t + 1 < len; ++t) {
        const V ct = A::from_coef(__ldg(cs + t));
#pragma unroll
        for (int p = 0; p < PPT; ++p) v[p] = A::mad(v[p], xp[p][1], ct);
      }
      const V cl = A::from_coef(__ldg(cs + len - 1));
#pragma unroll
      for (int p = 0; p < PPT; ++p) v[p] = A::mad(v[p], xp[p][1], partial ? acc[(S * PPT + p) * TPB + tid] : cl);
    } else {
      if constexpr (SCHEME != 0) {
        // a partial block's last node N starts from its slot (c_N plus N's
        // earlier children)
        const bool partial = kind == kOpPartial;
        V slot[PPT];
        if (partial) {
#pragma unroll
          for (int p = 0; p < PPT; ++p) slot[p] = acc[(S * PPT + p) * TPB + tid];
        }
        // Balanced trees: a run longer than kMaxBlock (f > 0) is T(b) +
        // T(a) x^f, b its f lowest nodes (ending at the op's last node), a
        // the others, each stored from an aligned offset.  When f is the
        // run's middle (the Balanced split, 17 to 22 nodes) one straight-line
        // case evaluates both parts and the join; otherwise the loop below
        // runs the parts through the same templates (f = 0: an ordinary block
        // of at most kMaxBlock nodes, its one part).  Other schemes have
        // single-part blocks only.
        if constexpr (SCHEME != kSchemeBExt) {
          block_dispatch<A, SCHEME, PPT>(len, partial, st, off, xp, slot, v);
        } else {
        const int f = (int)((h.y >> 8) & 255u);
        if (f > 0 && f == len / 2 && len >= 17 && len <= 22) {
          W xf[PPT];
#pragma unroll
          for (int p = 0; p < PPT; ++p) xf[p] = pw[((int)(h.y >> 16) * PPT + p) * TPB + tid];
          switch (len) {
            case 17: two_part_case<A, SCHEME, PPT, 17>(partial, st, off, xp, slot, xf, v); break;
            case 18: two_part_case<A, SCHEME, PPT, 18>(partial, st, off, xp, slot, xf, v); break;
            case 19: two_part_case<A, SCHEME, PPT, 19>(partial, st, off, xp, slot, xf, v); break;
            case 20: two_part_case<A, SCHEME, PPT, 20>(partial, st, off, xp, slot, xf, v); break;
            case 21: two_part_case<A, SCHEME, PPT, 21>(partial, st, off, xp, slot, xf, v); break;
            default: two_part_case<A, SCHEME, PPT, 22>(partial, st, off, xp, slot, xf, v); break;
          }
        } else {
        V va[PPT];
#pragma unroll 1
        for (int part = f > 0 ? 0 : 1; part < 2; ++part) {
          const bool lower = part == 1;
          const int plen = lower ? (f > 0 ? f : len) : len - f;
          const int64_t poff = lower && f > 0 ? off + ((len - f + kStreamAlign - 1) & ~(kStreamAlign - 1)) : off;
          V w[PPT];
          block_dispatch<A, SCHEME, PPT>(plen, lower && partial, st, poff, xp, slot, w);
#pragma unroll
          for (int p = 0; p < PPT; ++p) {
            if (lower) v[p] = w[p];
            else va[p] = w[p];
          }
        }
        if (f > 0) {
          const int cp = (int)(h.y >> 16);
#pragma unroll
          for (int p = 0; p < PPT; ++p) v[p] = A::mad(va[p], pw[(cp * PPT + p) * TPB + tid], v[p]);
        }
        }
        }
      }
    }
    // the outgoing edge of the op's last node; its power from the table, or
    // (kPidRecompute: a block of a Balanced tree whose power few ops read)
    // recomputed from a kept prefix x^(d >> m), or x, by the power program's
    // steps: square, then times x where the bit of d is set
    if constexpr (SPLIT) {
      if (half == 1 && (h.w >> 31)) {  // an edge into the root's slot: applied after warp 0
        defer[nd * TPB + tid] = v[0];
        ++nd;
        continue;
      }
    }
    if (SCHEME != kSchemeBExt || pid != (int)kPidRecompute) {
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        V* dst = &acc[(D * PPT + p) * TPB + tid];
        const V init = first ? A::from_coef(b) : *dst;
        *dst = A::mad(v[p], pw[(pid * PPT + p) * TPB + tid], init);
      }
    } else if constexpr (SCHEME == kSchemeBExt) {
      W xe[PPT];
#pragma unroll
      for (int p = 0; p < PPT; ++p) xe[p] = rebuild_power<A>(h.z, pw + p * TPB + tid, PPT * TPB, xp[p][1]);
#pragma unroll
      for (int p = 0; p < PPT; ++p) {
        V* dst = &acc[(D * PPT + p) * TPB + tid];
        const V init = first ? A::from_coef(b) : *dst;
        *dst = A::mad(v[p], xe[p], init);
      }
    }
  }

  if constexpr (SPLIT) {
    __syncthreads();
    if (half == 1) {
      const int64_t idx = base + col;
      V r = acc[o.root_lh * TPB + tid - 32];  // the root's slot after warp 0's part
      for (int k = 0; k < o.ndefer; ++k) {
        const uint2 e = __ldg(o.defer_edges + k);
        W xe;
        if (SCHEME != kSchemeBExt || e.x != kPidRecompute) xe = pw[e.x * TPB + tid];
        else xe = rebuild_power<A>(e.y, pw + tid, TPB, xp[0][1]);
        r = A::mad(defer[k * TPB + tid], xe, r);
      }
      if (o.root_pid >= 0) r = A::apply_root_power(r, pw[o.root_pid * TPB + tid]);
      if (idx < g.npts) A::store(g.out, idx, g.npts, r);
    }
    return;
  }
  const C rc = A::coef_from_bits(g.root_c);
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    const int64_t idx = base + p * TPB + tid;
    V r = A::root(g.root_leaf, rc, &acc[(o.root_lh * PPT + p) * TPB + tid]);
    if (o.root_pid >= 0) r = A::apply_root_power(r, pw[(o.root_pid * PPT + p) * TPB + tid]);
    if (idx < g.npts) A::store(g.out, idx, g.npts, r);
  }
}

// Minimum resident blocks per SM given to ptxas (0: none, its own register
// choice).  Left to itself ptxas holds the FP32C Estrin kernel at two points
// per thread to 56 registers, for a residency that its power table (>= 16
// entries, >= 32 KB per 128-thread block, at >= 3000 terms) never allows; a
// bound of one block lets it take 96, 7 % faster at 10007 terms (2^24 points)
// with the same 5 blocks per SM.  Every other instantiation measured level or
// slower with the bound (FP32C H and B, and MODP, at 1, 2 and 4 points).
template <class A, int PPT, int SCHEME>
constexpr int ops_min_blocks() {
  return (std::is_same<A, F32C>::value && SCHEME == FP_SCHEME_E && PPT == 2) ? 1 : 0;
}

template <class A, int PPT, int SCHEME, int TPB = kTPB, bool SPLIT = false>
__global__ void __launch_bounds__(TPB, (ops_min_blocks<A, PPT, SCHEME>())) eval_ops_kernel(const EvalArgs g, const OpArgs o) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ops_tile<A, PPT, SCHEME, TPB, SPLIT>(g, o, (int64_t)blockIdx.x * (SPLIT ? 32 : TPB * PPT), smem_raw);
}

// Launch helpers (defined per type in eval_<type>.cu).  variant: 0 = choose,
// 1 = register kernel, 2 = shared-memory kernel.
// variant 1 = grouped-op kernel (fused types only), 2 = node-by-node kernel.
cudaError_t launch_eval_f64(const EvalArgs& a, const OpArgs& o, int scheme, cudaStream_t s, int variant, int ppt);
cudaError_t launch_eval_f32c(const EvalArgs& a, const OpArgs& o, int scheme, cudaStream_t s, int variant, int ppt);
cudaError_t launch_eval_iv64(const EvalArgs& a, const OpArgs& o, int scheme, cudaStream_t s, int variant, int ppt);
cudaError_t launch_eval_modp(const EvalArgs& a, const OpArgs& o, int scheme, cudaStream_t s, int variant, int ppt);

// Shared memory of one block; the power table is used while it leaves room
// for at least two resident blocks per SM (228 KB per SM, 1 KB of it reserved
// per block).
constexpr size_t kTableSmemCap = 113 * 1024;
constexpr size_t kSmemMax = 227 * 1024;

template <class A, int PPT>
size_t eval_smem(const EvalArgs& a, bool table) {
  return (sizeof(typename A::val) * (size_t)a.nslot +
          sizeof(typename A::pw) * (size_t)(table ? a.npow : a.nvars)) * PPT * kTPB;
}

// Shared-memory kernel (any lazy height; power table or on-the-fly powers).
template <class A, int PPT>
cudaError_t launch_eval_smem(const EvalArgs& a, cudaStream_t s) {
  const bool table = eval_smem<A, PPT>(a, true) <= kTableSmemCap;
  const size_t smem = eval_smem<A, PPT>(a, table);
  if (smem > kSmemMax) return cudaErrorInvalidValue;
  // raise the dynamic shared-memory cap once per device (atomic: the server's
  // worker and the caller's threads may launch concurrently; a repeat is harmless)
  static std::atomic<int> configured_dev{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev.load(std::memory_order_relaxed) != dev) {
    cudaError_t e = cudaFuncSetAttribute(eval_kernel<A, PPT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(eval_kernel<A, PPT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    if (e != cudaSuccess) return e;
    configured_dev.store(dev, std::memory_order_relaxed);
  }
  const int64_t per_block = (int64_t)kTPB * PPT;
  const int64_t blocks = (a.npts + per_block - 1) / per_block;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  if (table) eval_kernel<A, PPT, true><<<(unsigned)blocks, kTPB, smem, s>>>(a);
  else eval_kernel<A, PPT, false><<<(unsigned)blocks, kTPB, smem, s>>>(a);
  return cudaGetLastError();
}

template <class A, int PPT>
size_t ops_smem(const OpArgs& o) {
  return sizeof(typename A::pw) * (size_t)o.entries * PPT * kTPB;
}

template <class A, int PPT, int SCHEME, int TPB>
cudaError_t launch_eval_ops_tpb(const EvalArgs& a, const OpArgs& o, cudaStream_t s) {
  const size_t smem = ops_smem<A, PPT>(o) / kTPB * TPB;
  if (smem > kSmemMax) return cudaErrorInvalidValue;
  static std::atomic<int> configured_dev{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev.load(std::memory_order_relaxed) != dev) {
    cudaError_t e = cudaFuncSetAttribute(eval_ops_kernel<A, PPT, SCHEME, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    if (e != cudaSuccess) return e;
    configured_dev.store(dev, std::memory_order_relaxed);
  }
  const int64_t per_block = (int64_t)TPB * PPT;
  const int64_t blocks = (a.npts + per_block - 1) / per_block;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  eval_ops_kernel<A, PPT, SCHEME, TPB><<<(unsigned)blocks, TPB, smem, s>>>(a, o);
  return cudaGetLastError();
}

// the split kernel: blocks of two warps over 32 points each
template <class A, int SCHEME>
cudaError_t launch_eval_ops_split(const EvalArgs& a, const OpArgs& o, cudaStream_t s) {
  const size_t smem = sizeof(typename A::pw) * (size_t)(o.entries + o.ndefer) * 64;
  if (smem > kSmemMax) return cudaErrorInvalidValue;
  static std::atomic<int> configured_dev{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev.load(std::memory_order_relaxed) != dev) {
    cudaError_t e = cudaFuncSetAttribute(eval_ops_kernel<A, 1, SCHEME, 64, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
    if (e != cudaSuccess) return e;
    configured_dev.store(dev, std::memory_order_relaxed);
  }
  const int64_t blocks = (a.npts + 31) / 32;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  eval_ops_kernel<A, 1, SCHEME, 64, true><<<(unsigned)blocks, 64, smem, s>>>(a, o);
  return cudaGetLastError();
}

// multiprocessors of the current device (cached per device)
inline int sm_count() {
  static std::atomic<int> cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return 152; }
  int c = cached[dev].load(std::memory_order_relaxed);
  if (!c) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 152;
    }
    cached[dev].store(n, std::memory_order_relaxed);
    c = n;
  }
  return c;
}

// registers per thread of a kernel (cached per instantiation)
template <class A, int PPT, int SCHEME, int TPB>
int ops_kernel_regs() {
  static std::atomic<int> regs{0};
  int r = regs.load(std::memory_order_relaxed);
  if (!r) {
    cudaFuncAttributes fa;
    r = cudaFuncGetAttributes(&fa, eval_ops_kernel<A, PPT, SCHEME, TPB>) == cudaSuccess && fa.numRegs > 0
            ? fa.numRegs
            : 255;
    cudaGetLastError();
    regs.store(r, std::memory_order_relaxed);
  }
  return r;
}

// Points resident per SM with blocks of tpb threads: shared memory (228 KB
// per SM, 1 KB of it reserved per block), registers (64 K per SM, allocated
// per warp in units of 256), at most 32 blocks and 2048 threads per SM.
inline int64_t ops_resident_points(size_t bytes_per_point, int tpb, int ppt, int regs) {
  const size_t blk = bytes_per_point * (size_t)tpb * ppt;
  if (blk > kSmemMax) return 0;
  const int64_t by_smem = (int64_t)((228 * 1024) / (blk + 1024));
  const int64_t warp_regs = ((int64_t)regs * 32 + 255) / 256 * 256;
  const int64_t by_regs = 65536 / (warp_regs * (tpb / 32));
  const int64_t nb = std::min<int64_t>(std::min<int64_t>(by_smem, by_regs), std::min<int64_t>(32, 2048 / tpb));
  return nb * tpb * ppt;
}

// Block width.  Small grids balance badly over the SMs (a grid of 3.4 blocks
// per SM runs as long as its SMs with 4): one point per thread and fewer than
// 16 blocks of kTPB threads per SM takes narrower blocks (64, or 32 under 4
// per SM), so the remainder is a smaller fraction of each SM's share.  Large
// grids take 64-thread blocks where more points stay resident per SM (the
// per-point table bounds the blocks per SM: a 47 KB block of 128 threads x 2
// points leaves four per SM, a 23.5 KB one of 64 threads nine).  Results do
// not depend on the block width.
template <class A, int PPT, int SCHEME>
cudaError_t launch_eval_ops(const EvalArgs& a, const OpArgs& o, cudaStream_t s) {
  if constexpr (PPT == 1 && SCHEME != 0) {
    // A small grid takes as long as the schedulers (4 per SM) with one warp
    // more than the others: w warps per scheduler cost ceil(w) / w of the
    // balanced time, the split's 2w half-warps ceil(2w) / 2w.  A tree with a
    // split takes it where that gains more than 5 %.
    if (o.split > 0) {
      const double w = (double)((a.npts + 31) / 32) / (4.0 * sm_count());
      if (w > 0 && w < 16 && (std::ceil(w) / w) > 1.05 * (std::ceil(2 * w) / (2 * w)))
        return launch_eval_ops_split<A, SCHEME>(a, o, s);
    }
  }
  if constexpr (PPT == 1) {
    const int64_t blocks = (a.npts + kTPB - 1) / kTPB;
    const int64_t sms = sm_count();
    if (blocks < 4 * sms) return launch_eval_ops_tpb<A, PPT, SCHEME, 32>(a, o, s);
    if (blocks < 16 * sms) return launch_eval_ops_tpb<A, PPT, SCHEME, 64>(a, o, s);
  }
  if constexpr (PPT <= 2) {
    const size_t per_point = sizeof(typename A::pw) * (size_t)o.entries;
    if (ops_resident_points(per_point, 64, PPT, ops_kernel_regs<A, PPT, SCHEME, 64>()) >
        ops_resident_points(per_point, kTPB, PPT, ops_kernel_regs<A, PPT, SCHEME, kTPB>()))
      return launch_eval_ops_tpb<A, PPT, SCHEME, 64>(a, o, s);
  }
  return launch_eval_ops_tpb<A, PPT, SCHEME, kTPB>(a, o, s);
}

// Kernel choice for the fused types: the grouped-op kernel whenever the power
// table fits in shared memory, else the node-by-node kernel (on-the-fly powers).
template <class A, int PPT_OPS, int PPT_NODE>
cudaError_t launch_eval_fused(const EvalArgs& a, const OpArgs& o, int scheme, cudaStream_t s, int variant) {
  const bool ops_ok = ops_smem<A, PPT_OPS>(o) <= kTableSmemCap && o.recs != nullptr;
  if (variant == 1 && !ops_ok) return cudaErrorInvalidValue;
  if (variant != 2 && ops_ok) {
    if (scheme == FP_SCHEME_E) return launch_eval_ops<A, PPT_OPS, FP_SCHEME_E>(a, o, s);
    if (scheme == FP_SCHEME_B)
      return o.ext ? launch_eval_ops<A, PPT_OPS, kSchemeBExt>(a, o, s) : launch_eval_ops<A, PPT_OPS, FP_SCHEME_B>(a, o, s);
    return launch_eval_ops<A, PPT_OPS, 0>(a, o, s);
  }
  return launch_eval_smem<A, PPT_NODE>(a, s);
}

}  // namespace fp
