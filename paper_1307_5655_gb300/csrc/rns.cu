// Exact integer evaluation through residues: the walk modulo several primes
// q = 2^64 - c (c < 2^32), one launch with the primes along blockIdx.y, and
// the Chinese remainder theorem (Garner's mixed-radix form) back to integers.
// The paper's multi-precision experiments (Sec. 3) evaluate integer
// polynomials at integer points; the residues carry the same exact values.
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "eval_kernel.cuh"
#include "tree.hpp"

namespace fp {

// ------------------------------------------------------------- primes (host)
namespace {

uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }
uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = h_mulmod(r, a, m);
    a = h_mulmod(a, a, m);
    e >>= 1;
  }
  return r;
}

// Miller-Rabin with the first twelve prime bases: deterministic below 3.3e24
bool is_prime_u64(uint64_t n) {
  if (n < 2) return false;
  static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (uint64_t p : bases)
    if (n % p == 0) return n == p;
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (uint64_t a : bases) {
    uint64_t x = h_powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool composite = true;
    for (int r = 1; r < s; ++r) {
      x = h_mulmod(x, x, n);
      if (x == n - 1) {
        composite = false;
        break;
      }
    }
    if (composite) return false;
  }
  return true;
}

// c_i of the FP_RNS_MAX_PRIMES largest primes 2^64 - c, in increasing c
const std::vector<uint64_t>& prime_offsets() {
  static std::vector<uint64_t> cs;
  static std::once_flag once;
  std::call_once(once, [] {
    for (uint64_t c = 1; (int)cs.size() < FP_RNS_MAX_PRIMES; c += 2)
      if (is_prime_u64(0 - c)) cs.push_back(c);
  });
  return cs;
}

}  // namespace

uint64_t rns_offset(int i) { return prime_offsets()[i]; }

// ------------------------------------------------------------ device arithmetic
// hi 2^64 + lo mod q, q = 2^64 - c, c < 2^32: 2^64 = c (mod q), so
//   hi 2^64 + lo = lo + hi c;  hi c = t1 2^64 + t0 with t1 < 2^32 (from
//   two 32 x 32 -> 64 products);
//   s = lo + t0 (carry k);  then s + (t1 + k) c, whose product is < 2^64;
//   a carry out of that sum is worth c again (it cannot carry twice);
//   one conditional subtraction of q leaves [0, q).
__device__ __forceinline__ uint64_t modq_reduce(uint64_t lo, uint64_t hi, uint64_t c) {
  // hi c from two 32 x 32 -> 64 products (c < 2^32): h0 c + (h1 c) 2^32
  const uint32_t c32 = (uint32_t)c;
  const uint64_t p0 = (uint64_t)(uint32_t)hi * c32, p1 = (uint64_t)(uint32_t)(hi >> 32) * c32;
  const uint64_t t0 = p0 + (p1 << 32);
  const uint64_t t1 = (p1 >> 32) + (t0 < p0 ? 1ull : 0ull);
  const uint64_t s = lo + t0;
  const uint64_t u = (uint64_t)(uint32_t)t1 * c32 + (s < t0 ? c : 0ull);  // (t1 + carry) c < 2^64
  uint64_t r = s + u;
  if (r < u) r += c;
  const uint64_t q = 0 - c;
  return r >= q ? r - q : r;
}
__device__ __forceinline__ uint64_t modq_mul_add(uint64_t a, uint64_t b, uint64_t d, uint64_t c) {
  uint64_t lo = a * b;
  uint64_t hi = __umul64hi(a, b);
  lo += d;
  hi += lo < d ? 1ull : 0ull;
  return modq_reduce(lo, hi, c);
}

namespace {

__constant__ uint64_t g_rns_c[FP_RNS_MAX_PRIMES];  // c_i of q_i = 2^64 - c_i

// Integers modulo q_y = 2^64 - c_y, y = blockIdx.y (the prime of this block).
// The interface of the MODP policy; exact, so blocks use Horner's rule.
struct MODQ {
  using coef = uint64_t;
  using val = uint64_t;
  using pw = uint64_t;
  static constexpr bool kSlotAtEnd = false;
  static constexpr bool kExact = true;
  static constexpr bool kKindRuns = false;
  static __device__ __forceinline__ uint64_t c() { return g_rns_c[blockIdx.y]; }
  static __device__ __forceinline__ coef coef_from_bits(uint64_t b) { return b; }
  static __device__ __forceinline__ uint64_t mul_add(uint64_t a, uint64_t b, uint64_t d) {
    return modq_mul_add(a, b, d, c());
  }
  static __device__ __forceinline__ pw load_point(const void* pts, int v, int64_t idx, int64_t npts) {
    const uint64_t x = __ldg((const unsigned long long*)pts + (int64_t)v * npts + idx);
    const uint64_t q = 0 - c();
    return x >= q ? x - q : x;
  }
  static __device__ __forceinline__ pw dummy_point() { return 2; }
  static __device__ __forceinline__ pw square(pw a) { return mul_add(a, a, 0); }
  static __device__ __forceinline__ pw mulx(pw a, pw x) { return mul_add(a, x, 0); }
  static __device__ __forceinline__ void node(bool leaf, bool first, coef ca, coef cb, const val* src, val* dst, pw xd) {
    const uint64_t s = leaf ? ca : *src;
    const uint64_t init = first ? cb : *dst;
    *dst = mul_add(s, xd, init);
  }
  static __device__ __forceinline__ val from_coef(coef x) { return x; }
  static __device__ __forceinline__ val mad(val s, pw xd, val init) { return mul_add(s, xd, init); }
  template <bool SC, bool IC, bool X1>
  static __device__ __forceinline__ val mad_k(val s, pw xd, val init) { return mul_add(s, xd, init); }
  static __device__ __forceinline__ val root(bool leaf, coef x, const val* acc) { return leaf ? x : *acc; }
  static __device__ __forceinline__ val apply_root_power(val r, pw xd) { return mul_add(r, xd, 0); }
  static __device__ __forceinline__ void store(void* out, int64_t idx, int64_t, val r) { ((uint64_t*)out)[idx] = r; }
};

// per-prime offsets of the arrays a block of prime y reads and writes
struct RnsStrides {
  int64_t points, out, coef, ops, stream;
  const uint64_t* root_c;  // [k] the root's coefficient per prime
};

__device__ __forceinline__ void rns_slice(EvalArgs& g, OpArgs& o, const RnsStrides& s) {
  const int64_t y = blockIdx.y;
  g.points = (const uint64_t*)g.points + y * s.points;
  g.out = (uint64_t*)g.out + y * s.out;
  g.ca = (const uint64_t*)g.ca + y * s.coef;
  g.cb = (const uint64_t*)g.cb + y * s.coef;
  g.root_c = s.root_c[y];
  o.recs = (const OpRec<uint64_t>*)o.recs + y * s.ops;
  o.stream = (const uint64_t*)o.stream + y * s.stream;
}

template <int PPT, int SCHEME>
__global__ void __launch_bounds__(kTPB) rns_ops_kernel(EvalArgs g, OpArgs o, RnsStrides s) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rns_slice(g, o, s);
  ops_tile<MODQ, PPT, SCHEME>(g, o, (int64_t)blockIdx.x * (kTPB * PPT), smem_raw);
}

template <int PPT, bool TABLE>
__global__ void __launch_bounds__(kTPB) rns_node_kernel(EvalArgs g, OpArgs o, RnsStrides s) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rns_slice(g, o, s);
  node_tile<MODQ, PPT, TABLE>(g, (int64_t)blockIdx.x * (kTPB * PPT), smem_raw);
}

// the offsets table on each device, once
int load_offsets() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FP_E_CUDA;
  }
  std::lock_guard<std::mutex> g(mu);
  if ((int)done.size() <= dev) done.resize(dev + 1, 0);
  if (done[dev]) return FP_OK;
  const std::vector<uint64_t>& cs = prime_offsets();
  if (cudaMemcpyToSymbol(g_rns_c, cs.data(), cs.size() * sizeof(uint64_t)) != cudaSuccess) {
    cudaGetLastError();
    return FP_E_CUDA;
  }
  done[dev] = 1;
  return FP_OK;
}

template <class K>
cudaError_t raise_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
}

}  // namespace

// Launch the walk for all k primes (grid y = prime): the grouped-op kernel
// when its table fits, else node by node (table, or powers on the fly).
int launch_eval_rns(const EvalArgs& a, const OpArgs& o, int scheme, int k, const int64_t* strides,
                    const uint64_t* root_c, cudaStream_t st) {
  int rc = load_offsets();
  if (rc != FP_OK) return rc;
  static std::mutex mu;
  static std::vector<int> configured;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> g(mu);
    if ((int)configured.size() <= dev) configured.resize(dev + 1, 0);
    if (!configured[dev]) {
      cudaError_t e = raise_smem(rns_ops_kernel<1, FP_SCHEME_E>);
      if (e == cudaSuccess) e = raise_smem(rns_ops_kernel<1, FP_SCHEME_B>);
      if (e == cudaSuccess) e = raise_smem(rns_ops_kernel<1, kSchemeBExt>);
      if (e == cudaSuccess) e = raise_smem(rns_ops_kernel<1, 0>);
      if (e == cudaSuccess) e = raise_smem(rns_node_kernel<1, true>);
      if (e == cudaSuccess) e = raise_smem(rns_node_kernel<1, false>);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return FP_E_CUDA;
      }
      configured[dev] = 1;
    }
  }
  RnsStrides s{strides[0], strides[1], strides[2], strides[3], strides[4], root_c};
  const int64_t blocks = (a.npts + kTPB - 1) / kTPB;
  if (blocks > 0x7FFFFFFFLL || k > 65535) return FP_E_TOO_LARGE;
  const dim3 grid((unsigned)blocks, (unsigned)k);
  const size_t ops_smem = sizeof(uint64_t) * (size_t)o.entries * kTPB;
  const size_t table = sizeof(uint64_t) * (size_t)(a.nslot + a.npow) * kTPB;
  const size_t fly = sizeof(uint64_t) * (size_t)(a.nslot + a.nvars) * kTPB;
  if (o.recs && ops_smem <= kTableSmemCap) {
    if (scheme == FP_SCHEME_E) rns_ops_kernel<1, FP_SCHEME_E><<<grid, kTPB, ops_smem, st>>>(a, o, s);
    else if (scheme == FP_SCHEME_B && o.ext) rns_ops_kernel<1, kSchemeBExt><<<grid, kTPB, ops_smem, st>>>(a, o, s);
    else if (scheme == FP_SCHEME_B) rns_ops_kernel<1, FP_SCHEME_B><<<grid, kTPB, ops_smem, st>>>(a, o, s);
    else rns_ops_kernel<1, 0><<<grid, kTPB, ops_smem, st>>>(a, o, s);
  } else if (table <= kTableSmemCap) {
    rns_node_kernel<1, true><<<grid, kTPB, table, st>>>(a, o, s);
  } else if (fly <= kSmemMax) {
    rns_node_kernel<1, false><<<grid, kTPB, fly, st>>>(a, o, s);
  } else {
    return FP_E_TOO_LARGE;
  }
  return cudaGetLastError() == cudaSuccess ? FP_OK : FP_E_CUDA;
}

// ------------------------------------------------------------------- CRT
namespace {

// Garner: digits v_i with X = v_0 + v_1 q_0 + v_2 q_0 q_1 + ...,
//   v_i = (r_i - (v_0 + v_1 q_0 + ... )) / (q_0 ... q_{i-1}) mod q_i,
// computed as t = r_i; t = (t - v_j) q_j^{-1} mod q_i for j < i; then X by
// Horner's rule over the limbs, and X - Q when X > Q/2.
__global__ void k_crt(int k, const uint64_t* __restrict__ res, int64_t npts, const uint64_t* __restrict__ tab,
                      uint64_t* __restrict__ limbs) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npts) return;
  // tab: c[k], inv[k][k] (inv[i][j] = q_j^-1 mod q_i), Q[k], halfQ[k]
  const uint64_t* cs = tab;
  const uint64_t* inv = tab + k;
  const uint64_t* Q = inv + (int64_t)k * k;
  const uint64_t* H = Q + k;
  uint64_t v[FP_RNS_MAX_PRIMES];
  for (int i = 0; i < k; ++i) {
    const uint64_t c = cs[i], q = 0 - c;
    uint64_t t = res[(int64_t)i * npts + j];
    for (int jj = 0; jj < i; ++jj) {
      uint64_t vj = v[jj];
      if (vj >= q) vj -= q;  // v_j < q_j < 2 q_i
      t = t >= vj ? t - vj : t + (q - vj);
      t = modq_mul_add(t, inv[(int64_t)i * k + jj], 0, c);
    }
    v[i] = t;
  }
  uint64_t L[FP_RNS_MAX_PRIMES];
  for (int l = 0; l < k; ++l) L[l] = 0;
  L[0] = v[k - 1];
  int len = 1;
  for (int i = k - 2; i >= 0; --i) {
    const uint64_t q = 0 - cs[i];
    uint64_t carry = v[i];
    for (int l = 0; l < len; ++l) {
      const uint64_t lo = L[l] * q, hi = __umul64hi(L[l], q);
      const uint64_t s = lo + carry;
      carry = hi + (s < lo ? 1ull : 0ull);
      L[l] = s;
    }
    if (carry && len < k) L[len++] = carry;
  }
  // X > Q/2 (limbs from the top): then X - Q, two's complement in k limbs
  bool above = false;
  for (int l = k - 1; l >= 0; --l)
    if (L[l] != H[l]) {
      above = L[l] > H[l];
      break;
    }
  if (above) {
    uint64_t borrow = 0;
    for (int l = 0; l < k; ++l) {
      const uint64_t d = L[l] - Q[l];
      const uint64_t b1 = L[l] < Q[l] ? 1ull : 0ull;
      const uint64_t d2 = d - borrow;
      const uint64_t b2 = d < borrow ? 1ull : 0ull;
      L[l] = d2;
      borrow = b1 | b2;
    }
  }
  for (int l = 0; l < k; ++l) limbs[j * k + l] = L[l];
}

// host tables for the first k primes, uploaded once per (device, k)
const uint64_t* crt_table(int k, int& rc) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, uint64_t*> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    rc = FP_E_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find({dev, k});
  if (it != cache.end()) return it->second;
  const std::vector<uint64_t>& cs = prime_offsets();
  std::vector<uint64_t> h((size_t)k + (size_t)k * k + 2 * (size_t)k, 0);
  for (int i = 0; i < k; ++i) h[i] = cs[i];
  for (int i = 0; i < k; ++i) {
    const uint64_t qi = 0 - cs[i];
    for (int j = 0; j < i; ++j) h[k + (size_t)i * k + j] = h_powmod((0 - cs[j]) % qi, qi - 2, qi);
  }
  // Q = q_0 ... q_{k-1} in k limbs, then Q / 2
  uint64_t* Q = &h[k + (size_t)k * k];
  uint64_t* H = Q + k;
  Q[0] = 1;
  for (int i = 0; i < k; ++i) {
    const uint64_t q = 0 - cs[i];
    uint64_t carry = 0;
    for (int l = 0; l < k; ++l) {
      const unsigned __int128 p = (unsigned __int128)Q[l] * q + carry;
      Q[l] = (uint64_t)p;
      carry = (uint64_t)(p >> 64);
    }
  }
  for (int l = 0; l < k; ++l) H[l] = (Q[l] >> 1) | (l + 1 < k ? Q[l + 1] << 63 : 0);
  uint64_t* d = nullptr;
  if (cudaMalloc((void**)&d, h.size() * sizeof(uint64_t)) != cudaSuccess) {
    cudaGetLastError();
    rc = FP_E_NOMEM;
    return nullptr;
  }
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d);
    rc = FP_E_CUDA;
    return nullptr;
  }
  cache[{dev, k}] = d;
  return d;
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" {

int fp_rns_primes(int k, uint64_t* q) {
  if (k < 1 || k > FP_RNS_MAX_PRIMES || !q) return FP_E_BAD_VALUE;
  const std::vector<uint64_t>& cs = prime_offsets();
  for (int i = 0; i < k; ++i) q[i] = 0 - cs[i];
  return FP_OK;
}

int fp_crt(int k, const uint64_t* residues, int64_t npts, uint64_t* limbs, void* stream) {
  if (k < 1 || k > FP_RNS_MAX_PRIMES || npts < 0) return FP_E_BAD_VALUE;
  if (npts == 0) return FP_OK;
  if (!residues || !limbs) return FP_E_BAD_VALUE;
  int rc = FP_OK;
  const uint64_t* tab = crt_table(k, rc);
  if (!tab) return rc;
  const int64_t blocks = (npts + 127) / 128;
  if (blocks > 0x7FFFFFFFLL) return FP_E_TOO_LARGE;
  k_crt<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(k, residues, npts, tab, limbs);
  return cudaGetLastError() == cudaSuccess ? FP_OK : FP_E_CUDA;
}

}  // extern "C"
