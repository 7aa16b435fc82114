// Batched composition r_j = p_j(q_j(y)) for many pairs (p_j, q_j): the
// coefficient walk of Moroz, Sec. 2.1, run over polynomial values -- the
// paper's "polynomial composition", where elements grow with every product
// (Sec. 1.2, Sec. 3).  All pairs share the tree of p (same terms and scheme),
// so every node step is one batched operation over the pairs:
//     acc[lh(P)] = (c_P if N is P's first child else acc[lh(P)]) + s * q^d(N)
//     s = c_N (leaf) or acc[lh(N)]
// Products are sized to the degrees they involve (the staircase of the
// Estrin scheme at 2^m + 1 terms comes from exactly this), computed
//   MODP: by number-theoretic transforms over p = 2^64 - 2^32 + 1 (roots of
//         unity of order 2^32 exist): in shared memory for lengths <= 4096,
//         by a four-step transform (two passes) above;
//   FP64: on the tensor cores (conv_tc.cu: bf16 slices of 64-coefficient
//         blocks with a block exponent each, exact integer recombination),
//         or by direct convolution for short operands.
// Powers q^d follow the tree's power program (squarings and products by q).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <cstring>
#include <map>
#include <vector>

#include <cuda_runtime.h>

#include "eval_kernel.cuh"
#include "tree.hpp"

namespace fp {

size_t conv_tc_workspace(int alen, int blen, int64_t npairs, int slices);
int conv_tc(const double* a, int64_t a_pitch, int alen, const double* b, int64_t b_pitch, int blen, double* out,
            int64_t out_pitch, int mode, const double* init, int64_t init_pitch, int64_t npairs, void* work,
            int* status, int slices, cudaStream_t st);

// FP64 products: slices per operand on the tensor cores, and the shortest
// operand length that goes to them (shorter ones: direct convolution)
static std::atomic<int> g_f64_slices{7};
static std::atomic<int> g_f64_tc_min{256};

namespace {

constexpr uint64_t kP = 0xFFFFFFFF00000001ull;
constexpr int kNttSmemMax = 4096;  // longest transform done in one block

// ------------------------------------------------------------ mod p (host)
uint64_t h_mul(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) % kP); }
uint64_t h_pow(uint64_t a, uint64_t e) {
  uint64_t r = 1;
  while (e) {
    if (e & 1) r = h_mul(r, a);
    a = h_mul(a, a);
    e >>= 1;
  }
  return r;
}

// ------------------------------------------------------------ mod p (device)
// The transforms are bound by integer ALU issue: the arithmetic mod p works
// on 32-bit halves with the carry flag (MODP::add, MODP::sub, MODP::reduce).
__device__ __forceinline__ uint64_t d_add(uint64_t a, uint64_t b) { return MODP::add(a, b); }
__device__ __forceinline__ uint64_t d_sub(uint64_t a, uint64_t b) { return MODP::sub(a, b); }
__device__ __forceinline__ uint64_t d_mul(uint64_t a, uint64_t b) { return MODP::reduce(a * b, __umul64hi(a, b)); }

// Transforms of `count` vectors of length n held one after the other in
// shared memory, all in lock step.  Forward: decimation in frequency, natural
// order in, bit-reversed order out.  Inverse: decimation in time,
// bit-reversed in, natural out (unscaled).  tw[j] = w^j for the length-n root
// w (inverse table: w^-j), j < n/2.  Two radix-2 stages are fused per pass
// (radix 4: one barrier and one shared-memory round trip per two stages),
// with one radix-2 stage when log2 n is odd.
__device__ __forceinline__ int ilog2_dev(int n) { return 31 - __clz(n); }

// upper_zero: the second half of every input vector is zero (a zero-padded
// product operand), so the first stage's butterflies reduce to (a, a w).
__device__ void ntt_dif(uint64_t* a, int n, int count, const uint64_t* tw, int stride, bool upper_zero = false) {
  // all sizes are powers of two: indices by shifts and masks; vector v starts
  // at a + v * stride (stride >= n)
  const int logn = ilog2_dev(n), lper = logn - 2;
  int lhalf = logn - 1;
  if (upper_zero && lhalf >= 1) {  // first two stages with x[i2] = x[i3] = 0 (half = n / 2: one group)
    __syncthreads();
    const int lq = lhalf - 1, q = 1 << lq;
    for (int e = threadIdx.x; e < (count << lper); e += blockDim.x) {
      const int v = e >> lper, pos = e & ((1 << lper) - 1);
      uint64_t* x = a + v * stride;
      const uint64_t b0 = x[pos], b1 = x[pos + q];
      const uint64_t b2 = d_mul(b0, __ldg(tw + pos)), b3 = d_mul(b1, __ldg(tw + pos + q));
      const uint64_t t = __ldg(tw + (pos << 1));
      x[pos] = d_add(b0, b1);
      x[pos + q] = d_mul(d_sub(b0, b1), t);
      x[pos + 2 * q] = d_add(b2, b3);
      x[pos + 3 * q] = d_mul(d_sub(b2, b3), t);
    }
    lhalf -= 2;
  }
  for (; lhalf >= 1; lhalf -= 2) {  // half = 2^lhalf >= 2: two stages
    __syncthreads();
    const int lq = lhalf - 1, q = 1 << lq;
    const int ls1 = logn - 1 - lhalf, ls2 = logn - lhalf;  // s1 = n / (2 half), s2 = n / half
    for (int e = threadIdx.x; e < (count << lper); e += blockDim.x) {
      const int v = e >> lper, u = e & ((1 << lper) - 1);
      const int grp = u >> lq, pos = u & (q - 1);
      uint64_t* x = a + v * stride + (grp << (lhalf + 1));
      const int i0 = pos, i1 = pos + q, i2 = pos + (1 << lhalf), i3 = pos + (1 << lhalf) + q;
      const uint64_t a0 = x[i0], a1 = x[i1], a2 = x[i2], a3 = x[i3];
      const uint64_t b0 = d_add(a0, a2), b2 = d_mul(d_sub(a0, a2), __ldg(tw + (pos << ls1)));
      const uint64_t b1 = d_add(a1, a3), b3 = d_mul(d_sub(a1, a3), __ldg(tw + ((pos + q) << ls1)));
      const uint64_t t = __ldg(tw + (pos << ls2));
      x[i0] = d_add(b0, b1);
      x[i1] = d_mul(d_sub(b0, b1), t);
      x[i2] = d_add(b2, b3);
      x[i3] = d_mul(d_sub(b2, b3), t);
    }
  }
  if (lhalf == 0) {  // last radix-2 stage: pairs (2g, 2g + 1), twiddle 1
    __syncthreads();
    for (int e = threadIdx.x; e < count * (n >> 1); e += blockDim.x) {
      uint64_t* x = a + (e >> (logn - 1)) * stride + 2 * (e & ((n >> 1) - 1));
      const uint64_t u = x[0], w = x[1];
      x[0] = d_add(u, w);
      x[1] = d_sub(u, w);
    }
  }
  __syncthreads();
}

__device__ void ntt_dit(uint64_t* a, int n, int count, const uint64_t* tw, int stride) {
  const int logn = ilog2_dev(n), lper = logn - 2;
  int lhalf = 0;
  if (n >= 2 && (logn & 1)) {  // first radix-2 stage: pairs (2g, 2g + 1), twiddle 1
    __syncthreads();
    for (int e = threadIdx.x; e < count * (n >> 1); e += blockDim.x) {
      uint64_t* x = a + (e >> (logn - 1)) * stride + 2 * (e & ((n >> 1) - 1));
      const uint64_t u = x[0], w = x[1];
      x[0] = d_add(u, w);
      x[1] = d_sub(u, w);
    }
    lhalf = 1;
  }
  for (; lhalf < logn; lhalf += 2) {  // half = 2^lhalf, 4 half <= n: two stages
    __syncthreads();
    const int half = 1 << lhalf;
    const int ls1 = logn - 1 - lhalf, ls2 = logn - 2 - lhalf;  // s1 = n / (2 half), s2 = n / (4 half)
    for (int e = threadIdx.x; e < (count << lper); e += blockDim.x) {
      const int v = e >> lper, u = e & ((1 << lper) - 1);
      const int grp = u >> lhalf, pos = u & (half - 1);
      uint64_t* x = a + v * stride + (grp << (lhalf + 2));
      const int i0 = pos, i1 = pos + half, i2 = pos + 2 * half, i3 = pos + 3 * half;
      const uint64_t t = __ldg(tw + (pos << ls1));
      const uint64_t a0 = x[i0], a1 = d_mul(x[i1], t), a2 = x[i2], a3 = d_mul(x[i3], t);
      const uint64_t b0 = d_add(a0, a1), b1 = d_sub(a0, a1), b2 = d_add(a2, a3), b3 = d_sub(a2, a3);
      const uint64_t c2 = d_mul(b2, __ldg(tw + (pos << ls2))), c3 = d_mul(b3, __ldg(tw + ((pos + half) << ls2)));
      x[i0] = d_add(b0, c2);
      x[i2] = d_sub(b0, c2);
      x[i1] = d_add(b1, c3);
      x[i3] = d_sub(b1, c3);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------ MODP kernels
// The first outlen coefficients of cnt inverse transforms in sh (vectors of
// length n), scaled by 1/n (SCALE; else the scale is already in them):
// written (mode 0), added into out (mode 1), or written with init[pair] added
// at degree 0 (mode 2).
template <bool SCALE>
__device__ __forceinline__ void store_product(const uint64_t* sh, int n, int cnt, int64_t p0, uint64_t ninv,
                                              uint64_t* out, int64_t out_pitch, int outlen, int mode,
                                              const uint64_t* init, int64_t init_pitch) {
  const int logn = ilog2_dev(n);
  for (int e = threadIdx.x; e < (cnt << logn); e += blockDim.x) {
    const int v = e >> logn, i = e & (n - 1);
    if (i >= outlen) continue;
    uint64_t* o = out + (p0 + v) * out_pitch + i;
    uint64_t val = SCALE ? d_mul(sh[e], ninv) : sh[e];
    if (mode == 1) val = d_add(*o, val);
    else if (mode == 2 && i == 0) val = d_add(val, init[(p0 + v) * init_pitch]);
    *o = val;
  }
}

// Forward transform of length n <= 4096 of src[pair][0..len) zero-padded,
// times `scale`, into dst[pair][0..n); vpb pairs per block.
__global__ void k_ntt_fwd_small(const uint64_t* src, int64_t src_pitch, int len, uint64_t* dst, int64_t dst_pitch,
                                int n, int vpb, int64_t npairs, const uint64_t* tw, uint64_t scale) {
  extern __shared__ uint64_t sh[];
  const int64_t p0 = (int64_t)blockIdx.x * vpb;
  const int cnt = (int)(npairs - p0 < vpb ? npairs - p0 : vpb);
  const int logn = ilog2_dev(n);
  for (int e = threadIdx.x; e < vpb * n; e += blockDim.x) {
    const int v = e >> logn, i = e & (n - 1);
    sh[e] = (v < cnt && i < len) ? src[(p0 + v) * src_pitch + i] : 0;
  }
  ntt_dif(sh, n, vpb, tw, n, 2 * len <= n);
  for (int e = threadIdx.x; e < cnt * n; e += blockDim.x) {
    const int v = e >> logn, i = e & (n - 1);
    dst[(p0 + v) * dst_pitch + i] = scale == 1 ? sh[e] : d_mul(sh[e], scale);
  }
}

// Inverse of a product: F(A) (in `prod`) times F(B) (`fb`), inverse
// transform, scaled by 1/n; the first `outlen` coefficients are written
// (mode 0), added into out (mode 1), or written with init[pair] added at
// degree 0 (mode 2).
__global__ void k_ntt_mul_inv_small(const uint64_t* prod, int64_t pitch, const uint64_t* fb, int64_t fb_pitch, int n,
                                    int vpb, int64_t npairs, const uint64_t* twi, uint64_t ninv, uint64_t* out,
                                    int64_t out_pitch, int outlen, int mode, const uint64_t* init, int64_t init_pitch) {
  extern __shared__ uint64_t sh[];
  const int64_t p0 = (int64_t)blockIdx.x * vpb;
  const int cnt = (int)(npairs - p0 < vpb ? npairs - p0 : vpb);
  const int logn = ilog2_dev(n);
  for (int e = threadIdx.x; e < vpb * n; e += blockDim.x) {
    const int v = e >> logn, i = e & (n - 1);
    sh[e] = v < cnt ? d_mul(prod[(p0 + v) * pitch + i], fb[(p0 + v) * fb_pitch + i]) : 0;
  }
  ntt_dit(sh, n, vpb, twi, n);
  store_product<true>(sh, n, cnt, p0, ninv, out, out_pitch, outlen, mode, init, init_pitch);
}

// A whole product for n <= 4096, one launch: transform of src (first len
// coefficients, zero-padded), times the cached transform fb (which carries
// the 1/n of the inverse), inverse, written per mode as in
// k_ntt_mul_inv_small.  src may be the destination: a block reads its rows
// completely before writing them.
__global__ void k_ntt_product_small(const uint64_t* src, int64_t src_pitch, int len, const uint64_t* fb,
                                    int64_t fb_pitch, int n, int vpb, int64_t npairs, const uint64_t* tw,
                                    const uint64_t* twi, uint64_t* out, int64_t out_pitch, int outlen, int mode,
                                    const uint64_t* init, int64_t init_pitch) {
  extern __shared__ uint64_t sh[];
  const int64_t p0 = (int64_t)blockIdx.x * vpb;
  const int cnt = (int)(npairs - p0 < vpb ? npairs - p0 : vpb);
  const int logn = ilog2_dev(n);
  for (int e = threadIdx.x; e < vpb * n; e += blockDim.x) {
    const int v = e >> logn, i = e & (n - 1);
    sh[e] = (v < cnt && i < len) ? src[(p0 + v) * src_pitch + i] : 0;
  }
  ntt_dif(sh, n, vpb, tw, n, 2 * len <= n);
  for (int e = threadIdx.x; e < vpb * n; e += blockDim.x) {
    const int v = e >> logn, i = e & (n - 1);
    if (v < cnt) sh[e] = d_mul(sh[e], fb[(p0 + v) * fb_pitch + i]);
  }
  ntt_dit(sh, n, vpb, twi, n);
  store_product<false>(sh, n, cnt, p0, 1, out, out_pitch, outlen, mode, init, init_pitch);
}

// Four-step transform of length n = R * C (R, C <= 4096), vector x[C n1 + n2].
// Column pass: a tile of TC columns (length R, stride C) per block, all
// transformed together; forward multiplies by w_n^(k1 n2) afterwards,
// inverse divides before.  Row pass: rows of length C, contiguous.  Position
// r of a transformed column holds k1 = bitrev(r), so the twiddle of element
// r C + n2 is tw4[r C + n2] = w_n^(+-bitrev(r) n2): a table in the layout of
// the data, read with the same coalesced pattern as the data (the inverse
// table also carries the 1/n of the inverse transform).
__global__ void k_ntt_cols(const uint64_t* src, int64_t src_pitch, int len, uint64_t* dst, int64_t dst_pitch, int R,
                           int C, int TC, const uint64_t* twR, const uint64_t* tw4, int inverse, int outlen, int mode,
                           const uint64_t* init, int64_t init_pitch) {
  extern __shared__ uint64_t sh[];  // [TC][R + 1]: the padding spreads a transposed row over the banks
  const int RS = R + 1;
  const int tiles = C / TC;
  const int64_t pr = blockIdx.x / tiles;
  const int c0 = (blockIdx.x % tiles) * TC;  // R, C, TC: powers of two
  const int lTC = ilog2_dev(TC);
  for (int e = threadIdx.x; e < R * TC; e += blockDim.x) {
    const int r = e >> lTC, c = e & (TC - 1);
    const int idx = r * C + c0 + c;
    uint64_t v = idx < len ? src[pr * src_pitch + idx] : 0;
    if (inverse) v = d_mul(v, __ldg(tw4 + idx));  // undo w^(k1 n2)
    sh[c * RS + r] = v;
  }
  if (inverse) ntt_dit(sh, R, TC, twR, RS);
  else ntt_dif(sh, R, TC, twR, RS, 2 * (int64_t)len <= (int64_t)R * C);  // rows r >= R/2 hold indices >= len
  for (int e = threadIdx.x; e < R * TC; e += blockDim.x) {
    const int r = e >> lTC, c = e & (TC - 1);
    const int idx = r * C + c0 + c;
    uint64_t v = sh[c * RS + r];
    if (!inverse) {
      dst[pr * dst_pitch + idx] = d_mul(v, __ldg(tw4 + idx));
    } else if (idx < outlen) {
      uint64_t* o = dst + pr * dst_pitch + idx;
      if (mode == 1) v = d_add(*o, v);
      else if (mode == 2 && idx == 0) v = d_add(v, init[pr * init_pitch]);
      *o = v;
    }
  }
}

// forward row pass: rows (length C) of data[pair][R][C], vpb rows per block
__global__ void k_ntt_rows(uint64_t* data, int64_t pitch, int R, int C, int vpb, const uint64_t* twC) {
  extern __shared__ uint64_t sh[];
  const int per_pair = R / vpb;
  const int64_t pr = blockIdx.x / per_pair;
  const int r0 = (blockIdx.x % per_pair) * vpb;
  uint64_t* rows = data + pr * pitch + (int64_t)r0 * C;
  for (int e = threadIdx.x; e < vpb * C; e += blockDim.x) sh[e] = rows[e];
  ntt_dif(sh, C, vpb, twC, C);
  for (int e = threadIdx.x; e < vpb * C; e += blockDim.x) rows[e] = sh[e];
}

// The row pass of a whole product: rows of the column-transformed A
// (data[pair][R][C], vpb rows per block) are transformed forward, multiplied
// by the matching rows of the transform fb, and transformed back, in shared
// memory: one pass over the data instead of a forward and an inverse pass.
__global__ void k_ntt_rows_product(uint64_t* data, int64_t pitch, int R, int C, int vpb, const uint64_t* twC,
                                   const uint64_t* twCi, const uint64_t* fb, int64_t fb_pitch) {
  extern __shared__ uint64_t sh[];
  const int per_pair = R / vpb;
  const int64_t pr = blockIdx.x / per_pair;
  const int r0 = (blockIdx.x % per_pair) * vpb;
  uint64_t* rows = data + pr * pitch + (int64_t)r0 * C;
  const uint64_t* frows = fb + pr * fb_pitch + (int64_t)r0 * C;
  for (int e = threadIdx.x; e < vpb * C; e += blockDim.x) sh[e] = rows[e];
  ntt_dif(sh, C, vpb, twC, C);
  for (int e = threadIdx.x; e < vpb * C; e += blockDim.x) sh[e] = d_mul(sh[e], frows[e]);
  ntt_dit(sh, C, vpb, twCi, C);
  for (int e = threadIdx.x; e < vpb * C; e += blockDim.x) rows[e] = sh[e];
}

// leaf step: dst[0..len) = (init at degree 0 if first) + c[pair] * q^d
template <class T>
__global__ void k_leaf(T* dst, int64_t dst_pitch, const T* qd, int64_t q_pitch, int len, const T* c, int64_t c_pitch,
                       int first, const T* init, int64_t init_pitch, int64_t npairs) {
  const int64_t total = npairs * (int64_t)len;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / len;
    const int i = (int)(e - pr * len);
    const T cv = c[pr * c_pitch];
    const T qv = qd[pr * q_pitch + i];
    T* o = dst + pr * dst_pitch + i;
    const T base = first ? ((i == 0 && init) ? init[pr * init_pitch] : T(0)) : *o;
    if constexpr (std::is_same<T, uint64_t>::value) *o = MODP::mul_add(cv, qv, base);
    else *o = fma(cv, qv, base);
  }
}

// FP64 product by direct convolution, out[j] = sum_i a[i] b[j-i] for
// j < outlen, written, accumulated or initialised as k_ntt_mul_inv_small.
__global__ void k_conv_f64(const double* a, int64_t a_pitch, int alen, const double* b, int64_t b_pitch, int blen,
                           double* out, int64_t out_pitch, int outlen, int mode, const double* init,
                           int64_t init_pitch, int tiles) {
  const int64_t pr = blockIdx.x / tiles;
  const int j = (blockIdx.x % tiles) * blockDim.x + threadIdx.x;
  if (j >= outlen) return;
  const double* ap = a + pr * a_pitch;
  const double* bp = b + pr * b_pitch;
  const int lo = j - blen + 1 > 0 ? j - blen + 1 : 0;
  const int hi = j < alen - 1 ? j : alen - 1;
  double s = 0.0;
  for (int i = lo; i <= hi; ++i) s = fma(ap[i], bp[j - i], s);
  double* o = out + pr * out_pitch + j;
  if (mode == 1) s += *o;
  else if (mode == 2 && j == 0) s += init[pr * init_pitch];
  *o = s;
}

// per-pair node coefficients: cn[pair][node] = coefficient of that node's term
template <class T>
__global__ void k_gather_coeffs(const T* pc, int64_t row_pitch, const int64_t* term_of_node, int64_t nnodes,
                                T* cn, int64_t npairs, int reduce_modp) {
  const int64_t total = npairs * nnodes;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / nnodes, i = e - pr * nnodes;
    const int64_t t = term_of_node[i];
    T v = t >= 0 ? pc[pr * row_pitch + t] : T(0);
    if constexpr (std::is_same<T, uint64_t>::value) {
      if (reduce_modp && v >= kP) v -= kP;
    }
    cn[e] = v;
  }
}

template <class T>
__global__ void k_copy_rows(const T* src, int64_t src_pitch, T* dst, int64_t dst_pitch, int len, int64_t npairs,
                            int reduce_modp) {
  const int64_t total = npairs * (int64_t)len;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / len;
    const int i = (int)(e - pr * len);
    T v = src[pr * src_pitch + i];
    if constexpr (std::is_same<T, uint64_t>::value) {
      if (reduce_modp && v >= kP) v -= kP;
    }
    dst[pr * dst_pitch + i] = v;
  }
}

template <class T>
__global__ void k_fill_zero(T* dst, int64_t pitch, int from, int len, int64_t npairs) {
  const int64_t w = len - from;
  const int64_t total = npairs * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pr = e / w;
    dst[pr * pitch + from + (e - pr * w)] = T(0);
  }
}

int grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}


// ------------------------------------------------------------ host plan
struct Buf {
  void* ptr = nullptr;
  int64_t pitch = 0;  // elements per pair
};

struct Composer {
  const fp_tree* t;
  int dtype;  // FP_MODP or FP_F64
  int degq;
  int64_t npairs;
  cudaStream_t st;
  int status = FP_OK;
  std::vector<void*> owned;
  // twiddles (MODP): forward/inverse powers of w_n for every length n used
  std::map<int, std::pair<uint64_t*, uint64_t*>> tw;
  // four-step twiddle tables (forward, inverse) per length n > 4096, n entries each
  std::map<int, std::pair<uint64_t*, uint64_t*>> tw4;
  // when set, work space is carved from this caller-provided region instead
  // of being allocated (fp_compose_noalloc)
  unsigned char* arena = nullptr;
  size_t arena_cap = 0, arena_used = 0;
  // dry run: every buffer is only counted (arena_used, 256-byte granules) and
  // nothing is launched, copied or computed -- the one account of the work
  // space, since the same driver code decides every buffer
  bool dry = false;
  bool live() const { return !dry && status == FP_OK; }
  int sms = 0;  // multiprocessors of the current device

  // vectors of length n <= 4096 per block of an in-shared-memory transform:
  // as many as fill 1024 elements (256 threads, one radix-4 butterfly each
  // per stage: the transforms of one product are a single partial wave, so
  // threads rather than work per thread hide the latencies), fewer when that
  // would leave the device with under two blocks per multiprocessor (short
  // transforms of few pairs)
  int small_vpb(int n) {
    if (sms == 0) {
      int dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 1;
      }
    }
    int vpb = std::max(1, 1024 / n);
    while (vpb > 1 && (npairs + vpb - 1) / vpb < 2 * (int64_t)sms) vpb >>= 1;
    return vpb;
  }
  // threads of such a block: one per radix-4 butterfly, 32 to 256
  static int small_threads(int vpb, int n) { return std::max(32, std::min(256, vpb * n / 4)); }

  void* alloc(size_t bytes) {
    void* p = nullptr;
    if (status != FP_OK) return nullptr;
    if (dry) {  // a distinct, never dereferenced stand-in address per buffer
      arena_used += (bytes + 255) & ~(size_t)255;
      return (void*)(uintptr_t)arena_used;
    }
    if (arena) {
      const size_t sz = (bytes + 255) & ~(size_t)255;
      if (arena_used + sz > arena_cap) {
        status = FP_E_TOO_LARGE;
        return nullptr;
      }
      p = arena + arena_used;
      arena_used += sz;
      return p;
    }
    if (pool_alloc(&p, bytes < 16 ? 16 : bytes, st) != cudaSuccess) {
      cudaGetLastError();
      status = FP_E_NOMEM;
      return nullptr;
    }
    owned.push_back(p);
    return p;
  }
  void release() {
    for (void* p : owned) cudaFreeAsync(p, st);
    owned.clear();
  }
  void check() {
    if (!dry && status == FP_OK && cudaGetLastError() != cudaSuccess) status = FP_E_CUDA;
  }

  std::pair<uint64_t*, uint64_t*> twiddles(int n) {
    auto it = tw.find(n);
    if (it != tw.end()) return it->second;
    if (dry) return tw[n] = {(uint64_t*)alloc(n * 8), (uint64_t*)alloc(n * 8)};
    std::vector<uint64_t> f(n), b(n);
    const uint64_t w = h_pow(7, (kP - 1) / (uint64_t)n);  // 7 generates (Z/pZ)^*
    const uint64_t wi = h_pow(w, kP - 2);
    uint64_t x = 1, y = 1;
    for (int j = 0; j < n; ++j) {
      f[j] = x;
      b[j] = y;
      x = h_mul(x, w);
      y = h_mul(y, wi);
    }
    uint64_t* df = (uint64_t*)alloc(n * 8);
    uint64_t* db = (uint64_t*)alloc(n * 8);
    if (status == FP_OK) {
      cudaMemcpyAsync(df, f.data(), n * 8, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(db, b.data(), n * 8, cudaMemcpyHostToDevice, st);
      // the host vectors must outlive the copies: wait for them
      cudaStreamSynchronize(st);
    }
    tw[n] = {df, db};
    return tw[n];
  }

  // the four-step twiddles of length n = R C in the layout of the data:
  // forward [r C + n2] = w^(bitrev(r) n2), inverse w^-(bitrev(r) n2) / n (the
  // inverse transform's scaling rides on its twiddle)
  std::pair<uint64_t*, uint64_t*> four_step_twiddles(int n) {
    auto it = tw4.find(n);
    if (it != tw4.end()) return it->second;
    if (dry) return tw4[n] = {(uint64_t*)alloc(n * 8), (uint64_t*)alloc(n * 8)};
    int R, C;
    split(n, R, C);
    int logR = 0;
    while ((1 << logR) < R) ++logR;
    std::vector<uint64_t> f(n), b(n);
    const uint64_t w = h_pow(7, (kP - 1) / (uint64_t)n);
    const uint64_t wi = h_pow(w, kP - 2), ninv = h_pow((uint64_t)n, kP - 2);
    for (int r = 0; r < R; ++r) {
      int k1 = 0;  // bitrev(r) over logR bits
      for (int j = 0; j < logR; ++j) k1 |= ((r >> j) & 1) << (logR - 1 - j);
      const uint64_t uf = h_pow(w, (uint64_t)k1), ub = h_pow(wi, (uint64_t)k1);
      uint64_t x = 1, y = ninv;
      for (int c = 0; c < C; ++c) {
        f[(size_t)r * C + c] = x;
        b[(size_t)r * C + c] = y;
        x = h_mul(x, uf);
        y = h_mul(y, ub);
      }
    }
    uint64_t* df = (uint64_t*)alloc(n * 8);
    uint64_t* db = (uint64_t*)alloc(n * 8);
    if (status == FP_OK) {
      cudaMemcpyAsync(df, f.data(), n * 8, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(db, b.data(), n * 8, cudaMemcpyHostToDevice, st);
      cudaStreamSynchronize(st);  // the host vectors must outlive the copies
    }
    tw4[n] = {df, db};
    return tw4[n];
  }

  static void split(int n, int& R, int& C) {
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    C = 1 << ((lg + 1) / 2);
    R = n / C;
  }

  // forward transform of length n of src (first len coefficients) into dst;
  // for n <= 4096 times `scale`
  void fwd(const Buf& src, int len, const Buf& dst, int n, uint64_t scale = 1) {
    if (status != FP_OK) return;
    if (n <= kNttSmemMax) {
      auto w = twiddles(n);
      if (!live()) return;
      const int vpb = small_vpb(n);
      k_ntt_fwd_small<<<(unsigned)((npairs + vpb - 1) / vpb), small_threads(vpb, n), (size_t)vpb * n * 8, st>>>(
          (const uint64_t*)src.ptr, src.pitch, len, (uint64_t*)dst.ptr, dst.pitch, n, vpb, npairs, w.first, scale);
    } else {
      int R, C;
      split(n, R, C);
      const int TC = kNttSmemMax / R;
      auto wR = twiddles(R);
      auto wC = twiddles(C);
      auto w4 = four_step_twiddles(n);
      if (!live()) return;
      k_ntt_cols<<<(unsigned)(npairs * (C / TC)), 256, (size_t)(R + 1) * TC * 8, st>>>(
          (const uint64_t*)src.ptr, src.pitch, len, (uint64_t*)dst.ptr, dst.pitch, R, C, TC, wR.first, w4.first, 0, 0,
          0, nullptr, 0);
      const int vpb = kNttSmemMax / C;
      k_ntt_rows<<<(unsigned)(npairs * (R / vpb)), 256, (size_t)vpb * C * 8, st>>>(
          (uint64_t*)dst.ptr, dst.pitch, R, C, vpb, wC.first);
    }
    check();
  }

  // out = first outlen coefficients of A * B for n > 4096, per mode, given
  // fb = F(B): column pass of A into work, one row pass for the forward
  // transform, the product and the inverse, inverse column pass into out
  void product_large(const Buf& a, int len, const Buf& fbuf, const Buf& work, int n, const Buf& out, int outlen,
                     int mode, const uint64_t* init, int64_t init_pitch) {
    if (status != FP_OK) return;
    int R, C;
    split(n, R, C);
    const int TC = kNttSmemMax / R;
    auto wR = twiddles(R);
    auto wC = twiddles(C);
    auto w4 = four_step_twiddles(n);
    if (!live()) return;
    k_ntt_cols<<<(unsigned)(npairs * (C / TC)), 256, (size_t)(R + 1) * TC * 8, st>>>(
        (const uint64_t*)a.ptr, a.pitch, len, (uint64_t*)work.ptr, work.pitch, R, C, TC, wR.first, w4.first, 0, 0, 0,
        nullptr, 0);
    const int vpb = kNttSmemMax / C;
    k_ntt_rows_product<<<(unsigned)(npairs * (R / vpb)), 256, (size_t)vpb * C * 8, st>>>(
        (uint64_t*)work.ptr, work.pitch, R, C, vpb, wC.first, wC.second, (const uint64_t*)fbuf.ptr, fbuf.pitch);
    k_ntt_cols<<<(unsigned)(npairs * (C / TC)), 256, (size_t)(R + 1) * TC * 8, st>>>(
        (const uint64_t*)work.ptr, work.pitch, n, (uint64_t*)out.ptr, out.pitch, R, C, TC, wR.second, w4.second, 1,
        outlen, mode, init, init_pitch);
    check();
  }

  // out = first outlen coefficients of inverse(F(A) * F(B)) for n <= 4096,
  // per mode (longer products go through product_large)
  void mul_inv(const Buf& fa, const Buf& fbuf, int n, const Buf& out, int outlen, int mode, const uint64_t* init,
               int64_t init_pitch) {
    if (status != FP_OK) return;
    auto w = twiddles(n);
    if (!live()) return;
    const uint64_t ninv = h_pow((uint64_t)n, kP - 2);
    const int vpb = small_vpb(n);
    k_ntt_mul_inv_small<<<(unsigned)((npairs + vpb - 1) / vpb), small_threads(vpb, n), (size_t)vpb * n * 8, st>>>(
        (const uint64_t*)fa.ptr, fa.pitch, (const uint64_t*)fbuf.ptr, fbuf.pitch, n, vpb, npairs, w.second, ninv,
        (uint64_t*)out.ptr, out.pitch, outlen, mode, init, init_pitch);
    check();
  }
};

int64_t next_pow2(int64_t x) {
  int64_t n = 1;
  while (n < x) n <<= 1;
  return n;
}

}  // namespace

// Composition entry (declared in capi.cu).
// With dry_bytes non-NULL nothing is launched, copied or allocated: the call
// only writes the bytes of work space the same arguments would use (buffers
// rounded up to 256 bytes, as the allocation-free entry carves them).
int compose_device(const fp_tree* t, fp_dtype dtype, const void* pcoeffs, const void* q, int32_t degq, int64_t npairs,
                   void* out, cudaStream_t st, unsigned char* arena = nullptr, size_t arena_cap = 0,
                   size_t* dry_bytes = nullptr) {
  if (!t || !q || !out || degq < 0 || npairs < 0) return FP_E_BAD_VALUE;
  if (t->nvars != 1) return FP_E_BAD_VALUE;
  if (dtype == FP_MODP ? t->coeff_type != FP_MODP : (dtype != FP_F64 || t->coeff_type != FP_F64)) return FP_E_DTYPE;
  if (t->dev.device < 0 && !dry_bytes) return FP_E_DTYPE;  // a dry run needs no device copy
  if (npairs == 0) {
    if (dry_bytes) *dry_bytes = 0;
    return FP_OK;
  }
  const bool modp = dtype == FP_MODP;
  const int64_t N = t->nnodes;
  const int64_t dmax = N > 0 ? t->node_e[0] : 0;  // degree of p (node 0 is the highest term)
  const int64_t outlen = dmax * (int64_t)degq + 1;
  const size_t esz = 8;
  if (outlen > (1 << 26)) return FP_E_TOO_LARGE;
  Composer cm{t, dtype, degq, npairs, st};
  cm.arena = arena;
  cm.arena_cap = arena_cap;
  cm.dry = dry_bytes != nullptr;
  if (cm.dry) *dry_bytes = 0;
  Buf outb{out, outlen};
  if (N == 0) {  // zero polynomial
    if (cm.dry) return FP_OK;
    k_fill_zero<uint64_t><<<grid_for(npairs * outlen), 256, 0, st>>>((uint64_t*)out, outlen, 0, (int)outlen, npairs);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_E_CUDA;
  }
  // ---- node coefficients per pair: cn[pair][node]
  Buf cn{cm.alloc(npairs * N * esz), N};
  {
    int64_t* d_map = (int64_t*)cm.alloc(N * 8);
    void* d_pc = nullptr;
    std::vector<uint64_t> own;
    if (!pcoeffs) {  // the tree's own coefficients, one row shared by every pair
      own.assign(t->nterms_in, 0);
      for (int64_t i = 0; i < N; ++i)
        if (t->term_of_node[i] >= 0) {
          if (modp) own[t->term_of_node[i]] = t->c_u64[i];
          else std::memcpy(&own[t->term_of_node[i]], &t->c_f64[i], 8);
        }
      d_pc = cm.alloc(own.size() * 8);
    }
    if (cm.status != FP_OK) { cm.release(); return cm.status; }
    if (cm.live()) {
      cudaMemcpyAsync(d_map, t->term_of_node.data(), N * 8, cudaMemcpyHostToDevice, st);
      if (!pcoeffs) cudaMemcpyAsync(d_pc, own.data(), own.size() * 8, cudaMemcpyHostToDevice, st);
      // term_of_node indexes the caller's input order (rows of nterms_in)
      const int64_t row = pcoeffs ? t->nterms_in : 0;
      if (modp)
        k_gather_coeffs<uint64_t><<<grid_for(npairs * N), 256, 0, st>>>(
            (const uint64_t*)(pcoeffs ? pcoeffs : d_pc), row, d_map, N, (uint64_t*)cn.ptr, npairs, 1);
      else
        k_gather_coeffs<double><<<grid_for(npairs * N), 256, 0, st>>>(
            (const double*)(pcoeffs ? pcoeffs : d_pc), row, d_map, N, (double*)cn.ptr, npairs, 0);
      cm.check();
      cudaStreamSynchronize(st);  // the host vectors above must outlive their copies
    }
  }
  // ---- degrees of node values: deg(N) = degq * (max exponent in subtree - e(N))
  std::vector<int64_t> maxe(N);
  for (int64_t i = 0; i < N; ++i) maxe[i] = t->node_e[i];
  for (int64_t i = 0; i + 1 < N; ++i) maxe[t->parent[i]] = std::max(maxe[t->parent[i]], maxe[i]);
  auto degval = [&](int64_t i) { return (maxe[i] - t->node_e[i]) * (int64_t)degq; };
  std::vector<int64_t> cap(t->max_lh + 1, 1);
  for (int64_t i = 0; i < N; ++i) cap[t->lh[i]] = std::max(cap[t->lh[i]], degval(i) + 1);
  std::vector<Buf> acc(cap.size());
  for (size_t s = 0; s < cap.size(); ++s) acc[s] = Buf{cm.alloc(npairs * cap[s] * esz), cap[s]};
  // ---- powers q^d (coefficient form) by the tree's power program
  const int npow = (int)t->pow_prog.size();
  std::vector<Buf> qp(npow);
  int64_t maxprod = 1;
  for (int k = 0; k < npow; ++k) qp[k] = Buf{cm.alloc(npairs * (t->pow_deg[k] * degq + 1) * esz), t->pow_deg[k] * degq + 1};
  for (int64_t i = 0; i + 1 < N; ++i) maxprod = std::max(maxprod, degval(i) + t->pd[i] * degq + 1);
  for (int k = 0; k < npow; ++k) maxprod = std::max(maxprod, t->pow_deg[k] * degq + 1);
  const int64_t Lmax = modp ? next_pow2(maxprod) : maxprod;
  Buf ta{cm.alloc(npairs * Lmax * esz), Lmax}, tb{cm.alloc(npairs * Lmax * esz), Lmax};
  // FP64 products on the tensor cores: one work buffer for the longest
  // operands (A: slots and powers, B: powers; the work space grows with both)
  const int slices = g_f64_slices.load(), tc_min = g_f64_tc_min.load();
  int64_t maxA = 1, maxB = 1;
  for (size_t s = 0; s < cap.size(); ++s) maxA = std::max(maxA, cap[s]);
  for (int k = 0; k < npow; ++k) maxB = std::max(maxB, qp[k].pitch);
  maxA = std::max(maxA, maxB);
  const bool tc_any = !modp && tc_min > 0 && maxB >= tc_min;
  void* tcw = nullptr;
  int* tc_status = nullptr;
  if (tc_any) {
    tcw = cm.alloc(conv_tc_workspace((int)maxA, (int)maxB, npairs, slices));
    tc_status = (int*)cm.alloc(sizeof(int));
    if (cm.live() && cudaMemsetAsync(tc_status, 0, sizeof(int), st) != cudaSuccess) cm.status = FP_E_CUDA;
  }
  if (cm.status != FP_OK) { cm.release(); return cm.status; }
  // transforms of the powers q^d at the lengths they are used at; for
  // n <= 4096 (used only by the fused product kernel) times 1/n, the scaling
  // of the products' inverse transforms
  std::map<std::pair<int, int64_t>, Buf> qhat;
  auto qhat_of = [&](int k, int64_t n) -> Buf {
    auto key = std::make_pair(k, n);
    auto it = qhat.find(key);
    if (it != qhat.end()) return it->second;
    Buf b{cm.alloc(npairs * n * esz), n};
    cm.fwd(qp[k], (int)qp[k].pitch, b, (int)n, n <= kNttSmemMax ? h_pow((uint64_t)n, kP - 2) : 1);
    qhat[key] = b;
    return b;
  };
  // product helper: dst (per mode) = A[0..alen) * B[0..blen); B = q^d when bk >= 0
  auto product = [&](const Buf& A, int64_t alen, const Buf& B, int64_t blen, int bk, const Buf& dst, int mode,
                     const void* init, int64_t init_pitch) {
    const int64_t rl = alen + blen - 1;
    if (modp) {
      const int n = (int)next_pow2(rl);
      if (bk >= 0 && n <= kNttSmemMax) {  // one fused launch
        const Buf fb = qhat_of(bk, n);
        auto w = cm.twiddles(n);
        if (!cm.live()) return;
        const int vpb = cm.small_vpb(n);
        k_ntt_product_small<<<(unsigned)((npairs + vpb - 1) / vpb), cm.small_threads(vpb, n), (size_t)vpb * n * 8, st>>>(
            (const uint64_t*)A.ptr, A.pitch, (int)alen, (const uint64_t*)fb.ptr, fb.pitch, n, vpb, npairs, w.first,
            w.second, (uint64_t*)dst.ptr, dst.pitch, (int)rl, mode, (const uint64_t*)init, init_pitch);
        cm.check();
        return;
      }
      if (n > kNttSmemMax) {
        Buf fb = tb;
        if (bk >= 0) fb = qhat_of(bk, n);
        else cm.fwd(B, (int)blen, tb, n);
        if (cm.status != FP_OK) return;
        cm.product_large(A, (int)alen, fb, ta, n, dst, (int)rl, mode, (const uint64_t*)init, init_pitch);
        return;
      }
      cm.fwd(A, (int)alen, ta, n);
      Buf fb = tb;
      if (bk >= 0) fb = qhat_of(bk, n);
      else cm.fwd(B, (int)blen, tb, n);
      if (cm.status != FP_OK) return;
      cm.mul_inv(ta, fb, n, dst, (int)rl, mode, (const uint64_t*)init, init_pitch);
    } else {
      if (!cm.live()) return;
      if (tc_any && alen >= tc_min && blen >= tc_min) {
        // the longer operand as the rows (fewer empty rows per tile); both
        // are sliced before the product is written, so dst may be A
        const bool swap = alen < blen;
        const int rc = conv_tc((const double*)(swap ? B.ptr : A.ptr), swap ? B.pitch : A.pitch,
                               (int)(swap ? blen : alen), (const double*)(swap ? A.ptr : B.ptr),
                               swap ? A.pitch : B.pitch, (int)(swap ? alen : blen), (double*)dst.ptr, dst.pitch,
                               mode, (const double*)init, init_pitch, npairs, tcw, tc_status, slices, st);
        if (rc != FP_OK) cm.status = rc;
        cm.check();
        return;
      }
      // the source may be the destination slot: convolve from a copy
      k_copy_rows<double><<<grid_for(npairs * alen), 256, 0, st>>>((const double*)A.ptr, A.pitch, (double*)ta.ptr,
                                                                    ta.pitch, (int)alen, npairs, 0);
      const int tiles = (int)((rl + 255) / 256);
      k_conv_f64<<<(unsigned)(npairs * tiles), 256, 0, st>>>((const double*)ta.ptr, ta.pitch, (int)alen,
                                                            (const double*)B.ptr, B.pitch, (int)blen,
                                                            (double*)dst.ptr, dst.pitch, (int)rl, mode,
                                                            (const double*)init, init_pitch, tiles);
      cm.check();
    }
  };
  for (int k = 0; k < npow && cm.status == FP_OK; ++k) {
    const uint32_t w = t->pow_prog[k];
    const uint32_t op = w & 3u, a1 = (w >> 2) & 0x7FFFu, a2 = w >> 17;
    if (op == kPowLoad) {
      if (cm.dry) continue;
      if (modp) k_copy_rows<uint64_t><<<grid_for(npairs * (degq + 1)), 256, 0, st>>>(
          (const uint64_t*)q, degq + 1, (uint64_t*)qp[k].ptr, qp[k].pitch, degq + 1, npairs, 1);
      else k_copy_rows<double><<<grid_for(npairs * (degq + 1)), 256, 0, st>>>(
          (const double*)q, degq + 1, (double*)qp[k].ptr, qp[k].pitch, degq + 1, npairs, 0);
      cm.check();
    } else if (op == kPowSq) {
      product(qp[a1], qp[a1].pitch, qp[a1], qp[a1].pitch, (int)a1, qp[k], 0, nullptr, 0);
    } else {
      product(qp[a1], qp[a1].pitch, qp[a2], qp[a2].pitch, (int)a2, qp[k], 0, nullptr, 0);
    }
  }
  // ---- the walk
  std::vector<uint8_t> has_child(N, 0), seen(N, 0);
  for (int64_t i = 0; i + 1 < N; ++i) has_child[t->parent[i]] = 1;
  std::map<std::pair<int32_t, int64_t>, int> pid;
  for (int k = 0; k < npow; ++k) pid[{t->pow_var[k], t->pow_deg[k]}] = k;
  for (int64_t i = 0; i + 1 < N && cm.status == FP_OK; ++i) {
    const int64_t P = t->parent[i];
    const bool first = !seen[P];
    seen[P] = 1;
    const Buf& dst = acc[t->lh[P]];
    const int qk = pid.at({0, t->pd[i]});
    const Buf& qd = qp[qk];
    const int mode = first ? 2 : 1;
    const void* init = (const char*)cn.ptr + P * esz;
    if (!has_child[i]) {  // leaf: c_i * q^d
      if (cm.dry) continue;
      const int len = (int)qd.pitch;
      if (modp)
        k_leaf<uint64_t><<<grid_for(npairs * len), 256, 0, st>>>(
            (uint64_t*)dst.ptr, dst.pitch, (const uint64_t*)qd.ptr, qd.pitch, len,
            (const uint64_t*)cn.ptr + i, N, first, (const uint64_t*)init, N, npairs);
      else
        k_leaf<double><<<grid_for(npairs * len), 256, 0, st>>>(
            (double*)dst.ptr, dst.pitch, (const double*)qd.ptr, qd.pitch, len, (const double*)cn.ptr + i, N, first,
            (const double*)init, N, npairs);
      cm.check();
    } else {
      product(acc[t->lh[i]], degval(i) + 1, qd, qd.pitch, qk, dst, mode, init, N);
    }
  }
  // ---- root: r = acc (or c) times q^d(root)
  if (cm.status == FP_OK) {
    const int64_t R = N - 1;
    const int64_t d0 = t->pd[R];
    if (!has_child[R]) {  // a single term c x^d: c * q^d
      if (cm.dry) {
      } else if (d0 == 0) {
        k_fill_zero<uint64_t><<<grid_for(npairs * outlen), 256, 0, st>>>((uint64_t*)out, outlen, 0, (int)outlen, npairs);
        if (modp) k_copy_rows<uint64_t><<<grid_for(npairs), 256, 0, st>>>((const uint64_t*)cn.ptr + R, N, (uint64_t*)out, outlen, 1, npairs, 0);
        else k_copy_rows<double><<<grid_for(npairs), 256, 0, st>>>((const double*)cn.ptr + R, N, (double*)out, outlen, 1, npairs, 0);
      } else {
        const Buf& qd = qp[pid.at({0, d0})];
        if (modp)
          k_leaf<uint64_t><<<grid_for(npairs * outlen), 256, 0, st>>>((uint64_t*)out, outlen, (const uint64_t*)qd.ptr,
                                                                      qd.pitch, (int)outlen, (const uint64_t*)cn.ptr + R,
                                                                      N, 1, nullptr, 0, npairs);
        else
          k_leaf<double><<<grid_for(npairs * outlen), 256, 0, st>>>((double*)out, outlen, (const double*)qd.ptr,
                                                                    qd.pitch, (int)outlen, (const double*)cn.ptr + R, N,
                                                                    1, nullptr, 0, npairs);
      }
      cm.check();
    } else if (d0 == 0) {
      const Buf& src = acc[t->lh[R]];
      if (cm.dry) {
      } else if (modp) k_copy_rows<uint64_t><<<grid_for(npairs * outlen), 256, 0, st>>>((const uint64_t*)src.ptr, src.pitch, (uint64_t*)out, outlen, (int)outlen, npairs, 0);
      else k_copy_rows<double><<<grid_for(npairs * outlen), 256, 0, st>>>((const double*)src.ptr, src.pitch, (double*)out, outlen, (int)outlen, npairs, 0);
      cm.check();
    } else {
      const int qk = pid.at({0, d0});
      const Buf& qd = qp[qk];
      product(acc[t->lh[R]], degval(R) + 1, qd, qd.pitch, qk, outb, 0, nullptr, 0);
    }
  }
  int rc = cm.status;
  if (rc == FP_OK && tc_any && cm.live()) {
    // a tensor-core tile that gave up waiting for its products reports here
    int flag = 0;
    if (cudaMemcpyAsync(&flag, tc_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = FP_E_CUDA;
    else if (flag)
      rc = FP_E_TIMEOUT;
  }
  cm.release();
  if (cm.dry) *dry_bytes = cm.arena_used;
  return rc;
}

int set_compose_f64(int slices, int min_len) {
  if (slices != 0 && (slices < 6 || slices > 8)) return FP_E_BAD_VALUE;
  g_f64_slices.store(slices ? slices : 7);
  g_f64_tc_min.store(min_len == 0 ? 256 : (min_len < 0 ? 0 : min_len));
  return FP_OK;
}


// ------------------------------------------------------------ allocation-free entry
// Work space of fp_compose_noalloc: one region per device, reserved when the
// library is loaded and held until the process exits.  Every call carves its
// buffers from the start of it; calls that overlap on the device race.
static __device__ __align__(256) unsigned char g_compose_scratch[FP_NOALLOC_SCRATCH_BYTES];

namespace {

// device address of g_compose_scratch, per device, looked up once under the lock
std::atomic<unsigned char*> g_scratch_ptr[256];
std::mutex g_scratch_lock;

}  // namespace

int compose_noalloc_device(const fp_tree* t, fp_dtype dtype, const void* pcoeffs, const void* q, int32_t degq,
                           int64_t npairs, void* out, cudaStream_t st) {
  if (!t || !q || !out || degq < 0 || npairs < 0) return FP_E_BAD_VALUE;
  if (t->nvars != 1) return FP_E_BAD_VALUE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) { cudaGetLastError(); return FP_E_CUDA; }
  unsigned char* base = g_scratch_ptr[dev].load();
  if (!base) {
    // set-up, once per device, with that device current: host code needs the
    // device address of the array (the symbol itself is a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_scratch_lock);
    base = g_scratch_ptr[dev].load();
    if (!base) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_compose_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return FP_E_CUDA;
      }
      base = (unsigned char*)ptr;
      g_scratch_ptr[dev].store(base);
    }
  }
  // the work space, counted by a dry run of the same driver code
  size_t need = 0;
  const int rc = compose_device(t, dtype, pcoeffs, q, degq, npairs, out, st, nullptr, 0, &need);
  if (rc != FP_OK) return rc;
  if (need > (size_t)FP_NOALLOC_SCRATCH_BYTES) return FP_E_TOO_LARGE;
  return compose_device(t, dtype, pcoeffs, q, degq, npairs, out, st, base, (size_t)FP_NOALLOC_SCRATCH_BYTES);
}

int compose_workspace_device(const fp_tree* t, fp_dtype dtype, int per_pair_coeffs, int32_t degq, int64_t npairs,
                             size_t* bytes) {
  if (!bytes) return FP_E_BAD_VALUE;
  static const uint64_t dummy = 0;  // stands for the caller's buffers: a dry run reads none of them
  return compose_device(t, dtype, per_pair_coeffs ? &dummy : nullptr, &dummy, degq, npairs, (void*)&dummy, nullptr,
                        nullptr, 0, bytes);
}

}  // namespace fp
