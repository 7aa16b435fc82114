// C ABI of the library (declarations and contracts in include/fastpoly.h).
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "eval_kernel.cuh"
#include "tree.hpp"

namespace fp {
uint64_t rns_offset(int i);
int launch_eval_rns(const EvalArgs& a, const OpArgs& o, int scheme, int k, const int64_t* strides,
                    const uint64_t* root_c, cudaStream_t st);

namespace {

template <class T>
int upload(const std::vector<T>& h, T** d) {
  const size_t n = h.empty() ? 1 : h.size();
  if (cudaMalloc((void**)d, n * sizeof(T)) != cudaSuccess) { cudaGetLastError(); return FP_E_NOMEM; }
  if (!h.empty() && cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return FP_E_CUDA;
  return FP_OK;
}

void release(fp_tree* t) {
  DeviceSchedule& d = t->dev;
  void* ptrs[] = {d.ctrl, d.pow_prog, d.pow_dv, d.ca_f64, d.cb_f64, d.ca_f32, d.cb_f32, d.ca_u64, d.cb_u64,
                  d.ops_f64, d.ops_f32, d.ops_u64, d.st_f64, d.st_f32, d.st_u64, d.ops_prog, d.ops_chain_pid, d.ops_defer,
                  d.ca_rns, d.cb_rns, d.ops_rns, d.st_rns, d.root_rns};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  d = DeviceSchedule{};
}

// op records and the coefficient stream in the coefficient type C
template <class C, class H>
void build_ops(const fp_tree* t, const std::vector<H>& c, std::vector<OpRec<C>>& recs, std::vector<C>& st) {
  recs.resize(t->ops.size());
  for (size_t i = 0; i < t->ops.size(); ++i) {
    OpRec<C> r{};
    r.x = t->ops[i].x; r.y = t->ops[i].y; r.z = t->ops[i].z; r.w = t->ops[i].w;
    r.a = t->op_a_node[i] >= 0 ? (C)c[t->op_a_node[i]] : C(0);
    r.b = t->op_b_node[i] >= 0 ? (C)c[t->op_b_node[i]] : C(0);
    recs[i] = r;
  }
  st.assign(t->stream.size() + kStreamAlign, C(0));  // padded so 4-wide loads stay in bounds
  for (size_t k = 0; k < t->stream.size(); ++k)
    if (t->stream[k] >= 0) st[k] = (C)c[t->stream[k]];
}

int upload_schedule(fp_tree* t) {
  DeviceSchedule& d = t->dev;
  if (cudaGetDevice(&d.device) != cudaSuccess) { cudaGetLastError(); return FP_E_CUDA; }
  if (t->nnodes == 0) return FP_OK;
  const int64_t N = t->nnodes, S = N - 1;
  int rc = upload(t->ctrl, &d.ctrl);
  if (rc == FP_OK) rc = upload(t->pow_prog, &d.pow_prog);
  if (rc == FP_OK) rc = upload(t->ops_prog, &d.ops_prog);
  if (rc == FP_OK) rc = upload(t->ops_chain_pid, &d.ops_chain_pid);
  if (rc == FP_OK) rc = upload(t->ops_defer, &d.ops_defer);
  if (rc != FP_OK) return rc;
  std::vector<uint2> dv(t->pow_prog.size());
  for (size_t k = 0; k < dv.size(); ++k) dv[k] = make_uint2((unsigned)t->pow_var[k], (unsigned)t->pow_deg[k]);
  rc = upload(dv, &d.pow_dv);
  if (rc != FP_OK) return rc;
  if (t->coeff_type == FP_MODP) {
    std::vector<uint64_t> a(S), b(S);
    for (int64_t i = 0; i < S; ++i) {
      a[i] = t->c_u64[i];
      b[i] = ((t->ctrl[i] >> kCtrlFirst) & 1u) ? t->c_u64[t->parent[i]] : 0;
    }
    rc = upload(a, &d.ca_u64);
    if (rc == FP_OK) rc = upload(b, &d.cb_u64);
    std::vector<OpRec<uint64_t>> recs;
    std::vector<uint64_t> st;
    build_ops(t, t->c_u64, recs, st);
    if (rc == FP_OK) rc = upload(recs, &d.ops_u64);
    if (rc == FP_OK) rc = upload(st, &d.st_u64);
  } else {
    std::vector<double> a(S), b(S);
    std::vector<float> af(S), bf(S);
    for (int64_t i = 0; i < S; ++i) {
      a[i] = t->c_f64[i];
      b[i] = ((t->ctrl[i] >> kCtrlFirst) & 1u) ? t->c_f64[t->parent[i]] : 0.0;
      af[i] = (float)a[i];
      bf[i] = (float)b[i];
    }
    rc = upload(a, &d.ca_f64);
    if (rc == FP_OK) rc = upload(b, &d.cb_f64);
    if (rc == FP_OK) rc = upload(af, &d.ca_f32);
    if (rc == FP_OK) rc = upload(bf, &d.cb_f32);
    std::vector<OpRec<double>> recs;
    std::vector<double> st;
    build_ops(t, t->c_f64, recs, st);
    if (rc == FP_OK) rc = upload(recs, &d.ops_f64);
    if (rc == FP_OK) rc = upload(st, &d.st_f64);
    std::vector<float> cf(t->c_f64.begin(), t->c_f64.end());
    std::vector<OpRec<float>> recs32;
    std::vector<float> st32;
    build_ops(t, cf, recs32, st32);
    if (rc == FP_OK) rc = upload(recs32, &d.ops_f32);
    if (rc == FP_OK) rc = upload(st32, &d.st_f32);
  }
  return rc;
}

__global__ void fill_zero_kernel(uint64_t* out, int64_t nwords) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 0;
}

__global__ void fill_zero32_kernel(uint32_t* out, int64_t nwords) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 0;
}

size_t value_bytes_out(fp_dtype dt) {  // bytes of output per point
  switch (dt) {
    case FP_F64: return 8;
    case FP_F32C: return 8;
    case FP_IV64: return 16;
    case FP_MODP: return 8;
  }
  return 0;
}

bool dtype_ok(const fp_tree* t, fp_dtype dt) {
  if (t->dev.device < 0) return false;  // host-only tree
  if (dt == FP_MODP) return t->coeff_type == FP_MODP;
  if (dt == FP_F64 || dt == FP_F32C || dt == FP_IV64) return t->coeff_type == FP_F64;
  return false;
}

__global__ void plain_horner_kernel(const double* __restrict__ c, int64_t nc, const double* __restrict__ x,
                                    int64_t npts, double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npts) return;
  const double xv = x[j];
  double r = c[nc - 1];
  for (int64_t i = nc - 2; i >= 0; --i) r = fma(r, xv, c[i]);
  out[j] = r;
}

}  // namespace

// Host buffers in, host buffers out: the points are cut into chunks that
// run as a pipeline -- the copy in of chunk i + 1 and the copy out of chunk
// i - 1 overlap the evaluation of chunk i -- on two copy streams of the
// library and the caller's stream, ordered by events; two device buffers
// per direction alternate.  Points and results are structure-of-arrays rows
// ([rows][npts]), so a chunk is a strided 2D copy.  Synchronous.
int eval_host_pipelined(const fp_tree* t, fp_dtype dtype, const void* points_host, int64_t npts, void* out_host,
                        cudaStream_t st);

// ---- autotuner cache: (value type, variables, block scheme, log2 nodes,
// log2 points) -> (kernel, points per thread), filled by fp_tune
struct TuneKey {
  int dt, nvars, scheme, lnodes, lpts;
  bool operator<(const TuneKey& o) const {
    return std::tie(dt, nvars, scheme, lnodes, lpts) < std::tie(o.dt, o.nvars, o.scheme, o.lnodes, o.lpts);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;

int log2_bucket(int64_t v) {
  int l = 0;
  while ((int64_t)1 << (l + 1) <= v) ++l;
  return l;
}

TuneKey tune_key(const fp_tree* t, fp_dtype dt, int64_t npts) {
  return TuneKey{(int)dt, t->nvars, t->block_scheme, log2_bucket(t->nnodes), log2_bucket(npts)};
}

void lookup_tuned(const fp_tree* t, fp_dtype dt, int64_t npts, int& variant, int& ppt) {
  if (t->tuned_kernel[dt] != 0) {
    variant = t->tuned_kernel[dt];
    ppt = t->tuned_ppt[dt];
    return;
  }
  std::lock_guard<std::mutex> g(g_tune_mu);
  auto it = g_tune.find(tune_key(t, dt, npts));
  if (it != g_tune.end()) {
    variant = it->second.first;
    ppt = it->second.second;
  }
}

// Kernel arguments of one evaluation (shared by fp_eval and the batch path).
int fill_eval_args(const fp_tree* t, fp_dtype dt, const void* points, int64_t npts, void* out, EvalArgs& a,
                   OpArgs& o) {
  if (!t || !dtype_ok(t, dt)) return FP_E_DTYPE;
  if (t->nnodes == 0) return FP_E_BAD_VALUE;
  a = EvalArgs{};
  a.ctrl = t->dev.ctrl;
  a.pow_prog = t->dev.pow_prog;
  a.pow_dv = t->dev.pow_dv;
  a.nsteps = t->nnodes - 1;
  a.npow = (int)t->pow_prog.size();
  a.nslot = t->max_lh + 1;
  a.nvars = t->nvars;
  a.root_leaf = t->root_leaf;
  a.root_lh = t->root_lh;
  a.root_pid = t->root_pid;
  a.points = points;
  a.npts = npts;
  a.out = out;
  o = OpArgs{};
  o.nops = (int64_t)t->ops.size();
  o.prog = t->dev.ops_prog;
  o.chain_pid = t->dev.ops_chain_pid;
  o.defer_edges = t->dev.ops_defer;
  o.nprog = (int)t->ops_prog.size();
  o.nlive = t->ops_nlive;
  o.nslot = t->ops_nslot;
  o.entries = t->ops_entries;
  o.root_lh = t->ops_root_lh;
  o.root_pid = t->ops_root_pid;
  o.pos_x1 = t->ops_pos_x1;
  o.ext = t->ops_ext;
  o.split = t->ops_split;
  o.ndefer = t->ops_ndefer;
  for (int d = 0; d <= kMaxBlock; ++d) o.pid_pow[d] = t->ops_pid_pow[d];
  const int64_t root = t->nnodes - 1;
  switch (dt) {
    case FP_F64:
      a.ca = t->dev.ca_f64; a.cb = t->dev.cb_f64;
      o.recs = t->dev.ops_f64; o.stream = t->dev.st_f64;
      std::memcpy(&a.root_c, &t->c_f64[root], 8);
      break;
    case FP_IV64:
      a.ca = t->dev.ca_f64; a.cb = t->dev.cb_f64;
      std::memcpy(&a.root_c, &t->c_f64[root], 8);
      break;
    case FP_F32C: {
      a.ca = t->dev.ca_f32; a.cb = t->dev.cb_f32;
      o.recs = t->dev.ops_f32; o.stream = t->dev.st_f32;
      const float c = (float)t->c_f64[root];
      uint32_t bits;
      std::memcpy(&bits, &c, 4);
      a.root_c = bits;
      break;
    }
    case FP_MODP:
      a.ca = t->dev.ca_u64; a.cb = t->dev.cb_u64;
      o.recs = t->dev.ops_u64; o.stream = t->dev.st_u64;
      a.root_c = t->c_u64[root];
      break;
  }
  return FP_OK;
}

int eval_device(const fp_tree* t, fp_dtype dt, const void* points, int64_t npts, void* out, cudaStream_t st,
                int variant = 0, int ppt = 0) {
  if (variant < 0 || variant > 2) return FP_E_BAD_VALUE;
  if (ppt != 0 && ppt != 1 && ppt != 2 && ppt != 4) return FP_E_BAD_VALUE;
  if (!t) return FP_E_BAD_VALUE;
  if ((int)dt < FP_F64 || (int)dt > FP_MODP) return FP_E_DTYPE;
  if (!dtype_ok(t, dt)) return FP_E_DTYPE;
  if (npts < 0) return FP_E_BAD_VALUE;
  if (npts == 0) return FP_OK;
  if (!points || !out) return FP_E_BAD_VALUE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != t->dev.device) { cudaGetLastError(); return FP_E_BAD_VALUE; }
  if (t->nnodes == 0) {  // zero polynomial
    const int64_t bytes = npts * (int64_t)value_bytes_out(dt);
    const int blocks = (int)((bytes / 8 + 255) / 256 < 4096 ? (bytes / 8 + 255) / 256 + 1 : 4096);
    if (bytes % 8 == 0) fill_zero_kernel<<<blocks, 256, 0, st>>>((uint64_t*)out, bytes / 8);
    else fill_zero32_kernel<<<blocks, 256, 0, st>>>((uint32_t*)out, bytes / 4);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_E_CUDA;
  }
  EvalArgs a;
  OpArgs o;
  const int frc = fill_eval_args(t, dt, points, npts, out, a, o);
  if (frc != FP_OK) return frc;
  if (variant == 0 && ppt == 0) {  // a tuned configuration, from the tree or the shared cache
    lookup_tuned(t, dt, npts, variant, ppt);
  }
  const size_t vbytes = dt == FP_IV64 ? 16 : 8, pbytes = vbytes;
  if (ppt == 0) ppt = (dt == FP_F32C || dt == FP_MODP) ? 2 : 1;
  if (dt == FP_F64 && ppt == 4) ppt = 2;
  if (dt == FP_IV64 && ppt == 4) ppt = 2;
  const size_t smem = (vbytes * (size_t)a.nslot + pbytes * (size_t)a.nvars) * ppt * kTPB;
  if (smem > kSmemMax) return FP_E_TOO_LARGE;
  cudaError_t e = cudaSuccess;
  switch (dt) {
    case FP_F64: e = launch_eval_f64(a, o, t->block_scheme, st, variant, ppt); break;
    case FP_F32C: e = launch_eval_f32c(a, o, t->block_scheme, st, variant, ppt); break;
    case FP_IV64: e = launch_eval_iv64(a, o, t->block_scheme, st, variant, ppt); break;
    case FP_MODP: e = launch_eval_modp(a, o, t->block_scheme, st, variant, ppt); break;
  }
  if (e == cudaErrorInvalidValue && variant == 1) { cudaGetLastError(); return FP_E_TOO_LARGE; }
  return e == cudaSuccess ? FP_OK : FP_E_CUDA;
}

int compose_device(const fp_tree* t, fp_dtype dtype, const void* pcoeffs, const void* q, int32_t degq, int64_t npairs,
                   void* out, cudaStream_t st, unsigned char* arena, size_t arena_cap, size_t* dry_bytes);
int compose_noalloc_device(const fp_tree* t, fp_dtype dtype, const void* pcoeffs, const void* q, int32_t degq,
                           int64_t npairs, void* out, cudaStream_t st);
int compose_workspace_device(const fp_tree* t, fp_dtype dtype, int per_pair_coeffs, int32_t degq, int64_t npairs,
                             size_t* bytes);
int set_compose_f64(int slices, int min_len);

}  // namespace fp

using namespace fp;

extern "C" {

int fp_compile(int nvars, int64_t nterms, const int32_t* exps, const void* coeffs, fp_dtype coeff_type,
               fp_scheme scheme, const int32_t* f_table, int64_t f_table_len, fp_tree** out) {
  if (!out) return FP_E_BAD_VALUE;
  fp_tree* t = new (std::nothrow) fp_tree();
  if (!t) return FP_E_NOMEM;
  int rc;
  try {
    rc = compile_host(nvars, nterms, exps, coeffs, coeff_type, scheme, f_table, f_table_len, t);
  } catch (const std::bad_alloc&) {
    rc = FP_E_NOMEM;
  }
  if (rc == FP_OK) rc = upload_schedule(t);
  if (rc != FP_OK) {
    release(t);
    delete t;
    return rc;
  }
  *out = t;
  return FP_OK;
}

int fp_compile_host(int nvars, int64_t nterms, const int32_t* exps, const void* coeffs, fp_dtype coeff_type,
                    fp_scheme scheme, const int32_t* f_table, int64_t f_table_len, fp_tree** out) {
  if (!out) return FP_E_BAD_VALUE;
  fp_tree* t = new (std::nothrow) fp_tree();
  if (!t) return FP_E_NOMEM;
  int rc;
  try {
    rc = compile_host(nvars, nterms, exps, coeffs, coeff_type, scheme, f_table, f_table_len, t);
  } catch (const std::bad_alloc&) {
    rc = FP_E_NOMEM;
  }
  if (rc != FP_OK) {
    delete t;
    return rc;
  }
  *out = t;
  return FP_OK;
}

void fp_free(fp_tree* t) {
  if (!t) return;
  release(t);
  delete t;
}

int fp_eval(const fp_tree* t, fp_dtype dtype, const void* points, int64_t npts, void* out, void* stream) {
  return eval_device(t, dtype, points, npts, out, (cudaStream_t)stream);
}

int fp_eval_ex(const fp_tree* t, fp_dtype dtype, const void* points, int64_t npts, void* out, void* stream,
               const fp_launch_cfg* cfg) {
  return eval_device(t, dtype, points, npts, out, (cudaStream_t)stream, cfg ? cfg->kernel : 0,
                     cfg ? cfg->points_per_thread : 0);
}

}  // extern "C"

namespace fp {
// Time every launch configuration of one tree on these points (3 runs each
// after a warm-up); the fastest one's (kernel, points per thread, ms per run).
int tune_device(const fp_tree* t, fp_dtype dtype, const void* points, int64_t npts, void* out, cudaStream_t st,
                int& bk, int& bp, float& best_ms) {
  const int kernels[2] = {1, 2};
  const int ppts[3] = {1, 2, 4};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { cudaGetLastError(); return FP_E_CUDA; }
  best_ms = 1e30f;
  bk = 0;
  bp = 0;
  for (int k : kernels) {
    if (k == 1 && dtype == FP_IV64) continue;
    for (int p : ppts) {
      if ((dtype == FP_F64 || dtype == FP_IV64) && p == 4) continue;
      // warm-up run (also rejects configurations that do not fit)
      if (eval_device(t, dtype, points, npts, out, st, k, p) != FP_OK) { cudaGetLastError(); continue; }
      cudaEventRecord(e0, st);
      int rc = FP_OK;
      for (int r = 0; r < 3 && rc == FP_OK; ++r) rc = eval_device(t, dtype, points, npts, out, st, k, p);
      cudaEventRecord(e1, st);
      if (rc != FP_OK || cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); continue; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; bk = k; bp = p; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (bk == 0) return FP_E_CUDA;
  best_ms /= 3;
  return FP_OK;
}
}  // namespace fp

extern "C" {

int fp_tune(fp_tree* t, fp_dtype dtype, const void* points, int64_t npts, void* out, void* stream,
            fp_launch_cfg* best) {
  if (!t || npts <= 0 || !points || !out) return FP_E_BAD_VALUE;
  if (!dtype_ok(t, dtype)) return FP_E_DTYPE;
  if (t->nnodes == 0) return FP_E_BAD_VALUE;
  cudaStream_t st = (cudaStream_t)stream;
  int bk = 0, bp = 0;
  float best_ms = 0;
  const int trc = tune_device(t, dtype, points, npts, out, st, bk, bp, best_ms);
  if (trc != FP_OK) return trc;
  t->tuned_kernel[dtype] = bk;
  t->tuned_ppt[dtype] = bp;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[tune_key(t, dtype, npts)] = {bk, bp};
  }
  // leave the tuned configuration's result in `out`
  const int rc = eval_device(t, dtype, points, npts, out, st, bk, bp);
  if (best) {
    best->kernel = bk;
    best->points_per_thread = bp;
  }
  return rc;
}

int fp_tune_scheme(int nvars, int64_t nterms, const int32_t* exps, const void* coeffs, fp_dtype coeff_type,
                   fp_dtype dtype, const void* points, int64_t npts, void* out, void* stream, int64_t* k0_out,
                   fp_tree** tree_out) {
  if (!tree_out || npts <= 0 || !points || !out || nterms < 1) return FP_E_BAD_VALUE;
  if (nterms > FP_MAX_TERMS) return FP_E_TOO_LARGE;
  cudaStream_t st = (cudaStream_t)stream;
  // candidates: k0 = 1, 2, 4, ..., the first power of two >= nterms (Horner
  // everywhere), then the Balanced scheme (k0 = 0)
  std::vector<int64_t> k0s;
  for (int64_t k0 = 1;; k0 <<= 1) {
    k0s.push_back(k0);
    if (k0 >= nterms) break;
  }
  k0s.push_back(0);
  std::vector<int32_t> ft;
  fp_tree* best = nullptr;
  float best_ms = 1e30f;
  int64_t best_k0 = -1;
  int last_rc = FP_OK;
  for (const int64_t k0 : k0s) {
    fp_tree* t = nullptr;
    int rc;
    if (k0 == 0) {
      rc = fp_compile(nvars, nterms, exps, coeffs, coeff_type, FP_SCHEME_B, nullptr, 0, &t);
    } else {
      // f(n) = 2^floor(log2 n) when the run has more than k0 terms (n + 1 > k0), else 1
      try {
        ft.assign((size_t)nterms, 1);
      } catch (const std::bad_alloc&) {
        return FP_E_NOMEM;
      }
      for (int64_t n = 1; n < nterms; ++n) {
        int64_t f = 1;
        if (n + 1 > k0)
          while ((f << 1) <= n) f <<= 1;
        ft[(size_t)n] = (int32_t)f;
      }
      rc = fp_compile(nvars, nterms, exps, coeffs, coeff_type, FP_SCHEME_CUSTOM, ft.data(), nterms, &t);
    }
    if (rc != FP_OK) {  // invalid terms fail every candidate alike
      if (best) fp_free(best);
      return rc;
    }
    int bk = 0, bp = 0;
    float ms = 0;
    rc = dtype_ok(t, dtype) ? (t->nnodes ? tune_device(t, dtype, points, npts, out, st, bk, bp, ms) : FP_OK)
                            : FP_E_DTYPE;
    if (rc != FP_OK) {
      last_rc = rc;
      fp_free(t);
      if (rc == FP_E_DTYPE) break;
      continue;
    }
    if (t->nnodes) {
      t->tuned_kernel[dtype] = bk;
      t->tuned_ppt[dtype] = bp;
    }
    if (!best || ms < best_ms) {
      if (best) fp_free(best);
      best = t;
      best_ms = ms;
      best_k0 = k0;
    } else {
      fp_free(t);
    }
  }
  if (!best) return last_rc != FP_OK ? last_rc : FP_E_CUDA;
  // the winner's result in `out`
  const int rc = eval_device(best, dtype, points, npts, out, st);
  if (rc != FP_OK) {
    fp_free(best);
    return rc;
  }
  if (k0_out) *k0_out = best_k0;
  *tree_out = best;
  return FP_OK;
}

int fp_eval_host(const fp_tree* t, fp_dtype dtype, const void* points_host, int64_t npts, void* out_host,
                 void* stream) {
  if (!t) return FP_E_BAD_VALUE;
  if (!dtype_ok(t, dtype)) return FP_E_DTYPE;
  if (npts < 0) return FP_E_BAD_VALUE;
  if (npts == 0) return FP_OK;
  if (!points_host || !out_host) return FP_E_BAD_VALUE;
  return eval_host_pipelined(t, dtype, points_host, npts, out_host, (cudaStream_t)stream);
}

int fp_tree_info(const fp_tree* t, int64_t* nnodes, int* nvars, int* max_lazy_height, int* npowers,
                 int* coeff_type) {
  if (!t) return FP_E_BAD_VALUE;
  if (nnodes) *nnodes = t->nnodes;
  if (nvars) *nvars = t->nvars;
  if (max_lazy_height) *max_lazy_height = t->max_lh;
  if (npowers) *npowers = (int)t->pow_prog.size();
  if (coeff_type) *coeff_type = t->coeff_type;
  return FP_OK;
}

int fp_tree_export(const fp_tree* t, int32_t* node_exps, int64_t* term_of_node, int64_t* parent, int32_t* pd_var,
                   int64_t* pd, int32_t* lazy_height) {
  if (!t) return FP_E_BAD_VALUE;
  const size_t N = (size_t)t->nnodes;
  if (N == 0) return FP_OK;
  if (node_exps) std::memcpy(node_exps, t->node_e.data(), N * t->nvars * sizeof(int32_t));
  if (term_of_node) std::memcpy(term_of_node, t->term_of_node.data(), N * sizeof(int64_t));
  if (parent) std::memcpy(parent, t->parent.data(), N * sizeof(int64_t));
  if (pd_var) std::memcpy(pd_var, t->pd_var.data(), N * sizeof(int32_t));
  if (pd) std::memcpy(pd, t->pd.data(), N * sizeof(int64_t));
  if (lazy_height) std::memcpy(lazy_height, t->lh.data(), N * sizeof(int32_t));
  return FP_OK;
}

int fp_tree_schedule(const fp_tree* t, int64_t* nops, uint32_t* op_words, int64_t* op_a_node, int64_t* op_b_node,
                     int64_t* stream_len, int64_t* stream, int32_t* nprog, uint32_t* prog, uint32_t* chain_pid,
                     int32_t* block_pow, int32_t* layout) {
  if (!t) return FP_E_BAD_VALUE;
  const size_t n = t->ops.size(), ns = t->stream.size(), np = t->ops_prog.size();
  const size_t nsteps = t->ops_chain_pid.size();
  if (nops) *nops = (int64_t)n;
  if (stream_len) *stream_len = (int64_t)ns;
  if (nprog) *nprog = (int32_t)np;
  if (op_words)
    for (size_t i = 0; i < n; ++i) {
      op_words[4 * i + 0] = t->ops[i].x;
      op_words[4 * i + 1] = t->ops[i].y;
      op_words[4 * i + 2] = t->ops[i].z;
      op_words[4 * i + 3] = t->ops[i].w;
    }
  if (op_a_node && n) std::memcpy(op_a_node, t->op_a_node.data(), n * sizeof(int64_t));
  if (op_b_node && n) std::memcpy(op_b_node, t->op_b_node.data(), n * sizeof(int64_t));
  if (stream && ns) std::memcpy(stream, t->stream.data(), ns * sizeof(int64_t));
  if (prog)
    for (size_t k = 0; k < np; ++k) {
      prog[2 * k] = t->ops_prog[k].x;
      prog[2 * k + 1] = t->ops_prog[k].y;
    }
  if (chain_pid && nsteps) std::memcpy(chain_pid, t->ops_chain_pid.data(), nsteps * sizeof(uint32_t));
  if (block_pow)
    for (int d = 0; d <= kMaxBlock; ++d) block_pow[d] = t->ops_pid_pow[d];
  if (layout) {
    layout[0] = t->ops_nlive;
    layout[1] = t->ops_nslot;
    layout[2] = t->ops_entries;
    layout[3] = t->block_scheme;
    layout[4] = t->root_leaf;
    layout[5] = t->ops_root_lh;
    layout[6] = t->ops_root_pid;
    layout[7] = (int32_t)t->ops_split;
  }
  return FP_OK;
}

int fp_compile_rns(int nvars, int64_t nterms, const int32_t* exps, int k, const uint64_t* residues,
                   fp_scheme scheme, const int32_t* f_table, int64_t f_table_len, fp_tree** out) {
  if (!out || k < 1 || k > FP_RNS_MAX_PRIMES || nterms < 0) return FP_E_BAD_VALUE;
  if (nterms > FP_MAX_TERMS) return FP_E_TOO_LARGE;
  if (nterms > 0 && !residues) return FP_E_BAD_VALUE;
  std::vector<uint64_t> present;
  try {
    present.assign((size_t)nterms, 0);
  } catch (const std::bad_alloc&) {
    return FP_E_NOMEM;
  }
  for (int i = 0; i < k; ++i) {
    const uint64_t q = 0 - rns_offset(i);
    for (int64_t t = 0; t < nterms; ++t) {
      const uint64_t r = residues[(size_t)i * nterms + t];
      if (r >= q) return FP_E_BAD_VALUE;
      present[t] |= r != 0 ? 1u : 0u;
    }
  }
  fp_tree* t = new (std::nothrow) fp_tree();
  if (!t) return FP_E_NOMEM;
  int rc;
  try {
    // the tree of the terms that are non-zero modulo some prime
    rc = compile_host(nvars, nterms, exps, present.data(), FP_MODP, scheme, f_table, f_table_len, t);
    if (rc == FP_OK) {
      const int64_t N = t->nnodes;
      t->rns_k = k;
      t->c_rns.assign((size_t)k * N, 0);
      for (int i = 0; i < k; ++i)
        for (int64_t j = 0; j < N; ++j)
          if (t->term_of_node[j] >= 0) t->c_rns[(size_t)i * N + j] = residues[(size_t)i * nterms + t->term_of_node[j]];
    }
  } catch (const std::bad_alloc&) {
    rc = FP_E_NOMEM;
  }
  if (rc == FP_OK) rc = upload_schedule(t);
  if (rc == FP_OK && t->nnodes > 0) {
    // per-prime slices of the node coefficients, the op records and streams
    const int64_t N = t->nnodes, S = N - 1;
    DeviceSchedule& d = t->dev;
    std::vector<uint64_t> a((size_t)k * S), b((size_t)k * S), root(k);
    std::vector<OpRec<uint64_t>> recs_all;
    std::vector<uint64_t> st_all;
    int64_t pitch = 0;
    for (int i = 0; i < k; ++i) {
      std::vector<uint64_t> ci(t->c_rns.begin() + (size_t)i * N, t->c_rns.begin() + (size_t)(i + 1) * N);
      for (int64_t j = 0; j < S; ++j) {
        a[(size_t)i * S + j] = ci[j];
        b[(size_t)i * S + j] = ((t->ctrl[j] >> kCtrlFirst) & 1u) ? ci[t->parent[j]] : 0;
      }
      root[i] = ci[N - 1];
      std::vector<OpRec<uint64_t>> recs;
      std::vector<uint64_t> st;
      build_ops(t, ci, recs, st);
      pitch = (int64_t)st.size();
      recs_all.insert(recs_all.end(), recs.begin(), recs.end());
      st_all.insert(st_all.end(), st.begin(), st.end());
    }
    d.st_rns_pitch = pitch;
    rc = upload(a, &d.ca_rns);
    if (rc == FP_OK) rc = upload(b, &d.cb_rns);
    if (rc == FP_OK) rc = upload(recs_all, &d.ops_rns);
    if (rc == FP_OK) rc = upload(st_all, &d.st_rns);
    if (rc == FP_OK) rc = upload(root, &d.root_rns);
  }
  if (rc != FP_OK) {
    release(t);
    delete t;
    return rc;
  }
  t->coeff_type = FP_RNS_COEFFS;
  *out = t;
  return FP_OK;
}

int fp_eval_rns(const fp_tree* t, const uint64_t* points, int64_t npts, uint64_t* out, void* stream) {
  if (!t || t->rns_k < 1) return t ? FP_E_DTYPE : FP_E_BAD_VALUE;
  if (npts < 0) return FP_E_BAD_VALUE;
  if (npts == 0) return FP_OK;
  if (!points || !out) return FP_E_BAD_VALUE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != t->dev.device) { cudaGetLastError(); return FP_E_BAD_VALUE; }
  cudaStream_t st = (cudaStream_t)stream;
  const int k = t->rns_k;
  if (t->nnodes == 0) {  // the zero polynomial: k rows of zeros
    const int64_t words = (int64_t)k * npts;
    fill_zero_kernel<<<(unsigned)std::min<int64_t>((words + 255) / 256, 4096), 256, 0, st>>>(out, words);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_E_CUDA;
  }
  EvalArgs a{};
  a.ctrl = t->dev.ctrl;
  a.pow_prog = t->dev.pow_prog;
  a.pow_dv = t->dev.pow_dv;
  a.nsteps = t->nnodes - 1;
  a.npow = (int)t->pow_prog.size();
  a.nslot = t->max_lh + 1;
  a.nvars = t->nvars;
  a.root_leaf = t->root_leaf;
  a.root_lh = t->root_lh;
  a.root_pid = t->root_pid;
  a.points = points;
  a.npts = npts;
  a.out = out;
  a.ca = t->dev.ca_rns;
  a.cb = t->dev.cb_rns;
  OpArgs o{};
  o.recs = t->dev.ops_rns;
  o.stream = t->dev.st_rns;
  o.nops = (int64_t)t->ops.size();
  o.prog = t->dev.ops_prog;
  o.chain_pid = t->dev.ops_chain_pid;
  o.defer_edges = t->dev.ops_defer;
  o.nprog = (int)t->ops_prog.size();
  o.nlive = t->ops_nlive;
  o.nslot = t->ops_nslot;
  o.entries = t->ops_entries;
  o.root_lh = t->ops_root_lh;
  o.root_pid = t->ops_root_pid;
  o.pos_x1 = t->ops_pos_x1;
  o.ext = t->ops_ext;
  o.split = t->ops_split;
  o.ndefer = t->ops_ndefer;
  for (int d = 0; d <= kMaxBlock; ++d) o.pid_pow[d] = t->ops_pid_pow[d];
  const int64_t strides[5] = {(int64_t)t->nvars * npts, npts, t->nnodes - 1, (int64_t)t->ops.size(),
                              t->dev.st_rns_pitch};
  return launch_eval_rns(a, o, t->block_scheme, k, strides, t->dev.root_rns, st);
}

int fp_compose(const fp_tree* p, fp_dtype dtype, const void* pcoeffs, const void* q, int32_t degq, int64_t npairs,
               void* out, void* stream) {
  int dev = -1;
  if (p && (cudaGetDevice(&dev) != cudaSuccess || dev != p->dev.device)) { cudaGetLastError(); return FP_E_BAD_VALUE; }
  return compose_device(p, dtype, pcoeffs, q, degq, npairs, out, (cudaStream_t)stream, nullptr, 0, nullptr);
}

int fp_set_compose_f64(int slices, int min_len) { return set_compose_f64(slices, min_len); }

int fp_compose_workspace(const fp_tree* p, fp_dtype dtype, int per_pair_coeffs, int32_t degq, int64_t npairs,
                         size_t* bytes) {
  return compose_workspace_device(p, dtype, per_pair_coeffs, degq, npairs, bytes);
}

int fp_compose_noalloc(const fp_tree* p, fp_dtype dtype, const void* pcoeffs, const void* q, int32_t degq,
                       int64_t npairs, void* out, void* stream) {
  int dev = -1;
  if (p && (cudaGetDevice(&dev) != cudaSuccess || dev != p->dev.device)) { cudaGetLastError(); return FP_E_BAD_VALUE; }
  return compose_noalloc_device(p, dtype, pcoeffs, q, degq, npairs, out, (cudaStream_t)stream);
}

int fp_eval_plain_f64(const double* coeffs, int64_t ncoeffs, const double* points, int64_t npts, double* out,
                      void* stream) {
  if (ncoeffs < 1 || npts < 0 || !coeffs) return FP_E_BAD_VALUE;
  if (npts == 0) return FP_OK;
  if (!points || !out) return FP_E_BAD_VALUE;
  const int64_t blocks = (npts + 255) / 256;
  if (blocks > 0x7FFFFFFFLL) return FP_E_TOO_LARGE;
  plain_horner_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(coeffs, ncoeffs, points, npts, out);
  return cudaGetLastError() == cudaSuccess ? FP_OK : FP_E_CUDA;
}

const char* fp_strerror(int status) {
  switch (status) {
    case FP_OK: return "ok";
    case FP_E_BAD_VALUE: return "bad value";
    case FP_E_DUP_TERM: return "duplicate term";
    case FP_E_BAD_SCHEME: return "bad scheme";
    case FP_E_DTYPE: return "value type not available for this tree";
    case FP_E_NOMEM: return "out of memory";
    case FP_E_TOO_LARGE: return "size beyond the supported limits";
    case FP_E_CUDA: return "CUDA error";
    case FP_E_TIMEOUT: return "device wait timed out";
    case FP_E_INTERNAL: return "internal schedule check failed";
  }
  return "unknown status";
}

}  // extern "C"
