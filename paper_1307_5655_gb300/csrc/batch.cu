// Many evaluation jobs (trees of uneven size, each with its own points) in
// one launch per shared-memory class.  Each block is one tile of one job: it
// finds its job in a descriptor table (binary search on the first tile of
// each job) and runs exactly the per-tile code of the single-job kernels, so
// a job's result is the same alone or in a batch.  Jobs are ordered by
// decreasing cost (nodes x tiles) so that the expensive tiles are scheduled
// first and the small ones fill the tail.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "eval_kernel.cuh"
#include "tree.hpp"

namespace fp {

// how a job is evaluated (the same choice fp_eval makes)
enum : int { kModeOps = 0, kModeNodeTable = 1, kModeNodeFly = 2 };

struct BatchJob {
  EvalArgs g;
  OpArgs o;
  int mode;
  int scheme;
  int64_t tile0;  // first block of this job in its launch
};

template <class A, int PPT>
__global__ void __launch_bounds__(kTPB) eval_batch_kernel(const BatchJob* __restrict__ jobs, int njobs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int lo = 0, hi = njobs - 1;
  const int64_t b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile0 <= b) lo = mid;
    else hi = mid - 1;
  }
  const EvalArgs g = jobs[lo].g;
  const int mode = jobs[lo].mode;
  const int64_t base = (b - jobs[lo].tile0) * (kTPB * PPT);
  if constexpr (std::is_same<A, IV64>::value) {
    if (mode == kModeNodeTable) node_tile<A, PPT, true>(g, base, smem_raw);
    else node_tile<A, PPT, false>(g, base, smem_raw);
  } else {
    if (mode == kModeOps) {
      const OpArgs o = jobs[lo].o;
      const int scheme = jobs[lo].scheme;
      if (scheme == FP_SCHEME_E) ops_tile<A, PPT, FP_SCHEME_E>(g, o, base, smem_raw);
      // Balanced: the extended path, which also runs plain Balanced schedules
      // (one instantiation less in this kernel, which serves every scheme)
      else if (scheme == FP_SCHEME_B) ops_tile<A, PPT, kSchemeBExt>(g, o, base, smem_raw);
      else ops_tile<A, PPT, 0>(g, o, base, smem_raw);
    } else if (mode == kModeNodeTable) {
      node_tile<A, PPT, true>(g, base, smem_raw);
    } else {
      node_tile<A, PPT, false>(g, base, smem_raw);
    }
  }
}

int fill_eval_args(const fp_tree* t, fp_dtype dt, const void* points, int64_t npts, void* out, EvalArgs& a, OpArgs& o);
void lookup_tuned(const fp_tree* t, fp_dtype dt, int64_t npts, int& variant, int& ppt);

namespace {

template <class A, int PPT>
cudaError_t launch_batch_t(const BatchJob* d_jobs, int njobs, int64_t nblocks, size_t smem, cudaStream_t st) {
  static std::atomic<int> configured_dev{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev.load(std::memory_order_relaxed) != dev) {
    cudaError_t e = cudaFuncSetAttribute(eval_batch_kernel<A, PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemMax);
    if (e != cudaSuccess) return e;
    configured_dev.store(dev, std::memory_order_relaxed);
  }
  if (nblocks <= 0) return cudaSuccess;
  if (nblocks > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  eval_batch_kernel<A, PPT><<<(unsigned)nblocks, kTPB, smem, st>>>(d_jobs, njobs);
  return cudaGetLastError();
}

int ppt_of(fp_dtype dt) { return (dt == FP_F32C || dt == FP_MODP) ? 2 : 1; }

size_t bytes_of(fp_dtype dt, bool val) {
  (void)val;
  return dt == FP_IV64 ? 16 : 8;
}

}  // namespace

// One launch: jobs [j0, j1) of the sorted list, with their shared memory.
struct BatchLaunch {
  int64_t job0 = 0;
  int njobs = 0;
  int64_t nblocks = 0;
  size_t smem = 0;
};

}  // namespace fp

struct fp_batch {
  fp_dtype dtype = FP_F64;
  std::vector<fp::BatchJob> jobs;  // host copy, sorted by decreasing cost
  std::vector<fp::BatchLaunch> launches;
  fp::BatchJob* d_jobs = nullptr;
  int device = -1;
  bool owns = true;  // device table allocated by fp_batch_create
};

namespace fp {

// Build the descriptor table and the launch split (host only).
int batch_build(fp_dtype dt, const fp_job* jobs, int64_t njobs, fp_batch* b) {
  if (njobs < 0 || (njobs > 0 && !jobs)) return FP_E_BAD_VALUE;
  if ((int)dt < FP_F64 || (int)dt > FP_MODP) return FP_E_DTYPE;
  b->dtype = dt;
  const int ppt = ppt_of(dt);
  const size_t vb = bytes_of(dt, true), pb = bytes_of(dt, false);
  struct Item {
    BatchJob j;
    double cost;
    size_t smem;
  };
  std::vector<Item> items;
  items.reserve(njobs);
  for (int64_t k = 0; k < njobs; ++k) {
    const fp_job& in = jobs[k];
    if (!in.tree) return FP_E_BAD_VALUE;
    if (in.npts < 0) return FP_E_BAD_VALUE;
    if (in.npts == 0) continue;
    if (!in.points || !in.out) return FP_E_BAD_VALUE;
    if (in.tree->nnodes == 0) return FP_E_BAD_VALUE;  // zero polynomials: use fp_eval
    Item it{};
    const int rc = fill_eval_args(in.tree, dt, in.points, in.npts, in.out, it.j.g, it.j.o);
    if (rc != FP_OK) return rc;
    const size_t table = (vb * it.j.g.nslot + pb * it.j.g.npow) * ppt * kTPB;
    const size_t fly = (vb * it.j.g.nslot + pb * it.j.g.nvars) * ppt * kTPB;
    const size_t ops_table = vb * (size_t)it.j.o.entries * ppt * kTPB;
    const bool fused = dt != FP_IV64;
    // the kernel variant fp_eval would use for this job (tuned or default);
    // points per thread do not change results, the variant can
    int tv = 0, tp = 0;
    lookup_tuned(in.tree, dt, in.npts, tv, tp);
    if (fused && tv != 2 && ops_table <= kTableSmemCap && it.j.o.recs) {
      it.j.mode = kModeOps;
      it.smem = ops_table;
    } else if (table <= kTableSmemCap) {
      it.j.mode = kModeNodeTable;
      it.smem = table;
    } else {
      it.j.mode = kModeNodeFly;
      it.smem = fly;
    }
    if (it.smem > kSmemMax) return FP_E_TOO_LARGE;
    it.j.scheme = in.tree->block_scheme;
    const int64_t tiles = (in.npts + (int64_t)kTPB * ppt - 1) / ((int64_t)kTPB * ppt);
    it.cost = (double)in.tree->nnodes * (double)tiles;
    items.push_back(it);
  }
  // launch classes by shared memory (a block holds the class maximum), most
  // expensive jobs first within each class
  auto cls = [](size_t smem) {
    size_t c = 16 * 1024;
    int k = 0;
    while (c < smem) { c *= 2; ++k; }
    return k;
  };
  std::stable_sort(items.begin(), items.end(), [&](const Item& x, const Item& y) {
    const int cx = cls(x.smem), cy = cls(y.smem);
    if (cx != cy) return cx < cy;
    return x.cost > y.cost;
  });
  b->jobs.clear();
  b->launches.clear();
  for (size_t i = 0; i < items.size();) {
    BatchLaunch L;
    L.job0 = (int64_t)b->jobs.size();
    const int c = cls(items[i].smem);
    int64_t tile = 0;
    size_t smem = 0;
    while (i < items.size() && cls(items[i].smem) == c) {
      BatchJob j = items[i].j;
      j.tile0 = tile;
      tile += (j.g.npts + (int64_t)kTPB * ppt - 1) / ((int64_t)kTPB * ppt);
      smem = std::max(smem, items[i].smem);
      b->jobs.push_back(j);
      ++i;
    }
    L.njobs = (int)(b->jobs.size() - L.job0);
    L.nblocks = tile;
    L.smem = smem;
    b->launches.push_back(L);
  }
  return FP_OK;
}

int batch_launch(const fp_batch* b, const BatchJob* d_jobs, cudaStream_t st) {
  for (const BatchLaunch& L : b->launches) {
    cudaError_t e = cudaSuccess;
    const BatchJob* dj = d_jobs + L.job0;
    switch (b->dtype) {
      case FP_F64: e = launch_batch_t<F64, 1>(dj, L.njobs, L.nblocks, L.smem, st); break;
      case FP_F32C: e = launch_batch_t<F32C, 2>(dj, L.njobs, L.nblocks, L.smem, st); break;
      case FP_IV64: e = launch_batch_t<IV64, 1>(dj, L.njobs, L.nblocks, L.smem, st); break;
      case FP_MODP: e = launch_batch_t<MODP, 2>(dj, L.njobs, L.nblocks, L.smem, st); break;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return FP_E_CUDA;
    }
  }
  return FP_OK;
}

}  // namespace fp

using namespace fp;

extern "C" {

int fp_batch_create(fp_dtype dtype, const fp_job* jobs, int64_t njobs, fp_batch** out) {
  if (!out) return FP_E_BAD_VALUE;
  fp_batch* b = new (std::nothrow) fp_batch();
  if (!b) return FP_E_NOMEM;
  int rc;
  try {
    rc = batch_build(dtype, jobs, njobs, b);
  } catch (const std::bad_alloc&) {
    rc = FP_E_NOMEM;
  }
  if (rc == FP_OK && cudaGetDevice(&b->device) != cudaSuccess) rc = FP_E_CUDA;
  if (rc == FP_OK && !b->jobs.empty()) {
    if (cudaMalloc((void**)&b->d_jobs, b->jobs.size() * sizeof(BatchJob)) != cudaSuccess) rc = FP_E_NOMEM;
    else if (cudaMemcpy(b->d_jobs, b->jobs.data(), b->jobs.size() * sizeof(BatchJob), cudaMemcpyHostToDevice) !=
             cudaSuccess)
      rc = FP_E_CUDA;
  }
  if (rc != FP_OK) {
    cudaGetLastError();
    if (b->d_jobs) cudaFree(b->d_jobs);
    delete b;
    return rc;
  }
  *out = b;
  return FP_OK;
}

int fp_batch_launch(const fp_batch* b, void* stream) {
  if (!b) return FP_E_BAD_VALUE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) { cudaGetLastError(); return FP_E_BAD_VALUE; }
  return batch_launch(b, b->d_jobs, (cudaStream_t)stream);
}

void fp_batch_free(fp_batch* b) {
  if (!b) return;
  if (b->d_jobs) cudaFree(b->d_jobs);
  delete b;
}

int fp_eval_batch(fp_dtype dtype, const fp_job* jobs, int64_t njobs, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  fp_batch b;
  int rc;
  try {
    rc = batch_build(dtype, jobs, njobs, &b);
  } catch (const std::bad_alloc&) {
    rc = FP_E_NOMEM;
  }
  if (rc != FP_OK || b.jobs.empty()) return rc;
  BatchJob* d = nullptr;
  const size_t bytes = b.jobs.size() * sizeof(BatchJob);
  if (pool_alloc((void**)&d, bytes, st) != cudaSuccess) { cudaGetLastError(); return FP_E_NOMEM; }
  // from pageable memory: the copy is staged before the call returns
  if (cudaMemcpyAsync(d, b.jobs.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) rc = FP_E_CUDA;
  if (rc == FP_OK) rc = batch_launch(&b, d, st);
  cudaFreeAsync(d, st);
  return rc;
}

}  // extern "C"
