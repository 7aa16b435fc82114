// A resident evaluation kernel with a device work queue: persistent blocks
// that stay on the GPU and evaluate tiles of jobs the host publishes while
// they run, so new work is admitted into a running kernel instead of waiting
// for a launch.  The tile code is the batch kernel's (the same result as
// fp_eval for each job).
//
// Queue (pinned host memory mapped into the device address space, so the host
// publishes with plain stores and no stream operation):
//   jobs[k]      descriptor of job k, written before its items are published
//   items[i]     a work item: job k, tiles [t, t + n) of it (n <= kItemTiles)
//   published    items published so far (host: release store after the
//                descriptors and items; device: acquire load)
//   stop         the host asks the blocks to exit once the published items
//                are claimed
//   done[k]      set by the block that finishes job k's last tile (release
//                store after the job's results; host: acquire load)
// Device memory: claimed (the next item, taken by compare-and-swap),
// tiles_done[k] (per-job counters), state (bit 0: an idle exit happened).
// A claim costs one read of the item (and of the job's descriptor when the
// block's previous item was another job's) over the host link.
//
// Bounded waits: an idle block sleeps between polls and exits after the
// configured idle time; the host relaunches the kernel when it submits to an
// exited one.  Nothing spins without a limit.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "eval_kernel.cuh"
#include "tree.hpp"

namespace fp {

// the batch kernel's descriptor and the job builder (batch.cu)
enum : int { kResModeOps = 0, kResModeNodeTable = 1, kResModeNodeFly = 2 };
struct ResJob {
  EvalArgs g;
  OpArgs o;
  int mode;
  int scheme;
  int64_t ntiles;
};

struct ResQueue {             // mapped host memory
  unsigned long long published;
  int stop;
  int active;                 // blocks of the current launch not yet exited
};

struct ResItem {  // one claim: tiles [tile, tile + ntiles) of job `job`
  int job;
  int ntiles;
  int64_t tile;
};
constexpr int kItemTiles = 4;

constexpr unsigned long long kNoTile = ~0ull;

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_sys_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys_i32(int* p, int v) {
  asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// acquire-release add at device scope: a block's tile count orders its
// results before the count, and the last block's acquire sees every block's
__device__ __forceinline__ int atom_add_acq_rel_gpu(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Claim the next published tile (thread 0 of a block): kNoTile when the
// block should exit -- stop requested and nothing left, or idle for idle_ns.
__device__ unsigned long long claim_tile(ResQueue* q, unsigned long long* claimed, unsigned long long idle_ns,
                                         int* state) {
  const unsigned long long t0 = global_ns();
  unsigned sleep = 32;
  for (;;) {
    const unsigned long long pub = ld_acquire_sys(&q->published);  // items
    unsigned long long c = atomicAdd(claimed, 0ull);
    while (c < pub) {
      const unsigned long long prev = atomicCAS(claimed, c, c + 1);
      if (prev == c) return c;
      c = prev;
    }
    if (ld_acquire_sys_i32(&q->stop)) return kNoTile;
    if (global_ns() - t0 > idle_ns) {
      atomicOr(state, 1);
      return kNoTile;
    }
    __nanosleep(sleep);
    if (sleep < 256) sleep *= 2;
  }
}

template <class A, int PPT>
__global__ void __launch_bounds__(kTPB) resident_kernel(ResQueue* q, const ResJob* jobs, const ResItem* items,
                                                         unsigned long long* claimed, int* tiles_done, int* done,
                                                         unsigned long long idle_ns, int* state) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long s_item;
  __shared__ int s_job, s_ntiles, s_cached;
  __shared__ int64_t s_tile;
  __shared__ ResJob s_desc;
  if (threadIdx.x == 0) s_cached = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      s_item = claim_tile(q, claimed, idle_ns, state);
      if (s_item != kNoTile) {
        const volatile ResItem* it = (const volatile ResItem*)&items[s_item];
        s_job = it->job;
        s_ntiles = it->ntiles;
        s_tile = it->tile;
      }
    }
    __syncthreads();
    if (s_item == kNoTile) {
      if (threadIdx.x == 0) atomicSub_system(&q->active, 1);
      break;
    }
    const int job = s_job;
    // the descriptor into shared memory, unless it is already there (it was
    // written before its items were published: the acquire load ordered it)
    if (s_cached != job) {
      const int words = (int)(sizeof(ResJob) / 4);
      const volatile int* src = (const volatile int*)&jobs[job];
      for (int i = threadIdx.x; i < words; i += blockDim.x) ((int*)&s_desc)[i] = src[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_cached = job;
    // the arguments in registers: read from shared memory inside the tile
    // code, every store to the per-point table (shared memory too) could
    // alias them and force reloads in the hot loops
    const EvalArgs g = s_desc.g;
    const int mode = s_desc.mode, scheme = s_desc.scheme, ntiles = s_ntiles;
    const int64_t tile = s_tile;
    for (int t = 0; t < ntiles; ++t) {
      const int64_t base = (tile + t) * (kTPB * PPT);
      if constexpr (std::is_same<A, IV64>::value) {
        if (mode == kResModeNodeTable) node_tile<A, PPT, true>(g, base, smem_raw);
        else node_tile<A, PPT, false>(g, base, smem_raw);
      } else {
        if (mode == kResModeOps) {
          const OpArgs o = s_desc.o;
          if (scheme == FP_SCHEME_E) ops_tile<A, PPT, FP_SCHEME_E>(g, o, base, smem_raw);
          // Balanced: the extended path, which also runs plain Balanced schedules
          // (one instantiation less in this kernel, which serves every scheme)
          else if (scheme == FP_SCHEME_B) ops_tile<A, PPT, kSchemeBExt>(g, o, base, smem_raw);
          else ops_tile<A, PPT, 0>(g, o, base, smem_raw);
        } else if (mode == kResModeNodeTable) {
          node_tile<A, PPT, true>(g, base, smem_raw);
        } else {
          node_tile<A, PPT, false>(g, base, smem_raw);
        }
      }
    }
    // the block's results happen before thread 0's release (the barrier),
    // which the count carries to the last block; its system-scope release of
    // the flag is cumulative, so the host's acquire sees every result
    __syncthreads();
    if (threadIdx.x == 0) {
      if (atom_add_acq_rel_gpu(&tiles_done[job], ntiles) + ntiles == (int)s_desc.ntiles)
        st_release_sys_i32(&done[job], 1);
    }
    __syncthreads();
  }
}

int fill_eval_args(const fp_tree* t, fp_dtype dt, const void* points, int64_t npts, void* out, EvalArgs& a, OpArgs& o);
void lookup_tuned(const fp_tree* t, fp_dtype dt, int64_t npts, int& variant, int& ppt);

namespace {

int res_ppt(fp_dtype dt) { return (dt == FP_F32C || dt == FP_MODP) ? 2 : 1; }

template <class A, int PPT>
cudaError_t res_launch(int grid, size_t smem, cudaStream_t st, ResQueue* q, const ResJob* jobs, const ResItem* items,
                       unsigned long long* claimed, int* tiles_done, int* done, unsigned long long idle_ns,
                       int* state) {
  cudaError_t e = cudaFuncSetAttribute(resident_kernel<A, PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  resident_kernel<A, PPT><<<grid, kTPB, smem, st>>>(q, jobs, items, claimed, tiles_done, done, idle_ns, state);
  return cudaGetLastError();
}

template <class A, int PPT>
int res_occupancy(size_t smem) {
  int n = 0;
  if (cudaFuncSetAttribute(resident_kernel<A, PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, resident_kernel<A, PPT>, kTPB, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace
}  // namespace fp

struct fp_resident {
  fp_dtype dtype = FP_F64;
  int device = -1;
  size_t smem = 0;
  int grid = 0;
  int max_jobs = 0;
  int64_t max_items = 0;
  unsigned long long idle_ns = 0;
  cudaStream_t stream = nullptr;
  bool running = false;
  // mapped host memory and its device addresses
  fp::ResQueue* q = nullptr;
  fp::ResQueue* dq = nullptr;
  fp::ResJob* jobs = nullptr;
  fp::ResJob* djobs = nullptr;
  fp::ResItem* items = nullptr;
  fp::ResItem* ditems = nullptr;
  int* done = nullptr;
  int* ddone = nullptr;
  // device memory
  unsigned long long* claimed = nullptr;
  int* tiles_done = nullptr;
  int* state = nullptr;
  int64_t njobs = 0;
  unsigned long long nitems = 0;  // items published
};

namespace fp {
namespace {

int res_start(fp_resident* r) {
  cudaError_t e = cudaSuccess;
  reinterpret_cast<std::atomic<int>*>(&r->q->active)->store(r->grid, std::memory_order_release);
#define FP_RES_LAUNCH(T, P)                                                                                      \
  e = res_launch<T, P>(r->grid, r->smem, r->stream, r->dq, r->djobs, r->ditems, r->claimed, r->tiles_done, r->ddone, \
                       r->idle_ns, r->state)
  switch (r->dtype) {
    case FP_F64: FP_RES_LAUNCH(F64, 1); break;
    case FP_F32C: FP_RES_LAUNCH(F32C, 2); break;
    case FP_IV64: FP_RES_LAUNCH(IV64, 1); break;
    case FP_MODP: FP_RES_LAUNCH(MODP, 2); break;
  }
#undef FP_RES_LAUNCH
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FP_E_CUDA;
  }
  r->running = true;
  return FP_OK;
}

void res_release(fp_resident* r) {
  if (r->q) cudaFreeHost(r->q);
  if (r->jobs) cudaFreeHost(r->jobs);
  if (r->items) cudaFreeHost(r->items);
  if (r->done) cudaFreeHost(r->done);
  if (r->claimed) cudaFree(r->claimed);
  if (r->tiles_done) cudaFree(r->tiles_done);
  if (r->state) cudaFree(r->state);
  if (r->stream) cudaStreamDestroy(r->stream);
  cudaGetLastError();
}

// A kernel whose blocks all left on an idle timeout is relaunched (the
// queue's counters persist); a block may time out just before a submission
// it did not see, so waits call this too.
int res_kick(fp_resident* r) {
  // every block of the launch has left (a plain read of the count the blocks
  // decrement on exit; no driver call on the submission path)
  if (r->running && reinterpret_cast<std::atomic<int>*>(&r->q->active)->load(std::memory_order_acquire) == 0) {
    if (cudaStreamSynchronize(r->stream) != cudaSuccess) {
      cudaGetLastError();
      return FP_E_CUDA;
    }
    r->running = false;
  }
  if (r->running || r->q->stop) return FP_OK;
  unsigned long long claimed = 0;
  if (cudaMemcpy(&claimed, r->claimed, sizeof(claimed), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return FP_E_CUDA;
  }
  return claimed < r->nitems ? res_start(r) : FP_OK;
}

// wait (at most timeout_s) for the resident kernel's stream to finish
int res_join(fp_resident* r, double timeout_s) {
  if (!r->running) return FP_OK;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(r->stream);
    if (e == cudaSuccess) {
      r->running = false;
      return FP_OK;
    }
    if (e != cudaErrorNotReady) {
      cudaGetLastError();
      r->running = false;
      return FP_E_CUDA;
    }
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout_s)
      return FP_E_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" {

int fp_resident_create(const fp_resident_cfg* cfg, fp_resident** out) {
  if (!cfg || !out) return FP_E_BAD_VALUE;
  if ((int)cfg->dtype < FP_F64 || (int)cfg->dtype > FP_MODP) return FP_E_DTYPE;
  if (cfg->max_jobs <= 0 || cfg->max_jobs > (1 << 24)) return FP_E_BAD_VALUE;
  const size_t smem = cfg->smem_bytes ? cfg->smem_bytes : (size_t)48 * 1024;
  if (smem > kSmemMax || smem < 1024) return FP_E_BAD_VALUE;
  fp_resident* r = new (std::nothrow) fp_resident();
  if (!r) return FP_E_NOMEM;
  r->dtype = cfg->dtype;
  r->smem = smem;
  r->max_jobs = cfg->max_jobs;
  r->idle_ns = (unsigned long long)((cfg->idle_exit_s > 0 ? cfg->idle_exit_s : 0.05) * 1e9);
  int rc = FP_OK;
  if (cudaGetDevice(&r->device) != cudaSuccess) rc = FP_E_CUDA;
  int per_sm = 0;
  if (rc == FP_OK) {
    switch (r->dtype) {
      case FP_F64: per_sm = res_occupancy<F64, 1>(smem); break;
      case FP_F32C: per_sm = res_occupancy<F32C, 2>(smem); break;
      case FP_IV64: per_sm = res_occupancy<IV64, 1>(smem); break;
      case FP_MODP: per_sm = res_occupancy<MODP, 2>(smem); break;
    }
    if (per_sm <= 0) rc = FP_E_TOO_LARGE;
  }
  if (rc == FP_OK) {
    const int blocks = cfg->blocks_per_sm > 0 ? std::min(cfg->blocks_per_sm, per_sm) : per_sm;
    r->grid = blocks * sm_count();
  }
  const size_t jbytes = sizeof(ResJob) * (size_t)r->max_jobs;
  r->max_items = cfg->max_items > 0 ? cfg->max_items : std::max<int64_t>(16 * (int64_t)r->max_jobs, 65536);
  if (rc == FP_OK && (cudaHostAlloc((void**)&r->q, sizeof(ResQueue), cudaHostAllocMapped) != cudaSuccess ||
                      cudaHostAlloc((void**)&r->jobs, jbytes, cudaHostAllocMapped) != cudaSuccess ||
                      cudaHostAlloc((void**)&r->items, sizeof(ResItem) * (size_t)r->max_items, cudaHostAllocMapped) !=
                          cudaSuccess ||
                      cudaHostAlloc((void**)&r->done, sizeof(int) * r->max_jobs, cudaHostAllocMapped) != cudaSuccess ||
                      cudaMalloc((void**)&r->claimed, sizeof(unsigned long long)) != cudaSuccess ||
                      cudaMalloc((void**)&r->tiles_done, sizeof(int) * r->max_jobs) != cudaSuccess ||
                      cudaMalloc((void**)&r->state, sizeof(int)) != cudaSuccess))
    rc = FP_E_NOMEM;
  if (rc == FP_OK && (cudaHostGetDevicePointer((void**)&r->dq, r->q, 0) != cudaSuccess ||
                      cudaHostGetDevicePointer((void**)&r->djobs, r->jobs, 0) != cudaSuccess ||
                      cudaHostGetDevicePointer((void**)&r->ditems, r->items, 0) != cudaSuccess ||
                      cudaHostGetDevicePointer((void**)&r->ddone, r->done, 0) != cudaSuccess))
    rc = FP_E_CUDA;
  if (rc == FP_OK) {
    std::memset(r->q, 0, sizeof(ResQueue));
    std::memset(r->jobs, 0, jbytes);
    std::memset(r->done, 0, sizeof(int) * r->max_jobs);
    if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemset(r->claimed, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(r->tiles_done, 0, sizeof(int) * r->max_jobs) != cudaSuccess ||
        cudaMemset(r->state, 0, sizeof(int)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      rc = FP_E_CUDA;
  }
  if (rc == FP_OK) rc = res_start(r);
  if (rc != FP_OK) {
    cudaGetLastError();
    res_release(r);
    delete r;
    return rc;
  }
  *out = r;
  return FP_OK;
}

int fp_resident_submit(fp_resident* r, const fp_job* job, int64_t* ticket) {
  if (!r || !job || !job->tree || job->npts < 0) return FP_E_BAD_VALUE;
  if (r->q->stop) return FP_E_BAD_VALUE;  // stopped: no further work
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != r->device) { cudaGetLastError(); return FP_E_BAD_VALUE; }
  if (r->njobs >= r->max_jobs) return FP_E_TOO_LARGE;
  if (job->npts > 0 && (!job->points || !job->out)) return FP_E_BAD_VALUE;
  if (job->tree->nnodes == 0) return FP_E_BAD_VALUE;  // zero polynomials: use fp_eval
  const int k = (int)r->njobs;
  ResJob j{};
  int rc = fill_eval_args(job->tree, r->dtype, job->points, job->npts, job->out, j.g, j.o);
  if (rc != FP_OK) return rc;
  const int ppt = res_ppt(r->dtype);
  const size_t vb = r->dtype == FP_IV64 ? 16 : 8;
  const size_t table = (vb * j.g.nslot + vb * j.g.npow) * ppt * kTPB;
  const size_t fly = (vb * j.g.nslot + vb * j.g.nvars) * ppt * kTPB;
  const size_t ops_table = vb * (size_t)j.o.entries * ppt * kTPB;
  int tv = 0, tp = 0;
  lookup_tuned(job->tree, r->dtype, job->npts, tv, tp);
  if (r->dtype != FP_IV64 && tv != 2 && ops_table <= r->smem && j.o.recs) j.mode = kResModeOps;
  else if (table <= r->smem) j.mode = kResModeNodeTable;
  else if (fly <= r->smem) j.mode = kResModeNodeFly;
  else return FP_E_TOO_LARGE;
  j.scheme = job->tree->block_scheme;
  j.ntiles = (job->npts + (int64_t)kTPB * ppt - 1) / ((int64_t)kTPB * ppt);
  const int64_t nit = (j.ntiles + kItemTiles - 1) / kItemTiles;
  if ((int64_t)r->nitems + nit > r->max_items) return FP_E_TOO_LARGE;
  if (j.ntiles > 0x7FFFFFFF) return FP_E_TOO_LARGE;
  // the descriptor and the items, then (release) the new count of published
  // items: a block that sees the count sees both
  std::memcpy(&r->jobs[k], &j, sizeof(ResJob));
  for (int64_t i = 0; i < nit; ++i) {
    ResItem& it = r->items[r->nitems + i];
    it.job = k;
    it.tile = i * kItemTiles;
    it.ntiles = (int)std::min<int64_t>(kItemTiles, j.ntiles - i * kItemTiles);
  }
  if (nit == 0) r->done[k] = 1;  // nothing to evaluate
  std::atomic_thread_fence(std::memory_order_release);
  r->nitems += (unsigned long long)nit;
  reinterpret_cast<std::atomic<unsigned long long>*>(&r->q->published)->store(r->nitems, std::memory_order_release);
  r->njobs = k + 1;
  if (ticket) *ticket = k;
  return nit > 0 ? res_kick(r) : FP_OK;
}

int fp_resident_query(const fp_resident* r, int64_t ticket) {
  if (!r || ticket < 0 || ticket >= r->njobs) return FP_E_BAD_VALUE;
  return reinterpret_cast<const std::atomic<int>*>(&r->done[ticket])->load(std::memory_order_acquire) ? FP_OK : 1;
}

int fp_resident_wait(fp_resident* r, int64_t ticket, double timeout_s) {
  if (!r || ticket < 0 || ticket >= r->njobs) return FP_E_BAD_VALUE;
  const auto t0 = std::chrono::steady_clock::now();
  for (int it = 0;; ++it) {
    if (fp_resident_query(r, ticket) == FP_OK) return FP_OK;
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout_s) return FP_E_TIMEOUT;
    if ((it & 1023) == 1023) {
      const int rc = res_kick(r);
      if (rc != FP_OK) return rc;
    }
    std::this_thread::yield();
  }
}

int fp_resident_state(const fp_resident* r, int* running, int* idle_exits, int64_t* jobs) {
  if (!r) return FP_E_BAD_VALUE;
  if (running) *running = r->running && cudaStreamQuery(r->stream) != cudaSuccess;
  cudaGetLastError();
  if (idle_exits) {
    int s = 0;
    if (cudaMemcpy(&s, r->state, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return FP_E_CUDA;
    }
    *idle_exits = s & 1;
  }
  if (jobs) *jobs = r->njobs;
  return FP_OK;
}

int fp_resident_stop(fp_resident* r, double timeout_s) {
  if (!r) return FP_E_BAD_VALUE;
  reinterpret_cast<std::atomic<int>*>(&r->q->stop)->store(1, std::memory_order_release);
  return res_join(r, timeout_s > 0 ? timeout_s : 60.0);
}

void fp_resident_free(fp_resident* r) {
  if (!r) return;
  if (fp_resident_stop(r, 60.0) == FP_OK) res_release(r);
  delete r;  // a kernel that did not stop keeps its buffers (leaked rather than freed under it)
}

}  // extern "C"
