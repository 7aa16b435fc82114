// Serving loop with continuous batching.
//
// Callers submit evaluation requests (a resident compiled tree, a value type,
// host points and a host result buffer) from any thread.  One worker thread:
//   - retires batches whose completion event has fired (requests complete,
//     their device memory returns to the budget);
//   - admits pending requests, oldest first, while their device footprint
//     (points + results) fits in the HBM budget, grouping requests of one
//     value type and one size class into one batched launch (fp_eval_batch)
//     in a free slot: host->device copies, the launch, device->host copies,
//     release of the buffers, then an event -- all stream-ordered.  A batch
//     lasts as long as its largest request, so small requests (estimated
//     work below kSmallWork) are never batched with large ones and run on
//     high-priority streams, and with two or more slots the first is kept
//     for small requests (an express lane);
//   - sleeps on a condition variable (bounded) when there is nothing to do.
// Requests arriving while batches run are admitted as soon as a slot and
// memory are free, so their work overlaps with the batches in flight.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fastpoly.h"
#include "tree.hpp"

namespace fp {
int eval_device(const fp_tree* t, fp_dtype dt, const void* points, int64_t npts, void* out, cudaStream_t st,
                int variant, int ppt);
}

namespace {

using Clock = std::chrono::steady_clock;

size_t in_bytes_of(fp_dtype dt, int nvars, int64_t npts) {
  const size_t b = dt == FP_F32C ? 4 : (dt == FP_IV64 ? 16 : 8);
  return b * (size_t)nvars * (size_t)npts;
}
size_t out_bytes_of(fp_dtype dt, int64_t npts) { return (dt == FP_IV64 ? 16 : 8) * (size_t)npts; }

// Estimated work of a request in FP64 node-evaluations: nodes x points x the
// value type's cost per node relative to FP64 (measured throughputs: FP32C
// about 4x faster, intervals about 4.7x slower, residues about as fast).
double work_of(const fp_tree* t, fp_dtype dt, int64_t npts) {
  const double w = dt == FP_F32C ? 0.25 : (dt == FP_IV64 ? 4.7 : 1.0);
  return w * (double)t->nnodes * (double)npts;
}
// below this a request is small: about 1.7 ms of FP64 work on the GPU
constexpr double kSmallWork = 1.0e9;

struct Request {
  int64_t ticket = 0;
  const fp_tree* tree = nullptr;
  fp_dtype dtype = FP_F64;
  const void* in_host = nullptr;
  void* out_host = nullptr;
  int64_t npts = 0;
  size_t in_bytes = 0, out_bytes = 0;
  bool small = true;  // estimated work below kSmallWork
  Clock::time_point t_submit;
  void* d_in = nullptr;
  void* d_out = nullptr;
};

struct Slot {
  cudaStream_t stream = nullptr;     // large requests (default priority)
  cudaStream_t stream_hi = nullptr;  // small requests (highest priority)
  cudaEvent_t done = nullptr;
  std::vector<Request> reqs;
  size_t bytes = 0;
  int status = FP_OK;
  bool busy = false;
};

}  // namespace

struct fp_server {
  fp_server_cfg cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> submitted;  // guarded by mu
  std::deque<fp_completion> completed;  // guarded by mu
  int64_t next_ticket = 0, n_submitted = 0, n_completed = 0;  // guarded by mu
  bool stop = false;  // guarded by mu
  // worker-owned
  std::deque<Request> pending;
  std::vector<Slot> slots;
  size_t used_bytes = 0;
  // statistics (worker writes)
  std::atomic<size_t> peak_bytes{0};
  std::atomic<int64_t> batches{0};
  std::thread worker;

  void complete(const Request& r, int status) {
    fp_completion c;
    c.ticket = r.ticket;
    c.status = status;
    c.latency_us = std::chrono::duration<double, std::micro>(Clock::now() - r.t_submit).count();
    std::lock_guard<std::mutex> g(mu);
    completed.push_back(c);
    ++n_completed;
    cv_done.notify_all();
  }

  // returns true if something was retired
  bool retire() {
    bool any = false;
    for (Slot& s : slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      int st = s.status;
      if (q != cudaSuccess) {
        cudaGetLastError();
        st = FP_E_CUDA;
      }
      for (const Request& r : s.reqs) complete(r, st);
      used_bytes -= s.bytes;
      s.reqs.clear();
      s.bytes = 0;
      s.busy = false;
      any = true;
    }
    return any;
  }

  // admit and launch one batch on slot s; returns true if launched.  The
  // batch takes the oldest pending request (the oldest small one on the
  // express slot, so that small requests always have a slot) and others of
  // its value type and size class.
  bool dispatch(Slot& s, bool express) {
    auto first = pending.begin();
    if (express)
      while (first != pending.end() && !first->small) ++first;
    if (first == pending.end()) return false;
    const fp_dtype dt = first->dtype;
    const bool small = first->small;
    const int maxjobs = cfg.max_batch_jobs > 0 ? cfg.max_batch_jobs : 1024;
    std::vector<Request> take;
    size_t bytes = 0;
    for (auto it = first; it != pending.end() && (int)take.size() < maxjobs;) {
      if (it->dtype != dt || it->small != small) { ++it; continue; }
      const size_t need = it->in_bytes + it->out_bytes;
      const bool alone = take.empty() && used_bytes == 0;  // larger than the budget: run it by itself
      if (used_bytes + bytes + need > cfg.hbm_budget_bytes && !alone) break;  // oldest first: no overtaking
      bytes += need;
      take.push_back(*it);
      it = pending.erase(it);
    }
    if (take.empty()) return false;
    // small batches run on the slot's high-priority stream: the block
    // scheduler then runs their blocks ahead of those a large batch still has
    // waiting on the other streams
    const cudaStream_t st = small ? s.stream_hi : s.stream;
    int status = FP_OK;
    std::vector<fp_job> jobs;
    jobs.reserve(take.size());
    for (Request& r : take) {
      if (fp::pool_alloc(&r.d_in, r.in_bytes ? r.in_bytes : 16, st) != cudaSuccess ||
          fp::pool_alloc(&r.d_out, r.out_bytes ? r.out_bytes : 16, st) != cudaSuccess) {
        cudaGetLastError();
        status = FP_E_NOMEM;
        break;
      }
      if (r.in_bytes && cudaMemcpyAsync(r.d_in, r.in_host, r.in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        status = FP_E_CUDA;
      if (r.tree->nnodes == 0) {  // the zero polynomial goes through fp_eval
        if (fp::eval_device(r.tree, r.dtype, r.d_in, r.npts, r.d_out, st, 0, 0) != FP_OK) status = FP_E_CUDA;
      } else {
        fp_job j;
        j.tree = r.tree;
        j.points = r.d_in;
        j.npts = r.npts;
        j.out = r.d_out;
        jobs.push_back(j);
      }
    }
    if (status == FP_OK && !jobs.empty()) status = fp_eval_batch(dt, jobs.data(), (int64_t)jobs.size(), st);
    for (Request& r : take) {
      if (status == FP_OK && r.out_bytes &&
          cudaMemcpyAsync(r.out_host, r.d_out, r.out_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        status = FP_E_CUDA;
      if (r.d_in) cudaFreeAsync(r.d_in, st);
      if (r.d_out) cudaFreeAsync(r.d_out, st);
    }
    cudaEventRecord(s.done, st);
    s.reqs = std::move(take);
    s.bytes = bytes;
    s.status = status;
    s.busy = true;
    used_bytes += bytes;
    if (used_bytes > peak_bytes) peak_bytes = used_bytes;
    ++batches;
    return true;
  }

  void run() {
    cudaSetDevice(device);
    for (;;) {
      bool stopping;
      {
        std::unique_lock<std::mutex> lk(mu);
        while (!submitted.empty()) {
          pending.push_back(std::move(submitted.front()));
          submitted.pop_front();
        }
        stopping = stop;
      }
      bool progress = retire();
      for (size_t i = 0; i < slots.size(); ++i)
        if (!slots[i].busy && dispatch(slots[i], i == 0 && slots.size() > 1)) progress = true;
      bool busy = false;
      for (const Slot& s : slots) busy = busy || s.busy;
      if (stopping && !busy && pending.empty()) {
        std::lock_guard<std::mutex> g(mu);
        if (submitted.empty()) break;
        continue;
      }
      if (!progress) {
        std::unique_lock<std::mutex> lk(mu);
        // bounded sleep: woken early by a submission; in-flight batches are polled
        cv_work.wait_for(lk, std::chrono::microseconds(busy ? 20 : 2000),
                         [&] { return !submitted.empty() || stop; });
      }
    }
  }
};

extern "C" {

int fp_server_create(const fp_server_cfg* cfg, fp_server** out) {
  if (!cfg || !out || cfg->hbm_budget_bytes == 0) return FP_E_BAD_VALUE;
  fp_server* s = new (std::nothrow) fp_server();
  if (!s) return FP_E_NOMEM;
  s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return FP_E_CUDA;
  }
  const int ns = cfg->streams > 0 ? cfg->streams : 4;
  s->slots.resize(ns);
  // per slot a default-priority stream (large batches) and a highest-priority
  // one (small batches)
  int prio_low = 0, prio_high = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
    cudaGetLastError();
    prio_low = prio_high = 0;
  }
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, prio_low) != cudaSuccess ||
        cudaStreamCreateWithPriority(&sl.stream_hi, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (Slot& x : s->slots) {
        if (x.stream) cudaStreamDestroy(x.stream);
        if (x.stream_hi) cudaStreamDestroy(x.stream_hi);
        if (x.done) cudaEventDestroy(x.done);
      }
      delete s;
      return FP_E_CUDA;
    }
  }
  try {
    s->worker = std::thread([s] { s->run(); });
  } catch (...) {
    for (Slot& x : s->slots) {
      cudaStreamDestroy(x.stream);
      cudaStreamDestroy(x.stream_hi);
      cudaEventDestroy(x.done);
    }
    delete s;
    return FP_E_NOMEM;
  }
  *out = s;
  return FP_OK;
}

int fp_server_submit(fp_server* s, const fp_tree* tree, fp_dtype dtype, const void* points_host, int64_t npts,
                     void* out_host, int64_t* ticket) {
  if (!s || !tree || npts < 0 || (npts > 0 && (!points_host || !out_host))) return FP_E_BAD_VALUE;
  if ((int)dtype < FP_F64 || (int)dtype > FP_MODP) return FP_E_DTYPE;
  if (tree->dev.device != s->device) return FP_E_BAD_VALUE;
  if (dtype == FP_MODP ? tree->coeff_type != FP_MODP : tree->coeff_type != FP_F64) return FP_E_DTYPE;
  Request r;
  r.tree = tree;
  r.dtype = dtype;
  r.in_host = points_host;
  r.out_host = out_host;
  r.npts = npts;
  r.in_bytes = in_bytes_of(dtype, tree->nvars, npts);
  r.out_bytes = out_bytes_of(dtype, npts);
  r.small = work_of(tree, dtype, npts) < kSmallWork;
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return FP_E_BAD_VALUE;
    r.ticket = s->next_ticket++;
    ++s->n_submitted;
    if (ticket) *ticket = r.ticket;
    if (npts == 0) {  // nothing to do
      fp_completion c{r.ticket, FP_OK, 0.0};
      s->completed.push_back(c);
      ++s->n_completed;
      s->cv_done.notify_all();
      return FP_OK;
    }
    s->submitted.push_back(r);
  }
  s->cv_work.notify_one();
  return FP_OK;
}

int fp_server_poll(fp_server* s, fp_completion* done, int max, int* n) {
  if (!s || !n || max < 0 || (max > 0 && !done)) return FP_E_BAD_VALUE;
  std::lock_guard<std::mutex> g(s->mu);
  int k = 0;
  while (k < max && !s->completed.empty()) {
    done[k++] = s->completed.front();
    s->completed.pop_front();
  }
  *n = k;
  return FP_OK;
}

int fp_server_drain(fp_server* s, double timeout_s) {
  if (!s) return FP_E_BAD_VALUE;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 60.0);
  while (s->n_completed < s->n_submitted) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->n_completed < s->n_submitted)
      return FP_E_TIMEOUT;
  }
  return FP_OK;
}

int fp_server_stats(const fp_server* s, size_t* peak_bytes, int64_t* batches) {
  if (!s) return FP_E_BAD_VALUE;
  if (peak_bytes) *peak_bytes = s->peak_bytes;
  if (batches) *batches = s->batches;
  return FP_OK;
}

void fp_server_destroy(fp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (Slot& x : s->slots) {
    cudaStreamSynchronize(x.stream);
    cudaStreamSynchronize(x.stream_hi);
    cudaStreamDestroy(x.stream);
    cudaStreamDestroy(x.stream_hi);
    cudaEventDestroy(x.done);
  }
  delete s;
}

}  // extern "C"
