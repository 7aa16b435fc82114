// fp_eval_host's data path: host points in, host results out, with the
// copies overlapping the evaluation.  Points are [rows][npts] rows of
// elements (rows = variables, twice that for intervals) and results
// [orows][npts]; a chunk of points [j0, j0 + m) is then one strided 2D copy
// each way, and the device buffers of a chunk are [rows][m] / [orows][m],
// the layout fp_eval expects for m points.
#include <algorithm>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "tree.hpp"

namespace fp {

int eval_device(const fp_tree* t, fp_dtype dt, const void* points, int64_t npts, void* out, cudaStream_t st,
                int variant, int ppt);

namespace {

constexpr int64_t kChunkPoints = 1 << 21;  // pipelining pays above about two chunks
constexpr int kMaxChunks = 16;

// two non-blocking copy streams per device (copies in, copies out)
int copy_streams(cudaStream_t& in, cudaStream_t& out) {
  static std::mutex mu;
  static std::vector<std::pair<cudaStream_t, cudaStream_t>> ss;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FP_E_CUDA;
  }
  std::lock_guard<std::mutex> g(mu);
  if ((int)ss.size() <= dev) ss.resize(dev + 1, {nullptr, nullptr});
  if (!ss[dev].first) {
    cudaStream_t a = nullptr, b = nullptr;
    if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      if (a) cudaStreamDestroy(a);
      return FP_E_CUDA;
    }
    ss[dev] = {a, b};
  }
  in = ss[dev].first;
  out = ss[dev].second;
  return FP_OK;
}

void shape(fp_dtype dt, int nvars, int& rows, size_t& elem, int& orows, size_t& oelem) {
  rows = dt == FP_IV64 ? 2 * nvars : nvars;
  elem = dt == FP_F32C ? 4 : 8;
  orows = (dt == FP_F32C || dt == FP_IV64) ? 2 : 1;
  oelem = dt == FP_F32C ? 4 : 8;
}

}  // namespace

int eval_host_pipelined(const fp_tree* t, fp_dtype dtype, const void* points_host, int64_t npts, void* out_host,
                        cudaStream_t st) {
  int rows, orows;
  size_t elem, oelem;
  shape(dtype, t->nvars, rows, elem, orows, oelem);
  int64_t nchunks = std::min<int64_t>(kMaxChunks, (npts + kChunkPoints - 1) / kChunkPoints);
  if (nchunks < 2) nchunks = 1;
  const int64_t m = (npts + nchunks - 1) / nchunks;  // points per chunk (the last may be shorter)
  const int nbuf = nchunks > 1 ? 2 : 1;
  const size_t in_bytes = (size_t)rows * m * elem, out_bytes = (size_t)orows * m * oelem;
  void* din[2] = {nullptr, nullptr};
  void* dout[2] = {nullptr, nullptr};
  int rc = FP_OK;
  for (int b = 0; b < nbuf && rc == FP_OK; ++b)
    if (pool_alloc(&din[b], in_bytes, st) != cudaSuccess || pool_alloc(&dout[b], out_bytes, st) != cudaSuccess)
      rc = FP_E_NOMEM;
  cudaStream_t s_in = st, s_out = st;
  if (rc == FP_OK && nchunks > 1) rc = copy_streams(s_in, s_out);
  std::vector<cudaEvent_t> ev;  // per chunk: in ready, evaluated, out copied
  if (rc == FP_OK && nchunks > 1) {
    ev.assign(3 * nchunks, nullptr);
    for (auto& e : ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = FP_E_CUDA;
    // the copy streams start after whatever the caller queued on its stream
    cudaEvent_t start = nullptr;
    if (rc == FP_OK && cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(start, st);
      cudaStreamWaitEvent(s_in, start, 0);
      cudaStreamWaitEvent(s_out, start, 0);
      cudaEventDestroy(start);
    } else {
      rc = FP_E_CUDA;
    }
  }
  for (int64_t i = 0; i < nchunks && rc == FP_OK; ++i) {
    const int64_t j0 = i * m, len = std::min<int64_t>(m, npts - j0);
    if (len <= 0) break;
    const int b = (int)(i % nbuf);
    if (nchunks > 1 && i >= 2) cudaStreamWaitEvent(s_in, ev[3 * (i - 2) + 1], 0);  // din[b] read by chunk i - 2
    if (cudaMemcpy2DAsync(din[b], len * elem, (const char*)points_host + j0 * elem, npts * elem, len * elem, rows,
                          cudaMemcpyHostToDevice, s_in) != cudaSuccess) {
      rc = FP_E_CUDA;
      break;
    }
    if (nchunks > 1) {
      cudaEventRecord(ev[3 * i], s_in);
      cudaStreamWaitEvent(st, ev[3 * i], 0);
      if (i >= 2) cudaStreamWaitEvent(st, ev[3 * (i - 2) + 2], 0);  // dout[b] copied out for chunk i - 2
    }
    rc = eval_device(t, dtype, din[b], len, dout[b], st, 0, 0);
    if (rc != FP_OK) break;
    if (nchunks > 1) {
      cudaEventRecord(ev[3 * i + 1], st);
      cudaStreamWaitEvent(s_out, ev[3 * i + 1], 0);
    }
    if (cudaMemcpy2DAsync((char*)out_host + j0 * oelem, npts * oelem, dout[b], len * oelem, len * oelem, orows,
                          cudaMemcpyDeviceToHost, s_out) != cudaSuccess) {
      rc = FP_E_CUDA;
      break;
    }
    if (nchunks > 1) cudaEventRecord(ev[3 * i + 2], s_out);
  }
  // the caller's stream waits for every copy out, then releases the buffers
  if (nchunks > 1) {
    cudaEvent_t done = nullptr;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(done, s_out);
      cudaStreamWaitEvent(st, done, 0);
      cudaEventRecord(done, s_in);
      cudaStreamWaitEvent(st, done, 0);
      cudaEventDestroy(done);
    } else if (rc == FP_OK) {
      rc = FP_E_CUDA;
    }
  }
  for (int b = 0; b < 2; ++b) {
    if (din[b]) cudaFreeAsync(din[b], st);
    if (dout[b]) cudaFreeAsync(dout[b], st);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == FP_OK) rc = FP_E_CUDA;
  if (nchunks > 1) {  // copy streams idle again (also after an error part-way)
    cudaStreamSynchronize(s_in);
    cudaStreamSynchronize(s_out);
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  return rc;
}

}  // namespace fp
