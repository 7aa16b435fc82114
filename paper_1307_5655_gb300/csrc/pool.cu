// Device memory for the library's own work space: one stream-ordered pool per
// device that keeps up to kPoolKeepBytes of freed memory mapped for reuse, so
// that repeated calls (host-buffer evaluations, batches, compositions, the
// server) do not map and unmap device memory every time.  The default pool
// of the CUDA runtime returns freed memory at every synchronisation.
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "tree.hpp"

namespace fp {

namespace {
constexpr uint64_t kPoolKeepBytes = 4ull << 30;
}

cudaMemPool_t device_pool() {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> g(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = kPoolKeepBytes;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaGetLastError();
    pools[dev] = p;
  }
  return pools[dev];
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = device_pool();
  if (!pool) return cudaMallocAsync(p, bytes, st);
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

}  // namespace fp
