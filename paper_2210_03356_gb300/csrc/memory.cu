// Device memory of the library: its stream-ordered pool and the per-thread
// cache of freed blocks in front of it.
#include <map>
#include <mutex>

#include "../../include/sign.h"
#include "common.cuh"

namespace sgn {

cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  SGN_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error(5, "device index out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    SGN_CUDA(cudaMemPoolCreate(&p, &props));
    uint64_t keep = ~uint64_t(0);
    SGN_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
    pools[dev] = p;
  }
  return pools[dev];
}

namespace {
// the parked blocks of this thread, by size
struct BlockCache {
  struct Block {
    void *p;
    cudaStream_t s;
  };
  std::multimap<size_t, Block> free;
  size_t bytes = 0;
  // No CUDA call here: at process exit the runtime may already be gone, and
  // the process's memory goes with it. Threads that end before the process
  // call block_cache_flush() first.
  ~BlockCache() = default;
  // The streams the blocks were parked with may have been destroyed since
  // (a server's upload stream, a caller's stream), so none of them is used:
  // once the device is idle, every parked block is unused and freed directly.
  void flush() {
    if (free.empty()) return;
    cudaDeviceSynchronize();
    for (auto &kv : free) cudaFree(kv.second.p);
    free.clear();
    bytes = 0;
  }
};
thread_local BlockCache t_blocks;
thread_local bool t_cache_on = true;
constexpr size_t kCacheMaxBytes = size_t(96) << 30;  // parked at most, per thread
}  // namespace

void block_cache_enable(bool on) {
  if (!on) t_blocks.flush();
  t_cache_on = on;
}

void *block_alloc(size_t bytes, cudaStream_t s, size_t &cap, const void *&owner) {
  BlockCache &c = t_blocks;
  owner = t_cache_on ? &c : nullptr;
  for (auto it = c.free.lower_bound(bytes); it != c.free.end() && it->first <= 2 * bytes + (1 << 20);
       ++it) {
    if (it->second.s != s) continue;
    void *p = it->second.p;
    cap = it->first;
    c.bytes -= it->first;
    c.free.erase(it);
    return p;
  }
  void *p = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, lib_pool(), s);
  if (e == cudaErrorMemoryAllocation && !c.free.empty()) {
    cudaGetLastError();
    c.flush();  // parked blocks back to the pool, then once more
    e = cudaMallocFromPoolAsync(&p, bytes, lib_pool(), s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? 2 : 5,
                std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
  }
  cap = bytes;
  return p;
}

void block_cache_flush() { t_blocks.flush(); }

void block_free(void *p, size_t cap, cudaStream_t s, const void *owner) {
  BlockCache &c = t_blocks;
  if (!t_cache_on || owner != &c || c.bytes + cap > kCacheMaxBytes) {
    cudaFreeAsync(p, s);
    return;
  }
  try {  // runs in destructors: no exception may leave
    c.free.emplace(cap, BlockCache::Block{p, s});
    c.bytes += cap;
  } catch (...) {
    cudaFreeAsync(p, s);
  }
}

}  // namespace sgn

extern "C" {

sign_status sign_trim_memory(void) {
  try {
    sgn::block_cache_flush();
    SGN_CUDA(cudaDeviceSynchronize());  // frees queued on streams take effect first
    SGN_CUDA(cudaMemPoolTrimTo(sgn::lib_pool(), 0));
  } catch (const sgn::Error &e) {
    sgn::set_last_error(e.what());
    return sign_status(e.status);
  }
  return SIGN_OK;
}

}  // extern "C"
