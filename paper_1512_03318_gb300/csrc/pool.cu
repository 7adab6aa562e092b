// Device memory cache of the library.
//
// A two-site update builds an H_eff (charge tables, folded environments, packed tensor-core
// and float-float operands, Lanczos vectors: a few GB at chi = 3200) and frees it when the
// update ends. cudaMalloc and cudaFree of that much memory cost milliseconds and cudaFree
// synchronises the device, so released blocks are kept here and handed out again to later
// requests. A block is reused only on the stream that released it: work already queued on
// that stream precedes any new use in stream order. When cudaMalloc runs out of memory the
// cached blocks of the device are freed and the allocation is retried.
#include <map>
#include <mutex>
#include <unordered_map>

#include "mrd_internal.h"

namespace mrd {

namespace {

struct Block {
  size_t bytes;
  int device;
};

struct Cache {
  std::mutex mu;
  std::map<std::pair<int, cudaStream_t>, std::multimap<size_t, void*>> free_blocks;
  std::unordered_map<void*, Block> live;     // every block the cache owns (in use or free)
};

Cache& cache() {
  static Cache* c = new Cache();   // never destroyed: blocks may be released during exit
  return *c;
}

size_t round_bytes(size_t b) {
  if (b < 256) b = 256;
  const size_t g = b >= ((size_t)1 << 20) ? ((size_t)2 << 20) : 512;
  return (b + g - 1) / g * g;
}

void trim_locked(Cache& c, int device) {
  for (auto& kv : c.free_blocks) {
    if (kv.first.first != device) continue;
    for (auto& fb : kv.second) {
      cudaFree(fb.second);
      c.live.erase(fb.second);
    }
    kv.second.clear();
  }
}

}  // namespace

cudaError_t cache_alloc(void** out, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const size_t want = round_bytes(bytes);
  Cache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  auto& fl = c.free_blocks[{dev, s}];
  auto it = fl.lower_bound(want);
  if (it != fl.end() && it->first <= 2 * want) {   // best fit, at most twice the request
    *out = it->second;
    fl.erase(it);
    return cudaSuccess;
  }
  void* p = nullptr;
  e = cudaMalloc(&p, want);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    trim_locked(c, dev);
    e = cudaMalloc(&p, want);
  }
  if (e != cudaSuccess) return e;
  c.live[p] = {want, dev};
  *out = p;
  return cudaSuccess;
}

void cache_free(void* p, cudaStream_t s) {
  if (!p) return;
  Cache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  auto it = c.live.find(p);
  if (it == c.live.end()) return;
  c.free_blocks[{it->second.device, s}].insert({it->second.bytes, p});
}

// Pinned host blocks (small: Lanczos state mirrors), reused by size.
namespace {
struct HostCache {
  std::mutex mu;
  std::multimap<size_t, void*> free_blocks;
  std::unordered_map<void*, size_t> live;
};
HostCache& host_cache() {
  static HostCache* c = new HostCache();
  return *c;
}
}  // namespace

cudaError_t cache_alloc_host(void** out, size_t bytes) {
  HostCache& c = host_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  auto it = c.free_blocks.lower_bound(bytes);
  if (it != c.free_blocks.end() && it->first <= 2 * bytes + 4096) {
    *out = it->second;
    c.free_blocks.erase(it);
    return cudaSuccess;
  }
  void* p = nullptr;
  cudaError_t e = cudaMallocHost(&p, bytes);
  if (e != cudaSuccess) return e;
  c.live[p] = bytes;
  *out = p;
  return cudaSuccess;
}

void cache_free_host(void* p) {
  if (!p) return;
  HostCache& c = host_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  auto it = c.live.find(p);
  if (it != c.live.end()) c.free_blocks.insert({it->second, p});
}

void cache_trim(int device) {
  Cache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  trim_locked(c, device);
}

}  // namespace mrd
