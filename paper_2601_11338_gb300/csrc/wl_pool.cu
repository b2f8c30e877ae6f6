// Caching allocator for the library's device and pinned host buffers.
//
// Handles are short-lived (a graph is built, solved, destroyed), and each one
// allocates gigabytes of vectors and Krylov basis. cudaMalloc / cudaFree of
// that much memory costs tens of milliseconds per handle (cudaFree also
// synchronises the device), so freed blocks are kept in a per-device cache
// and handed out again to the next request of a fitting size. A request that
// cudaMalloc cannot satisfy first returns every cached block of that device
// to the driver and retries. wl_pool_release() empties the cache.
//
// A block returns to the cache only when no queued work can still touch it:
// callers free after synchronising the stream that used it (handle destroy
// synchronises its stream first; buffer growth inside a call synchronises
// before the old buffer is released).
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <unordered_map>

#include "wl.h"
#include "wl_host.h"

namespace wl {
namespace {

constexpr size_t kSmall = 1u << 20;     // below: 512-byte size classes
constexpr size_t kLargeQ = 2u << 20;    // at or above: 2 MB size classes
constexpr int kMaxDev = 64;

size_t round_size(size_t b) {
  if (b == 0) b = 16;
  if (b < kSmall) return (b + 511) & ~(size_t)511;
  return (b + kLargeQ - 1) / kLargeQ * kLargeQ;
}

struct Cache {
  std::multimap<size_t, void*> free_blocks;
  std::unordered_map<void*, size_t> live;
  size_t cached = 0;
};

std::mutex g_mtx;
Cache g_dev[kMaxDev];
Cache g_host;

int cur_dev() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDev) {
    (void)cudaGetLastError();
    return 0;
  }
  return d;
}

void drop_all(Cache& c, bool host) {
  for (auto& kv : c.free_blocks) {
    if (host)
      cudaFreeHost(kv.second);
    else
      cudaFree(kv.second);
  }
  c.free_blocks.clear();
  c.cached = 0;
}

// a cached block of at least `sz` bytes, at most a quarter larger
void* take(Cache& c, size_t sz) {
  auto it = c.free_blocks.lower_bound(sz);
  if (it == c.free_blocks.end() || it->first > sz + sz / 4) return nullptr;
  void* p = it->second;
  const size_t bsz = it->first;
  c.free_blocks.erase(it);
  c.cached -= bsz;
  c.live[p] = bsz;
  return p;
}

}  // namespace

cudaError_t pool_malloc(void** out, size_t bytes) {
  const size_t sz = round_size(bytes);
  std::lock_guard<std::mutex> lk(g_mtx);
  Cache& c = g_dev[cur_dev()];
  if (void* p = take(c, sz)) {
    *out = p;
    return cudaSuccess;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sz);
  if (e == cudaErrorMemoryAllocation && c.cached > 0) {
    (void)cudaGetLastError();
    drop_all(c, false);
    e = cudaMalloc(&p, sz);
  }
  if (e != cudaSuccess) {
    *out = nullptr;
    return e;
  }
  c.live[p] = sz;
  *out = p;
  return cudaSuccess;
}

void pool_free(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_mtx);
  for (Cache& c : g_dev) {
    auto it = c.live.find(p);
    if (it == c.live.end()) continue;
    c.free_blocks.emplace(it->second, p);
    c.cached += it->second;
    c.live.erase(it);
    return;
  }
  cudaFree(p);  // not from the pool
}

cudaError_t pool_malloc_host(void** out, size_t bytes) {
  const size_t sz = round_size(bytes);
  std::lock_guard<std::mutex> lk(g_mtx);
  if (void* p = take(g_host, sz)) {
    *out = p;
    return cudaSuccess;
  }
  void* p = nullptr;
  cudaError_t e = cudaMallocHost(&p, sz);
  if (e != cudaSuccess) {
    *out = nullptr;
    return e;
  }
  g_host.live[p] = sz;
  *out = p;
  return cudaSuccess;
}

void pool_free_host(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_mtx);
  auto it = g_host.live.find(p);
  if (it == g_host.live.end()) {
    cudaFreeHost(p);
    return;
  }
  g_host.free_blocks.emplace(it->second, p);
  g_host.cached += it->second;
  g_host.live.erase(it);
}

}  // namespace wl

extern "C" {

void wl_pool_release(void) {
  std::lock_guard<std::mutex> lk(wl::g_mtx);
  int dev = 0;
  cudaGetDevice(&dev);
  for (int d = 0; d < wl::kMaxDev; ++d) {
    if (wl::g_dev[d].free_blocks.empty()) continue;
    cudaSetDevice(d);
    wl::drop_all(wl::g_dev[d], false);
  }
  cudaSetDevice(dev);
  wl::drop_all(wl::g_host, true);
}

size_t wl_pool_cached_bytes(void) {
  std::lock_guard<std::mutex> lk(wl::g_mtx);
  size_t t = wl::g_host.cached;
  for (const auto& c : wl::g_dev) t += c.cached;
  return t;
}

}  // extern "C"
