// Device memory of the library: a per-process cache of freed blocks.
//
// A handle owns a few large buffers (FFT work grids, D-matrix octants,
// Krylov vectors, the D-matrix build scratch) whose sizes depend only on the
// lattice.  Workloads that make one handle per particle (a batch, or a user
// who builds, solves and frees per call) would otherwise pay a cudaMalloc and
// a device-synchronising cudaFree for each of them every time.  Freed blocks
// go to a cache keyed by (device, size) instead, each with an event recorded
// on the stream that last used it; an allocation of (nearly) the same size on
// the same device takes a cached block after that event has completed.  At
// most kCacheCap bytes stay cached (larger blocks are released at once);
// when cudaMalloc runs out of memory the cache of that device is released and
// the allocation retried.  dda_release_cached_memory() releases it on demand.
#include <cstdint>
#include <map>
#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace dda {
namespace {

constexpr size_t kCacheCap = (size_t)4 << 30;

struct Cached {
  void* p;
  cudaEvent_t ev;   // recorded on the freeing stream (null: nothing pending)
};

struct Live {
  size_t bytes;
  int dev;
};

std::mutex g_mu;
std::unordered_map<void*, Live> g_live;
std::multimap<std::pair<int, size_t>, Cached> g_cache;
size_t g_cached = 0;

void release_block(const Cached& c) {
  if (c.ev) {
    cudaEventSynchronize(c.ev);
    cudaEventDestroy(c.ev);
  }
  cudaFree(c.p);
}

// Caller holds g_mu.  Releases every cached block of device dev (-1: all).
void release_locked(int dev) {
  for (auto it = g_cache.begin(); it != g_cache.end();) {
    if (dev >= 0 && it->first.first != dev) {
      ++it;
      continue;
    }
    release_block(it->second);
    g_cached -= it->first.second;
    it = g_cache.erase(it);
  }
}

}  // namespace

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  Cached c{nullptr, nullptr};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.lower_bound(std::make_pair(dev, bytes));
    if (it != g_cache.end() && it->first.first == dev && it->first.second <= bytes + bytes / 8) {
      const size_t sz = it->first.second;
      c = it->second;
      g_cache.erase(it);
      g_cached -= sz;
      g_live[c.p] = Live{sz, dev};
    }
  }
  if (c.p) {
    // the block is this caller's now; wait (outside the lock) until the
    // stream that freed it is done with it
    if (c.ev) {
      cudaEventSynchronize(c.ev);
      cudaEventDestroy(c.ev);
    }
    *p = c.p;
    return cudaSuccess;
  }
  e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    {
      std::lock_guard<std::mutex> lk(g_mu);
      release_locked(dev);
    }
    e = cudaMalloc(p, bytes);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_live[*p] = Live{bytes, dev};
  return cudaSuccess;
}

cudaError_t dev_free(void* p, cudaStream_t st) {
  if (!p) return cudaSuccess;
  Live b{};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_live.find(p);
    if (it == g_live.end()) return cudaFree(p);   // not ours: plain release
    b = it->second;
    g_live.erase(it);
  }
  if (b.bytes > kCacheCap) return cudaFree(p);
  int cur = 0;
  cudaGetDevice(&cur);
  cudaEvent_t ev = nullptr;
  if (cur == b.dev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
    if (cudaEventRecord(ev, st) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(ev);
      ev = nullptr;
      cudaStreamSynchronize(st);
      cudaGetLastError();
    }
  } else {
    cudaGetLastError();
    ev = nullptr;
    cudaDeviceSynchronize();
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.emplace(std::make_pair(b.dev, b.bytes), Cached{p, ev});
  g_cached += b.bytes;
  // keep at most kCacheCap bytes: release the largest blocks first
  while (g_cached > kCacheCap && !g_cache.empty()) {
    auto last = std::prev(g_cache.end());
    release_block(last->second);
    g_cached -= last->first.second;
    g_cache.erase(last);
  }
  return cudaSuccess;
}

}  // namespace dda

extern "C" int dda_release_cached_memory(void) {
  std::lock_guard<std::mutex> lk(dda::g_mu);
  dda::release_locked(-1);
  cudaGetLastError();
  return DDA_OK;
}
