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
// dda_set_memory_limit() caps the bytes held by live handles: an allocation
// beyond the cap fails as an out-of-memory would (DDA_ERR_OOM at the entry
// point), for services that share a GPU and budget each library's memory.
#include <cstdint>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace dda {
namespace {

constexpr size_t kCacheCap = (size_t)4 << 30;

struct Cached {
  void* p;
  cudaEvent_t ev;   // recorded on the freeing stream (null: nothing pending)
  int dev;
};

struct Live {
  size_t bytes;
  int dev;
};

std::mutex g_mu;
std::unordered_map<void*, Live> g_live;
std::multimap<std::pair<int, size_t>, Cached> g_cache;
size_t g_cached = 0;
size_t g_live_bytes = 0;
size_t g_limit = 0;                 // 0: no limit (dda_set_memory_limit)

// Waits for a block's pending work and returns it to the driver, on the
// block's own device.  Called without g_mu held.
void release_block(const Cached& c) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); cur = -1; }
  if (cur != c.dev) cudaSetDevice(c.dev);
  if (c.ev) {
    cudaEventSynchronize(c.ev);
    cudaEventDestroy(c.ev);
  }
  cudaFree(c.p);
  if (cur >= 0 && cur != c.dev) cudaSetDevice(cur);
  cudaGetLastError();
}

// Caller holds g_mu.  Moves every cached block of device dev (-1: all) to
// out, for release after the lock is dropped.
void take_cached_locked(int dev, std::vector<Cached>& out) {
  for (auto it = g_cache.begin(); it != g_cache.end();) {
    if (dev >= 0 && it->first.first != dev) {
      ++it;
      continue;
    }
    out.push_back(it->second);
    g_cached -= it->first.second;
    it = g_cache.erase(it);
  }
}

void release_all(const std::vector<Cached>& v) {
  for (const Cached& c : v) release_block(c);
}

}  // namespace

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  Cached c{nullptr, nullptr, dev};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    // the caller's limit on the bytes held by live handles
    if (g_limit && g_live_bytes + bytes > g_limit) return cudaErrorMemoryAllocation;
    auto it = g_cache.lower_bound(std::make_pair(dev, bytes));
    if (it != g_cache.end() && it->first.first == dev && it->first.second <= bytes + bytes / 8 &&
        (!g_limit || g_live_bytes + it->first.second <= g_limit)) {
      const size_t sz = it->first.second;
      c = it->second;
      g_cache.erase(it);
      g_cached -= sz;
      g_live[c.p] = Live{sz, dev};
      g_live_bytes += sz;
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
    std::vector<Cached> victims;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      take_cached_locked(dev, victims);
    }
    release_all(victims);
    e = cudaMalloc(p, bytes);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_live[*p] = Live{bytes, dev};
  g_live_bytes += bytes;
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
    g_live_bytes -= b.bytes;
  }
  if (b.bytes > kCacheCap) return cudaFree(p);
  // the event is recorded with the block's own device current (st belongs to
  // that device), then the caller's device is restored
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); cur = -1; }
  if (cur != b.dev) cudaSetDevice(b.dev);
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
    if (cudaEventRecord(ev, st) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(ev);
      ev = nullptr;
      cudaStreamSynchronize(st);
    }
  } else {
    ev = nullptr;
    cudaDeviceSynchronize();
  }
  cudaGetLastError();
  if (cur >= 0 && cur != b.dev) cudaSetDevice(cur);
  std::vector<Cached> victims;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache.emplace(std::make_pair(b.dev, b.bytes), Cached{p, ev, b.dev});
    g_cached += b.bytes;
    // keep at most kCacheCap bytes: evict the largest blocks first, whatever
    // their device (the map is ordered by device, then size)
    while (g_cached > kCacheCap && !g_cache.empty()) {
      auto big = g_cache.begin();
      for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
        if (it->first.second > big->first.second) big = it;
      victims.push_back(big->second);
      g_cached -= big->first.second;
      g_cache.erase(big);
    }
  }
  release_all(victims);
  return cudaSuccess;
}

}  // namespace dda

extern "C" int dda_release_cached_memory(void) {
  std::vector<dda::Cached> victims;
  {
    std::lock_guard<std::mutex> lk(dda::g_mu);
    dda::take_cached_locked(-1, victims);
  }
  dda::release_all(victims);
  cudaGetLastError();
  return DDA_OK;
}

extern "C" int dda_set_memory_limit(unsigned long long bytes) {
  std::vector<dda::Cached> victims;
  {
    std::lock_guard<std::mutex> lk(dda::g_mu);
    dda::g_limit = (size_t)bytes;
    // with a limit in force the cache is given back too, so that the device
    // memory the library holds is the live handles' alone
    if (bytes) dda::take_cached_locked(-1, victims);
  }
  dda::release_all(victims);
  cudaGetLastError();
  return DDA_OK;
}

extern "C" int dda_memory_in_use(unsigned long long* live_bytes, unsigned long long* cached_bytes) {
  if (!live_bytes || !cached_bytes) return DDA_ERR_ARG;
  std::lock_guard<std::mutex> lk(dda::g_mu);
  *live_bytes = dda::g_live_bytes;
  *cached_bytes = dda::g_cached;
  return DDA_OK;
}
