// Per-kernel CUDA-event timing behind dda_trace / dda_trace_read: an event
// pair is recorded around each traced launch on the launching stream and
// resolved (cudaEventElapsedTime) at the next flush.
#include <atomic>
#include <cstdio>

#include "internal.h"

namespace dda {

static const char* kNames[TR_COUNT] = {
    "p1_xfft_c64", "p2_yfft_c64", "p3_zconv_c64", "p4_yifft_c64", "p5_xifft_c64",
    "p1_xfft_c128", "p2_yfft_c128", "p3_zconv_c128", "p4_yifft_c128", "p5_xifft_c128",
    "dbuild_green", "dbuild_lines", "dbuild_octant", "farfield", "qsums", "p1_xfft_df", "p2_yfft_df", "p3_zconv_df", "p4_yifft_df",
    "p5_xifft_df",
    "qmr_k1", "qmr_k2", "qmr_scalars"};

const char* trace_name(int id) { return (id >= 0 && id < TR_COUNT) ? kNames[id] : "?"; }

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_total() { return g_launches.load(std::memory_order_relaxed); }

static cudaEvent_t take(Tracer* t) {
  if (!t->pool.empty()) {
    cudaEvent_t e = t->pool.back();
    t->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

void tr_begin(Tracer* t, cudaStream_t st) {
  if (!t || !t->on) return;
  t->open = take(t);
  if (t->open) cudaEventRecord(t->open, st);
}

void tr_end(Tracer* t, cudaStream_t st, int id) {
  if (!t || !t->on || !t->open) return;
  cudaEvent_t b = take(t);
  if (!b) return;
  cudaEventRecord(b, st);
  t->pending.push_back({id, t->open, b});
  t->open = nullptr;
}

void tr_flush(Tracer* t) {
  if (!t) return;
  for (auto& r : t->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      t->ms[r.id] += ms;
      t->cnt[r.id] += 1;
    }
    cudaGetLastError();
    t->pool.push_back(r.a);
    t->pool.push_back(r.b);
  }
  t->pending.clear();
}

void tr_reset(Tracer* t) {
  tr_flush(t);
  t->launch_base = launch_total();
  for (int i = 0; i < TR_COUNT; ++i) { t->ms[i] = 0.0; t->cnt[i] = 0; }
}

void tr_destroy(Tracer* t) {
  tr_flush(t);
  for (cudaEvent_t e : t->pool) cudaEventDestroy(e);
  t->pool.clear();
  if (t->open) cudaEventDestroy(t->open);
  t->open = nullptr;
}

}  // namespace dda

using namespace dda;

extern "C" int dda_trace(dda_t h, int enable) {
  DDA_ON_DEVICE(h);
  tr_reset(&h->tracer);
  h->tracer.on = enable != 0;
  return DDA_OK;
}

extern "C" int dda_trace_read(dda_t h, int max_n, char* names, double* ms, long long* count,
                              int* n_out) {
  if (!h || max_n < 0 || (max_n > 0 && (!names || !ms || !count)) || !n_out) return DDA_ERR_ARG;
  DDA_ON_DEVICE(h);
  tr_flush(&h->tracer);
  int k = 0;
  if (max_n > 0) {
    std::snprintf(names, 32, "%s", "all_launches");
    ms[0] = 0.0;
    count[0] = launch_total() - h->tracer.launch_base;
  }
  ++k;
  for (int i = 0; i < TR_COUNT; ++i) {
    if (h->tracer.cnt[i] == 0) continue;
    if (k < max_n) {
      std::snprintf(names + 32 * k, 32, "%s", trace_name(i));
      ms[k] = h->tracer.ms[i];
      count[k] = h->tracer.cnt[i];
    }
    ++k;
  }
  *n_out = k;
  return DDA_OK;
}

// ---------------------------------------------------------------- kernel attributes
#include <map>
#include <mutex>
#include <utility>

namespace dda {

static std::mutex g_attr_mu;
static std::map<std::pair<const void*, int>, size_t> g_smem;
static std::map<std::pair<const void*, int>, bool> g_carve;

cudaError_t ensure_smem(const void* func, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto key = std::make_pair(func, dev);
  auto it = g_smem.find(key);
  if (it != g_smem.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) g_smem[key] = bytes;
  return e;
}

cudaError_t ensure_carveout_max(const void* func) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  auto key = std::make_pair(func, dev);
  if (g_carve.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) g_carve[key] = true;
  return e;
}

}  // namespace dda

namespace dda {

int num_sms() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 1;                       // not cached: asked again next time
  }
  cache[dev] = n;
  return n;
}

}  // namespace dda
