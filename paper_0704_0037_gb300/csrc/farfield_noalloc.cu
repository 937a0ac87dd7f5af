// dda_farfield_noalloc: the far-field amplitude of dda_scatter for callers
// that must not allocate device memory.
//
// dda_scatter allocates its working memory (per-direction phase tables and
// per-chunk partial sums) with cudaMalloc on first use.  Some callers cannot
// let a library do that: code that runs while a CUDA stream is being
// captured into a graph, processes whose device memory is handed out by their
// own allocator or reserved up front, and long-running services that forbid
// allocation after start-up.  This entry point runs the same far-field
// kernels, but keeps their working memory in one fixed array in device
// global memory, kFarfieldScratchBytes long, that is part of the library
// image: every GPU that loads the library holds it until the process exits.
//
// Rules of use:
//  * The handle's device must be the calling thread's current device (the
//    entry point does not switch devices); otherwise DDA_ERR_ARG.
//  * The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before starting any stream capture.
//  * All calls share the one array.  Calls whose kernels overlap on the GPU
//    (different streams, or different handles on the same device) race on
//    it and give wrong results; serialise them.
//  * The array keeps whatever the last call left in it.  Every entry of it
//    that a call reads is written earlier by the same call, so nothing needs
//    clearing between calls.
//  * A problem whose working memory exceeds the limit is rejected with
//    DDA_ERR_ARG before anything is launched.
#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr size_t kFarfieldScratchBytes = 8u << 20;   // 8 MiB

static __device__ __align__(256) unsigned char g_farfield_scratch[kFarfieldScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_farfield_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

using namespace dda;

extern "C" int dda_farfield_noalloc(dda_t h, const void* P_dev, int n_dir, const double* dirs_dev,
                                    void* F_dev) {
  if (!h) return DDA_ERR_ARG;
  if (!P_dev || !dirs_dev || !F_dev || n_dir < 1)
    return dda_fail(h, DDA_ERR_ARG, "dda_farfield_noalloc: NULL buffer or n_dir < 1");
  // The scratch address and the kernels belong to the current device, which
  // this entry point does not change (a stream capture in progress on the
  // caller's thread is left alone): it must be the handle's.
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return dda_fail(h, DDA_ERR_CUDA, "dda_farfield_noalloc: cudaGetDevice failed");
  }
  if (cur != h->device)
    return dda_fail(h, DDA_ERR_ARG,
                    "dda_farfield_noalloc: the handle's device (" + std::to_string(h->device) +
                        ") is not the current device (" + std::to_string(cur) + ")");
  const Geom& g = h->g;
  const int L = g.nx + g.ny + g.nz;
  const int dblocks = (n_dir + kFarfieldDB - 1) / kFarfieldDB;
  int n_chunks = std::max(1, std::min((4 * num_sms() + dblocks - 1) / dblocks, (g.nrows + 31) / 32));
  const int rows_per_chunk = (g.nrows + n_chunks - 1) / n_chunks;
  n_chunks = (g.nrows + rows_per_chunk - 1) / rows_per_chunk;
  const size_t tab_bytes = ((size_t)n_dir * L * sizeof(c128) + 255) / 256 * 256;
  const size_t part_bytes = (size_t)n_chunks * n_dir * 6 * sizeof(double);
  if (tab_bytes + part_bytes > kFarfieldScratchBytes)
    return dda_fail(h, DDA_ERR_ARG,
                    "dda_farfield_noalloc: needs " + std::to_string(tab_bytes + part_bytes) +
                        " bytes of working memory, above its fixed limit of " +
                        std::to_string(kFarfieldScratchBytes) + " bytes (use fewer directions)");
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "dda_farfield_noalloc: scratch address");
  c128* tab = (c128*)base;
  double* part = (double*)((unsigned char*)base + tab_bytes);
  cudaStream_t st = h->stream;
  const long long tt = (long long)n_dir * L;
  k_phase_tab<<<(int)std::min<long long>((tt + 255) / 256, 4096), 256, 0, st>>>(
      dirs_dev, n_dir, h->kd, g.nx, g.ny, g.nz, tab);
  count_launch();
  dim3 grid(dblocks, n_chunks);
  k_farfield<<<grid, 256, 0, st>>>((const c128*)P_dev, h->lat(), tab, n_dir, g.nx, g.ny, g.nz,
                                   g.nrows, g.n_occ, rows_per_chunk, part);
  count_launch();
  k_farfield_fin<<<(n_dir + 127) / 128, 128, 0, st>>>(part, n_chunks, n_dir, dirs_dev, h->kd,
                                                      (double*)F_dev);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "dda_farfield_noalloc: launch");
  return DDA_OK;
}
