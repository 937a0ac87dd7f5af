// Many particles at once: a pool of host threads, each taking the next
// particle and running its D-matrix build (if missing) and dda_solve_batch on
// the particle's own stream, so that the kernels of different particles
// overlap on the device.  No counterpart in the paper (one particle per run).
#include <atomic>
#include <thread>
#include <vector>

#include "internal.h"

using namespace dda;

extern "C" int dda_build_Dmatrix(dda_t h, int prec);
extern "C" int dda_solve_batch(dda_t h, const dda_solve_opts* o, int nrhs, const double* prop,
                               const double* pol, void* P_dev, dda_solve_info* info);

extern "C" int dda_solve_many(int n_part, dda_t const* hs, const dda_solve_opts* o,
                              const int* nrhs, const double* const* prop, const double* const* pol,
                              void* const* P, dda_solve_info* const* info, int n_threads,
                              int* status_out) {
  if (n_part < 1 || !hs || !o || !nrhs || !prop || !pol || !P || !info || !status_out ||
      n_threads < 1)
    return DDA_ERR_ARG;
  for (int i = 0; i < n_part; ++i)
    if (!hs[i] || nrhs[i] < 1 || !prop[i] || !pol[i] || !P[i] || !info[i]) return DDA_ERR_ARG;
  if (o->checkpoint_every != 0 || o->resume) return DDA_ERR_ARG;   // one buffer cannot hold many solves
  for (int i = 0; i < n_part; ++i)
    for (int j = 0; j < i; ++j)
      if (hs[i] == hs[j]) return DDA_ERR_ARG;          // a handle is not thread-safe
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n_part) break;
      dda_t h = hs[i];
      // the entry points below make the handle's device current themselves
      // and restore this thread's device afterwards
      int rc = DDA_OK;
      const bool need64 = !h->w64.have_D;
      const bool need32 = o->prec == DDA_FP32_REFINED && !h->w32.have_D;
      if (need64 || need32) rc = dda_build_Dmatrix(h, o->prec);
      if (rc == DDA_OK) rc = dda_solve_batch(h, o, nrhs[i], prop[i], pol[i], P[i], info[i]);
      status_out[i] = rc;
    }
  };
  const int nt = n_threads < n_part ? n_threads : n_part;
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int t = 0; t < nt; ++t) {
    try {
      pool.emplace_back(worker);
    } catch (...) {               // no more threads: the started ones share the work
      break;
    }
  }
  if (pool.empty()) worker();     // none could be started: this thread does it all
  for (auto& t : pool) t.join();
  int worst = DDA_OK;
  for (int i = 0; i < n_part; ++i) {
    const int s = status_out[i];
    const int rs = s < 0 ? 100 - s : s, rw = worst < 0 ? 100 - worst : worst;
    if (rs > rw) worst = s;
  }
  return worst;
}
