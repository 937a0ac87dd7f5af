// C-ABI entry points: handle, lattice, beta tables, products, queries.
// Equation and section references are to Yurkin, Maltsev & Hoekstra,
// arXiv:0704.0037.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <utility>

#include "internal.h"

using namespace dda;

int dda_fail(dda_t h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int dda_cuda_fail(dda_t h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a non-sticky error so the handle stays usable
  return dda_fail(h, e == cudaErrorMemoryAllocation ? DDA_ERR_OOM : DDA_ERR_CUDA, m);
}

namespace {

// exp(-2 pi i m / M) for m < M, in long double, for the three axes.
// cos and sin of 2 pi m / M, m < M, in long double, computed once per M in
// the process (long double is software-emulated on some hosts, and every new
// handle needs the tables of its three padded lengths)
static const std::vector<std::pair<long double, long double>>& unit_roots(int M) {
  static std::mutex mu;
  static std::map<int, std::vector<std::pair<long double, long double>>> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(M);
  if (it != cache.end()) return it->second;
  std::vector<std::pair<long double, long double>>& v = cache[M];
  const long double twopi = 6.283185307179586476925286766559L;
  v.resize(M);
  for (int m = 0; m < M; ++m) {
    const long double a = twopi * (long double)m / (long double)M;
    v[m] = std::make_pair(cosl(a), sinl(a));
  }
  return v;
}

template <typename R>
std::vector<cpx<R>> twiddles(const Geom& g) {
  std::vector<cpx<R>> t;
  for (int M : {g.Mx, g.My, g.Mz}) {
    const std::vector<std::pair<long double, long double>>& u = unit_roots(M);
    for (int m = 0; m < M; ++m) t.push_back(mk<R>((R)u[m].first, (R)(-u[m].second)));
  }
  return t;
}

template <typename R>
int ensure_work(dda_t h, Work<R>& w, bool buffers = true) {
  const Geom& g = h->g;
  if (!w.tw) {
    std::vector<cpx<R>> t = twiddles<R>(g);
    if (dev_malloc(&w.tw, t.size() * sizeof(cpx<R>)) != cudaSuccess) {
      w.tw = nullptr;
      cudaGetLastError();
      return dda_fail(h, DDA_ERR_OOM, "cannot allocate twiddle tables");
    }
    DDA_CK(h, cudaMemcpy(w.tw, t.data(), t.size() * sizeof(cpx<R>), cudaMemcpyHostToDevice));
  }
  if (!buffers) return DDA_OK;
  if (!w.B1) {
    if (dev_malloc(&w.B1, g.b1() * sizeof(cpx<R>)) != cudaSuccess) {
      w.B1 = nullptr;
      cudaGetLastError();
      return dda_fail(h, DDA_ERR_OOM, "cannot allocate FFT work buffer B1");
    }
  }
  if (!w.B2) {
    if (dev_malloc(&w.B2, g.b2() * sizeof(cpx<R>)) != cudaSuccess) {
      w.B2 = nullptr;
      cudaGetLastError();
      return dda_fail(h, DDA_ERR_OOM, "cannot allocate FFT work buffer B2");
    }
  }
  if (w.cap < 1) w.cap = 1;
  return DDA_OK;
}


template <typename R>
void free_work(Work<R>& w, cudaStream_t st) {
  dev_free(w.B1, st); dev_free(w.B2, st); dev_free(w.tw, st); dev_free(w.D, st); dev_free(w.beta, st);
  w = Work<R>();
}

// ---------------------------------------------------------------- beta (O3)
__device__ c128 csqrt_principal(c128 z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return mk<double>(0.0, 0.0);
  if (z.x >= 0.0) {
    const double t = sqrt(0.5 * (r + z.x));
    return mk<double>(t, z.y / (2.0 * t));
  }
  const double t = sqrt(0.5 * (r - z.x));
  return mk<double>(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

__device__ c128 cdiv(c128 a, c128 b) {
  const double d = b.x * b.x + b.y * b.y;
  return mk<double>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// Polarizability prescriptions of Sec. 2 (formulas of the cited works):
//   1/alpha = 1/alpha_CM + c_corr kd^2 - (2/3) i kd^3   (RR: c_corr = 0),
//   LDR: c_corr = b1 + b2 m^2 + b3 S m^2, S = sum (a_mu e_mu)^2;
//   CLDR: component mu uses b3 m^2 a_mu^2;  CM: 1/alpha = 1/alpha_CM.
// beta = sqrt(alpha) (Eq. (2)), principal branch.
__global__ void k_beta(int nrhs, int n_mat, const double* __restrict__ m, int presc,
                       const double* __restrict__ prop, const double* __restrict__ pol, double kd,
                       c128* __restrict__ b64, c64* __restrict__ b32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrhs * n_mat * 3) return;
  const int mu = i % 3;
  const int k = (i / 3) % n_mat;
  const int r = i / (3 * n_mat);
  const double b1 = -1.8915316, b2 = 0.1648469, b3 = -1.7700004;
  const c128 mm = mk<double>(m[2 * k], m[2 * k + 1]);
  const c128 eps = mm * mm;
  const double pi = 3.141592653589793238462643;
  // alpha_CM = (3/4pi)(eps-1)/(eps+2)  ->  1/alpha_CM = (4pi/3)(eps+2)/(eps-1)
  c128 inv = cdiv(eps + mk<double>(2.0, 0.0), eps - mk<double>(1.0, 0.0));
  inv = mk<double>(inv.x * (4.0 * pi / 3.0), inv.y * (4.0 * pi / 3.0));
  const double k2 = kd * kd, k3 = kd * kd * kd;
  const c128 m2 = eps;
  if (presc != DDA_CM) inv = inv + mk<double>(0.0, -(2.0 / 3.0) * k3);
  if (presc == DDA_LDR) {
    const double* a = prop + 3 * r;
    const double* e = pol + 6 * r;
    c128 S = mk<double>(0.0, 0.0);
    for (int q = 0; q < 3; ++q) {
      const c128 ae = mk<double>(a[q] * e[2 * q], a[q] * e[2 * q + 1]);
      S = S + ae * ae;
    }
    const c128 corr = mk<double>(b1, 0.0) + mk<double>(b2, 0.0) * m2 + mk<double>(b3, 0.0) * S * m2;
    inv = inv + mk<double>(corr.x * k2, corr.y * k2);
  } else if (presc == DDA_CLDR) {
    const double am = prop[3 * r + mu];
    const c128 corr = mk<double>(b1, 0.0) + mk<double>(b2, 0.0) * m2 + mk<double>(b3 * am * am, 0.0) * m2;
    inv = inv + mk<double>(corr.x * k2, corr.y * k2);
  }
  const c128 alpha = cdiv(mk<double>(1.0, 0.0), inv);
  const c128 beta = csqrt_principal(alpha);
  b64[i] = beta;
  b32[i] = mk<float>((float)beta.x, (float)beta.y);
}

bool finite_all(const double* p, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

}  // namespace

namespace dda {

// Several right-hand sides per launch need B1/B2 for each: grow to
// min(want, 64, what a quarter of the free device memory holds).
template <typename R>
int ensure_work_cap(dda_t h, Work<R>& w, int want) {
  int rc = ensure_work<R>(h, w);
  if (rc != DDA_OK) return rc;
  if (want <= w.cap) return DDA_OK;
  const Geom& g = h->g;
  const size_t per = (size_t)(g.b1() + g.b2()) * sizeof(cpx<R>);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); fr = 0; }
  long long fit = (long long)((fr / 4 + (size_t)w.cap * per) / per);
  int target = want < 64 ? want : 64;
  if (fit < target) target = (int)(fit > 1 ? fit : 1);
  if (target <= w.cap) return DDA_OK;
  cpx<R>* b1 = nullptr;
  cpx<R>* b2 = nullptr;
  if (dev_malloc(&b1, (size_t)target * g.b1() * sizeof(cpx<R>)) != cudaSuccess ||
      dev_malloc(&b2, (size_t)target * g.b2() * sizeof(cpx<R>)) != cudaSuccess) {
    cudaGetLastError();
    dev_free(b1, h->stream);
    return DDA_OK;            // keep the current capacity: the product runs in more chunks
  }
  dev_free(w.B1, h->stream);
  dev_free(w.B2, h->stream);
  w.B1 = b1;
  w.B2 = b2;
  w.cap = target;
  return DDA_OK;
}
template int ensure_work_cap<float>(dda_t, Work<float>&, int);
template int ensure_work_cap<double>(dda_t, Work<double>&, int);
template int ensure_work_cap<df>(dda_t, Work<df>&, int);

}  // namespace dda

int dda_beta_internal(dda_t h, int presc, int nrhs, const double* prop, const double* pol) {
  if (presc < DDA_CM || presc > DDA_CLDR) return dda_fail(h, DDA_ERR_ARG, "unknown polarizability prescription");
  if (nrhs < 1) return dda_fail(h, DDA_ERR_ARG, "nrhs must be >= 1");
  if (!prop || !pol) return dda_fail(h, DDA_ERR_ARG, "prop and pol must not be NULL");
  if (!finite_all(prop, 3 * nrhs) || !finite_all(pol, 6 * nrhs))
    return dda_fail(h, DDA_ERR_ARG, "non-finite propagation or polarisation vector");
  const int nb = nrhs * h->n_mat * 3;
  if (h->beta_cap < nrhs) {
    dev_free(h->w64.beta, h->stream); dev_free(h->w32.beta, h->stream);
    h->w64.beta = nullptr; h->w32.beta = nullptr; h->beta_cap = 0; h->beta_nrhs = 0;
    if (dev_malloc(&h->w64.beta, nb * sizeof(c128)) != cudaSuccess ||
        dev_malloc(&h->w32.beta, nb * sizeof(c64)) != cudaSuccess) {
      cudaGetLastError();
      return dda_fail(h, DDA_ERR_OOM, "cannot allocate beta tables");
    }
  }
  double* dbuf = nullptr;
  const size_t nd = 2 * h->n_mat + 3 * nrhs + 6 * nrhs;
  DDA_CK(h, dev_malloc(&dbuf, nd * sizeof(double)));
  std::vector<double> hb(nd);
  std::memcpy(hb.data(), h->m.data(), 2 * h->n_mat * sizeof(double));
  std::memcpy(hb.data() + 2 * h->n_mat, prop, 3 * nrhs * sizeof(double));
  std::memcpy(hb.data() + 2 * h->n_mat + 3 * nrhs, pol, 6 * nrhs * sizeof(double));
  cudaError_t e = cudaMemcpyAsync(dbuf, hb.data(), nd * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    k_beta<<<(nb + 127) / 128, 128, 0, h->stream>>>(nrhs, h->n_mat, dbuf, presc, dbuf + 2 * h->n_mat,
                                                    dbuf + 2 * h->n_mat + 3 * nrhs, h->kd,
                                                    h->w64.beta, h->w32.beta); count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(dbuf, h->stream);
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "beta build");
  if (nrhs > h->beta_cap) h->beta_cap = nrhs;
  h->beta_nrhs = nrhs;
  h->beta_presc = presc;
  return DDA_OK;
}

// DDA_SYM_* flags of the lattice, examined on first use from the host copy
// of the occupied cells: the rotation by +90 degrees about z maps cell
// (x = i, y = j) to (x = n - 1 - j, y = i); the lattice is invariant when nx
// == ny and every occupied cell maps to an occupied cell of the same
// material (the map is a bijection of the box, so that suffices).
static int lattice_symmetry(dda_t h) {
  if (h->sym_flags >= 0) return h->sym_flags;
  const Geom& g = h->g;
  int flags = 0;
  if (g.nx == g.ny) {
    const int n = g.nx;
    std::vector<uint8_t> cell((size_t)n * n * g.nz, 0);   // material + 1
    for (int r = 0; r < g.nrows; ++r)
      for (long long k = h->row_off_h[r]; k < h->row_off_h[r + 1]; ++k)
        cell[(size_t)r * n + h->xi_h[k]] = (uint8_t)(h->mat_h[k] + 1);
    bool sym = true;
    for (int r = 0; r < g.nrows && sym; ++r) {
      const int j = r % n, iz = r / n;
      for (long long k = h->row_off_h[r]; k < h->row_off_h[r + 1]; ++k) {
        const int i = h->xi_h[k];
        const size_t rot = ((size_t)iz * n + i) * n + (n - 1 - j);
        if (cell[rot] != h->mat_h[k] + 1) { sym = false; break; }
      }
    }
    if (sym) flags |= DDA_SYM_ROT90_Z;
  }
  h->sym_flags = flags;
  return flags;
}

// ---------------------------------------------------------------- C-ABI

extern "C" int dda_init_lattice(dda_t* out, int nx, int ny, int nz, const uint8_t* occ,
                                int n_mat, const double* m, double kd, int volume_corrected,
                                void* cuda_stream) {
  if (!out) return DDA_ERR_ARG;
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || nx > 65535 || ny > 65535 || nz > 65535 || !occ || !m ||
      n_mat < 1 || n_mat > 255 || !(kd > 0.0) || !std::isfinite(kd))
    return DDA_ERR_ARG;
  if (!finite_all(m, 2 * n_mat)) return DDA_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return DDA_ERR_CUDA;
  }
  dda_ctx* h = new (std::nothrow) dda_ctx();
  if (!h) return DDA_ERR_OOM;
  static std::atomic<long long> next_uid{1};
  h->uid = next_uid.fetch_add(1);
  if (cudaGetDevice(&h->device) != cudaSuccess) { cudaGetLastError(); h->device = 0; }
  Geom& g = h->g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.nrows = ny * nz;
  h->row_off_h.assign((size_t)g.nrows + 1, 0);
  // Count the occupied cells of every row, then fill the compact arrays: both
  // passes split over host threads by blocks of rows (a 134^3 box is 2.4 M
  // cells), the row offsets a prefix sum in between.
  {
    const int nrows = g.nrows;
    const unsigned hw = std::thread::hardware_concurrency();
    const long long cells = (long long)nrows * nx;
    const int nt = (int)std::max(1LL, std::min<long long>(hw ? hw : 1, cells / (1LL << 18)));
    std::vector<uint8_t> bad(nt, 0);
    // block t of rows on thread t; blocks whose thread could not be started
    // run on the calling thread (no exception leaves the C-ABI)
    auto run = [&](auto&& body) {
      std::vector<std::thread> th;
      for (int t = 1; t < nt; ++t) {
        try {
          th.emplace_back(body, t);
        } catch (...) {
          break;
        }
      }
      body(0);
      for (int t = 1 + (int)th.size(); t < nt; ++t) body(t);
      for (auto& x : th) x.join();
    };
    auto rows_of = [&](int t, int& r0, int& r1) {
      r0 = (int)((long long)nrows * t / nt);
      r1 = (int)((long long)nrows * (t + 1) / nt);
    };
    run([&](int t) {
      int r0, r1;
      rows_of(t, r0, r1);
      for (int r = r0; r < r1; ++r) {
        const uint8_t* row = occ + (size_t)r * nx;
        long long c = 0;
        uint8_t mx = 0;
        for (int ix = 0; ix < nx; ++ix) {
          c += row[ix] != 0;
          mx = row[ix] > mx ? row[ix] : mx;
        }
        h->row_off_h[r + 1] = c;
        if (mx > n_mat) bad[t] = 1;
      }
    });
    for (int r = 0; r < nrows; ++r) h->row_off_h[r + 1] += h->row_off_h[r];
    const long long cnt = h->row_off_h[nrows];
    bool any_bad = false;
    for (int t = 0; t < nt; ++t) any_bad = any_bad || bad[t];
    if (cnt == 0 || any_bad) { delete h; return DDA_ERR_ARG; }
    h->xi_h.resize((size_t)cnt);
    h->mat_h.resize((size_t)cnt);
    run([&](int t) {
      int r0, r1;
      rows_of(t, r0, r1);
      for (int r = r0; r < r1; ++r) {
        const uint8_t* row = occ + (size_t)r * nx;
        long long k = h->row_off_h[r];
        for (int ix = 0; ix < nx; ++ix) {
          if (row[ix]) {
            h->xi_h[k] = (uint16_t)ix;
            h->mat_h[k] = (uint8_t)(row[ix] - 1);
            ++k;
          }
        }
      }
    });
  }
  g.n_occ = h->row_off_h[g.nrows];
  // per z plane the span of its occupied rows, and the rows of all spans
  std::vector<int> yr_h(2 * (size_t)nz), arow_h;
  std::vector<long long> aoff_h;
  for (int z = 0; z < nz; ++z) {
    int lo = ny, hi = -1;
    for (int y = 0; y < ny; ++y) {
      const size_t r = (size_t)z * ny + y;
      if (h->row_off_h[r + 1] > h->row_off_h[r]) {
        lo = std::min(lo, y);
        hi = y;
      }
    }
    if (hi < 0) { lo = 1; hi = 0; }
    yr_h[2 * z] = lo;
    yr_h[2 * z + 1] = hi;
    for (int y = lo; y <= hi; ++y) {
      arow_h.push_back(z * ny + y);
      aoff_h.push_back(h->row_off_h[(size_t)z * ny + y]);
    }
  }
  aoff_h.push_back(g.n_occ);
  h->nact = (int)arow_h.size();
  const std::vector<uint8_t>& mat = h->mat_h;
  g.Mx = padded_length(2 * nx - 1, DDA_ENGINE_AUTO);
  g.My = padded_length(2 * ny - 1, DDA_ENGINE_AUTO);
  g.Mz = padded_length(2 * nz - 1, DDA_ENGINE_AUTO);
  g.px = make_plan(g.Mx); g.py = make_plan(g.My); g.pz = make_plan(g.Mz);
  g.tr = &h->tracer;
  g.engine = DDA_ENGINE_AUTO;
  h->n_mat = n_mat;
  h->m.assign(m, m + 2 * n_mat);
  // Sec. 3.1 volume correction: N_occ d^3 = (4/3) pi a^3  =>  kd = x (4 pi / (3 N_occ))^(1/3)
  h->kd = volume_corrected ? kd * std::cbrt(4.0 * M_PI / (3.0 * (double)g.n_occ)) : kd;
  h->stream = (cudaStream_t)cuda_stream;
  int rc = DDA_OK;
  if (dev_malloc(&h->d_row_off, h->row_off_h.size() * sizeof(long long)) != cudaSuccess ||
      dev_malloc(&h->d_xi, h->xi_h.size() * sizeof(uint16_t)) != cudaSuccess ||
      dev_malloc(&h->d_mat, mat.size()) != cudaSuccess ||
      dev_malloc(&h->d_arow, arow_h.size() * sizeof(int)) != cudaSuccess ||
      dev_malloc(&h->d_aoff, aoff_h.size() * sizeof(long long)) != cudaSuccess ||
      dev_malloc(&h->d_yr, yr_h.size() * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    rc = DDA_ERR_OOM;
  } else if (cudaMemcpy(h->d_row_off, h->row_off_h.data(), h->row_off_h.size() * sizeof(long long),
                        cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(h->d_xi, h->xi_h.data(), h->xi_h.size() * sizeof(uint16_t),
                        cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(h->d_mat, mat.data(), mat.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(h->d_arow, arow_h.data(), arow_h.size() * sizeof(int),
                        cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(h->d_aoff, aoff_h.data(), aoff_h.size() * sizeof(long long),
                        cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(h->d_yr, yr_h.data(), yr_h.size() * sizeof(int), cudaMemcpyHostToDevice) !=
                 cudaSuccess) {
    cudaGetLastError();
    rc = DDA_ERR_CUDA;
  }
  if (rc != DDA_OK) { dda_free(h); return rc; }
  *out = h;
  return DDA_OK;
}

extern "C" int dda_set_fft_engine(dda_t h, int engine) {
  if (!h) return DDA_ERR_ARG;
  if (engine != DDA_ENGINE_AUTO && engine != DDA_ENGINE_STOCKHAM)
    return dda_fail(h, DDA_ERR_ARG, "unknown FFT engine");
  if (h->w64.have_D || h->w32.have_D || h->wdf.have_D)
    return dda_fail(h, DDA_ERR_STATE, "dda_set_fft_engine must precede dda_build_Dmatrix");
  // the padded lengths follow the engine: compiled lengths for the
  // register-resident passes, the smallest 7-smooth ones for Stockham; work
  // memory sized for the old lengths (a failed build) is released
  auto drop_grid_buffers = [&](auto& w) {
    dev_free(w.B1, h->stream); dev_free(w.B2, h->stream); dev_free(w.tw, h->stream);
    dev_free(w.D, h->stream);
    w.B1 = nullptr; w.B2 = nullptr; w.tw = nullptr; w.D = nullptr; w.cap = 0;
  };
  drop_grid_buffers(h->w64);
  drop_grid_buffers(h->w32);
  drop_grid_buffers(h->wdf);
  dev_free(h->d_dscratch, h->stream);
  h->d_dscratch = nullptr;
  h->dscratch_bytes = 0;
  Geom& g = h->g;
  g.engine = engine;
  g.Mx = padded_length(2 * g.nx - 1, engine);
  g.My = padded_length(2 * g.ny - 1, engine);
  g.Mz = padded_length(2 * g.nz - 1, engine);
  g.px = make_plan(g.Mx); g.py = make_plan(g.My); g.pz = make_plan(g.Mz);
  return DDA_OK;
}

extern "C" int dda_build_Dmatrix(dda_t h, int prec) {
  DDA_ON_DEVICE(h);
  if (prec != DDA_FP64 && prec != DDA_FP32_REFINED) return dda_fail(h, DDA_ERR_ARG, "unknown precision");
  if (h->g.px.nst < 0 || h->g.py.nst < 0 || h->g.pz.nst < 0)
    return dda_fail(h, DDA_ERR_ARG, "padded grid is not 7-smooth");
  // double-float tables when every axis has register-resident passes; the
  // FP32-refined form then needs no complex128 product buffers (they are
  // made on the first FP64 product)
  const Geom& g = h->g;
  const bool dfok = prec == DDA_FP32_REFINED && g.engine == 0 && fast_supported(g.Mx) &&
                    fast_supported(g.My) && fast_supported(g.Mz);
  int rc = ensure_work<double>(h, h->w64, !dfok);
  if (rc != DDA_OK) return rc;
  if (prec == DDA_FP32_REFINED) {
    rc = ensure_work<float>(h, h->w32);
    if (rc != DDA_OK) return rc;
    if (dfok) {
      rc = ensure_work<df>(h, h->wdf);
      if (rc != DDA_OK) return rc;
    }
  }
  rc = dda_build_D_internal(h, prec == DDA_FP32_REFINED);
  if (rc != DDA_OK) return rc;
  // the tile variants of the product's y and z passes, picked by timing
  // (cached per grid shape; entries pinned by dda_set_pass_tiles are kept)
  cudaError_t e;
  if (prec == DDA_FP32_REFINED) {
    e = tune_tiles<float>(h->g, h->lat(), h->w32, h->stream);
    if (e == cudaSuccess && dfok) e = tune_tiles<df>(h->g, h->lat(), h->wdf, h->stream);
  } else {
    e = tune_tiles<double>(h->g, h->lat(), h->w64, h->stream);
  }
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "product pass tile autotuning");
  return DDA_OK;
}

static int tile_kind(int prec) {
  return prec == DDA_FP32_REFINED ? 0 : prec == DDA_FP64 ? 1 : prec == DDA_FP64_PAIR ? 2 : -1;
}

extern "C" int dda_set_pass_tiles(dda_t h, int prec, const int* tiles) {
  if (!h) return DDA_ERR_ARG;
  const int k = tile_kind(prec);
  if (k < 0) return dda_fail(h, DDA_ERR_ARG, "unknown precision");
  for (int i = 0; i < 3; ++i) {
    const int v = tiles ? tiles[i] : -1;
    if (v < -1 || v > 1) return dda_fail(h, DDA_ERR_ARG, "tile variant must be -1, 0 or 1");
  }
  for (int i = 0; i < 3; ++i) h->g.tiles[k][i] = tiles ? tiles[i] : -1;
  return DDA_OK;
}

extern "C" int dda_get_pass_tiles(dda_t h, int prec, int* tiles) {
  if (!h || !tiles) return DDA_ERR_ARG;
  const int k = tile_kind(prec);
  if (k < 0) return dda_fail(h, DDA_ERR_ARG, "unknown precision");
  for (int i = 0; i < 3; ++i) tiles[i] = h->g.tiles[k][i];
  return DDA_OK;
}

extern "C" int dda_set_beta(dda_t h, int presc, int nrhs, const double* prop, const double* pol) {
  DDA_ON_DEVICE(h);
  return dda_beta_internal(h, presc, nrhs, prop, pol);
}

static int matvec_common(dda_t h, int prec, const void* x, void* y, int nrhs, bool adjoint) {
  DDA_ON_DEVICE(h);
  if (!x || !y) return dda_fail(h, DDA_ERR_ARG, "x and y must not be NULL");
  if (x == y) return dda_fail(h, DDA_ERR_ARG, "x and y must not alias");
  if (nrhs < 1) return dda_fail(h, DDA_ERR_ARG, "nrhs must be >= 1");
  if (nrhs > h->beta_nrhs) return dda_fail(h, DDA_ERR_STATE, "beta not set for that many RHS (dda_set_beta)");
  cudaError_t e;
  if (prec == DDA_FP64) {
    if (!h->w64.have_D) return dda_fail(h, DDA_ERR_STATE, "FP64 D-matrix not built");
    int rc = ensure_d64(h);
    if (rc != DDA_OK) return rc;
    rc = ensure_work_cap<double>(h, h->w64, nrhs);
    if (rc != DDA_OK) return rc;
    e = launch_matvec<double>(h->g, h->lat(), h->w64, h->w64.beta, h->n_mat, (const c128*)x,
                              (c128*)y, nrhs, adjoint, h->stream);
  } else if (prec == DDA_FP32_REFINED) {
    if (!h->w32.have_D) return dda_fail(h, DDA_ERR_STATE, "FP32 D-matrix not built");
    const int rc = ensure_work_cap<float>(h, h->w32, nrhs);
    if (rc != DDA_OK) return rc;
    e = launch_matvec<float>(h->g, h->lat(), h->w32, h->w32.beta, h->n_mat, (const c64*)x,
                             (c64*)y, nrhs, adjoint, h->stream);
  } else if (prec == DDA_FP64_PAIR) {
    if (adjoint) return dda_fail(h, DDA_ERR_ARG, "no adjoint in double-float");
    if (!h->wdf.have_D)
      return dda_fail(h, DDA_ERR_STATE, "double-float D-matrix not built (FP32_REFINED build "
                                        "on a grid with register-resident passes)");
    const int rc = ensure_work_cap<df>(h, h->wdf, nrhs);
    if (rc != DDA_OK) return rc;
    e = launch_matvec_df(h->g, h->lat(), h->wdf, h->w64.beta, h->n_mat, (const c128*)x, (c128*)y,
                         nrhs, h->stream);
  } else {
    return dda_fail(h, DDA_ERR_ARG, "unknown precision");
  }
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "matvec launch");
  return DDA_OK;
}

extern "C" int dda_matvec(dda_t h, int prec, const void* x, void* y, int nrhs) {
  return matvec_common(h, prec, x, y, nrhs, false);
}

extern "C" int dda_matvec_adjoint(dda_t h, int prec, const void* x, void* y, int nrhs) {
  return matvec_common(h, prec, x, y, nrhs, true);
}

// checkpoint options: a host buffer large enough, and only where the
// batched QMR-CS driver runs
static int check_ckpt_opts(dda_t h, const dda_solve_opts* o, int nrhs, bool batched) {
  if (o->checkpoint_every < 0) return dda_fail(h, DDA_ERR_ARG, "checkpoint_every must be >= 0");
  if (o->checkpoint_every == 0 && !o->resume) return DDA_OK;
  if (!batched)
    return dda_fail(h, DDA_ERR_ARG, "checkpoints are taken by QMR-CS without a residual history");
  if (!o->checkpoint_host ||
      o->checkpoint_bytes < dda_checkpoint_bytes_internal(h, o->prec, nrhs))
    return dda_fail(h, DDA_ERR_ARG, "checkpoint buffer missing or smaller than dda_checkpoint_bytes");
  return DDA_OK;
}

extern "C" int dda_checkpoint_bytes(dda_t h, int prec, int nrhs, long long* bytes) {
  if (!h) return DDA_ERR_ARG;
  if (!bytes || nrhs < 1 || (prec != DDA_FP64 && prec != DDA_FP32_REFINED))
    return dda_fail(h, DDA_ERR_ARG, "bad dda_checkpoint_bytes arguments");
  *bytes = dda_checkpoint_bytes_internal(h, prec, nrhs);
  return DDA_OK;
}

extern "C" int dda_solve(dda_t h, const dda_solve_opts* o, int nrhs, const double* prop,
                         const double* pol, void* P_dev, double* hist, int hist_len,
                         dda_solve_info* info) {
  DDA_ON_DEVICE(h);
  if (!o || !prop || !pol || !P_dev || !info || nrhs < 1 || (hist && hist_len < 1))
    return dda_fail(h, DDA_ERR_ARG, "bad dda_solve arguments");
  if (o->solver < DDA_QMR_CS || o->solver > DDA_CGNR) return dda_fail(h, DDA_ERR_ARG, "unknown solver");
  if (o->prec != DDA_FP64 && o->prec != DDA_FP32_REFINED) return dda_fail(h, DDA_ERR_ARG, "unknown precision");
  if (!(o->tol > 0.0) || o->maxiter < 1) return dda_fail(h, DDA_ERR_ARG, "tol must be > 0 and maxiter >= 1");
  if (o->prec == DDA_FP32_REFINED && !(o->inner_tol > 0.0 && o->inner_tol < 1.0))
    return dda_fail(h, DDA_ERR_ARG, "inner_tol must be in (0, 1)");
  if (!h->w64.have_D) return dda_fail(h, DDA_ERR_STATE, "FP64 D-matrix not built");
  if (o->prec == DDA_FP32_REFINED && !h->w32.have_D)
    return dda_fail(h, DDA_ERR_STATE, "FP32 D-matrix not built");
  // QMR-CS without a residual history runs on the batched driver (same
  // arithmetic; the host reads the scalars every 8 steps instead of every
  // step, and converged right-hand sides skip their products)
  const bool batched = o->solver == DDA_QMR_CS && !hist;
  const int rc = check_ckpt_opts(h, o, nrhs, batched);
  if (rc != DDA_OK) return rc;
  if (batched) return dda_solve_batch_internal(h, o, nrhs, prop, pol, P_dev, info);
  return dda_solve_internal(h, o, nrhs, prop, pol, P_dev, hist, hist_len, info);
}

extern "C" int dda_solve_batch(dda_t h, const dda_solve_opts* o, int nrhs, const double* prop,
                               const double* pol, void* P_dev, dda_solve_info* info) {
  DDA_ON_DEVICE(h);
  if (!o || !prop || !pol || !P_dev || !info || nrhs < 1)
    return dda_fail(h, DDA_ERR_ARG, "bad dda_solve_batch arguments");
  if (o->solver != DDA_QMR_CS) return dda_fail(h, DDA_ERR_ARG, "dda_solve_batch runs QMR-CS only");
  if (o->prec != DDA_FP64 && o->prec != DDA_FP32_REFINED) return dda_fail(h, DDA_ERR_ARG, "unknown precision");
  if (!(o->tol > 0.0) || o->maxiter < 1) return dda_fail(h, DDA_ERR_ARG, "tol must be > 0 and maxiter >= 1");
  if (o->prec == DDA_FP32_REFINED && !(o->inner_tol > 0.0 && o->inner_tol < 1.0))
    return dda_fail(h, DDA_ERR_ARG, "inner_tol must be in (0, 1)");
  if (!h->w64.have_D) return dda_fail(h, DDA_ERR_STATE, "FP64 D-matrix not built");
  if (o->prec == DDA_FP32_REFINED && !h->w32.have_D)
    return dda_fail(h, DDA_ERR_STATE, "FP32 D-matrix not built");
  const int rc = check_ckpt_opts(h, o, nrhs, true);
  if (rc != DDA_OK) return rc;
  return dda_solve_batch_internal(h, o, nrhs, prop, pol, P_dev, info);
}

extern "C" int dda_residual(dda_t h, int presc, int nrhs, const double* prop, const double* pol,
                            const void* P_dev, double* res) {
  DDA_ON_DEVICE(h);
  if (!prop || !pol || !P_dev || !res || nrhs < 1)
    return dda_fail(h, DDA_ERR_ARG, "bad dda_residual arguments");
  if (presc < DDA_CM || presc > DDA_CLDR) return dda_fail(h, DDA_ERR_ARG, "unknown polarizability prescription");
  if (!h->w64.have_D) return dda_fail(h, DDA_ERR_STATE, "D-matrix not built");
  const int rc = dda_residual_internal(h, presc, nrhs, prop, pol, P_dev, res);
  if (rc == DDA_OK) DDA_CK(h, cudaStreamSynchronize(h->stream));
  return rc;
}

extern "C" int dda_scatter(dda_t h, int presc, const void* P_dev, int nrhs, const double* prop,
                           const double* pol, int n_dir, const double* dirs, const double* w,
                           double* F_out, double* q_out) {
  DDA_ON_DEVICE(h);
  if (!P_dev || nrhs < 1 || !prop || !pol || n_dir < 0 || (n_dir > 0 && (!dirs || !F_out)) || !q_out)
    return dda_fail(h, DDA_ERR_ARG, "bad dda_scatter arguments");
  if (presc < DDA_CM || presc > DDA_CLDR) return dda_fail(h, DDA_ERR_ARG, "unknown polarizability prescription");
  if (n_dir > 0 && !finite_all(dirs, 3 * n_dir)) return dda_fail(h, DDA_ERR_ARG, "non-finite direction");
  return dda_scatter_internal(h, presc, P_dev, nrhs, prop, pol, n_dir, dirs, w, F_out, q_out);
}

extern "C" int dda_mueller_plane(int n_theta, const double* th, const double* Fx, const double* Fy,
                                 double* s11) {
  if (n_theta < 0 || (n_theta > 0 && (!th || !Fx || !Fy || !s11))) return DDA_ERR_ARG;
  for (int i = 0; i < n_theta; ++i) {
    const double t = th[i] * (M_PI / 180.0);
    const double ct = std::cos(t), st = std::sin(t);
    // theta_hat = (cos t, 0, -sin t), y_hat = (0, 1, 0)
    const double* fx = Fx + 6 * i;
    const double* fy = Fy + 6 * i;
    const double s2r = ct * fx[0] - st * fx[4], s2i = ct * fx[1] - st * fx[5];
    const double s4r = -fx[2], s4i = -fx[3];
    const double s3r = -(ct * fy[0] - st * fy[4]), s3i = -(ct * fy[1] - st * fy[5]);
    const double s1r = fy[2], s1i = fy[3];
    s11[i] = 0.5 * (s1r * s1r + s1i * s1i + s2r * s2r + s2i * s2i + s3r * s3r + s3i * s3i +
                    s4r * s4r + s4i * s4i);
  }
  return DDA_OK;
}

static inline double cabs2h(c128 a) { return a.x * a.x + a.y * a.y; }

// Amplitude matrix in the xz plane from F_x, F_y at n = (sin t, 0, cos t):
// S2 = theta.F_x, S4 = -y.F_x, S3 = -theta.F_y, S1 = y.F_y (theta = (cos t, 0, -sin t))
static void plane_amplitudes(double t_deg, const double* fx, const double* fy, c128 S[4]) {
  const double t = t_deg * (M_PI / 180.0);
  const double ct = std::cos(t), st = std::sin(t);
  S[1] = mk<double>(ct * fx[0] - st * fx[4], ct * fx[1] - st * fx[5]);        // S2
  S[3] = mk<double>(-fx[2], -fx[3]);                                          // S4
  S[2] = mk<double>(-(ct * fy[0] - st * fy[4]), -(ct * fy[1] - st * fy[5]));  // S3
  S[0] = mk<double>(fy[2], fy[3]);                                            // S1
}

// The 16 Mueller elements of the amplitude matrix [[S2, S3], [S4, S1]] acting
// on (E_par, E_perp), Stokes (I, Q, U, V) = (|E_par|^2+|E_perp|^2,
// |E_par|^2-|E_perp|^2, 2 Re(E_par E_perp^*), -2 Im(E_par E_perp^*)):
// with a = S2, b = S3, c = S4, d = S1, expand the Stokes vector of
// (a E_par + b E_perp, c E_par + d E_perp).  S[] = {S1, S2, S3, S4}.
void mueller_from_S(const c128 S[4], double* m) {
  const c128 a = S[1], b = S[2], c = S[3], d = S[0];
  const double A = cabs2h(a), B = cabs2h(b), C = cabs2h(c), D = cabs2h(d);
  const c128 ab = a * conjg(b), cd = c * conjg(d), ac = a * conjg(c), bd = b * conjg(d);
  const c128 ad = a * conjg(d), bc = b * conjg(c);
  m[0] = 0.5 * (A + B + C + D);  m[1] = 0.5 * (A - B + C - D);
  m[2] = ab.x + cd.x;            m[3] = ab.y + cd.y;
  m[4] = 0.5 * (A + B - C - D);  m[5] = 0.5 * (A - B - C + D);
  m[6] = ab.x - cd.x;            m[7] = ab.y - cd.y;
  m[8] = ac.x + bd.x;            m[9] = ac.x - bd.x;
  m[10] = ad.x + bc.x;           m[11] = ad.y - bc.y;
  m[12] = -(ac.y + bd.y);        m[13] = -(ac.y - bd.y);
  m[14] = -(ad.y + bc.y);        m[15] = ad.x - bc.x;
}

extern "C" int dda_mueller_plane_full(int n_theta, const double* th, const double* Fx,
                                      const double* Fy, double* M) {
  if (n_theta < 0 || (n_theta > 0 && (!th || !Fx || !Fy || !M))) return DDA_ERR_ARG;
  for (int i = 0; i < n_theta; ++i) {
    c128 S[4];
    plane_amplitudes(th[i], Fx + 6 * i, Fy + 6 * i, S);
    mueller_from_S(S, M + 16 * i);
  }
  return DDA_OK;
}

extern "C" int dda_asymmetry(int n_dir, const double* dirs, const double* w, const double* F,
                             const double* prop, double* g) {
  if (n_dir < 1 || !dirs || !w || !F || !prop || !g) return DDA_ERR_ARG;
  double s = 0.0, v[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < n_dir; ++k) {
    double f2 = 0.0;
    for (int q = 0; q < 6; ++q) f2 += F[6 * k + q] * F[6 * k + q];
    const double wf = w[k] * f2;
    s += wf;
    for (int q = 0; q < 3; ++q) v[q] += wf * dirs[3 * k + q];
  }
  if (!(s > 0.0) || !std::isfinite(s)) return DDA_ERR_ARG;
  for (int q = 0; q < 3; ++q) g[1 + q] = v[q] / s;
  g[0] = g[1] * prop[0] + g[2] * prop[1] + g[3] * prop[2];
  return DDA_OK;
}

extern "C" int dda_symmetry(dda_t h, int* flags) {
  if (!h || !flags) return DDA_ERR_ARG;
  *flags = lattice_symmetry(h);
  return DDA_OK;
}

extern "C" int dda_mueller_plane_sym(dda_t h, int presc, const void* P_dev, int n_theta,
                                     const double* th, double* M, double* F_out) {
  DDA_ON_DEVICE(h);
  if (!(lattice_symmetry(h) & DDA_SYM_ROT90_Z))
    return dda_fail(h, DDA_ERR_ARG, "lattice is not invariant under the 90 degree rotation about z");
  if (n_theta < 1 || !th || !M || !P_dev) return dda_fail(h, DDA_ERR_ARG, "bad arguments");
  std::vector<double> dirs((size_t)6 * n_theta), F((size_t)12 * n_theta);
  for (int i = 0; i < n_theta; ++i) {
    const double t = th[i] * (M_PI / 180.0);
    double* a = dirs.data() + 3 * i;
    double* b = dirs.data() + 3 * (n_theta + i);
    a[0] = std::sin(t); a[1] = 0.0; a[2] = std::cos(t);      // n
    b[0] = 0.0; b[1] = -std::sin(t); b[2] = std::cos(t);     // R^-1 n
  }
  const double prop[3] = {0.0, 0.0, 1.0};
  const double pol[6] = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double q[3];
  const int rc = dda_scatter_internal(h, presc, P_dev, 1, prop, pol, 2 * n_theta, dirs.data(),
                                      nullptr, F.data(), q);
  if (rc != DDA_OK) return rc;
  std::vector<double> Fy((size_t)6 * n_theta);
  for (int i = 0; i < n_theta; ++i) {
    const double* fr = F.data() + 6 * (n_theta + i);     // F_x at R^-1 n
    double* fy = Fy.data() + 6 * i;                      // R applied: (x, y, z) -> (-y, x, z)
    fy[0] = -fr[2]; fy[1] = -fr[3];
    fy[2] = fr[0];  fy[3] = fr[1];
    fy[4] = fr[4];  fy[5] = fr[5];
  }
  if (F_out) {
    for (int i = 0; i < n_theta; ++i) {
      for (int q2 = 0; q2 < 6; ++q2) {
        F_out[12 * i + q2] = F[6 * i + q2];
        F_out[12 * i + 6 + q2] = Fy[6 * i + q2];
      }
    }
  }
  return dda_mueller_plane_full(n_theta, th, F.data(), Fy.data(), M);
}

extern "C" int dda_n_occ(dda_t h, long long* n) {
  if (!h || !n) return DDA_ERR_ARG;
  *n = h->g.n_occ;
  return DDA_OK;
}

extern "C" int dda_kd(dda_t h, double* kd) {
  if (!h || !kd) return DDA_ERR_ARG;
  *kd = h->kd;
  return DDA_OK;
}

extern "C" int dda_grid(dda_t h, int* g3) {
  if (!h || !g3) return DDA_ERR_ARG;
  g3[0] = h->g.Mx; g3[1] = h->g.My; g3[2] = h->g.Mz;
  return DDA_OK;
}

extern "C" int dda_positions(dda_t h, int* ijk) {
  if (!h || !ijk) return DDA_ERR_ARG;
  for (int r = 0; r < h->g.nrows; ++r) {
    const int iy = r % h->g.ny, iz = r / h->g.ny;
    for (long long i = h->row_off_h[r]; i < h->row_off_h[r + 1]; ++i) {
      ijk[3 * i] = h->xi_h[i];
      ijk[3 * i + 1] = iy;
      ijk[3 * i + 2] = iz;
    }
  }
  return DDA_OK;
}

extern "C" const char* dda_last_error(dda_t h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

extern "C" int dda_free(dda_t h) {
  if (!h) return DDA_OK;
  dda::DeviceGuard dev_guard(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  tr_destroy(&h->tracer);
  free_work(h->w64, h->stream);
  free_work(h->w32, h->stream);
  free_work(h->wdf, h->stream);
  dev_free(h->d_row_off, h->stream); dev_free(h->d_xi, h->stream); dev_free(h->d_mat, h->stream);
  dev_free(h->d_arow, h->stream); dev_free(h->d_aoff, h->stream); dev_free(h->d_yr, h->stream);
  dev_free(h->sv, h->stream); dev_free(h->d_part, h->stream); dev_free(h->d_mvpart, h->stream); dev_free(h->d_scal, h->stream); cudaFreeHost(h->h_scal);
  batch_free(h);
  dev_free(h->d_tab, h->stream); dev_free(h->d_fpart, h->stream); dev_free(h->d_coll, h->stream); dev_free(h->d_dscratch, h->stream);
  dev_free(h->d_ptab, h->stream);
  cudaGetLastError();
  delete h;
  return DDA_OK;
}
