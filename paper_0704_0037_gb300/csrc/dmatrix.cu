// D-matrix build: FFT of the Green's tensor on the padded grid (FP64).
//
// G_ij depends only on r_i - r_j, so the interaction sum is a lattice
// convolution (arXiv:0704.0037, Sec. 2, performance paragraph).  On an
// Mx*My*Mz periodic grid with M >= 2n - 1, grid index j along an axis stands
// for the offset j (j < n) or j - M (j > M - n); other indices hold zero.
// G itself (Eq. (1); free-space dyadic Green's tensor, d = 1, kappa = kd):
//   G = exp(i kappa rho)/rho^3 [(kappa^2 rho^2 - 1 + i kappa rho) I
//                               - (kappa^2 rho^2 - 3 + 3 i kappa rho) D D^T / rho^2],
// G(0) = 0.  Each of the 6 components is transformed by three FP64 line-FFT
// passes and only the octant k_mu <= M_mu/2 is kept: component (mu, nu) is
// even or odd along axis a (odd iff exactly one of mu, nu is a), and the DFT
// keeps that parity, which is how Sec. 2's "symmetry of the interaction
// matrix" reduces the memory of its Fourier transform.  1/(Mx My Mz) is folded in.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "internal.h"

namespace dda {

__device__ __forceinline__ c128 store_as(c128 v, c128*) { return v; }
__device__ __forceinline__ cdf store_as(c128 v, cdf*) { return to_cdf(v); }
__device__ __forceinline__ c128 neg_of(c128 v) { return mk<double>(-v.x, -v.y); }
__device__ __forceinline__ cdf neg_of(cdf v) { return mk<df>(-v.x, -v.y); }
// an integer below 2^24, exactly, in either arithmetic
__device__ __forceinline__ double from_int(int v, double*) { return (double)v; }
__device__ __forceinline__ df from_int(int v, df*) { return df((float)v, 0.0f); }

// G depends on the offset d through rho^2 = |d|^2, an integer n, and the
// products d_mu d_nu: G_mu,nu(d) = A(n) delta_mu,nu - B(n) d_mu d_nu with
//   A(n) = exp(i kappa rho)/rho^3 (kappa^2 rho^2 - 1 + i kappa rho),
//   B(n) = exp(i kappa rho)/rho^5 (kappa^2 rho^2 - 3 + 3 i kappa rho).
// ab[2n], ab[2n+1] = A(n), B(n) for 1 <= n <= nmax (FP64, one sincos per n),
// stored in the table's arithmetic.
template <typename T>
__global__ void k_green_radial(T* __restrict__ ab, double kd, int nmax) {
  for (int n = 1 + blockIdx.x * blockDim.x + threadIdx.x; n <= nmax; n += gridDim.x * blockDim.x) {
    const double r2 = (double)n;
    const double rho = sqrt(r2);
    const double kr = kd * rho;
    double sn, cn;
    sincos(kr, &sn, &cn);
    const double inv3 = 1.0 / (r2 * rho);
    const c128 pref = mk<double>(cn * inv3, sn * inv3);
    ab[2 * n] = store_as(pref * mk<double>(kr * kr - 1.0, kr), (T*)nullptr);
    ab[2 * n + 1] = store_as(pref * mk<double>((kr * kr - 3.0) / r2, 3.0 * kr / r2), (T*)nullptr);
  }
}

// G for every non-negative offset (dx, dy, dz) < (nx, ny, nz), all six
// components from A(n), B(n): table[6][nz][ny][nx].  d_mu d_nu is an integer
// below 2^24, exact in either arithmetic.
template <typename R>
__global__ void k_green_table(cpx<R>* __restrict__ table, const cpx<R>* __restrict__ ab, int nx,
                              int ny, int nz) {
  const long long total = (long long)nx * ny * nz;
  const int rows = ny * nz;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {     // a block per (y, z) row
    const int iy = row % ny, iz = row / ny;
    for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
      const long long i = (long long)row * nx + ix;
      const int d[3] = {ix, iy, iz};
      const int n = ix * ix + iy * iy + iz * iz;
      cpx<R> g[6];
      if (n > 0) {
        const cpx<R> A = ab[2 * n], B = ab[2 * n + 1];
        const int mu_of[6] = {0, 0, 0, 1, 1, 2}, nu_of[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const cpx<R> t = scale<R>(B, from_int(d[mu_of[k]] * d[nu_of[k]], (R*)nullptr));
          g[k] = mu_of[k] == nu_of[k] ? A - t : neg_of(t);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) g[k] = mk<R>(from_int(0, (R*)nullptr), from_int(0, (R*)nullptr));
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) table[(long long)k * total + i] = g[k];
    }
  }
}

// Component (mu, nu) of G on the padded grid from the table: grid index j
// stands for offset j (j < n) or j - M (j > M - n), zero otherwise; a
// negative offset along an axis flips the sign iff exactly one of mu, nu is
// that axis (G_mu,nu is odd along it).  A block per (y, z) row of the grid;
// only rows y < ry, z < rz are written (the rows the first pass reads).
template <typename T>
__global__ void k_green_fill(T* __restrict__ grid, const T* __restrict__ table, int mu,
                             int nu, int nx, int ny, int nz, int Mx, int My, int Mz, int ry,
                             int rz) {
  const long long tsz = (long long)nx * ny * nz;
  const int comp = mu == 0 ? nu : (mu == 1 ? 2 + nu : 5);
  const bool oddx = (mu == 0) != (nu == 0), oddy = (mu == 1) != (nu == 1),
             oddz = (mu == 2) != (nu == 2);
  const int rows = ry * rz;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int iy = r % ry, iz = r / ry;
    const long long row = (long long)iz * My + iy;
    const bool uyz = (iy < ny || iy > My - ny) && (iz < nz || iz > Mz - nz);
    const int ay = iy < ny ? iy : My - iy;
    const int az = iz < nz ? iz : Mz - iz;
    const bool flip_yz = ((iy >= ny) && oddy) != ((iz >= nz) && oddz);
    const T* trow = table + comp * tsz + ((long long)az * ny + ay) * nx;
    T* out = grid + row * Mx;
    T zero;
    zero.x = decltype(zero.x)(0.0);
    zero.y = decltype(zero.y)(0.0);
    for (int ix = threadIdx.x; ix < Mx; ix += blockDim.x) {
      T v = zero;
      if (uyz && (ix < nx || ix > Mx - nx)) {
        v = trow[ix < nx ? ix : Mx - ix];
        if (flip_yz != ((ix >= nx) && oddx)) v = neg_of(v);
      }
      out[ix] = v;
    }
  }
}

// octant of the transformed FP64 grid, scaled by inv
// D: component c of the (planar, complex128) octant, the caller passing its
// base D + c * octant size
__global__ void k_octant(const c128* __restrict__ grid, c128* __restrict__ D, int Mx, int My, int Mz,
                         double inv) {
  const int hx = Mx / 2 + 1, hy = My / 2 + 1, hz = Mz / 2 + 1;
  const int rows = hy * hz;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int fy = row % hy, fz = row / hy;
    const c128* src = grid + ((long long)fz * My + fy) * Mx;
    for (int fx = threadIdx.x; fx < hx; fx += blockDim.x) {
      const c128 v = src[fx];
      D[(long long)row * hx + fx] = mk<double>(v.x * inv, v.y * inv);
    }
  }
}

// octant of the transformed double-float grid, scaled by inv (double-float
// arithmetic), and its complex64 rounding (the high words)
__global__ void k_octant_df(const cdf* __restrict__ grid, cdf* __restrict__ Ddf,
                            c64* __restrict__ D32, int Mx, int My, int Mz, df inv) {
  const int hx = Mx / 2 + 1, hy = My / 2 + 1, hz = Mz / 2 + 1;
  const int rows = hy * hz;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int fy = row % hy, fz = row / hy;
    const cdf* src = grid + ((long long)fz * My + fy) * Mx;
    for (int fx = threadIdx.x; fx < hx; fx += blockDim.x) {
      const cdf v = src[fx];
      const cdf sv = mk<df>(v.x * inv, v.y * inv);
      const long long i = (long long)row * hx + fx;
      Ddf[i] = sv;                                   // planar: Ddf = base + c * octant size
      D32[6 * i] = mk<float>(sv.x.hi, sv.y.hi);      // interleaved: D32 = base + c
    }
  }
}

// complex128 from double-float (the FP64 octant derived on demand)
__global__ void k_df_to128(const cdf* __restrict__ a, c128* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = to128(a[i]);
}

// complex64 rounding of the planar complex128 octant a ([6][oct]) into the
// interleaved complex64 octant b ([oct][6])
__global__ void k_to32(const c128* __restrict__ a, c64* __restrict__ b, long long oct) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 6 * oct;
       i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / oct, o = i - c * oct;
    b[6 * o + c] = mk<float>((float)a[i].x, (float)a[i].y);
  }
}

// The remaining components of the octant of a cubic lattice (nx = ny = nz,
// padded to Mx = My = Mz, octant side h) from xx and xy.  G_mn(r) =
// A(|r|) d_mn - B(|r|) r_m r_n is then carried into itself by permuting the
// axes, and the 3D DFT commutes with the permutation:
//   D_yy(kx,ky,kz) = D_xx(ky,kx,kz),  D_zz(kx,ky,kz) = D_xx(kz,ky,kx),
//   D_xz(kx,ky,kz) = D_xy(kx,kz,ky),  D_yz(kx,ky,kz) = D_xy(kz,ky,kx)
// (the parity of each component in each axis permutes the same way).  The
// octant is planar ([6][oct]) or interleaved by point ([oct][6]).
template <typename T, bool INTERLEAVED>
__global__ void k_oct_permute(T* __restrict__ D, int h, long long oct) {
  auto at = [&](int c, long long q) -> T& { return INTERLEAVED ? D[6 * q + c] : D[c * oct + q]; };
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < oct;
       p += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(p % h), ky = (int)((p / h) % h), kz = (int)(p / ((long long)h * h));
    at(3, p) = at(0, ((long long)kz * h + kx) * h + ky);
    at(5, p) = at(0, ((long long)kx * h + ky) * h + kz);
    at(2, p) = at(1, ((long long)ky * h + kz) * h + kx);
    at(4, p) = at(1, ((long long)kx * h + ky) * h + kz);
  }
}

static int rows_grid(int rows) { return std::min(rows, num_sms() * 64); }

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 16LL * num_sms()) b = 16LL * num_sms();
  if (b < 1) b = 1;
  return (int)b;
}

template <typename R> Work<R>& dwork(dda_t h);
template <> Work<double>& dwork<double>(dda_t h) { return h->w64; }
template <> Work<df>& dwork<df>(dda_t h) { return h->wdf; }

// One component (mu, nu) with the register-resident passes in arithmetic R
// (double or double-float): fill, x pass grid -> grid2, y pass grid2 -> grid,
// z pass grid -> grid2, octant.  Component (mu, nu) is even or odd along y and
// z, and transforms along the other axes keep that: line y > My/2 is sy times
// line My - y.  So the x pass runs only on rows y <= My/2, z <= Mz/2, the y
// pass only on planes z <= Mz/2 and reads rows y <= My/2 (mirroring the rest),
// and the z pass reads planes z <= Mz/2; the y and z passes transform only the
// lines the octant keeps (kx <= Mx/2, and ky <= My/2 for z).
template <typename R>
cudaError_t build_component_fast(dda_t h, cpx<R>* grid, cpx<R>* grid2, const cpx<R>* table,
                                 const int comp[2], int c, double inv) {
  const Geom& g = h->g;
  cudaStream_t st = h->stream;
  const long long oct = g.oct();
  const cpx<R>* twx = dwork<R>(h).tw;
  const cpx<R>* twy = twx + g.Mx;
  const cpx<R>* twz = twy + g.My;
  tr_begin(g.tr, st);
  k_green_fill<cpx<R>><<<rows_grid((g.My / 2 + 1) * (g.Mz / 2 + 1)), 256, 0, st>>>(
      grid, table, comp[0], comp[1], g.nx, g.ny, g.nz, g.Mx, g.My, g.Mz, g.My / 2 + 1, g.Mz / 2 + 1);
  count_launch();
  tr_end(g.tr, st, TR_DB_GREEN);
  tr_begin(g.tr, st);
  const int hx = g.Mx / 2 + 1, hy = g.My / 2 + 1, hz = g.Mz / 2 + 1;
  const int mu = comp[0], nu = comp[1];
  const int sy = ((mu == 1) != (nu == 1)) ? -1 : 1;
  const int sz = ((mu == 2) != (nu == 2)) ? -1 : 1;
  FastArgs fa{};
  fa.st = st;
  fa.in = grid; fa.out = grid2; fa.tw = twx;
  fa.nrows = hy * hz; fa.ny = hy; fa.My = g.My;
  cudaError_t e;
  if ((e = fast_pass<R>(g.Mx, FP_XFULL, fa)) != cudaSuccess) return e;
  fa.in = grid2; fa.out = grid; fa.tw = twy; fa.nrows = hx; fa.nz = hz; fa.Mx = g.Mx;
  fa.msign = sy;
  if ((e = fast_pass<R>(g.My, FP_SFULL, fa)) != cudaSuccess) return e;
  // z lines (kx, ky), kx <= Mx/2, ky <= My/2 (the octant's): hx adjacent
  // lines per ky, the ky groups Mx elements apart
  fa.in = grid; fa.out = grid2; fa.tw = twz; fa.nrows = hx; fa.nz = hy;
  fa.Mx = g.My * g.Mx; fa.msign = sz; fa.ostride = g.Mx;
  if ((e = fast_pass<R>(g.Mz, FP_SFULL, fa)) != cudaSuccess) return e;
  tr_end(g.tr, st, TR_DB_LINES);
  tr_begin(g.tr, st);
  const int orows = rows_grid((g.My / 2 + 1) * (g.Mz / 2 + 1));
  if constexpr (std::is_same<R, df>::value) {
    k_octant_df<<<orows, 256, 0, st>>>(grid2, h->wdf.D + c * oct, h->w32.D + c, g.Mx, g.My,
                                       g.Mz, df(inv)); count_launch();
  } else {
    k_octant<<<orows, 256, 0, st>>>(grid2, h->w64.D + c * oct, g.Mx, g.My, g.Mz, inv); count_launch();
  }
  tr_end(g.tr, st, TR_DB_OCTANT);
  return cudaGetLastError();
}

// One component with the shared-memory Stockham passes (FP64, in place).
cudaError_t build_component_generic(dda_t h, c128* grid, const c128* table, const int comp[2],
                                    int c, double inv) {
  const Geom& g = h->g;
  cudaStream_t st = h->stream;
  const long long oct = g.oct();
  const c128* twx = h->w64.tw;
  const c128* twy = twx + g.Mx;
  const c128* twz = twy + g.My;
  tr_begin(g.tr, st);
  k_green_fill<c128><<<rows_grid(g.My * g.Mz), 256, 0, st>>>(grid, table, comp[0], comp[1], g.nx, g.ny,
                                                     g.nz, g.Mx, g.My, g.Mz, g.My, g.Mz); count_launch();
  tr_end(g.tr, st, TR_DB_GREEN);
  tr_begin(g.tr, st);
  // x lines (contiguous) over the whole grid; then only the octant is
  // needed, so y lines run for kx <= Mx/2 and z lines for kx <= Mx/2,
  // ky <= My/2 (the other entries are left untransformed).
  const int hx = g.Mx / 2 + 1, hy = g.My / 2 + 1;
  cudaError_t e = launch_lines<double>(g, grid, grid, g.px, twx, false, g.Mx, g.Mx,
                                       g.My * g.Mz, 1, 1, true, 1, g.Mx, 0, 0, 1, g.Mx, 0, 0, st);
  if (e != cudaSuccess) return e;
  e = launch_lines<double>(g, grid, grid, g.py, twy, false, g.My, g.My, hx, g.Mz, 1, false,
                           g.Mx, 1, (long long)g.My * g.Mx, 0, g.Mx, 1,
                           (long long)g.My * g.Mx, 0, st);
  if (e != cudaSuccess) return e;
  e = launch_lines<double>(g, grid, grid, g.pz, twz, false, g.Mz, g.Mz, hx, hy, 1, false,
                           (long long)g.My * g.Mx, 1, g.Mx, 0, (long long)g.My * g.Mx, 1,
                           g.Mx, 0, st);
  if (e != cudaSuccess) return e;
  tr_end(g.tr, st, TR_DB_LINES);
  tr_begin(g.tr, st);
  k_octant<<<rows_grid((g.My / 2 + 1) * (g.Mz / 2 + 1)), 256, 0, st>>>(grid, h->w64.D + c * oct,
                                                                        g.Mx, g.My, g.Mz, inv); count_launch();
  tr_end(g.tr, st, TR_DB_OCTANT);
  return cudaGetLastError();
}

}  // namespace dda

using namespace dda;

int dda_build_D_internal(dda_t h, bool want32) {
  const Geom& g = h->g;
  cudaStream_t st = h->stream;
  const long long full = (long long)g.Mx * g.My * g.Mz;
  const long long oct = g.oct();
  const long long tsz = (long long)g.nx * g.ny * g.nz;
  const bool fast = g.engine == 0 && fast_supported(g.Mx) && fast_supported(g.My) &&
                    fast_supported(g.Mz);
  // FP32_REFINED builds in double-float when every axis has register-resident
  // passes: the FP64-class D-matrix then costs FP32-pipe arithmetic (the FP64
  // pipe is ~1/58 of it on this part); the double-float octant serves the
  // refinement's residual products, its high words are the complex64 octant,
  // and the complex128 octant is derived only if an FP64 product asks for it
  const bool use_df = want32 && fast && h->wdf.tw != nullptr;
  auto alloc = [&](void** p, size_t bytes, const char* what) -> int {
    if (*p) return DDA_OK;
    if (dev_malloc(p, bytes) != cudaSuccess) {
      *p = nullptr;
      cudaGetLastError();
      return dda_fail(h, DDA_ERR_OOM, what);
    }
    return DDA_OK;
  };
  int rc = DDA_OK;
  if (use_df) {
    rc = alloc((void**)&h->wdf.D, 6 * oct * sizeof(cdf), "cannot allocate the double-float D-matrix octant");
    if (rc == DDA_OK) rc = alloc((void**)&h->w32.D, 6 * oct * sizeof(c64), "cannot allocate the FP32 D-matrix octant");
  } else {
    rc = alloc((void**)&h->w64.D, 6 * oct * sizeof(c128), "cannot allocate the FP64 D-matrix octant");
  }
  if (rc != DDA_OK) return rc;
  // scratch: two padded grids, the offset table and the A, B table; kept in
  // the handle for later builds when it is small (the bench and batch
  // workloads rebuild per particle), allocated per build otherwise
  const int nmax = (g.nx - 1) * (g.nx - 1) + (g.ny - 1) * (g.ny - 1) + (g.nz - 1) * (g.nz - 1);
  const size_t grid_b = (size_t)full * sizeof(c128);
  const size_t table_b = (size_t)6 * tsz * sizeof(c128);
  const size_t ab_b = (size_t)2 * (nmax + 1) * sizeof(c128);
  const size_t need = (fast ? 2 : 1) * grid_b + table_b + ab_b;
  constexpr size_t kKeepScratch = (size_t)2 << 30;
  void* scratch = nullptr;
  if (h->d_dscratch && h->dscratch_bytes >= need) {
    scratch = h->d_dscratch;
  } else {
    dev_free(h->d_dscratch, h->stream);
    h->d_dscratch = nullptr;
    h->dscratch_bytes = 0;
    if (dev_malloc(&scratch, need) != cudaSuccess) {
      cudaGetLastError();
      return dda_fail(h, DDA_ERR_OOM, "cannot allocate the Green's tensor grid");
    }
    if (need <= kKeepScratch) {
      h->d_dscratch = scratch;
      h->dscratch_bytes = need;
    }
  }
  void* grid = scratch;
  void* table = (char*)scratch + grid_b;
  void* ab = (char*)table + table_b;
  void* grid2 = fast ? (char*)ab + ab_b : nullptr;
  auto release = [&]() {
    if (scratch != h->d_dscratch) dev_free(scratch, h->stream);
  };
  tr_begin(g.tr, st);
  const int rgrid = (int)std::max<long long>(1, std::min<long long>((nmax + 255) / 256, 8LL * num_sms()));
  if (use_df) {
    k_green_radial<cdf><<<rgrid, 256, 0, st>>>((cdf*)ab, h->kd, nmax); count_launch();
    k_green_table<df><<<rows_grid(g.ny * g.nz), 128, 0, st>>>((cdf*)table, (const cdf*)ab, g.nx, g.ny, g.nz); count_launch();
  } else {
    k_green_radial<c128><<<rgrid, 256, 0, st>>>((c128*)ab, h->kd, nmax); count_launch();
    k_green_table<double><<<rows_grid(g.ny * g.nz), 128, 0, st>>>((c128*)table, (const c128*)ab, g.nx, g.ny, g.nz); count_launch();
  }
  tr_end(g.tr, st, TR_DB_GREEN);
  const int comps[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
  const double inv = 1.0 / (double)full;
  // a cubic lattice on a cubic grid: xx and xy transformed, the other four
  // components permuted from them
  const bool cubic = g.nx == g.ny && g.ny == g.nz && g.Mx == g.My && g.My == g.Mz;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < (cubic ? 2 : 6) && e == cudaSuccess; ++c) {
    if (use_df) e = build_component_fast<df>(h, (cdf*)grid, (cdf*)grid2, (const cdf*)table, comps[c], c, inv);
    else if (fast) e = build_component_fast<double>(h, (c128*)grid, (c128*)grid2, (const c128*)table, comps[c], c, inv);
    else e = build_component_generic(h, (c128*)grid, (const c128*)table, comps[c], c, inv);
  }
  if (cubic && e == cudaSuccess) {
    tr_begin(g.tr, st);
    const int hh = g.Mx / 2 + 1;
    if (use_df) {
      k_oct_permute<cdf, false><<<grid_for(oct), 256, 0, st>>>(h->wdf.D, hh, oct); count_launch();
      k_oct_permute<c64, true><<<grid_for(oct), 256, 0, st>>>(h->w32.D, hh, oct); count_launch();
    } else {
      k_oct_permute<c128, false><<<grid_for(oct), 256, 0, st>>>(h->w64.D, hh, oct); count_launch();
    }
    e = cudaGetLastError();
    tr_end(g.tr, st, TR_DB_OCTANT);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  tr_flush(g.tr);
  release();
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "D-matrix build");
  h->w64.have_D = true;
  h->d64_from_df = use_df;
  h->wdf.have_D = use_df;
  if (want32) {
    if (!use_df) {
      rc = alloc((void**)&h->w32.D, 6 * oct * sizeof(c64), "cannot allocate the FP32 D-matrix octant");
      if (rc != DDA_OK) return rc;
      k_to32<<<grid_for(6 * oct), 256, 0, st>>>(h->w64.D, h->w32.D, oct); count_launch();
      e = cudaGetLastError();
      if (e != cudaSuccess) return dda_cuda_fail(h, e, "D-matrix FP32 copy");
    }
    h->w32.have_D = true;
  }
  return DDA_OK;
}

// The complex128 octant of a double-float build, made when first needed.
int ensure_d64(dda_t h) {
  if (!h->d64_from_df) return DDA_OK;
  const long long n = 6 * h->g.oct();
  if (!h->w64.D && dev_malloc(&h->w64.D, n * sizeof(c128)) != cudaSuccess) {
    h->w64.D = nullptr;
    cudaGetLastError();
    return dda_fail(h, DDA_ERR_OOM, "cannot allocate the FP64 D-matrix octant");
  }
  k_df_to128<<<grid_for(n), 256, 0, h->stream>>>(h->wdf.D, h->w64.D, n); count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "FP64 D-matrix from double-float");
  h->d64_from_df = false;
  return DDA_OK;
}
