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
#include <cmath>

#include "internal.h"

namespace dda {

__global__ void k_green_fill(c128* __restrict__ grid, int mu, int nu, double kd, int nx, int ny,
                             int nz, int Mx, int My, int Mz) {
  const long long total = (long long)Mx * My * Mz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % Mx);
    const long long q = i / Mx;
    const int iy = (int)(q % My);
    const int iz = (int)(q / My);
    c128 out = mk<double>(0.0, 0.0);
    const bool ux = ix < nx || ix > Mx - nx;
    const bool uy = iy < ny || iy > My - ny;
    const bool uz = iz < nz || iz > Mz - nz;
    if (ux && uy && uz) {
      double d[3];
      d[0] = ix < nx ? (double)ix : (double)(ix - Mx);
      d[1] = iy < ny ? (double)iy : (double)(iy - My);
      d[2] = iz < nz ? (double)iz : (double)(iz - Mz);
      const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 > 0.0) {
        const double rho = sqrt(r2);
        const double kr = kd * rho;
        double s, c;
        sincos(kr, &s, &c);
        const double inv3 = 1.0 / (r2 * rho);
        const c128 pref = mk<double>(c * inv3, s * inv3);
        const c128 a = mk<double>(kr * kr - 1.0, kr);
        const c128 b = mk<double>((kr * kr - 3.0) / r2, 3.0 * kr / r2);
        const double dd = d[mu] * d[nu];
        c128 t = mk<double>(-b.x * dd, -b.y * dd);
        if (mu == nu) t = t + a;
        out = pref * t;
      }
    }
    grid[i] = out;
  }
}

__global__ void k_octant(const c128* __restrict__ grid, c128* __restrict__ D, int Mx, int My,
                         int Mz, double inv) {
  const int hx = Mx / 2 + 1, hy = My / 2 + 1, hz = Mz / 2 + 1;
  const long long total = (long long)hx * hy * hz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int fx = (int)(i % hx);
    const long long q = i / hx;
    const int fy = (int)(q % hy);
    const int fz = (int)(q / hy);
    const c128 v = grid[((long long)fz * My + fy) * Mx + fx];
    D[i] = mk<double>(v.x * inv, v.y * inv);
  }
}

__global__ void k_to32(const c128* __restrict__ a, c64* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = mk<float>((float)a[i].x, (float)a[i].y);
}

static int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace dda

using namespace dda;

int dda_build_D_internal(dda_t h, bool want32) {
  const Geom& g = h->g;
  cudaStream_t st = h->stream;
  const long long full = (long long)g.Mx * g.My * g.Mz;
  const long long oct = g.oct();
  if (!h->w64.D) {
    if (cudaMalloc(&h->w64.D, 6 * oct * sizeof(c128)) != cudaSuccess) {
      h->w64.D = nullptr;
      cudaGetLastError();
      return dda_fail(h, DDA_ERR_OOM, "cannot allocate the FP64 D-matrix octant");
    }
  }
  c128* grid = nullptr;
  if (cudaMalloc(&grid, full * sizeof(c128)) != cudaSuccess) {
    cudaGetLastError();
    return dda_fail(h, DDA_ERR_OOM, "cannot allocate the Green's tensor grid");
  }
  const int comps[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
  const double inv = 1.0 / (double)full;
  const c128* twx = h->w64.tw;
  const c128* twy = twx + g.Mx;
  const c128* twz = twy + g.My;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < 6 && e == cudaSuccess; ++c) {
    tr_begin(g.tr, st);
    k_green_fill<<<grid_for(full), 256, 0, st>>>(grid, comps[c][0], comps[c][1], h->kd, g.nx, g.ny,
                                                 g.nz, g.Mx, g.My, g.Mz); count_launch();
    tr_end(g.tr, st, TR_DB_GREEN);
    tr_begin(g.tr, st);
    // x lines (contiguous) over the whole grid; then only the octant is
    // needed, so y lines run for kx <= Mx/2 and z lines for kx <= Mx/2,
    // ky <= My/2 (in place; the other entries are left untransformed).
    const int hx = g.Mx / 2 + 1, hy = g.My / 2 + 1;
    e = launch_lines<double>(g, grid, grid, g.px, twx, false, g.Mx, g.Mx,
                             g.My * g.Mz, 1, 1, true, 1, g.Mx, 0, 0, 1, g.Mx, 0, 0, st);
    if (e != cudaSuccess) break;
    e = launch_lines<double>(g, grid, grid, g.py, twy, false, g.My, g.My, hx, g.Mz, 1, false,
                             g.Mx, 1, (long long)g.My * g.Mx, 0, g.Mx, 1,
                             (long long)g.My * g.Mx, 0, st);
    if (e != cudaSuccess) break;
    e = launch_lines<double>(g, grid, grid, g.pz, twz, false, g.Mz, g.Mz, hx, hy, 1, false,
                             (long long)g.My * g.Mx, 1, g.Mx, 0, (long long)g.My * g.Mx, 1, g.Mx,
                             0, st);
    if (e != cudaSuccess) break;
    tr_end(g.tr, st, TR_DB_LINES);
    tr_begin(g.tr, st);
    k_octant<<<grid_for(oct), 256, 0, st>>>(grid, h->w64.D + c * oct, g.Mx, g.My, g.Mz, inv); count_launch();
    tr_end(g.tr, st, TR_DB_OCTANT);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  tr_flush(g.tr);
  cudaFree(grid);
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "D-matrix build");
  h->w64.have_D = true;
  if (want32) {
    if (!h->w32.D) {
      if (cudaMalloc(&h->w32.D, 6 * oct * sizeof(c64)) != cudaSuccess) {
        h->w32.D = nullptr;
        cudaGetLastError();
        return dda_fail(h, DDA_ERR_OOM, "cannot allocate the FP32 D-matrix octant");
      }
    }
    k_to32<<<grid_for(6 * oct), 256, 0, st>>>(h->w64.D, h->w32.D, 6 * oct); count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return dda_cuda_fail(h, e, "D-matrix FP32 copy");
    h->w32.have_D = true;
  }
  return DDA_OK;
}
