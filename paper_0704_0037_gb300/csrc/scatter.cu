// Scattering quantities from the dipole polarizations (arXiv:0704.0037,
// Sec. 3.1: extinction, and the Mueller matrix in one scattering plane).
// FP64 sums throughout.  Units d = 1, kappa = kd, dimensionless P = beta x:
//   F(n)  = -i kappa^3 (I - n n) sum_j P_j exp(-i kappa n . r_j)
//   Q_ext = (4 kappa^3 / x^2) sum_j Im(E_inc,j^* . P_j)
//   Q_abs = (4 kappa^3 / x^2) sum_j sum_mu [-Im(1/alpha_mu) - (2/3) kappa^3] |P_mu,j|^2
//   Q_sca = (1/(pi x^2)) sum_k w_k |F(n_k)|^2       (caller's quadrature)
// with x = kappa (3 N_occ / (4 pi))^(1/3), the volume-equivalent size parameter.
//
// The phase of dipole j factorises over the lattice axes, so each direction
// gets three 1D tables exp(-i kappa n_mu r_mu) and a row of the lattice
// shares its (y, z) factor.
#include <cmath>

#include "internal.h"

namespace dda {

constexpr int kDB = kFarfieldDB;        // directions per block

__global__ void k_phase_tab(const double* __restrict__ dirs, int n_dir, double kd, int nx, int ny,
                            int nz, c128* __restrict__ tab) {
  const int L = nx + ny + nz;
  const long long total = (long long)n_dir * L;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int d = (int)(i / L);
    int k = (int)(i - (long long)d * L);
    int axis = 0, n = nx;
    if (k >= nx) { k -= nx; axis = 1; n = ny; if (k >= ny) { k -= ny; axis = 2; n = nz; } }
    const double r = 0.5 * (2 * k + 1 - n);
    double s, c;
    sincos(-kd * dirs[3 * d + axis] * r, &s, &c);
    tab[i] = mk<double>(c, s);
  }
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Partial sums S_d = sum_j P_j phase_d(j) over a chunk of rows for kDB
// directions; part[((chunk * n_dir + d) * 3 + c) * 2 + {re,im}].
__global__ void __launch_bounds__(256) k_farfield(const c128* __restrict__ P, LatticeDev lat,
                                                  const c128* __restrict__ tab, int n_dir, int nx,
                                                  int ny, int nz, int nrows, long long n_occ,
                                                  int rows_per_chunk, double* __restrict__ part) {
  const int L = nx + ny + nz;
  const int d0 = blockIdx.x * kDB;
  const int chunk = blockIdx.y;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double acc[kDB][6];
#pragma unroll
  for (int d = 0; d < kDB; ++d)
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[d][q] = 0.0;
  const int rs = chunk * rows_per_chunk;
  const int re = min(nrows, rs + rows_per_chunk);
  for (int row = rs + wid; row < re; row += 8) {
    const int iy = row % ny, iz = row / ny;
    c128 pyz[kDB];
#pragma unroll
    for (int d = 0; d < kDB; ++d) {
      const int dd = min(d0 + d, n_dir - 1);
      pyz[d] = tab[(long long)dd * L + nx + iy] * tab[(long long)dd * L + nx + ny + iz];
    }
    for (long long i = lat.row_off[row] + lane; i < lat.row_off[row + 1]; i += 32) {
      const int ix = lat.xi[i];
      const c128 p0 = P[i], p1 = P[n_occ + i], p2 = P[2 * n_occ + i];
#pragma unroll
      for (int d = 0; d < kDB; ++d) {
        const int dd = min(d0 + d, n_dir - 1);
        const c128 ph = tab[(long long)dd * L + ix] * pyz[d];
        const c128 a = p0 * ph, b = p1 * ph, c = p2 * ph;
        acc[d][0] += a.x; acc[d][1] += a.y;
        acc[d][2] += b.x; acc[d][3] += b.y;
        acc[d][4] += c.x; acc[d][5] += c.y;
      }
    }
  }
  __shared__ double sh[kDB * 6][8];
#pragma unroll
  for (int d = 0; d < kDB; ++d)
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const double s = wsum(acc[d][q]);
      if (lane == 0) sh[d * 6 + q][wid] = s;
    }
  __syncthreads();
  if (threadIdx.x < kDB * 6) {
    const int d = threadIdx.x / 6, q = threadIdx.x % 6;
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[threadIdx.x][w];
    if (d0 + d < n_dir) part[((long long)chunk * n_dir + d0 + d) * 6 + q] = s;
  }
}

// F(n_d) from the chunk partials (fixed order), then the transverse projection
__global__ void k_farfield_fin(const double* __restrict__ part, int n_chunks, int n_dir,
                               const double* __restrict__ dirs, double kd, double* __restrict__ F) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n_dir) return;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int c = 0; c < n_chunks; ++c)
    for (int q = 0; q < 6; ++q) s[q] += part[((long long)c * n_dir + d) * 6 + q];
  const double nx = dirs[3 * d], ny = dirs[3 * d + 1], nz = dirs[3 * d + 2];
  const double dr = nx * s[0] + ny * s[2] + nz * s[4];
  const double di = nx * s[1] + ny * s[3] + nz * s[5];
  const double n3[3] = {nx, ny, nz};
  const double k3 = kd * kd * kd;
  for (int c = 0; c < 3; ++c) {
    const double tr = s[2 * c] - n3[c] * dr;
    const double ti = s[2 * c + 1] - n3[c] * di;
    // -i k3 (tr + i ti) = k3 ti - i k3 tr
    F[6 * d + 2 * c] = k3 * ti;
    F[6 * d + 2 * c + 1] = -k3 * tr;
  }
}

// Directions with n_y = 0 (e.g. the xz scattering plane) see no phase along
// y, so sum_j P_j exp(-i kappa n.r_j) = sum_{x,z} Q(x, z) exp(-i kappa n.r)
// with Q(x, z) = sum_y P(x, y, z).  One block per z: the rows of that z-slab
// are added in y order into a shared [nx][3] accumulator (dipoles of one row
// have distinct x, so the order of every sum is fixed).  Q is laid out as the
// dipole vector of a full nx x 1 x nz lattice: [3][nz*nx].
// Sum of P over y for every (x, z): the far field in a plane with n_y = 0
// needs only that.  Block (z, gy) sums the rows y of group gy (of G) into
// shared memory and writes them as a partial; k_collapse_fin adds the G
// partials in order (deterministic).  part [G][3][nq], Q [3][nq], nq = nx nz.
__global__ void __launch_bounds__(256) k_collapse_y(const c128* __restrict__ P, LatticeDev lat,
                                                    long long n_occ, int nx, int ny,
                                                    c128* __restrict__ part, long long nq) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c128* acc = reinterpret_cast<c128*>(smem_raw);
  const int z = blockIdx.x, gy = blockIdx.y, G = gridDim.y;
  const int y0 = (int)((long long)gy * ny / G), y1 = (int)((long long)(gy + 1) * ny / G);
  for (int i = threadIdx.x; i < 3 * nx; i += blockDim.x) acc[i] = mk<double>(0.0, 0.0);
  __syncthreads();
  for (int y = y0; y < y1; ++y) {
    const int row = z * ny + y;
    for (long long i = lat.row_off[row] + threadIdx.x; i < lat.row_off[row + 1]; i += blockDim.x) {
      const int x = lat.xi[i];
      for (int c = 0; c < 3; ++c) acc[3 * x + c] = acc[3 * x + c] + P[c * n_occ + i];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < 3 * nx; i += blockDim.x) {
    const int x = i / 3, c = i - 3 * x;
    part[((long long)gy * 3 + c) * nq + (long long)z * nx + x] = acc[i];
  }
}

__global__ void k_collapse_fin(const c128* __restrict__ part, int G, long long nq,
                               c128* __restrict__ Q) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * nq;
       i += (long long)gridDim.x * blockDim.x) {
    c128 s = part[i];
    for (int g = 1; g < G; ++g) s = s + part[(long long)g * 3 * nq + i];
    Q[i] = s;
  }
}

struct Wave2 { double a[3]; double e[6]; };

constexpr int kCollapseG = 8;   // y groups of the collapse (partials per (x, z))

// per-row-chunk partials of sum Im(E_inc^* . P) and sum w |P|^2.  ptab holds
// exp(-i kd a_mu r_mu) along x, then y, then z (k_phase_tab for the incidence
// direction a), so exp(-i kd a.r) is a product of three table entries.
__global__ void __launch_bounds__(256) k_qsums(const c128* __restrict__ P, LatticeDev lat,
                                               const c128* __restrict__ beta, int n_mat,
                                               long long n_occ, int nx, int ny, int nrows, double kd,
                                               Wave2 w, const c128* __restrict__ ptab,
                                               double* __restrict__ part) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const double k3 = kd * kd * kd;
  // absorption weight -Im(1/alpha) - (2/3) kd^3 per material and component
  __shared__ double wab[3 * 256];
  for (int i = threadIdx.x; i < 3 * n_mat; i += blockDim.x) {
    const c128 al = beta[i] * beta[i];
    wab[i] = al.y / (al.x * al.x + al.y * al.y) - (2.0 / 3.0) * k3;
  }
  __syncthreads();
  // E = e exp(i phi); E^* . P = conj(e) exp(-i phi) P
  const c128 e0 = mk<double>(w.e[0], -w.e[1]), e1 = mk<double>(w.e[2], -w.e[3]),
             e2 = mk<double>(w.e[4], -w.e[5]);
  double se = 0.0, sa = 0.0;
  for (int row = blockIdx.x * 8 + wid; row < nrows; row += nwarps) {
    const int iy = row % ny, iz = row / ny;
    const c128 pyz = ptab[nx + iy] * ptab[nx + ny + iz];
    for (long long i = lat.row_off[row] + lane; i < lat.row_off[row + 1]; i += 32) {
      const c128 ph = ptab[lat.xi[i]] * pyz;
      const int m = lat.mat[i];
      const c128 p0 = P[i], p1 = P[n_occ + i], p2 = P[2 * n_occ + i];
      const c128 t = (e0 * p0 + e1 * p1 + e2 * p2) * ph;
      se += t.y;
      sa += wab[3 * m] * (p0.x * p0.x + p0.y * p0.y) + wab[3 * m + 1] * (p1.x * p1.x + p1.y * p1.y) +
            wab[3 * m + 2] * (p2.x * p2.x + p2.y * p2.y);
    }
  }
  __shared__ double sh[2][8];
  se = wsum(se); sa = wsum(sa);
  if (lane == 0) { sh[0][wid] = se; sh[1][wid] = sa; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += sh[threadIdx.x][q];
    part[2 * blockIdx.x + threadIdx.x] = s;
  }
}

}  // namespace dda

using namespace dda;

int dda_scatter_internal(dda_t h, int presc, const void* P_dev, int nrhs, const double* prop,
                         const double* pol, int n_dir, const double* dirs, const double* wts,
                         double* F_out, double* q_out) {
  int rc = dda_beta_internal(h, presc, nrhs, prop, pol);
  if (rc != DDA_OK) return rc;
  const Geom& g = h->g;
  cudaStream_t st = h->stream;
  const long long n = 3 * g.n_occ;
  const double xsz = h->kd * std::cbrt(3.0 * (double)g.n_occ / (4.0 * M_PI));
  const double k3 = h->kd * h->kd * h->kd;
  // far-field lattice: the particle's, or its y-collapse when no direction
  // has a y component (the xz scattering plane of Sec. 3.1)
  bool collapse = n_dir > 0 && g.ny > 1 && (size_t)g.nx * 3 * sizeof(c128) <= 96 * 1024;
  for (int d = 0; d < n_dir && collapse; ++d)
    if (dirs[3 * d + 1] != 0.0) collapse = false;
  const int fnx = g.nx, fny = collapse ? 1 : g.ny, fnz = g.nz;
  const int fnrows = collapse ? g.nz : g.nrows;
  const long long fnocc = collapse ? (long long)g.nx * g.nz : g.n_occ;
  LatticeDev flat = h->lat();
  c128* Qc = nullptr;
  c128* Qpart = nullptr;
  if (collapse) {
    const size_t need = (size_t)fnocc * 3 * sizeof(c128) * (1 + kCollapseG) +
                        (size_t)(g.nz + 1) * sizeof(long long) + (size_t)fnocc * sizeof(uint16_t) + 64;
    if (h->coll_bytes < need) {
      dev_free(h->d_coll, h->stream); h->d_coll = nullptr; h->coll_bytes = 0;
      if (dev_malloc(&h->d_coll, need) != cudaSuccess) { cudaGetLastError(); return dda_fail(h, DDA_ERR_OOM, "scatter collapse buffer"); }
      h->coll_bytes = need;
    }
    Qc = (c128*)h->d_coll;
    Qpart = Qc + (size_t)fnocc * 3;
    long long* roff = (long long*)(Qpart + (size_t)fnocc * 3 * kCollapseG);
    uint16_t* xis = (uint16_t*)(roff + g.nz + 1);
    std::vector<long long> ro(g.nz + 1);
    std::vector<uint16_t> xv((size_t)fnocc);
    for (int z = 0; z <= g.nz; ++z) ro[z] = (long long)z * g.nx;
    for (long long i = 0; i < fnocc; ++i) xv[i] = (uint16_t)(i % g.nx);
    DDA_CK(h, cudaMemcpy(roff, ro.data(), ro.size() * sizeof(long long), cudaMemcpyHostToDevice));
    DDA_CK(h, cudaMemcpy(xis, xv.data(), xv.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    flat.row_off = roff;
    flat.xi = xis;
    flat.mat = nullptr;
    flat.arow = nullptr;
    flat.aoff = nullptr;
    flat.yr = nullptr;
    flat.nact = 0;
  }
  const int L = fnx + fny + fnz;
  const int qblocks = (int)std::min<long long>((g.nrows + 7) / 8, 1024);
  int n_chunks = 1, rows_per_chunk = fnrows;
  if (n_dir > 0) {
    const int dblocks = (n_dir + kDB - 1) / kDB;
    n_chunks = std::max(1, std::min((4 * num_sms() + dblocks - 1) / dblocks, (fnrows + 31) / 32));
    rows_per_chunk = (fnrows + n_chunks - 1) / n_chunks;
    n_chunks = (fnrows + rows_per_chunk - 1) / rows_per_chunk;
  }
  const int Lq = g.nx + g.ny + g.nz;   // incidence phase table of the Q sums
  const size_t tab_b = (size_t)std::max(n_dir, 1) * L * sizeof(c128) + (size_t)Lq * sizeof(c128) +
                       (size_t)(std::max(n_dir, 1) + 1) * 3 * sizeof(double);
  const size_t fp_b = std::max((size_t)n_chunks * std::max(n_dir, 1) * 6, (size_t)2 * qblocks) * sizeof(double) +
                      (size_t)std::max(n_dir, 1) * 6 * sizeof(double);
  if (h->tab_bytes < tab_b) {
    dev_free(h->d_tab, h->stream); h->d_tab = nullptr; h->tab_bytes = 0;
    if (dev_malloc(&h->d_tab, tab_b) != cudaSuccess) { cudaGetLastError(); return dda_fail(h, DDA_ERR_OOM, "scatter tables"); }
    h->tab_bytes = tab_b;
  }
  if (h->fpart_bytes < fp_b) {
    dev_free(h->d_fpart, h->stream); h->d_fpart = nullptr; h->fpart_bytes = 0;
    if (dev_malloc(&h->d_fpart, fp_b) != cudaSuccess) { cudaGetLastError(); return dda_fail(h, DDA_ERR_OOM, "scatter partials"); }
    h->fpart_bytes = fp_b;
  }
  c128* tab = (c128*)h->d_tab;
  c128* qtab = tab + (size_t)std::max(n_dir, 1) * L;
  double* d_dirs = (double*)(qtab + Lq);
  double* d_qdir = d_dirs + (size_t)std::max(n_dir, 1) * 3;
  double* part = h->d_fpart;
  double* d_F = part + std::max((size_t)n_chunks * std::max(n_dir, 1) * 6, (size_t)2 * qblocks);
  if (n_dir > 0) {
    DDA_CK(h, cudaMemcpyAsync(d_dirs, dirs, (size_t)n_dir * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    const long long tt = (long long)n_dir * L;
    k_phase_tab<<<(int)std::min<long long>((tt + 255) / 256, 4096), 256, 0, st>>>(d_dirs, n_dir, h->kd, fnx, fny, fnz, tab); count_launch();
    DDA_CK(h, cudaGetLastError());
  }
  std::vector<double> qp(2 * qblocks);
  for (int r = 0; r < nrhs; ++r) {
    const c128* P = (const c128*)P_dev + (size_t)r * n;
    const c128* beta = h->w64.beta + (long long)r * h->n_mat * 3;
    if (n_dir > 0) {
      dim3 grid((n_dir + kDB - 1) / kDB, n_chunks);
      tr_begin(g.tr, st);
      const c128* Pf = P;
      if (collapse) {
        const size_t sm = (size_t)g.nx * 3 * sizeof(c128);
        DDA_CK(h, cudaFuncSetAttribute(k_collapse_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const int G = std::min(g.ny, kCollapseG);
        k_collapse_y<<<dim3(g.nz, G), 256, sm, st>>>(P, h->lat(), g.n_occ, g.nx, g.ny, Qpart, fnocc); count_launch();
        k_collapse_fin<<<(int)std::min<long long>((3 * fnocc + 255) / 256, 2048), 256, 0, st>>>(Qpart, G, fnocc, Qc); count_launch();
        Pf = Qc;
      }
      k_farfield<<<grid, 256, 0, st>>>(Pf, flat, tab, n_dir, fnx, fny, fnz, fnrows, fnocc,
                                       rows_per_chunk, part); count_launch();
      tr_end(g.tr, st, TR_FARFIELD);
      k_farfield_fin<<<(n_dir + 127) / 128, 128, 0, st>>>(part, n_chunks, n_dir, d_dirs, h->kd, d_F); count_launch();
      DDA_CK(h, cudaGetLastError());
      DDA_CK(h, cudaMemcpyAsync(F_out + (size_t)r * n_dir * 6, d_F, (size_t)n_dir * 6 * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
    }
    Wave2 w;
    for (int q = 0; q < 3; ++q) w.a[q] = prop[3 * r + q];
    for (int q = 0; q < 6; ++q) w.e[q] = pol[6 * r + q];
    DDA_CK(h, cudaMemcpyAsync(d_qdir, prop + 3 * r, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    tr_begin(g.tr, st);
    k_phase_tab<<<(Lq + 255) / 256, 256, 0, st>>>(d_qdir, 1, h->kd, g.nx, g.ny, g.nz, qtab); count_launch();
    k_qsums<<<qblocks, 256, 0, st>>>(P, h->lat(), beta, h->n_mat, g.n_occ, g.nx, g.ny, g.nrows, h->kd, w,
                                     qtab, part); count_launch();
    tr_end(g.tr, st, TR_QSUMS);
    DDA_CK(h, cudaGetLastError());
    DDA_CK(h, cudaMemcpyAsync(qp.data(), part, 2 * qblocks * sizeof(double), cudaMemcpyDeviceToHost, st));
    DDA_CK(h, cudaStreamSynchronize(st));
    tr_flush(g.tr);
    double se = 0.0, sa = 0.0;
    for (int b = 0; b < qblocks; ++b) { se += qp[2 * b]; sa += qp[2 * b + 1]; }
    q_out[3 * r] = 4.0 * k3 / (xsz * xsz) * se;
    q_out[3 * r + 1] = 4.0 * k3 / (xsz * xsz) * sa;
    double qs = NAN;
    if (n_dir > 0 && wts) {
      const double* F = F_out + (size_t)r * n_dir * 6;
      qs = 0.0;
      for (int d = 0; d < n_dir; ++d) {
        double f2 = 0.0;
        for (int q = 0; q < 6; ++q) f2 += F[6 * d + q] * F[6 * d + q];
        qs += wts[d] * f2;
      }
      qs /= M_PI * xsz * xsz;
    }
    q_out[3 * r + 2] = qs;
  }
  return DDA_OK;
}
