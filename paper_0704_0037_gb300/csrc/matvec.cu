// The FFT interaction-matrix product y = A x of Eq. (2)-(3):
//     y_i = x_i - beta_i sum_j G(r_i - r_j) beta_j x_j ,
// done as a zero-padded circular convolution on an Mx*My*Mz grid
// (M >= 2n - 1), split into 1D transforms with pruning (arXiv:0704.0037,
// Sec. 2: the forward input is mostly zeros and only part of the backward
// output is used; only the real dipoles carry vector data).
//
// Five passes, per right-hand side:
//   P1  x-FFT of the n_y*n_z occupied rows, fused with the gather of x from
//       the compact dipole order and the multiply by beta   -> B1[3][nz][ny][Mx]
//   P2  y-FFT of n_y nonzero inputs, all My outputs          -> B2[3][nz][My][Mx]
//   P3  per (kx, ky): z-FFT of n_z nonzero inputs, 3x3 product with the octant
//       of FFT(G) (parity signs restore the other octants), inverse z-FFT,
//       keep z < n_z; in place in B2
//   P4  inverse y-FFT, keep y < n_y                          -> B1
//   P5  inverse x-FFT, keep the occupied x, y = x - beta u   -> compact y
#include <array>
#include <map>
#include <mutex>

#include "internal.h"

namespace dda {

static __device__ __forceinline__ int ldm_for(int logT, bool contig) {
  return (1 << logT) + (contig ? 1 : 0);
}

template <typename R>
__device__ __forceinline__ void load_tw(cpx<R>* s_tw, const cpx<R>* __restrict__ tw, int M) {
  for (int i = threadIdx.x; i < M; i += blockDim.x) s_tw[i] = tw[i];
}

// ---------------------------------------------------------------- P1
template <typename R, bool CONJ>
__global__ void __launch_bounds__(256) k_p1(const cpx<R>* __restrict__ x, cpx<R>* __restrict__ B1,
                                            LatticeDev lat, const cpx<R>* __restrict__ beta,
                                            long long n_occ, int nrows, FftPlan p,
                                            const cpx<R>* __restrict__ tw, int logT, int bstride,
                                            const int* __restrict__ skip) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = p.M;
  const int T = 1 << logT;
  const int ldm = ldm_for(logT, true);
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* b0 = s_tw + M;
  cpx<R>* b1 = b0 + (size_t)M * ldm;
  const int cc = blockIdx.y, c = cc % 3;     // 3 * (right-hand side) + component
  if (skip && skip[cc / 3]) return;
  beta += (long long)(cc / 3) * bstride;
  const int r0 = blockIdx.x * T;
  load_tw(s_tw, tw, M);
  for (int i = threadIdx.x; i < M * ldm; i += blockDim.x) b0[i] = mk<R>(0, 0);
  __syncthreads();
  const cpx<R>* xc = x + (long long)cc * n_occ;
  for (int t = 0; t < T; ++t) {
    const int row = r0 + t;
    if (row >= nrows) break;
    const long long s = lat.row_off[row], e = lat.row_off[row + 1];
    for (long long i = s + threadIdx.x; i < e; i += blockDim.x) {
      cpx<R> v = xc[i];
      if (CONJ) v = conjg(v);
      b0[(int)lat.xi[i] * ldm + t] = beta[lat.mat[i] * 3 + c] * v;
    }
  }
  __syncthreads();
  cpx<R>* res = stockham<R, false>(b0, b1, ldm, logT, p, s_tw);
  cpx<R>* out = B1 + (long long)cc * nrows * M;
  for (int it = threadIdx.x; it < M * T; it += blockDim.x) {
    const int t = it / M, m = it - t * M;
    const int row = r0 + t;
    if (row < nrows) out[(long long)row * M + m] = res[m * ldm + t];
  }
}

// ---------------------------------------------------------------- P5
template <typename R, bool CONJ>
__global__ void __launch_bounds__(256) k_p5(const cpx<R>* __restrict__ B1, const cpx<R>* __restrict__ x,
                                            cpx<R>* __restrict__ y, LatticeDev lat,
                                            const cpx<R>* __restrict__ beta, long long n_occ,
                                            int nrows, FftPlan p, const cpx<R>* __restrict__ tw,
                                            int logT, int bstride, const int* __restrict__ skip) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = p.M;
  const int T = 1 << logT;
  const int ldm = ldm_for(logT, true);
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* b0 = s_tw + M;
  cpx<R>* b1 = b0 + (size_t)M * ldm;
  const int cc = blockIdx.y, c = cc % 3;
  if (skip && skip[cc / 3]) return;
  beta += (long long)(cc / 3) * bstride;
  const int r0 = blockIdx.x * T;
  load_tw(s_tw, tw, M);
  const cpx<R>* in = B1 + (long long)cc * nrows * M;
  for (int it = threadIdx.x; it < M * T; it += blockDim.x) {
    const int t = it / M, m = it - t * M;
    const int row = r0 + t;
    b0[m * ldm + t] = row < nrows ? in[(long long)row * M + m] : mk<R>(0, 0);
  }
  __syncthreads();
  cpx<R>* res = stockham<R, true>(b0, b1, ldm, logT, p, s_tw);
  const cpx<R>* xc = x + (long long)cc * n_occ;
  cpx<R>* yc = y + (long long)cc * n_occ;
  for (int t = 0; t < T; ++t) {
    const int row = r0 + t;
    if (row >= nrows) break;
    const long long s = lat.row_off[row], e = lat.row_off[row + 1];
    for (long long i = s + threadIdx.x; i < e; i += blockDim.x) {
      cpx<R> v = xc[i];
      if (CONJ) v = conjg(v);
      cpx<R> o = v - beta[lat.mat[i] * 3 + c] * res[(int)lat.xi[i] * ldm + t];
      if (CONJ) o = conjg(o);
      yc[i] = o;
    }
  }
}

// ---------------------------------------------------------------- P2 / P4 and generic lines
struct LineGeom {
  int n_in, n_out, nt;
  int contig;
  long long in_sm, in_st, in_so, in_sb;
  long long out_sm, out_st, out_so, out_sb;
  const int* skip;     // batch b is skipped when skip[b / per] != 0 (null: none)
  int per;
};

// in may equal out (in-place passes of the D-matrix build): every block reads
// all its lines before the barrier and writes the same lines after it.
template <typename R, bool INV>
__global__ void __launch_bounds__(256) k_lines(const cpx<R>* in, cpx<R>* out,
                                               LineGeom lg, FftPlan p, const cpx<R>* __restrict__ tw,
                                               int logT) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = p.M;
  const int T = 1 << logT;
  const int Tm = T - 1;
  const int ldm = ldm_for(logT, lg.contig != 0);
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* b0 = s_tw + M;
  cpx<R>* b1 = b0 + (size_t)M * ldm;
  if (lg.skip && lg.skip[blockIdx.z / lg.per]) return;
  const int t0 = blockIdx.x * T;
  const long long ib = blockIdx.z * lg.in_sb + blockIdx.y * lg.in_so;
  const long long ob = blockIdx.z * lg.out_sb + blockIdx.y * lg.out_so;
  load_tw(s_tw, tw, M);
  const int nload = lg.n_in * T;
  for (int it = threadIdx.x; it < nload; it += blockDim.x) {
    int t, m;
    if (lg.contig) { t = it / lg.n_in; m = it - t * lg.n_in; }
    else { t = it & Tm; m = it >> logT; }
    const int tt = t0 + t;
    b0[m * ldm + t] = tt < lg.nt ? in[ib + (long long)tt * lg.in_st + (long long)m * lg.in_sm]
                                 : mk<R>(0, 0);
  }
  for (int it = nload + threadIdx.x; it < M * T; it += blockDim.x) {
    const int t = it & Tm, m = it >> logT;
    b0[m * ldm + t] = mk<R>(0, 0);
  }
  __syncthreads();
  cpx<R>* res = stockham<R, INV>(b0, b1, ldm, logT, p, s_tw);
  const int nst = lg.n_out * T;
  for (int it = threadIdx.x; it < nst; it += blockDim.x) {
    int t, m;
    if (lg.contig) { t = it / lg.n_out; m = it - t * lg.n_out; }
    else { t = it & Tm; m = it >> logT; }
    const int tt = t0 + t;
    if (tt < lg.nt) out[ob + (long long)tt * lg.out_st + (long long)m * lg.out_sm] = res[m * ldm + t];
  }
}

// ---------------------------------------------------------------- P3
// D octant index and parity sign for frequency k on an axis of length M.
static __device__ __forceinline__ int fold(int k, int M, int& neg) {
  if (2 * k > M) { neg = 1; return M - k; }
  neg = 0;
  return k;
}

template <typename R>
__global__ void __launch_bounds__(256) k_p3(cpx<R>* __restrict__ B2, const cpx<R>* __restrict__ D,
                                            int nz, int Mx, int My, FftPlan p,
                                            const cpx<R>* __restrict__ tw, int logT,
                                            const int* __restrict__ skip) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Mz = p.M;
  if (skip && skip[blockIdx.z]) return;
  B2 += (long long)blockIdx.z * 3 * nz * My * Mx;      // right-hand side blockIdx.z
  const int T = 1 << logT;
  const int Tm = T - 1;
  const int ldm = T;
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* buf[4];
  buf[0] = s_tw + Mz;
  for (int i = 1; i < 4; ++i) buf[i] = buf[i - 1] + (size_t)Mz * ldm;
  const int kx0 = blockIdx.x * T;
  const int ky = blockIdx.y;
  const long long plane = (long long)My * Mx;
  const long long comp = (long long)nz * plane;
  load_tw(s_tw, tw, Mz);
  // load the three components (z < nz), zero the padding
  for (int c = 0; c < 3; ++c) {
    cpx<R>* b = buf[c];
    for (int it = threadIdx.x; it < Mz * T; it += blockDim.x) {
      const int t = it & Tm, z = it >> logT;
      const int kx = kx0 + t;
      b[z * ldm + t] = (z < nz && kx < Mx) ? B2[c * comp + z * plane + (long long)ky * Mx + kx]
                                           : mk<R>(0, 0);
    }
  }
  __syncthreads();
  cpx<R>* cp[3] = {buf[0], buf[1], buf[2]};
  cpx<R>* fr = buf[3];
  for (int c = 0; c < 3; ++c) {
    cpx<R>* res = stockham<R, false>(cp[c], fr, ldm, logT, p, s_tw);
    if (res == fr) { fr = cp[c]; cp[c] = res; }
  }
  // 3x3 symmetric multiply in Fourier space
  const int hx = Mx / 2 + 1, hy = My / 2 + 1, hz = Mz / 2 + 1;
  const long long octs = (long long)hx * hy * hz;
  int ny_;
  const int fy = fold(ky, My, ny_);
  for (int it = threadIdx.x; it < Mz * T; it += blockDim.x) {
    const int t = it & Tm, kz = it >> logT;
    const int kx = kx0 + t;
    if (kx >= Mx) continue;
    int nx_, nz_;
    const int fx = fold(kx, Mx, nx_);
    const int fz = fold(kz, Mz, nz_);
    const long long p = ((long long)fz * hy + fy) * hx + fx;
    // octant entry k of point p: interleaved (complex64) or planar
    const long long o = kOctInterleaved<R> ? 6 * p : p, ks = kOctInterleaved<R> ? 1 : octs;
    cpx<R> dxx = D[o], dxy = D[o + ks], dxz = D[o + 2 * ks];
    cpx<R> dyy = D[o + 3 * ks], dyz = D[o + 4 * ks], dzz = D[o + 5 * ks];
    if (nx_ ^ ny_) dxy = mk<R>(-dxy.x, -dxy.y);
    if (nx_ ^ nz_) dxz = mk<R>(-dxz.x, -dxz.y);
    if (ny_ ^ nz_) dyz = mk<R>(-dyz.x, -dyz.y);
    const int e = kz * ldm + t;
    const cpx<R> vx = cp[0][e], vy = cp[1][e], vz = cp[2][e];
    cp[0][e] = dxx * vx + dxy * vy + dxz * vz;
    cp[1][e] = dxy * vx + dyy * vy + dyz * vz;
    cp[2][e] = dxz * vx + dyz * vy + dzz * vz;
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    cpx<R>* res = stockham<R, true>(cp[c], fr, ldm, logT, p, s_tw);
    if (res == fr) { fr = cp[c]; cp[c] = res; }
  }
  for (int c = 0; c < 3; ++c) {
    const cpx<R>* b = cp[c];
    for (int it = threadIdx.x; it < nz * T; it += blockDim.x) {
      const int t = it & Tm, z = it >> logT;
      const int kx = kx0 + t;
      if (kx < Mx) B2[c * comp + z * plane + (long long)ky * Mx + kx] = b[z * ldm + t];
    }
  }
}

// ---------------------------------------------------------------- host side

static int pick_logT(int M, size_t elem, int nbuf, int extra_col, int logTmax) {
  const size_t budget = 100 * 1024;
  int lt = logTmax;
  while (lt > 0) {
    size_t need = ((size_t)nbuf * M * ((1 << lt) + extra_col) + M) * elem;
    if (need <= budget) break;
    --lt;
  }
  return lt;
}

static size_t smem_bytes(int M, size_t elem, int nbuf, int logT, int extra_col) {
  return ((size_t)nbuf * M * ((1 << logT) + extra_col) + M) * elem;
}

template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
  return ensure_smem((const void*)kernel, bytes);
}

template <typename R>
cudaError_t launch_lines(const Geom& g, const cpx<R>* in, cpx<R>* out, const FftPlan& p,
                         const cpx<R>* tw, bool inverse, int n_in, int n_out, int nt, int n_outer,
                         int n_batch, bool contig, long long in_sm, long long in_st,
                         long long in_so, long long in_sb, long long out_sm, long long out_st,
                         long long out_so, long long out_sb, cudaStream_t st, const int* skip) {
  (void)g;
  const int logTmax = sizeof(R) == 4 ? 4 : 3;
  const int lt = pick_logT(p.M, sizeof(cpx<R>), 2, contig ? 1 : 0, logTmax);
  const size_t sm = smem_bytes(p.M, sizeof(cpx<R>), 2, lt, contig ? 1 : 0);
  LineGeom lg{n_in, n_out, nt, contig ? 1 : 0, in_sm, in_st, in_so, in_sb,
              out_sm, out_st, out_so, out_sb, skip, 3};
  dim3 grid((nt + (1 << lt) - 1) >> lt, n_outer, n_batch);
  cudaError_t e;
  if (inverse) {
    e = allow_smem(k_lines<R, true>, sm);
    if (e != cudaSuccess) return e;
    k_lines<R, true><<<grid, 256, sm, st>>>(in, out, lg, p, tw, lt); count_launch();
  } else {
    e = allow_smem(k_lines<R, false>, sm);
    if (e != cudaSuccess) return e;
    k_lines<R, false><<<grid, 256, sm, st>>>(in, out, lg, p, tw, lt); count_launch();
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_matvec(const Geom& g, const LatticeDev& lat, Work<R>& w, const cpx<R>* beta,
                          int n_mat, const cpx<R>* x, cpx<R>* y, int nrhs, bool adjoint,
                          cudaStream_t st, double* dotp, int* dot_nb, const int* skip) {
  if (dot_nb) *dot_nb = 0;
  const int logTmax = sizeof(R) == 4 ? 4 : 3;
  const size_t el = sizeof(cpx<R>);
  const cpx<R>* twx = w.tw;
  const cpx<R>* twy = w.tw + g.Mx;
  const cpx<R>* twz = w.tw + g.Mx + g.My;
  const int lt1 = pick_logT(g.Mx, el, 2, 1, logTmax);
  const size_t sm1 = smem_bytes(g.Mx, el, 2, lt1, 1);
  const int lt3 = pick_logT(g.Mz, el, 4, 0, logTmax - 1);
  const size_t sm3 = smem_bytes(g.Mz, el, 4, lt3, 0);
  cudaError_t e;
  if ((e = allow_smem(k_p1<R, false>, sm1)) != cudaSuccess) return e;
  if ((e = allow_smem(k_p1<R, true>, sm1)) != cudaSuccess) return e;
  if ((e = allow_smem(k_p5<R, false>, sm1)) != cudaSuccess) return e;
  if ((e = allow_smem(k_p5<R, true>, sm1)) != cudaSuccess) return e;
  if ((e = allow_smem(k_p3<R>, sm3)) != cudaSuccess) return e;
  const long long nv = 3LL * g.n_occ;
  const int bstride = n_mat * 3;
  // per axis: the register-resident passes when the padded length has a
  // compile-time split, the shared-memory Stockham passes otherwise
  auto has_fast = [](int M) { return sizeof(R) == 4 ? fast_supported_c64(M) : fast_supported(M); };
  const bool fx = g.engine == 0 && has_fast(g.Mx);
  const bool fy = g.engine == 0 && has_fast(g.My);
  const bool fz = g.engine == 0 && has_fast(g.Mz);
  // the register-resident x and y passes skip the rows outside the planes'
  // spans of occupied rows when all four are register-resident (the
  // Stockham passes transform every row)
  LatticeDev la = lat;
  if (!(fx && fy)) {
    la.arow = nullptr;
    la.aoff = nullptr;
    la.yr = nullptr;
    la.nact = 0;
  }
  const int dnb = fast_xinv_blocks(la.arow ? la.nact : g.nrows, sizeof(R) == 4, g.Mx);
  if (dotp && dot_nb && fx) *dot_nb = dnb;
  // right-hand sides in chunks of the work buffers' capacity, each chunk in
  // one launch per pass
  const int cap = w.cap > 0 ? w.cap : 1;
  for (int r0 = 0; r0 < nrhs; r0 += cap) {
    const int cnt = nrhs - r0 < cap ? nrhs - r0 : cap;
    const cpx<R>* xr = x + r0 * nv;
    cpx<R>* yr = y + r0 * nv;
    const cpx<R>* br = beta + (long long)r0 * bstride;
    const int* sk = skip ? skip + r0 : nullptr;
    FastArgs fa{};
    fa.lat = la; fa.beta = br; fa.D = w.D; fa.n_occ = g.n_occ; fa.nrows = g.nrows;
    fa.ny = g.ny; fa.nz = g.nz; fa.Mx = g.Mx; fa.My = g.My; fa.adj = adjoint; fa.st = st;
    fa.nrhs = cnt; fa.bstride = bstride; fa.skip = sk;
    fa.pdl = fast_pdl(std::is_same<R, double>::value, g.Mx, g.My, g.Mz, cnt);
    {
      const int* tl = g.tiles[std::is_same<R, float>::value ? 0 : 1];
      fa.var_yf = tl[0] > 0 ? tl[0] : 0; fa.var_z = tl[1] > 0 ? tl[1] : 0; fa.var_yi = tl[2] > 0 ? tl[2] : 0;
    }
    dim3 g1((g.nrows + (1 << lt1) - 1) >> lt1, 3 * cnt);
    const int tb = sizeof(R) == 4 ? TR_P1_C64 : TR_P1_C128;
    // P1: x lines of the occupied rows, gather and beta -> B1 [rhs][3][nz][ny][Mx]
    tr_begin(g.tr, st);
    if (fx) {
      fa.in = xr; fa.out = w.B1; fa.tw = twx;
      if ((e = fast_pass<R>(g.Mx, FP_XFWD, fa)) != cudaSuccess) return e;
    } else if (adjoint) {
      k_p1<R, true><<<g1, 256, sm1, st>>>(xr, w.B1, lat, br, g.n_occ, g.nrows, g.px, twx, lt1,
                                          bstride, sk); count_launch();
    } else {
      k_p1<R, false><<<g1, 256, sm1, st>>>(xr, w.B1, lat, br, g.n_occ, g.nrows, g.px, twx, lt1,
                                           bstride, sk); count_launch();
    }
    tr_end(g.tr, st, tb);
    tr_begin(g.tr, st);
    // P2: y lines of B1 [rhs][3][nz][ny][Mx] -> B2 [rhs][3][nz][My][Mx]
    if (fy) {
      fa.in = w.B1; fa.out = w.B2; fa.tw = twy;
      e = fast_pass<R>(g.My, FP_YFWD, fa);
    } else {
      e = launch_lines<R>(g, w.B1, w.B2, g.py, twy, false, g.ny, g.My, g.Mx, g.nz, 3 * cnt, false,
                          g.Mx, 1, (long long)g.ny * g.Mx, (long long)g.nz * g.ny * g.Mx,
                          g.Mx, 1, (long long)g.My * g.Mx, (long long)g.nz * g.My * g.Mx, st, sk);
    }
    if (e != cudaSuccess) return e;
    tr_end(g.tr, st, tb + 1);
    dim3 g3((g.Mx + (1 << lt3) - 1) >> lt3, g.My, cnt);
    tr_begin(g.tr, st);
    // P3: z lines, product with the octant of FFT(G), inverse z lines (in place)
    if (fz) {
      fa.out = w.B2; fa.tw = twz;
      if ((e = fast_pass<R>(g.Mz, FP_ZCONV, fa)) != cudaSuccess) return e;
    } else {
      k_p3<R><<<g3, 256, sm3, st>>>(w.B2, w.D, g.nz, g.Mx, g.My, g.pz, twz, lt3, sk); count_launch();
    }
    tr_end(g.tr, st, tb + 2);
    tr_begin(g.tr, st);
    // P4: inverse y, keep y < ny
    if (fy) {
      fa.in = w.B2; fa.out = w.B1; fa.tw = twy;
      e = fast_pass<R>(g.My, FP_YINV, fa);
    } else {
      e = launch_lines<R>(g, w.B2, w.B1, g.py, twy, true, g.My, g.ny, g.Mx, g.nz, 3 * cnt, false,
                          g.Mx, 1, (long long)g.My * g.Mx, (long long)g.nz * g.My * g.Mx,
                          g.Mx, 1, (long long)g.ny * g.Mx, (long long)g.nz * g.ny * g.Mx, st, sk);
    }
    if (e != cudaSuccess) return e;
    tr_end(g.tr, st, tb + 3);
    tr_begin(g.tr, st);
    // P5: inverse x, keep the occupied x, y = x - beta u (+ partials of x^T y)
    if (fx) {
      fa.in = w.B1; fa.x = xr; fa.out = yr; fa.tw = twx;
      if (dotp && dot_nb) fa.dotp = dotp + (size_t)r0 * 2 * dnb;
      if ((e = fast_pass<R>(g.Mx, FP_XINV, fa)) != cudaSuccess) return e;
    } else if (adjoint) {
      k_p5<R, true><<<g1, 256, sm1, st>>>(w.B1, xr, yr, lat, br, g.n_occ, g.nrows, g.px, twx, lt1,
                                          bstride, sk); count_launch();
    } else {
      k_p5<R, false><<<g1, 256, sm1, st>>>(w.B1, xr, yr, lat, br, g.n_occ, g.nrows, g.px, twx, lt1,
                                           bstride, sk); count_launch();
    }
    tr_end(g.tr, st, tb + 4);
  }
  return cudaGetLastError();
}

__global__ void k_beta_df(const c128* __restrict__ b, cdf* __restrict__ o, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = to_cdf(b[i]);
}

cudaError_t launch_matvec_df(const Geom& g, const LatticeDev& lat, Work<df>& w, const c128* beta,
                             int n_mat, const c128* x, c128* y, int nrhs, cudaStream_t st,
                             const int* skip) {
  if (!(fast_supported(g.Mx) && fast_supported(g.My) && fast_supported(g.Mz)) || g.engine != 0)
    return cudaErrorNotSupported;
  const int bstride = n_mat * 3;
  // beta as double-float, grown with the number of right-hand sides
  if (w.cap_beta < nrhs * bstride) {
    dev_free(w.beta, st);
    w.beta = nullptr;
    w.cap_beta = 0;
    cudaError_t e = dev_malloc(&w.beta, (size_t)nrhs * bstride * sizeof(cdf));
    if (e != cudaSuccess) return e;
    w.cap_beta = nrhs * bstride;
  }
  const int nb = nrhs * bstride;
  k_beta_df<<<(nb + 127) / 128, 128, 0, st>>>(beta, w.beta, nb); count_launch();
  const long long nv = 3LL * g.n_occ;
  const cdf* twx = w.tw;
  const cdf* twy = w.tw + g.Mx;
  const cdf* twz = w.tw + g.Mx + g.My;
  const int cap = w.cap > 0 ? w.cap : 1;
  cudaError_t e = cudaSuccess;
  for (int r0 = 0; r0 < nrhs; r0 += cap) {
    const int cnt = nrhs - r0 < cap ? nrhs - r0 : cap;
    FastArgs fa{};
    fa.lat = lat; fa.beta = w.beta + (long long)r0 * bstride; fa.D = w.D; fa.n_occ = g.n_occ;
    fa.nrows = g.nrows; fa.ny = g.ny; fa.nz = g.nz; fa.Mx = g.Mx; fa.My = g.My; fa.adj = false;
    fa.st = st; fa.nrhs = cnt; fa.bstride = bstride; fa.skip = skip ? skip + r0 : nullptr;
    fa.pdl = fast_pdl(false, g.Mx, g.My, g.Mz, cnt);
    fa.var_yf = g.tiles[2][0] > 0 ? g.tiles[2][0] : 0;
    fa.var_z = g.tiles[2][1] > 0 ? g.tiles[2][1] : 0;
    fa.var_yi = g.tiles[2][2] > 0 ? g.tiles[2][2] : 0;
    tr_begin(g.tr, st);
    fa.in = x + r0 * nv; fa.out = w.B1; fa.tw = twx;
    if ((e = fast_pass<df>(g.Mx, FP_XFWD, fa)) != cudaSuccess) return e;
    tr_end(g.tr, st, TR_P1_DF);
    tr_begin(g.tr, st);
    fa.in = w.B1; fa.out = w.B2; fa.tw = twy;
    if ((e = fast_pass<df>(g.My, FP_YFWD, fa)) != cudaSuccess) return e;
    tr_end(g.tr, st, TR_P2_DF);
    tr_begin(g.tr, st);
    fa.out = w.B2; fa.tw = twz;
    if ((e = fast_pass<df>(g.Mz, FP_ZCONV, fa)) != cudaSuccess) return e;
    tr_end(g.tr, st, TR_P3_DF);
    tr_begin(g.tr, st);
    fa.in = w.B2; fa.out = w.B1; fa.tw = twy;
    if ((e = fast_pass<df>(g.My, FP_YINV, fa)) != cudaSuccess) return e;
    tr_end(g.tr, st, TR_P4_DF);
    tr_begin(g.tr, st);
    fa.in = w.B1; fa.x = x + r0 * nv; fa.out = y + r0 * nv; fa.tw = twx;
    if ((e = fast_pass<df>(g.Mx, FP_XINV, fa)) != cudaSuccess) return e;
    tr_end(g.tr, st, TR_P5_DF);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t tune_tiles(Geom& g, const LatticeDev& lat, Work<R>& w, cudaStream_t st) {
  const int kind = std::is_same<R, float>::value ? 0 : std::is_same<R, double>::value ? 1 : 2;
  int* tl = g.tiles[kind];
  if (tl[0] >= 0 && tl[1] >= 0 && tl[2] >= 0) return cudaSuccess;
  auto has = [](int M) { return std::is_same<R, float>::value ? fast_supported_c64(M) : fast_supported(M); };
  if (g.engine != 0 || !w.B1 || !w.B2 || !w.D || !w.tw) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::array<int, 8>, std::array<int, 3>> cache;
  const std::array<int, 8> key{dev, kind, g.Mx, g.My, g.Mz, g.ny, g.nz, 0};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      for (int k = 0; k < 3; ++k)
        if (tl[k] < 0) tl[k] = it->second[k];
      return cudaSuccess;
    }
  }
  FastArgs fa{};
  fa.lat = lat; fa.D = w.D; fa.n_occ = g.n_occ; fa.nrows = g.nrows;
  fa.ny = g.ny; fa.nz = g.nz; fa.Mx = g.Mx; fa.My = g.My; fa.st = st; fa.nrhs = 1;
  const cpx<R>* twy = w.tw + g.Mx;
  const cpx<R>* twz = w.tw + g.Mx + g.My;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  std::array<int, 3> best{0, 0, 0};
  for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
    if (!has(pass == 1 ? g.Mz : g.My)) continue;       // that axis runs the Stockham passes
    float tbest = 0.f;
    for (int var = 0; var < 2 && e == cudaSuccess; ++var) {
      FastArgs a = fa;
      int op, M;
      if (pass == 0) { op = FP_YFWD; M = g.My; a.in = w.B1; a.out = w.B2; a.tw = twy; a.var_yf = var; }
      else if (pass == 1) { op = FP_ZCONV; M = g.Mz; a.out = w.B2; a.tw = twz; a.var_z = var; }
      else { op = FP_YINV; M = g.My; a.in = w.B2; a.out = w.B1; a.tw = twy; a.var_yi = var; }
      if ((e = fast_pass<R>(M, op, a)) != cudaSuccess) break;   // warm-up (attributes, code)
      if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
      for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = fast_pass<R>(M, op, a);
      if (e != cudaSuccess) break;
      if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      // the half tiles only when clearly faster (3 %): a choice between variants
      // within the launch-to-launch noise would change from run to run
      if (var == 0 || ms < 0.97f * tbest) { tbest = ms; best[pass] = var; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = best;
  }
  for (int k = 0; k < 3; ++k)
    if (tl[k] < 0) tl[k] = best[k];
  return cudaSuccess;
}

template cudaError_t tune_tiles<float>(Geom&, const LatticeDev&, Work<float>&, cudaStream_t);
template cudaError_t tune_tiles<double>(Geom&, const LatticeDev&, Work<double>&, cudaStream_t);
template cudaError_t tune_tiles<df>(Geom&, const LatticeDev&, Work<df>&, cudaStream_t);

template cudaError_t launch_matvec<float>(const Geom&, const LatticeDev&, Work<float>&,
                                          const c64*, int, const c64*, c64*, int, bool,
                                          cudaStream_t, double*, int*, const int*);
template cudaError_t launch_matvec<double>(const Geom&, const LatticeDev&, Work<double>&,
                                           const c128*, int, const c128*, c128*, int, bool,
                                           cudaStream_t, double*, int*, const int*);
template cudaError_t launch_lines<double>(const Geom&, const c128*, c128*, const FftPlan&,
                                          const c128*, bool, int, int, int, int, int, bool,
                                          long long, long long, long long, long long, long long,
                                          long long, long long, long long, cudaStream_t,
                                          const int*);
template cudaError_t launch_lines<float>(const Geom&, const c64*, c64*, const FftPlan&,
                                         const c64*, bool, int, int, int, int, int, bool,
                                         long long, long long, long long, long long, long long,
                                         long long, long long, long long, cudaStream_t,
                                         const int*);

// Factor M into radices 8, 4, 2, 3, 5, 7 (in that order of preference).
FftPlan make_plan(int M) {
  FftPlan p{};
  p.M = M;
  p.nst = 0;
  int r = M;
  const int order[] = {8, 4, 2, 3, 5, 7};
  for (int q : order) {
    while (r % q == 0 && p.nst < kMaxStages) {
      p.radix[p.nst++] = q;
      r /= q;
    }
  }
  if (r != 1) p.nst = -1;  // not 7-smooth
  return p;
}

int padded_length(int lo, int engine) {
  const int smooth = smooth_size(lo);
  if (engine != 0) return smooth;
  // compiled lengths, ascending (complex64 passes also exist for 512 and 1080)
  static const int kFast[] = {32, 40, 48, 64, 80, 96, 128, 256, 270, 512, 1080};
  for (int M : kFast)
    if (M >= lo) return (double)M <= 1.35 * smooth ? M : smooth;
  return smooth;
}

int smooth_size(int lo) {
  int m = lo < 1 ? 1 : lo;
  for (;; ++m) {
    int r = m;
    for (int q : {2, 3, 5, 7})
      while (r % q == 0) r /= q;
    if (r == 1) return m;
  }
}

}  // namespace dda
