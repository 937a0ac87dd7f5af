// Krylov solvers of arXiv:0704.0037, Sec. 2 (CGNR, Bi-CGSTAB, Bi-CG, QMR),
// for A x = b of Eq. (3), with A of Eq. (2) applied by the FFT product.
//
// QMR and Bi-CG use the complex symmetry A = A^T (bilinear form u^T v);
// Bi-CGSTAB and CGNR use Hermitian products (CGNR on A^H A, with
// A^H y = conj(A conj y)).  Stopping rule (Sec. 2, 3.1): relative residual
// ||b - A x|| / ||b|| < tol.  x0 = 0.
//
// Vectors live on the device in complex64 or complex128; every inner
// product is accumulated in FP64 per thread, reduced per block with warp
// shuffles, and the per-block partials are summed by a one-block kernel in a
// fixed order, so reruns are bitwise identical.  The scalar recurrences
// (Lanczos coefficients, Givens rotations, step lengths) run in FP64 on the
// device; the host reads a small status record once per iteration.
//
// DDA_FP32_REFINED: complex64 inner solves of A d = r / ||r|| inside an FP64
// iterative refinement x += ||r|| d, r = b - A x (FP64 product), which is
// also the true residual the stop test uses.
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>

#include <cstdlib>

#include "internal.h"

namespace dda {

constexpr int kNB = 1024;     // max blocks of a vector kernel (partials per slot)
// Breakdown of the bilinear-form solvers (QMR-CS, Bi-CG-CS; no look-ahead):
// a bilinear form u^T u at the rounding level of the Hermitian one,
// |u^T u| <= 1e-12 ||u||^2, counts as zero (kBreak2 is the square of 1e-12)
constexpr double kBreak2 = 1e-24;
constexpr int kSlots = 8;     // doubles per block in the partials array
constexpr int kVT = 256;      // threads of vector kernels
constexpr long long kPS = (long long)kSlots * kNB;   // partials per right-hand side
// Batched launches: vector kernels take right-hand side blockIdx.y (vectors
// [nrhs][n], partials at part + r * kPS, scalars at s + r), scalar kernels
// take right-hand side blockIdx.x (one block each).  Single right-hand-side
// launches have gridDim.y = 1 and one block, i.e. r = 0.

// QMR-CS scalars (see the QMR-CS section)
struct QmrScal {
  double rho, inv_rho, g, theta, cd;
  c128 delta, eps, eps_new, beta, eta, cp;
};

struct Scal {
  double bnorm, res, sres, tol;
  int done, status, half, iters;   // iters: steps taken (batched QMR)
  int cnt;                         // blocks of the current sweep that have finished
  c128 alpha, beta_k, beta_next, inv_beta, t, tau, delta, eps, inv_gamma, s1, s2;
  double c1, c2;
  c128 rho, rho_prev, omega, bstep;
  double zz, ww;
  QmrScal q;
};

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Reduce K per-thread values over the block and store them as this block's
// partials part[k * kNB + blockIdx.x] (k = slot0 .. slot0+K-1).  A = float
// (partials of complex64 vectors, FP32-accurate already) sums within each
// warp in FP32 and across warps in FP64; A = double sums in FP64 throughout.
template <int K, typename A = double>
__device__ void block_store(double (&v)[K], double* part, int slot0) {
  __shared__ double sh[K][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double s = (double)warp_sum((A)v[k]);
    if (lane == 0) sh[k][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = lane < nw ? sh[k][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) part[(slot0 + k) * kNB + blockIdx.x] = s;
    }
  }
}

// Sum slot `slot` of the partials of nb blocks; one block of kVT threads, fixed order.
__device__ double fin(const double* part, int slot, int nb) {
  __shared__ double sh[kVT];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[slot * kNB + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ c128 cfin(const double* part, int slot, int nb) {
  const double re = fin(part, slot, nb);
  const double im = fin(part, slot + 1, nb);
  return mk<double>(re, im);
}

// K sums at once: entry (k, i) of the partials sits at p[k * ks + i * is],
// i < nb.  One block of kVT threads; fixed order (per-thread strided sums,
// warp shuffles, then the warps in order), the same result in every thread.
template <int K>
__device__ void fin_k(const double* p, long long ks, long long is, int nb, double (&out)[K]) {
  __shared__ double sh[K][kVT / 32];
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0.0;
  // four strides' loads in flight per thread (the partials come from L2)
#pragma unroll 4
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __ldcg(p + k * ks + i * is);   // other blocks' writes
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = warp_sum(v[k]);
    if (lane == 0) sh[k][wid] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += sh[k][w];
    out[k] = x;
  }
  __syncthreads();
}

// True in every thread of the block that finishes last among the gridDim.x
// blocks working on one right-hand side (counter *cnt, reset here for the
// next sweep); every block's partials are then visible to it.  A sweep ends
// with its reduction in that block instead of a separate one-block launch.
// Thread 0 wrote the block's partials (block_store), so it alone fences
// before counting; the last block reads the partials through L2 (fin_k).
__device__ bool last_block(int* cnt) {
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(cnt, 1) == (int)gridDim.x - 1;
    if (is_last) *cnt = 0;
  }
  __syncthreads();
  return is_last != 0;
}

// Running sum of the products for complex128 vectors in FP64; for complex64
// vectors a compensated (Kahan) sum in FP32, whose error is a few units of
// 2^-24 of the sum of magnitudes whatever the number of terms, with no FP64
// work per term (the FP64 pipe is ~1/58 of the FP32 rate on this part, and a
// conditional FP64 flush every few terms gets if-converted into an FP64 add
// per term).
template <typename R> struct Acc {
  double d = 0.0;
  __device__ __forceinline__ void add(R v) { d += v; }
  __device__ __forceinline__ double get() const { return d; }
};
template <> struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

__device__ __forceinline__ c128 csqrt_p(c128 z) {
  const double r = hypot(z.x, z.y);
  if (r == 0.0) return mk<double>(0.0, 0.0);
  if (z.x >= 0.0) {
    const double t = sqrt(0.5 * (r + z.x));
    return mk<double>(t, z.y / (2.0 * t));
  }
  const double t = sqrt(0.5 * (r - z.x));
  return mk<double>(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}
__device__ __forceinline__ c128 cdivd(c128 a, c128 b) {
  const double d = b.x * b.x + b.y * b.y;
  return mk<double>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double cabs2(c128 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ bool cfinite(c128 a) { return isfinite(a.x) && isfinite(a.y); }

template <typename R> __device__ __forceinline__ cpx<R> cs(c128 a) { return mk<R>((R)a.x, (R)a.y); }

#define VLOOP(n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); \
                      i += (long long)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- generic kernels
template <typename R, bool HERM>
__global__ void __launch_bounds__(kVT) k_dot(const cpx<R>* __restrict__ a, const cpx<R>* __restrict__ b,
                                             long long n, double* part, int slot, const Scal* s) {
  a += blockIdx.y * n; b += blockIdx.y * n; part += blockIdx.y * kPS;
  if (s) s += blockIdx.y;
  if (s && s->done) return;
  Acc<R> a0, a1;
  VLOOP(n) {
    const R ax = a[i].x, ay = HERM ? -a[i].y : a[i].y;
    const R bx = b[i].x, by = b[i].y;
    a0.add(ax * bx - ay * by);
    a1.add(ax * by + ay * bx);
  }
  double v[2] = {a0.get(), a1.get()};
  block_store<2, R>(v, part, slot);
}

// |a|^2 and, optionally, a^T a (bilinear)
template <typename R>
__global__ void __launch_bounds__(kVT) k_norms(const cpx<R>* __restrict__ a, long long n, double* part,
                                               const Scal* s) {
  a += blockIdx.y * n; part += blockIdx.y * kPS;
  if (s) s += blockIdx.y;
  if (s && s->done) return;
  double v[3] = {0.0, 0.0, 0.0};
  VLOOP(n) {
    const double x = a[i].x, y = a[i].y;
    v[0] += x * x - y * y;
    v[1] += 2.0 * x * y;
    v[2] += x * x + y * y;
  }
  block_store<3>(v, part, 0);
}

template <typename R>
__global__ void k_zero(cpx<R>* a, long long n) { VLOOP(n) a[i] = mk<R>(0, 0); }

template <typename R>
__global__ void k_copy(const cpx<R>* __restrict__ a, cpx<R>* __restrict__ b, long long n) {
  VLOOP(n) b[i] = a[i];
}

// ---------------------------------------------------------------- RHS and P

// exp(i kd a_mu r_mu) along x (nx entries), then y, then z: the incident
// phase exp(i kd a.r) of a dipole is the product of three entries
__global__ void k_axis_phase(c128* __restrict__ tab, double kd, Wave w, int nx, int ny, int nz) {
  const int L = nx + ny + nz;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
    int j = k, axis = 0, n = nx;
    if (j >= nx) { j -= nx; axis = 1; n = ny; if (j >= ny) { j -= ny; axis = 2; n = nz; } }
    double sn, cn;
    sincos(kd * w.a[axis] * (0.5 * (2 * j + 1 - n)), &sn, &cn);
    tab[k] = mk<double>(cn, sn);
  }
}

// b_i = beta_i e exp(i kd a.r_i)  (Eq. (3)), rows in parallel, a warp per
// row; ptab from k_axis_phase
template <typename R>
__global__ void k_rhs(cpx<R>* __restrict__ b, LatticeDev lat, const c128* __restrict__ beta,
                      long long n_occ, int nx, int ny, int nrows, const c128* __restrict__ ptab,
                      Wave w) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int row = warp; row < nrows; row += nwarps) {
    const int iy = row % ny, iz = row / ny;
    const c128 pyz = ptab[nx + iy] * ptab[nx + ny + iz];
    for (long long i = lat.row_off[row] + lane; i < lat.row_off[row + 1]; i += 32) {
      const c128 ph = ptab[lat.xi[i]] * pyz;
      for (int c = 0; c < 3; ++c) {
        const c128 e = mk<double>(w.e[2 * c], w.e[2 * c + 1]);
        const c128 v = beta[lat.mat[i] * 3 + c] * (e * ph);
        b[c * n_occ + i] = cs<R>(v);
      }
    }
  }
}

// b = beta e exp(i kd a.r) for one right-hand side on stream st
int launch_rhs(dda_t h, c128* b, const c128* beta, const Wave& wv, cudaStream_t st) {
  const Geom& g = h->g;
  if (!h->d_ptab) {
    if (dev_malloc(&h->d_ptab, (size_t)(g.nx + g.ny + g.nz) * sizeof(c128)) != cudaSuccess) {
      h->d_ptab = nullptr;
      cudaGetLastError();
      return dda_fail(h, DDA_ERR_OOM, "incident phase table");
    }
  }
  const int L = g.nx + g.ny + g.nz;
  c128* ptab = (c128*)h->d_ptab;
  k_axis_phase<<<(L + 255) / 256, 256, 0, st>>>(ptab, h->kd, wv, g.nx, g.ny, g.nz); count_launch();
  const int rows_grid = (int)std::min<long long>((g.nrows + 7) / 8, 32LL * num_sms());
  k_rhs<double><<<rows_grid, 256, 0, st>>>(b, h->lat(), beta, g.n_occ, g.nx, g.ny, g.nrows, ptab,
                                           wv); count_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DDA_OK : dda_cuda_fail(h, e, "right-hand side");
}

// P = beta x (Eq. (3)), FP64 output
template <typename R>
__global__ void k_pfinal(const cpx<R>* __restrict__ x, c128* __restrict__ P, const uint8_t* __restrict__ mat,
                         const c128* __restrict__ beta, long long n_occ) {
  VLOOP(3 * n_occ) {
    const int c = (int)(i / n_occ);
    const long long j = i - c * n_occ;
    P[i] = beta[mat[j] * 3 + c] * to128(x[i]);
  }
}

// ---------------------------------------------------------------- QMR-CS
// Freund's QMR for A = A^T without look-ahead, on coupled two-term
// recurrences (Freund and Nachtigal's implementation; the left and right
// Lanczos sequences coincide, one product per step).  Lanczos vectors have
// unit Euclidean norm; delta_i = v_i^T v_i carries the bilinear form.
//   p_i = v_i - cp p_{i-1},  cp = rho_i delta_i / eps_{i-1};   pt = A p_i
//   eps_i = p_i^T pt,  beta_i = eps_i / delta_i,  vt = pt - beta_i v_i
//   rho_{i+1} = ||vt||,  theta_i = rho_{i+1} / (g_{i-1} |beta_i|),
//   g_i = 1/sqrt(1 + theta_i^2),  eta_i = -eta_{i-1} rho_i g_i^2 / (beta_i g_{i-1}^2)
//   d = eta_i p_i + (theta_{i-1} g_i)^2 d,  s = eta_i pt + (theta_{i-1} g_i)^2 s
//   x += d,  r -= s
// The three-term, bilinear-scaled form of the same Lanczos process loses its
// convergence rate in complex64 for large size parameters; this form tracks
// the FP64 iteration.  Scalars live in QmrScal (FP64), vectors in R.

// part: slots 0/1 = b^T b, slot 2 = |b|^2 (k_norms).  tols (device, or null:
// tol for all) per right-hand side; off (device, or null) marks right-hand
// sides that start done; mask (device, or null) mirrors the done flags.
__global__ void k_qmr_init(Scal* s, const double* part, int nb, double tol, const double* tols,
                           const int* off, int* mask) {
  const int rr = blockIdx.x;
  s += rr; part += rr * kPS;
  const c128 bb = cfin(part, 0, nb);
  const double bn2 = fin(part, 2, nb);
  if (threadIdx.x) return;
  QmrScal& q = s->q;
  s->tol = tols ? tols[rr] : tol;
  s->iters = 0;
  s->cnt = 0;
  s->bnorm = sqrt(bn2);
  s->res = 1.0;
  s->done = 0; s->half = 0;
  s->status = DDA_NOT_CONVERGED;
  q.rho = s->bnorm;
  q.inv_rho = bn2 > 0.0 ? 1.0 / q.rho : 0.0;
  q.delta = bn2 > 0.0 ? scale<double>(bb, 1.0 / bn2) : mk<double>(0.0, 0.0);
  q.g = 1.0; q.theta = 0.0; q.cd = 0.0;
  q.eta = mk<double>(-1.0, 0.0);
  q.eps = mk<double>(1.0, 0.0);
  q.cp = mk<double>(0.0, 0.0);
  q.beta = mk<double>(0.0, 0.0);
  if (bn2 == 0.0) { s->done = 1; s->status = DDA_OK; s->res = 0.0; }
  else if (!isfinite(bn2) || !cfinite(bb)) { s->done = 1; s->status = DDA_ERR_NONFINITE; }
  else if (cabs2(q.delta) <= kBreak2) { s->done = 1; s->status = DDA_BREAKDOWN; }
  if (off && off[rr]) { s->done = 1; s->status = DDA_OK; }
  if (mask) mask[rr] = s->done;
}

// v_1 = b / rho_1, p_1 = v_1, r = b, x = d = s = 0
template <typename R>
__global__ void k_qmr_start(const cpx<R>* __restrict__ b, cpx<R>* __restrict__ v,
                            cpx<R>* __restrict__ p, cpx<R>* __restrict__ r, cpx<R>* __restrict__ x,
                            cpx<R>* __restrict__ d, cpx<R>* __restrict__ sv, long long n,
                            const Scal* s) {
  const long long o = blockIdx.y * n;
  b += o; v += o; p += o; r += o; x += o; d += o; sv += o;
  s += blockIdx.y;
  const R ir = (R)s->q.inv_rho;
  const cpx<R> z = mk<R>(0, 0);
  VLOOP(n) {
    const cpx<R> bi = b[i];
    const cpx<R> vi = scale<R>(bi, ir);
    v[i] = vi; p[i] = vi; r[i] = bi; x[i] = z; d[i] = z; sv[i] = z;
  }
}

// End right-hand side rr's solve with `status` (one thread); its products
// are skipped from then on when a mask is kept
__device__ __forceinline__ void qmr_stop(Scal* s, int status, int* mask, int rr) {
  s->status = status;
  s->done = 1;
  if (mask) mask[rr] = 1;
}

// eps_i = p^T A p from partials (entry (k, i) at part[k * ks + i * is],
// right-hand side r's partials at part + r * rs); beta_i
__global__ void k_qmr_a(Scal* s, const double* part, long long ks, long long is, long long rs,
                        int nb, int* mask) {
  pdl_wait();
  pdl_launch();
  const int rr = blockIdx.x;
  s += rr; part += rr * rs;
  if (s->done) return;
  double a[2];
  fin_k<2>(part, ks, is, nb, a);
  if (threadIdx.x) return;
  QmrScal& q = s->q;
  const c128 eps = mk<double>(a[0], a[1]);
  const c128 beta = cdivd(eps, q.delta);
  if (!cfinite(eps) || !cfinite(beta)) { qmr_stop(s, DDA_ERR_NONFINITE, mask, rr); return; }
  if (cabs2(eps) == 0.0 || cabs2(beta) == 0.0) { qmr_stop(s, DDA_BREAKDOWN, mask, rr); return; }
  q.eps_new = eps;
  q.beta = beta;
}

// rho_{i+1}, delta_{i+1}, the quasi-minimisation scalars of step i and the
// coefficients of the update and of the next direction, from the nb partials
// of the k1 sweep (all threads of one block)
__device__ void qmr_b_fin(Scal* s, const double* part, int nb, int* mask, int rr) {
  double f[3];
  fin_k<3>(part, kNB, 1, nb, f);
  if (threadIdx.x) return;
  QmrScal& q = s->q;
  const c128 vtv = mk<double>(f[0], f[1]);
  const double rho_n = sqrt(f[2]);
  const double theta = rho_n / (q.g * sqrt(cabs2(q.beta)));
  const double g = 1.0 / sqrt(1.0 + theta * theta);
  const c128 eta = scale<double>(cdivd(q.eta, q.beta), -q.rho * g * g / (q.g * q.g));
  if (!isfinite(rho_n) || !cfinite(vtv) || !isfinite(theta) || !cfinite(eta)) {
    qmr_stop(s, DDA_ERR_NONFINITE, mask, rr);
    return;
  }
  q.cd = (q.theta * g) * (q.theta * g);
  q.eta = eta;
  q.g = g;
  q.theta = theta;
  s->half = 0;
  if (rho_n == 0.0) {            // invariant subspace: this step's update is exact
    q.inv_rho = 0.0;
    q.cp = mk<double>(0.0, 0.0);
    s->half = 2;
  } else {
    const c128 delta = scale<double>(vtv, 1.0 / (rho_n * rho_n));
    q.inv_rho = 1.0 / rho_n;
    q.cp = scale<double>(cdivd(delta, q.eps_new), rho_n);
    q.delta = delta;
    if (cabs2(delta) <= kBreak2) s->half = 1;      // next v^T v vanishes: breakdown after this step
  }
  q.rho = rho_n;
  q.eps = q.eps_new;
}

// stop test on the nb partials of |r|^2 of the k2 sweep (all threads of one block)
__device__ void qmr_c_fin(Scal* s, const double* part, int nb, int* mask, int rr) {
  double f[1];
  fin_k<1>(part, kNB, 1, nb, f);
  const double rn2 = f[0];
  if (threadIdx.x) return;
  const double res = sqrt(rn2) / s->bnorm;
  s->res = res;
  s->iters++;
  if (!isfinite(res)) { s->status = DDA_ERR_NONFINITE; s->done = 1; }
  else if (res < s->tol) { s->status = DDA_OK; s->done = 1; }
  else if (s->half) { s->status = DDA_BREAKDOWN; s->done = 1; }
  if (mask) mask[rr] = s->done;
}

// vt = pt - beta v (into v); partials of vt^T vt and |vt|^2, reduced by the
// last block to finish (qmr_b_fin)
template <typename R>
__global__ void __launch_bounds__(kVT) k_qmr_k1(const cpx<R>* __restrict__ pt, cpx<R>* __restrict__ v,
                                                long long n, Scal* s, double* part, int* mask) {
  pdl_wait();
  pdl_launch();
  pt += blockIdx.y * n; v += blockIdx.y * n; part += blockIdx.y * kPS; s += blockIdx.y;
  if (s->done) return;
  const cpx<R> be = cs<R>(s->q.beta);
  Acc<R> q0, q1, q2;
  // four elements per step with their loads issued together (two short
  // streams: without that the sweep is latency-bound)
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    cpx<R> a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { a[u] = pt[i + u * stride]; b[u] = v[i + u * stride]; }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const cpx<R> t = a[u] - be * b[u];
      v[i + u * stride] = t;
      const R x = t.x, y = t.y;
      q0.add(x * x - y * y);
      q1.add((R)2 * x * y);
      q2.add(x * x + y * y);
    }
  }
  for (; i < n; i += stride) {
    const cpx<R> t = pt[i] - be * v[i];
    v[i] = t;
    const R x = t.x, y = t.y;
    q0.add(x * x - y * y);
    q1.add((R)2 * x * y);
    q2.add(x * x + y * y);
  }
  double acc[3] = {q0.get(), q1.get(), q2.get()};
  block_store<3, R>(acc, part, 0);
  if (last_block(&s->cnt)) qmr_b_fin(s, part, gridDim.x, mask, blockIdx.y);
}

// d = eta p + cd d;  s = eta pt + cd s;  x += d;  r -= s (partial |r|^2);
// then v_{i+1} = vt / rho_{i+1} and p_{i+1} = v_{i+1} - cp p_i; the last
// block to finish takes the stop test (qmr_c_fin)
template <typename R>
__global__ void __launch_bounds__(kVT) k_qmr_k2(cpx<R>* __restrict__ v, cpx<R>* __restrict__ p,
                                                const cpx<R>* __restrict__ pt, cpx<R>* __restrict__ d,
                                                cpx<R>* __restrict__ sv, cpx<R>* __restrict__ x,
                                                cpx<R>* __restrict__ r, long long n, Scal* s,
                                                double* part, int* mask) {
  pdl_wait();
  pdl_launch();
  const long long o = blockIdx.y * n;
  v += o; p += o; pt += o; d += o; sv += o; x += o; r += o;
  part += blockIdx.y * kPS; s += blockIdx.y;
  if (s->done) return;
  const QmrScal& q = s->q;
  const cpx<R> et = cs<R>(q.eta), cp = cs<R>(q.cp);
  const R cd = (R)q.cd, ir = (R)q.inv_rho;
  Acc<R> acc;
  // two elements per step with their fourteen loads issued together
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i < n; i += 2 * stride) {
    const int m = i + stride < n ? 2 : 1;
    cpx<R> pv[2], dv[2], tv[2], sw[2], xv[2], rv[2], vv[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u < m) {
        const long long j = i + u * stride;
        pv[u] = p[j]; dv[u] = d[j]; tv[u] = pt[j]; sw[u] = sv[j];
        xv[u] = x[j]; rv[u] = r[j]; vv[u] = v[j];
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u < m) {
        const long long j = i + u * stride;
        const cpx<R> di = fmas<R>(dv[u], cd, et * pv[u]);
        const cpx<R> si = fmas<R>(sw[u], cd, et * tv[u]);
        d[j] = di;
        sv[j] = si;
        x[j] = xv[u] + di;
        const cpx<R> rr = rv[u] - si;
        r[j] = rr;
        acc.add(rr.x * rr.x + rr.y * rr.y);
        const cpx<R> vn = scale<R>(vv[u], ir);
        v[j] = vn;
        p[j] = vn - cp * pv[u];
      }
    }
  }
  double a[1] = {acc.get()};
  block_store<1, R>(a, part, 0);
  if (last_block(&s->cnt)) qmr_c_fin(s, part, gridDim.x, mask, blockIdx.y);
}

// ---------------------------------------------------------------- Bi-CG-CS (COCG)
__global__ void k_bicg_init(Scal* s, const double* part, int nb, double tol) {
  const c128 bb = cfin(part, 0, nb);
  const double bn2 = fin(part, 2, nb);
  if (threadIdx.x) return;
  s->tol = tol; s->bnorm = sqrt(bn2); s->res = 1.0; s->done = 0; s->half = 0;
  s->status = DDA_NOT_CONVERGED;
  s->rho = bb;
  if (bn2 == 0.0) { s->done = 1; s->status = DDA_OK; s->res = 0.0; }
  else if (!isfinite(bn2)) { s->done = 1; s->status = DDA_ERR_NONFINITE; }
  else if (cabs2(bb) <= kBreak2 * bn2 * bn2) { s->done = 1; s->status = DDA_BREAKDOWN; }
}

template <typename R>
__global__ void k_start3(const cpx<R>* __restrict__ b, cpx<R>* x, cpx<R>* r, cpx<R>* p, long long n) {
  VLOOP(n) { const cpx<R> bi = b[i]; x[i] = mk<R>(0, 0); r[i] = bi; p[i] = bi; }
}

__global__ void k_bicg_a(Scal* s, const double* part, int nb) {
  if (s->done) return;
  const c128 mu = cfin(part, 0, nb);
  if (threadIdx.x) return;
  if (!cfinite(mu)) { s->status = DDA_ERR_NONFINITE; s->done = 1; return; }
  if (cabs2(mu) == 0.0) { s->status = DDA_BREAKDOWN; s->done = 1; return; }
  s->alpha = cdivd(s->rho, mu);
}

// x += alpha p; r -= alpha q; partials r^T r and |r|^2
template <typename R>
__global__ void __launch_bounds__(kVT) k_bicg_k1(cpx<R>* __restrict__ x, cpx<R>* __restrict__ r,
                                                 const cpx<R>* __restrict__ p, const cpx<R>* __restrict__ q,
                                                 long long n, const Scal* s, double* part) {
  if (s->done) return;
  const cpx<R> al = cs<R>(s->alpha);
  double acc[3] = {0.0, 0.0, 0.0};
  VLOOP(n) {
    x[i] = x[i] + al * p[i];
    const cpx<R> t = r[i] - al * q[i];
    r[i] = t;
    const double a = t.x, b = t.y;
    acc[0] += a * a - b * b;
    acc[1] += 2.0 * a * b;
    acc[2] += a * a + b * b;
  }
  block_store<3>(acc, part, 0);
}

__global__ void k_bicg_b(Scal* s, const double* part, int nb) {
  if (s->done) return;
  const c128 rn = cfin(part, 0, nb);
  const double r2 = fin(part, 2, nb);
  if (threadIdx.x) return;
  const double res = sqrt(r2) / s->bnorm;
  s->res = res;
  if (!isfinite(res) || !cfinite(rn)) { s->status = DDA_ERR_NONFINITE; s->done = 1; return; }
  if (res < s->tol) { s->status = DDA_OK; s->done = 1; return; }
  if (cabs2(rn) <= kBreak2 * r2 * r2) { s->status = DDA_BREAKDOWN; s->done = 1; return; }
  s->bstep = cdivd(rn, s->rho);
  s->rho = rn;
}

// p = r + bstep p
template <typename R>
__global__ void k_bicg_k2(const cpx<R>* __restrict__ r, cpx<R>* __restrict__ p, long long n, const Scal* s) {
  if (s->done) return;
  const cpx<R> bs = cs<R>(s->bstep);
  VLOOP(n) p[i] = r[i] + bs * p[i];
}

// ---------------------------------------------------------------- Bi-CGSTAB
__global__ void k_bs_init(Scal* s, const double* part, int nb, double tol) {
  const double bn2 = fin(part, 2, nb);
  if (threadIdx.x) return;
  s->tol = tol; s->bnorm = sqrt(bn2); s->res = 1.0; s->done = 0; s->half = 0;
  s->status = DDA_NOT_CONVERGED;
  s->rho = mk<double>(bn2, 0.0);       // rhat^H r0 with rhat = r0 = b
  s->rho_prev = mk<double>(1.0, 0.0);
  s->alpha = mk<double>(1.0, 0.0);
  s->omega = mk<double>(1.0, 0.0);
  s->bstep = mk<double>(0.0, 0.0);     // p = r on the first step (p = v = 0)
  if (bn2 == 0.0) { s->done = 1; s->status = DDA_OK; s->res = 0.0; }
  else if (!isfinite(bn2)) { s->done = 1; s->status = DDA_ERR_NONFINITE; }
}

template <typename R>
__global__ void k_bs_start(const cpx<R>* __restrict__ b, cpx<R>* x, cpx<R>* r, cpx<R>* rh, cpx<R>* p,
                           cpx<R>* v, cpx<R>* t, long long n) {
  VLOOP(n) {
    const cpx<R> bi = b[i];
    x[i] = mk<R>(0, 0); r[i] = bi; rh[i] = bi; p[i] = mk<R>(0, 0); v[i] = mk<R>(0, 0);
    t[i] = mk<R>(0, 0);
  }
}

// p = r + bstep (p - omega v)
template <typename R>
__global__ void k_bs_p(const cpx<R>* __restrict__ r, cpx<R>* __restrict__ p, const cpx<R>* __restrict__ v,
                       long long n, const Scal* s) {
  if (s->done) return;
  const cpx<R> bs = cs<R>(s->bstep), om = cs<R>(s->omega);
  VLOOP(n) p[i] = r[i] + bs * (p[i] - om * v[i]);
}

__global__ void k_bs_a(Scal* s, const double* part, int nb) {
  if (s->done) return;
  const c128 q = cfin(part, 0, nb);
  if (threadIdx.x) return;
  if (!cfinite(q)) { s->status = DDA_ERR_NONFINITE; s->done = 1; return; }
  if (cabs2(q) == 0.0) { s->status = DDA_BREAKDOWN; s->done = 1; return; }
  s->alpha = cdivd(s->rho, q);
}

// s = r - alpha v ; partial |s|^2
template <typename R>
__global__ void __launch_bounds__(kVT) k_bs_s(const cpx<R>* __restrict__ r, const cpx<R>* __restrict__ v,
                                              cpx<R>* __restrict__ sv, long long n, const Scal* s,
                                              double* part) {
  if (s->done) return;
  const cpx<R> al = cs<R>(s->alpha);
  double acc[1] = {0.0};
  VLOOP(n) {
    const cpx<R> t = r[i] - al * v[i];
    sv[i] = t;
    acc[0] += (double)(t.x * t.x + t.y * t.y);
  }
  block_store<1>(acc, part, 0);
}

__global__ void k_bs_b(Scal* s, const double* part, int nb) {
  if (s->done) return;
  const double s2 = fin(part, 0, nb);
  if (threadIdx.x) return;
  s->sres = sqrt(s2) / s->bnorm;
  if (!isfinite(s->sres)) { s->status = DDA_ERR_NONFINITE; s->done = 1; return; }
  s->half = s->sres < s->tol ? 1 : 0;
}

// t^H s and t^H t
template <typename R>
__global__ void __launch_bounds__(kVT) k_bs_ts(const cpx<R>* __restrict__ t, const cpx<R>* __restrict__ sv,
                                               long long n, const Scal* s, double* part) {
  if (s->done) return;
  double acc[3] = {0.0, 0.0, 0.0};
  VLOOP(n) {
    const double tx = t[i].x, ty = t[i].y, sx = sv[i].x, sy = sv[i].y;
    acc[0] += tx * sx + ty * sy;
    acc[1] += tx * sy - ty * sx;
    acc[2] += tx * tx + ty * ty;
  }
  block_store<3>(acc, part, 0);
}

__global__ void k_bs_c(Scal* s, const double* part, int nb) {
  if (s->done) return;
  const c128 ts = cfin(part, 0, nb);
  const double tt = fin(part, 2, nb);
  if (threadIdx.x) return;
  if (s->half || tt == 0.0) s->omega = mk<double>(0.0, 0.0);
  else s->omega = scale<double>(ts, 1.0 / tt);
}

// x += alpha p + omega s ; r = s - omega t ; partials |r|^2 and rhat^H r
template <typename R>
__global__ void __launch_bounds__(kVT) k_bs_xr(cpx<R>* __restrict__ x, cpx<R>* __restrict__ r,
                                               const cpx<R>* __restrict__ p, const cpx<R>* __restrict__ sv,
                                               const cpx<R>* __restrict__ t, const cpx<R>* __restrict__ rh,
                                               long long n, const Scal* s, double* part) {
  if (s->done) return;
  const cpx<R> al = cs<R>(s->alpha), om = cs<R>(s->omega);
  double acc[3] = {0.0, 0.0, 0.0};
  VLOOP(n) {
    const cpx<R> si = sv[i];
    x[i] = x[i] + al * p[i] + om * si;
    const cpx<R> ri = si - om * t[i];
    r[i] = ri;
    const double a = ri.x, b = ri.y, hx = rh[i].x, hy = rh[i].y;
    acc[0] += a * a + b * b;
    acc[1] += hx * a + hy * b;
    acc[2] += hx * b - hy * a;
  }
  block_store<3>(acc, part, 0);
}

__global__ void k_bs_d(Scal* s, const double* part, int nb) {
  if (s->done) return;
  const double r2 = fin(part, 0, nb);
  const c128 rho = cfin(part, 1, nb);
  if (threadIdx.x) return;
  const double res = s->half ? s->sres : sqrt(r2) / s->bnorm;
  s->res = res;
  if (!isfinite(res)) { s->status = DDA_ERR_NONFINITE; s->done = 1; return; }
  if (res < s->tol) { s->status = DDA_OK; s->done = 1; return; }
  if (cabs2(rho) == 0.0 || cabs2(s->omega) == 0.0) { s->status = DDA_BREAKDOWN; s->done = 1; return; }
  s->rho_prev = s->rho;
  s->rho = rho;
  s->bstep = cdivd(rho, s->rho_prev) * cdivd(s->alpha, s->omega);
}

// ---------------------------------------------------------------- CGNR
__global__ void k_set_bnorm(Scal* s, const double* part, int nb, double tol) {
  const double bn2 = fin(part, 2, nb);
  if (threadIdx.x) return;
  s->tol = tol; s->bnorm = sqrt(bn2); s->res = 1.0; s->done = 0; s->half = 0;
  s->status = DDA_NOT_CONVERGED;
  s->zz = 0.0;
  if (bn2 == 0.0) { s->done = 1; s->status = DDA_OK; s->res = 0.0; }
  else if (!isfinite(bn2)) { s->done = 1; s->status = DDA_ERR_NONFINITE; }
}

template <typename R>
__global__ void k_start2(const cpx<R>* __restrict__ b, cpx<R>* x, cpx<R>* r, long long n) {
  VLOOP(n) { x[i] = mk<R>(0, 0); r[i] = b[i]; }
}

// store |.|^2 partial sum (slot 2 of k_norms) into zz (which = 0) or ww (1)
__global__ void k_cg_take(Scal* s, const double* part, int nb, int which) {
  if (s->done) return;
  const double v = fin(part, 2, nb);
  if (threadIdx.x) return;
  if (!isfinite(v)) { s->status = DDA_ERR_NONFINITE; s->done = 1; return; }
  if (which == 0) {           // zz of the new z: step for p = z + (zz_new/zz) p
    s->bstep = mk<double>(s->zz > 0.0 ? v / s->zz : 0.0, 0.0);
    s->zz = v;
  } else {                    // ww = |A p|^2 : alpha = zz / ww
    if (v == 0.0) { s->status = DDA_BREAKDOWN; s->done = 1; return; }
    s->ww = v;
    s->alpha = mk<double>(s->zz / v, 0.0);
  }
}

// x += alpha p; r -= alpha w; partial |r|^2 (slot 0)
template <typename R>
__global__ void __launch_bounds__(kVT) k_cg_k1(cpx<R>* __restrict__ x, cpx<R>* __restrict__ r,
                                               const cpx<R>* __restrict__ p, const cpx<R>* __restrict__ w,
                                               long long n, const Scal* s, double* part) {
  if (s->done) return;
  const cpx<R> al = cs<R>(s->alpha);
  double acc[1] = {0.0};
  VLOOP(n) {
    x[i] = x[i] + al * p[i];
    const cpx<R> t = r[i] - al * w[i];
    r[i] = t;
    acc[0] += (double)(t.x * t.x + t.y * t.y);
  }
  block_store<1>(acc, part, 0);
}

__global__ void k_res_check(Scal* s, const double* part, int nb) {
  if (s->done) return;
  const double r2 = fin(part, 0, nb);
  if (threadIdx.x) return;
  const double res = sqrt(r2) / s->bnorm;
  s->res = res;
  if (!isfinite(res)) { s->status = DDA_ERR_NONFINITE; s->done = 1; }
  else if (res < s->tol) { s->status = DDA_OK; s->done = 1; }
}

// ---------------------------------------------------------------- refinement (FP64 outer)
// r32 = (complex64)(r64 * scl)
__global__ void k_to32s(const c128* __restrict__ a, c64* __restrict__ b, long long n, double scl) {
  VLOOP(n) b[i] = mk<float>((float)(a[i].x * scl), (float)(a[i].y * scl));
}
// x64 += scl * d32
__global__ void k_axpy64(c128* __restrict__ x, const c64* __restrict__ d, long long n, double scl) {
  VLOOP(n) x[i] = mk<double>(x[i].x + scl * (double)d[i].x, x[i].y + scl * (double)d[i].y);
}
// r = b - w ; partial |r|^2 in slot 2 (as k_norms)
__global__ void __launch_bounds__(kVT) k_resid(const c128* __restrict__ b, const c128* __restrict__ w,
                                               c128* __restrict__ r, long long n, double* part) {
  double acc[3] = {0.0, 0.0, 0.0};
  VLOOP(n) {
    const c128 t = b[i] - w[i];
    r[i] = t;
    acc[2] += t.x * t.x + t.y * t.y;
  }
  block_store<3>(acc, part, 0);
}
__global__ void k_take_norm(Scal* s, const double* part, int nb) {
  const double v = fin(part, 2, nb);
  if (threadIdx.x == 0) s->sres = sqrt(v);
}

// ---------------------------------------------------------------- host orchestration
namespace {

struct Run {
  dda_t h;
  cudaStream_t st;
  long long n;       // 3 * N_occ
  int nb;            // blocks of vector kernels
  double* part;
  Scal* ds;
  Scal* hs;
  int rhs;           // RHS index (beta table)
  int matvecs = 0, matvecs64 = 0, iters = 0;
  std::vector<double>* hist = nullptr;
  double hist_scale = 1.0;
  // Inner complex64 solves stop when their residual, already below 1e-4,
  // has not improved by 1 % in stall_window iterations (the complex64
  // rounding floor); the FP64 refinement then continues.  0 = off.
  int stall_window = 0;
  double best = 1e300;
  int best_k = 0;
};

int sync_read(Run& R_) {
  dda_t h = R_.h;
  DDA_CK(h, cudaMemcpyAsync(R_.hs, R_.ds, sizeof(Scal), cudaMemcpyDeviceToHost, R_.st));
  DDA_CK(h, cudaStreamSynchronize(R_.st));
  return DDA_OK;
}

template <typename R> Work<R>& work(dda_t h);
template <> Work<double>& work<double>(dda_t h) { return h->w64; }
template <> Work<float>& work<float>(dda_t h) { return h->w32; }

template <typename R>
int matvec(Run& ru, const cpx<R>* x, cpx<R>* y, bool adj, double* dotp = nullptr,
           int* dot_nb = nullptr) {
  dda_t h = ru.h;
  Work<R>& w = work<R>(h);
  cudaError_t e = launch_matvec<R>(h->g, h->lat(), w, w.beta + (long long)ru.rhs * h->n_mat * 3,
                                   h->n_mat, x, y, 1, adj, ru.st, dotp, dot_nb);
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "matvec in solver");
  ru.matvecs++;
  if (sizeof(R) == 8) ru.matvecs64++;
  return DDA_OK;
}

#define RK(call) do { int rc_ = (call); if (rc_ != DDA_OK) return rc_; } while (0)
#define LK(h) do { cudaError_t e_ = cudaGetLastError(); if (e_ != cudaSuccess) return dda_cuda_fail(h, e_, "solver kernel"); } while (0)

// Run one solver in precision R on b (vector pool vec[0..]); the solution is
// left in x.  Returns DDA_OK or an error; the solver outcome is in ru.hs->status.
template <typename R>
int run_solver(Run& ru, int solver, const cpx<R>* b, cpx<R>* x, cpx<R>** vec, double tol, int maxiter) {
  dda_t h = ru.h;
  const long long n = ru.n;
  const int nb = ru.nb;
  cudaStream_t st = ru.st;
  double* part = ru.part;
  Scal* s = ru.ds;
  ru.best = 1e300;
  ru.best_k = ru.iters;
  auto rec = [&](void) {
    const double r = ru.hs->res;
    if (ru.hist) ru.hist->push_back(r * ru.hist_scale);
    if (r < 0.99 * ru.best) {
      ru.best = r;
      ru.best_k = ru.iters;
    } else if (ru.stall_window > 0 && r < 1e-4 && ru.iters - ru.best_k >= ru.stall_window) {
      ru.hs->done = 1;   // host copy only: ends this loop, status stays NOT_CONVERGED
    }
  };
  k_norms<R><<<nb, kVT, 0, st>>>(b, n, part, nullptr); count_launch();
  if (solver == DDA_QMR_CS) {
    cpx<R>*v = vec[0], *p = vec[1], *pt = vec[2], *d = vec[3], *sv = vec[4], *r = vec[5];
    k_qmr_init<<<1, kVT, 0, st>>>(s, part, nb, tol, nullptr, nullptr, nullptr); count_launch();
    k_qmr_start<R><<<nb, kVT, 0, st>>>(b, v, p, r, x, d, sv, n, s); count_launch();
    LK(h);
    RK(sync_read(ru));
    for (int k = 1; k <= maxiter && !ru.hs->done; ++k) {
      // pt = A p; eps = p^T pt, from the product's last pass when it can
      int dnb = 0;
      RK(matvec<R>(ru, p, pt, false, h->d_mvpart, &dnb));
      if (dnb > 0) {
        k_qmr_a<<<1, kVT, 0, st>>>(s, h->d_mvpart, 1, 2, 0, dnb, nullptr); count_launch();
      } else {
        k_dot<R, false><<<nb, kVT, 0, st>>>(p, pt, n, part, 0, s); count_launch();
        k_qmr_a<<<1, kVT, 0, st>>>(s, part, kNB, 1, 0, nb, nullptr); count_launch();
      }
      k_qmr_k1<R><<<nb, kVT, 0, st>>>(pt, v, n, s, part, nullptr); count_launch();
      k_qmr_k2<R><<<nb, kVT, 0, st>>>(v, p, pt, d, sv, x, r, n, s, part, nullptr); count_launch();
      LK(h);
      ru.iters++;
      RK(sync_read(ru));
      rec();
    }
  } else if (solver == DDA_BICG_CS) {
    cpx<R>*r = vec[0], *p = vec[1], *q = vec[2];
    k_bicg_init<<<1, kVT, 0, st>>>(s, part, nb, tol); count_launch();
    k_start3<R><<<nb, kVT, 0, st>>>(b, x, r, p, n); count_launch();
    LK(h);
    RK(sync_read(ru));
    for (int k = 1; k <= maxiter && !ru.hs->done; ++k) {
      RK(matvec<R>(ru, p, q, false));
      k_dot<R, false><<<nb, kVT, 0, st>>>(p, q, n, part, 0, s); count_launch();
      k_bicg_a<<<1, kVT, 0, st>>>(s, part, nb); count_launch();
      k_bicg_k1<R><<<nb, kVT, 0, st>>>(x, r, p, q, n, s, part); count_launch();
      k_bicg_b<<<1, kVT, 0, st>>>(s, part, nb); count_launch();
      k_bicg_k2<R><<<nb, kVT, 0, st>>>(r, p, n, s); count_launch();
      LK(h);
      ru.iters++;
      RK(sync_read(ru));
      rec();
    }
  } else if (solver == DDA_BICGSTAB) {
    cpx<R>*r = vec[0], *rh = vec[1], *p = vec[2], *v = vec[3], *sv = vec[4], *t = vec[5];
    k_bs_init<<<1, kVT, 0, st>>>(s, part, nb, tol); count_launch();
    k_bs_start<R><<<nb, kVT, 0, st>>>(b, x, r, rh, p, v, t, n); count_launch();
    LK(h);
    RK(sync_read(ru));
    for (int k = 1; k <= maxiter && !ru.hs->done; ++k) {
      k_bs_p<R><<<nb, kVT, 0, st>>>(r, p, v, n, s); count_launch();
      RK(matvec<R>(ru, p, v, false));
      k_dot<R, true><<<nb, kVT, 0, st>>>(rh, v, n, part, 0, s); count_launch();
      k_bs_a<<<1, kVT, 0, st>>>(s, part, nb); count_launch();
      k_bs_s<R><<<nb, kVT, 0, st>>>(r, v, sv, n, s, part); count_launch();
      k_bs_b<<<1, kVT, 0, st>>>(s, part, nb); count_launch();
      LK(h);
      RK(sync_read(ru));
      if (!ru.hs->done && !ru.hs->half) {
        RK(matvec<R>(ru, sv, t, false));
        k_bs_ts<R><<<nb, kVT, 0, st>>>(t, sv, n, s, part); count_launch();
      }
      k_bs_c<<<1, kVT, 0, st>>>(s, part, nb); count_launch();
      k_bs_xr<R><<<nb, kVT, 0, st>>>(x, r, p, sv, t, rh, n, s, part); count_launch();
      k_bs_d<<<1, kVT, 0, st>>>(s, part, nb); count_launch();
      LK(h);
      ru.iters++;
      RK(sync_read(ru));
      rec();
    }
  } else {  // CGNR
    cpx<R>*r = vec[0], *z = vec[1], *p = vec[2], *w = vec[3];
    k_set_bnorm<<<1, kVT, 0, st>>>(s, part, nb, tol); count_launch();
    k_start2<R><<<nb, kVT, 0, st>>>(b, x, r, n); count_launch();
    LK(h);
    RK(sync_read(ru));
    if (!ru.hs->done) {
      RK(matvec<R>(ru, r, z, true));
      k_copy<R><<<nb, kVT, 0, st>>>(z, p, n); count_launch();
      k_norms<R><<<nb, kVT, 0, st>>>(z, n, part, s); count_launch();
      k_cg_take<<<1, kVT, 0, st>>>(s, part, nb, 0); count_launch();
      LK(h);
    }
    for (int k = 1; k <= maxiter && !ru.hs->done; ++k) {
      RK(matvec<R>(ru, p, w, false));
      k_norms<R><<<nb, kVT, 0, st>>>(w, n, part, s); count_launch();
      k_cg_take<<<1, kVT, 0, st>>>(s, part, nb, 1); count_launch();
      k_cg_k1<R><<<nb, kVT, 0, st>>>(x, r, p, w, n, s, part); count_launch();
      k_res_check<<<1, kVT, 0, st>>>(s, part, nb); count_launch();
      LK(h);
      ru.iters++;
      RK(sync_read(ru));
      rec();
      if (ru.hs->done) break;
      RK(matvec<R>(ru, r, z, true));
      k_norms<R><<<nb, kVT, 0, st>>>(z, n, part, s); count_launch();
      k_cg_take<<<1, kVT, 0, st>>>(s, part, nb, 0); count_launch();
      k_bicg_k2<R><<<nb, kVT, 0, st>>>(z, p, n, s); count_launch();   // p = z + bstep p
      LK(h);
    }
  }
  return DDA_OK;
}

int ensure_solver_mem(dda_t h, size_t bytes) {
  if (!h->d_part) {
    if (dev_malloc(&h->d_part, kSlots * kNB * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return dda_fail(h, DDA_ERR_OOM, "solver partials"); }
    if (dev_malloc(&h->d_scal, sizeof(Scal)) != cudaSuccess) { cudaGetLastError(); return dda_fail(h, DDA_ERR_OOM, "solver scalars"); }
    const size_t mvp = 2 * (size_t)fast_xinv_blocks_max(h->g.nrows);
    if (dev_malloc(&h->d_mvpart, mvp * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return dda_fail(h, DDA_ERR_OOM, "product partials"); }
    if (cudaMallocHost(&h->h_scal, sizeof(Scal)) != cudaSuccess) { cudaGetLastError(); return dda_fail(h, DDA_ERR_OOM, "pinned scalars"); }
  }
  if (h->sv_bytes < bytes) {
    dev_free(h->sv, h->stream);
    h->sv = nullptr;
    h->sv_bytes = 0;
    if (dev_malloc(&h->sv, bytes) != cudaSuccess) { cudaGetLastError(); return dda_fail(h, DDA_ERR_OOM, "solver vectors"); }
    h->sv_bytes = bytes;
  }
  return DDA_OK;
}

int status_rank(int s) {          // larger = worse
  if (s < 0) return 100 - s;
  return s;                        // OK 0 < NOT_CONVERGED 1 < BREAKDOWN 2
}

}  // namespace
}  // namespace dda

using namespace dda;

int dda_solve_internal(dda_t h, const dda_solve_opts* o, int nrhs, const double* prop,
                       const double* pol, void* P_dev, double* hist, int hist_len,
                       dda_solve_info* info) {
  int rc = dda_beta_internal(h, o->pol, nrhs, prop, pol);
  if (rc != DDA_OK) return rc;
  if (o->prec == DDA_FP64 || !h->wdf.have_D) {   // FP64 products
    rc = ensure_d64(h);
    if (rc == DDA_OK) rc = ensure_work_cap<double>(h, h->w64, 1);
    if (rc != DDA_OK) return rc;
  }
  const long long n = 3 * h->g.n_occ;
  const bool refined = o->prec == DDA_FP32_REFINED;
  const int nvec = 10;
  const size_t bytes = refined ? (size_t)n * (nvec * sizeof(c64) + 5 * sizeof(c128))
                               : (size_t)n * (nvec + 1) * sizeof(c128);
  rc = ensure_solver_mem(h, bytes);
  if (rc != DDA_OK) return rc;
  Run ru;
  ru.h = h; ru.st = h->stream; ru.n = n;
  long long nb = (n + 4LL * kVT - 1) / (4LL * kVT);
  ru.nb = (int)(nb < 1 ? 1 : (nb > kNB ? kNB : nb));
  ru.part = h->d_part;
  ru.ds = (Scal*)h->d_scal;
  ru.hs = (Scal*)h->h_scal;
  const int rows_grid = (int)std::min<long long>((h->g.nrows + 7) / 8, 32LL * num_sms());
  int worst = DDA_OK;
  for (int r = 0; r < nrhs; ++r) {
    auto t0 = std::chrono::steady_clock::now();
    ru.rhs = r; ru.matvecs = 0; ru.matvecs64 = 0; ru.iters = 0;
    std::vector<double> hv;
    hv.push_back(1.0);
    ru.hist = &hv;
    ru.hist_scale = 1.0;
    Wave wv;
    for (int q = 0; q < 3; ++q) wv.a[q] = prop[3 * r + q];
    for (int q = 0; q < 6; ++q) wv.e[q] = pol[6 * r + q];
    const c128* beta64 = h->w64.beta + (long long)r * h->n_mat * 3;
    dda_solve_info& inf = info[r];
    inf = dda_solve_info{};
    int st_rhs = DDA_NOT_CONVERGED;
    double res_true = NAN, res_recur = NAN;
    int outer = 0;
    if (!refined) {
      c128* base = (c128*)h->sv;
      c128* vec[nvec];
      for (int i = 0; i < nvec; ++i) vec[i] = base + (size_t)i * n;
      c128* b = base + (size_t)nvec * n;   // b lives after the pool
      c128* x = vec[9];
      RK(launch_rhs(h, b, beta64, wv, ru.st));
      LK(h);
      RK(run_solver<double>(ru, o->solver, b, x, vec, o->tol, o->maxiter));
      st_rhs = ru.hs->status;
      res_recur = ru.hs->res;
      const double bn = ru.hs->bnorm;
      // true residual in FP64 (stop test at exit)
      c128* w = vec[0];
      c128* rr = vec[1];
      RK(matvec<double>(ru, x, w, false));
      k_resid<<<ru.nb, kVT, 0, ru.st>>>(b, w, rr, n, ru.part); count_launch();
      k_take_norm<<<1, kVT, 0, ru.st>>>(ru.ds, ru.part, ru.nb); count_launch();
      LK(h);
      RK(sync_read(ru));
      res_true = bn > 0 ? ru.hs->sres / bn : 0.0;
      if (st_rhs == DDA_OK && !(res_true < o->tol)) st_rhs = DDA_NOT_CONVERGED;
      k_pfinal<double><<<ru.nb, kVT, 0, ru.st>>>(x, (c128*)P_dev + (size_t)r * n, h->d_mat, beta64, h->g.n_occ); count_launch();
      LK(h);
    } else {
      c64* base = (c64*)h->sv;
      c64* vec[nvec];
      for (int i = 0; i < nvec; ++i) vec[i] = base + (size_t)i * n;
      c64* x32 = vec[9];
      c64* b32 = vec[8];
      c128* b64 = (c128*)(base + (size_t)nvec * n);
      c128* x64 = b64 + n;
      c128* r64 = x64 + n;
      c128* w64 = r64 + n;
      RK(launch_rhs(h, b64, beta64, wv, ru.st));
      k_norms<double><<<ru.nb, kVT, 0, ru.st>>>(b64, n, ru.part, nullptr); count_launch();
      k_take_norm<<<1, kVT, 0, ru.st>>>(ru.ds, ru.part, ru.nb); count_launch();
      k_copy<double><<<ru.nb, kVT, 0, ru.st>>>(b64, r64, n); count_launch();
      k_zero<double><<<ru.nb, kVT, 0, ru.st>>>(x64, n); count_launch();
      LK(h);
      RK(sync_read(ru));
      const double bn = ru.hs->sres;
      double rn = bn;
      int left = o->maxiter;
      st_rhs = bn > 0 ? DDA_NOT_CONVERGED : DDA_OK;
      res_true = bn > 0 ? 1.0 : 0.0;
      if (!std::isfinite(bn)) { st_rhs = DDA_ERR_NONFINITE; res_true = NAN; }  // NaN/Inf in b
      while (bn > 0 && std::isfinite(bn) && left > 0 && outer < 64) {
        if (rn / bn < o->tol) { st_rhs = DDA_OK; break; }
        const double target = std::max(o->inner_tol, 0.5 * o->tol * bn / rn);
        k_to32s<<<ru.nb, kVT, 0, ru.st>>>(r64, b32, n, 1.0 / rn); count_launch();
        LK(h);
        ru.hist_scale = rn / bn;
        const int it0 = ru.iters;
        ru.stall_window = 10;
        RK(run_solver<float>(ru, o->solver, b32, x32, vec, target, left));
        ru.stall_window = 0;
        const int inner_status = ru.hs->status;
        left -= ru.iters - it0;
        outer++;
        k_axpy64<<<ru.nb, kVT, 0, ru.st>>>(x64, x32, n, rn); count_launch();
        if (h->wdf.have_D) {       // residual product in double-float
          cudaError_t e = launch_matvec_df(h->g, h->lat(), h->wdf,
                                           h->w64.beta + (long long)r * h->n_mat * 3, h->n_mat,
                                           x64, w64, 1, ru.st);
          if (e != cudaSuccess) return dda_cuda_fail(h, e, "double-float residual product");
          ru.matvecs++;
          ru.matvecs64++;
        } else {
          RK(matvec<double>(ru, x64, w64, false));
        }
        k_resid<<<ru.nb, kVT, 0, ru.st>>>(b64, w64, r64, n, ru.part); count_launch();
        k_take_norm<<<1, kVT, 0, ru.st>>>(ru.ds, ru.part, ru.nb); count_launch();
        LK(h);
        RK(sync_read(ru));
        const double rn_new = ru.hs->sres;
        res_true = rn_new / bn;
        if (!std::isfinite(rn_new)) { st_rhs = DDA_ERR_NONFINITE; break; }
        if (res_true < o->tol) { st_rhs = DDA_OK; break; }
        if (inner_status == DDA_BREAKDOWN || inner_status == DDA_ERR_NONFINITE) { st_rhs = inner_status; break; }
        if (!(rn_new < 0.999 * rn)) { st_rhs = DDA_NOT_CONVERGED; break; }   // refinement stalled
        rn = rn_new;
      }
      res_recur = res_true;
      k_pfinal<double><<<ru.nb, kVT, 0, ru.st>>>(x64, (c128*)P_dev + (size_t)r * n, h->d_mat, beta64, h->g.n_occ); count_launch();
      LK(h);
    }
    DDA_CK(h, cudaStreamSynchronize(ru.st));
    tr_flush(&h->tracer);
    auto t1 = std::chrono::steady_clock::now();
    inf.status = st_rhs;
    inf.iters = ru.iters;
    inf.matvecs = ru.matvecs;
    inf.matvecs_fp64 = ru.matvecs64;
    inf.outer = outer;
    inf.rel_res_true = res_true;
    inf.rel_res_recur = res_recur;
    inf.seconds = std::chrono::duration<double>(t1 - t0).count();
    if (hist) {
      double* hr = hist + (size_t)r * hist_len;
      for (int i = 0; i < hist_len; ++i) hr[i] = i < (int)hv.size() ? hv[i] : -1.0;
    }
    if (status_rank(st_rhs) > status_rank(worst)) worst = st_rhs;
  }
  return worst;
}

// ---------------------------------------------------------------- true residual
namespace dda {
namespace {
// x = P / beta (Eq. (3)); a dipole with beta = 0 (m = 1, alpha = 0) has
// P = 0 and b = 0, and takes x = 0
__global__ void k_x_from_P(const c128* __restrict__ P, c128* __restrict__ x,
                           const uint8_t* __restrict__ mat, const c128* __restrict__ beta,
                           long long n_occ) {
  VLOOP(3 * n_occ) {
    const int c = (int)(i / n_occ);
    const long long j = i - c * n_occ;
    const c128 b = beta[mat[j] * 3 + c];
    const double d = b.x * b.x + b.y * b.y;
    const c128 p = P[i];
    x[i] = d > 0.0 ? mk<double>((p.x * b.x + p.y * b.y) / d, (p.y * b.x - p.x * b.y) / d)
                   : mk<double>(0.0, 0.0);
  }
}
}  // namespace
}  // namespace dda

int dda_residual_internal(dda_t h, int presc, int nrhs, const double* prop, const double* pol,
                          const void* P_dev, double* res) {
  int rc = dda_beta_internal(h, presc, nrhs, prop, pol);
  if (rc != DDA_OK) return rc;
  rc = ensure_d64(h);
  if (rc == DDA_OK) rc = ensure_work_cap<double>(h, h->w64, 1);
  if (rc != DDA_OK) return rc;
  const long long n = 3 * h->g.n_occ;
  rc = ensure_solver_mem(h, (size_t)n * 4 * sizeof(c128));
  if (rc != DDA_OK) return rc;
  Run ru;
  ru.h = h; ru.st = h->stream; ru.n = n;
  const long long nb = (n + 4LL * kVT - 1) / (4LL * kVT);
  ru.nb = (int)(nb < 1 ? 1 : (nb > kNB ? kNB : nb));
  ru.part = h->d_part;
  ru.ds = (Scal*)h->d_scal;
  ru.hs = (Scal*)h->h_scal;
  c128* x = (c128*)h->sv;
  c128* b = x + n;
  c128* w = b + n;
  c128* r = w + n;
  for (int k = 0; k < nrhs; ++k) {
    Wave wv;
    for (int q = 0; q < 3; ++q) wv.a[q] = prop[3 * k + q];
    for (int q = 0; q < 6; ++q) wv.e[q] = pol[6 * k + q];
    const c128* beta64 = h->w64.beta + (long long)k * h->n_mat * 3;
    RK(launch_rhs(h, b, beta64, wv, ru.st));
    k_x_from_P<<<ru.nb, kVT, 0, ru.st>>>((const c128*)P_dev + (size_t)k * n, x, h->d_mat, beta64,
                                         h->g.n_occ); count_launch();
    LK(h);
    k_norms<double><<<ru.nb, kVT, 0, ru.st>>>(b, n, ru.part, nullptr); count_launch();
    k_take_norm<<<1, kVT, 0, ru.st>>>(ru.ds, ru.part, ru.nb); count_launch();
    LK(h);
    RK(sync_read(ru));
    const double bn = ru.hs->sres;
    // the FP64 product of this right-hand side's beta table
    cudaError_t e = launch_matvec<double>(h->g, h->lat(), h->w64, beta64, h->n_mat, x, w, 1,
                                          false, ru.st);
    if (e != cudaSuccess) return dda_cuda_fail(h, e, "residual product");
    k_resid<<<ru.nb, kVT, 0, ru.st>>>(b, w, r, n, ru.part); count_launch();
    k_take_norm<<<1, kVT, 0, ru.st>>>(ru.ds, ru.part, ru.nb); count_launch();
    LK(h);
    RK(sync_read(ru));
    res[k] = bn > 0 ? ru.hs->sres / bn : 0.0;
  }
  return DDA_OK;
}

// ---------------------------------------------------------------- batched QMR-CS
// All right-hand sides of one particle advance together: every QMR step is
// one launch per product pass and per solver kernel for all of them (the
// right-hand side is the grid's y index), converged ones are skipped through
// a device mask, and the host reads the scalars every kSyncEvery steps only
// (a converged right-hand side's kernels are no-ops in between).
namespace dda {
namespace {

constexpr int kSyncEvery = 8;
// An inner solve with complex64 Krylov vectors gets at most this many steps
// per refinement step.  If it needs more (hard problems: thousands of
// iterations, where the complex64 Lanczos process loses its biorthogonality
// and convergence slows far below the FP64 rate), the following inner solves
// keep the Krylov vectors and scalars in complex128 with the double-float
// products (FP64-class accuracy at the FP32 pipe's cost; FP64 products where
// the grid has no double-float D-matrix): measured on the
// 128^3 sphere with m = 2, complex128 vectors with complex64 products still
// stall (1.5e-3 after 100,000 steps; the FP64 form needs 50,872), so the
// product's accuracy, not only the vectors', sets the rate.
constexpr int kC64InnerCap = 1000;
// the cap of a solve: dda_solve_opts.inner_cap when positive, else the default
int c64_inner_cap(const dda_solve_opts* o) { return o->inner_cap > 0 ? o->inner_cap : kC64InnerCap; }

// b32[r] = (complex64)(a64[r] * scl[r]) for right-hand sides with off[r] == 0
__global__ void k_to32s_b(const c128* __restrict__ a, c64* __restrict__ b, long long n,
                          const double* __restrict__ scl, const int* __restrict__ off) {
  const int rr = blockIdx.y;
  if (off[rr]) return;
  a += rr * n; b += rr * n;
  const double sc = scl[rr];
  VLOOP(n) b[i] = mk<float>((float)(a[i].x * sc), (float)(a[i].y * sc));
}
// x64[r] += scl[r] * d32[r]
__global__ void k_axpy64_b(c128* __restrict__ x, const c64* __restrict__ d, long long n,
                           const double* __restrict__ scl, const int* __restrict__ off) {
  const int rr = blockIdx.y;
  if (off[rr]) return;
  x += rr * n; d += rr * n;
  const double sc = scl[rr];
  VLOOP(n) x[i] = mk<double>(x[i].x + sc * (double)d[i].x, x[i].y + sc * (double)d[i].y);
}
// r = b - w with |r|^2 partials (slot 2) per right-hand side
__global__ void __launch_bounds__(kVT) k_resid_b(const c128* __restrict__ b, const c128* __restrict__ w,
                                                 c128* __restrict__ r, long long n, double* part,
                                                 const int* __restrict__ off) {
  const int rr = blockIdx.y;
  if (off && off[rr]) return;
  b += rr * n; w += rr * n; r += rr * n; part += rr * kPS;
  double acc[3] = {0.0, 0.0, 0.0};
  VLOOP(n) {
    const c128 t = b[i] - w[i];
    r[i] = t;
    acc[2] += t.x * t.x + t.y * t.y;
  }
  block_store<3>(acc, part, 0);
}
__global__ void k_take_norms_b(Scal* s, const double* part, int nb, const int* off) {
  const int rr = blockIdx.x;
  if (off && off[rr]) return;
  const double v = fin(part + rr * kPS, 2, nb);
  if (threadIdx.x == 0) s[rr].sres = sqrt(v);
}

// b[r] = a[r] * scl[r] (complex128)
__global__ void k_scale_b(const c128* __restrict__ a, c128* __restrict__ b, long long n,
                          const double* __restrict__ scl, const int* __restrict__ off) {
  const int rr = blockIdx.y;
  if (off[rr]) return;
  a += rr * n; b += rr * n;
  const double sc = scl[rr];
  VLOOP(n) b[i] = mk<double>(a[i].x * sc, a[i].y * sc);
}
// x64[r] += scl[r] * d64[r]
__global__ void k_axpy_b(c128* __restrict__ x, const c128* __restrict__ d, long long n,
                         const double* __restrict__ scl, const int* __restrict__ off) {
  const int rr = blockIdx.y;
  if (off[rr]) return;
  x += rr * n; d += rr * n;
  const double sc = scl[rr];
  VLOOP(n) x[i] = mk<double>(x[i].x + sc * d[i].x, x[i].y + sc * d[i].y);
}

// Device and pinned memory of one batched solve, grown on demand.
struct BatchMem {
  int cap = 0;
  Scal* ds = nullptr;        // [cap] scalars
  Scal* hs = nullptr;        // pinned mirror
  double* part = nullptr;    // [cap][kPS] partials
  double* mvpart = nullptr;  // [cap][2 * xinv blocks] product partials
  int* mask = nullptr;       // [cap] done flags (skip in the product)
  int* off = nullptr;        // [cap] right-hand sides left out of an inner solve
  double* dvals = nullptr;   // [2 cap]: tolerances, scales
  int* h_off = nullptr;      // pinned [cap]
  double* h_vals = nullptr;  // pinned [2 cap]
  void* sv = nullptr;        // solver vectors
  size_t sv_bytes = 0;
  void* sv2 = nullptr;       // vectors of the mixed inner solves (allocated on first use)
  size_t sv2_bytes = 0;
};

void bm_release(BatchMem* m, cudaStream_t st) {
  dev_free(m->ds, st); cudaFreeHost(m->hs); dev_free(m->part, st); dev_free(m->mvpart, st); dev_free(m->mask, st);
  dev_free(m->off, st); dev_free(m->dvals, st); cudaFreeHost(m->h_off); cudaFreeHost(m->h_vals);
  dev_free(m->sv, st);
  dev_free(m->sv2, st);
  *m = BatchMem();
}

int bm_ensure(dda_t h, int nrhs, size_t sv_bytes) {
  BatchMem* m = (BatchMem*)h->bm;
  if (!m) {
    m = new (std::nothrow) BatchMem();
    if (!m) return dda_fail(h, DDA_ERR_OOM, "batch state");
    h->bm = m;
  }
  if (m->cap < nrhs) {
    BatchMem fresh;
    fresh.sv = m->sv; fresh.sv_bytes = m->sv_bytes;
    fresh.sv2 = m->sv2; fresh.sv2_bytes = m->sv2_bytes;
    m->sv = nullptr; m->sv_bytes = 0;
    m->sv2 = nullptr; m->sv2_bytes = 0;
    bm_release(m, h->stream);
    *m = fresh;
    const size_t mvp = 2 * (size_t)fast_xinv_blocks_max(h->g.nrows) * nrhs;
    if (dev_malloc(&m->ds, nrhs * sizeof(Scal)) != cudaSuccess ||
        cudaMallocHost(&m->hs, nrhs * sizeof(Scal)) != cudaSuccess ||
        dev_malloc(&m->part, (size_t)nrhs * kPS * sizeof(double)) != cudaSuccess ||
        dev_malloc(&m->mvpart, mvp * sizeof(double)) != cudaSuccess ||
        dev_malloc(&m->mask, nrhs * sizeof(int)) != cudaSuccess ||
        dev_malloc(&m->off, nrhs * sizeof(int)) != cudaSuccess ||
        dev_malloc(&m->dvals, 2 * nrhs * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&m->h_off, nrhs * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&m->h_vals, 2 * nrhs * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      bm_release(m, h->stream);
      return dda_fail(h, DDA_ERR_OOM, "batched solver state");
    }
    m->cap = nrhs;
  }
  if (m->sv_bytes < sv_bytes) {
    dev_free(m->sv, h->stream);
    m->sv = nullptr; m->sv_bytes = 0;
    if (dev_malloc(&m->sv, sv_bytes) != cudaSuccess) {
      cudaGetLastError();
      return dda_fail(h, DDA_ERR_OOM, "batched solver vectors");
    }
    m->sv_bytes = sv_bytes;
  }
  return DDA_OK;
}

struct BRun {
  dda_t h;
  cudaStream_t st;
  long long n;
  int nb, nrhs;
  BatchMem* m;
  // inner-solve stagnation stop (complex64 only): per right-hand side best
  // residual and the step it was reached at
  bool stall = false;
  std::vector<double> best;
  std::vector<int> best_k;
};

int bsync(BRun& b) {
  DDA_CK(b.h, cudaMemcpyAsync(b.m->hs, b.m->ds, b.nrhs * sizeof(Scal), cudaMemcpyDeviceToHost, b.st));
  DDA_CK(b.h, cudaStreamSynchronize(b.st));
  return DDA_OK;
}

// Batched QMR-CS (same kernels and arithmetic as the single right-hand-side
// path) on b[nrhs][n] -> x; tol per right-hand side from m->dvals (or tol);
// right-hand sides with off[r] (device) start done.  Returns after every
// right-hand side is done or maxiter steps.
template <typename R>
int run_qmr_batched(BRun& b, const cpx<R>* rhs, cpx<R>* x, cpx<R>** vec, double tol,
                    const double* tols_dev, const int* off_dev, int maxiter, int* steps_out,
                    bool df_products = false, int resume_k = -1,
                    const std::function<int(int)>* on_sync = nullptr) {
  // resume_k >= 0: the vectors, x, the scalars and the skip mask hold a
  // saved state after resume_k steps; continue from there.  on_sync(k) runs
  // at every host synchronisation (every kSyncEvery steps): a negative
  // status aborts, 1 stops the solve after a checkpoint.
  // df_products (R = double): the products in double-float from the
  // double-float D-matrix (FP64-class accuracy), Krylov vectors and scalars in
  // complex128
  dda_t h = b.h;
  cudaStream_t st = b.st;
  const long long n = b.n;
  const int nb = b.nb, nr = b.nrhs;
  BatchMem* m = b.m;
  Scal* s = m->ds;
  double* part = m->part;
  cpx<R>*v = vec[0], *p = vec[1], *pt = vec[2], *d = vec[3], *sv = vec[4], *r = vec[5];
  const dim3 vg(nb, nr);
  if (resume_k < 0) {
    k_norms<R><<<vg, kVT, 0, st>>>(rhs, n, part, nullptr); count_launch();
    k_qmr_init<<<nr, kVT, 0, st>>>(s, part, nb, tol, tols_dev, off_dev, m->mask); count_launch();
    k_qmr_start<R><<<vg, kVT, 0, st>>>(rhs, v, p, r, x, d, sv, n, s); count_launch();
    LK(h);
  }
  RK(bsync(b));
  if (b.stall) {
    b.best.assign(nr, 1e300);
    b.best_k.assign(nr, 0);
  }
  Work<R>& w = work<R>(h);
  const cpx<R>* beta = w.beta;
  int k = resume_k > 0 ? resume_k : 0;
  bool active = false;
  for (int i = 0; i < nr; ++i) active = active || !m->hs[i].done;
  // Blocks of kSyncEvery steps after the first (which sets the kernels'
  // attributes) are captured once into a CUDA graph and replayed: every
  // argument of the block's launches is a device buffer or a value fixed for
  // the whole call, so one graph serves every block.  Not while tracing
  // (its events are host bookkeeping per launch).
  cudaGraphExec_t gexec = nullptr;
  long long glaunches = 0;
  bool graphs_ok = !(h->g.tr && h->g.tr->on);
  int blocks = 0;
  while (active && k < maxiter) {
    const bool full = k + kSyncEvery <= maxiter;
    if (graphs_ok && full && blocks >= 1 && !gexec) {
      // capture one block
      const long long l0 = launch_total();
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      int kk = k;
      if (ok) {
        for (int j = 0; j < kSyncEvery; ++j, ++kk) {
          int dnb = 0;
          cudaError_t e;
          if (df_products) {
            e = launch_matvec_df(h->g, h->lat(), h->wdf, h->w64.beta, h->n_mat, (const c128*)p,
                                 (c128*)pt, nr, st, m->mask);
          } else {
            e = launch_matvec<R>(h->g, h->lat(), w, beta, h->n_mat, p, pt, nr, false, st, m->mvpart,
                                 &dnb, m->mask);
          }
          if (e != cudaSuccess) { ok = false; break; }
          if (dnb > 0) {
            launch_pdl(true, k_qmr_a, dim3(nr), dim3(kVT), 0, st, s, (const double*)m->mvpart, 1LL, 2LL, 2LL * dnb, dnb, m->mask); count_launch();
          } else {
            k_dot<R, false><<<vg, kVT, 0, st>>>(p, pt, n, part, 0, s); count_launch();
            launch_pdl(true, k_qmr_a, dim3(nr), dim3(kVT), 0, st, s, (const double*)part, (long long)kNB, 1LL, (long long)kPS, nb, m->mask); count_launch();
          }
          launch_pdl(true, k_qmr_k1<R>, vg, dim3(kVT), 0, st, (const cpx<R>*)pt, v, n, s, part, m->mask); count_launch();
          launch_pdl(true, k_qmr_k2<R>, vg, dim3(kVT), 0, st, v, p, (const cpx<R>*)pt, d, sv, x, r, n, s, part, m->mask); count_launch();
        }
        const cudaError_t ec = cudaStreamEndCapture(st, &graph);
        ok = ok && ec == cudaSuccess && graph &&
             cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess;
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      glaunches = launch_total() - l0;
      if (!ok) {
        // the block was not launched: run it the ordinary way from now on
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        graphs_ok = false;
        count_launches(-glaunches);
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
          cudaGraph_t g2 = nullptr;
          cudaStreamEndCapture(st, &g2);
          if (g2) cudaGraphDestroy(g2);
        }
        cudaGetLastError();
      } else {
        count_launches(-glaunches);   // counted again as they run
      }
    }
    if (gexec && full) {
      DDA_CK(h, cudaGraphLaunch(gexec, st));
      count_launches(glaunches);
      k += kSyncEvery;
    }
    for (int j = 0; !(gexec && full) && j < kSyncEvery && k < maxiter; ++j, ++k) {
      int dnb = 0;
      cudaError_t e;
      if (df_products) {
        e = launch_matvec_df(h->g, h->lat(), h->wdf, h->w64.beta, h->n_mat, (const c128*)p,
                             (c128*)pt, nr, st, m->mask);
      } else {
        e = launch_matvec<R>(h->g, h->lat(), w, beta, h->n_mat, p, pt, nr, false, st, m->mvpart,
                             &dnb, m->mask);
      }
      if (e != cudaSuccess) return dda_cuda_fail(h, e, "batched product");
      Tracer* tr = h->g.tr;
      tr_begin(tr, st);
      if (dnb > 0) {
        launch_pdl(true, k_qmr_a, dim3(nr), dim3(kVT), 0, st, s, (const double*)m->mvpart, 1LL, 2LL, 2LL * dnb, dnb, m->mask); count_launch();
      } else {
        k_dot<R, false><<<vg, kVT, 0, st>>>(p, pt, n, part, 0, s); count_launch();
        launch_pdl(true, k_qmr_a, dim3(nr), dim3(kVT), 0, st, s, (const double*)part, (long long)kNB, 1LL, (long long)kPS, nb, m->mask); count_launch();
      }
      tr_end(tr, st, TR_QMR_SCALARS);
      tr_begin(tr, st);
      launch_pdl(true, k_qmr_k1<R>, vg, dim3(kVT), 0, st, (const cpx<R>*)pt, v, n, s, part, m->mask); count_launch();
      tr_end(tr, st, TR_QMR_K1);
      tr_begin(tr, st);
      launch_pdl(true, k_qmr_k2<R>, vg, dim3(kVT), 0, st, v, p, (const cpx<R>*)pt, d, sv, x, r, n, s, part, m->mask); count_launch();
      tr_end(tr, st, TR_QMR_K2);
      LK(h);
    }
    ++blocks;
    {
      const int rc = bsync(b);
      if (rc != DDA_OK) {
        if (gexec) cudaGraphExecDestroy(gexec);
        return rc;
      }
    }
    active = false;
    for (int i = 0; i < nr; ++i) {
      Scal& q = m->hs[i];
      if (q.done) continue;
      if (b.stall) {
        if (q.res < 0.99 * b.best[i]) {
          b.best[i] = q.res;
          b.best_k[i] = q.iters;
        } else if (q.res < 1e-4 && q.iters - b.best_k[i] >= 10) {
          // stagnated at the complex64 floor: end this inner solve
          const int one = 1;
          DDA_CK(h, cudaMemcpyAsync(&s[i].done, &one, sizeof(int), cudaMemcpyHostToDevice, st));
          DDA_CK(h, cudaMemcpyAsync(&m->mask[i], &one, sizeof(int), cudaMemcpyHostToDevice, st));
          DDA_CK(h, cudaStreamSynchronize(st));
          q.done = 1;
          continue;
        }
      }
      active = true;
    }
    if (on_sync && active) {
      const int rc = (*on_sync)(k);
      if (rc < 0) {
        if (gexec) cudaGraphExecDestroy(gexec);
        return rc;
      }
      if (rc == 1) break;
    }
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  *steps_out = k;
  return DDA_OK;
}

// ---------------------------------------------------------------- checkpoints
// Host image of a batched QMR-CS solve (dda_solve_opts.checkpoint_*): a
// header, the incidence of every right-hand side, then
//   FP64: the six QMR vectors, b and x ([8][nrhs][3 N_occ] complex128), the
//         device scalars of each right-hand side and the skip mask;
//   FP32_REFINED (saved between refinement steps): b, x, r ([3][nrhs][3 N_occ]
//         complex128) and the per-right-hand-side counters and norms.
struct CkptHead {
  char magic[8];
  int prec, nrhs, k, it_out, left, mixed;
  long long n;
  long long bytes;
};
constexpr char kCkptMagic[8] = {'D', 'D', 'A', 'C', 'K', 'P', 'T', '1'};

long long ckpt_bytes(int prec, int nrhs, long long n) {
  long long b = (long long)sizeof(CkptHead) + (long long)nrhs * 9 * sizeof(double);
  if (prec == DDA_FP64) b += 8LL * nrhs * n * (long long)sizeof(c128) + (long long)nrhs * (sizeof(Scal) + sizeof(int));
  else b += 3LL * nrhs * n * (long long)sizeof(c128) + (long long)nrhs * (5 * sizeof(int) + 3 * sizeof(double));
  return b;
}

// Sequential reader/writer over the caller's host buffer.
struct CkptCursor {
  unsigned char* p;
  long long at = 0;
  void put(const void* src, size_t nbytes) { std::memcpy(p + at, src, nbytes); at += (long long)nbytes; }
  void get(void* dst, size_t nbytes) { std::memcpy(dst, p + at, nbytes); at += (long long)nbytes; }
};

}  // namespace
}  // namespace dda

long long dda_checkpoint_bytes_internal(dda_t h, int prec, int nrhs) {
  return ckpt_bytes(prec, nrhs, 3 * h->g.n_occ);
}

void batch_free(dda_t h) {
  if (h && h->bm) {
    BatchMem* m = (BatchMem*)h->bm;
    bm_release(m, h->stream);
    delete m;
    h->bm = nullptr;
  }
}

int dda_solve_batch_internal(dda_t h, const dda_solve_opts* o, int nrhs, const double* prop,
                             const double* pol, void* P_dev, dda_solve_info* info) {
  auto t0 = std::chrono::steady_clock::now();
  int rc = dda_beta_internal(h, o->pol, nrhs, prop, pol);
  if (rc != DDA_OK) return rc;
  if (o->prec == DDA_FP64 || !h->wdf.have_D) {
    rc = ensure_d64(h);
    if (rc != DDA_OK) return rc;
  }
  const long long n = 3 * h->g.n_occ;
  const bool refined = o->prec == DDA_FP32_REFINED;
  const int nvec = 6;
  // complex64: the 6 QMR vectors, x32 and the inner right-hand side, then
  // b64, x64, r64, w64; FP64: the 6 QMR vectors, b64, x64
  const size_t bytes = refined ? (size_t)nrhs * n * ((nvec + 2) * sizeof(c64) + 4 * sizeof(c128))
                               : (size_t)nrhs * n * (nvec + 2) * sizeof(c128);
  rc = bm_ensure(h, nrhs, bytes);
  if (rc != DDA_OK) return rc;
  if (!refined || !h->wdf.have_D) {                // FP64 products
    rc = ensure_work_cap<double>(h, h->w64, nrhs);
    if (rc != DDA_OK) return rc;
  }
  if (refined) {
    rc = ensure_work_cap<float>(h, h->w32, nrhs);
    if (rc != DDA_OK) return rc;
    if (h->wdf.have_D) {
      rc = ensure_work_cap<df>(h, h->wdf, nrhs);
      if (rc != DDA_OK) return rc;
    }
  }
  BatchMem* m = (BatchMem*)h->bm;
  BRun b;
  b.h = h; b.st = h->stream; b.n = n; b.nrhs = nrhs; b.m = m;
  long long nbl = (n + 4LL * kVT - 1) / (4LL * kVT);
  b.nb = (int)(nbl < 1 ? 1 : (nbl > kNB ? kNB : nbl));
  const int rows_grid = (int)std::min<long long>((h->g.nrows + 7) / 8, 32LL * num_sms());
  cudaStream_t st = b.st;
  std::vector<int> status(nrhs, DDA_NOT_CONVERGED), iters(nrhs, 0), outer(nrhs, 0);
  std::vector<int> mv64(nrhs, 0);
  std::vector<double> res_true(nrhs, NAN), res_recur(nrhs, NAN);
  // b64 per right-hand side (FP64, Eq. (3))
  c128* b64;
  c128* x64;
  c128* r64 = nullptr;
  c128* w64;
  if (!refined) {
    c128* base = (c128*)m->sv;
    b64 = base + (size_t)nvec * nrhs * n;
    x64 = b64 + (size_t)nrhs * n;
    w64 = base;                                    // reused after the solve
  } else {
    c64* base = (c64*)m->sv;
    b64 = (c128*)(base + (size_t)(nvec + 2) * nrhs * n);
    x64 = b64 + (size_t)nrhs * n;
    r64 = x64 + (size_t)nrhs * n;
    w64 = r64 + (size_t)nrhs * n;
  }
  for (int r = 0; r < nrhs && !(o->resume && !refined); ++r) {
    Wave wv;
    for (int q = 0; q < 3; ++q) wv.a[q] = prop[3 * r + q];
    for (int q = 0; q < 6; ++q) wv.e[q] = pol[6 * r + q];
    RK(launch_rhs(h, b64 + (size_t)r * n, h->w64.beta + (long long)r * h->n_mat * 3, wv, st));
  }
  LK(h);
  const dim3 vg(b.nb, nrhs);
  std::vector<double> bn(nrhs, 0.0);
  // checkpoint image: header and incidences, checked on resume
  const long long ck_need = ckpt_bytes(o->prec, nrhs, n);
  CkptHead ck_head{};
  CkptCursor ck{(unsigned char*)o->checkpoint_host};
  if (o->resume) {
    ck.get(&ck_head, sizeof(ck_head));
    std::vector<double> inc((size_t)9 * nrhs);
    ck.get(inc.data(), inc.size() * sizeof(double));
    bool same = std::memcmp(ck_head.magic, kCkptMagic, 8) == 0 && ck_head.prec == o->prec &&
                ck_head.nrhs == nrhs && ck_head.n == n && ck_head.bytes == ck_need;
    for (int r = 0; same && r < nrhs; ++r)
      same = std::memcmp(inc.data() + 9 * r, prop + 3 * r, 3 * sizeof(double)) == 0 &&
             std::memcmp(inc.data() + 9 * r + 3, pol + 6 * r, 6 * sizeof(double)) == 0;
    if (!same)
      return dda_fail(h, DDA_ERR_ARG, "checkpoint does not match this handle, precision or incidence");
  }
  auto ck_begin = [&](int k, int it_out, int left, int mixed) {
    ck.at = 0;
    CkptHead hd{};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.prec = o->prec; hd.nrhs = nrhs; hd.k = k; hd.it_out = it_out; hd.left = left; hd.mixed = mixed;
    hd.n = n; hd.bytes = ck_need;
    ck.put(&hd, sizeof(hd));
    for (int r = 0; r < nrhs; ++r) {
      ck.put(prop + 3 * r, 3 * sizeof(double));
      ck.put(pol + 6 * r, 6 * sizeof(double));
    }
  };
  int ck_next = o->checkpoint_every > 0 ? o->checkpoint_every : 0;
  bool ck_stopped = false;
  if (!refined) {
    c128* base = (c128*)m->sv;
    c128* vec[nvec];
    for (int i = 0; i < nvec; ++i) vec[i] = base + (size_t)i * nrhs * n;
    int steps = 0;
    const size_t vbytes = (size_t)(nvec + 2) * nrhs * n * sizeof(c128);   // vectors, b, x
    int resume_k = -1;
    if (o->resume) {
      DDA_CK(h, cudaMemcpyAsync(base, ck.p + ck.at, vbytes, cudaMemcpyHostToDevice, st));
      ck.at += (long long)vbytes;
      DDA_CK(h, cudaMemcpyAsync(m->ds, ck.p + ck.at, nrhs * sizeof(Scal), cudaMemcpyHostToDevice, st));
      ck.at += (long long)(nrhs * sizeof(Scal));
      DDA_CK(h, cudaMemcpyAsync(m->mask, ck.p + ck.at, nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
      DDA_CK(h, cudaStreamSynchronize(st));
      resume_k = ck_head.k;
      while (ck_next > 0 && ck_next <= resume_k) ck_next += o->checkpoint_every;
    }
    std::function<int(int)> save = [&](int k) -> int {
      if (ck_next <= 0 || k < ck_next) return 0;
      while (ck_next <= k) ck_next += o->checkpoint_every;
      ck_begin(k, 0, 0, 0);
      DDA_CK(h, cudaMemcpyAsync(ck.p + ck.at, base, vbytes, cudaMemcpyDeviceToHost, st));
      ck.at += (long long)vbytes;
      DDA_CK(h, cudaMemcpyAsync(ck.p + ck.at, m->ds, nrhs * sizeof(Scal), cudaMemcpyDeviceToHost, st));
      ck.at += (long long)(nrhs * sizeof(Scal));
      DDA_CK(h, cudaMemcpyAsync(ck.p + ck.at, m->mask, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
      DDA_CK(h, cudaStreamSynchronize(st));
      if (o->checkpoint_stop) { ck_stopped = true; return 1; }
      return 0;
    };
    RK(run_qmr_batched<double>(b, b64, x64, vec, o->tol, nullptr, nullptr, o->maxiter, &steps, false,
                               resume_k, ck_next > 0 ? &save : nullptr));
    for (int r = 0; r < nrhs; ++r) {
      status[r] = m->hs[r].status;
      iters[r] = m->hs[r].iters;
      res_recur[r] = m->hs[r].res;
      bn[r] = m->hs[r].bnorm;
    }
    // true residuals in FP64, one batched product
    cudaError_t e = launch_matvec<double>(h->g, h->lat(), h->w64, h->w64.beta, h->n_mat, x64, w64,
                                          nrhs, false, st);
    if (e != cudaSuccess) return dda_cuda_fail(h, e, "batched product");
    k_resid_b<<<vg, kVT, 0, st>>>(b64, w64, base + (size_t)nrhs * n, n, m->part, nullptr); count_launch();
    k_take_norms_b<<<nrhs, kVT, 0, st>>>(m->ds, m->part, b.nb, nullptr); count_launch();
    LK(h);
    RK(bsync(b));
    for (int r = 0; r < nrhs; ++r) {
      res_true[r] = bn[r] > 0 ? m->hs[r].sres / bn[r] : 0.0;
      if (status[r] == DDA_OK && !(res_true[r] < o->tol)) status[r] = DDA_NOT_CONVERGED;
      mv64[r] = iters[r] + 1;
    }
  } else {
    c64* base = (c64*)m->sv;
    c64* vec[nvec];
    for (int i = 0; i < nvec; ++i) vec[i] = base + (size_t)i * nrhs * n;
    c64* x32 = base + (size_t)nvec * nrhs * n;
    c64* rhs32 = x32 + (size_t)nrhs * n;
    k_norms<double><<<vg, kVT, 0, st>>>(b64, n, m->part, nullptr); count_launch();
    k_take_norms_b<<<nrhs, kVT, 0, st>>>(m->ds, m->part, b.nb, nullptr); count_launch();
    k_copy<double><<<b.nb, kVT, 0, st>>>(b64, r64, (long long)nrhs * n); count_launch();
    k_zero<double><<<b.nb, kVT, 0, st>>>(x64, (long long)nrhs * n); count_launch();
    LK(h);
    RK(bsync(b));
    std::vector<double> rn(nrhs);
    std::vector<char> fin_(nrhs, 0);
    for (int r = 0; r < nrhs; ++r) {
      bn[r] = m->hs[r].sres;
      rn[r] = bn[r];
      if (!std::isfinite(bn[r])) { fin_[r] = 1; status[r] = DDA_ERR_NONFINITE; res_true[r] = NAN; }
      else if (!(bn[r] > 0)) { fin_[r] = 1; status[r] = DDA_OK; res_true[r] = 0.0; }
      else res_true[r] = 1.0;
    }
    int left = o->maxiter;
    b.stall = true;
    bool mixed = false;
    c128* mvec[nvec] = {};
    c128 *xm = nullptr, *rhsm = nullptr;
    // inner solves with complex128 Krylov vectors and FP64-class products
    auto make_mixed = [&]() -> int {
      const size_t need = (size_t)nrhs * n * (nvec + 2) * sizeof(c128);
      if (m->sv2_bytes < need) {
        dev_free(m->sv2, h->stream);
        m->sv2 = nullptr; m->sv2_bytes = 0;
        if (dev_malloc(&m->sv2, need) != cudaSuccess) {
          cudaGetLastError();
          return dda_fail(h, DDA_ERR_OOM, "mixed inner-solve vectors");
        }
        m->sv2_bytes = need;
      }
      c128* b2 = (c128*)m->sv2;
      for (int i = 0; i < nvec; ++i) mvec[i] = b2 + (size_t)i * nrhs * n;
      xm = b2 + (size_t)nvec * nrhs * n;
      rhsm = xm + (size_t)nrhs * n;
      mixed = true;
      return DDA_OK;
    };
    // the refinement state between outer steps: b, x, r on the device, the
    // per-right-hand-side counters and norms on the host
    const size_t sbytes = (size_t)3 * nrhs * n * sizeof(c128);
    std::vector<int> fin_i(nrhs);
    auto ck_ints = [&](bool save) {
      for (int r = 0; r < nrhs; ++r) fin_i[r] = fin_[r];
      int* arr[5] = {fin_i.data(), status.data(), iters.data(), outer.data(), mv64.data()};
      for (int* a : arr) {
        if (save) ck.put(a, nrhs * sizeof(int));
        else ck.get(a, nrhs * sizeof(int));
      }
      double* dar[3] = {rn.data(), bn.data(), res_true.data()};
      for (double* a : dar) {
        if (save) ck.put(a, nrhs * sizeof(double));
        else ck.get(a, nrhs * sizeof(double));
      }
      for (int r = 0; r < nrhs; ++r) fin_[r] = (char)fin_i[r];
    };
    int it_out0 = 0;
    if (o->resume) {
      DDA_CK(h, cudaMemcpyAsync(b64, ck.p + ck.at, sbytes, cudaMemcpyHostToDevice, st));
      ck.at += (long long)sbytes;
      DDA_CK(h, cudaStreamSynchronize(st));
      ck_ints(false);
      left = ck_head.left;
      it_out0 = ck_head.it_out;
      if (ck_head.mixed) RK(make_mixed());
      int kmax = 0;
      for (int r = 0; r < nrhs; ++r) kmax = std::max(kmax, iters[r]);
      while (ck_next > 0 && ck_next <= kmax) ck_next += o->checkpoint_every;
    }
    for (int it_out = it_out0; it_out < 64 && left > 0; ++it_out) {
      bool any = false;
      for (int r = 0; r < nrhs; ++r) {
        if (!fin_[r] && rn[r] / bn[r] < o->tol) { fin_[r] = 1; status[r] = DDA_OK; }
        m->h_off[r] = fin_[r];
        m->h_vals[r] = std::max(o->inner_tol, 0.5 * o->tol * bn[r] / rn[r]);   // inner targets
        m->h_vals[nrhs + r] = fin_[r] ? 0.0 : 1.0 / rn[r];                     // scales
        any = any || !fin_[r];
      }
      if (!any) break;
      DDA_CK(h, cudaMemcpyAsync(m->off, m->h_off, nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
      DDA_CK(h, cudaMemcpyAsync(m->dvals, m->h_vals, 2 * nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
      int steps = 0;
      bool capped = false;
      b.stall = !mixed;          // the stagnation stop is for the complex64 rounding floor
      if (!mixed) {
        k_to32s_b<<<vg, kVT, 0, st>>>(r64, rhs32, n, m->dvals + nrhs, m->off); count_launch();
        LK(h);
        const int cap = std::min(left, c64_inner_cap(o));
        RK(run_qmr_batched<float>(b, rhs32, x32, vec, 0.0, m->dvals, m->off, cap, &steps));
        capped = steps >= cap && cap < left;
      } else {
        k_scale_b<<<vg, kVT, 0, st>>>(r64, rhsm, n, m->dvals + nrhs, m->off); count_launch();
        LK(h);
        RK(run_qmr_batched<double>(b, rhsm, xm, mvec, 0.0, m->dvals, m->off, left, &steps,
                                   h->wdf.have_D));
      }
      left -= steps;
      for (int r = 0; r < nrhs; ++r) {
        if (fin_[r]) continue;
        iters[r] += m->hs[r].iters;
        outer[r] += 1;
        m->h_vals[nrhs + r] = rn[r];
      }
      DDA_CK(h, cudaMemcpyAsync(m->dvals + nrhs, m->h_vals + nrhs, nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
      std::vector<int> inner_status(nrhs);
      bool unfinished = false;
      for (int r = 0; r < nrhs; ++r) {
        inner_status[r] = m->hs[r].status;
        if (!fin_[r] && !m->hs[r].done) unfinished = true;
      }
      if (!mixed) {
        k_axpy64_b<<<vg, kVT, 0, st>>>(x64, x32, n, m->dvals + nrhs, m->off); count_launch();
      } else {
        k_axpy_b<<<vg, kVT, 0, st>>>(x64, xm, n, m->dvals + nrhs, m->off); count_launch();
      }
      cudaError_t e = h->wdf.have_D
          ? launch_matvec_df(h->g, h->lat(), h->wdf, h->w64.beta, h->n_mat, x64, w64, nrhs, st,
                             m->off)
          : launch_matvec<double>(h->g, h->lat(), h->w64, h->w64.beta, h->n_mat, x64, w64, nrhs,
                                  false, st, nullptr, nullptr, m->off);
      if (e != cudaSuccess) return dda_cuda_fail(h, e, "batched product");
      k_resid_b<<<vg, kVT, 0, st>>>(b64, w64, r64, n, m->part, m->off); count_launch();
      k_take_norms_b<<<nrhs, kVT, 0, st>>>(m->ds, m->part, b.nb, m->off); count_launch();
      LK(h);
      RK(bsync(b));
      for (int r = 0; r < nrhs; ++r) {
        if (fin_[r]) continue;
        mv64[r] += 1;
        const double rn_new = m->hs[r].sres;
        res_true[r] = rn_new / bn[r];
        if (!std::isfinite(rn_new)) { fin_[r] = 1; status[r] = DDA_ERR_NONFINITE; continue; }
        if (res_true[r] < o->tol) { fin_[r] = 1; status[r] = DDA_OK; continue; }
        if (inner_status[r] == DDA_BREAKDOWN || inner_status[r] == DDA_ERR_NONFINITE) {
          fin_[r] = 1; status[r] = inner_status[r]; continue;
        }
        if (!(rn_new < 0.999 * rn[r])) { fin_[r] = 1; status[r] = DDA_NOT_CONVERGED; continue; }
        rn[r] = rn_new;
      }
      if (!mixed && capped && unfinished) {
        // switch the remaining inner solves to complex128 Krylov vectors and
        // FP64-class products
        RK(make_mixed());
      }
      // checkpoint between refinement steps, at the first boundary after
      // every checkpoint_every inner iterations
      int kmax = 0;
      for (int r = 0; r < nrhs; ++r) kmax = std::max(kmax, iters[r]);
      if (ck_next > 0 && kmax >= ck_next) {
        while (ck_next <= kmax) ck_next += o->checkpoint_every;
        ck_begin(0, it_out + 1, left, mixed ? 1 : 0);
        DDA_CK(h, cudaMemcpyAsync(ck.p + ck.at, b64, sbytes, cudaMemcpyDeviceToHost, st));
        ck.at += (long long)sbytes;
        DDA_CK(h, cudaStreamSynchronize(st));
        ck_ints(true);
        if (o->checkpoint_stop) { ck_stopped = true; break; }
      }
    }
    for (int r = 0; r < nrhs; ++r) res_recur[r] = res_true[r];
  }
  for (int r = 0; r < nrhs; ++r) {
    k_pfinal<double><<<b.nb, kVT, 0, st>>>(x64 + (size_t)r * n, (c128*)P_dev + (size_t)r * n,
                                           h->d_mat, h->w64.beta + (long long)r * h->n_mat * 3,
                                           h->g.n_occ); count_launch();
  }
  LK(h);
  DDA_CK(h, cudaStreamSynchronize(st));
  tr_flush(&h->tracer);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = DDA_OK;
  for (int r = 0; r < nrhs; ++r) {
    dda_solve_info& inf = info[r];
    inf = dda_solve_info{};
    inf.status = status[r];
    inf.iters = iters[r];
    inf.matvecs = iters[r] + mv64[r];
    inf.matvecs_fp64 = refined ? mv64[r] : iters[r] + 1;
    if (!refined) inf.matvecs = iters[r] + 1;
    inf.outer = outer[r];
    inf.rel_res_true = res_true[r];
    inf.rel_res_recur = res_recur[r];
    inf.seconds = secs;
    if (status_rank(status[r]) > status_rank(worst)) worst = status[r];
  }
  return worst;
}
