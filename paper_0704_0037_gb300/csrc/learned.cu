// Learned right preconditioner: a small 3D convolutional network that maps a
// residual r of Eq. (3) to an approximation of the error A^-1 r, trained on
// (residual -> error) pairs the solver itself produces, and used inside a
// flexible Bi-CGSTAB whose residual is that of the exact product.  Sec. 4 of
// the paper traces the slow convergence for large m to the system itself and
// Sec. 5 names better preconditioning as the way forward; the paper trains
// nothing, so this whole file has no counterpart there.
//
// Network (1,033,430 parameters; BF16 weights in every product, FP32
// master copy, activations and accumulation):
//   features at half resolution s0 = ceil(n/2) per axis: the 2x2x2 average of
//   (Re, Im) of the three components of r / rms(r) and the occupied fraction
//   L0 conv3 7->16 relu [s0] -> pool2 -> L1 conv3 16->32 relu [s1]
//   -> pool2 -> L2 conv3 32->160 relu, L3 conv3 160->160 relu [s2]
//   -> up2, concat L1 -> L4 conv3 192->32 relu [s1]
//   -> up2, concat L0 -> L5 conv3 48->16 relu [s0] -> L6 conv1 16->6 [s0]
//   output: r plus the value of each dipole's half-resolution cell times
//   rms(r) (identity plus a learned correction: an untrained network with
//   its small last layer is close to no preconditioner at all).
// conv3 = 3x3x3, zero padding 1; pool2 = average of the existing children;
// up2 = nearest.  Loss: |N(r) - e|^2 / |e|^2 over the dipoles; Adam.
// Every reduction has a fixed order (per-block partials, then one block), so
// training and inference are deterministic.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "internal.h"

namespace dda {
namespace pc {

constexpr int NL = 7;
struct LayerSpec { int cin, cout, k, relu; };
constexpr LayerSpec kSpec[NL] = {{7, 16, 3, 1},   {16, 32, 3, 1},  {32, 160, 3, 1}, {160, 160, 3, 1},
                                 {192, 32, 3, 1}, {48, 16, 3, 1},  {16, 6, 1, 0}};
constexpr int kTX = 8, kTY = 8, kTZ = 4, kTV = kTX * kTY * kTZ;  // voxel tile of the conv kernels
constexpr int kCO = 8;                                           // output channels per block

struct Dims {
  int x, y, z;
  __host__ __device__ long long n() const { return (long long)x * y * z; }
};
inline Dims halved(Dims d) { return {(d.x + 1) / 2, (d.y + 1) / 2, (d.z + 1) / 2}; }

// ---------------------------------------------------------------- conv kernels
// out[co][v] = b[co] + sum_ci sum_k w[co][ci][k] in[ci][v + k - c]  (relu optional)
// grid (tiles, Cout / kCO); 256 threads, one voxel each, kCO accumulators
template <int K>
__global__ void __launch_bounds__(kTV) k_conv_fwd(const float* __restrict__ in, int cin,
                                                  const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias,
                                                  float* __restrict__ out, int cout, Dims d,
                                                  int relu) {
  constexpr int K3 = K * K * K, H = K / 2;
  constexpr int HX = kTX + 2 * H, HY = kTY + 2 * H, HZ = kTZ + 2 * H;
  __shared__ float s_in[HZ * HY * HX];
  __shared__ float s_w[kCO * K3];
  const int ntx = (d.x + kTX - 1) / kTX, nty = (d.y + kTY - 1) / kTY;
  const int tile = blockIdx.x;
  const int tx0 = (tile % ntx) * kTX, ty0 = ((tile / ntx) % nty) * kTY, tz0 = (tile / (ntx * nty)) * kTZ;
  const int co0 = blockIdx.y * kCO;
  const int lx = threadIdx.x % kTX, ly = (threadIdx.x / kTX) % kTY, lz = threadIdx.x / (kTX * kTY);
  const int x = tx0 + lx, y = ty0 + ly, z = tz0 + lz;
  const long long nv = d.n();
  float acc[kCO];
#pragma unroll
  for (int c = 0; c < kCO; ++c) acc[c] = (bias && co0 + c < cout) ? bias[co0 + c] : 0.0f;
  for (int ci = 0; ci < cin; ++ci) {
    __syncthreads();
    for (int k = threadIdx.x; k < HZ * HY * HX; k += kTV) {
      const int hx = k % HX, hy = (k / HX) % HY, hz = k / (HX * HY);
      const int gx = tx0 + hx - H, gy = ty0 + hy - H, gz = tz0 + hz - H;
      const bool ok = gx >= 0 && gy >= 0 && gz >= 0 && gx < d.x && gy < d.y && gz < d.z;
      s_in[k] = ok ? in[ci * nv + ((long long)gz * d.y + gy) * d.x + gx] : 0.0f;
    }
    for (int k = threadIdx.x; k < kCO * K3; k += kTV) {
      const int c = k / K3, t = k - c * K3;
      s_w[k] = co0 + c < cout ? __bfloat162float(w[((long long)(co0 + c) * cin + ci) * K3 + t]) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < K3; ++t) {
      const int kx = t % K, ky = (t / K) % K, kz = t / (K * K);
      const float v = s_in[((lz + kz) * HY + ly + ky) * HX + lx + kx];
#pragma unroll
      for (int c = 0; c < kCO; ++c) acc[c] = fmaf(s_w[c * K3 + t], v, acc[c]);
    }
  }
  if (x < d.x && y < d.y && z < d.z) {
    const long long v = ((long long)z * d.y + y) * d.x + x;
#pragma unroll
    for (int c = 0; c < kCO; ++c)
      if (co0 + c < cout) out[(co0 + c) * nv + v] = relu ? fmaxf(acc[c], 0.0f) : acc[c];
  }
}

// Partial weight gradients: part[chunk][co][ci][k] = sum over the voxels of
// this chunk's tiles of gout[co][v] in[ci][v + k - c]; grid (chunks, Cout /
// kCO, Cin), one thread per (co, k)
template <int K>
__global__ void __launch_bounds__(kCO * K * K * K) k_conv_wgrad(const float* __restrict__ in, int cin,
                                                               const float* __restrict__ gout,
                                                               int cout, Dims d,
                                                               float* __restrict__ part,
                                                               int tiles_per_chunk) {
  constexpr int K3 = K * K * K, H = K / 2, NT = kCO * K3;
  constexpr int HX = kTX + 2 * H, HY = kTY + 2 * H, HZ = kTZ + 2 * H;
  __shared__ float s_in[HZ * HY * HX];
  __shared__ float s_g[kCO * kTV];
  const int ntx = (d.x + kTX - 1) / kTX, nty = (d.y + kTY - 1) / kTY, ntz = (d.z + kTZ - 1) / kTZ;
  const int ntiles = ntx * nty * ntz;
  const int co0 = blockIdx.y * kCO, ci = blockIdx.z;
  const int c = threadIdx.x / K3, t = threadIdx.x - (threadIdx.x / K3) * K3;
  const int kx = t % K, ky = (t / K) % K, kz = t / (K * K);
  const long long nv = d.n();
  float acc = 0.0f;
  const int t0 = blockIdx.x * tiles_per_chunk, t1 = min(ntiles, t0 + tiles_per_chunk);
  for (int tile = t0; tile < t1; ++tile) {
    const int tx0 = (tile % ntx) * kTX, ty0 = ((tile / ntx) % nty) * kTY, tz0 = (tile / (ntx * nty)) * kTZ;
    __syncthreads();
    for (int k = threadIdx.x; k < HZ * HY * HX; k += NT) {
      const int hx = k % HX, hy = (k / HX) % HY, hz = k / (HX * HY);
      const int gx = tx0 + hx - H, gy = ty0 + hy - H, gz = tz0 + hz - H;
      const bool ok = gx >= 0 && gy >= 0 && gz >= 0 && gx < d.x && gy < d.y && gz < d.z;
      s_in[k] = ok ? in[ci * nv + ((long long)gz * d.y + gy) * d.x + gx] : 0.0f;
    }
    for (int k = threadIdx.x; k < kCO * kTV; k += NT) {
      const int cc = k / kTV, u = k - cc * kTV;
      const int gx = tx0 + u % kTX, gy = ty0 + (u / kTX) % kTY, gz = tz0 + u / (kTX * kTY);
      const bool ok = co0 + cc < cout && gx < d.x && gy < d.y && gz < d.z;
      s_g[k] = ok ? gout[(co0 + cc) * nv + ((long long)gz * d.y + gy) * d.x + gx] : 0.0f;
    }
    __syncthreads();
    for (int u = 0; u < kTV; ++u) {
      const int lx = u % kTX, ly = (u / kTX) % kTY, lz = u / (kTX * kTY);
      acc = fmaf(s_g[c * kTV + u], s_in[((lz + kz) * HY + ly + ky) * HX + lx + kx], acc);
    }
  }
  if (co0 + c < cout)
    part[(((long long)blockIdx.x * cout + co0 + c) * cin + ci) * K3 + t] = acc;
}

// g[i] += sum over chunks of part[chunk][i] (fixed order)
__global__ void k_sum_chunks(const float* __restrict__ part, int chunks, long long n,
                             float* __restrict__ g) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < chunks; ++c) s += part[c * n + i];
    g[i] += s;
  }
}

// gb[co] += sum_v gout[co][v]: one block per channel, fixed-order reduction
__global__ void k_bias_grad(const float* __restrict__ gout, long long nv, float* __restrict__ gb) {
  __shared__ float sh[256];
  float s = 0.0f;
  for (long long v = threadIdx.x; v < nv; v += 256) s += gout[blockIdx.x * nv + v];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) gb[blockIdx.x] += sh[0];
}

// wT[ci][co][K3-1-t] = w[co][ci][t] (the transposed, flipped kernel of the
// input gradient)
__global__ void k_wtrans(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt,
                         int cin, int cout, int K3) {
  const long long n = (long long)cin * cout * K3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i % K3);
    const long long r = i / K3;
    const int ci = (int)(r % cin), co = (int)(r / cin);
    wt[((long long)ci * cout + co) * K3 + (K3 - 1 - t)] = w[i];
  }
}

// g[c][v] *= (a[c][v] > 0)
__global__ void k_relu_mask(float* __restrict__ g, const float* __restrict__ a, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!(a[i] > 0.0f)) g[i] = 0.0f;
}

// ---------------------------------------------------------------- pooling
// out[c][p] = mean of in[c][children of p] (children inside the grid)
__global__ void k_pool2(const float* __restrict__ in, Dims di, float* __restrict__ out, Dims dout,
                        int ch) {
  const long long n = dout.n() * ch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / dout.n());
    const long long p = i - c * dout.n();
    const int X = (int)(p % dout.x), Y = (int)((p / dout.x) % dout.y), Z = (int)(p / ((long long)dout.x * dout.y));
    float s = 0.0f;
    int cnt = 0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
          if (x < di.x && y < di.y && z < di.z) {
            s += in[c * di.n() + ((long long)z * di.y + y) * di.x + x];
            ++cnt;
          }
        }
    out[i] = s / (float)cnt;
  }
}
// gin[c][v] += gout[c][parent(v)] / children(parent)
__global__ void k_pool2_back(const float* __restrict__ gout, Dims dout, float* __restrict__ gin,
                             Dims di, int ch) {
  const long long n = di.n() * ch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / di.n());
    const long long v = i - c * di.n();
    const int x = (int)(v % di.x), y = (int)((v / di.x) % di.y), z = (int)(v / ((long long)di.x * di.y));
    const int X = x / 2, Y = y / 2, Z = z / 2;
    const int cnt = (min(2, di.x - 2 * X)) * (min(2, di.y - 2 * Y)) * (min(2, di.z - 2 * Z));
    gin[i] += gout[c * dout.n() + ((long long)Z * dout.y + Y) * dout.x + X] / (float)cnt;
  }
}
// out[c][v] = in[c][parent(v)] (nearest)
__global__ void k_up2(const float* __restrict__ in, Dims dc, float* __restrict__ out, Dims df,
                      int ch) {
  const long long n = df.n() * ch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / df.n());
    const long long v = i - c * df.n();
    const int x = (int)(v % df.x), y = (int)((v / df.x) % df.y), z = (int)(v / ((long long)df.x * df.y));
    out[i] = in[c * dc.n() + ((long long)(z / 2) * dc.y + y / 2) * dc.x + x / 2];
  }
}
// gin[c][p] = sum of gout[c][children of p]
__global__ void k_up2_back(const float* __restrict__ gout, Dims df, float* __restrict__ gin,
                           Dims dc, int ch) {
  const long long n = dc.n() * ch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / dc.n());
    const long long p = i - c * dc.n();
    const int X = (int)(p % dc.x), Y = (int)((p / dc.x) % dc.y), Z = (int)(p / ((long long)dc.x * dc.y));
    float s = 0.0f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
          if (x < df.x && y < df.y && z < df.z) s += gout[c * df.n() + ((long long)z * df.y + y) * df.x + x];
        }
    gin[i] = s;
  }
}

// ---------------------------------------------------------------- lattice <-> grid
// map[(z ny + y) nx + x] = dipole index (or -1), one thread per dipole
__global__ void k_idx_map(LatticeDev lat, int nx, int ny, int nrows, int* __restrict__ map) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int row = warp; row < nrows; row += nwarps)
    for (long long i = lat.row_off[row] + lane; i < lat.row_off[row + 1]; i += 32)
      map[(long long)row * nx + lat.xi[i]] = (int)i;
}
// features at s0: channel 2c / 2c+1 = mean of Re / Im of v_c / rms over the
// cell's children (void children count as zero), channel 6 = occupied fraction
__global__ void k_feat_in(const c128* __restrict__ v, long long n_occ, const int* __restrict__ map,
                          Dims dl, Dims d0, const double* __restrict__ scl, float* __restrict__ f) {
  const double inv = scl[0] > 0.0 ? 1.0 / scl[0] : 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d0.n();
       p += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(p % d0.x), Y = (int)((p / d0.x) % d0.y), Z = (int)(p / ((long long)d0.x * d0.y));
    double acc[6] = {0, 0, 0, 0, 0, 0};
    int occ = 0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
          if (x >= dl.x || y >= dl.y || z >= dl.z) continue;
          const int i = map[((long long)z * dl.y + y) * dl.x + x];
          if (i < 0) continue;
          ++occ;
          for (int c = 0; c < 3; ++c) {
            const c128 a = v[c * n_occ + i];
            acc[2 * c] += a.x;
            acc[2 * c + 1] += a.y;
          }
        }
    for (int c = 0; c < 6; ++c) f[c * d0.n() + p] = (float)(acc[c] * inv * 0.125);
    f[6 * d0.n() + p] = occ * 0.125f;
  }
}
// z_i = v_i + rms * out6[.][cell(i)] for every dipole (complex128): the
// identity plus the learned correction
__global__ void k_feat_out(const float* __restrict__ o6, Dims d0, LatticeDev lat, int nx, int ny,
                           int nrows, long long n_occ, const double* __restrict__ scl,
                           const c128* __restrict__ v, c128* __restrict__ z) {
  const double s = scl[0];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int row = warp; row < nrows; row += nwarps) {
    const int y = row % ny, zz = row / ny;
    for (long long i = lat.row_off[row] + lane; i < lat.row_off[row + 1]; i += 32) {
      const long long p = ((long long)(zz / 2) * d0.y + y / 2) * d0.x + lat.xi[i] / 2;
      for (int c = 0; c < 3; ++c)
        z[c * n_occ + i] = v[c * n_occ + i] +
                           mk<double>(s * o6[(2 * c) * d0.n() + p], s * o6[(2 * c + 1) * d0.n() + p]);
    }
  }
}
// gradient of |z - e|^2 / |e|^2 with respect to out6 (z = rms * out6[cell]):
// g6[ch][p] = rms * sum over the cell's dipoles of 2 (z - e)_ch / |e|^2
__global__ void k_loss_grad(const c128* __restrict__ zz, const c128* __restrict__ e, long long n_occ,
                            const int* __restrict__ map, Dims dl, Dims d0,
                            const double* __restrict__ scl, float* __restrict__ g6) {
  const double s = scl[0], inv_e = scl[1] > 0.0 ? 1.0 / scl[1] : 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < d0.n();
       p += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(p % d0.x), Y = (int)((p / d0.x) % d0.y), Z = (int)(p / ((long long)d0.x * d0.y));
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
          if (x >= dl.x || y >= dl.y || z >= dl.z) continue;
          const int i = map[((long long)z * dl.y + y) * dl.x + x];
          if (i < 0) continue;
          for (int c = 0; c < 3; ++c) {
            const c128 d = zz[c * n_occ + i] - e[c * n_occ + i];
            acc[2 * c] += d.x;
            acc[2 * c + 1] += d.y;
          }
        }
    for (int c = 0; c < 6; ++c) g6[c * d0.n() + p] = (float)(2.0 * s * inv_e * acc[c]);
  }
}

// per-block partial sums of |a|^2 (slot 0) and |a - b|^2 (slot 1; b may be
// null), then one block adds them in order: out[0], out[1]
__global__ void k_sq_part(const c128* __restrict__ a, const c128* __restrict__ b, long long n,
                          double* __restrict__ part) {
  __shared__ double sh[2][256];
  double s0 = 0.0, s1 = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const c128 x = a[i];
    s0 += x.x * x.x + x.y * x.y;
    if (b) {
      const c128 d = x - b[i];
      s1 += d.x * d.x + d.y * d.y;
    }
  }
  sh[0][threadIdx.x] = s0;
  sh[1][threadIdx.x] = s1;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sh[0][0];
    part[2 * blockIdx.x + 1] = sh[1][0];
  }
}
__global__ void k_sq_fin(const double* __restrict__ part, int nb, double* __restrict__ out, int mode) {
  if (threadIdx.x != 0) return;
  double s0 = 0.0, s1 = 0.0;
  for (int b = 0; b < nb; ++b) { s0 += part[2 * b]; s1 += part[2 * b + 1]; }
  out[0] = s0;
  out[1] = s1;
  // mode 1: out[2] = rms = sqrt(s0 / n) is set by the caller's second launch
  (void)mode;
}
__global__ void k_rms(double* __restrict__ sc, long long n) {
  if (threadIdx.x == 0) sc[0] = n > 0 ? sqrt(sc[0] / (double)n) : 0.0;
}

// Adam (bias-corrected), then the BF16 copy used by the products
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                       float* __restrict__ m1, float* __restrict__ m2, long long n, float lr, float b1,
                       float b2, float c1, float c2, float eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float wi = w[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
  }
}
__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16(w[i]);
}

inline int gs(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)); }

}  // namespace pc
}  // namespace dda

using namespace dda;
using namespace dda::pc;

// The network and its working memory (grown to the largest lattice seen).
struct dda_pcnet {
  int device = 0;
  long long nparam = 0;
  long long woff[NL] = {}, boff[NL] = {};
  float* w = nullptr;           // FP32 master weights and biases
  __nv_bfloat16* wb = nullptr;  // BF16 copy (weights and biases; products use the weights)
  __nv_bfloat16* wt = nullptr;  // transposed, flipped kernels of the input gradients
  float* g = nullptr;           // gradients
  float* m1 = nullptr;
  float* m2 = nullptr;
  int step = 0;
  // activations and gradients
  void* arena = nullptr;
  size_t arena_bytes = 0;
  float* part = nullptr;        // weight-gradient partials
  size_t part_bytes = 0;
  int* map = nullptr;           // dipole index map of the current handle
  size_t map_bytes = 0;
  long long map_of = 0;         // uid of the handle the map was built for
  double* scal = nullptr;       // [0] rms(v), [1] |e|^2, [2..] scratch
  double* red = nullptr;        // reduction partials
  std::string err;
};

namespace {

int pc_fail(dda_pcnet_t n, int code, const std::string& m) {
  if (n) n->err = m;
  return code;
}

// Buffers of one forward/backward pass for lattice dims dl.
struct Acts {
  Dims d0, d1, d2;
  float *f0, *cat0, *a5, *o6, *p1, *cat1, *a4, *p2, *a2, *a3;
  float *g6, *ga5, *gcat0, *gcat1, *ga4, *ga3, *ga2, *gp2, *gp1;
};

size_t acts_floats(Dims d0, Dims d1, Dims d2) {
  return (size_t)d0.n() * (7 + 48 + 16 + 6 + 6 + 16 + 48) + (size_t)d1.n() * (16 + 192 + 32 + 192 + 32 + 16) +
         (size_t)d2.n() * (32 + 160 + 160 + 160 + 160 + 32);
}

int ensure_arena(dda_pcnet_t net, dda_t h, Acts& A) {
  const Dims dl{h->g.nx, h->g.ny, h->g.nz};
  A.d0 = halved(dl);
  A.d1 = halved(A.d0);
  A.d2 = halved(A.d1);
  const size_t need = acts_floats(A.d0, A.d1, A.d2) * sizeof(float) + 256;
  if (net->arena_bytes < need) {
    dev_free(net->arena, h->stream);
    net->arena = nullptr;
    net->arena_bytes = 0;
    if (dev_malloc(&net->arena, need) != cudaSuccess) {
      cudaGetLastError();
      return pc_fail(net, DDA_ERR_OOM, "network activations");
    }
    net->arena_bytes = need;
  }
  float* p = (float*)net->arena;
  auto take = [&](long long n) { float* r = p; p += n; return r; };
  A.f0 = take(7 * A.d0.n());
  A.cat0 = take(48 * A.d0.n());
  A.a5 = take(16 * A.d0.n());
  A.o6 = take(6 * A.d0.n());
  A.g6 = take(6 * A.d0.n());
  A.ga5 = take(16 * A.d0.n());
  A.gcat0 = take(48 * A.d0.n());
  A.p1 = take(16 * A.d1.n());
  A.cat1 = take(192 * A.d1.n());
  A.a4 = take(32 * A.d1.n());
  A.gcat1 = take(192 * A.d1.n());
  A.ga4 = take(32 * A.d1.n());
  A.gp1 = take(16 * A.d1.n());
  A.p2 = take(32 * A.d2.n());
  A.a2 = take(160 * A.d2.n());
  A.a3 = take(160 * A.d2.n());
  A.ga3 = take(160 * A.d2.n());
  A.ga2 = take(160 * A.d2.n());
  A.gp2 = take(32 * A.d2.n());
  // the dipole index map of this handle
  const long long nbox = (long long)dl.x * dl.y * dl.z;
  if (net->map_bytes < (size_t)nbox * sizeof(int)) {
    dev_free(net->map, h->stream);
    net->map = nullptr;
    net->map_bytes = 0;
    if (dev_malloc(&net->map, (size_t)nbox * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return pc_fail(net, DDA_ERR_OOM, "network index map");
    }
    net->map_bytes = (size_t)nbox * sizeof(int);
    net->map_of = 0;
  }
  if (net->map_of != h->uid) {
    if (cudaMemsetAsync(net->map, 0xff, (size_t)nbox * sizeof(int), h->stream) != cudaSuccess)
      return pc_fail(net, DDA_ERR_CUDA, "index map");
    k_idx_map<<<std::min(4096, (h->g.nrows + 7) / 8), 256, 0, h->stream>>>(h->lat(), h->g.nx, h->g.ny,
                                                                           h->g.nrows, net->map);
    count_launch();
    net->map_of = h->uid;
  }
  return DDA_OK;
}

void conv_fwd(dda_pcnet_t net, int L, const float* in, float* out, Dims d, cudaStream_t st) {
  const LayerSpec& s = kSpec[L];
  const int tiles = ((d.x + kTX - 1) / kTX) * ((d.y + kTY - 1) / kTY) * ((d.z + kTZ - 1) / kTZ);
  dim3 grid(tiles, (s.cout + kCO - 1) / kCO);
  if (s.k == 3)
    k_conv_fwd<3><<<grid, kTV, 0, st>>>(in, s.cin, net->wb + net->woff[L], net->w + net->boff[L], out,
                                        s.cout, d, s.relu);
  else
    k_conv_fwd<1><<<grid, kTV, 0, st>>>(in, s.cin, net->wb + net->woff[L], net->w + net->boff[L], out,
                                        s.cout, d, s.relu);
  count_launch();
}

// input gradient of layer L: gin = conv(gout, wT) (no bias, no relu)
void conv_bwd_data(dda_pcnet_t net, int L, const float* gout, float* gin, Dims d, cudaStream_t st) {
  const LayerSpec& s = kSpec[L];
  const int K3 = s.k * s.k * s.k;
  const long long nw = (long long)s.cin * s.cout * K3;
  k_wtrans<<<gs(nw), 256, 0, st>>>(net->wb + net->woff[L], net->wt, s.cin, s.cout, K3);
  count_launch();
  const int tiles = ((d.x + kTX - 1) / kTX) * ((d.y + kTY - 1) / kTY) * ((d.z + kTZ - 1) / kTZ);
  dim3 grid(tiles, (s.cin + kCO - 1) / kCO);
  if (s.k == 3)
    k_conv_fwd<3><<<grid, kTV, 0, st>>>(gout, s.cout, net->wt, nullptr, gin, s.cin, d, 0);
  else
    k_conv_fwd<1><<<grid, kTV, 0, st>>>(gout, s.cout, net->wt, nullptr, gin, s.cin, d, 0);
  count_launch();
}

int conv_bwd_weight(dda_pcnet_t net, int L, const float* in, const float* gout, Dims d,
                    cudaStream_t st) {
  const LayerSpec& s = kSpec[L];
  const int K3 = s.k * s.k * s.k;
  const int tiles = ((d.x + kTX - 1) / kTX) * ((d.y + kTY - 1) / kTY) * ((d.z + kTZ - 1) / kTZ);
  const int chunks = std::max(1, std::min(tiles, 16));
  const int per = (tiles + chunks - 1) / chunks;
  const long long nw = (long long)s.cout * s.cin * K3;
  const size_t need = (size_t)chunks * nw * sizeof(float);
  if (net->part_bytes < need) {
    dev_free(net->part, st);
    net->part = nullptr;
    net->part_bytes = 0;
    if (dev_malloc(&net->part, need) != cudaSuccess) {
      cudaGetLastError();
      return pc_fail(net, DDA_ERR_OOM, "weight-gradient partials");
    }
    net->part_bytes = need;
  }
  dim3 grid(chunks, (s.cout + kCO - 1) / kCO, s.cin);
  if (s.k == 3)
    k_conv_wgrad<3><<<grid, kCO * 27, 0, st>>>(in, s.cin, gout, s.cout, d, net->part, per);
  else
    k_conv_wgrad<1><<<grid, kCO, 0, st>>>(in, s.cin, gout, s.cout, d, net->part, per);
  count_launch();
  k_sum_chunks<<<gs(nw), 256, 0, st>>>(net->part, chunks, nw, net->g + net->woff[L]);
  count_launch();
  k_bias_grad<<<s.cout, 256, 0, st>>>(gout, d.n(), net->g + net->boff[L]);
  count_launch();
  return DDA_OK;
}

// z = N(v) on the handle's lattice (v, z complex128 [3][N_occ]); leaves the
// activations in A for a backward pass
int forward(dda_pcnet_t net, dda_t h, const c128* v, c128* z, Acts& A) {
  cudaStream_t st = h->stream;
  const long long n = 3 * h->g.n_occ;
  const Dims dl{h->g.nx, h->g.ny, h->g.nz};
  // rms(v)
  const int nb = 256;
  k_sq_part<<<nb, 256, 0, st>>>(v, nullptr, n, net->red);
  count_launch();
  k_sq_fin<<<1, 32, 0, st>>>(net->red, nb, net->scal, 0);
  count_launch();
  k_rms<<<1, 32, 0, st>>>(net->scal, n);
  count_launch();
  k_feat_in<<<gs(A.d0.n()), 256, 0, st>>>(v, h->g.n_occ, net->map, dl, A.d0, net->scal, A.f0);
  count_launch();
  float* a0 = A.cat0 + 32 * A.d0.n();
  float* a1 = A.cat1 + 160 * A.d1.n();
  conv_fwd(net, 0, A.f0, a0, A.d0, st);
  k_pool2<<<gs(16 * A.d1.n()), 256, 0, st>>>(a0, A.d0, A.p1, A.d1, 16); count_launch();
  conv_fwd(net, 1, A.p1, a1, A.d1, st);
  k_pool2<<<gs(32 * A.d2.n()), 256, 0, st>>>(a1, A.d1, A.p2, A.d2, 32); count_launch();
  conv_fwd(net, 2, A.p2, A.a2, A.d2, st);
  conv_fwd(net, 3, A.a2, A.a3, A.d2, st);
  k_up2<<<gs(160 * A.d1.n()), 256, 0, st>>>(A.a3, A.d2, A.cat1, A.d1, 160); count_launch();
  conv_fwd(net, 4, A.cat1, A.a4, A.d1, st);
  k_up2<<<gs(32 * A.d0.n()), 256, 0, st>>>(A.a4, A.d1, A.cat0, A.d0, 32); count_launch();
  conv_fwd(net, 5, A.cat0, A.a5, A.d0, st);
  conv_fwd(net, 6, A.a5, A.o6, A.d0, st);
  k_feat_out<<<std::min(4096, (h->g.nrows + 7) / 8), 256, 0, st>>>(A.o6, A.d0, h->lat(), h->g.nx, h->g.ny,
                                                                  h->g.nrows, h->g.n_occ, net->scal, v, z);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DDA_OK : pc_fail(net, DDA_ERR_CUDA, cudaGetErrorString(e));
}

int backward(dda_pcnet_t net, dda_t h, const c128* z, const c128* e, Acts& A) {
  cudaStream_t st = h->stream;
  const Dims dl{h->g.nx, h->g.ny, h->g.nz};
  float* a0 = A.cat0 + 32 * A.d0.n();
  float* a1 = A.cat1 + 160 * A.d1.n();
  float* ga0 = A.gcat0 + 32 * A.d0.n();
  float* ga1 = A.gcat1 + 160 * A.d1.n();
  k_loss_grad<<<gs(A.d0.n()), 256, 0, st>>>(z, e, h->g.n_occ, net->map, dl, A.d0, net->scal, A.g6);
  count_launch();
  int rc;
  // L6 (conv1, linear)
  if ((rc = conv_bwd_weight(net, 6, A.a5, A.g6, A.d0, st)) != DDA_OK) return rc;
  conv_bwd_data(net, 6, A.g6, A.ga5, A.d0, st);
  k_relu_mask<<<gs(16 * A.d0.n()), 256, 0, st>>>(A.ga5, A.a5, 16 * A.d0.n()); count_launch();
  // L5
  if ((rc = conv_bwd_weight(net, 5, A.cat0, A.ga5, A.d0, st)) != DDA_OK) return rc;
  conv_bwd_data(net, 5, A.ga5, A.gcat0, A.d0, st);
  // up2 back to L4's output
  k_up2_back<<<gs(32 * A.d1.n()), 256, 0, st>>>(A.gcat0, A.d0, A.ga4, A.d1, 32); count_launch();
  k_relu_mask<<<gs(32 * A.d1.n()), 256, 0, st>>>(A.ga4, A.a4, 32 * A.d1.n()); count_launch();
  // L4
  if ((rc = conv_bwd_weight(net, 4, A.cat1, A.ga4, A.d1, st)) != DDA_OK) return rc;
  conv_bwd_data(net, 4, A.ga4, A.gcat1, A.d1, st);
  k_up2_back<<<gs(160 * A.d2.n()), 256, 0, st>>>(A.gcat1, A.d1, A.ga3, A.d2, 160); count_launch();
  k_relu_mask<<<gs(160 * A.d2.n()), 256, 0, st>>>(A.ga3, A.a3, 160 * A.d2.n()); count_launch();
  // L3
  if ((rc = conv_bwd_weight(net, 3, A.a2, A.ga3, A.d2, st)) != DDA_OK) return rc;
  conv_bwd_data(net, 3, A.ga3, A.ga2, A.d2, st);
  k_relu_mask<<<gs(160 * A.d2.n()), 256, 0, st>>>(A.ga2, A.a2, 160 * A.d2.n()); count_launch();
  // L2
  if ((rc = conv_bwd_weight(net, 2, A.p2, A.ga2, A.d2, st)) != DDA_OK) return rc;
  conv_bwd_data(net, 2, A.ga2, A.gp2, A.d2, st);
  // pool back into L1's output (skip gradient already in gcat1[160..])
  k_pool2_back<<<gs(32 * A.d1.n()), 256, 0, st>>>(A.gp2, A.d2, ga1, A.d1, 32); count_launch();
  k_relu_mask<<<gs(32 * A.d1.n()), 256, 0, st>>>(ga1, a1, 32 * A.d1.n()); count_launch();
  // L1
  if ((rc = conv_bwd_weight(net, 1, A.p1, ga1, A.d1, st)) != DDA_OK) return rc;
  conv_bwd_data(net, 1, ga1, A.gp1, A.d1, st);
  k_pool2_back<<<gs(16 * A.d0.n()), 256, 0, st>>>(A.gp1, A.d1, ga0, A.d0, 16); count_launch();
  k_relu_mask<<<gs(16 * A.d0.n()), 256, 0, st>>>(ga0, a0, 16 * A.d0.n()); count_launch();
  // L0 (no input gradient)
  if ((rc = conv_bwd_weight(net, 0, A.f0, ga0, A.d0, st)) != DDA_OK) return rc;
  const cudaError_t er = cudaGetLastError();
  return er == cudaSuccess ? DDA_OK : pc_fail(net, DDA_ERR_CUDA, cudaGetErrorString(er));
}

bool pc_device_ok(dda_pcnet_t net, dda_t h) { return net->device == h->device; }

}  // namespace

// ---------------------------------------------------------------- C-ABI
extern "C" int dda_pcnet_create(dda_pcnet_t* out, unsigned long long seed) {
  if (!out) return DDA_ERR_ARG;
  *out = nullptr;
  dda_pcnet* net = new (std::nothrow) dda_pcnet();
  if (!net) return DDA_ERR_OOM;
  if (cudaGetDevice(&net->device) != cudaSuccess) {
    cudaGetLastError();
    delete net;
    return DDA_ERR_CUDA;
  }
  long long off = 0;
  for (int L = 0; L < NL; ++L) {
    net->woff[L] = off;
    off += (long long)kSpec[L].cout * kSpec[L].cin * kSpec[L].k * kSpec[L].k * kSpec[L].k;
    net->boff[L] = off;
    off += kSpec[L].cout;
  }
  net->nparam = off;
  size_t wtmax = 0;
  for (int L = 0; L < NL; ++L)
    wtmax = std::max(wtmax, (size_t)kSpec[L].cout * kSpec[L].cin * kSpec[L].k * kSpec[L].k * kSpec[L].k);
  // He-normal weights from a seeded host generator, zero biases; the last
  // layer starts small so that the untrained network is close to zero
  std::vector<float> hw((size_t)off, 0.0f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.0f, 1.0f);
  for (int L = 0; L < NL; ++L) {
    const int fan = kSpec[L].cin * kSpec[L].k * kSpec[L].k * kSpec[L].k;
    const float sd = std::sqrt(2.0f / fan) * (L == NL - 1 ? 0.1f : 1.0f);
    for (long long i = net->woff[L]; i < net->boff[L]; ++i) hw[i] = sd * nd(rng);
  }
  int rc = DDA_OK;
  if (dev_malloc(&net->w, off * sizeof(float)) != cudaSuccess ||
      dev_malloc(&net->wb, off * sizeof(__nv_bfloat16)) != cudaSuccess ||
      dev_malloc(&net->wt, wtmax * sizeof(__nv_bfloat16)) != cudaSuccess ||
      dev_malloc(&net->g, off * sizeof(float)) != cudaSuccess ||
      dev_malloc(&net->m1, off * sizeof(float)) != cudaSuccess ||
      dev_malloc(&net->m2, off * sizeof(float)) != cudaSuccess ||
      dev_malloc(&net->scal, 8 * sizeof(double)) != cudaSuccess ||
      dev_malloc(&net->red, 2 * 256 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rc = DDA_ERR_OOM;
  } else if (cudaMemcpy(net->w, hw.data(), off * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(net->m1, 0, off * sizeof(float)) != cudaSuccess ||
             cudaMemset(net->m2, 0, off * sizeof(float)) != cudaSuccess ||
             cudaMemset(net->scal, 0, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    rc = DDA_ERR_CUDA;
  } else {
    k_to_bf16<<<gs(off), 256>>>(net->w, net->wb, off);
    count_launch();
    if (cudaDeviceSynchronize() != cudaSuccess) { cudaGetLastError(); rc = DDA_ERR_CUDA; }
  }
  if (rc != DDA_OK) {
    dda_pcnet_free(net);
    return rc;
  }
  *out = net;
  return DDA_OK;
}

extern "C" int dda_pcnet_free(dda_pcnet_t net) {
  if (!net) return DDA_OK;
  DeviceGuard dg(net->device);
  cudaDeviceSynchronize();
  dev_free(net->w, 0); dev_free(net->wb, 0); dev_free(net->wt, 0); dev_free(net->g, 0);
  dev_free(net->m1, 0); dev_free(net->m2, 0); dev_free(net->arena, 0); dev_free(net->part, 0);
  dev_free(net->map, 0); dev_free(net->scal, 0); dev_free(net->red, 0);
  cudaGetLastError();
  delete net;
  return DDA_OK;
}

extern "C" int dda_pcnet_params(dda_pcnet_t net, long long* n) {
  if (!net || !n) return DDA_ERR_ARG;
  *n = net->nparam;
  return DDA_OK;
}

extern "C" const char* dda_pcnet_last_error(dda_pcnet_t net) { return net ? net->err.c_str() : "null network"; }

extern "C" int dda_pcnet_get_weights(dda_pcnet_t net, float* host) {
  if (!net || !host) return DDA_ERR_ARG;
  DeviceGuard dg(net->device);
  if (cudaMemcpy(host, net->w, net->nparam * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return pc_fail(net, DDA_ERR_CUDA, "weights to host");
  }
  return DDA_OK;
}

extern "C" int dda_pcnet_set_weights(dda_pcnet_t net, const float* host) {
  if (!net || !host) return DDA_ERR_ARG;
  DeviceGuard dg(net->device);
  if (cudaMemcpy(net->w, host, net->nparam * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return pc_fail(net, DDA_ERR_CUDA, "weights from host");
  }
  k_to_bf16<<<gs(net->nparam), 256>>>(net->w, net->wb, net->nparam);
  count_launch();
  cudaMemset(net->m1, 0, net->nparam * sizeof(float));
  cudaMemset(net->m2, 0, net->nparam * sizeof(float));
  net->step = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return pc_fail(net, DDA_ERR_CUDA, "bf16 copy");
  }
  return DDA_OK;
}

extern "C" int dda_pcnet_apply(dda_pcnet_t net, dda_t h, const void* v_dev, void* z_dev) {
  if (!net || !h || !v_dev || !z_dev) return DDA_ERR_ARG;
  if (!pc_device_ok(net, h)) return pc_fail(net, DDA_ERR_ARG, "network and handle on different devices");
  DDA_ON_DEVICE(h);
  Acts A;
  int rc = ensure_arena(net, h, A);
  if (rc == DDA_OK) rc = forward(net, h, (const c128*)v_dev, (c128*)z_dev, A);
  return rc;
}

// One Adam step on the pair (r, e): loss |N(r) - e|^2 / |e|^2; z_dev receives
// N(r) before the step; loss_out (host) the loss.
extern "C" int dda_pcnet_train_step(dda_pcnet_t net, dda_t h, const void* r_dev, const void* e_dev,
                                    void* z_dev, float lr, double* loss_out) {
  if (!net || !h || !r_dev || !e_dev || !z_dev || !(lr > 0.0f)) return DDA_ERR_ARG;
  if (!pc_device_ok(net, h)) return pc_fail(net, DDA_ERR_ARG, "network and handle on different devices");
  DDA_ON_DEVICE(h);
  cudaStream_t st = h->stream;
  Acts A;
  int rc = ensure_arena(net, h, A);
  if (rc != DDA_OK) return rc;
  const c128* r = (const c128*)r_dev;
  const c128* e = (const c128*)e_dev;
  c128* z = (c128*)z_dev;
  if ((rc = forward(net, h, r, z, A)) != DDA_OK) return rc;
  // |e|^2 into scal[1] (scal[0] keeps rms(r)), |z - e|^2 into scal[2]
  const long long n = 3 * h->g.n_occ;
  k_sq_part<<<256, 256, 0, st>>>(e, z, n, net->red);
  count_launch();
  k_sq_fin<<<1, 32, 0, st>>>(net->red, 256, net->scal + 3, 0);   // scal[3] = |e|^2, scal[4] = |e - z|^2
  count_launch();
  if (cudaMemcpyAsync(net->scal + 1, net->scal + 3, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return pc_fail(net, DDA_ERR_CUDA, "loss scalars");
  if (cudaMemsetAsync(net->g, 0, net->nparam * sizeof(float), st) != cudaSuccess)
    return pc_fail(net, DDA_ERR_CUDA, "gradient reset");
  if ((rc = backward(net, h, z, e, A)) != DDA_OK) return rc;
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)net->step), c2 = 1.0f - std::pow(b2, (float)net->step);
  k_adam<<<gs(net->nparam), 256, 0, st>>>(net->w, net->wb, net->g, net->m1, net->m2, net->nparam, lr,
                                         b1, b2, c1, c2, 1e-8f);
  count_launch();
  double hs[2];
  if (cudaMemcpyAsync(hs, net->scal + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return pc_fail(net, DDA_ERR_CUDA, "loss readback");
  }
  if (loss_out) *loss_out = hs[0] > 0.0 ? hs[1] / hs[0] : 0.0;
  return std::isfinite(hs[1]) ? DDA_OK : pc_fail(net, DDA_ERR_NONFINITE, "non-finite loss");
}

// Gradients of the last train step (host, nparam floats): for tests.
extern "C" int dda_pcnet_get_grads(dda_pcnet_t net, float* host) {
  if (!net || !host) return DDA_ERR_ARG;
  DeviceGuard dg(net->device);
  if (cudaMemcpy(host, net->g, net->nparam * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return pc_fail(net, DDA_ERR_CUDA, "gradients to host");
  }
  return DDA_OK;
}

// ---------------------------------------------------------------- flexible Bi-CGSTAB
// Right-preconditioned Bi-CGSTAB whose preconditioner may change from one
// application to the next (the network): with p^ = N(p), s^ = N(s),
//   v = A p^, alpha = rho / (r0, v), s = r - alpha v, t = A s^,
//   omega = (t, s) / (t, t), x += alpha p^ + omega s^, r = s - omega t.
// Hermitian products (Sec. 2's Bi-CGSTAB), complex128 vectors, the exact
// product (double-float where the handle has the double-float D-matrix, else
// FP64).  Convergence is declared on the true residual b - A x.  When the
// preconditioned iteration stalls (its residual has not improved by 1 % in
// 50 iterations) or breaks down, the solve continues from the current x
// without the network: the plain solver is the fallback.
namespace dda {
namespace pc {

// per-block partials of (a, b) = sum conj(a) b for up to three pairs
__global__ void k_hdot3(const c128* __restrict__ a0, const c128* __restrict__ b0,
                        const c128* __restrict__ a1, const c128* __restrict__ b1,
                        const c128* __restrict__ a2, const c128* __restrict__ b2, long long n,
                        double* __restrict__ part) {
  __shared__ double sh[6][256];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const c128* as[3] = {a0, a1, a2};
    const c128* bs[3] = {b0, b1, b2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (!as[k]) continue;
      const c128 x = as[k][i], y = bs[k][i];
      acc[2 * k] += x.x * y.x + x.y * y.y;
      acc[2 * k + 1] += x.x * y.y - x.y * y.x;
    }
  }
  for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) part[6 * blockIdx.x + k] = sh[k][0];
}
__global__ void k_hdot_fin(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 6; ++k) s[k] += part[6 * b + k];
  for (int k = 0; k < 6; ++k) out[k] = s[k];
}
// y = a x + b y + c z (complex scalars; z may be null)
__global__ void k_axpbypcz(c128 a, const c128* __restrict__ x, c128 b, c128* __restrict__ y, c128 c,
                           const c128* __restrict__ z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    c128 r = a * x[i] + b * y[i];
    if (z) r = r + c * z[i];
    y[i] = r;
  }
}
// P = beta x (Eq. (3))
__global__ void k_p_from_x(const c128* __restrict__ x, c128* __restrict__ P, const uint8_t* __restrict__ mat,
                           const c128* __restrict__ beta, long long n_occ) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * n_occ;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / n_occ);
    P[i] = beta[mat[i - c * n_occ] * 3 + c] * x[i];
  }
}

}  // namespace pc
}  // namespace dda

namespace {

struct PcRun {
  dda_t h;
  cudaStream_t st;
  long long n;
  bool df;
  double* part;
  double* out;     // device [6]
  double* hout;    // host [6]
};

int pc_matvec(PcRun& R, const c128* x, c128* y) {
  dda_t h = R.h;
  const cudaError_t e = R.df ? launch_matvec_df(h->g, h->lat(), h->wdf, h->w64.beta, h->n_mat, x, y, 1, R.st)
                             : launch_matvec<double>(h->g, h->lat(), h->w64, h->w64.beta, h->n_mat, x, y, 1,
                                                     false, R.st);
  return e == cudaSuccess ? DDA_OK : dda_cuda_fail(h, e, "product");
}

// up to three Hermitian products, read back to R.hout as (re, im) pairs
int pc_dots(PcRun& R, const c128* a0, const c128* b0, const c128* a1 = nullptr, const c128* b1 = nullptr,
            const c128* a2 = nullptr, const c128* b2 = nullptr) {
  k_hdot3<<<256, 256, 0, R.st>>>(a0, b0, a1, b1, a2, b2, R.n, R.part);
  count_launch();
  k_hdot_fin<<<1, 32, 0, R.st>>>(R.part, 256, R.out);
  count_launch();
  DDA_CK(R.h, cudaMemcpyAsync(R.hout, R.out, 6 * sizeof(double), cudaMemcpyDeviceToHost, R.st));
  DDA_CK(R.h, cudaStreamSynchronize(R.st));
  return DDA_OK;
}

c128 cplx(const double* p) { return mk<double>(p[0], p[1]); }
double cabs2h(c128 a) { return a.x * a.x + a.y * a.y; }
c128 cdivh(c128 a, c128 b) {
  const double d = b.x * b.x + b.y * b.y;
  return mk<double>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

}  // namespace

extern "C" int dda_solve_pc(dda_t h, dda_pcnet_t net, const dda_solve_opts* o, const double* prop,
                            const double* pol, void* P_dev, double* hist, int hist_len,
                            dda_solve_info* info) {
  DDA_ON_DEVICE(h);
  if (!o || !prop || !pol || !P_dev || !info || (hist && hist_len < 1))
    return dda_fail(h, DDA_ERR_ARG, "bad dda_solve_pc arguments");
  if (net && net->device != h->device) return dda_fail(h, DDA_ERR_ARG, "network on another device");
  if (!(o->tol > 0.0) || o->maxiter < 1 || o->pol < DDA_CM || o->pol > DDA_CLDR)
    return dda_fail(h, DDA_ERR_ARG, "bad solver options");
  if (!h->w64.have_D) return dda_fail(h, DDA_ERR_STATE, "D-matrix not built");
  auto t0 = std::chrono::steady_clock::now();
  int rc = dda_beta_internal(h, o->pol, 1, prop, pol);
  if (rc != DDA_OK) return rc;
  PcRun R;
  R.h = h;
  R.st = h->stream;
  R.n = 3 * h->g.n_occ;
  R.df = h->wdf.have_D;
  if (R.df) {
    if ((rc = ensure_work_cap<df>(h, h->wdf, 1)) != DDA_OK) return rc;
  } else {
    if ((rc = ensure_d64(h)) != DDA_OK || (rc = ensure_work_cap<double>(h, h->w64, 1)) != DDA_OK) return rc;
  }
  const long long n = R.n;
  c128* buf = nullptr;
  double* dbuf = nullptr;
  if (dev_malloc(&buf, (size_t)10 * n * sizeof(c128)) != cudaSuccess ||
      dev_malloc(&dbuf, (size_t)(6 * 256 + 6) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    dev_free(buf, R.st);
    return dda_fail(h, DDA_ERR_OOM, "preconditioned solver vectors");
  }
  double hout[6];
  R.part = dbuf;
  R.out = dbuf + 6 * 256;
  R.hout = hout;
  c128 *b = buf, *x = buf + n, *r = buf + 2 * n, *r0 = buf + 3 * n, *p = buf + 4 * n, *v = buf + 5 * n;
  c128 *s = buf + 6 * n, *t = buf + 7 * n, *ph = buf + 8 * n, *sh = buf + 9 * n;
  const int nbk = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * num_sms()));
  const c128 one = mk<double>(1.0, 0.0), zero = mk<double>(0.0, 0.0);
  Wave wv;
  for (int q = 0; q < 3; ++q) wv.a[q] = prop[q];
  for (int q = 0; q < 6; ++q) wv.e[q] = pol[q];
  int status = DDA_NOT_CONVERGED, iters = 0, matvecs = 0, napps = 0, fallback = 0;
  double res_true = NAN, res_rec = NAN;
  std::vector<double> hv;
  hv.push_back(1.0);
  auto done = [&](int code) {
    dev_free(buf, R.st);
    dev_free(dbuf, R.st);
    return code;
  };
#define PCK(call) do { const int rc_ = (call); if (rc_ != DDA_OK) return done(rc_); } while (0)
  PCK(launch_rhs(h, b, h->w64.beta, wv, R.st));
  DDA_CK(h, cudaMemsetAsync(x, 0, n * sizeof(c128), R.st));
  DDA_CK(h, cudaMemcpyAsync(r, b, n * sizeof(c128), cudaMemcpyDeviceToDevice, R.st));
  PCK(pc_dots(R, b, b));
  const double bn = std::sqrt(hout[0]);
  bool use_net = net != nullptr;
  auto precond = [&](const c128* in, c128* out) -> int {
    if (use_net) {
      ++napps;
      return dda_pcnet_apply(net, h, in, out) == DDA_OK ? DDA_OK
                                                        : dda_fail(h, DDA_ERR_CUDA, "network: " + net->err);
    }
    const cudaError_t e = cudaMemcpyAsync(out, in, n * sizeof(c128), cudaMemcpyDeviceToDevice, R.st);
    return e == cudaSuccess ? DDA_OK : dda_cuda_fail(h, e, "copy");
  };
  if (!(bn > 0.0)) {
    status = std::isfinite(bn) ? DDA_OK : DDA_ERR_NONFINITE;
    res_true = res_rec = std::isfinite(bn) ? 0.0 : NAN;
  }
  double best = 1.0;
  int best_it = 0;
  while (status == DDA_NOT_CONVERGED && iters < o->maxiter) {
    // (re)start from the current x: r0 = r, p = v = 0, rho = alpha = omega = 1
    DDA_CK(h, cudaMemcpyAsync(r0, r, n * sizeof(c128), cudaMemcpyDeviceToDevice, R.st));
    DDA_CK(h, cudaMemsetAsync(p, 0, n * sizeof(c128), R.st));
    DDA_CK(h, cudaMemsetAsync(v, 0, n * sizeof(c128), R.st));
    c128 rho = one, alpha = one, omega = one;
    PCK(pc_dots(R, r0, r));
    c128 rho_new = cplx(hout);
    bool restart = false;
    while (!restart && iters < o->maxiter) {
      if (cabs2h(rho_new) == 0.0) { restart = true; break; }
      const c128 beta = cdivh(rho_new, rho) * cdivh(alpha, omega);
      rho = rho_new;
      // p = r + beta (p - omega v)
      k_axpbypcz<<<nbk, 256, 0, R.st>>>(one, r, beta, p, mk<double>(-(beta * omega).x, -(beta * omega).y), v, n);
      count_launch();
      PCK(precond(p, ph));
      PCK(pc_matvec(R, ph, v));
      ++matvecs;
      PCK(pc_dots(R, r0, v));
      const c128 rv = cplx(hout);
      if (cabs2h(rv) == 0.0) { restart = true; break; }
      alpha = cdivh(rho, rv);
      // s = r - alpha v
      DDA_CK(h, cudaMemcpyAsync(s, r, n * sizeof(c128), cudaMemcpyDeviceToDevice, R.st));
      k_axpbypcz<<<nbk, 256, 0, R.st>>>(mk<double>(-alpha.x, -alpha.y), v, one, s, zero, nullptr, n);
      count_launch();
      PCK(precond(s, sh));
      PCK(pc_matvec(R, sh, t));
      ++matvecs;
      PCK(pc_dots(R, t, s, t, t));
      const c128 ts = cplx(hout);
      const double tt = hout[2];
      omega = tt > 0.0 ? mk<double>(ts.x / tt, ts.y / tt) : zero;
      // x += alpha p^ + omega s^ ; r = s - omega t
      k_axpbypcz<<<nbk, 256, 0, R.st>>>(alpha, ph, one, x, omega, sh, n);
      count_launch();
      DDA_CK(h, cudaMemcpyAsync(r, s, n * sizeof(c128), cudaMemcpyDeviceToDevice, R.st));
      k_axpbypcz<<<nbk, 256, 0, R.st>>>(mk<double>(-omega.x, -omega.y), t, one, r, zero, nullptr, n);
      count_launch();
      ++iters;
      PCK(pc_dots(R, r, r, r0, r));
      const double res = std::sqrt(hout[0]) / bn;
      rho_new = cplx(hout + 2);
      res_rec = res;
      hv.push_back(res);
      if (!std::isfinite(res)) { status = DDA_ERR_NONFINITE; break; }
      if (res < best * 0.99) { best = res; best_it = iters; }
      if (res < o->tol) break;
      if (cabs2h(omega) == 0.0) { restart = true; break; }
      if (use_net && iters - best_it >= 50) {   // stalled: continue without the network
        use_net = false;
        fallback = iters;
        restart = true;
        best_it = iters;
      }
    }
    if (status != DDA_NOT_CONVERGED) break;
    // the judge: the true residual with the exact product
    PCK(pc_matvec(R, x, t));
    ++matvecs;
    DDA_CK(h, cudaMemcpyAsync(r, b, n * sizeof(c128), cudaMemcpyDeviceToDevice, R.st));
    k_axpbypcz<<<nbk, 256, 0, R.st>>>(mk<double>(-1.0, 0.0), t, one, r, zero, nullptr, n);
    count_launch();
    PCK(pc_dots(R, r, r));
    res_true = std::sqrt(hout[0]) / bn;
    if (!std::isfinite(res_true)) { status = DDA_ERR_NONFINITE; break; }
    if (res_true < o->tol) { status = DDA_OK; break; }
  }
  if (status == DDA_NOT_CONVERGED && std::isnan(res_true)) {
    PCK(pc_matvec(R, x, t));
    ++matvecs;
    DDA_CK(h, cudaMemcpyAsync(r, b, n * sizeof(c128), cudaMemcpyDeviceToDevice, R.st));
    k_axpbypcz<<<nbk, 256, 0, R.st>>>(mk<double>(-1.0, 0.0), t, one, r, zero, nullptr, n);
    count_launch();
    PCK(pc_dots(R, r, r));
    res_true = std::sqrt(hout[0]) / bn;
  }
  k_p_from_x<<<nbk, 256, 0, R.st>>>(x, (c128*)P_dev, h->d_mat, h->w64.beta, h->g.n_occ);
  count_launch();
  DDA_CK(h, cudaStreamSynchronize(R.st));
#undef PCK
  dda_solve_info& inf = info[0];
  inf = dda_solve_info{};
  inf.status = status;
  inf.iters = iters;
  inf.matvecs = matvecs;
  inf.matvecs_fp64 = matvecs;
  inf.outer = fallback;             // iteration at which the network was dropped (0: never)
  inf.rel_res_true = res_true;
  inf.rel_res_recur = res_rec;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (hist)
    for (int i = 0; i < hist_len; ++i) hist[i] = i < (int)hv.size() ? hv[i] : -1.0;
  (void)napps;
  return done(status);
}

// ---------------------------------------------------------------- training pairs
namespace dda {
namespace pc {
// e = (Ps - Pk) / beta per dipole and component (beta = 0: e = 0)
__global__ void k_err_from_P(const c128* __restrict__ Ps, const c128* __restrict__ Pk,
                             const uint8_t* __restrict__ mat, const c128* __restrict__ beta,
                             long long n_occ, c128* __restrict__ e) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * n_occ;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / n_occ);
    const c128 b = beta[mat[i - c * n_occ] * 3 + c];
    const double d = b.x * b.x + b.y * b.y;
    const c128 p = Ps[i] - Pk[i];
    e[i] = d > 0.0 ? mk<double>((p.x * b.x + p.y * b.y) / d, (p.y * b.x - p.x * b.y) / d)
                   : mk<double>(0.0, 0.0);
  }
}
}  // namespace pc
}  // namespace dda

extern "C" int dda_pcnet_pair(dda_t h, int pol_prescription, const double* prop_host,
                              const double* pol_host, const void* P_star, const void* P_k, void* r_out,
                              void* e_out) {
  DDA_ON_DEVICE(h);
  if (!prop_host || !pol_host || !P_star || !P_k || !r_out || !e_out)
    return dda_fail(h, DDA_ERR_ARG, "bad dda_pcnet_pair arguments");
  if (!h->w64.have_D) return dda_fail(h, DDA_ERR_STATE, "D-matrix not built");
  int rc = dda_beta_internal(h, pol_prescription, 1, prop_host, pol_host);
  if (rc != DDA_OK) return rc;
  const bool use_df = h->wdf.have_D;
  if (use_df) rc = ensure_work_cap<dda::df>(h, h->wdf, 1);
  else if ((rc = ensure_d64(h)) == DDA_OK) rc = ensure_work_cap<double>(h, h->w64, 1);
  if (rc != DDA_OK) return rc;
  const long long n = 3 * h->g.n_occ;
  k_err_from_P<<<(int)std::min<long long>((n + 255) / 256, 8LL * num_sms()), 256, 0, h->stream>>>(
      (const c128*)P_star, (const c128*)P_k, h->d_mat, h->w64.beta, h->g.n_occ, (c128*)e_out);
  count_launch();
  const cudaError_t e = use_df ? launch_matvec_df(h->g, h->lat(), h->wdf, h->w64.beta, h->n_mat,
                                                  (const c128*)e_out, (c128*)r_out, 1, h->stream)
                           : launch_matvec<double>(h->g, h->lat(), h->w64, h->w64.beta, h->n_mat,
                                                   (const c128*)e_out, (c128*)r_out, 1, false, h->stream);
  if (e != cudaSuccess) return dda_cuda_fail(h, e, "pair product");
  DDA_CK(h, cudaStreamSynchronize(h->stream));
  return DDA_OK;
}
