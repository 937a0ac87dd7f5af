// Register-resident two-level FFT passes of the interaction-matrix product.
//
// Same five passes as matvec.cu (arXiv:0704.0037, Sec. 2: 1D transforms with
// pruned input and partial output), for padded lengths M = M1 * M2 known at
// compile time.  A length-M line is split with n = j + M2 i (j < M2, i < M1)
// and k = k1 + M1 k2:
//   phase 1: for each column j, an M1-point DFT over i (registers), then the
//            twiddle exp(-2 pi i j k1 / M) (shared-memory table);
//   phase 2: for each k1, an M2-point DFT over j (registers) gives X[k1 + M1 k2].
// The inverse runs the two phases in reverse with conjugate twiddles.
// Element (r, t) of T lines lives in shared memory as row r = k1 * M2 + j.
// Thread (t, q) handles line t: q is the column j in phase 1 and k1 in phase 2,
// so each thread only ever touches its own rows between the two barriers.
//
// Lines along y and z are strided in global memory; T adjacent lines (along
// x) are contiguous, so every global access of a warp covers T consecutive
// complex numbers.  Lines along x are contiguous; their tiles sit in shared
// memory as [t][LD] with LD odd (bank-conflict free) and are loaded and
// stored row by row.
#pragma once

#include <type_traits>

#include "codelets.cuh"
#include "internal.h"

namespace dda {
namespace fast {

template <int M1, int M2> constexpr int kQ = M1 > M2 ? M1 : M2;
// The product's padded lengths are M >= 2 n - 1, so its lines hold input (and
// keep output) only at n < (M + 1) / 2: of the elements n = j + M2 i of a
// line only i < kHalf can.  With this bound known at compile time the other
// inputs are constant zeros and the arithmetic of the discarded outputs is
// dead code (the zero input and partial output of Sec. 2).
template <int M1, int M2> constexpr int kHalf = ((M1 * M2 + 1) / 2 + M2 - 1) / M2;
// Blocks per SM a launch bound asks for: `want` for blocks of up to 288
// threads, one for the larger blocks of the long lines (512 and 1080), and
// never more than smem_bytes of shared memory per block lets reside
constexpr int kMinB(int nt, int want, long long smem_bytes) {
  const int by_smem = (int)((227LL * 1024) / (smem_bytes > 0 ? smem_bytes : 1));
  const int w = nt <= 288 ? want : 1;
  const int r = w < by_smem ? w : by_smem;
  return r >= 1 ? r : 1;
}

template <typename R>
__device__ __forceinline__ cpx<R> zero() { return mk<R>((R)0, (R)0); }

// Element type of the product's input and output vectors: the arithmetic
// type for complex64 and complex128, complex128 for the double-float passes
// (their vectors are the FP64 refinement's).
template <typename R> struct VecOf { using type = cpx<R>; };
template <> struct VecOf<df> { using type = c128; };

__device__ __forceinline__ c64 vload(const c64& v, c64*) { return v; }
__device__ __forceinline__ c128 vload(const c128& v, c128*) { return v; }
__device__ __forceinline__ cdf vload(const c128& v, cdf*) { return to_cdf(v); }
__device__ __forceinline__ c64 vstore(const c64& v) { return v; }
__device__ __forceinline__ c128 vstore(const c128& v) { return v; }
__device__ __forceinline__ c128 vstore(const cdf& v) { return to128(v); }
template <typename R> __device__ __forceinline__ cpx<R> vin(const typename VecOf<R>::type& v) {
  return vload(v, (cpx<R>*)nullptr);
}
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(df v) { return df_to_double(v); }

template <typename R>
__device__ __forceinline__ void load_tw(cpx<R>* s_tw, const cpx<R>* __restrict__ tw, int M, int nt) {
  for (int i = threadIdx.x; i < M; i += nt) s_tw[i] = tw[i];
}

// ---------------------------------------------------------------- P2: y forward
// B1 [3][nz][ny][Mx] -> B2 [3][nz][M][Mx]; grid (ceil(Mx/T), nz, 3).
// msign != 0 (D-matrix build, whole lines): only elements y <= M/2 are read;
// element y > M/2 is msign times element M - y (the line has that parity).
// ostr != 0: line group blockIdx.y starts at element blockIdx.y * ostr of
// both arrays (sub-blocks of whole lines, ny == M).  PRUNE: the product's
// lines (ny <= (M + 1) / 2, inputs past kHalf known zero).
template <typename R, int M1, int M2, int T, bool PRUNE>
__global__ void __launch_bounds__(T * kQ<M1, M2>) fk_yfwd(const cpx<R>* __restrict__ in,
                                                          cpx<R>* __restrict__ out, int ny, int nz,
                                                          int Mx, const cpx<R>* __restrict__ tw,
                                                          int msign, const int* __restrict__ skip,
                                                          long long ostr, const int* __restrict__ yr) {
  constexpr int M = M1 * M2, NT = T * kQ<M1, M2>;
  pdl_wait();
  pdl_launch();
  if (skip && skip[blockIdx.z / 3]) return;     // right-hand side already converged
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* s = s_tw + M;
  const int t = threadIdx.x % T, q = threadIdx.x / T;
  const int kx = blockIdx.x * T + t;
  const long long og = (long long)blockIdx.z * nz + blockIdx.y;
  const long long ib = ostr ? og * ostr : og * ny * Mx;
  const long long ob = ostr ? og * ostr : og * M * Mx;
  // rows of plane blockIdx.y outside its span of occupied rows are not read
  // (zero; the x pass does not write them) when the spans are given; the
  // span is fetched with the twiddles
  __shared__ int s_yr[2];
  if (threadIdx.x < 2) s_yr[threadIdx.x] = yr ? yr[2 * blockIdx.y + threadIdx.x] : (threadIdx.x ? ny - 1 : 0);
  load_tw(s_tw, tw, M, NT);
  __syncthreads();
  const int ylo = s_yr[0], yhi = s_yr[1];
  if (q < M2) {
    const int j = q;
    cpx<R> v[M1];
    if (msign == 0) {
#pragma unroll
      for (int i = 0; i < M1; ++i) {
        const int y = j + M2 * i;
        v[i] = ((!PRUNE || i < kHalf<M1, M2>) && y >= ylo && y <= yhi && kx < Mx)
                   ? in[ib + (long long)y * Mx + kx]
                   : zero<R>();
      }
    } else {
#pragma unroll
      for (int i = 0; i < M1; ++i) {
        const int y = j + M2 * i;
        const bool mir = 2 * y > M;
        const int ys = mir ? M - y : y;
        cpx<R> w = kx < Mx ? in[ib + (long long)ys * Mx + kx] : zero<R>();
        if (mir && msign < 0) w = mk<R>(-w.x, -w.y);
        v[i] = w;
      }
    }
    cl::Dft<R, false, M1>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < M1; ++k1) v[k1] = twiddle<R, false>(v[k1], s_tw[j * k1]);
#pragma unroll
    for (int k1 = 0; k1 < M1; ++k1) s[(k1 * M2 + j) * T + t] = v[k1];
  }
  __syncthreads();
  if (q < M1 && kx < Mx) {
    const int k1 = q;
    cpx<R> u[M2];
#pragma unroll
    for (int j = 0; j < M2; ++j) u[j] = s[(k1 * M2 + j) * T + t];
    cl::Dft<R, false, M2>::run(u);
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) out[ob + (long long)(k1 + M1 * k2) * Mx + kx] = u[k2];
  }
}

// ---------------------------------------------------------------- P4: y inverse
// B2 [3][nz][M][Mx] -> B1 [3][nz][ny][Mx] (y < ny kept); grid (ceil(Mx/T), nz, 3)
template <typename R, int M1, int M2, int T>
__global__ void __launch_bounds__(T * kQ<M1, M2>) fk_yinv(const cpx<R>* __restrict__ in,
                                                          cpx<R>* __restrict__ out, int ny, int nz,
                                                          int Mx, const cpx<R>* __restrict__ tw,
                                                          const int* __restrict__ skip) {
  constexpr int M = M1 * M2, NT = T * kQ<M1, M2>;
  pdl_wait();
  pdl_launch();
  if (skip && skip[blockIdx.z / 3]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* s = s_tw + M;
  const int t = threadIdx.x % T, q = threadIdx.x / T;
  const int kx = blockIdx.x * T + t;
  const long long ib = ((long long)blockIdx.z * nz + blockIdx.y) * M * Mx;
  const long long ob = ((long long)blockIdx.z * nz + blockIdx.y) * ny * Mx;
  load_tw(s_tw, tw, M, NT);
  __syncthreads();
  if (q < M1) {
    const int k1 = q;
    cpx<R> u[M2];
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2)
      u[k2] = kx < Mx ? in[ib + (long long)(k1 + M1 * k2) * Mx + kx] : zero<R>();
    cl::Dft<R, true, M2>::run(u);
#pragma unroll
    for (int j = 1; j < M2; ++j) u[j] = twiddle<R, true>(u[j], s_tw[j * k1]);
#pragma unroll
    for (int j = 0; j < M2; ++j) s[(k1 * M2 + j) * T + t] = u[j];
  }
  __syncthreads();
  if (q < M2 && kx < Mx) {
    const int j = q;
    cpx<R> v[M1];
#pragma unroll
    for (int k1 = 0; k1 < M1; ++k1) v[k1] = s[(k1 * M2 + j) * T + t];
    cl::Dft<R, true, M1>::run(v);
#pragma unroll
    for (int i = 0; i < M1; ++i) {
      const int y = j + M2 * i;
      if (i < kHalf<M1, M2> && y < ny) out[ob + (long long)y * Mx + kx] = v[i];
    }
  }
}

// ---------------------------------------------------------------- async copies
// 16-byte global -> shared copies that complete in the background (the
// pre-TMA asynchronous copy of sm_80 and later); a zero source size fills the
// destination with zeros without reading.  Waits are on commit groups, with
// no spin loop of ours.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n)
               : "memory");
}
// Asynchronous copy of one complex element (8 or 16 bytes) global -> shared;
// !valid fills zeros without reading.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(n)
               : "memory");
}
template <int S>
__device__ __forceinline__ void cp_async_elem(void* smem, const void* gmem, bool valid) {
  static_assert(S == 8 || S == 16, "8- or 16-byte elements");
  if constexpr (S == 8) cp_async8(smem, gmem, valid);
  else cp_async16(smem, gmem, valid);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Fetch the 128-byte line holding p into L2 (no data returned to the thread)
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- P3: z fused
// In place on B2 [3][nz][My][Mx]: per (kx, ky) line, forward z transform of the
// nz nonzero inputs, 3x3 product with the octant of FFT(G) (parity signs),
// inverse z transform, z < nz kept.  grid (ceil(Mx/T), My).
__device__ __forceinline__ int fold_axis(int k, int M, int& neg) {
  if (2 * k > M) { neg = 1; return M - k; }
  neg = 0;
  return k;
}

// Shared-memory rows of one component of the fused z pass: row k1 M2 + j of
// the two-level split (j < M2) lives in physical row k1 (M2 + 1) + j when a
// tile row is narrower than the 32 banks (T complex64 < 16 columns), so that
// the rows M2 apart read together by the second phase fall in different
// banks; otherwise in row k1 M2 + j.
template <typename R, int M1, int M2, int T>
struct ZRows {
  static constexpr bool pad = T * (int)sizeof(cpx<R>) < 128;
  static constexpr int rows = pad ? M1 * M2 + M1 : M1 * M2;
  // physical row of row k1 M2 + j (j < M2)
  static __device__ __forceinline__ int at(int k1, int j) { return k1 * (pad ? M2 + 1 : M2) + j; }
};

// Row ky of the z pass taken by block row b: 0, 1, My - 1, 2, My - 2, ...
// (a permutation of 0 .. My - 1), so that the rows ky and My - ky, whose
// products read the same octant entries (fy = min(ky, My - ky)), run one
// after the other and the second finds them in L2.
__device__ __forceinline__ int ky_order(int b, int My) {
  if (b == 0) return 0;
  const int j = (b + 1) / 2;
  return (b & 1) ? j : My - j;
}

// Pieces of the fused z pass.  A tile is T adjacent columns (kx from bx T) of
// one ky; s is [3][rows][T] (component, row, column) in shared memory.
//
// Stage the nz x T input tile of component c in the first nz rows of that
// component's own region (its first transform phase reads it all before
// overwriting the region): asynchronous 16-byte copies, one commit group per
// call.  Chunks past the last column are zero-filled without reading.  Rows
// of an odd number of complex64 elements (x padded to an odd length: this z
// pass runs whenever the z length has a compiled split) do not start on
// 16-byte boundaries, so their elements are copied one by one.
template <typename R, int T, int NT>
__device__ __forceinline__ void zc_stage(cpx<R>* tile, const cpx<R>* B2, int c, int nz, int Mx,
                                         int My, int bx, int ky) {
  constexpr int E = 16 / (int)sizeof(cpx<R>);   // elements per chunk
  constexpr int CPR = T / E;                     // chunks per tile row
  const long long plane = (long long)My * Mx;
  const int kx0 = bx * T;
  const bool by_elem = E > 1 && (Mx % E) != 0;
  const cpx<R>* src = B2 + c * (long long)nz * plane + (long long)ky * Mx + kx0;
  if (by_elem) {
    for (int k = threadIdx.x; k < nz * T; k += NT) {
      const int z = k / T, u = k - z * T;
      const bool ok = kx0 + u < Mx;
      cp_async_elem<sizeof(cpx<R>)>(tile + z * T + u,
                                    ok ? (const void*)(src + z * plane + u) : (const void*)B2, ok);
    }
  } else {
    for (int k = threadIdx.x; k < nz * CPR; k += NT) {
      const int z = k / CPR, u = k - z * CPR;
      const bool ok = kx0 + u * E < Mx;
      cp_async16(tile + z * T + u * E, ok ? (const void*)(src + z * plane + u * E) : (const void*)B2,
                 ok);
    }
  }
  cp_async_commit();
}

// The six octant entries (xx, xy, xz, yy, yz, zz) of point o: of the
// interleaved complex64 octant [Mz/2+1][My/2+1][Mx/2+1][6] with three 16-byte
// loads, of the planar octant [6][octs] of the wider types with six.
template <typename R>
__device__ __forceinline__ void load_oct(const cpx<R>* __restrict__ D, long long o, long long octs,
                                         cpx<R> (&d)[6]) {
  if constexpr (kOctInterleaved<R>) {
    const float4* q = reinterpret_cast<const float4*>(D + 6 * o);   // 48 bytes, 16-byte aligned
    const float4 a = q[0], b = q[1], c = q[2];
    d[0] = mk<float>(a.x, a.y); d[1] = mk<float>(a.z, a.w); d[2] = mk<float>(b.x, b.y);
    d[3] = mk<float>(b.z, b.w); d[4] = mk<float>(c.x, c.y); d[5] = mk<float>(c.z, c.w);
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) d[k] = D[k * octs + o];
  }
}

// Warm L2 with the octant entries of the Fourier-space product of a tile (fy
// of its ky, its range of fx, every fz and component): they arrive from HBM
// while the forward transforms run, so the product's loads hit L2.  Each fz
// row of the tile is one contiguous run of the interleaved octant (every
// 128-byte line it touches prefetched), or six runs of the planar one (their
// first and last lines).
template <typename R, int M, int T, int NT>
__device__ __forceinline__ void zc_prefetch(const cpx<R>* D, int Mx, int My, int bx, int ky) {
  const int hx = Mx / 2 + 1, hy = My / 2 + 1, hz = M / 2 + 1;
  int nys, na, nb;
  const int fy = fold_axis(ky, My, nys);
  const int kxa = bx * T, kxb = min(kxa + T, Mx) - 1;
  const int fa = fold_axis(kxa, Mx, na), fb = fold_axis(kxb, Mx, nb);
  const int fmin = min(fa, fb);
  const int fmax = (2 * kxa <= Mx && 2 * kxb >= Mx) ? Mx / 2 : max(fa, fb);
  if constexpr (kOctInterleaved<R>) {
    const int nl = (int)(((size_t)(fmax - fmin + 1) * 6 * sizeof(cpx<R>) + 127) / 128) + 1;
    for (int k = threadIdx.x; k < hz * nl; k += NT) {
      const int fz = k / nl, l = k - fz * nl;
      const long long o = ((long long)fz * hy + fy) * hx;
      const size_t a0 = (size_t)(D + 6 * (o + fmin)) >> 7;
      const size_t a1 = ((size_t)(D + 6 * (o + fmax + 1)) - 1) >> 7;
      if (a0 + l <= a1) prefetch_l2((const void*)((a0 + l) << 7));
    }
  } else {
    const long long octs = (long long)hx * hy * hz;
    for (int k = threadIdx.x; k < 6 * hz; k += NT) {
      const int c6 = k / hz, fz = k - c6 * hz;
      const cpx<R>* row = D + c6 * octs + ((long long)fz * hy + fy) * hx;
      prefetch_l2(row + fmin);
      if (((size_t)(row + fmax) >> 7) != ((size_t)(row + fmin) >> 7)) prefetch_l2(row + fmax);
    }
  }
}

// Fourier-space product with the octant of FFT(G).  Work item (t, fz): the
// six octant values at (fx, fy, fz) are loaded once and applied to both
// kz = fz and kz = M - fz (sign flips for the components odd in z); the
// spectrum value kz = k1 + M1 k2 of column t lives in row Z::at(k1, k2);
// components are CS elements apart.  A thread keeps its column t and steps
// fz by NT / T, so its octant index and the (k1, k2) of both kz advance by
// constants instead of being recomputed (no division per item).
template <typename R, int M1, int M2, int T, int NT, int CS>
__device__ __forceinline__ void zc_product(cpx<R>* s, const cpx<R>* __restrict__ D, int Mx, int My,
                                           int bx, int ky) {
  using Z = ZRows<R, M1, M2, T>;
  constexpr int M = M1 * M2, hz = M / 2 + 1;
  static_assert(NT % T == 0, "a thread's work items share its column");
  constexpr int FS = NT / T, S1 = FS % M1, S2 = FS / M1;
  const int hx = Mx / 2 + 1, hy = My / 2 + 1;
  int nys;
  const int fy = fold_axis(ky, My, nys);
  const int t2 = threadIdx.x % T;
  const int kx2 = bx * T + t2;
  if (kx2 >= Mx) return;
  int nxs;
  const int fx = fold_axis(kx2, Mx, nxs);
  const long long octs = (long long)hx * hy * hz;
  const long long ostep = (long long)FS * hy * hx;
  int fz = threadIdx.x / T;
  long long o = ((long long)fz * hy + fy) * hx + fx;
  int a1 = fz % M1, a2 = fz / M1;                // kz = fz
  int b1 = (M - fz) % M1, b2 = (M - fz) / M1;    // kz = M - fz
#pragma unroll 2
  for (; fz < hz; fz += FS, o += ostep) {
    cpx<R> d6[6];
    load_oct<R>(D, o, octs, d6);
    const cpx<R> dxx = d6[0], dyy = d6[3], dzz = d6[5];
    cpx<R> dxy = d6[1], ez = d6[2], fzz = d6[4];
    if (nxs ^ nys) dxy = mk<R>(-dxy.x, -dxy.y);
    if (nxs) ez = mk<R>(-ez.x, -ez.y);           // xz and yz at kz = fz
    if (nys) fzz = mk<R>(-fzz.x, -fzz.y);
    {
      const int e = Z::at(a1, a2) * T + t2;
      const cpx<R> vx = s[e], vy = s[CS + e], vz = s[2 * CS + e];
      s[e] = dxx * vx + dxy * vy + ez * vz;
      s[CS + e] = dxy * vx + dyy * vy + fzz * vz;
      s[2 * CS + e] = ez * vx + fzz * vy + dzz * vz;
    }
    if (fz != 0 && 2 * fz != M) {
      // kz = M - fz: xz and yz change sign (odd in z); the negated terms are
      // subtracted, which rounds exactly as adding the negated products
      const int e = Z::at(b1, b2) * T + t2;
      const cpx<R> vx = s[e], vy = s[CS + e], vz = s[2 * CS + e];
      s[e] = dxx * vx + dxy * vy - ez * vz;
      s[CS + e] = dxy * vx + dyy * vy - fzz * vz;
      s[2 * CS + e] = dzz * vz - (ez * vx + fzz * vy);
    }
    a1 += S1;
    a2 += S2;
    if (a1 >= M1) { a1 -= M1; ++a2; }
    b1 -= S1;
    b2 -= S2;
    if (b1 < 0) { b1 += M1; --b2; }
  }
}

// The double-float z pass runs its forward phase 2 and its inverse phase A
// through one M2-point codelet (zc_m2_one_codelet): its unrolled double-float
// transforms are long enough that separate forward and inverse copies miss
// the instruction cache (sharing the M1-point codelet too would give up the
// compile-time pruning of the first and last phases, and measured slower)
template <typename R> constexpr bool kZOneM2 = std::is_same<R, df>::value;
// a.y times sg (+1 or -1): conjugation by a runtime sign
__device__ __forceinline__ cpx<df> imag_sign(cpx<df> a, float sg) {
  cpx<df> r;
  r.x = a.x;
  r.y = df(a.y.hi * sg, a.y.lo * sg);
  return r;
}

// Forward phase 2 of every component, the product and inverse phase A of
// every component with one M2-point codelet: the inverse transform is the
// conjugate of the forward transform of the conjugate (pass 0 forward, then
// the product, pass 1 inverse).  Starts after a barrier, ends with one.
template <typename R, int M1, int M2, int T, int NT>
__device__ __forceinline__ void zc_m2_one_codelet(cpx<R>* s, const cpx<R>* s_tw,
                                                  const cpx<R>* __restrict__ D, int Mx, int My,
                                                  int bx, int ky) {
  using Z = ZRows<R, M1, M2, T>;
  constexpr int M = M1 * M2, CS = Z::rows * T;
  const int t = threadIdx.x % T, q = threadIdx.x / T;
  const int kx = bx * T + t;
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      zc_product<R, M1, M2, T, NT, CS>(s, D, Mx, My, bx, ky);
      __syncthreads();
    }
    if (q < M1 && kx < Mx) {
      const int k1 = q;
      const float sg = pass ? -1.0f : 1.0f;
#pragma unroll 1
      for (int c = 0; c < 3; ++c) {
        cpx<R>* sc = s + c * CS;
        cpx<R> u[M2];
#pragma unroll
        for (int j = 0; j < M2; ++j) u[j] = imag_sign(sc[Z::at(k1, j) * T + t], sg);
        cl::Dft<R, false, M2>::run(u);
#pragma unroll
        for (int j = 0; j < M2; ++j) u[j] = imag_sign(u[j], sg);
        if (pass) {
#pragma unroll
          for (int j = 1; j < M2; ++j) u[j] = twiddle<R, true>(u[j], s_tw[j * k1]);
        }
#pragma unroll
        for (int j = 0; j < M2; ++j) sc[Z::at(k1, j) * T + t] = u[j];
      }
    }
    __syncthreads();
  }
}

// Forward z transforms of the three staged components of a tile (phase 1
// waits for each component's copies), the product, and the inverse z
// transforms up to the inverse phase A of every component; the caller runs
// inverse phase B (zc_inverse_b) per component.
template <typename R, int M1, int M2, int T, int NT>
__device__ __forceinline__ void zc_forward_product_inva(cpx<R>* s, const cpx<R>* s_tw,
                                                       const cpx<R>* __restrict__ D, int nz, int Mx,
                                                       int My, int bx, int ky) {
  using Z = ZRows<R, M1, M2, T>;
  constexpr int M = M1 * M2, CS = Z::rows * T, kZin = kHalf<M1, M2>;
  const int t = threadIdx.x % T, q = threadIdx.x / T;
  const int kx = bx * T + t;
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    if (c == 0) cp_async_wait<2>();
    else if (c == 1) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();           // this component's tile (and the twiddles) complete
    cpx<R>* sc = s + c * CS;
    const int j = q;
    cpx<R> v[M1];
    if (q < M2) {
#pragma unroll
      for (int i = 0; i < M1; ++i) {
        const int z = j + M2 * i;
        v[i] = (i < kZin && z < nz) ? sc[z * T + t] : zero<R>();
      }
    }
    __syncthreads();           // every read of the tile before the region is rewritten
    if (q < M2) {
      cl::Dft<R, false, M1>::run(v);
#pragma unroll
      for (int k1 = 1; k1 < M1; ++k1) v[k1] = twiddle<R, false>(v[k1], s_tw[j * k1]);
#pragma unroll
      for (int k1 = 0; k1 < M1; ++k1) sc[Z::at(k1, j) * T + t] = v[k1];
    }
  }
  __syncthreads();
  if constexpr (kZOneM2<R>) {
    zc_m2_one_codelet<R, M1, M2, T, NT>(s, s_tw, D, Mx, My, bx, ky);
    return;
  }
  if (q < M1 && kx < Mx) {
    const int k1 = q;
    // forward phase 2 of each component, written back to this thread's rows
    // (row k1*M2 + k2 holds kz = k1 + M1*k2)
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      cpx<R>* sc = s + c * CS;
      cpx<R> u[M2];
#pragma unroll
      for (int j = 0; j < M2; ++j) u[j] = sc[Z::at(k1, j) * T + t];
      cl::Dft<R, false, M2>::run(u);
#pragma unroll
      for (int k2 = 0; k2 < M2; ++k2) sc[Z::at(k1, k2) * T + t] = u[k2];
    }
  }
  __syncthreads();
  // kz = k1 + M1 k2 lives in row k1*M2 + k2
  zc_product<R, M1, M2, T, NT, CS>(s, D, Mx, My, bx, ky);
  __syncthreads();
  if (q < M1 && kx < Mx) {
    const int k1 = q;
    // inverse phase A of each component: M2-point inverse over k2, conjugate twiddle
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      cpx<R>* sc = s + c * CS;
      cpx<R> u[M2];
#pragma unroll
      for (int k2 = 0; k2 < M2; ++k2) u[k2] = sc[Z::at(k1, k2) * T + t];
      cl::Dft<R, true, M2>::run(u);
#pragma unroll
      for (int j = 1; j < M2; ++j) u[j] = twiddle<R, true>(u[j], s_tw[j * k1]);
#pragma unroll
      for (int j = 0; j < M2; ++j) sc[Z::at(k1, j) * T + t] = u[j];
    }
  }
  __syncthreads();
}

// Inverse phase B of component c of a tile: M1-point inverse over k1, rows
// z = j + M2 i < nz stored to B2.
template <typename R, int M1, int M2, int T>
__device__ __forceinline__ void zc_inverse_b(const cpx<R>* sc, cpx<R>* __restrict__ B2c, int nz,
                                             int Mx, long long plane, long long col, int kx) {
  using Z = ZRows<R, M1, M2, T>;
  constexpr int kZin = kHalf<M1, M2>;
  const int t = threadIdx.x % T, q = threadIdx.x / T;
  if (q < M2 && kx < Mx) {
    const int j = q;
    cpx<R> v[M1];
#pragma unroll
    for (int k1 = 0; k1 < M1; ++k1) v[k1] = sc[Z::at(k1, j) * T + t];
    cl::Dft<R, true, M1>::run(v);
#pragma unroll
    for (int i = 0; i < M1; ++i) {
      const int z = j + M2 * i;
      if (i < kZin && z < nz) B2c[z * plane + col] = v[i];
    }
  }
}

template <typename R, int M1, int M2, int T>
__global__ void __launch_bounds__(T * kQ<M1, M2>,
                                  kMinB(T * kQ<M1, M2>, 2, (M1 * M2 + 3LL * ZRows<R, M1, M2, T>::rows * T) * sizeof(cpx<R>)))
    fk_zconv(cpx<R>* __restrict__ B2, const cpx<R>* __restrict__ D, int nz, int Mx, int My,
             const cpx<R>* __restrict__ tw, const int* __restrict__ skip) {
  constexpr int M = M1 * M2, NT = T * kQ<M1, M2>, CS = ZRows<R, M1, M2, T>::rows * T;
  pdl_wait();
  pdl_launch();
  if (skip && skip[blockIdx.z]) return;
  B2 += (long long)blockIdx.z * 3 * nz * My * Mx;      // right-hand side blockIdx.z
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* s = s_tw + M;                      // [3][rows][T]
  // complex64 (interleaved octant): mirrored rows together; the double-width
  // passes measured faster in natural order
  const int bx = blockIdx.x, ky = kOctInterleaved<R> ? ky_order(blockIdx.y, My) : (int)blockIdx.y;
  const int kx = bx * T + threadIdx.x % T;
  const long long plane = (long long)My * Mx;
  const long long comp = (long long)nz * plane;
  const long long col = (long long)ky * Mx + kx;
  for (int c = 0; c < 3; ++c) zc_stage<R, T, NT>(s + c * CS, B2, c, nz, Mx, My, bx, ky);
  zc_prefetch<R, M, T, NT>(D, Mx, My, bx, ky);
  load_tw(s_tw, tw, M, NT);
  zc_forward_product_inva<R, M1, M2, T, NT>(s, s_tw, D, nz, Mx, My, bx, ky);
#pragma unroll 1
  for (int c = 0; c < 3; ++c) zc_inverse_b<R, M1, M2, T>(s + c * CS, B2 + c * comp, nz, Mx, plane, col, kx);
}

// ---------------------------------------------------------------- P1: x forward
// gather beta*x of T rows into a [t][LD] tile, transform, store rows of
// B1 [3][nrows][M]; grid (ceil(nrows/T), 3)
template <int M> constexpr int kLD = (M % 2 == 1) ? M : M + 1;

// Row t (0 <= t < T) of the block holding dipole i: the last t with
// off[t] <= i, for the non-decreasing offsets off[0..T] of the block's rows
// (off[0] <= i < off[T]; empty rows are skipped over).
template <int T>
__device__ __forceinline__ int row_of(const long long* off, long long i) {
  static_assert((T & (T - 1)) == 0, "tile rows must be a power of two");
  int t = 0;
#pragma unroll
  for (int b = T / 2; b >= 1; b >>= 1)
    if (off[t + b] <= i) t += b;
  return t;
}

// Loads per thread issued together in the gather and scatter loops over a
// block's dipoles
// in the x forward and x inverse passes: more for the long lines, whose
// blocks of few rows hold many dipoles, as far as the registers of the
// blocks an SM holds allow
template <int M> constexpr int kGUF = M >= 1000 ? 8 : 4;
template <int M> constexpr int kGUI = M >= 1000 ? 16 : 4;

template <typename R, int M1, int M2, int T, bool CONJ>
__global__ void __launch_bounds__(T * kQ<M1, M2>, kMinB(T * kQ<M1, M2>, 3, (M1 * M2 + T * kLD<M1 * M2>) * sizeof(cpx<R>))) fk_xfwd(const typename VecOf<R>::type* __restrict__ x,
                                                          cpx<R>* __restrict__ B1, LatticeDev lat,
                                                          const cpx<R>* __restrict__ beta,
                                                          long long n_occ, int nrows,
                                                          const cpx<R>* __restrict__ tw,
                                                          int bstride, const int* __restrict__ skip) {
  constexpr int M = M1 * M2, NT = T * kQ<M1, M2>, LD = kLD<M>, kGU = kGUF<M1 * M2>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_off[T + 1];
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* a = s_tw + M;                      // [T][LD]
  // blockIdx.y = 3 * (right-hand side) + component; vectors [rhs][3][n_occ]
  const int cc = blockIdx.y, c = cc % 3;
  pdl_wait();
  pdl_launch();
  if (skip && skip[cc / 3]) return;
  beta += (long long)(cc / 3) * bstride;
  // the rows transformed: those within the planes' spans of occupied rows
  // when the lattice lists them, else every row
  __shared__ int s_row[T];
  const int nr = lat.arow ? lat.nact : nrows;
  const int r0 = blockIdx.x * T;
  if (threadIdx.x <= T) {
    const int i = min(r0 + (int)threadIdx.x, nr);
    s_off[threadIdx.x] = lat.arow ? lat.aoff[i] : lat.row_off[i];
    if (threadIdx.x < T) s_row[threadIdx.x] = lat.arow ? lat.arow[min(i, nr - 1)] : i;
  }
  load_tw(s_tw, tw, M, NT);
  for (int i = threadIdx.x; i < T * LD; i += NT) a[i] = zero<R>();
  __syncthreads();
  {
    // all threads over the block's dipoles (contiguous in x: rows r0..r0+T-1),
    // kGU independent loads of x, xi and mat in flight per thread
    const typename VecOf<R>::type* __restrict__ xc = x + (long long)cc * n_occ;
    const uint16_t* __restrict__ xi = lat.xi;
    const uint8_t* __restrict__ mt = lat.mat;
    const long long S0 = s_off[0];
    const int span = (int)(s_off[T] - S0);
    for (int k0 = threadIdx.x; k0 < span; k0 += kGU * NT) {
      typename VecOf<R>::type xv[kGU];
      int xk[kGU], mk_[kGU];
#pragma unroll
      for (int u = 0; u < kGU; ++u) {
        const int k = k0 + u * NT;
        if (k < span) {
          xv[u] = xc[S0 + k];
          xk[u] = xi[S0 + k];
          mk_[u] = mt[S0 + k];
        }
      }
#pragma unroll
      for (int u = 0; u < kGU; ++u) {
        const int k = k0 + u * NT;
        if (k < span) {
          cpx<R> v = vin<R>(xv[u]);
          if (CONJ) v = conjg(v);
          a[row_of<T>(s_off, S0 + k) * LD + xk[u]] = beta[mk_[u] * 3 + c] * v;
        }
      }
    }
  }
  __syncthreads();
  const int t = threadIdx.x % T, q = threadIdx.x / T;
  cpx<R>* at = a + t * LD;
  if (q < M2) {              // phase 1: reads and writes the same set {j + M2 i}
    const int j = q;
    cpx<R> v[M1];
#pragma unroll
    for (int i = 0; i < M1; ++i) v[i] = i < kHalf<M1, M2> ? at[j + M2 * i] : zero<R>();
    cl::Dft<R, false, M1>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < M1; ++k1) v[k1] = twiddle<R, false>(v[k1], s_tw[j * k1]);
#pragma unroll
    for (int k1 = 0; k1 < M1; ++k1) at[k1 * M2 + j] = v[k1];
  }
  __syncthreads();
  cpx<R> u[M2];
  if (q < M1) {
    const int k1 = q;
#pragma unroll
    for (int j = 0; j < M2; ++j) u[j] = at[k1 * M2 + j];
    cl::Dft<R, false, M2>::run(u);
  }
  __syncthreads();
  if (q < M1) {              // natural order k = k1 + M1 k2
    const int k1 = q;
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) at[k1 + M1 * k2] = u[k2];
  }
  __syncthreads();
  // row tt of the block is row s_row[tt] of B1
  cpx<R>* out = B1 + (long long)cc * nrows * M;
  const int nel = min(T, nr - r0) * M;
  for (int idx = threadIdx.x; idx < nel; idx += NT) {
    const int tt = idx / M, m = idx - tt * M;
    out[(long long)s_row[tt] * M + m] = a[tt * LD + m];
  }
}


// ---------------------------------------------------------------- P5: x inverse
// rows of B1 -> [t][LD] tile, inverse transform, y = x - beta u at the
// occupied x; grid (ceil(nrows/T), 3).  The tile rows (contiguous in B1) and
// the block's slice of x are staged by asynchronous copies before the
// transform, so their latency overlaps; the slice holds up to kXS elements
// (a row has at most (M + 1) / 2 dipoles when M >= 2 n_x - 1; any excess is
// read directly).
// staged elements of x per tile row: a row holds at most (M + 1) / 2
// dipoles; the long lines stage up to 384 (about the mean of the 536^3
// sphere's 4-row tiles) and read the rest directly
template <int M> constexpr int kXRow = (M + 1) / 2 < 384 ? (M + 1) / 2 : 384;
// blocks per SM the x inverse pass's launch bound asks for: four in
// complex64 (at 270 points 56 registers, no spill: P5 of the 134^3 sphere
// 59 -> 55 us), three in the wider arithmetic
template <typename R, int M> constexpr int kXinvB = (sizeof(R) == 4) ? 4 : 3;

template <typename R, int M1, int M2, int T, bool CONJ>
__global__ void __launch_bounds__(T * kQ<M1, M2>, kMinB(T * kQ<M1, M2>, kXinvB<R, M1 * M2>, (M1 * M2 + T * kLD<M1 * M2>) * sizeof(cpx<R>) + T * kXRow<M1 * M2> * sizeof(typename VecOf<R>::type))) fk_xinv(const cpx<R>* __restrict__ B1,
                                                          const typename VecOf<R>::type* __restrict__ x,
                                                          typename VecOf<R>::type* __restrict__ y,
                                                          LatticeDev lat,
                                                          const cpx<R>* __restrict__ beta,
                                                          long long n_occ, int nrows,
                                                          const cpx<R>* __restrict__ tw,
                                                          double* __restrict__ dotp, int bstride,
                                                          const int* __restrict__ skip) {
  constexpr int M = M1 * M2, NT = T * kQ<M1, M2>, LD = kLD<M>, kXS = T * kXRow<M>, kGU = kGUI<M1 * M2>;
  using V = typename VecOf<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_off[T + 1];
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* a = s_tw + M;                      // [T][LD]
  V* s_x = reinterpret_cast<V*>(a + T * LD); // [kXS]
  const int cc = blockIdx.y, c = cc % 3;     // 3 * (right-hand side) + component
  pdl_wait();
  pdl_launch();
  if (skip && skip[cc / 3]) return;
  beta += (long long)(cc / 3) * bstride;
  // the rows transformed: those within the planes' spans of occupied rows
  // when the lattice lists them (the rows outside hold no dipole), else
  // every row; a block's rows are consecutive in B1 unless they cross planes
  const int nr = lat.arow ? lat.nact : nrows;
  const int r0 = blockIdx.x * T;
  const int rows = min(T, nr - r0);
  const long long* off = lat.arow ? lat.aoff : lat.row_off;
  int rb = r0;
  bool runs = false;
  if (lat.arow) {
    rb = lat.arow[r0];
    runs = lat.arow[r0 + rows - 1] - rb != rows - 1;
  }
  const cpx<R>* in = B1 + (long long)cc * nrows * M;
  for (int idx = threadIdx.x; idx < T * M; idx += NT) {
    const int tt = idx / M, m = idx - tt * M;
    const bool ok = tt < rows;
    const long long row = runs ? (ok ? lat.arow[r0 + tt] : 0) : rb + tt;
    cp_async_elem<sizeof(cpx<R>)>(a + tt * LD + m, ok ? (const void*)(in + row * M + m) : (const void*)B1,
                                  ok);
  }
  const V* xc = x + (long long)cc * n_occ;
  V* yc = y + (long long)cc * n_occ;
  const long long S0 = off[r0];
  const int span = (int)(off[r0 + rows] - S0);
  const int staged = min(span, kXS);
  for (int k = threadIdx.x; k < staged; k += NT) cp_async_elem<sizeof(V)>(s_x + k, xc + S0 + k, true);
  cp_async_commit();
  if (threadIdx.x <= T) s_off[threadIdx.x] = off[min(r0 + (int)threadIdx.x, nr)];
  load_tw(s_tw, tw, M, NT);
  cp_async_wait<0>();
  __syncthreads();
  const int t = threadIdx.x % T, q = threadIdx.x / T;
  cpx<R>* at = a + t * LD;
  cpx<R> u[M2];
  if (q < M1) {              // phase A reads k = k1 + M1 k2
    const int k1 = q;
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) u[k2] = at[k1 + M1 * k2];
    cl::Dft<R, true, M2>::run(u);
#pragma unroll
    for (int j = 1; j < M2; ++j) u[j] = twiddle<R, true>(u[j], s_tw[j * k1]);
  }
  __syncthreads();
  if (q < M1) {
    const int k1 = q;
#pragma unroll
    for (int j = 0; j < M2; ++j) at[k1 * M2 + j] = u[j];
  }
  __syncthreads();
  if (q < M2) {              // phase B reads and writes the same set {j + M2 i}
    const int j = q;
    cpx<R> v[M1];
#pragma unroll
    for (int k1 = 0; k1 < M1; ++k1) v[k1] = at[k1 * M2 + j];
    cl::Dft<R, true, M1>::run(v);
#pragma unroll
    for (int i = 0; i < kHalf<M1, M2>; ++i) at[j + M2 * i] = v[i];   // x < n_x only
  }
  __syncthreads();
  constexpr int NW = (NT + 31) / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // partial x^T y (bilinear) when dotp is set: per thread and per warp in
  // the arithmetic's precision (FP32 for complex64: no FP64 work per
  // element), across warps in FP64
  R tr = (R)0, ti = (R)0;
  {
    const uint16_t* __restrict__ xi = lat.xi;
    const uint8_t* __restrict__ mt = lat.mat;
    for (int k0 = threadIdx.x; k0 < span; k0 += kGU * NT) {
      int xk[kGU], mk_[kGU];
#pragma unroll
      for (int u2 = 0; u2 < kGU; ++u2) {
        const int k = k0 + u2 * NT;
        if (k < span) {
          xk[u2] = xi[S0 + k];
          mk_[u2] = mt[S0 + k];
        }
      }
#pragma unroll
      for (int u2 = 0; u2 < kGU; ++u2) {
        const int k = k0 + u2 * NT;
        if (k < span) {
          const cpx<R> xv = vin<R>(k < kXS ? s_x[k] : xc[S0 + k]);
          cpx<R> v = xv;
          if (CONJ) v = conjg(v);
          cpx<R> o = v - beta[mk_[u2] * 3 + c] * a[row_of<T>(s_off, S0 + k) * LD + xk[u2]];
          if (CONJ) o = conjg(o);
          yc[S0 + k] = vstore(o);
          if (dotp) {
            tr = tr + (xv.x * o.x - xv.y * o.y);
            ti = ti + (xv.x * o.y + xv.y * o.x);
          }
        }
      }
    }
  }
  if (dotp) {
    // block partial of the product's input times its output, for the solver;
    // a trailing partial warp (NT % 32 threads, a power of two) reduces over
    // its own lanes only
    __shared__ double sd[2][NW];
    constexpr int kTail = NT % 32;
    static_assert((kTail & (kTail - 1)) == 0, "partial warp of a power-of-two size");
    const bool part = kTail != 0 && wid == NW - 1;
    const unsigned mask = part ? (1u << kTail) - 1u : 0xffffffffu;
    const int width = part ? kTail : 32;
    double dre, dim;
    if constexpr (std::is_same<R, float>::value) {
      float fr = tr, fi = ti;
      for (int o = width / 2; o > 0; o >>= 1) {
        fr += __shfl_down_sync(mask, fr, o, width);
        fi += __shfl_down_sync(mask, fi, o, width);
      }
      dre = fr;
      dim = fi;
    } else {
      dre = to_d(tr);
      dim = to_d(ti);
      for (int o = width / 2; o > 0; o >>= 1) {
        dre += __shfl_down_sync(mask, dre, o, width);
        dim += __shfl_down_sync(mask, dim, o, width);
      }
    }
    if (lane == 0) { sd[0][wid] = dre; sd[1][wid] = dim; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0.0, si = 0.0;
      for (int w = 0; w < NW; ++w) { sr += sd[0][w]; si += sd[1][w]; }
      const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
      dotp[2 * b] = sr;
      dotp[2 * b + 1] = si;
    }
  }
}

// ---------------------------------------------------------------- full x lines
// Whole contiguous lines of length M (no pruning): rows of in -> rows of out;
// grid (ceil(nrows/T)).  Used by the D-matrix build.  Row r of the launch is
// memory row (r / rows_y) * plane_rows + r % rows_y, so a sub-block of rows
// (y < rows_y in every plane) can be transformed.
template <typename R, int M1, int M2, int T>
__global__ void __launch_bounds__(T * kQ<M1, M2>, kMinB(T * kQ<M1, M2>, 3, 1)) fk_xfull(const cpx<R>* __restrict__ in,
                                                           cpx<R>* __restrict__ out, long long nrows,
                                                           int rows_y, long long plane_rows,
                                                           const cpx<R>* __restrict__ tw) {
  constexpr int M = M1 * M2, NT = T * kQ<M1, M2>, LD = kLD<M>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* s_tw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* a = s_tw + M;                      // [T][LD]
  const long long r0 = (long long)blockIdx.x * T;
  load_tw(s_tw, tw, M, NT);
  for (int idx = threadIdx.x; idx < T * M; idx += NT) {
    const int tt = idx / M, m = idx - tt * M;
    const long long r = r0 + tt;
    const long long mr = (r / rows_y) * plane_rows + r % rows_y;
    a[tt * LD + m] = r < nrows ? in[mr * M + m] : zero<R>();
  }
  __syncthreads();
  const int t = threadIdx.x % T, q = threadIdx.x / T;
  cpx<R>* at = a + t * LD;
  if (q < M2) {
    const int j = q;
    cpx<R> v[M1];
#pragma unroll
    for (int i = 0; i < M1; ++i) v[i] = at[j + M2 * i];
    cl::Dft<R, false, M1>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < M1; ++k1) v[k1] = twiddle<R, false>(v[k1], s_tw[j * k1]);
#pragma unroll
    for (int k1 = 0; k1 < M1; ++k1) at[k1 * M2 + j] = v[k1];
  }
  __syncthreads();
  cpx<R> u[M2];
  if (q < M1) {
    const int k1 = q;
#pragma unroll
    for (int j = 0; j < M2; ++j) u[j] = at[k1 * M2 + j];
    cl::Dft<R, false, M2>::run(u);
  }
  __syncthreads();
  if (q < M1) {
    const int k1 = q;
#pragma unroll
    for (int k2 = 0; k2 < M2; ++k2) at[k1 + M1 * k2] = u[k2];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < T * M; idx += NT) {
    const int tt = idx / M, m = idx - tt * M;
    const long long r = r0 + tt;
    const long long mr = (r / rows_y) * plane_rows + r % rows_y;
    if (r < nrows) out[mr * M + m] = a[tt * LD + m];
  }
}

// ---------------------------------------------------------------- launchers
template <typename R> constexpr int kT = sizeof(R) == 4 ? 16 : 8;
// rows per block of the x passes (fast_x_rows gives the same on the host)
template <typename R, int M> constexpr int kTX = (sizeof(R) == 4 && M >= 1000) ? 4 : kT<R>;

template <typename K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  return ensure_smem((const void*)kernel, bytes);
}

// Launches of one pass for a compile-time length; returns cudaErrorNotSupported
// for a length without a specialisation.
template <typename R, int M1, int M2>
struct Passes {
  static constexpr int M = M1 * M2, T = kT<R>, NT = T * kQ<M1, M2>;
  // rows per block of the x passes: 4 for the complex64 lines of 1000 points
  // and more (four blocks of 4.5 warps per SM; 16 rows of 1080 points would
  // take 147 KB, one block per SM)
  static constexpr int TX = kTX<R, M>, NTX = TX * kQ<M1, M2>;
  // columns per block of the fused z pass: the three spectra of TZ columns
  // must fit in shared memory (two blocks per SM where they can)
  static constexpr int TZ = (size_t)(M + 3 * M * T) * sizeof(cpx<R>) <= 113 * 1024 ? T
                           : (size_t)(M + 3 * M * (T / 2)) * sizeof(cpx<R>) <= 226 * 1024 ? T / 2
                           : T / 4;
  // Tile variants (lines per block) of the y passes and the z pass: 0 the
  // default, 1 half as many lines per block.  Every variant computes each line
  // with the same arithmetic, so the products agree bit for bit; the
  // autotuner picks one by timing.
  template <int TY>
  static cudaError_t yfwd_t(const cpx<R>* in, cpx<R>* out, int ny, int nz, int Mx,
                            const cpx<R>* tw, int nrhs, const int* skip, cudaStream_t st, bool pdl,
                            const int* yr) {
    const size_t sm = (size_t)(M + M * TY) * sizeof(cpx<R>);
    cudaError_t e = set_smem(fk_yfwd<R, M1, M2, TY, true>, sm);
    if (e != cudaSuccess) return e;
    e = launch_pdl(pdl, fk_yfwd<R, M1, M2, TY, true>, dim3((Mx + TY - 1) / TY, nz, 3 * nrhs),
                   dim3(TY * kQ<M1, M2>), sm, st, in, out, ny, nz, Mx, tw, 0, skip, 0LL, yr);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  static cudaError_t yfwd(const cpx<R>* in, cpx<R>* out, int ny, int nz, int Mx,
                          const cpx<R>* tw, int nrhs, const int* skip, cudaStream_t st, int var,
                          bool pdl, const int* yr) {
    return var == 1 ? yfwd_t<T / 2>(in, out, ny, nz, Mx, tw, nrhs, skip, st, pdl, yr)
                    : yfwd_t<T>(in, out, ny, nz, Mx, tw, nrhs, skip, st, pdl, yr);
  }
  template <int TY>
  static cudaError_t yinv_t(const cpx<R>* in, cpx<R>* out, int ny, int nz, int Mx,
                            const cpx<R>* tw, int nrhs, const int* skip, cudaStream_t st, bool pdl) {
    const size_t sm = (size_t)(M + M * TY) * sizeof(cpx<R>);
    cudaError_t e = set_smem(fk_yinv<R, M1, M2, TY>, sm);
    if (e != cudaSuccess) return e;
    e = launch_pdl(pdl, fk_yinv<R, M1, M2, TY>, dim3((Mx + TY - 1) / TY, nz, 3 * nrhs),
                   dim3(TY * kQ<M1, M2>), sm, st, in, out, ny, nz, Mx, tw, skip);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  static cudaError_t yinv(const cpx<R>* in, cpx<R>* out, int ny, int nz, int Mx,
                          const cpx<R>* tw, int nrhs, const int* skip, cudaStream_t st, int var,
                          bool pdl) {
    return var == 1 ? yinv_t<T / 2>(in, out, ny, nz, Mx, tw, nrhs, skip, st, pdl)
                    : yinv_t<T>(in, out, ny, nz, Mx, tw, nrhs, skip, st, pdl);
  }
  template <int TC>
  static cudaError_t zconv_t(cpx<R>* B2, const cpx<R>* D, int nz, int Mx, int My, const cpx<R>* tw,
                             int nrhs, const int* skip, cudaStream_t st, bool pdl) {
    const size_t sm = (size_t)(M + 3 * ZRows<R, M1, M2, TC>::rows * TC) * sizeof(cpx<R>);
    cudaError_t e = set_smem(fk_zconv<R, M1, M2, TC>, sm);
    if (e != cudaSuccess) return e;
    // two ~106 KB blocks per SM need the largest shared-memory carveout
    e = ensure_carveout_max((const void*)fk_zconv<R, M1, M2, TC>);
    if (e != cudaSuccess) return e;
    e = launch_pdl(pdl, fk_zconv<R, M1, M2, TC>, dim3((Mx + TC - 1) / TC, My, nrhs), dim3(TC * kQ<M1, M2>),
                   sm, st, B2, D, nz, Mx, My, tw, skip);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  static cudaError_t zconv(cpx<R>* B2, const cpx<R>* D, int nz, int Mx, int My, const cpx<R>* tw,
                           int nrhs, const int* skip, cudaStream_t st, int var, bool pdl) {
    return var == 1 ? zconv_t<TZ / 2>(B2, D, nz, Mx, My, tw, nrhs, skip, st, pdl)
                    : zconv_t<TZ>(B2, D, nz, Mx, My, tw, nrhs, skip, st, pdl);
  }
  using V = typename VecOf<R>::type;
  static cudaError_t xfwd(const V* x, cpx<R>* B1, const LatticeDev& lat, const cpx<R>* beta,
                          long long n_occ, int nrows, const cpx<R>* tw, bool adj, int nrhs,
                          int bstride, const int* skip, cudaStream_t st, bool pdl) {
    const size_t sm = (size_t)(M + TX * kLD<M>) * sizeof(cpx<R>);
    const int nr = lat.arow ? lat.nact : nrows;
    const dim3 grid((nr + TX - 1) / TX, 3 * nrhs);
    cudaError_t e;
    if (adj) {
      if ((e = set_smem(fk_xfwd<R, M1, M2, TX, true>, sm)) != cudaSuccess) return e;
      e = launch_pdl(pdl, fk_xfwd<R, M1, M2, TX, true>, grid, dim3(NTX), sm, st, x, B1, lat, beta, n_occ,
                     nrows, tw, bstride, skip);
    } else {
      if ((e = set_smem(fk_xfwd<R, M1, M2, TX, false>, sm)) != cudaSuccess) return e;
      e = launch_pdl(pdl, fk_xfwd<R, M1, M2, TX, false>, grid, dim3(NTX), sm, st, x, B1, lat, beta, n_occ,
                     nrows, tw, bstride, skip);
    }
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  // whole contiguous lines (rows of length M): rows y < rows_y of each plane
  // of plane_rows rows, nrows rows in all
  static cudaError_t xfull(const cpx<R>* in, cpx<R>* out, long long nrows, int rows_y,
                           long long plane_rows, const cpx<R>* tw, cudaStream_t st) {
    const size_t sm = (size_t)(M + T * kLD<M>) * sizeof(cpx<R>);
    cudaError_t e = set_smem(fk_xfull<R, M1, M2, T>, sm);
    if (e != cudaSuccess) return e;
    fk_xfull<R, M1, M2, T><<<(unsigned)((nrows + T - 1) / T), NT, sm, st>>>(in, out, nrows, rows_y,
                                                                          plane_rows, tw);
    count_launch();
    return cudaGetLastError();
  }
  // whole lines along a strided axis: element stride `stride`, lines 0..nlines-1
  // adjacent in memory, n_outer groups M*stride apart (the y pass kernel with
  // every input present); msign != 0 reads only elements <= M/2 and mirrors
  static cudaError_t sfull(const cpx<R>* in, cpx<R>* out, int nlines, int n_outer, int stride,
                           int msign, const cpx<R>* tw, cudaStream_t st, long long ostride) {
    const size_t sm = (size_t)(M + M * T) * sizeof(cpx<R>);
    cudaError_t e = set_smem(fk_yfwd<R, M1, M2, T, false>, sm);
    if (e != cudaSuccess) return e;
    fk_yfwd<R, M1, M2, T, false><<<dim3((nlines + T - 1) / T, n_outer, 1), NT, sm, st>>>(in, out, M, n_outer,
                                                                                 stride, tw, msign,
                                                                                 nullptr, ostride, nullptr);
    count_launch();
    return cudaGetLastError();
  }
  static cudaError_t xinv(const cpx<R>* B1, const V* x, V* y, const LatticeDev& lat,
                          const cpx<R>* beta, long long n_occ, int nrows, const cpx<R>* tw, bool adj,
                          double* dotp, int nrhs, int bstride, const int* skip, cudaStream_t st,
                          bool pdl) {
    const size_t sm = (size_t)(M + TX * kLD<M>) * sizeof(cpx<R>) + (size_t)TX * kXRow<M> * sizeof(V);
    const int nr = lat.arow ? lat.nact : nrows;
    const dim3 grid((nr + TX - 1) / TX, 3 * nrhs);
    cudaError_t e;
    // three blocks of up to ~56 KB per SM need a large shared-memory carveout
    if ((e = ensure_carveout_max((const void*)fk_xinv<R, M1, M2, TX, true>)) != cudaSuccess) return e;
    if ((e = ensure_carveout_max((const void*)fk_xinv<R, M1, M2, TX, false>)) != cudaSuccess) return e;
    if (adj) {
      if ((e = set_smem(fk_xinv<R, M1, M2, TX, true>, sm)) != cudaSuccess) return e;
      e = launch_pdl(pdl, fk_xinv<R, M1, M2, TX, true>, grid, dim3(NTX), sm, st, B1, x, y, lat, beta, n_occ,
                     nrows, tw, dotp, bstride, skip);
    } else {
      if ((e = set_smem(fk_xinv<R, M1, M2, TX, false>, sm)) != cudaSuccess) return e;
      e = launch_pdl(pdl, fk_xinv<R, M1, M2, TX, false>, grid, dim3(NTX), sm, st, B1, x, y, lat, beta,
                     n_occ, nrows, tw, dotp, bstride, skip);
    }
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
  }
};

}  // namespace fast
}  // namespace dda
