// Batched 1D mixed-radix FFT of T lines held in shared memory.
//
// The interaction-matrix product is an FFT convolution split into 1D
// transforms (arXiv:0704.0037, Sec. 2, performance paragraph).  Each CTA
// holds T lines of length M in shared memory, element (m, t) at
// buf[m*ldm + t], and runs a self-sorting (Stockham) radix-r sequence over
// them: stage s with radix r and Ns = product of the earlier radices maps
// element j + i*M/r (i < r) to (j/Ns)*Ns*r + j%Ns + i*Ns after twiddling by
// w_M^{i*(j%Ns)*M/(Ns*r)} and an r-point DFT.  Forward transforms use
// exp(-2 pi i jk/M); inverse transforms use the conjugate and no 1/M scale.
// Radix-2/3/4/5/7/8 butterflies are written out below from the DFT
// definition; their constants are cos/sin of 2 pi k/r.
#pragma once

#include "common.cuh"

namespace dda {

constexpr int kMaxStages = 24;

struct FftPlan {
  int M;                     // transform length
  int nst;                   // number of stages
  int radix[kMaxStages];     // radix of each stage (2, 3, 4, 5, 7 or 8)
};

// cos/sin(2 pi k / r) for the odd-prime butterflies
#define DDA_S3 0.8660254037844386467637232
#define DDA_C51 0.3090169943749474241022934
#define DDA_S51 0.9510565162951535721164393
#define DDA_C52 (-0.8090169943749474241022934)
#define DDA_S52 0.5877852522924731291687060
#define DDA_C71 0.6234898018587335305250049
#define DDA_S71 0.7818314824680298087084445
#define DDA_C72 (-0.2225209339563144042889026)
#define DDA_S72 0.9749279121818236070181317
#define DDA_C73 (-0.9009688679024191262361023)
#define DDA_S73 0.4338837391175581204757683
#define DDA_R2 0.7071067811865475244008444

template <typename R, bool INV>
__host__ __device__ __forceinline__ void bfly2(cpx<R>& a, cpx<R>& b) {
  cpx<R> t = a - b;
  a = a + b;
  b = t;
}

template <typename R, bool INV>
__host__ __device__ __forceinline__ void bfly3(cpx<R>& a, cpx<R>& b, cpx<R>& c) {
  cpx<R> t = b + c;
  cpx<R> d = fmas<R>(t, (R)-0.5, a);
  cpx<R> e = mul_mi<R, INV>(scale<R>(b - c, (R)DDA_S3));
  a = a + t;
  b = d + e;
  c = d - e;
}

template <typename R, bool INV>
__host__ __device__ __forceinline__ void bfly4(cpx<R>& a, cpx<R>& b, cpx<R>& c, cpx<R>& d) {
  cpx<R> s0 = a + c, s1 = a - c, s2 = b + d;
  cpx<R> s3 = mul_mi<R, INV>(b - d);
  a = s0 + s2;
  c = s0 - s2;
  b = s1 + s3;
  d = s1 - s3;
}

template <typename R, bool INV>
__host__ __device__ __forceinline__ void bfly5(cpx<R>* v) {
  cpx<R> t1 = v[1] + v[4], t2 = v[2] + v[3], t3 = v[1] - v[4], t4 = v[2] - v[3];
  cpx<R> a1 = fmas<R>(t2, (R)DDA_C52, fmas<R>(t1, (R)DDA_C51, v[0]));
  cpx<R> a2 = fmas<R>(t2, (R)DDA_C51, fmas<R>(t1, (R)DDA_C52, v[0]));
  cpx<R> b1 = mul_mi<R, INV>(fmas<R>(t4, (R)DDA_S52, scale<R>(t3, (R)DDA_S51)));
  cpx<R> b2 = mul_mi<R, INV>(fmas<R>(t4, (R)(-DDA_S51), scale<R>(t3, (R)DDA_S52)));
  v[0] = v[0] + t1 + t2;
  v[1] = a1 + b1;
  v[4] = a1 - b1;
  v[2] = a2 + b2;
  v[3] = a2 - b2;
}

template <typename R, bool INV>
__host__ __device__ __forceinline__ void bfly7(cpx<R>* v) {
  cpx<R> t1 = v[1] + v[6], t2 = v[2] + v[5], t3 = v[3] + v[4];
  cpx<R> u1 = v[1] - v[6], u2 = v[2] - v[5], u3 = v[3] - v[4];
  cpx<R> x0 = v[0];
  cpx<R> a1 = fmas<R>(t3, (R)DDA_C73, fmas<R>(t2, (R)DDA_C72, fmas<R>(t1, (R)DDA_C71, x0)));
  cpx<R> a2 = fmas<R>(t3, (R)DDA_C71, fmas<R>(t2, (R)DDA_C73, fmas<R>(t1, (R)DDA_C72, x0)));
  cpx<R> a3 = fmas<R>(t3, (R)DDA_C72, fmas<R>(t2, (R)DDA_C71, fmas<R>(t1, (R)DDA_C73, x0)));
  cpx<R> b1 = mul_mi<R, INV>(fmas<R>(u3, (R)DDA_S73, fmas<R>(u2, (R)DDA_S72, scale<R>(u1, (R)DDA_S71))));
  cpx<R> b2 = mul_mi<R, INV>(fmas<R>(u3, (R)(-DDA_S71), fmas<R>(u2, (R)(-DDA_S73), scale<R>(u1, (R)DDA_S72))));
  cpx<R> b3 = mul_mi<R, INV>(fmas<R>(u3, (R)DDA_S72, fmas<R>(u2, (R)(-DDA_S71), scale<R>(u1, (R)DDA_S73))));
  v[0] = x0 + t1 + t2 + t3;
  v[1] = a1 + b1; v[6] = a1 - b1;
  v[2] = a2 + b2; v[5] = a2 - b2;
  v[3] = a3 + b3; v[4] = a3 - b3;
}

// z * w8^k, w8 = exp(-i pi/4) (forward) or its conjugate (inverse)
// (w8^1 = (1 -+ i)/sqrt2, w8^3 = (-1 -+ i)/sqrt2: z w8^1 = (z + mul_mi(z))/sqrt2,
// z w8^3 = (mul_mi(z) - z)/sqrt2)
template <typename R, bool INV, int K>
__host__ __device__ __forceinline__ cpx<R> rot8(cpx<R> z) {
  const R r2 = (R)DDA_R2;
  if (K == 1) return scale<R>(z + mul_mi<R, INV>(z), r2);
  if (K == 2) return mul_mi<R, INV>(z);
  // K == 3
  return scale<R>(mul_mi<R, INV>(z) - z, r2);
}

template <typename R, bool INV>
__host__ __device__ __forceinline__ void bfly8(cpx<R>* v) {
  cpx<R> a0 = v[0] + v[4], a1 = v[1] + v[5], a2 = v[2] + v[6], a3 = v[3] + v[7];
  cpx<R> b0 = v[0] - v[4];
  cpx<R> b1 = rot8<R, INV, 1>(v[1] - v[5]);
  cpx<R> b2 = rot8<R, INV, 2>(v[2] - v[6]);
  cpx<R> b3 = rot8<R, INV, 3>(v[3] - v[7]);
  bfly4<R, INV>(a0, a1, a2, a3);
  bfly4<R, INV>(b0, b1, b2, b3);
  v[0] = a0; v[2] = a1; v[4] = a2; v[6] = a3;
  v[1] = b0; v[3] = b1; v[5] = b2; v[7] = b3;
}

template <typename R, bool INV>
__device__ __forceinline__ void dft_r(int r, cpx<R>* v) {
  switch (r) {
    case 2: bfly2<R, INV>(v[0], v[1]); break;
    case 3: bfly3<R, INV>(v[0], v[1], v[2]); break;
    case 4: bfly4<R, INV>(v[0], v[1], v[2], v[3]); break;
    case 5: bfly5<R, INV>(v); break;
    case 7: bfly7<R, INV>(v); break;
    case 8: bfly8<R, INV>(v); break;
    default: break;
  }
}

// Run all stages of plan p over T = 1 << logT lines; data starts in buf0.
// Returns the buffer that holds the result (buf0 or buf1).  Caller must
// __syncthreads() before (data in buf0 complete); this returns after a barrier.
template <typename R, bool INV>
__device__ cpx<R>* stockham(cpx<R>* buf0, cpx<R>* buf1, int ldm, int logT, const FftPlan& p,
                            const cpx<R>* __restrict__ tw) {
  const int M = p.M;
  const int Tm = (1 << logT) - 1;
  cpx<R>* src = buf0;
  cpx<R>* dst = buf1;
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int r = p.radix[s];
    const int Mr = M / r;
    const int tws = M / (Ns * r);
    const int items = Mr << logT;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int t = it & Tm;
      const int j = it >> logT;
      const int k = j % Ns;
      cpx<R> v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < r) v[i] = src[(j + i * Mr) * ldm + t];
      if (k != 0) {
#pragma unroll
        for (int i = 1; i < 8; ++i)
          if (i < r) v[i] = twiddle<R, INV>(v[i], tw[i * k * tws]);
      }
      dft_r<R, INV>(r, v);
      const int base = (j - k) * r + k;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i < r) dst[(base + i * Ns) * ldm + t] = v[i];
    }
    __syncthreads();
    cpx<R>* tmp = src; src = dst; dst = tmp;
    Ns *= r;
  }
  return src;
}

}  // namespace dda
