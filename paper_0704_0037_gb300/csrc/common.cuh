// Shared device helpers: complex arithmetic in float/double, launch sizing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dda {

template <typename R> struct cpx;
template <> struct __align__(8) cpx<float> { float x, y; };
template <> struct __align__(16) cpx<double> { double x, y; };

using c64 = cpx<float>;
using c128 = cpx<double>;

template <typename R> __host__ __device__ __forceinline__ cpx<R> mk(R a, R b) {
  cpx<R> r; r.x = a; r.y = b; return r;
}
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x + b.x, a.y + b.y);
}
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x - b.x, a.y - b.y);
}
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R> __host__ __device__ __forceinline__ cpx<R> scale(cpx<R> a, R s) {
  return mk<R>(a.x * s, a.y * s);
}
template <typename R> __host__ __device__ __forceinline__ cpx<R> conjg(cpx<R> a) { return mk<R>(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <typename R, bool INV> __host__ __device__ __forceinline__ cpx<R> mul_mi(cpx<R> a) {
  return INV ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x);
}
// a * conj(w) when INV else a * w  (twiddles are stored for the forward sign)
template <typename R, bool INV> __host__ __device__ __forceinline__ cpx<R> twiddle(cpx<R> a, cpx<R> w) {
  return INV ? mk<R>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y)
             : mk<R>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

template <typename R> __host__ __device__ __forceinline__ cpx<R> cvt(c128 a) {
  return mk<R>((R)a.x, (R)a.y);
}

__host__ __device__ __forceinline__ c128 to128(c64 a) { return mk<double>(a.x, a.y); }
__host__ __device__ __forceinline__ c128 to128(c128 a) { return a; }

}  // namespace dda
