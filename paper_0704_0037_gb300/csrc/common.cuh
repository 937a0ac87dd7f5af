// Shared device helpers: complex arithmetic in float/double, launch sizing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dda {

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialization (launch_pdl) may start before the kernel
// ahead of it on its stream has finished; it calls pdl_wait() before touching
// anything that kernel wrote (the wait returns once it has completed and its
// writes are visible).  pdl_launch() lets the next such kernel be scheduled
// as soon as every block of this one has called it.  Both are no-ops in an
// ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }


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
  return INV ? a * conjg(w) : a * w;
}

// a * s + c for complex a, c and real s
template <typename R> __host__ __device__ __forceinline__ cpx<R> fmas(cpx<R> a, R s, cpx<R> c) {
  return mk<R>(a.x * s + c.x, a.y * s + c.y);
}

// Complex64 on sm_100-class devices: a complex number is one 64-bit register
// pair and the componentwise add / sub / real-scale / real-fma map to the
// paired FP32 instructions (add, sub, mul, fma with type .f32x2), one
// instruction per complex operation instead of two.  Each lane is rounded
// exactly as the scalar instruction would be.
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && !defined(DDA_NO_F32X2)
#define DDA_F32X2 1
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ c64 upk2(unsigned long long r) {
  c64 o;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
  return o;
}
#endif

template <> __host__ __device__ __forceinline__ c64 operator+<float>(c64 a, c64 b) {
#ifdef DDA_F32X2
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
  return upk2(r);
#else
  return mk<float>(a.x + b.x, a.y + b.y);
#endif
}
template <> __host__ __device__ __forceinline__ c64 operator-<float>(c64 a, c64 b) {
#ifdef DDA_F32X2
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
  return upk2(r);
#else
  return mk<float>(a.x - b.x, a.y - b.y);
#endif
}
template <> __host__ __device__ __forceinline__ c64 scale<float>(c64 a, float s) {
#ifdef DDA_F32X2
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a.x, a.y)), "l"(pk2(s, s)));
  return upk2(r);
#else
  return mk<float>(a.x * s, a.y * s);
#endif
}
template <> __host__ __device__ __forceinline__ c64 fmas<float>(c64 a, float s, c64 c) {
#ifdef DDA_F32X2
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk2(a.x, a.y)), "l"(pk2(s, s)),
      "l"(pk2(c.x, c.y)));
  return upk2(r);
#else
  return mk<float>(fmaf(a.x, s, c.x), fmaf(a.y, s, c.y));
#endif
}

// ---------------------------------------------------------------- double-float
// A real number carried as an unevaluated sum hi + lo of two floats
// (|lo| <= ulp(hi)/2), about 48 significant bits; the FP32 pipe runs the
// arithmetic.  The algorithms are the classical error-free transformations:
// Knuth's two-sum for the rounding error of a sum, Dekker's fast two-sum to
// renormalise, and the exact product error a*b - fl(a*b) from one fused
// multiply-add.  Sum and product use the cheap ("sloppy") double-word forms:
// their error is a small multiple of 2^-46 relative to the operands' magnitude,
// which is the error an FFT's rounding analysis needs.  Used for the FP64-class
// products (the refinement residual, the D-matrix build) on parts whose FP64
// pipe is a small fraction of the FP32 one.
struct __align__(8) df {
  float hi, lo;
  __host__ __device__ constexpr df() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // split of a double (compile-time constants, table entries)
  __host__ __device__ constexpr explicit df(double v)
      : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

#if defined(__CUDA_ARCH__)
#define DDA_FADD(a, b) __fadd_rn((a), (b))
#define DDA_FSUB(a, b) __fsub_rn((a), (b))
#define DDA_FMUL(a, b) __fmul_rn((a), (b))
#define DDA_FFMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
#define DDA_FADD(a, b) ((a) + (b))
#define DDA_FSUB(a, b) ((a) - (b))
#define DDA_FMUL(a, b) ((a) * (b))
#define DDA_FFMA(a, b, c) fmaf((a), (b), (c))
#endif

__host__ __device__ __forceinline__ df operator+(df a, df b) {
  const float s = DDA_FADD(a.hi, b.hi);
  const float bb = DDA_FSUB(s, a.hi);
  float e = DDA_FADD(DDA_FSUB(a.hi, DDA_FSUB(s, bb)), DDA_FSUB(b.hi, bb));   // two-sum error
  e = DDA_FADD(e, DDA_FADD(a.lo, b.lo));
  const float h = DDA_FADD(s, e);
  return df(h, DDA_FSUB(e, DDA_FSUB(h, s)));                                 // fast two-sum
}
__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__host__ __device__ __forceinline__ df operator*(df a, df b) {
  const float p = DDA_FMUL(a.hi, b.hi);
  float e = DDA_FFMA(a.hi, b.hi, -p);                                        // exact product error
  e = DDA_FFMA(a.hi, b.lo, e);
  e = DDA_FFMA(a.lo, b.hi, e);
  const float h = DDA_FADD(p, e);
  return df(h, DDA_FSUB(e, DDA_FSUB(h, p)));
}

template <> struct __align__(16) cpx<df> { df x, y; };
using cdf = cpx<df>;

// Complex double-float on sm_100-class devices: the two real parts' high
// words form one f32x2 register pair and the low words another, so each step
// of the double-float algorithms above runs once for both parts (the same
// roundings per part as the scalar form).
#ifdef DDA_F32X2
struct df2 { unsigned long long h, l; };   // (re.hi, im.hi), (re.lo, im.lo)
__device__ __forceinline__ unsigned long long f2add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2fma(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ df2 dpack(const cpx<df>& a) {
  return df2{pk2(a.x.hi, a.y.hi), pk2(a.x.lo, a.y.lo)};
}
__device__ __forceinline__ cpx<df> dunpack(df2 p) {
  const c64 h = upk2(p.h), l = upk2(p.l);
  cpx<df> r;
  r.x = df(h.x, l.x);
  r.y = df(h.y, l.y);
  return r;
}
// Componentwise double-float sum and difference of the two parts, without
// the final renormalisation: the result (s, e) is the two-sum of the high
// words with the low words' sum added to its error term.  It represents the
// same value as the renormalised sum (which only redistributes s + e between
// the words), but e may exceed ulp(s) / 2.  Every product renormalises its
// result, so between two products the low word stays within a few ulp of the
// operands' magnitude (a DFT codelet chains a few sums at most), and the
// error stays a small multiple of 2^-46 of the operands' magnitude; long
// accumulations do not use these.
__device__ __forceinline__ df2 dadd2(df2 a, df2 b) {
  const unsigned long long s = f2add(a.h, b.h);
  const unsigned long long bb = f2sub(s, a.h);
  const unsigned long long e = f2add(f2sub(a.h, f2sub(s, bb)), f2sub(b.h, bb));
  return df2{s, f2add(e, f2add(a.l, b.l))};
}
__device__ __forceinline__ df2 dsub2(df2 a, df2 b) {
  const unsigned long long s = f2sub(a.h, b.h);
  const unsigned long long bb = f2sub(s, a.h);
  const unsigned long long e = f2sub(f2sub(a.h, f2sub(s, bb)), f2add(b.h, bb));
  return df2{s, f2add(e, f2sub(a.l, b.l))};
}
__device__ __forceinline__ df2 dmul2(df2 a, df2 b) {
  // The rounded product comes from an fma with a zero addend the compiler
  // cannot see through (a - a): a paired multiply followed by the paired add
  // below may otherwise be contracted into one fused operation, which adds
  // the product's rounding error a second time.
  const unsigned long long z = f2sub(a.h, a.h);
  const unsigned long long p = f2fma(a.h, b.h, z);
  unsigned long long e = f2fma(a.h, b.h, f2sub(0ull, p));
  e = f2fma(a.h, b.l, e);
  e = f2fma(a.l, b.h, e);
  const unsigned long long h = f2add(p, e);
  return df2{h, f2sub(e, f2sub(h, p))};
}
// the pair (v, v) of a double-float scalar
__device__ __forceinline__ df2 dsplat(df v) { return df2{pk2(v.hi, v.hi), pk2(v.lo, v.lo)}; }
// multiply the first part by -1 (exact)
__device__ __forceinline__ df2 dneg_re(df2 a) {
  const unsigned long long m = pk2(-1.0f, 1.0f);
  return df2{f2mul(a.h, m), f2mul(a.l, m)};
}
// (a + ib)(c + id) = (ac - bd) + i(ad + bc): (ac, ad) + (-bd, bc)
__device__ __forceinline__ cpx<df> dcmul(const cpx<df>& z, const cpx<df>& w) {
  const df2 wp = dpack(w);
  const df2 ws{pk2(w.y.hi, w.x.hi), pk2(w.y.lo, w.x.lo)};
  const df2 p1 = dmul2(dsplat(z.x), wp);
  const df2 p2 = dmul2(dsplat(z.y), ws);
  return dunpack(dadd2(p1, dneg_re(p2)));
}
#endif

template <> __host__ __device__ __forceinline__ cpx<df> operator+<df>(cpx<df> a, cpx<df> b) {
#ifdef DDA_F32X2
  return dunpack(dadd2(dpack(a), dpack(b)));
#else
  return mk<df>(a.x + b.x, a.y + b.y);
#endif
}
template <> __host__ __device__ __forceinline__ cpx<df> operator-<df>(cpx<df> a, cpx<df> b) {
#ifdef DDA_F32X2
  return dunpack(dsub2(dpack(a), dpack(b)));
#else
  return mk<df>(a.x - b.x, a.y - b.y);
#endif
}
template <> __host__ __device__ __forceinline__ cpx<df> operator*<df>(cpx<df> a, cpx<df> b) {
#ifdef DDA_F32X2
  return dcmul(a, b);
#else
  return mk<df>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
#endif
}
template <> __host__ __device__ __forceinline__ cpx<df> scale<df>(cpx<df> a, df s) {
#ifdef DDA_F32X2
  return dunpack(dmul2(dpack(a), dsplat(s)));
#else
  return mk<df>(a.x * s, a.y * s);
#endif
}
template <> __host__ __device__ __forceinline__ cpx<df> fmas<df>(cpx<df> a, df s, cpx<df> c) {
#ifdef DDA_F32X2
  return dunpack(dadd2(dmul2(dpack(a), dsplat(s)), dpack(c)));
#else
  return mk<df>(a.x * s + c.x, a.y * s + c.y);
#endif
}

__host__ __device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ c128 to128(cdf a) {
  return mk<double>(df_to_double(a.x), df_to_double(a.y));
}
__host__ __device__ __forceinline__ cdf to_cdf(c128 a) { return mk<df>(df(a.x), df(a.y)); }

template <typename R> __host__ __device__ __forceinline__ cpx<R> cvt(c128 a) {
  return mk<R>((R)a.x, (R)a.y);
}

__host__ __device__ __forceinline__ c128 to128(c64 a) { return mk<double>(a.x, a.y); }
__host__ __device__ __forceinline__ c128 to128(c128 a) { return a; }

}  // namespace dda
