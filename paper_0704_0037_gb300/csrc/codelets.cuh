// Register-resident DFT codelets of compile-time length N.
//
// Dft<R, INV, N>::run(v) transforms v[0..N-1] in place (forward
// X_k = sum_n x_n exp(-2 pi i n k / N); INV uses the conjugate, no 1/N).
// Lengths 2, 3, 4, 5, 7, 8 are the butterflies of fft.cuh; other lengths are
// composed at compile time:
//  * N = A B with gcd(A, B) = 1: Good-Thomas prime-factor mapping
//    n = (B n1 + A n2) mod N, k = (k1 e_A + k2 e_B) mod N with
//    e_A = 1 mod A, 0 mod B and e_B = 0 mod A, 1 mod B -- no twiddles;
//  * N = A B a prime power: Cooley-Tukey, n = j + B i, k = k1 + A k2, with
//    twiddles exp(-2 pi i j k1 / N) that are compile-time constants.
// All indices are compile-time after unrolling, so the arrays stay in
// registers.  The twiddle constants come from a constexpr Taylor series of
// sin/cos on [0, pi/4] after an exact rational reduction of 2 pi p/q.
#pragma once

#include <utility>

#include "common.cuh"
#include "fft.cuh"

namespace dda {
namespace cl {

constexpr double kTwoPi = 6.283185307179586476925286766559;

constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 13; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}

constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 13; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}

struct CS { double c, s; };

// cos and sin of 2 pi p / q: reflect the angle into [0, pi/4] with exact
// integer arithmetic, then sum the series.
constexpr CS cs2pi(long long p, long long q) {
  p %= q;
  if (p < 0) p += q;
  double sc = 1.0, ss = 1.0;
  if (2 * p > q) { p = q - p; ss = -ss; }                   // a -> 1 - a
  if (4 * p > q) { p = q - 2 * p; q = 2 * q; sc = -sc; }    // a -> 1/2 - a
  bool swap = false;
  if (8 * p > q) { p = q - 4 * p; q = 4 * q; swap = true; } // a -> 1/4 - a
  const double x = kTwoPi * (double)p / (double)q;
  double c = taylor_cos(x), s = taylor_sin(x);
  if (swap) { const double t = c; c = s; s = t; }
  return CS{sc * c, ss * s};
}

template <int P, int Q> constexpr double kCos = cs2pi(P, Q).c;
template <int P, int Q> constexpr double kSin = cs2pi(P, Q).s;

// z * w_N^M with w_N = exp(-2 pi i / N) (forward) or its conjugate (INV)
template <typename R, bool INV, int M, int N>
__host__ __device__ __forceinline__ cpx<R> tw_mul(cpx<R> z) {
  constexpr int m = ((M % N) + N) % N;
  if constexpr (m == 0) {
    return z;
  } else if constexpr (2 * m == N) {
    return mk<R>(-z.x, -z.y);
  } else if constexpr (4 * m == N) {
    return mul_mi<R, INV>(z);
  } else if constexpr (4 * m == 3 * N) {
    return mul_mi<R, !INV>(z);
  } else {
    constexpr R c = (R)kCos<m, N>;
    constexpr R s = INV ? (R)kSin<m, N> : (R)(-kSin<m, N>);
    return z * mk<R>(c, s);
  }
}

constexpr int smallest_prime(int n) {
  for (int p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

constexpr int prime_power_part(int n) {
  const int p = smallest_prime(n);
  int a = 1;
  while (n % p == 0) { n /= p; a *= p; }
  return a;
}

// first factor of a prime-power length for Cooley-Tukey
constexpr int ct_radix(int n) {
  if (n % 2 == 0) {
    if (n == 16 || n == 32) return 4;
    if (n % 8 == 0) return 8;
    if (n % 4 == 0) return 4;
    return 2;
  }
  return smallest_prime(n);
}

constexpr int modinv(int a, int m) {
  a %= m;
  for (int x = 1; x < m; ++x)
    if ((a * x) % m == 1) return x;
  return 1;
}

template <typename R, bool INV, int N> struct Dft;

template <typename R, bool INV> struct Dft<R, INV, 1> {
  static __host__ __device__ __forceinline__ void run(cpx<R>*) {}
};
template <typename R, bool INV> struct Dft<R, INV, 2> {
  static __host__ __device__ __forceinline__ void run(cpx<R>* v) { bfly2<R, INV>(v[0], v[1]); }
};
template <typename R, bool INV> struct Dft<R, INV, 3> {
  static __host__ __device__ __forceinline__ void run(cpx<R>* v) { bfly3<R, INV>(v[0], v[1], v[2]); }
};
template <typename R, bool INV> struct Dft<R, INV, 4> {
  static __host__ __device__ __forceinline__ void run(cpx<R>* v) { bfly4<R, INV>(v[0], v[1], v[2], v[3]); }
};
template <typename R, bool INV> struct Dft<R, INV, 5> {
  static __host__ __device__ __forceinline__ void run(cpx<R>* v) { bfly5<R, INV>(v); }
};
template <typename R, bool INV> struct Dft<R, INV, 7> {
  static __host__ __device__ __forceinline__ void run(cpx<R>* v) { bfly7<R, INV>(v); }
};
template <typename R, bool INV> struct Dft<R, INV, 8> {
  static __host__ __device__ __forceinline__ void run(cpx<R>* v) { bfly8<R, INV>(v); }
};

template <typename R, bool INV, int N, int A, int... I>
__host__ __device__ __forceinline__ void tw_all(cpx<R>* t, std::integer_sequence<int, I...>) {
  ((t[I] = tw_mul<R, INV, (I / A) * (I % A), N>(t[I])), ...);
}

// Good-Thomas, gcd(A, B) = 1
template <typename R, bool INV, int A, int B>
__host__ __device__ __forceinline__ void pfa(cpx<R>* v) {
  constexpr int N = A * B;
  cpx<R> t[N];
#pragma unroll
  for (int n1 = 0; n1 < A; ++n1)
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) t[n2 * A + n1] = v[(B * n1 + A * n2) % N];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) Dft<R, INV, A>::run(t + n2 * A);
  cpx<R> u[N];
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1)
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) u[k1 * B + n2] = t[n2 * A + k1];
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) Dft<R, INV, B>::run(u + k1 * B);
  constexpr int eA = B * modinv(B, A);
  constexpr int eB = A * modinv(A, B);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[(k1 * eA + k2 * eB) % N] = u[k1 * B + k2];
}

// Cooley-Tukey, n = j + B i (i < A), k = k1 + A k2 (k2 < B)
template <typename R, bool INV, int A, int B>
__host__ __device__ __forceinline__ void ct(cpx<R>* v) {
  constexpr int N = A * B;
  cpx<R> t[N];
#pragma unroll
  for (int j = 0; j < B; ++j)
#pragma unroll
    for (int i = 0; i < A; ++i) t[j * A + i] = v[j + B * i];
#pragma unroll
  for (int j = 0; j < B; ++j) Dft<R, INV, A>::run(t + j * A);
  tw_all<R, INV, N, A>(t, std::make_integer_sequence<int, N>{});
  cpx<R> u[N];
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1)
#pragma unroll
    for (int j = 0; j < B; ++j) u[k1 * B + j] = t[j * A + k1];
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) Dft<R, INV, B>::run(u + k1 * B);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = u[k1 * B + k2];
}

template <typename R, bool INV, int N>
struct Dft {
  static __host__ __device__ __forceinline__ void run(cpx<R>* v) {
    constexpr int A = prime_power_part(N);
    if constexpr (A != N) {
      pfa<R, INV, A, N / A>(v);
    } else {
      constexpr int a = ct_radix(N);
      ct<R, INV, a, N / a>(v);
    }
  }
};

}  // namespace cl
}  // namespace dda
