// Host-side check of the register DFT codelets against the DFT definition
// (direct O(N^2) sum in long double).  Prints one line per (length,
// precision, direction): "N prec dir max_rel_error".
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "codelets.cuh"

using namespace dda;

template <typename R, bool INV, int N>
void check(const char* pname) {
  cpx<R> v[N];
  long double xr[N], xi[N];
  unsigned s = 12345u + N;
  for (int n = 0; n < N; ++n) {
    s = s * 1103515245u + 12345u; double a = ((s >> 8) & 0xffff) / 65536.0 - 0.5;
    s = s * 1103515245u + 12345u; double b = ((s >> 8) & 0xffff) / 65536.0 - 0.5;
    v[n] = mk<R>((R)a, (R)b);
    xr[n] = (long double)v[n].x; xi[n] = (long double)v[n].y;
  }
  cl::Dft<R, INV, N>::run(v);
  const long double tp = 6.283185307179586476925286766559L;
  long double err = 0, nrm = 0;
  for (int k = 0; k < N; ++k) {
    long double sr = 0, si = 0;
    for (int n = 0; n < N; ++n) {
      long double a = tp * (long double)((long long)n * k % N) / N;
      long double c = cosl(a), sn = INV ? sinl(a) : -sinl(a);
      sr += xr[n] * c - xi[n] * sn;
      si += xr[n] * sn + xi[n] * c;
    }
    long double dr = sr - v[k].x, di = si - v[k].y;
    err += dr * dr + di * di;
    nrm += sr * sr + si * si;
  }
  std::printf("%d %s %s %.3Le\n", N, pname, INV ? "inv" : "fwd", sqrtl(err / nrm));
}

template <int N>
void both() {
  check<double, false, N>("f64");
  check<double, true, N>("f64");
  check<float, false, N>("f32");
  check<float, true, N>("f32");
}

int main() {
  both<2>(); both<3>(); both<4>(); both<5>(); both<6>(); both<7>(); both<8>(); both<9>();
  both<10>(); both<12>(); both<15>(); both<16>(); both<18>(); both<20>(); both<24>();
  both<25>(); both<27>(); both<30>(); both<32>(); both<36>(); both<45>(); both<64>();
  return 0;
}
