// GPU check of the double-float arithmetic (common.cuh): complex sums,
// products, real scaling and fused multiply-add of double-float numbers on
// the device, in the paired FP32 form and the scalar form, against FP64
// results of the same inputs.  Prints the largest relative error of each
// operation (sums relative to |a| + |b|, products to |a| |b|).
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "common.cuh"

using namespace dda;

__global__ void k_ops(const double* in, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cdf a = to_cdf(mk<double>(in[4 * i], in[4 * i + 1]));
  const cdf b = to_cdf(mk<double>(in[4 * i + 2], in[4 * i + 3]));
  const cdf r[7] = {a + b, a - b, a * b, scale<df>(a, b.x), fmas<df>(a, b.x, b),
                    mk<df>(a.x + b.x, a.y + b.y),
                    mk<df>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x)};
  for (int k = 0; k < 7; ++k) {
    const c128 v = to128(r[k]);
    out[14 * i + 2 * k] = v.x;
    out[14 * i + 2 * k + 1] = v.y;
  }
}

int main() {
  const int n = 4096;
  std::mt19937_64 gen(7);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::vector<double> h(4 * n), o(14 * n);
  for (auto& v : h) v = nd(gen) * std::exp(nd(gen));
  double *di = nullptr, *dout = nullptr;
  if (cudaMalloc(&di, h.size() * 8) != cudaSuccess || cudaMalloc(&dout, o.size() * 8) != cudaSuccess) return 2;
  cudaMemcpy(di, h.data(), h.size() * 8, cudaMemcpyHostToDevice);
  k_ops<<<(n + 127) / 128, 128>>>(di, dout, n);
  if (cudaMemcpy(o.data(), dout, o.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
  const char* names[7] = {"add", "sub", "mul", "scale", "fmas", "add_scalar", "mul_scalar"};
  double worst[7] = {0};
  for (int i = 0; i < n; ++i) {
    const double ar = h[4 * i], ai = h[4 * i + 1], br = h[4 * i + 2], bi = h[4 * i + 3];
    const double na = std::hypot(ar, ai), nb = std::hypot(br, bi);
    const double ref[7][3] = {{ar + br, ai + bi, na + nb}, {ar - br, ai - bi, na + nb},
                              {ar * br - ai * bi, ar * bi + ai * br, na * nb},
                              {ar * br, ai * br, na * std::fabs(br)},
                              {ar * br + br, ai * br + bi, na * std::fabs(br) + nb},
                              {ar + br, ai + bi, na + nb},
                              {ar * br - ai * bi, ar * bi + ai * br, na * nb}};
    for (int k = 0; k < 7; ++k) {
      const double e = std::hypot(o[14 * i + 2 * k] - ref[k][0], o[14 * i + 2 * k + 1] - ref[k][1]) / ref[k][2];
      if (e > worst[k]) worst[k] = e;
    }
  }
  for (int k = 0; k < 7; ++k) std::printf("%s %.6e\n", names[k], worst[k]);
  cudaFree(di);
  cudaFree(dout);
  return 0;
}
