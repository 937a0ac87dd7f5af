// Register-resident product passes for M = 32 = 4 x 8, 64 = 8 x 8 and
// 128 = 8 x 16 (the 16^3, 32^3 and 64^3 spheres), and the length dispatch.
#include "fast_impl.cuh"

namespace dda {

template <typename R> cudaError_t fast_pass_small(int M, int pass, const FastArgs& a) {
  switch (M) {
    case 32: return fast::run_pass<R, 4, 8>(pass, a);
    case 64: return fast::run_pass<R, 8, 8>(pass, a);
    case 128: return fast::run_pass<R, 8, 16>(pass, a);
  }
  return cudaErrorNotSupported;
}
template cudaError_t fast_pass_small<float>(int, int, const FastArgs&);
template cudaError_t fast_pass_small<double>(int, int, const FastArgs&);

bool fast_supported(int M) {
  return M == 32 || M == 40 || M == 48 || M == 64 || M == 80 || M == 96 || M == 128 || M == 256 ||
         M == 270;
}
bool fast_supported_c64(int M) { return fast_supported(M) || M == 512 || M == 1080; }

template <typename R> cudaError_t fast_pass(int M, int pass, const FastArgs& a) {
  if (M == 270) return fast_pass_270<R>(pass, a);
  if (M == 256) return fast_pass_256<R>(pass, a);
  if constexpr (std::is_same<R, float>::value) {
    if (M == 512) return fast_pass_512_c64(pass, a);
    if (M == 1080) return fast_pass_1080_c64(pass, a);
  }
  if (M == 40 || M == 48 || M == 80 || M == 96) return fast_pass_mid<R>(M, pass, a);
  return fast_pass_small<R>(M, pass, a);
}
template cudaError_t fast_pass<float>(int, int, const FastArgs&);
template cudaError_t fast_pass<double>(int, int, const FastArgs&);
template <> cudaError_t fast_pass<df>(int M, int pass, const FastArgs& a) {
  if (M == 270) return fast_pass_270_df(pass, a);
  if (M == 256) return fast_pass_256_df(pass, a);
  if (M == 40 || M == 48 || M == 80 || M == 96) return fast_pass_mid_df(M, pass, a);
  return fast_pass_small_df(M, pass, a);
}

}  // namespace dda
